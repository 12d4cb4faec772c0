"""One instance split by eigenpair ranges (arrow_eig_part), parts run one after
another on one GPU.

Each part repeats the reduction and solves an even share of the computed
eigenpairs, the deflated rows in its value range, and (for the remedy test of
Eq. K0) the eigenpair just outside each end of its range.  Checked: the
device's part bounds equal the host's bookkeeping (shard.part_items on the
oracle's reduction, bit-exact index results); the parts' blocks cover the
output once; put side by side they equal the whole arrow_eig bit for bit,
except eigenpairs a remedy re-solved (a team of another width may re-solve
them), which meet the 10 n eps64 bar against the oracle like everything else;
a buffer too small for a part is refused before anything is solved.
"""
import numpy as np
import pytest

import oracle
from parity import assert_parity
from paper_1302_7203_gb300 import shard, workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ae():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1302_7203_gb300 import arrowhead, build
    build.build()
    return arrowhead


def t(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float64), device="cuda")


def deflating(n=301, seed=3):
    d, z, a = W.uniform_arrow(n, seed=seed)
    d, z = d.copy(), z.copy()
    z[[4, 20, 21, 150]] = 0.0
    d[[9, 10]] = d[8]
    d[[60, 61]] = d[59]
    z[61] = 0.0
    return d, z, a


def reduced(d, z):
    order, kind, head, m = oracle.reduce(d, z)
    return (np.array([d[r] for r in order if kind[r] == 0]),
            np.array([d[r] for r in order if kind[r] != 0]))


CASES = {"graded3001": lambda: W.graded_arrow(3001, seed=13),
         "deflating301": deflating,
         "uniform1000": lambda: W.uniform_arrow(1000, seed=0)}


@pytest.mark.parametrize("form", [(0, 0, 0), (1, 1, 1)])
@pytest.mark.parametrize("nparts", [1, 2, 3, 7])
@pytest.mark.parametrize("case", sorted(CASES))
def test_parts_equal_the_whole(ae, case, nparts, form):
    d, z, a = CASES[case]()
    n = len(d) + 1
    o = ae.default_opts(precision=form[0], finish=form[1], bgate=form[2])
    whole = ae.arrow_eig(t(d), t(z), a, opts=o, diag=True)
    torch.cuda.synchronize()
    lam_w, V_w = whole["lam"].cpu().numpy(), whole["V"].cpu().numpy()
    remedy = ae.FLAG_NEARZERO | ae.FLAG_OTHERPOLE | ae.FLAG_DPR1SHIFT
    fixed = (whole["diag"]["flags"].cpu().numpy() & remedy) != 0
    poles, defl = reduced(d, z)
    blocks = []
    for p in range(nparts):
        k0, k1, u0, u1, pos0, cnt = shard.part_items(poles, defl, p, nparts)
        assert ae.arrow_eig_part_size(t(d), t(z), p, nparts) == (pos0, cnt)
        r = ae.arrow_eig_part(t(d), t(z), a, p, nparts, opts=o, info=True)
        torch.cuda.synchronize()
        assert (r["pos0"], r["count"]) == (pos0, cnt)
        assert r["info"]["n_capped"] == 0
        blocks.append((r["pos0"], r["lam"].cpu().numpy(), r["V"].cpu().numpy()))
    lam, V = shard.merge_parts(n, blocks)
    same = ~fixed
    np.testing.assert_array_equal(lam[same], lam_w[same])
    np.testing.assert_array_equal(V[:, same], V_w[:, same])
    if nparts == 1:
        np.testing.assert_array_equal(lam, lam_w)
        np.testing.assert_array_equal(V, V_w)
    assert_parity(lam, V, oracle.arrow_eig(d, z, a), n, what=f"split {case} into {nparts}")


def test_part_of_the_benchmark_matrix(ae):
    # a middle part of the n = 16384 graded matrix in the benchmarked form,
    # sampled against the oracle
    n = 16384
    d, z, a = W.graded_arrow(n, seed=1)
    o = ae.default_opts(precision=1, finish=1, bgate=1)
    r = ae.arrow_eig_part(t(d), t(z), a, 3, 8, opts=o)
    torch.cuda.synchronize()
    assert (r["pos0"], r["count"]) == (3 * n // 8, n // 8)
    rng = np.random.default_rng(3)
    loc = np.unique(np.concatenate([[0, r["count"] - 1], rng.choice(r["count"], 60, False)]))
    ks = r["pos0"] + loc
    ref = oracle.arrow_eig(d, z, a, ks=ks)
    assert_parity(r["lam"].cpu().numpy()[loc], r["V"].cpu().numpy()[:, loc], ref, n, cols=ks,
                  what="part 3 of 8 of the benchmark matrix")


def test_part_buffer_too_small_is_refused(ae):
    d, z, a = W.uniform_arrow(500, seed=2)
    pos0, cnt = ae.arrow_eig_part_size(t(d), t(z), 1, 4)
    with pytest.raises(ae.AeError) as ei:
        ae.arrow_eig_part(t(d), t(z), a, 1, 4, cap=cnt - 1)
    assert ei.value.status == ae.AE_ERR_TOO_LARGE
    with pytest.raises(ae.AeError) as ei:
        ae.arrow_eig_part(t(d), t(z), a, 4, 4, cap=10)
    assert ei.value.status == -5


@pytest.mark.parametrize("n", [1, 2, 3, 9])
def test_more_parts_than_eigenpairs(ae, n):
    # parts may be empty (nparts > m + 1); the non-empty ones still tile the output
    d, z, a = W.uniform_arrow(n, seed=90 + n)
    whole = ae.arrow_eig(t(d), t(z), a)
    torch.cuda.synchronize()
    nparts = n + 3
    blocks = []
    for p in range(nparts):
        r = ae.arrow_eig_part(t(d), t(z), a, p, nparts)
        torch.cuda.synchronize()
        if r["count"]:
            blocks.append((r["pos0"], r["lam"].cpu().numpy(), r["V"].cpu().numpy()))
    lam, V = shard.merge_parts(n, blocks)
    np.testing.assert_array_equal(lam, whole["lam"].cpu().numpy())
    np.testing.assert_array_equal(V, whole["V"].cpu().numpy())
