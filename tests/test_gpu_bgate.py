"""Algorithm 5's precision gates on the GPU (ae_opts.bgate = 1).

With the gate, the element b of Eq. (b_ob) is formed in standard precision
unless the spike ratio sum_{j != i} |zeta_j| / |zeta_i| exceeds n and K_b of
Eq. (K2) exceeds kb_max; only then is it recomputed in double-double
(Theorem 6), flagged AE_FLAG_DDB.  Checked: parity with the oracle at 10 n
eps64 on every workload and both finishes; the paper's Example 3, whose
K_b ~ 3e9 needs doubled precision, takes the double-double path and
reproduces the paper's doubled-precision b; with the gate forced open (never
double-double) the same eigenvalues miss the tolerance, which is what the
gate is for.
"""
import numpy as np
import pytest

import oracle
from conftest import read_golden
from parity import assert_parity, lam_errors, widened
from paper_1302_7203_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ae():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1302_7203_gb300 import arrowhead, build
    build.build()
    return arrowhead


def solve(ae, d, z, a, o):
    r = ae.arrow_eig(torch.as_tensor(d, device="cuda"), torch.as_tensor(z, device="cuda"), a,
                     opts=o, info=True, diag=True, want_shift=True)
    torch.cuda.synchronize()
    return ({k: r[k].cpu().numpy() for k in ("lam", "V", "shift")},
            {k: v.cpu().numpy() for k, v in r["diag"].items()}, r["info"])


def case(name):
    if name.startswith("ex"):
        return W.paper_example(int(name[2]))
    if name == "uniform1000":
        return W.uniform_arrow(1000, seed=0)
    if name == "graded3001":
        return W.graded_arrow(3001, seed=13)
    if name == "qdot":
        return W.quantum_dot_like(2501)
    return W.mirrored_arrow(41)


@pytest.mark.parametrize("form", [(0, 0), (0, 1), (1, 1)])     # (precision, finish)
@pytest.mark.parametrize("name", ["ex1", "ex2", "ex3", "uniform1000", "graded3001", "qdot",
                                  "mirrored"])
def test_gated_parity(ae, name, form):
    d, z, a = case(name)
    g, dg, info = solve(ae, d, z, a, ae.default_opts(bgate=1, precision=form[0],
                                                     finish=form[1]))
    o = oracle.arrow_eig(d, z, a)
    assert_parity(g["lam"], g["V"], o, len(d) + 1, what=f"bgate {name} form {form}")
    assert info["n_capped"] == 0
    # every eigenpair whose b went to double-double is flagged, and counted
    assert info["n_ddb"] >= int(np.count_nonzero(dg["flags"] & ae.FLAG_DDB))


def test_example3_takes_the_double_double_path(ae):
    d, z, a = W.paper_example(3)
    g, dg, info = solve(ae, d, z, a, ae.default_opts(bgate=1))
    # eigenvalues 2..5 (indices 1..4) have K_b ~ 3e9-5e9 and spike ratio ~1e10
    assert np.all(dg["flags"][1:5] & ae.FLAG_DDB)
    rows = read_golden("example3.txt")
    b_doubled = [float(v[0]) for key, v in rows if key == "b_doubled"][0]
    assert g["shift"][1] == 4.0
    assert abs(dg["b"][1] - b_doubled) <= 2 * np.spacing(b_doubled)
    # the largest eigenvalue (K_b ~ 1) stays in standard precision
    assert not (dg["flags"][0] & ae.FLAG_DDB)


def test_example3_needs_the_gate(ae):
    # with the gate held open (kb_max huge) b is formed in standard precision:
    # b of A_2^{-1} loses ~10 digits and eigenvalue 2 misses the tolerance,
    # as Sec. 5 shows for Example 3
    d, z, a = W.paper_example(3)
    n = len(d) + 1
    g, dg, _ = solve(ae, d, z, a, ae.default_opts(bgate=1, kb_max=1e300))
    rows = read_golden("example3.txt")
    b_doubled = [float(v[0]) for key, v in rows if key == "b_doubled"][0]
    assert abs(dg["b"][1] - b_doubled) > 1e-12 * b_doubled
    o = oracle.arrow_eig(d, z, a)
    assert lam_errors(g["lam"], o, n)[1] > 10.0


def test_gate_spares_most_pairs_of_the_benchmark_matrix(ae):
    d, z, a = W.graded_arrow(4000, seed=17)
    g, dg, info = solve(ae, d, z, a, ae.default_opts(bgate=1, finish=1))
    o = oracle.arrow_eig(d, z, a)
    assert_parity(g["lam"], g["V"], o, len(d) + 1, what="bgate graded 4000")
    # only a small share of eigenpairs needs double-double
    assert info["n_ddb"] < 0.25 * len(d)


def test_gated_full_size_sampled(ae):
    """n = 16384 graded (the benchmark workload) in the gated Newton form."""
    n = 16384
    d, z, a = W.graded_arrow(n, seed=1)
    g, dg, info = solve(ae, d, z, a, ae.default_opts(bgate=1, finish=1))
    lam, V = g["lam"], g["V"]
    assert np.all(lam[:-1] >= d) and np.all(d >= lam[1:])
    ddb = np.nonzero(dg["flags"] & ae.FLAG_DDB)[0]
    fixed = np.nonzero(dg["flags"] & (ae.FLAG_NEARZERO | ae.FLAG_OTHERPOLE |
                                      ae.FLAG_DPR1SHIFT))[0]
    # the pairs the gate kept in standard precision with the largest K_b are
    # the ones most at risk: sample them with the rest
    std = np.nonzero(~(dg["flags"] & ae.FLAG_DDB).astype(bool))[0]
    risky = std[np.argsort(-dg["Kb"][std])[:48]]
    rng = np.random.default_rng(11)
    ks = np.unique(np.concatenate([[0, 1, n // 2, n - 2, n - 1], rng.choice(n, 64, False),
                                   ddb[:32], fixed[:32], risky]))
    o = oracle.arrow_eig(d, z, a, ks=ks)
    assert not widened(o, n).any()   # every comparison at the full 10 n eps64 bar
    assert_parity(lam[ks], V[:, ks], o, n, cols=ks, what="bgate graded n=16384 sampled")
