"""The serving loop: continuous batching of arrowhead / DPR1 / SVD requests.

Each result served in a mix of kinds and sizes equals the same solve made
alone through the direct entry points: bitwise (the same kernels run, only on
another stream, or, for a run of small arrowheads admitted together, the
batched stages with one 32-lane team per eigenpair), except eigenpairs a
remedy re-solved inside a merged pass (a warp there, a wider team alone),
which agree within the 10 n eps64 tolerance.  Small requests submitted behind a
large one finish while it is still running (their work overlaps), a burst of
small arrowheads is merged into batched passes, the memory budget and queue
bound apply backpressure, and a bad request fails alone, also inside a merged
pass.
"""
import time

import numpy as np
import pytest

import oracle
from parity import assert_parity
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


def t(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float64), device="cuda")


def mix():
    reqs = []
    for n, seed in [(64, 1), (300, 2), (2000, 3)]:
        d, z, a = W.uniform_arrow(n, seed=seed)
        reqs.append((0, d, z, a))
    for n, seed in [(100, 4), (1000, 5)]:
        d, u, rho = W.uniform_dpr1(n, seed=seed)
        reqs.append((1, d, u, rho))
    for n, seed in [(80, 6), (700, 7)]:
        d, z, a = W.uniform_tsvd(n, seed=seed)
        reqs.append((2, d, z, a))
    return reqs


REMEDY = 2 | 4 | 8         # AE_FLAG_NEARZERO | AE_FLAG_OTHERPOLE | AE_FLAG_DPR1SHIFT


def alone(ae, kind, d, z, a):
    if kind == 0:
        r = ae.arrow_eig(t(d), t(z), a, diag=True)
        return {"lam": r["lam"], "V": r["V"],
                "fixed": (r["diag"]["flags"] & REMEDY) != 0}
    if kind == 1:
        r = ae.dpr1_eig(t(d), t(z), a)
        return {"lam": r["lam"], "V": r["Q"]}
    r = ae.tri_arrow_svd(t(d), t(z), a)
    return {"lam": r["s"], "V": r["V"], "U": r["U"]}


def same_as_alone(got, ref, n):
    """Bitwise, except remedied eigenpairs of a merged pass: within tolerance."""
    if "fixed" not in ref:
        assert torch.equal(got["lam"], ref["lam"])
        assert torch.equal(got["V"], ref["V"])
        return
    keep = ~ref["fixed"]
    assert torch.equal(got["lam"][keep], ref["lam"][keep])
    assert torch.equal(got["V"][:, keep], ref["V"][:, keep])
    tol = 10 * n * 2.0 ** -53
    assert torch.all((got["lam"] - ref["lam"]).abs() <= tol * ref["lam"].abs())
    assert torch.all((got["V"] - ref["V"]).abs() <= tol * ref["V"].abs() + 1e-300)


def test_served_results_equal_solo_results(ae):
    srv = ae.Server(budget_bytes=8 << 30, max_inflight=6)
    reqs = mix() * 2
    tickets = [srv.submit(k, t(d), t(z), a) for k, d, z, a in reqs]
    assert all(tk is not None for tk in tickets)
    for tk, (k, d, z, a) in zip(tickets, reqs):
        st, lat = srv.wait(tk)
        assert st == ae.REQ_DONE and lat > 0
        got = srv.result(tk)
        ref = alone(ae, k, d, z, a)
        same_as_alone(got, ref, len(ref["lam"]))
        if k == 2:
            assert torch.equal(got["U"], ref["U"])
        assert srv.release(tk) == 0
    s = srv.stats()
    assert s["completed"] == len(reqs) and s["failed"] == 0
    assert 0 < s["p50_s"] <= s["p99_s"] <= s["max_s"]
    assert s["bytes_in_use"] == 0
    srv.close()


def test_small_arrowheads_are_merged(ae):
    # a burst of small arrowheads waits at the head of the queue while a large
    # request holds the GPU: they are admitted as merged batched passes, each
    # result equal to its solo solve (bitwise outside remedies) and to the oracle
    srv = ae.Server(budget_bytes=16 << 30, max_inflight=2)
    d, z, a = W.graded_arrow(8000, seed=12)
    big = srv.submit(0, t(d), t(z), a, vectors=False)
    small = []
    for i in range(40):
        n = int(W.batch_sizes(1, lo=8, hi=1024, seed=200 + i)[0])
        ds, zs, als = (W.graded_arrow if i % 2 else W.uniform_arrow)(n, seed=300 + i)
        small.append((srv.submit(0, t(ds), t(zs), als), ds, zs, als))
    for tk, ds, zs, als in small:
        st, _ = srv.wait(tk)
        assert st == ae.REQ_DONE
        got = srv.result(tk)
        same_as_alone(got, alone(ae, 0, ds, zs, als), len(ds) + 1)
        if len(ds) % 5 == 0:
            assert_parity(got["lam"].cpu().numpy(), got["V"].cpu().numpy(),
                          oracle.arrow_eig(ds, zs, als), len(ds) + 1, what="merged request")
        srv.release(tk)
    assert srv.wait(big)[0] == ae.REQ_DONE
    s = srv.stats()
    assert s["merged"] >= 10 and s["failed"] == 0
    srv.close()


def test_served_results_match_oracle(ae):
    srv = ae.Server(budget_bytes=4 << 30, max_inflight=4)
    d, z, a = W.graded_arrow(500, seed=8)
    tk = srv.submit(0, t(d), t(z), a)
    srv.wait(tk)
    got = srv.result(tk)
    o = oracle.arrow_eig(d, z, a)
    assert_parity(got["lam"].cpu().numpy(), got["V"].cpu().numpy(), o, 500, what="served")
    srv.close()


def test_small_requests_overlap_a_large_one(ae):
    srv = ae.Server(budget_bytes=16 << 30, max_inflight=8)
    d, z, a = W.graded_arrow(12000, seed=9)
    big = srv.submit(0, t(d), t(z), a, vectors=False)
    small = []
    for i in range(6):
        ds, zs, als = W.uniform_arrow(128, seed=100 + i)
        small.append(srv.submit(0, t(ds), t(zs), als))
    lat_small = [srv.wait(tk)[1] for tk in small]
    st_big, lat_big = srv.wait(big)
    assert st_big == ae.REQ_DONE
    # the small requests were admitted while the big one ran and finished first
    assert max(lat_small) < lat_big
    srv.close()


def test_budget_and_queue_backpressure(ae):
    # a 1-byte budget admits one request at a time; the queue holds 3 waiting
    # requests, so a burst of 20 gets AE_EAGAIN for most of them
    srv = ae.Server(budget_bytes=1, max_inflight=4, queue_cap=3)
    d, z, a = W.uniform_arrow(3000, seed=11)
    dt, zt = t(d), t(z)
    tickets = [srv.submit(0, dt, zt, a) for _ in range(20)]
    accepted = [tk for tk in tickets if tk is not None]
    assert 1 <= len(accepted) < 20
    assert srv.stats()["rejected"] == 20 - len(accepted)
    first = None
    for tk in accepted:
        st, _ = srv.wait(tk)
        assert st == ae.REQ_DONE
        got = srv.result(tk)["lam"]
        first = got if first is None else first
        assert torch.equal(got, first)
        srv.release(tk)
    srv.close()


def test_bad_request_fails_alone(ae):
    # the two are small arrowheads submitted together: one merged pass
    srv = ae.Server(budget_bytes=4 << 30, max_inflight=4)
    d, z, a = W.uniform_arrow(200, seed=10)
    bad = d.copy()
    bad[7] = np.inf
    t_bad = srv.submit(0, t(bad), t(z), a)
    t_ok = srv.submit(0, t(d), t(z), a)
    assert srv.wait(t_bad)[0] == ae.REQ_ERROR
    assert srv.wait(t_ok)[0] == ae.REQ_DONE
    got = srv.result(t_ok)
    same_as_alone(got, alone(ae, 0, d, z, a), 200)
    assert srv.stats()["failed"] == 1
    srv.close()
