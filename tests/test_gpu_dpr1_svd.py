"""GPU parity of dpr1_eig (Sec. 6.3) and tri_arrow_svd (Sec. 6.2) with the oracle.

The oracle solves the DPR1 secular equation over all n poles and the SVD from
B^T B with exact shifted differences, independently of the arrowhead reductions
the library uses.  Tolerance 10 n eps64 relative per value and per vector
component, as for arrow_eig.
"""
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


def gpu_dpr1(ae, d, u, rho, **kw):
    r = ae.dpr1_eig(t(d), t(u), rho, info=True, **kw)
    torch.cuda.synchronize()
    return r["lam"].cpu().numpy(), r["Q"].cpu().numpy(), r["info"]


def gpu_svd(ae, d, z, a, **kw):
    r = ae.tri_arrow_svd(t(d), t(z), a, info=True, **kw)
    torch.cuda.synchronize()
    return r["s"].cpu().numpy(), r["U"].cpu().numpy(), r["V"].cpu().numpy(), r["info"]


def dpr1_parity(ae, d, u, rho, what, **kw):
    n = len(d)
    lam, Q, info = gpu_dpr1(ae, d, u, rho, **kw)
    o = oracle.dpr1_eig(d, u, rho)
    o["abserr"] = np.zeros(n)
    o["V"] = o["Q"]
    assert_parity(lam, Q, o, n, what=what)
    return lam, Q, info


# ---------------------------------------------------------------------------
# DPR1
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("rho", [0.5, 2.0, -0.75])
@pytest.mark.parametrize("n", [1, 2, 3, 33, 65, 300])
def test_dpr1_parity(ae, n, rho):
    d, u, _ = W.uniform_dpr1(n, seed=100 + n)
    dpr1_parity(ae, d, u, rho, f"dpr1 n={n} rho={rho}")


@pytest.mark.parametrize("prec", [0, 1])
def test_dpr1_uniform_n1000(ae, prec):
    d, u, rho = W.uniform_dpr1(1000, seed=3)
    dpr1_parity(ae, d, u, rho, "dpr1 n=1000", opts=ae.default_opts(precision=prec))


def test_dpr1_last_eigenvalue_near_last_pole(ae):
    # a tiny u_n puts lambda_n just above d_n: its offset must stay accurate
    d, u, rho = W.uniform_dpr1(200, seed=9)
    u = u.copy()
    u[-1] = 1e-9
    lam, Q, info = dpr1_parity(ae, d, u, rho, "dpr1 tiny u_n")
    assert info["n_dpr1shift"] >= 1


def test_dpr1_deflation_unsorted_and_rho_zero(ae):
    d = np.array([0.3, 0.9, 0.1, 0.9, 0.5, 0.7, 0.2])
    u = np.array([0.4, -0.3, 0.0, 0.5, 0.2, -0.6, 0.1])
    dpr1_parity(ae, d, u, 0.8, "dpr1 deflation")
    dpr1_parity(ae, d, u, -1.3, "dpr1 deflation rho<0")
    lam, Q, _ = gpu_dpr1(ae, d, u, 0.0)
    np.testing.assert_array_equal(lam, np.sort(d)[::-1])
    np.testing.assert_array_equal(np.abs(Q).sum(axis=0), np.ones(len(d)))


def test_dpr1_full_size_sampled(ae):
    n = 8192
    d, u, rho = W.uniform_dpr1(n, seed=3)
    lam, Q, info = gpu_dpr1(ae, d, u, rho)
    assert np.all(lam > d) and np.all(lam[1:] < d[:-1])        # interlacing
    rng = np.random.default_rng(3)
    ks = np.unique(np.concatenate([[0, 1, n // 2, n - 2, n - 1], rng.choice(n, 60, False)]))
    o = oracle.dpr1_eig(d, u, rho, ks=ks)
    o["abserr"] = np.zeros(ks.size)
    o["V"] = o["Q"]
    assert_parity(lam[ks], Q[:, ks], o, n, cols=ks, what="dpr1 n=8192 sampled")


# ---------------------------------------------------------------------------
# triangular-arrowhead SVD
# ---------------------------------------------------------------------------
def svd_parity(ae, d, z, a, what, **kw):
    n = len(d) + 1
    s, U, V, info = gpu_svd(ae, d, z, a, **kw)
    o = oracle.tsvd(d, z, a)
    ov = {"lam": o["s"], "abserr": np.zeros(n), "V": o["V"]}
    assert_parity(s, V, ov, n, what=what + " (s, V)")
    ou = {"lam": o["s"], "abserr": np.zeros(n), "V": o["U"]}
    assert_parity(s, U, ou, n, what=what + " (U)")
    return s, U, V, info


@pytest.mark.parametrize("n", [2, 3, 33, 65, 300, 1000])
def test_svd_parity(ae, n):
    d, z, a = W.uniform_tsvd(n, seed=200 + n)
    svd_parity(ae, d, z, a, f"svd n={n}")


def test_svd_fp32_bracket(ae):
    d, z, a = W.uniform_tsvd(1000, seed=4)
    svd_parity(ae, d, z, a, "svd fp32", opts=ae.default_opts(precision=1))


def test_svd_unsorted_and_deflation(ae):
    d, z, a = W.uniform_tsvd(50, seed=5)
    s0, U0, V0, _ = gpu_svd(ae, d, z, a)
    perm = np.random.default_rng(0).permutation(len(d))
    s1, U1, V1, _ = gpu_svd(ae, d[perm], z[perm], a)
    np.testing.assert_array_equal(s1, s0)
    np.testing.assert_array_equal(V1[:-1], V0[:-1][perm])
    np.testing.assert_array_equal(U1[:-1], U0[:-1][perm])
    # zero spikes deflate to (d_r, e_r, e_r); check against binary128 one-sided Jacobi
    z2 = z.copy()
    z2[[3, 17]] = 0.0
    s2, U2, V2, info = gpu_svd(ae, d, z2, a)
    n = len(d) + 1
    B = np.zeros((n, n))
    B[np.arange(n - 1), np.arange(n - 1)] = d
    B[:-1, -1] = z2
    B[-1, -1] = a
    sj, _, _ = oracle.jacobi_svd(B)
    np.testing.assert_allclose(s2, sj, rtol=10 * n * 2.0 ** -53)
    np.testing.assert_allclose(B @ V2, U2 * s2[None, :], atol=10 * n * 2.0 ** -53)
    np.testing.assert_allclose(V2.T @ V2, np.eye(n), atol=10 * n * 2.0 ** -53)
    assert info["n_deflated"] == 2


def test_svd_rejects_nonpositive_diagonal(ae):
    d, z, a = W.uniform_tsvd(10, seed=6)
    d = d.copy()
    d[4] = -d[4]
    with pytest.raises(ae.AeError) as ei:
        gpu_svd(ae, d, z, a)
    assert ei.value.status == ae.AE_ERR_INPUT


def test_svd_full_size_sampled(ae):
    n = 8192
    d, z, a = W.uniform_tsvd(n, seed=4)
    s, U, V, info = gpu_svd(ae, d, z, a)
    assert np.all(s[:-1] >= d) and np.all(d >= s[1:])        # interlacing of sigma
    rng = np.random.default_rng(4)
    ks = np.unique(np.concatenate([[0, 1, n // 2, n - 2, n - 1], rng.choice(n, 60, False)]))
    o = oracle.tsvd(d, z, a, ks=ks)
    assert_parity(s[ks], V[:, ks], {"lam": o["s"], "abserr": np.zeros(ks.size), "V": o["V"]},
                  n, cols=ks, what="svd n=8192 sampled (V)")
    assert_parity(s[ks], U[:, ks], {"lam": o["s"], "abserr": np.zeros(ks.size), "V": o["U"]},
                  n, cols=ks, what="svd n=8192 sampled (U)")
