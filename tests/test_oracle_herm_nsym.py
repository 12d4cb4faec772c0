"""Pins of the Hermitian and non-symmetric oracles (Sec. 6.1 and its Remark).

The oracle solves both through the Pick function with weights |zeta_r|^2,
resp. zc_r zr_r, and writes the vectors from the rows of (C - l I) u = 0.
Pinned here, without a GPU, against things other than itself: 2 x 2 closed
forms, high-precision mpmath eigensolvers on tiny graded matrices, LAPACK
(numpy eigh / eig) on the dense matrix at n = 150-200, the real symmetric
oracle when the spikes are real (the Hermitian case then IS the real one), and
the invariants of each decomposition (residuals, unitarity, biorthonormality
y^T x = 1, interlacing).  A wrong conjugation, a swapped row/column spike, a
missing phase or a wrong weight fails one of them.
"""
import numpy as np
import pytest

import oracle
from paper_1302_7203_gb300 import workloads as W

EPS = 2.0 ** -53


def herm_dense(d, z, a):
    n = len(d) + 1
    C = np.zeros((n, n), complex)
    C[np.arange(n - 1), np.arange(n - 1)] = d
    C[:-1, -1] = z
    C[-1, :-1] = np.conj(z)
    C[-1, -1] = a
    return C


def nsym_dense(d, zc, zr, a):
    n = len(d) + 1
    G = np.zeros((n, n))
    G[np.arange(n - 1), np.arange(n - 1)] = d
    G[:-1, -1] = zc
    G[-1, :-1] = zr
    G[-1, -1] = a
    return G


# ----------------------------------------------------------------------------
# Hermitian
# ----------------------------------------------------------------------------
def test_herm_closed_form_order_two():
    # C = [d z; conj(z) a]: l = (d+a)/2 +- sqrt(((d-a)/2)^2 + |z|^2)
    from decimal import Decimal, getcontext
    getcontext().prec = 60
    for d0, z0, a0 in [(0.75, 0.5 - 0.25j, 2.0), (-1.5, 3.0j, 0.5), (2.0, -1e-9 + 1e-9j, 2.5)]:
        r = oracle.herm_eig([d0], [z0], a0)
        D, A = Decimal(d0), Decimal(a0)
        Z2 = Decimal(z0.real) ** 2 + Decimal(z0.imag) ** 2
        h = (D + A) / 2
        s = (((D - A) / 2) ** 2 + Z2).sqrt()
        for got, lo, ref in [(r["lam"][0], r["lam_lo"][0], h + s), (r["lam"][1], r["lam_lo"][1], h - s)]:
            assert abs(Decimal(got) + Decimal(lo) - ref) <= abs(ref) * Decimal("1e-28")
        C = herm_dense([d0], [z0], a0)
        U = r["U"]
        np.testing.assert_allclose(C @ U, U * r["lam"], atol=4 * EPS * np.abs(C).sum())


def test_herm_graded_tiny_against_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    for seed in range(3):
        d, z, a = W.graded_herm(8, seed=300 + seed)
        r = oracle.herm_eig(d, z, a)
        n = len(d) + 1
        C = mp.matrix(n, n)
        for i in range(n - 1):
            C[i, i] = mp.mpf(d[i])
            C[i, n - 1] = mp.mpc(z[i].real, z[i].imag)
            C[n - 1, i] = mp.mpc(z[i].real, -z[i].imag)
        C[n - 1, n - 1] = mp.mpf(a)
        E, _ = mp.eighe(C)
        ev = sorted([mp.re(E[i]) for i in range(n)], reverse=True)
        for k in range(n):
            got = mp.mpf(float(r["lam"][k])) + mp.mpf(float(r["lam_lo"][k]))
            assert abs(got - ev[k]) <= abs(ev[k]) * mp.mpf("1e-25"), (seed, k)
        # vectors: u_r = zeta_r/(d_r - l), u_n = -1, normalised, at 60 digits
        for k in range(n):
            x = [mp.mpc(z[i].real, z[i].imag) / (mp.mpf(d[i]) - ev[k]) for i in range(n - 1)]
            x.append(mp.mpc(-1))
            nr = mp.sqrt(sum(abs(t) ** 2 for t in x))
            for i in range(n):
                ref = complex(x[i] / nr)
                assert abs(r["U"][i, k] - ref) <= 4e-16 * abs(ref), (seed, k, i)


def test_herm_against_numpy_eigh():
    n = 200
    d, z, a = W.uniform_herm(n, seed=8)
    r = oracle.herm_eig(d, z, a)
    C = herm_dense(d, z, a)
    ev = np.linalg.eigvalsh(C)[::-1]
    nrm = np.linalg.norm(C, 2)
    assert np.abs(r["lam"] - ev).max() <= 50 * n * EPS * nrm
    U = r["U"]
    assert np.abs(C @ U - U * r["lam"]).max() <= 8 * EPS * nrm
    assert np.abs(U.conj().T @ U - np.eye(n)).max() <= 2 * n * EPS
    assert np.all(r["lam"][:-1] > d) and np.all(d > r["lam"][1:])   # interlacing


def test_herm_real_spikes_equal_real_oracle():
    # with real zeta the Hermitian arrowhead is the real symmetric one: the same
    # weights zeta^2, so the same eigenvalues bit for bit and the same vectors
    d, z, a = W.uniform_arrow(300, seed=4)
    rh = oracle.herm_eig(d, z.astype(complex), a)
    rr = oracle.arrow_eig(d, z, a)
    np.testing.assert_array_equal(rh["lam"], rr["lam"])
    np.testing.assert_array_equal(rh["lam_lo"], rr["lam_lo"])
    assert np.abs(rh["U"].imag).max() == 0.0
    np.testing.assert_allclose(rh["U"].real, rr["V"], rtol=4 * EPS, atol=1e-300)


def test_herm_phases_only_rotate_rows():
    # C' = Phi C Phi^* with Phi = diag(e^{i t_r}, 1): spikes e^{i t_r} zeta_r,
    # eigenvalues unchanged, vector rows rotated by e^{i t_r} (Sec. 6.1)
    d, z, a = W.graded_herm(60, seed=12)
    t = np.random.default_rng(5).uniform(0, 2 * np.pi, len(d))
    ph = np.exp(1j * t)
    r0 = oracle.herm_eig(d, z, a)
    r1 = oracle.herm_eig(d, z * ph, a)
    np.testing.assert_allclose(r1["lam"], r0["lam"], rtol=8 * EPS)
    U0 = r0["U"].copy()
    U0[:-1] *= ph[:, None]
    np.testing.assert_allclose(r1["U"], U0, rtol=1e-14, atol=1e-300)


def test_herm_deflation():
    d = np.array([3.0, 1.0, 1.0, 1.0, -2.0, -4.0])
    z = np.array([0.5 + 0.5j, 1.0 - 2.0j, 0.0, 0.25j, 1.0, 0.0])
    a = 0.5
    r = oracle.herm_eig(d, z, a)
    C = herm_dense(d, z, a)
    n = len(d) + 1
    U = r["U"]
    nrm = np.abs(C).sum()
    np.testing.assert_allclose(C @ U, U * r["lam"], atol=8 * EPS * nrm)
    np.testing.assert_allclose(U.conj().T @ U, np.eye(n), atol=8 * EPS)
    ev = np.linalg.eigvalsh(C)[::-1]
    np.testing.assert_allclose(r["lam"], ev, atol=20 * EPS * nrm)
    # zero spikes give unit vectors e_r
    for row, val in [(2, 1.0), (5, -4.0)]:
        k = int(np.nonzero(np.abs(U[row]) == 1.0)[0][0])
        assert r["lam"][k] == val


def test_herm_invalid():
    with pytest.raises(ValueError):
        oracle.herm_eig([1.0, np.nan], [1.0, 1j], 0.0)


# ----------------------------------------------------------------------------
# non-symmetric (Remark of Sec. 6.1)
# ----------------------------------------------------------------------------
def test_nsym_closed_form_order_two():
    from decimal import Decimal, getcontext
    getcontext().prec = 60
    for d0, c0, r0, a0 in [(0.75, 0.5, 2.0, 2.0), (-1.5, -3.0, -0.125, 0.5), (2.0, 1e-9, 4e-9, 2.5)]:
        r = oracle.nsym_eig([d0], [c0], [r0], a0)
        D, A = Decimal(d0), Decimal(a0)
        P = Decimal(c0) * Decimal(r0)
        h = (D + A) / 2
        s = (((D - A) / 2) ** 2 + P).sqrt()
        for got, lo, ref in [(r["lam"][0], r["lam_lo"][0], h + s), (r["lam"][1], r["lam_lo"][1], h - s)]:
            assert abs(Decimal(got) + Decimal(lo) - ref) <= abs(ref) * Decimal("1e-28")
        G = nsym_dense([d0], [c0], [r0], a0)
        X, Y = r["X"], r["Y"]
        nrm = np.abs(G).sum()
        np.testing.assert_allclose(G @ X, X * r["lam"], atol=4 * EPS * nrm * np.abs(X).max())
        np.testing.assert_allclose(Y.T @ G, (Y * r["lam"]).T, atol=4 * EPS * nrm * np.abs(Y).max())
        np.testing.assert_allclose(Y.T @ X, np.eye(2), atol=8 * EPS)


def test_nsym_graded_tiny_against_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    for seed in range(3):
        d, zc, zr, a = W.graded_nsym(7, seed=400 + seed)
        r = oracle.nsym_eig(d, zc, zr, a)
        n = len(d) + 1
        G = mp.matrix(n, n)
        for i in range(n - 1):
            G[i, i] = mp.mpf(d[i])
            G[i, n - 1] = mp.mpf(zc[i])
            G[n - 1, i] = mp.mpf(zr[i])
        G[n - 1, n - 1] = mp.mpf(a)
        E = mp.eig(G, left=False, right=False)
        ev = sorted([mp.re(e) for e in E], reverse=True)
        assert max(abs(mp.im(e)) for e in E) < mp.mpf("1e-40") * max(abs(x) for x in ev)
        for k in range(n):
            got = mp.mpf(float(r["lam"][k])) + mp.mpf(float(r["lam_lo"][k]))
            assert abs(got - ev[k]) <= abs(ev[k]) * mp.mpf("1e-25"), (seed, k)
        for k in range(n):
            xs = [mp.mpf(zc[i]) / (mp.mpf(d[i]) - ev[k]) for i in range(n - 1)] + [mp.mpf(-1)]
            ys = [mp.mpf(zr[i]) / (mp.mpf(d[i]) - ev[k]) for i in range(n - 1)] + [mp.mpf(-1)]
            s = mp.sqrt(sum(x * y for x, y in zip(xs, ys)))
            for i in range(n):
                for got, ref in [(r["X"][i, k], float(xs[i] / s)), (r["Y"][i, k], float(ys[i] / s))]:
                    assert abs(got - ref) <= 4e-16 * abs(ref), (seed, k, i)


def test_nsym_against_numpy_eig():
    n = 150
    d, zc, zr, a = W.uniform_nsym(n, seed=10)
    r = oracle.nsym_eig(d, zc, zr, a)
    G = nsym_dense(d, zc, zr, a)
    ev = np.linalg.eigvals(G)
    assert np.abs(ev.imag).max() <= 1e-10
    ev = np.sort(ev.real)[::-1]
    nrm = np.linalg.norm(G, 2)
    assert np.abs(r["lam"] - ev).max() <= 1e-9 * nrm     # dgeev: non-normal, looser
    X, Y = r["X"], r["Y"]
    assert np.abs(G @ X - X * r["lam"]).max() <= 16 * EPS * nrm * np.abs(X).max()
    assert np.abs(Y.T @ G - (Y * r["lam"]).T).max() <= 16 * EPS * nrm * np.abs(Y).max()
    assert np.abs(Y.T @ X - np.eye(n)).max() <= 1e-11
    assert np.all(r["lam"][:-1] > d) and np.all(d > r["lam"][1:])


def test_nsym_symmetric_case_equals_real_oracle():
    # zc = zr = z: G is the real symmetric arrowhead and X = Y = V
    d, z, a = W.uniform_arrow(200, seed=6)
    rs = oracle.nsym_eig(d, z, z, a)
    rr = oracle.arrow_eig(d, z, a)
    np.testing.assert_array_equal(rs["lam"], rr["lam"])
    np.testing.assert_allclose(rs["X"], rr["V"], rtol=4 * EPS, atol=1e-300)
    np.testing.assert_allclose(rs["Y"], rr["V"], rtol=4 * EPS, atol=1e-300)


def test_nsym_deflation_and_invalid():
    d = np.array([2.0, 1.0, 1.0, -0.5, -3.0])
    zc = np.array([0.5, -1.0, -0.25, 0.0, 2.0])
    zr = np.array([2.0, -0.5, -1.0, 0.0, 0.125])
    a = 0.75
    r = oracle.nsym_eig(d, zc, zr, a)
    G = nsym_dense(d, zc, zr, a)
    n = len(d) + 1
    X, Y = r["X"], r["Y"]
    nrm = np.abs(G).sum()
    np.testing.assert_allclose(G @ X, X * r["lam"], atol=16 * EPS * nrm * np.abs(X).max())
    np.testing.assert_allclose(Y.T @ G, (Y * r["lam"]).T, atol=16 * EPS * nrm * np.abs(Y).max())
    np.testing.assert_allclose(Y.T @ X, np.eye(n), atol=16 * EPS)
    k = int(np.nonzero(X[3] == 1.0)[0][0])
    assert r["lam"][k] == -0.5 and Y[3, k] == 1.0
    with pytest.raises(ValueError):
        oracle.nsym_eig([1.0, 0.0], [1.0, -1.0], [1.0, 1.0], 0.0)      # opposite signs
    with pytest.raises(ValueError):
        oracle.nsym_eig([1.0, 0.0], [1.0, 0.0], [1.0, 1.0], 0.0)       # one-sided zero
