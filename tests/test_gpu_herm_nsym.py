"""GPU parity of herm_arrow_eig (Sec. 6.1) and nsym_arrow_eig (Remark of Sec. 6.1).

Both run the real arrowhead pipeline on the moduli |zeta_r| (resp.
sqrt(zc_r zr_r)) with the exact squares in double-double and differ only in
the vector epilogue (U = Phi V; X = Psi V, Y = Psi^{-1} V).  Each eigenvalue
and each (complex) vector component must be within 10 n eps64 of the oracle,
which solves the Pick function with the exact weights and writes the vectors
from the rows of (C - l I) u = 0.  Covered for both finishes, with the FP32
bracket, on uniform and graded spectra, with deflation, and against the real
solver when the spikes are real.
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


def t(x, dtype=torch.float64):
    return torch.as_tensor(np.asarray(x), dtype=dtype, device="cuda")


def herm(ae, d, z, a, **kw):
    r = ae.herm_arrow_eig(t(d), t(z, torch.complex128), a, info=True, **kw)
    torch.cuda.synchronize()
    return r["lam"].cpu().numpy(), r["U"].cpu().numpy(), r["info"]


def nsym(ae, d, zc, zr, a, **kw):
    r = ae.nsym_arrow_eig(t(d), t(zc), t(zr), a, info=True, **kw)
    torch.cuda.synchronize()
    return r["lam"].cpu().numpy(), r["X"].cpu().numpy(), r["Y"].cpu().numpy(), r["info"]


# (precision, finish, bgate); the last is the benchmarked form
FORMS = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (1, 1, 1)]


def herm_case(case):
    if case == "uniform300":
        return W.uniform_herm(300, seed=8)
    if case == "uniform1000":
        return W.uniform_herm(1000, seed=18)
    if case == "graded700":
        return W.graded_herm(700, seed=9)
    if case == "n2":
        return np.array([0.75]), np.array([0.5 - 0.25j]), 2.0
    if case == "n65":
        return W.uniform_herm(65, seed=65)
    d = np.array([3.0, 1.0, 1.0, 1.0, -2.0, -4.0, 0.5])
    z = np.array([0.5 + 0.5j, 1.0 - 2.0j, 0.0, 0.25j, 1.0, 0.0, -0.75 + 0.1j])
    return d, z, 0.5


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("case", ["n2", "n65", "uniform300", "uniform1000", "graded700",
                                  "deflation"])
def test_herm_parity(ae, case, form):
    d, z, a = herm_case(case)
    o = oracle.herm_eig(d, z, a)
    o["V"] = o["U"]
    lam, U, info = herm(ae, d, z, a, opts=ae.default_opts(precision=form[0], finish=form[1], bgate=form[2]))
    assert_parity(lam, U, o, len(d) + 1, what=f"herm {case} form {form}")
    assert info["n_capped"] == 0


def test_herm_real_spikes_match_arrow_eig(ae):
    d, z, a = W.graded_arrow(500, seed=31)
    lam_h, U, _ = herm(ae, d, z.astype(complex), a)
    r = ae.arrow_eig(t(d), t(z), a)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(lam_h, r["lam"].cpu().numpy())
    assert np.abs(U.imag).max() == 0.0
    V = r["V"].cpu().numpy()
    assert np.all(np.abs(U.real - V) <= 4 * 2.0 ** -53 * np.abs(V))


def test_herm_residual_and_unitarity(ae):
    d, z, a = W.uniform_herm(800, seed=3)
    lam, U, _ = herm(ae, d, z, a)
    n = len(d) + 1
    CU = np.empty_like(U)
    CU[:-1] = d[:, None] * U[:-1] + z[:, None] * U[-1][None, :]
    CU[-1] = np.conj(z) @ U[:-1] + a * U[-1]
    nrm = np.abs(d).max() + np.linalg.norm(z) + abs(a)
    assert np.abs(CU - U * lam[None, :]).max() <= 8 * 2.0 ** -53 * nrm
    assert np.abs(U.conj().T @ U - np.eye(n)).max() <= 2 * n * 2.0 ** -53


def test_herm_sampled_n4096(ae):
    n = 4096
    d, z, a = W.graded_herm(n, seed=41)
    lam, U, _ = herm(ae, d, z, a, opts=ae.default_opts(finish=1))
    assert np.all(lam[:-1] >= d) and np.all(d >= lam[1:])
    ks = np.unique(np.concatenate([[0, 1, n // 2, n - 1],
                                   np.random.default_rng(2).choice(n, 48, replace=False)]))
    o = oracle.herm_eig(d, z, a, ks=ks)
    o["V"] = o["U"]
    assert_parity(lam[ks], U[:, ks], o, n, cols=ks, what="herm n=4096 sampled")


def nsym_case(case):
    if case == "uniform300":
        return W.uniform_nsym(300, seed=10)
    if case == "uniform1000":
        return W.uniform_nsym(1000, seed=20)
    if case == "graded700":
        return W.graded_nsym(700, seed=11)
    if case == "n2":
        return np.array([0.75]), np.array([-0.5]), np.array([-2.0]), 2.0
    d = np.array([2.0, 1.0, 1.0, -0.5, -3.0, 0.25])
    zc = np.array([0.5, -1.0, -0.25, 0.0, 2.0, 1.5])
    zr = np.array([2.0, -0.5, -1.0, 0.0, 0.125, 0.5])
    return d, zc, zr, 0.75


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("case", ["n2", "uniform300", "uniform1000", "graded700", "deflation"])
def test_nsym_parity(ae, case, form):
    d, zc, zr, a = nsym_case(case)
    o = oracle.nsym_eig(d, zc, zr, a)
    lam, X, Y, info = nsym(ae, d, zc, zr, a,
                           opts=ae.default_opts(precision=form[0], finish=form[1], bgate=form[2]))
    n = len(d) + 1
    o["V"] = o["X"]
    assert_parity(lam, X, o, n, what=f"nsym {case} form {form} (X)")
    o["V"] = o["Y"]
    assert_parity(lam, Y, o, n, what=f"nsym {case} form {form} (Y)")
    assert info["n_capped"] == 0


def test_nsym_biorthonormal(ae):
    d, zc, zr, a = W.graded_nsym(600, seed=12)
    lam, X, Y, _ = nsym(ae, d, zc, zr, a)
    n = len(d) + 1
    assert np.abs(Y.T @ X - np.eye(n)).max() <= 4 * n * 2.0 ** -53


def test_nsym_rejects_mixed_signs(ae):
    d = np.array([1.0, 0.5, -1.0])
    zc = np.array([1.0, -1.0, 0.5])
    zr = np.array([1.0, 1.0, 0.5])
    with pytest.raises(ae.AeError) as ei:
        nsym(ae, d, zc, zr, 0.0)
    assert ei.value.status == ae.AE_ERR_INPUT
    zr = np.array([1.0, 0.0, 0.5])
    zc = np.array([1.0, 0.25, 0.5])
    with pytest.raises(ae.AeError) as ei:
        nsym(ae, d, zc, zr, 0.0)
    assert ei.value.status == ae.AE_ERR_INPUT
