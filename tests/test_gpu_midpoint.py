"""GPU check of Algorithm 1's midpoint test evaluated in FP32 (AE_FP32_BRACKET).

With precision = AE_FP32_BRACKET the sign of F at the midpoint of lambda's
interval is first taken from an FP32 evaluation on the scaled copies, which
carries an error bound; it decides only where that bound, plus a bound on the
FP64 evaluation's own error, leaves the sign in no doubt, and otherwise the
FP64 pass runs (flag AE_FLAG_MID64).  So the shift chosen must be the one the
all-FP64 test picks.  Checked: the shift equals the all-FP64 run's for every
eigenpair that neither run remedied, for real, Hermitian and non-symmetric
arrowheads over uniform, graded, clustered and quantum-dot-like spectra; the
FP64 pass runs on a small fraction only; where F vanishes at the midpoint (a
mirrored spectrum) the FP64 pass is the one that decides.
"""
import numpy as np
import pytest

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
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


REMEDY = 2 | 4 | 8   # AE_FLAG_NEARZERO | AE_FLAG_OTHERPOLE | AE_FLAG_DPR1SHIFT


def run(ae, fn, args, precision):
    o = ae.default_opts(precision=precision, finish=ae.AE_FINISH_NEWTON, bgate=1)
    r = fn(*args, vectors=False, want_shift=True, opts=o, info=True, diag=True)
    torch.cuda.synchronize()
    return (r["shift"].cpu().numpy(), r["diag"]["flags"].cpu().numpy(), r["info"],
            r["lam"].cpu().numpy())


def compare(ae, fn, args, n, frac_max):
    s0, f0, _, _ = run(ae, fn, args, 0)
    s1, f1, i1, lam1 = run(ae, fn, args, 1)
    keep = ((f0 | f1) & REMEDY) == 0
    np.testing.assert_array_equal(s1[keep], s0[keep])
    assert np.all(np.isfinite(lam1))
    mid = int(np.count_nonzero(f1 & ae.FLAG_MID64))
    assert i1["n_mid64"] == mid
    assert not np.any(f0 & ae.FLAG_MID64)       # the flag belongs to the FP32 mode
    assert mid <= frac_max * n, (mid, n)
    return f1


@pytest.mark.parametrize("case", ["uniform", "graded", "clustered", "qdot", "ex1", "ex3"])
def test_midpoint_f32_picks_the_fp64_shift(ae, case):
    if case == "uniform":
        d, z, a = W.uniform_arrow(3000, seed=31)
    elif case == "graded":
        d, z, a = W.graded_arrow(4096, seed=32)
    elif case == "clustered":
        # poles in tight clusters: relative gaps down to 1e-12
        rng = np.random.default_rng(33)
        c = rng.uniform(-5, 5, 40)
        d = np.unique((c[:, None] * (1 + 1e-12 * np.arange(1, 26))).ravel())[::-1]
        z = 1.0 - rng.random(d.size)
        a = 0.5
    elif case == "qdot":
        d, z, a = W.quantum_dot_like(2501)
    else:
        d, z, a = W.paper_example(int(case[2]))
    n = len(d) + 1
    # tight clusters leave the FP32 copy too coarse for most midpoints there
    compare(ae, ae.arrow_eig, (t(d), t(z), a), n,
            0.05 if n > 100 and case != "clustered" else 1.0)


def test_midpoint_f32_hermitian_and_nonsymmetric(ae):
    d, z, a = W.uniform_herm(2000, seed=34)
    compare(ae, ae.herm_arrow_eig, (t(d), t(z), a), 2000, 0.05)
    d, zc, zr, a = W.graded_nsym(2000, seed=35)
    compare(ae, ae.nsym_arrow_eig, (t(d), t(zc), t(zr), a), 2000, 0.05)


def test_midpoint_zero_goes_to_fp64(ae):
    # d_j = -d_{n-j}, mirrored z, alpha = 0: F vanishes at the midpoint 0 of
    # the middle eigenvalue's interval, which no FP32 bound can sign
    d, z, a = W.mirrored_arrow(41)
    f1 = compare(ae, ae.arrow_eig, (t(d), t(z), a), 41, 1.0)
    assert f1[20] & ae.FLAG_MID64
