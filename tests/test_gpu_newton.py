"""GPU parity of the bracketed-Newton finish (ae_opts.finish = AE_FINISH_NEWTON).

The Newton finish searches the same Pick function of the shifted inverse as
Algorithm 3, keeps a sign-change bracket of it and stops on the same test, so
its eigenpairs must meet the same bar against the CPU oracle: 10 n eps64 per
eigenvalue and per vector component.  Covered with and without the FP32
opening bracket, on the paper's examples, uniform, graded and quantum-dot-like
spectra, deflation, the DPR1 and SVD wrappers and the batched path; plus exact
invariances and the evaluation count it exists to cut.
"""
import numpy as np
import pytest

import oracle
from parity import assert_parity, widened
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


def opts(ae, precision):
    return ae.default_opts(precision=precision, finish=ae.AE_FINISH_NEWTON)


def solve(ae, d, z, a, o, **kw):
    r = ae.arrow_eig(t(d), t(z), a, opts=o, info=True, **kw)
    torch.cuda.synchronize()
    out = {"lam": r["lam"].cpu().numpy(), "V": r["V"].cpu().numpy(), "info": r["info"]}
    if "diag" in r:
        out["diag"] = {k: v.cpu().numpy() for k, v in r["diag"].items()}
    return out


CASES = ["ex1", "ex2", "ex3", "uniform1000", "graded3001", "qdot", "mirrored", "deflation",
         "n2", "n33"]


def case_data(case):
    if case.startswith("ex"):
        return W.paper_example(int(case[2]))
    if case == "uniform1000":
        return W.uniform_arrow(1000, seed=0)
    if case == "graded3001":
        return W.graded_arrow(3001, seed=13)
    if case == "qdot":
        return W.quantum_dot_like(2501)
    if case == "mirrored":
        return W.mirrored_arrow(41)
    if case == "n2":
        return np.array([0.75]), np.array([-0.5]), 2.0
    if case == "n33":
        return W.uniform_arrow(33, seed=33)
    d = np.array([0.5, 3.0, 2.0, 3.0, -1.0, 3.0, 2.0, 7.5, -1.0, 0.25])
    z = np.array([0.5, -1.0, 0.0, 2.0, 1.0, -0.0, 0.25, -3.0, 0.125, 1.5])
    return d, z, 0.3


@pytest.mark.parametrize("gate", [0, 1])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("case", CASES)
def test_newton_parity(ae, case, precision, gate):
    d, z, a = case_data(case)
    o_ = opts(ae, precision)
    o_.bgate = gate
    g = solve(ae, d, z, a, o_)
    o = oracle.arrow_eig(d, z, a)
    assert_parity(g["lam"], g["V"], o, len(d) + 1,
                  what=f"newton p={precision} gate={gate} {case}")
    assert g["info"]["n_capped"] == 0


def test_newton_cuts_fp64_evaluations(ae):
    d, z, a = W.graded_arrow(4000, seed=17)
    gb = solve(ae, d, z, a, ae.default_opts(precision=1))
    gn = solve(ae, d, z, a, opts(ae, 1))
    ib, inn = gb["info"], gn["info"]
    n_pairs = len(d) + 1
    # bisection needs ~30 FP64 steps after the FP32 bracket; Newton a handful
    assert ib["total_iter"] > 25 * n_pairs
    assert inn["total_iter"] < 6 * n_pairs
    assert inn["n_fp32_fallback"] <= 0.01 * n_pairs


def test_newton_close_to_bisection(ae):
    # both return the right end of a 2 eps-wide bracket of the same computed
    # function; away from rounding noise they agree to a few ulps
    d, z, a = W.uniform_arrow(1500, seed=2)
    gb = solve(ae, d, z, a, ae.default_opts(precision=1))
    gn = solve(ae, d, z, a, opts(ae, 1))
    rel = np.abs(gn["lam"] - gb["lam"]) / np.abs(gb["lam"])
    assert np.median(rel) <= 2.0 ** -52
    assert rel.max() <= 10 * len(z) * 2.0 ** -53


def test_newton_scale_and_sign_invariance(ae):
    d, z, a = W.graded_arrow(700, seed=21)
    o = opts(ae, 1)
    g0 = solve(ae, d, z, a, o)
    g2 = solve(ae, d * 2.0 ** 40, z * 2.0 ** 40, a * 2.0 ** 40, o)
    np.testing.assert_array_equal(g2["lam"], g0["lam"] * 2.0 ** 40)
    np.testing.assert_array_equal(g2["V"], g0["V"])
    zs = z.copy()
    zs[[0, 5, 99]] *= -1
    g3 = solve(ae, d, zs, a, o)
    V = g0["V"].copy()
    V[[0, 5, 99]] *= -1
    np.testing.assert_array_equal(g3["lam"], g0["lam"])
    np.testing.assert_array_equal(g3["V"], V)


def test_newton_full_size_sampled(ae):
    n = 16384
    d, z, a = W.graded_arrow(n, seed=1)
    g = solve(ae, d, z, a, opts(ae, 1), diag=True)
    lam, V = g["lam"], g["V"]
    assert np.all(lam[:-1] >= d) and np.all(d >= lam[1:])
    np.testing.assert_allclose(np.linalg.norm(V, axis=0), 1.0, atol=4 * n * 2.0 ** -53)
    flags = g["diag"]["flags"]
    fixed = np.nonzero(flags & (ae.FLAG_NEARZERO | ae.FLAG_OTHERPOLE | ae.FLAG_DPR1SHIFT))[0]
    fb = np.nonzero(flags & ae.FLAG_FP32_FALLBACK)[0]
    rng = np.random.default_rng(9)
    ks = np.unique(np.concatenate([[0, 1, n // 2, n - 2, n - 1],
                                   rng.choice(n, 96, replace=False), fixed[:32], fb[:32]]))
    o = oracle.arrow_eig(d, z, a, ks=ks)
    assert not widened(o, n).any()   # every comparison at the full 10 n eps64 bar
    assert_parity(lam[ks], V[:, ks], o, n, cols=ks, what="newton graded n=16384 sampled")
    assert g["info"]["total_iter"] < 6 * n


@pytest.mark.parametrize("n", [3, 65, 1000])
def test_newton_dpr1_and_svd(ae, n):
    o = opts(ae, 1)
    d, u, rho = W.uniform_dpr1(n, seed=300 + n)
    r = ae.dpr1_eig(t(d), t(u), rho, opts=o)
    torch.cuda.synchronize()
    ref = oracle.dpr1_eig(d, u, rho)
    assert_parity(r["lam"].cpu().numpy(), r["Q"].cpu().numpy(),
                  {"lam": ref["lam"], "abserr": np.zeros(n), "V": ref["Q"]}, n,
                  what=f"newton dpr1 n={n}")
    d, z, a = W.uniform_tsvd(n, seed=400 + n)
    r = ae.tri_arrow_svd(t(d), t(z), a, opts=o)
    torch.cuda.synchronize()
    ref = oracle.tsvd(d, z, a)
    s = r["s"].cpu().numpy()
    assert_parity(s, r["V"].cpu().numpy(), {"lam": ref["s"], "abserr": np.zeros(n), "V": ref["V"]},
                  n, what=f"newton svd n={n} (V)")
    assert_parity(s, r["U"].cpu().numpy(), {"lam": ref["s"], "abserr": np.zeros(n), "V": ref["U"]},
                  n, what=f"newton svd n={n} (U)")


@pytest.mark.parametrize("precision", [0, 1])
def test_many_remedies_one_warp_each(ae, precision):
    # K_nu > 1 sends about a third of the eigenpairs to Remark 2: more than a
    # quarter of the remedy grid's warps (at most 3648 on 152 SMs), so the
    # remedy kernel gives each its own warp (with few remedies it uses a CTA
    # each); same parity bar
    d, z, a = W.uniform_arrow(4000, seed=51)
    o = opts(ae, precision)
    o.knu_max = 1.0
    g = solve(ae, d, z, a, o)
    info = g["info"]
    assert info["n_otherpole"] + info["n_dpr1shift"] >= 1000
    assert_parity(g["lam"], g["V"], oracle.arrow_eig(d, z, a), len(d) + 1,
                  what=f"many remedies p={precision}")


def test_newton_batched(ae):
    sizes = W.batch_sizes(40, lo=2, hi=900, seed=44)
    inst = [W.uniform_arrow(int(n), seed=4400 + i) for i, n in enumerate(sizes)]
    inst.append(W.graded_arrow(500, seed=45))
    B = ae.Batch(inst, opts=opts(ae, 1))
    B.run()
    torch.cuda.synchronize()
    assert np.all(B.status.cpu().numpy() == 0)
    for i, (d, z, a) in enumerate(inst):
        assert_parity(B.lam(i).cpu().numpy(), B.V(i).cpu().numpy(), oracle.arrow_eig(d, z, a),
                      len(d) + 1, what=f"newton batch instance {i}")
    B.close()


@pytest.mark.parametrize("e", [-400, -300, 300, 400])
@pytest.mark.parametrize("form", [(0, 0, 0), (0, 1, 1), (1, 1, 0), (1, 1, 1)])
def test_extreme_power_of_two_scaling(ae, e, form):
    # A -> 2^e A scales every eigenvalue by 2^e and leaves the vectors, exactly,
    # as long as the squares the solve forms (zeta^2, delta^2, 1/zeta_i^2) stay
    # in range: here |entries| from 2^-450 to 2^400
    d, z, a = W.graded_arrow(300, seed=23)
    o = ae.default_opts(precision=form[0], finish=form[1], bgate=form[2])
    g0 = solve(ae, d, z, a, o)
    s = 2.0 ** e
    g1 = solve(ae, d * s, z * s, a * s, o)
    if form[0] == 0:
        np.testing.assert_array_equal(g1["lam"], g0["lam"] * s)
        np.testing.assert_array_equal(g1["V"], g0["V"])
    else:
        # the FP32 opening bracket has float's narrower exponent range: where
        # its rescaled copy cannot represent the problem it falls back, so the
        # FP64 finish starts elsewhere; same tolerance, not the same bits
        tol = 10 * len(d) * 2.0 ** -53
        assert np.all(np.abs(g1["lam"] - g0["lam"] * s) <= tol * np.abs(g0["lam"] * s))
        assert np.all(np.abs(g1["V"] - g0["V"]) <= tol * np.abs(g0["V"]) + 1e-300)


def _pick_function(k):
    # the shifted inverse of the n = 16384 graded matrix at eigenvalue k's pole
    # sigma (the oracle's shift), as the finish sees it: differences, c_j, b, c
    import math
    n = 16384
    d, z, a = W.graded_arrow(n, seed=1)
    order = np.argsort(-d)
    ds, zs = d[order], np.abs(z[order])
    ref = oracle.arrow_eig(d, z, a, ks=[k], vectors=False)
    sigma = ref["sigma"][0]
    i = int(np.flatnonzero(ds == sigma)[0])
    nu = 1.0 / (ref["mu_hi"][0] + ref["mu_lo"][0])
    keep = np.arange(n - 1) != i
    delta = ds[keep] - sigma
    cj = zs[keep] ** 2 / delta
    c = 1.0 / zs[i] ** 2
    b = math.fsum(list(cj) + [-(a - sigma)]) * c
    side = 1 if nu > 0 else -1
    jn = i - 1 if side > 0 else i + 1
    pole = 1.0 / (ds[jn] - sigma)
    return delta, cj, b, c, side, pole, nu


def _dF(delta, cj, c, x):
    t = 1.0 / (1.0 - x * delta)
    return -1.0 - c * (1.0 / x ** 2 + np.sum(cj * delta * t * t))


@pytest.mark.parametrize("k", [6340, 9953])
def test_stale_derivative_near_a_pole_does_not_stall(ae, k):
    # two eigenvalues within 1e-11 of zero whose shifted inverse has its zero
    # 5x (k = 6340) and 3x (k = 9953) farther out than its nearest pole.  A
    # start 1e-7 (relative) beyond that pole, with F' taken 1e-9 beyond it (as
    # a short FP32 opening step can hand over, |F'| there 10^4 too large):
    # the finish must evaluate F' again once its steps stay short against the
    # pole's distance, and close on the zero the oracle gives.  Reusing F'
    # while steps were short against |x| kept every step short: 300 FP64
    # evaluations ended next to the pole.
    delta, cj, b, c, side, pole, nu = _pick_function(k)
    far = nu * 8.0 if side < 0 else nu * 8.0
    left, right = (far, pole) if side < 0 else (pole, far)
    x0 = pole * (1.0 + 1e-7)
    xs = pole * (1.0 + 1e-9)
    dF0 = _dF(delta, cj, c, xs)
    got, it, itd = ae.debug_newton(t(delta), t(cj), b, c, side, pole, left, right, x0=x0,
                                   dF0=dF0, max_iter=300)
    assert it < 40, (it, itd)
    assert itd >= 1
    assert abs(got - nu) <= 1e-12 * abs(nu), (got, nu)
    # the same from the bracket's middle with no estimate
    got2, it2, _ = ae.debug_newton(t(delta), t(cj), b, c, side, pole, left, right, max_iter=300)
    assert it2 < 40 and abs(got2 - nu) <= 1e-12 * abs(nu)
