"""CPU checks of two error bounds the GPU solver relies on (no GPU, no oracle).

1. The local expansion that closes the Newton finish: within the radius
   H = min(2^-27 rho, err / (4 drel |c S'|)) of an FP64 evaluation at x,
       F(y) ~ F64(x) + (y - x) F'(x) + c (y - x)^2 / (x^2 y)
   differs from the exact F(y) by at most the error of F64(x) plus err / 2
   (err = 2^-52 (|b| + |x| + c (|S| + |1/x|)), the evaluation's rounding bound).
   Checked against 60-digit mpmath evaluations of the same function on the
   same double inputs, with a fresh F' and with one formed elsewhere.

2. Algorithm 1's midpoint test in FP32: the error bound that lets the FP32 sum
   decide the sign.  The FP32 computation is emulated in numpy float32 (IEEE
   round to nearest; the approximate reciprocal as the rounded one moved by up
   to one ulp), per lane and through the butterfly as the kernel sums, and the
   bound must cover the exact sum; where it decides, the FP64 sign agrees.
"""
import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")
mp = mpmath.mp


def _arrow(n, kind, seed):
    rng = np.random.default_rng(seed)
    if kind == "uniform":
        d = np.sort(rng.uniform(-10, 10, n - 1))[::-1]
        z = 1.0 - rng.random(n - 1)
        a = float(rng.normal())
    else:   # graded, as the benchmark matrix
        d = np.sort(rng.choice([-1.0, 1.0], n - 1) * 10.0 ** rng.uniform(-15, 0, n - 1))[::-1]
        z = 10.0 ** rng.uniform(-10, 0, n - 1)
        a = 1e3
    return d, z, a


def _shifted_problem(d, z, a, k):
    """Shift pole i nearest eigenvalue k, side, and the double inputs of F."""
    n = len(d) + 1
    A = np.diag(np.append(d, a))
    A[:-1, -1] = z
    A[-1, :-1] = z
    lam = np.sort(np.linalg.eigvalsh(A))[::-1][k]
    i = int(np.argmin(np.abs(d - lam)))
    side = 1 if lam > d[i] else -1
    mask = np.arange(n - 1) != i
    delta = d[mask] - d[i]                       # exact for these inputs or rounded once
    cj = z[mask] ** 2 / delta
    c = 1.0 / z[i] ** 2
    b = float(c * (-(a - d[i]) + np.sum(cj)))
    return delta, cj, c, b, side, lam - d[i]


def _F_exact(delta, cj, c, b, y):
    y = mp.mpf(y)
    S = mp.fsum(mp.mpf(q) / (1 - y * mp.mpf(dl)) for dl, q in zip(delta, cj))
    return (mp.mpf(b) - y) - mp.mpf(c) * (S - 1 / y)


def _F64(delta, cj, c, b, x):
    r = 1.0 / (1.0 - x * delta)
    q = cj * r
    S = q.sum()
    Sd = (q * delta * r).sum()
    rx = 1.0 / x
    F = (b - x) - c * (S - rx)
    dF = -1.0 - c * (Sd + rx * rx)
    err = 2.0 ** -52 * (abs(b) + abs(x) + c * (abs(S) + abs(rx)))
    return F, dF, err


@pytest.mark.parametrize("kind,seed", [("uniform", 1), ("uniform", 2), ("graded", 3),
                                       ("graded", 4)])
def test_local_expansion_within_rounding_bound(kind, seed):
    mp.dps = 60
    n = 40
    d, z, a = _arrow(n, kind, seed)
    checked = 0
    for k in range(1, n - 1, 3):
        delta, cj, c, b, side, mu0 = _shifted_problem(d, z, a, k)
        inv = 1.0 / delta
        on_side = inv[inv > 0] if side > 0 else inv[inv < 0]
        pole = (on_side.max() if side > 0 else on_side.min()) if on_side.size else 0.0
        nu = mp.findroot(lambda y: _F_exact(delta, cj, c, b, y), mp.mpf(1.0 / mu0))
        for rel in (2.0 ** -40, -3 * 2.0 ** -38):
            x = float(nu) * (1.0 + rel)
            rho = abs(x - pole)
            F, dF, err = _F64(delta, cj, c, b, x)
            e0 = abs(mp.mpf(F) - _F_exact(delta, cj, c, b, x))
            for xs, rsrc in ((x, 2.0 ** -40), (x * (1.0 + 2.0 ** -24), 2.0 ** -40)):
                # c S' at its source xs, moved to x as the kernel does
                _, dFs, _ = _F64(delta, cj, c, b, xs)
                cSs = -1.0 - dFs - c / xs / xs
                drel = rsrc + 4.0 * abs(x - xs) / rho
                H = min(2.0 ** -27 * rho, 0.25 * err / (drel * abs(cSs)))
                dFa = -1.0 - cSs - c / x / x
                for t in np.linspace(-1.0, 1.0, 9):
                    y = x + t * H
                    if y == x:
                        continue
                    h = y - x
                    Ft = F + h * (dFa + (c / x) * (h / x) / y)
                    dev = abs(mp.mpf(Ft) - _F_exact(delta, cj, c, b, y))
                    assert dev <= e0 + 0.5 * err + 4 * 2.0 ** -53 * abs(Ft), \
                        (kind, k, rel, t, float(dev), float(e0), err)
                    checked += 1
    assert checked > 100


def _emulate_midpoint_f32(d, z2, alpha_hi, k, rng):
    """The kernel's FP32 midpoint evaluation and its bound, in numpy float32."""
    f32 = np.float32
    m = len(d)
    ds = 2.0 ** -np.floor(np.log2(np.max(np.abs(d))))
    zs = 2.0 ** -np.floor(np.log2(np.max(z2)))
    v = d * ds
    pdh = v.astype(f32)
    pdl = (v - pdh.astype(np.float64)).astype(f32)
    pz2f = (z2 * zs).astype(f32)
    sk = d[k]
    middle = 0.5 * (d[k - 1] - sk)
    am = (alpha_hi - sk) - middle
    ss = sk * ds
    sh = f32(ss)
    sl = f32(ss - np.float64(sh))
    mf = f32(middle * ds)
    D = ((pdh - sh) + (pdl - sl)) - mf
    g = np.abs(pdh) + abs(sh)
    bad = bool(np.any(~(np.abs(D) >= g * f32(2.0 ** -20) + f32(2.0 ** -100))))
    r = (f32(1.0) / D).astype(f32)
    # the approximate reciprocal: within one ulp of the rounded one
    up = np.nextafter(r, np.float32(np.inf))
    dn = np.nextafter(r, np.float32(-np.inf))
    pick = rng.integers(0, 3, m)
    r = np.where(pick == 1, up, np.where(pick == 2, dn, r)).astype(f32)
    t = (pz2f * r).astype(f32)
    # per lane: j = lane, lane + 32, ...; two interleaved accumulators
    lanes = []
    for lane in range(32):
        idx = np.arange(lane, m, 32)
        acc = [[f32(0), f32(0), f32(0)], [f32(0), f32(0), f32(0)]]
        for q, j in enumerate(idx):
            a_ = acc[q % 2]              # pairs alternate; an odd last term goes first
            a_[0] = f32(a_[0] + t[j])
            a_[1] = f32(a_[1] + abs(t[j]))
            a_[2] = f32(a_[2] + abs(r[j]))
        lanes.append([f32(acc[0][i] + acc[1][i]) for i in range(3)])
    vals = np.array(lanes, dtype=f32)
    for o in (16, 8, 4, 2, 1):
        vals = (vals + vals[np.arange(32) ^ o]).astype(f32)
    tf, af, bf = (float(x) for x in vals[0])
    if bad:
        bf = np.inf
    L = float((m + 31) // 32)
    f = ds / zs
    F32 = am - f * tf
    ET = 2.0 * (L + 24.0) * 2.0 ** -24 * (2.0 * af) + 2.0 ** -148 * (bf + m)
    M = f * ET * (1.0 + 2.0 ** -20) + (L + 16.0) * 2.0 ** -52 * abs(am)
    return F32, M, f * ET, am, tf * f, bad


@pytest.mark.parametrize("kind,seed", [("uniform", 5), ("graded", 6), ("clustered", 7)])
def test_midpoint_f32_bound_covers_exact_sum(kind, seed):
    mp.dps = 50
    rng = np.random.default_rng(seed)
    n = 300
    if kind == "clustered":
        c = rng.uniform(-5, 5, 30)
        d = np.unique((c[:, None] * (1 + 1e-9 * np.arange(1, 11))).ravel())[::-1]
        z = 1.0 - rng.random(d.size)
        a = 0.5
    else:
        d, z, a = _arrow(n, kind, seed)
    z2 = z * z
    decided = 0
    for k in range(1, len(d)):
        F32, M, bound, am, S32, bad = _emulate_midpoint_f32(d, z2, a, k, rng)
        sk = d[k]
        middle = 0.5 * (d[k - 1] - sk)
        S_ex = mp.fsum(mp.mpf(q) / ((mp.mpf(dj) - mp.mpf(sk)) - mp.mpf(middle))
                       for dj, q in zip(d, z2))
        if not bad:
            assert abs(mp.mpf(S32) - S_ex) <= bound, (kind, k)
        if np.isfinite(F32) and abs(F32) > M * (1.0 + 2.0 ** -40):
            # the FP64 test, as the kernel runs it
            F64 = am - np.sum(z2 / ((d - sk) - middle))
            assert np.sign(F64) == np.sign(F32), (kind, k)
            decided += 1
    if kind != "clustered":
        assert decided >= 0.9 * (len(d) - 1)
