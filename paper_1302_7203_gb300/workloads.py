"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the eigen-solver: it only draws inputs
(numpy PCG64, fixed draw order) so that the CUDA path and the CPU oracle can
be fed identical data.  The matrix order is ``n``; an arrowhead has
``n - 1`` poles ``d`` and spikes ``z`` plus the corner ``alpha``.

Recipes (the paper measures on no public data; its only application matrix,
the quantum-dot example of Sec. 5, is not published, so a stand-in with the
printed ranges is provided):

* ``uniform_arrow``  -- d ~ U[-10, 10] sorted descending, z = 1 - U[0, 1)
  (so z in (0, 1]), alpha ~ N(0, 1).
* ``graded_arrow``   -- |d| = 10^u, u ~ U[-15, 0], random signs, sorted
  descending; z = 10^w, w ~ U[-10, 0]; alpha = 1e3.
* ``batch_sizes``    -- instance orders round(exp(U[ln 32, ln 4096])).
* ``uniform_dpr1``   -- d ~ U[0, 1] sorted descending, u ~ N(0, 1) / ||u||,
  rho = 0.5.
* ``uniform_tsvd``   -- d ~ U(0, 1] sorted descending, z ~ N(0, 1),
  alpha ~ U(0, 1].
* ``quantum_dot_like`` -- n = 2501-style stand-in: d ~ U[5.87e14, 1.38e15],
  z log-uniform in [1.05e4, 1.10e7], alpha = 9.7949881500060375e14.
* ``paper_example(k)`` -- the 6x6, 5x5 and 6x6 matrices of Examples 1-3.

Distinctness of d is enforced by redrawing duplicates (never needed in
practice for these continuous distributions).
"""
from __future__ import annotations

import math

import numpy as np

EPS_M = 2.0 ** -52   # the paper's machine precision (Sec. 1 footnote)


def _sorted_distinct(draw, count, rng):
    vals = draw(count)
    for _ in range(100):
        vals = np.sort(vals)[::-1].copy()
        dup = np.nonzero(vals[1:] == vals[:-1])[0]
        if dup.size == 0:
            return vals
        vals[dup + 1] = draw(dup.size)
    raise RuntimeError("could not draw distinct poles")


def uniform_arrow(n: int, seed: int = 0):
    """Arrowhead of order n: d ~ U[-10,10] desc, z in (0,1], alpha ~ N(0,1)."""
    rng = np.random.default_rng(seed)
    d = _sorted_distinct(lambda c: rng.uniform(-10.0, 10.0, c), n - 1, rng)
    z = 1.0 - rng.random(n - 1)
    alpha = float(rng.standard_normal())
    return d, z, alpha


def graded_arrow(n: int, seed: int = 1):
    """Graded arrowhead: |d| = 10^U[-15,0] with random signs, z = 10^U[-10,0]."""
    rng = np.random.default_rng(seed)

    def draw(c):
        u = rng.uniform(-15.0, 0.0, c)
        s = np.where(rng.random(c) < 0.5, -1.0, 1.0)
        return s * 10.0 ** u

    d = _sorted_distinct(draw, n - 1, rng)
    z = 10.0 ** rng.uniform(-10.0, 0.0, n - 1)
    alpha = 1.0e3
    return d, z, alpha


def uniform_herm(n: int, seed: int = 8):
    """Hermitian arrowhead (Sec. 6.1): d as uniform_arrow, |zeta| = 1 - U[0,1),
    phase U[0, 2 pi), alpha ~ N(0,1).  Returns (d, z complex, alpha)."""
    d, r, alpha = uniform_arrow(n, seed=seed)
    rng = np.random.default_rng(seed + 1000)
    z = r * np.exp(1j * rng.uniform(0.0, 2.0 * np.pi, n - 1))
    return d, z, alpha


def graded_herm(n: int, seed: int = 9):
    """Graded Hermitian arrowhead: d, |zeta| as graded_arrow, uniform phases."""
    d, r, alpha = graded_arrow(n, seed=seed)
    rng = np.random.default_rng(seed + 1000)
    z = r * np.exp(1j * rng.uniform(0.0, 2.0 * np.pi, n - 1))
    return d, z, alpha


def uniform_nsym(n: int, seed: int = 10):
    """Non-symmetric arrowhead (Remark, Sec. 6.1): d as uniform_arrow; column
    spikes zc with random signs and |zc| = 1 - U[0,1); row spikes zr = zc t,
    t = 10^U[-2,2] (same sign).  Returns (d, zc, zr, alpha)."""
    d, r, alpha = uniform_arrow(n, seed=seed)
    rng = np.random.default_rng(seed + 1000)
    zc = np.where(rng.random(n - 1) < 0.5, -1.0, 1.0) * r
    zr = zc * 10.0 ** rng.uniform(-2.0, 2.0, n - 1)
    return d, zc, zr, alpha


def graded_nsym(n: int, seed: int = 11):
    """Graded non-symmetric arrowhead: d as graded_arrow, |zc| = 10^U[-10,0],
    zr = zc 10^U[-3,3]."""
    d, r, alpha = graded_arrow(n, seed=seed)
    rng = np.random.default_rng(seed + 1000)
    zc = np.where(rng.random(n - 1) < 0.5, -1.0, 1.0) * r
    zr = zc * 10.0 ** rng.uniform(-3.0, 3.0, n - 1)
    return d, zc, zr, alpha


def batch_sizes(count: int = 4096, lo: int = 32, hi: int = 4096, seed: int = 2):
    """Instance orders, log-uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    n = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), count))).astype(np.int64)
    return np.clip(n, lo, hi)


def uniform_batch(count: int = 4096, lo: int = 32, hi: int = 4096, seed: int = 2):
    """A batch of uniform arrowheads of log-uniform orders (list of (d, z, alpha))."""
    sizes = batch_sizes(count, lo, hi, seed)
    return [uniform_arrow(int(n), seed=int(seed) * 1_000_003 + i) for i, n in enumerate(sizes)]


def uniform_dpr1(n: int, seed: int = 3):
    """DPR1 D + rho u u^T of order n: d ~ U[0,1] desc, u ~ N(0,1)/||u||, rho = 0.5."""
    rng = np.random.default_rng(seed)
    d = _sorted_distinct(lambda c: rng.uniform(0.0, 1.0, c), n, rng)
    u = rng.standard_normal(n)
    u /= np.linalg.norm(u)
    return d, u, 0.5


def uniform_tsvd(n: int, seed: int = 4):
    """Upper triangular arrowhead [diag(d) z; 0 alpha] of order n."""
    rng = np.random.default_rng(seed)
    d = _sorted_distinct(lambda c: 1.0 - rng.random(c), n - 1, rng)
    z = rng.standard_normal(n - 1)
    alpha = float(1.0 - rng.random())
    return d, z, alpha


def quantum_dot_like(n: int = 2501, seed: int = 6):
    """Stand-in with the ranges printed for the quantum-dot example (Sec. 5)."""
    rng = np.random.default_rng(seed)
    d = _sorted_distinct(lambda c: rng.uniform(5.87e14, 1.38e15, c), n - 1, rng)
    z = 10.0 ** rng.uniform(math.log10(1.05e4), math.log10(1.10e7), n - 1)
    return d, z, 9.7949881500060375e14


def paper_example(k: int):
    """Inputs (d, z, alpha) of Examples 1, 2 and 3 of Sec. 5."""
    if k == 1:
        return (np.array([2e-3, 1e-7, 0.0, -1e-7, -2e-3]),
                np.array([1e7, 1e7, 1.0, 1e7, 1e7]), 1e20)
    if k == 2:
        e = EPS_M
        return (np.array([1 + 4 * e, 1 + 3 * e, 1 + 2 * e, 1 + e]),
                np.array([1.0, 2.0, 3.0, 4.0]), 0.0)
    if k == 3:
        return (np.array([1e10, 4.0, 3.0, 2.0, 1.0]),
                np.array([1e10, 1.0, 1.0, 1.0, 1.0]), 1e10)
    raise ValueError(k)


def mirrored_arrow(n: int, seed: int = 7):
    """Odd-order arrowhead with d_j = -d_{n-j}, mirrored z, alpha = 0.

    Its spectrum is symmetric about 0 and contains 0 exactly (the symmetric
    middle eigenvalue)."""
    assert n % 2 == 1
    rng = np.random.default_rng(seed)
    h = (n - 1) // 2
    pos = _sorted_distinct(lambda c: rng.uniform(0.1, 10.0, c), h, rng)
    zp = 1.0 - rng.random(h)
    d = np.concatenate([pos, -pos[::-1]])
    z = np.concatenate([zp, zp[::-1]])
    return d, z, 0.0


def serve_stream(rate: float, count: int, seed: int = 5, lo: int = 64, hi: int = 16384):
    """Poisson arrivals: (t_arrival[s], kind[0 arrow|1 dpr1|2 tsvd], n) per request."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, count)
    kinds = rng.integers(0, 3, count)
    n = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), count))).astype(np.int64)
    return np.cumsum(gaps), kinds, np.clip(n, lo, hi)
