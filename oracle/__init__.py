"""CPU oracle for the arrowhead eigen-solver -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product path never does, and the oracle shares no code with it.

The numerics live in ``arrow_oracle.c`` (plain C, double-double arithmetic
plus binary128 Jacobi for brute force); this module only compiles it and
marshals numpy arrays through ctypes.  What each routine computes, with the
paper passage it follows, is stated in the C file's header.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "arrow_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def _cpu_has_fma() -> bool:
    try:
        with open("/proc/cpuinfo") as f:
            return " fma " in f.read()
    except OSError:
        return False


def build_oracle(force: bool = False) -> str:
    """Compile arrow_oracle.c into oracle/_lib/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-std=gnu11", _SRC, "-o", _LIB + ".tmp", "-lm"]
    mach = platform.machine()
    if mach in ("x86_64", "AMD64"):
        cmd.append("-lquadmath")
        if _cpu_has_fma():
            cmd.insert(1, "-mfma")
    subprocess.run(cmd, check=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build_oracle()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        lib.oracle_arrow_eig.argtypes = [I, P, P, D, P, I, P, P, P, P, P, P, P, P, I]
        lib.oracle_arrow_eig.restype = I
        lib.oracle_herm_eig.argtypes = [I, P, P, P, D, P, I, P, P, P, P, P, P, P, P, P, I]
        lib.oracle_herm_eig.restype = I
        lib.oracle_nsym_eig.argtypes = [I, P, P, P, D, P, I, P, P, P, P, P, P, P, P, P, I]
        lib.oracle_nsym_eig.restype = I
        lib.oracle_reduce.argtypes = [I, P, P, P, P, P]
        lib.oracle_reduce.restype = I
        lib.oracle_inverse_element.argtypes = [I, P, P, D, I, P, P, P]
        lib.oracle_inverse_element.restype = I
        lib.oracle_dpr1_eig.argtypes = [I, P, P, D, P, I, P, P, P, I]
        lib.oracle_dpr1_eig.restype = I
        lib.oracle_tsvd.argtypes = [I, P, P, D, P, I, P, P, P, P, I]
        lib.oracle_tsvd.restype = I
        lib.oracle_jacobi_sym.argtypes = [I, P, P, P, P, I]
        lib.oracle_jacobi_sym.restype = I
        lib.oracle_jacobi_svd.argtypes = [I, P, P, P, P, I]
        lib.oracle_jacobi_svd.restype = I
        lib.oracle_dd_ops.argtypes = [D, D, D, D, P]
        lib.oracle_dd_ops.restype = None
        lib.oracle_threads.argtypes = []
        lib.oracle_threads.restype = I
        _lib = lib
        return lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data


def threads() -> int:
    """Number of OpenMP threads the oracle uses by default."""
    return _load().oracle_threads()


def arrow_eig(d, z, alpha, ks=None, vectors=True, nthreads=0):
    """Eigen-decomposition of A = [diag(d) z; z^T alpha] (order n = len(d)+1).

    Returns a dict with ``lam`` (descending), ``lam_lo`` (dd tail), the shift
    representation ``sigma`` + (``mu_hi`` + ``mu_lo``), ``relerr`` (the oracle's
    own relative error bound per eigenvalue; ``abserr`` the absolute one) and ``V`` (n x len(ks), rows in
    input order) when ``vectors``.  ``ks`` selects output positions.
    """
    lib = _load()
    d = _f64(d)
    z = _f64(z)
    n = d.size + 1
    if ks is None:
        kk = None
        nk = n
    else:
        kk = np.ascontiguousarray(ks, dtype=np.int32)
        nk = kk.size
    out = {k: np.zeros(nk) for k in ("lam", "lam_lo", "sigma", "mu_hi", "mu_lo", "relerr",
                                     "abserr")}
    V = np.zeros((nk, n)) if vectors else None   # row-major (nk, n) == col-major (n, nk)
    rc = lib.oracle_arrow_eig(n, _ptr(d), _ptr(z), float(alpha), _ptr(kk), nk,
                              _ptr(out["lam"]), _ptr(out["lam_lo"]), _ptr(out["sigma"]),
                              _ptr(out["mu_hi"]), _ptr(out["mu_lo"]), _ptr(out["relerr"]),
                              _ptr(out["abserr"]), _ptr(V), int(nthreads))
    if rc != 0:
        raise ValueError("oracle_arrow_eig: invalid input")
    if vectors:
        out["V"] = V.T.copy()
    return out


def _scalars(nk):
    return {k: np.zeros(nk) for k in ("lam", "lam_lo", "sigma", "mu_hi", "mu_lo", "relerr",
                                      "abserr")}


def _ks(ks, n):
    if ks is None:
        return None, n
    kk = np.ascontiguousarray(ks, dtype=np.int32)
    return kk, kk.size


def herm_eig(d, z, alpha, ks=None, vectors=True, nthreads=0):
    """Eigen-decomposition of the Hermitian arrowhead C = [diag(d) z; z^* alpha]
    (Sec. 6.1), z complex (len(d) entries, the column above the corner).

    Same keys as arrow_eig; ``U`` is complex (n x len(ks)), rows in input order.
    """
    lib = _load()
    d = _f64(d)
    z = np.asarray(z, dtype=np.complex128)
    zre, zim = _f64(z.real), _f64(z.imag)
    n = d.size + 1
    kk, nk = _ks(ks, n)
    out = _scalars(nk)
    Ur = np.zeros((nk, n)) if vectors else None
    Ui = np.zeros((nk, n)) if vectors else None
    rc = lib.oracle_herm_eig(n, _ptr(d), _ptr(zre), _ptr(zim), float(alpha), _ptr(kk), nk,
                             _ptr(out["lam"]), _ptr(out["lam_lo"]), _ptr(out["sigma"]),
                             _ptr(out["mu_hi"]), _ptr(out["mu_lo"]), _ptr(out["relerr"]),
                             _ptr(out["abserr"]), _ptr(Ur), _ptr(Ui), int(nthreads))
    if rc != 0:
        raise ValueError("oracle_herm_eig: invalid input")
    if vectors:
        out["U"] = (Ur + 1j * Ui).T.copy()
    return out


def nsym_eig(d, zc, zr, alpha, ks=None, vectors=True, nthreads=0):
    """Eigen-decomposition of the non-symmetric arrowhead G = [diag(d) zc; zr^T alpha]
    (Remark, Sec. 6.1), zc_r zr_r > 0 or both zero.

    Same keys as arrow_eig; ``X`` right and ``Y`` left eigenvectors (n x len(ks)),
    scaled so that y_k^T x_k = 1.
    """
    lib = _load()
    d = _f64(d)
    zc = _f64(zc)
    zr = _f64(zr)
    n = d.size + 1
    kk, nk = _ks(ks, n)
    out = _scalars(nk)
    X = np.zeros((nk, n)) if vectors else None
    Y = np.zeros((nk, n)) if vectors else None
    rc = lib.oracle_nsym_eig(n, _ptr(d), _ptr(zc), _ptr(zr), float(alpha), _ptr(kk), nk,
                             _ptr(out["lam"]), _ptr(out["lam_lo"]), _ptr(out["sigma"]),
                             _ptr(out["mu_hi"]), _ptr(out["mu_lo"]), _ptr(out["relerr"]),
                             _ptr(out["abserr"]), _ptr(X), _ptr(Y), int(nthreads))
    if rc != 0:
        raise ValueError("oracle_nsym_eig: invalid input")
    if vectors:
        out["X"] = X.T.copy()
        out["Y"] = Y.T.copy()
    return out


def reduce(d, z):
    """Reduction decisions: (order, kind, head, m); see arrow_oracle.c."""
    lib = _load()
    d = _f64(d)
    z = _f64(z)
    n1 = d.size
    order = np.zeros(n1, np.int32)
    kind = np.zeros(n1, np.int32)
    head = np.zeros(n1, np.int32)
    m = lib.oracle_reduce(n1, _ptr(d), _ptr(z), _ptr(order), _ptr(kind), _ptr(head))
    return order, kind, head, m


def inverse_element(d, z, alpha, i):
    """b = [(A - d_i I)^{-1}]_{ii} in double-double and K_b (Eq. K2)."""
    lib = _load()
    d = _f64(d)
    z = _f64(z)
    hi = np.zeros(1)
    lo = np.zeros(1)
    kb = np.zeros(1)
    rc = lib.oracle_inverse_element(d.size + 1, _ptr(d), _ptr(z), float(alpha), int(i),
                                    _ptr(hi), _ptr(lo), _ptr(kb))
    if rc != 0:
        raise ValueError("bad index")
    return float(hi[0]), float(lo[0]), float(kb[0])


def dpr1_eig(d, u, rho, ks=None, vectors=True, nthreads=0):
    """Eigen-decomposition of D + rho u u^T: ``lam`` descending, ``Q`` columns."""
    lib = _load()
    d = _f64(d)
    u = _f64(u)
    n = d.size
    kk = None if ks is None else np.ascontiguousarray(ks, dtype=np.int32)
    nk = n if ks is None else kk.size
    lam = np.zeros(nk)
    rel = np.zeros(nk)
    Q = np.zeros((nk, n)) if vectors else None
    rc = lib.oracle_dpr1_eig(n, _ptr(d), _ptr(u), float(rho), _ptr(kk), nk, _ptr(lam),
                             _ptr(rel), _ptr(Q), int(nthreads))
    if rc != 0:
        raise ValueError("oracle_dpr1_eig: invalid input")
    out = {"lam": lam, "relerr": rel}
    if vectors:
        out["Q"] = Q.T.copy()
    return out


def tsvd(d, z, alpha, ks=None, vectors=True, nthreads=0):
    """SVD of B = [diag(d) z; 0 alpha]: ``s`` descending, ``U``, ``V`` columns."""
    lib = _load()
    d = _f64(d)
    z = _f64(z)
    n = d.size + 1
    kk = None if ks is None else np.ascontiguousarray(ks, dtype=np.int32)
    nk = n if ks is None else kk.size
    s = np.zeros(nk)
    rel = np.zeros(nk)
    U = np.zeros((nk, n)) if vectors else None
    V = np.zeros((nk, n)) if vectors else None
    rc = lib.oracle_tsvd(n, _ptr(d), _ptr(z), float(alpha), _ptr(kk), nk, _ptr(s),
                         _ptr(rel), _ptr(U), _ptr(V), int(nthreads))
    if rc != 0:
        raise ValueError("oracle_tsvd: invalid input")
    out = {"s": s, "relerr": rel}
    if vectors:
        out["U"] = U.T.copy()
        out["V"] = V.T.copy()
    return out


def jacobi_sym(A, max_sweeps=60):
    """Binary128 cyclic Jacobi: (lam_hi, lam_lo, V) sorted descending."""
    lib = _load()
    A = np.asfortranarray(A, dtype=np.float64)
    n = A.shape[0]
    hi = np.zeros(n)
    lo = np.zeros(n)
    V = np.zeros((n, n), order="F")
    lib.oracle_jacobi_sym(n, A.ctypes.data, _ptr(hi), _ptr(lo), V.ctypes.data, max_sweeps)
    idx = np.lexsort((-lo, -hi))
    return hi[idx], lo[idx], np.asarray(V)[:, idx]


def jacobi_svd(B, max_sweeps=60):
    """Binary128 one-sided Jacobi SVD: (s, U, V) sorted descending."""
    lib = _load()
    B = np.asfortranarray(B, dtype=np.float64)
    n = B.shape[0]
    s = np.zeros(n)
    U = np.zeros((n, n), order="F")
    V = np.zeros((n, n), order="F")
    lib.oracle_jacobi_svd(n, B.ctypes.data, _ptr(s), U.ctypes.data, V.ctypes.data, max_sweeps)
    idx = np.argsort(-s, kind="stable")
    return s[idx], np.asarray(U)[:, idx], np.asarray(V)[:, idx]


def dd_ops(a_hi, a_lo, b_hi, b_lo):
    """(a+b, a*b, a/b, sqrt|a|) in the oracle's double-double, as (hi, lo) pairs."""
    out = np.zeros(8)
    _load().oracle_dd_ops(a_hi, a_lo, b_hi, b_lo, out.ctypes.data)
    return [(out[2 * i], out[2 * i + 1]) for i in range(4)]
