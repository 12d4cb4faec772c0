"""Thin ctypes binding of libarrowhead.so (include/arrowhead.h).

Argument marshalling only: every step of the solve runs in the CUDA library.
PyTorch supplies device memory and the stream.  There is no CPU fallback: if
the library has not been built, or no GPU is present, calls raise.

Low-level symbols carry the C names (``lib().arrow_eig`` ...); the wrappers
below with the same names take torch tensors and return torch tensors.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libarrowhead.so")

AE_OK = 0
AE_ERR_CUDA = 1001
AE_ERR_INPUT = 1002
AE_ERR_NOCONV = 1003
AE_FP64 = 0
AE_FP32_BRACKET = 1
AE_FINISH_BISECT = 0
AE_FINISH_NEWTON = 1
FLAG_DEFLATED, FLAG_NEARZERO, FLAG_OTHERPOLE, FLAG_DPR1SHIFT = 1, 2, 4, 8
FLAG_CAPPED, FLAG_SINGULAR, FLAG_FP32_FALLBACK, FLAG_DDB = 16, 32, 64, 128
FLAG_MID64 = 256

# every symbol include/arrowhead.h declares
EXPORTED = ["ae_default_opts", "ae_status_string", "ae_last_cuda_error", "arrow_eig",
            "herm_arrow_eig", "nsym_arrow_eig",
            "dpr1_eig", "tri_arrow_svd", "arrow_eig_batched", "ae_batch_create",
            "ae_batch_run", "ae_batch_info", "ae_batch_destroy", "ae_autotune",
            "ae_team_width", "ae_serve_create", "ae_serve_submit", "ae_serve_poll",
            "ae_serve_result", "ae_serve_release", "ae_serve_stats", "ae_serve_destroy",
            "arrow_eig_host", "arrow_eig_noalloc", "arrow_eig_part", "arrow_eig_part_size",
            "ae_fma_peaks", "ae_debug_rcp", "ae_debug_newton"]
AE_EAGAIN = 1005
KIND_ARROW, KIND_DPR1, KIND_SVD = 0, 1, 2
REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_ERROR = 0, 1, 2, 3
AE_ERR_TOO_LARGE = 1004


class AeOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("knu_max", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("fixup", ctypes.c_int),
                ("profile", ctypes.c_int), ("finish", ctypes.c_int),
                ("bgate", ctypes.c_int), ("kb_max", ctypes.c_double)]


class AeInfo(ctypes.Structure):
    _fields_ = [("n_reduced", ctypes.c_int), ("n_deflated", ctypes.c_int),
                ("n_nearzero", ctypes.c_int), ("n_otherpole", ctypes.c_int),
                ("n_dpr1shift", ctypes.c_int), ("n_capped", ctypes.c_int),
                ("n_fp32_fallback", ctypes.c_int), ("max_iter_used", ctypes.c_int),
                ("total_iter", ctypes.c_longlong), ("fix_iter", ctypes.c_longlong),
                ("max_Kb", ctypes.c_double),
                ("max_Knu", ctypes.c_double), ("ms_reduce", ctypes.c_float),
                ("ms_eig", ctypes.c_float), ("ms_fix", ctypes.c_float),
                ("ms_vectors", ctypes.c_float), ("n_ddb", ctypes.c_int),
                ("total_deriv", ctypes.c_longlong), ("n_mid64", ctypes.c_int),
                ("n_f32_passes", ctypes.c_longlong), ("n_df_passes", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class AeRequest(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n", ctypes.c_int), ("d", ctypes.c_void_p),
                ("z", ctypes.c_void_p), ("alpha", ctypes.c_double), ("want_vectors", ctypes.c_int)]


class AeServeStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_longlong) for k in ("submitted", "admitted", "completed", "rejected",
                                                  "failed", "queued", "running")] + \
        [("bytes_in_use", ctypes.c_size_t), ("eigenpairs", ctypes.c_longlong),
         ("p50_s", ctypes.c_double), ("p99_s", ctypes.c_double), ("max_s", ctypes.c_double),
         ("eigenpairs_per_s", ctypes.c_double), ("cuda_error", ctypes.c_int),
         ("merged", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class AeDiag(ctypes.Structure):
    _fields_ = [("b", ctypes.c_void_p), ("Kb", ctypes.c_void_p), ("Knu", ctypes.c_void_p),
                ("iters", ctypes.c_void_p), ("flags", ctypes.c_void_p)]


_lock = threading.Lock()
_lib = None


def lib():
    """Load libarrowhead.so (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                "(the solver has no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.ae_default_opts.argtypes = [ctypes.POINTER(AeOpts)]
        L.ae_default_opts.restype = None
        L.ae_status_string.argtypes = [I]
        L.ae_status_string.restype = ctypes.c_char_p
        L.ae_last_cuda_error.argtypes = []
        L.ae_last_cuda_error.restype = ctypes.c_char_p
        L.arrow_eig.argtypes = [I, P, P, D, P, P, I, P, P, ctypes.POINTER(AeOpts),
                                ctypes.POINTER(AeInfo), ctypes.POINTER(AeDiag), P]
        L.arrow_eig.restype = I
        L.arrow_eig_host.argtypes = [I, P, P, D, P, P, P, P, ctypes.POINTER(AeOpts),
                                     ctypes.POINTER(AeInfo), P]
        IP = ctypes.POINTER(I)
        L.arrow_eig_part.argtypes = [I, P, P, D, I, I, P, P, I, I, IP, IP,
                                     ctypes.POINTER(AeOpts), ctypes.POINTER(AeInfo), P]
        L.arrow_eig_part.restype = I
        L.arrow_eig_part_size.argtypes = [I, P, P, I, I, IP, IP, P]
        L.arrow_eig_part_size.restype = I
        L.arrow_eig_host.restype = I
        L.dpr1_eig.argtypes = [I, P, P, D, P, P, I, ctypes.POINTER(AeOpts),
                               ctypes.POINTER(AeInfo), ctypes.POINTER(AeDiag), P]
        L.dpr1_eig.restype = I
        L.tri_arrow_svd.argtypes = [I, P, P, D, P, P, I, P, I, ctypes.POINTER(AeOpts),
                                    ctypes.POINTER(AeInfo), ctypes.POINTER(AeDiag), P]
        L.tri_arrow_svd.restype = I
        L.herm_arrow_eig.argtypes = [I, P, P, D, P, P, I, P, P, ctypes.POINTER(AeOpts),
                                     ctypes.POINTER(AeInfo), ctypes.POINTER(AeDiag), P]
        L.herm_arrow_eig.restype = I
        L.nsym_arrow_eig.argtypes = [I, P, P, P, D, P, P, I, P, I, P, P,
                                     ctypes.POINTER(AeOpts), ctypes.POINTER(AeInfo),
                                     ctypes.POINTER(AeDiag), P]
        L.nsym_arrow_eig.restype = I
        LLP = ctypes.POINTER(ctypes.c_longlong)
        L.arrow_eig_batched.argtypes = [I, LLP, LLP, P, P, P, P, P, P, ctypes.POINTER(AeOpts),
                                        ctypes.POINTER(AeInfo), P]
        L.arrow_eig_batched.restype = I
        L.ae_batch_create.argtypes = [ctypes.POINTER(P), I, LLP, LLP, P, P, P, P, P, P,
                                      ctypes.POINTER(AeOpts), P]
        L.ae_batch_create.restype = I
        L.ae_batch_run.argtypes = [P, P]
        L.ae_batch_run.restype = I
        L.ae_batch_info.argtypes = [P, ctypes.POINTER(AeInfo), P]
        L.ae_batch_info.restype = I
        L.ae_batch_destroy.argtypes = [P]
        L.ae_batch_destroy.restype = None
        L.ae_autotune.argtypes = [I, P]
        L.ae_autotune.restype = I
        L.ae_team_width.argtypes = [I]
        L.ae_team_width.restype = I
        L.ae_serve_create.argtypes = [ctypes.POINTER(P), ctypes.c_size_t, I, I,
                                      ctypes.POINTER(AeOpts)]
        L.ae_serve_create.restype = I
        L.ae_serve_submit.argtypes = [P, ctypes.POINTER(AeRequest),
                                      ctypes.POINTER(ctypes.c_ulonglong)]
        L.ae_serve_submit.restype = I
        L.ae_serve_poll.argtypes = [P, ctypes.c_ulonglong, ctypes.POINTER(I),
                                    ctypes.POINTER(D)]
        L.ae_serve_poll.restype = I
        L.ae_serve_result.argtypes = [P, ctypes.c_ulonglong, ctypes.POINTER(P),
                                      ctypes.POINTER(P), ctypes.POINTER(P)]
        L.ae_serve_result.restype = I
        L.ae_serve_release.argtypes = [P, ctypes.c_ulonglong]
        L.ae_serve_release.restype = I
        L.ae_serve_stats.argtypes = [P, ctypes.POINTER(AeServeStats)]
        L.ae_serve_stats.restype = I
        L.ae_serve_destroy.argtypes = [P]
        L.ae_serve_destroy.restype = I
        L.arrow_eig_noalloc.argtypes = L.arrow_eig.argtypes
        L.arrow_eig_noalloc.restype = I
        L.ae_fma_peaks.argtypes = [ctypes.POINTER(D), ctypes.POINTER(D), P]
        L.ae_fma_peaks.restype = I
        L.ae_debug_rcp.argtypes = [I, P, P, P]
        L.ae_debug_rcp.restype = I
        L.ae_debug_newton.argtypes = [I, P, P, D, D, I, D, D, D, D, D, D, D, I, P, P]
        L.ae_debug_newton.restype = I
        _lib = L
        return L


class AeError(RuntimeError):
    def __init__(self, fn, status):
        L = lib()
        msg = L.ae_status_string(status).decode()
        if status == AE_ERR_CUDA:
            msg += ": " + L.ae_last_cuda_error().decode()
        super().__init__(f"{fn} returned {status} ({msg})")
        self.status = status


def default_opts(**kw) -> AeOpts:
    o = AeOpts()
    lib().ae_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _check(fn, status):
    if status != AE_OK:
        raise AeError(fn, status)


def arrow_eig(d, z, alpha, *, vectors=True, want_shift=False, opts=None, info=False,
              diag=False, stream=None, out=None):
    """Eigen-decomposition of [diag(d) z; z^T alpha] on the GPU.

    ``d``, ``z``: float64 CUDA tensors of length n-1.  Returns a dict with
    ``lam`` (n, descending), ``V`` (n x n column-major: column k is
    ``V[:, k]`` of the returned (n, n) tensor) when ``vectors``, ``shift`` and
    ``mu`` when ``want_shift``, ``info`` (dict, synchronises) and per-eigenpair
    ``diag`` tensors when requested.  ``out`` may supply preallocated
    ``lam``/``V`` tensors.
    """
    import torch
    dev = d.device
    n = int(d.numel()) + 1
    out = dict(out or {})
    lam = out.get("lam")
    if lam is None:
        lam = torch.empty(n, dtype=torch.float64, device=dev)
    V = out.get("V") if vectors else None
    if vectors and V is None:
        # storage is column-major n x n: allocate (n, n) row-major and view transposed
        V = torch.empty((n, n), dtype=torch.float64, device=dev)
    shift = torch.empty(n, dtype=torch.float64, device=dev) if want_shift else None
    mu = torch.empty(n, dtype=torch.float64, device=dev) if want_shift else None
    o = opts if opts is not None else default_opts()
    inf = AeInfo() if info else None
    dg = None
    dgt = {}
    if diag:
        dgt = {"b": torch.empty(n, dtype=torch.float64, device=dev),
               "Kb": torch.empty(n, dtype=torch.float64, device=dev),
               "Knu": torch.empty(n, dtype=torch.float64, device=dev),
               "iters": torch.empty(n, dtype=torch.int32, device=dev),
               "flags": torch.empty(n, dtype=torch.int32, device=dev)}
        dg = AeDiag(*(t.data_ptr() for t in dgt.values()))
    st = lib().arrow_eig(n, _ptr(d), _ptr(z), float(alpha), _ptr(lam), _ptr(V), n,
                         _ptr(shift), _ptr(mu), ctypes.byref(o),
                         ctypes.byref(inf) if inf is not None else None,
                         ctypes.byref(dg) if dg is not None else None,
                         _stream_handle(stream))
    _check("arrow_eig", st)
    res = {"lam": lam}
    if vectors:
        res["V"] = V.t()          # column k of the column-major matrix
    if want_shift:
        res["shift"], res["mu"] = shift, mu
    if info:
        res["info"] = inf.as_dict()
    if diag:
        res["diag"] = dgt
    return res


def arrow_eig_part_size(d, z, part, nparts, stream=None):
    """(first output position, item count) of part `part` of `nparts` of the
    arrowhead (d, z) (float64 CUDA tensors of length n-1)."""
    n = int(d.numel()) + 1
    p0, cnt = ctypes.c_int(), ctypes.c_int()
    _check("arrow_eig_part_size", lib().arrow_eig_part_size(
        n, _ptr(d), _ptr(z), int(part), int(nparts), ctypes.byref(p0), ctypes.byref(cnt),
        _stream_handle(stream)))
    return p0.value, cnt.value


def arrow_eig_part(d, z, alpha, part, nparts, *, vectors=True, opts=None, info=False,
                   stream=None, cap=None, out=None):
    """Part `part` of `nparts` of arrow_eig on the GPU (include/arrowhead.h).

    Returns ``lam`` (the part's eigenvalues, descending), ``V`` (n x count,
    columns ``V[:, j]``) when ``vectors``, ``pos0`` (the output position of
    its first item in the whole decomposition) and ``info`` when requested.
    ``cap`` defaults to the part's exact size (one extra size query); ``out``
    may supply ``lam`` (cap) and ``V`` (cap x n, row j = column j) tensors."""
    import torch
    dev = d.device
    n = int(d.numel()) + 1
    out = dict(out or {})
    if cap is None:
        cap = (int(out["lam"].numel()) if "lam" in out
               else arrow_eig_part_size(d, z, part, nparts, stream=stream)[1])
    lam = out.get("lam")
    if lam is None:
        lam = torch.empty(max(cap, 1), dtype=torch.float64, device=dev)
    V = out.get("V") if vectors else None
    if vectors and V is None:
        V = torch.empty((max(cap, 1), n), dtype=torch.float64, device=dev)
    o = opts if opts is not None else default_opts()
    inf = AeInfo() if info else None
    p0, cnt = ctypes.c_int(), ctypes.c_int()
    st = lib().arrow_eig_part(n, _ptr(d), _ptr(z), float(alpha), int(part), int(nparts),
                              _ptr(lam), _ptr(V), n, int(cap), ctypes.byref(p0),
                              ctypes.byref(cnt), ctypes.byref(o),
                              ctypes.byref(inf) if inf is not None else None,
                              _stream_handle(stream))
    _check("arrow_eig_part", st)
    c = cnt.value
    res = {"lam": lam[:c], "pos0": p0.value, "count": c}
    if vectors:
        res["V"] = V[:c].t()
    if info:
        res["info"] = inf.as_dict()
    return res


def _diag_arrays(n, dev):
    import torch
    return {"b": torch.empty(n, dtype=torch.float64, device=dev),
            "Kb": torch.empty(n, dtype=torch.float64, device=dev),
            "Knu": torch.empty(n, dtype=torch.float64, device=dev),
            "iters": torch.empty(n, dtype=torch.int32, device=dev),
            "flags": torch.empty(n, dtype=torch.int32, device=dev)}


def dpr1_eig(d, u, rho, *, vectors=True, opts=None, info=False, diag=False, stream=None,
             out=None):
    """Eigen-decomposition of diag(d) + rho u u^T (float64 CUDA tensors, length n).

    Returns ``lam`` (descending), ``Q`` (columns ``Q[:, k]``) when ``vectors``,
    ``info`` and ``diag`` when requested."""
    import torch
    dev = d.device
    n = int(d.numel())
    out = dict(out or {})
    lam = out.get("lam")
    if lam is None:
        lam = torch.empty(n, dtype=torch.float64, device=dev)
    Q = out.get("Q") if vectors else None
    if vectors and Q is None:
        Q = torch.empty((n, n), dtype=torch.float64, device=dev)
    o = opts if opts is not None else default_opts()
    inf = AeInfo() if info else None
    dgt = _diag_arrays(n, dev) if diag else {}
    dg = AeDiag(*(t.data_ptr() for t in dgt.values())) if diag else None
    st = lib().dpr1_eig(n, _ptr(d), _ptr(u), float(rho), _ptr(lam), _ptr(Q), n,
                        ctypes.byref(o), ctypes.byref(inf) if inf is not None else None,
                        ctypes.byref(dg) if dg is not None else None, _stream_handle(stream))
    _check("dpr1_eig", st)
    res = {"lam": lam}
    if vectors:
        res["Q"] = Q.t()
    if info:
        res["info"] = inf.as_dict()
    if diag:
        res["diag"] = dgt
    return res


def tri_arrow_svd(d, z, alpha, *, vectors=True, opts=None, info=False, diag=False,
                  stream=None, out=None):
    """SVD of [diag(d) z; 0 alpha] (d > 0, length n-1 float64 CUDA tensors).

    Returns ``s`` (descending), ``U`` and ``V`` (columns) when ``vectors``."""
    import torch
    dev = d.device
    n = int(d.numel()) + 1
    out = dict(out or {})
    s = out.get("s")
    if s is None:
        s = torch.empty(n, dtype=torch.float64, device=dev)
    U = out.get("U") if vectors else None
    V = out.get("V") if vectors else None
    if vectors and U is None:
        U = torch.empty((n, n), dtype=torch.float64, device=dev)
    if vectors and V is None:
        V = torch.empty((n, n), dtype=torch.float64, device=dev)
    o = opts if opts is not None else default_opts()
    inf = AeInfo() if info else None
    dgt = _diag_arrays(n, dev) if diag else {}
    dg = AeDiag(*(t.data_ptr() for t in dgt.values())) if diag else None
    st = lib().tri_arrow_svd(n, _ptr(d), _ptr(z), float(alpha), _ptr(s), _ptr(U), n, _ptr(V),
                             n, ctypes.byref(o), ctypes.byref(inf) if inf is not None else None,
                             ctypes.byref(dg) if dg is not None else None,
                             _stream_handle(stream))
    _check("tri_arrow_svd", st)
    res = {"s": s}
    if vectors:
        res["U"] = U.t()
        res["V"] = V.t()
    if info:
        res["info"] = inf.as_dict()
    if diag:
        res["diag"] = dgt
    return res


def herm_arrow_eig(d, z, alpha, *, vectors=True, want_shift=False, opts=None, info=False,
                   diag=False, stream=None, out=None):
    """Eigen-decomposition of the Hermitian arrowhead [diag(d) z; z^* alpha] (Sec. 6.1).

    ``d``: float64 CUDA tensor of length n-1, ``z``: complex128 CUDA tensor of
    length n-1 (the column above the real corner).  Returns ``lam`` (descending)
    and ``U`` (complex, columns ``U[:, k]``) when ``vectors``; ``shift``/``mu``,
    ``info`` and ``diag`` as arrow_eig."""
    import torch
    dev = d.device
    n = int(d.numel()) + 1
    if z.dtype != torch.complex128:
        raise TypeError("herm_arrow_eig: z must be complex128")
    z = z.contiguous()
    out = dict(out or {})
    lam = out.get("lam")
    if lam is None:
        lam = torch.empty(n, dtype=torch.float64, device=dev)
    U = out.get("U") if vectors else None
    if vectors and U is None:
        U = torch.empty((n, n), dtype=torch.complex128, device=dev)
    shift = torch.empty(n, dtype=torch.float64, device=dev) if want_shift else None
    mu = torch.empty(n, dtype=torch.float64, device=dev) if want_shift else None
    o = opts if opts is not None else default_opts()
    inf = AeInfo() if info else None
    dgt = _diag_arrays(n, dev) if diag else {}
    dg = AeDiag(*(t.data_ptr() for t in dgt.values())) if diag else None
    st = lib().herm_arrow_eig(n, _ptr(d), _ptr(z), float(alpha), _ptr(lam), _ptr(U), n,
                              _ptr(shift), _ptr(mu), ctypes.byref(o),
                              ctypes.byref(inf) if inf is not None else None,
                              ctypes.byref(dg) if dg is not None else None,
                              _stream_handle(stream))
    _check("herm_arrow_eig", st)
    res = {"lam": lam}
    if vectors:
        res["U"] = U.t()
    if want_shift:
        res["shift"], res["mu"] = shift, mu
    if info:
        res["info"] = inf.as_dict()
    if diag:
        res["diag"] = dgt
    return res


def nsym_arrow_eig(d, zc, zr, alpha, *, vectors=True, left=True, want_shift=False, opts=None,
                   info=False, diag=False, stream=None, out=None):
    """Eigen-decomposition of the non-symmetric arrowhead [diag(d) zc; zr^T alpha]
    (Remark of Sec. 6.1; zc_r zr_r > 0 or both zero).

    Returns ``lam`` (descending), right vectors ``X`` and (``left``) left
    vectors ``Y`` (columns, Y^T X = I) when ``vectors``; the rest as arrow_eig."""
    import torch
    dev = d.device
    n = int(d.numel()) + 1
    out = dict(out or {})
    lam = out.get("lam")
    if lam is None:
        lam = torch.empty(n, dtype=torch.float64, device=dev)
    X = out.get("X") if vectors else None
    Y = out.get("Y") if (vectors and left) else None
    if vectors and X is None:
        X = torch.empty((n, n), dtype=torch.float64, device=dev)
    if vectors and left and Y is None:
        Y = torch.empty((n, n), dtype=torch.float64, device=dev)
    shift = torch.empty(n, dtype=torch.float64, device=dev) if want_shift else None
    mu = torch.empty(n, dtype=torch.float64, device=dev) if want_shift else None
    o = opts if opts is not None else default_opts()
    inf = AeInfo() if info else None
    dgt = _diag_arrays(n, dev) if diag else {}
    dg = AeDiag(*(t.data_ptr() for t in dgt.values())) if diag else None
    st = lib().nsym_arrow_eig(n, _ptr(d), _ptr(zc), _ptr(zr), float(alpha), _ptr(lam),
                              _ptr(X), n, _ptr(Y), n, _ptr(shift), _ptr(mu), ctypes.byref(o),
                              ctypes.byref(inf) if inf is not None else None,
                              ctypes.byref(dg) if dg is not None else None,
                              _stream_handle(stream))
    _check("nsym_arrow_eig", st)
    res = {"lam": lam}
    if vectors:
        res["X"] = X.t()
        if left:
            res["Y"] = Y.t()
    if want_shift:
        res["shift"], res["mu"] = shift, mu
    if info:
        res["info"] = inf.as_dict()
    if diag:
        res["diag"] = dgt
    return res


class Batch:
    """Packed device buffers for a batch of arrowheads and the C plan over them.

    ``instances`` is a list of (d, z, alpha) (numpy, length n_i - 1).  The
    inputs are uploaded once; ``run()`` replays the captured solve; results are
    views into ``lam_all`` / ``V_all``.  ``graph=False`` uses the one-shot
    arrow_eig_batched instead of a plan.
    """

    def __init__(self, instances, *, vectors=True, opts=None, graph=True, stream=None,
                 device="cuda"):
        import torch
        self.count = len(instances)
        ns = np.array([len(d) + 1 for d, _, _ in instances], dtype=np.int64)
        self.n = ns
        self.n_off = np.zeros(self.count + 1, dtype=np.int64)
        np.cumsum(ns, out=self.n_off[1:])
        self.v_off = np.zeros(self.count + 1, dtype=np.int64)
        np.cumsum(ns * ns, out=self.v_off[1:])
        cat = lambda k: np.concatenate([np.asarray(x[k], dtype=np.float64) for x in instances]) \
            if self.n_off[-1] > self.count else np.zeros(1)
        self.d_all = torch.as_tensor(cat(0), device=device)
        self.z_all = torch.as_tensor(cat(1), device=device)
        self.alpha_all = torch.as_tensor(np.array([x[2] for x in instances], dtype=np.float64),
                                         device=device)
        self.lam_all = torch.empty(int(self.n_off[-1]), dtype=torch.float64, device=device)
        self.V_all = torch.empty(int(self.v_off[-1]), dtype=torch.float64, device=device) \
            if vectors else None
        self.status = torch.empty(self.count, dtype=torch.int32, device=device)
        self.opts = opts if opts is not None else default_opts()
        self.stream = stream
        self.plan = None
        if graph:
            h = ctypes.c_void_p()
            st = lib().ae_batch_create(ctypes.byref(h), self.count, self._ll(self.n_off),
                                       self._ll(self.v_off), _ptr(self.d_all), _ptr(self.z_all),
                                       _ptr(self.alpha_all), _ptr(self.lam_all), _ptr(self.V_all),
                                       _ptr(self.status), ctypes.byref(self.opts),
                                       _stream_handle(stream))
            _check("ae_batch_create", st)
            self.plan = h

    @staticmethod
    def _ll(a):
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong))

    def run(self, info=False):
        inf = AeInfo() if info else None
        if self.plan is not None:
            _check("ae_batch_run", lib().ae_batch_run(self.plan, _stream_handle(self.stream)))
            if info:
                _check("ae_batch_info", lib().ae_batch_info(self.plan, ctypes.byref(inf),
                                                            _stream_handle(self.stream)))
        else:
            st = lib().arrow_eig_batched(self.count, self._ll(self.n_off), self._ll(self.v_off),
                                         _ptr(self.d_all), _ptr(self.z_all),
                                         _ptr(self.alpha_all), _ptr(self.lam_all),
                                         _ptr(self.V_all), _ptr(self.status),
                                         ctypes.byref(self.opts),
                                         ctypes.byref(inf) if inf is not None else None,
                                         _stream_handle(self.stream))
            _check("arrow_eig_batched", st)
        return inf.as_dict() if info else None

    def lam(self, i):
        return self.lam_all[self.n_off[i]:self.n_off[i + 1]]

    def V(self, i):
        n = int(self.n[i])
        return self.V_all[self.v_off[i]:self.v_off[i + 1]].view(n, n).t()

    def close(self):
        if self.plan is not None:
            lib().ae_batch_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _DeviceView:
    """Zero-copy view of a device buffer for torch.as_tensor (CUDA array interface)."""

    def __init__(self, ptr, shape):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<f8",
                                         "data": (int(ptr), False), "version": 3, "strides": None}


class Server:
    """Continuous-batching request loop over the solvers (ae_serve_*).

    ``submit(kind, d, z, alpha)`` takes float64 CUDA tensors (kept referenced
    until ``release``) and returns a ticket; ``poll`` gives (state, latency s);
    ``result`` copies a finished request's outputs into new tensors."""

    def __init__(self, budget_bytes, max_inflight=8, queue_cap=4096, opts=None):
        self.h = ctypes.c_void_p()
        o = opts if opts is not None else default_opts()
        _check("ae_serve_create", lib().ae_serve_create(ctypes.byref(self.h), int(budget_bytes),
                                                        int(max_inflight), int(queue_cap),
                                                        ctypes.byref(o)))
        self.refs = {}
        self.meta = {}

    def submit(self, kind, d, z, alpha, vectors=True):
        n = int(d.numel()) + (0 if kind == KIND_DPR1 else 1)
        req = AeRequest(kind, n, d.data_ptr() if d.numel() else None,
                        z.data_ptr() if z.numel() else None, float(alpha), 1 if vectors else 0)
        t = ctypes.c_ulonglong()
        st = lib().ae_serve_submit(self.h, ctypes.byref(req), ctypes.byref(t))
        if st == AE_EAGAIN:
            return None
        _check("ae_serve_submit", st)
        self.refs[t.value] = (d, z)
        self.meta[t.value] = (kind, n, vectors)
        return t.value

    def poll(self, ticket):
        state = ctypes.c_int()
        lat = ctypes.c_double()
        lib().ae_serve_poll(self.h, ctypes.c_ulonglong(ticket), ctypes.byref(state),
                            ctypes.byref(lat))
        return state.value, lat.value

    def wait(self, ticket, timeout=120.0):
        import time
        t0 = time.time()
        while True:
            st, lat = self.poll(ticket)
            if st in (REQ_DONE, REQ_ERROR):
                return st, lat
            if time.time() - t0 > timeout:
                raise TimeoutError(f"request {ticket} not finished")
            time.sleep(0.0005)

    def result(self, ticket):
        import torch
        kind, n, vectors = self.meta[ticket]
        pl, pv, pu = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        _check("ae_serve_result", lib().ae_serve_result(self.h, ctypes.c_ulonglong(ticket),
                                                        ctypes.byref(pl), ctypes.byref(pv),
                                                        ctypes.byref(pu)))
        out = {"lam": torch.as_tensor(_DeviceView(pl.value, (n,)), device="cuda").clone()}
        if vectors:
            out["V"] = torch.as_tensor(_DeviceView(pv.value, (n, n)), device="cuda").t().clone()
            if kind == KIND_SVD:
                out["U"] = torch.as_tensor(_DeviceView(pu.value, (n, n)),
                                           device="cuda").t().clone()
        return out

    def release(self, ticket):
        st = lib().ae_serve_release(self.h, ctypes.c_ulonglong(ticket))
        if st == AE_OK:
            self.refs.pop(ticket, None)
            self.meta.pop(ticket, None)
        return st

    def stats(self):
        s = AeServeStats()
        _check("ae_serve_stats", lib().ae_serve_stats(self.h, ctypes.byref(s)))
        return s.as_dict()

    def close(self):
        if self.h:
            lib().ae_serve_destroy(self.h)
            self.h = None
            self.refs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(n_max=4096, stream=None):
    """Run the team-width tuner and store its choices in the JSON cache."""
    _check("ae_autotune", lib().ae_autotune(int(n_max), _stream_handle(stream)))
    return {b: lib().ae_team_width(b) for b in (32, 64, 128, 256, 512)}


def arrow_eig_host(d, z, alpha, *, vectors=True, want_shift=False, opts=None, stream=None,
                   out=None):
    """arrow_eig on host arrays (numpy or pinned torch CPU tensors).

    The library copies the inputs to the device, solves and copies the results
    back on ``stream`` and synchronises.  ``out`` may supply pinned host
    ``lam``/``V`` buffers (torch CPU tensors)."""
    import torch
    d = torch.as_tensor(d, dtype=torch.float64)
    z = torch.as_tensor(z, dtype=torch.float64)
    n = int(d.numel()) + 1
    out = dict(out or {})
    lam = out.get("lam")
    if lam is None:
        lam = torch.empty(n, dtype=torch.float64)
    V = out.get("V") if vectors else None
    if vectors and V is None:
        V = torch.empty((n, n), dtype=torch.float64)
    shift = torch.empty(n, dtype=torch.float64) if want_shift else None
    mu = torch.empty(n, dtype=torch.float64) if want_shift else None
    o = opts if opts is not None else default_opts()
    st = lib().arrow_eig_host(n, _ptr(d.contiguous()), _ptr(z.contiguous()), float(alpha),
                              _ptr(lam), _ptr(V), _ptr(shift), _ptr(mu), ctypes.byref(o), None,
                              _stream_handle(stream))
    _check("arrow_eig_host", st)
    res = {"lam": lam}
    if vectors:
        res["V"] = V.t()
    if want_shift:
        res["shift"], res["mu"] = shift, mu
    return res


def fma_peaks(stream=None):
    """Measured FMA throughput (TFLOP/s) of the FP64 and FP32 pipes."""
    f64, f32 = ctypes.c_double(), ctypes.c_double()
    _check("ae_fma_peaks", lib().ae_fma_peaks(ctypes.byref(f64), ctypes.byref(f32),
                                              _stream_handle(stream)))
    return {"fp64_tflops": f64.value, "fp32_tflops": f32.value}


def debug_rcp(x, stream=None):
    """The solver's FP64 reciprocal applied elementwise (device tensor)."""
    import torch
    y = torch.empty_like(x)
    _check("ae_debug_rcp", lib().ae_debug_rcp(int(x.numel()), _ptr(x), _ptr(y),
                                              _stream_handle(stream)))
    return y


def debug_newton(delta, cj, b, c, side, pole, left, right, x0=float("nan"),
                 dF0=float("nan"), xdF0=float("nan"), rel0=float("inf"), max_iter=300,
                 stream=None):
    """The solver's FP64 finish on one shifted inverse's Pick function
    (include/arrowhead.h, ae_debug_newton).  delta, cj: float64 CUDA tensors.
    Returns (nu, FP64 evaluations, evaluations with F')."""
    import torch
    out = torch.empty(3, dtype=torch.float64, device=delta.device)
    _check("ae_debug_newton", lib().ae_debug_newton(
        int(delta.numel()), _ptr(delta), _ptr(cj), float(b), float(c), int(side), float(pole),
        float(left), float(right), float(x0), float(dF0), float(xdF0), float(rel0),
        int(max_iter), _ptr(out), _stream_handle(stream)))
    nu, it, itd = out.cpu().tolist()
    return nu, int(it), int(itd)


def exported_symbols(path=LIB_PATH):
    """Names of the C-ABI symbols present in the library (no GPU needed)."""
    L = ctypes.CDLL(path)
    return [s for s in EXPORTED if hasattr(L, s)]


__all__ = ["arrow_eig", "arrow_eig_part", "arrow_eig_part_size", "herm_arrow_eig", "nsym_arrow_eig", "dpr1_eig", "tri_arrow_svd",
           "Batch", "Server", "autotune", "arrow_eig_host",
           "fma_peaks", "debug_rcp", "default_opts", "lib", "AeOpts",
           "AeInfo", "AeDiag", "AeError", "exported_symbols", "EXPORTED"]

_ = np  # numpy is used by callers passing host arrays
