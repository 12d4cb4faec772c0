"""arrow_eig_noalloc, the entry point for callers that cannot allocate.

Some callers may not allocate device memory while they run (an application
that reserved all GPU memory up front and passes the library only its input
and output buffers, or a latency-critical loop where an allocation could block
or fail).  arrow_eig_noalloc serves them from a static device array instead of
cudaMallocAsync.  These tests call it through the C ABI and check it against
arrow_eig at the suite's tolerance (10 n eps64, relative, per eigenvalue and
eigenvector component), on two calls in a row that reuse the shared array
with different sizes, so stale contents from the first call would show; at
the largest order the array admits (n = 20928) a sample of eigenvalues is
checked against the oracle.
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

EPS64 = 2.0 ** -53


@pytest.fixture(scope="module")
def ae():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1302_7203_gb300 import arrowhead, build
    build.build()
    return arrowhead


def _noalloc(ae, d, z, alpha):
    n = len(d) + 1
    dt = torch.as_tensor(d, device="cuda")
    zt = torch.as_tensor(z, device="cuda")
    lam = torch.empty(n, dtype=torch.float64, device="cuda")
    V = torch.empty((n, n), dtype=torch.float64, device="cuda")
    info = ae.AeInfo()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = ae.lib().arrow_eig_noalloc(n, ctypes.c_void_p(dt.data_ptr()),
                                    ctypes.c_void_p(zt.data_ptr()), float(alpha),
                                    ctypes.c_void_p(lam.data_ptr()),
                                    ctypes.c_void_p(V.data_ptr()), n, None, None, None,
                                    ctypes.byref(info), None, stream)
    assert st == ae.AE_OK, ae.lib().ae_status_string(st)
    torch.cuda.synchronize()
    return lam.cpu().numpy(), V.t().cpu().numpy(), info


def _reference(ae, d, z, alpha):
    r = ae.arrow_eig(torch.as_tensor(d, device="cuda"), torch.as_tensor(z, device="cuda"),
                     alpha)
    torch.cuda.synchronize()
    return r["lam"].cpu().numpy(), r["V"].cpu().numpy()


def test_noalloc_matches_arrow_eig_on_two_calls(ae):
    from paper_1302_7203_gb300 import workloads as W
    cases = [W.graded_arrow(3000, seed=41), W.uniform_arrow(1200, seed=42)]
    for d, z, alpha in cases:                       # two calls in a row
        n = len(d) + 1
        tol = 10 * n * EPS64
        lam, V, info = _noalloc(ae, d, z, alpha)
        lam_ref, V_ref = _reference(ae, d, z, alpha)
        assert info.n_reduced == n
        assert np.all(np.abs(lam - lam_ref) <= tol * np.abs(lam_ref))
        tiny = np.finfo(np.float64).tiny
        assert np.all(np.abs(V - V_ref) <= tol * np.maximum(np.abs(V_ref), tiny))


def test_noalloc_rejects_sizes_beyond_its_scratch(ae):
    n = 20929                                       # first order that does not fit
    st = ae.lib().arrow_eig_noalloc(n, ctypes.c_void_p(1), ctypes.c_void_p(1), 0.0,
                                    ctypes.c_void_p(1), None, n, None, None, None, None, None,
                                    None)
    assert st == ae.AE_ERR_TOO_LARGE
    assert b"static scratch" in ae.lib().ae_status_string(st)


def _cudart():
    """The CUDA runtime (any copy: the memory pool queried is the device's)."""
    import glob
    import os
    cands = ["libcudart.so.13", "libcudart.so"]
    cands += glob.glob("/usr/local/cuda/lib64/libcudart.so*")
    try:
        import nvidia
        for base in nvidia.__path__:
            cands += glob.glob(os.path.join(base, "*", "lib", "libcudart.so*"))
    except ImportError:
        pass
    for c in cands:
        try:
            return ctypes.CDLL(c)
        except OSError:
            continue
    pytest.skip("no CUDA runtime library to query the memory pool with")


def _pool_bytes(rt):
    """(used, reserved) bytes of the current device's default memory pool,
    which every cudaMallocAsync of this library draws from."""
    dev = ctypes.c_int()
    assert rt.cudaGetDevice(ctypes.byref(dev)) == 0
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0
    used, res = ctypes.c_uint64(), ctypes.c_uint64()
    assert rt.cudaMemPoolGetAttribute(pool, 0x7, ctypes.byref(used)) == 0   # UsedMemCurrent
    assert rt.cudaMemPoolGetAttribute(pool, 0x5, ctypes.byref(res)) == 0    # ReservedMemCurrent
    return used.value, res.value


def test_noalloc_allocates_nothing(ae):
    # what the entry point exists for: after a first call on the device (which
    # loads the library's kernels and looks up the array), a call changes
    # neither the device's free memory nor its stream-ordered memory pool
    from paper_1302_7203_gb300 import workloads as W
    rt = _cudart()
    d, z, alpha = W.graded_arrow(2000, seed=43)
    _noalloc(ae, d, z, alpha)                       # warm-up call
    n = len(d) + 1
    dt = torch.as_tensor(d, device="cuda")
    zt = torch.as_tensor(z, device="cuda")
    lam = torch.empty(n, dtype=torch.float64, device="cuda")
    V = torch.empty((n, n), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    pool0 = _pool_bytes(rt)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = ae.lib().arrow_eig_noalloc(n, ctypes.c_void_p(dt.data_ptr()),
                                    ctypes.c_void_p(zt.data_ptr()), float(alpha),
                                    ctypes.c_void_p(lam.data_ptr()), ctypes.c_void_p(V.data_ptr()),
                                    n, None, None, None, None, None, stream)
    assert st == ae.AE_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert _pool_bytes(rt) == pool0


def test_noalloc_accepts_its_largest_order(ae):
    # n = 20928 is the largest order whose scratch fits the static array
    from paper_1302_7203_gb300 import workloads as W
    n = 20928
    d, z, alpha = W.uniform_arrow(n, seed=44)
    dt = torch.as_tensor(d, device="cuda")
    zt = torch.as_tensor(z, device="cuda")
    lam = torch.empty(n, dtype=torch.float64, device="cuda")
    info = ae.AeInfo()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = ae.lib().arrow_eig_noalloc(n, ctypes.c_void_p(dt.data_ptr()),
                                    ctypes.c_void_p(zt.data_ptr()), float(alpha),
                                    ctypes.c_void_p(lam.data_ptr()), None, n, None, None, None,
                                    ctypes.byref(info), None, stream)
    assert st == ae.AE_OK, ae.lib().ae_status_string(st)
    torch.cuda.synchronize()
    lam = lam.cpu().numpy()
    assert info.n_reduced == n and np.all(np.diff(lam) <= 0)
    assert np.all(lam[:-1] >= d) and np.all(d >= lam[1:])   # interlacing (Sec. 1)
    # and the values themselves: sampled against the oracle at 10 n eps64
    import oracle
    ks = np.unique(np.r_[0, 1, n // 3, n // 2, n - 2, n - 1,
                         np.random.default_rng(44).choice(n, 26, replace=False)])
    ref = oracle.arrow_eig(d, z, alpha, ks=ks, vectors=False)
    tol = 10 * n * 2.0 ** -53
    assert np.all(np.abs(lam[ks] - ref["lam"]) <= tol * np.abs(ref["lam"]))
