// ae_noalloc.cu -- arrow_eig_noalloc: the arrowhead solve with its scratch in a
// static device array, for callers that must not allocate device memory.
//
// Who cannot allocate: an application that reserves all device memory up
// front and hands this library only its input and output buffers (a host
// framework with its own memory budget, or a latency-critical service loop),
// where a cudaMalloc/cudaMallocAsync could block on the driver, fail under
// memory pressure or fragment the reserved pool.  For them the O(n) scratch of
// the solve lives in g_noalloc_scratch below: AE_NOALLOC_SCRATCH_BYTES bytes
// that every GPU holds until the process exits once this code has been loaded
// onto it -- with CUDA's lazy module loading, at the first call there, which
// is why callers make one call per device before reserving its memory.
//
// Host code must not pass g_noalloc_scratch itself to a kernel: on the host
// that name denotes a host-side shadow, not a device address.  The device
// address is looked up once per device with cudaGetSymbolAddress (with that
// device current) and cached.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "ae_internal.h"

static __device__ __align__(256) unsigned char g_noalloc_scratch[AE_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mu;

// device address of g_noalloc_scratch on the current device (set-up on first use)
cudaError_t scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int arrow_eig_noalloc(int n, const double *d, const double *z, double alpha,
                                 double *lambda, double *V, int ldv, double *shift, double *mu,
                                 const ae_opts *opts, ae_info *info, const ae_diag *diag,
                                 void *stream) {
    if (n < 1) return -1;
    if (n > 1 && !d) return -2;
    if (n > 1 && !z) return -3;
    if (!isfinite(alpha)) return -4;
    if (!lambda) return -5;
    if (V && ldv < n) return -7;
    if (ae::arrow_scratch_bytes(n) > (size_t)AE_NOALLOC_SCRATCH_BYTES) return AE_ERR_TOO_LARGE;
    ae::RunOpts ro;
    if (ae::resolve_opts(opts, ro)) return -10;      // opts->profile is ignored here
    cudaStream_t st = (cudaStream_t)stream;
    void *base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) {
        ae::record_cuda_error(e);
        return AE_ERR_CUDA;
    }
    // launch_arrow zeroes the counters it relies on; every other scratch array
    // is written before it is read, so the previous call's contents do no harm
    ae::Scratch S = ae::carve_scratch(base, n);
    ae::Outputs out;
    out.lambda = lambda;
    out.V = V;
    out.ldv = ldv;
    out.U = nullptr;
    out.ldu = 0;
    out.shift = shift;
    out.mu = mu;
    out.dg_b = diag ? diag->b : nullptr;
    out.dg_Kb = diag ? diag->Kb : nullptr;
    out.dg_Knu = diag ? diag->Knu : nullptr;
    out.dg_iters = diag ? diag->iters : nullptr;
    out.dg_flags = diag ? diag->flags : nullptr;
    e = ae::launch_arrow(n, d, z, alpha, out, ro, S, st);
    if (e != cudaSuccess) {
        ae::record_cuda_error(e);
        return AE_ERR_CUDA;
    }
    if (!info) return AE_OK;
    int cnt[ae::C_COUNT];
    unsigned long long c64[ae::C64_COUNT];
    e = cudaMemcpyAsync(cnt, S.cnt, sizeof(cnt), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c64, S.cnt64, sizeof(c64), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        ae::record_cuda_error(e);
        return AE_ERR_CUDA;
    }
    memset(info, 0, sizeof(*info));
    info->n_reduced = cnt[ae::C_M] + 1;
    info->n_deflated = cnt[ae::C_ND];
    info->n_nearzero = cnt[ae::C_NEARZERO];
    info->n_otherpole = cnt[ae::C_OTHERPOLE];
    info->n_dpr1shift = cnt[ae::C_DPR1];
    info->n_capped = cnt[ae::C_CAPPED];
    info->n_fp32_fallback = cnt[ae::C_FP32FB];
    info->max_iter_used = cnt[ae::C_MAXIT];
    info->total_iter = (long long)c64[ae::C64_ITERS];
    info->fix_iter = (long long)c64[ae::C64_ITERS_FIX];
    memcpy(&info->max_Kb, &c64[ae::C64_MAXKB], sizeof(double));
    memcpy(&info->max_Knu, &c64[ae::C64_MAXKNU], sizeof(double));
    info->n_ddb = cnt[ae::C_DDB];
    info->n_mid64 = cnt[ae::C_MID64];
    info->total_deriv = (long long)c64[ae::C64_DERIV];
    info->n_f32_passes = (long long)c64[ae::C64_F32];
    info->n_df_passes = (long long)c64[ae::C64_DF];
    if (cnt[ae::C_FLAGS] & ae::CF_BAD) return AE_ERR_INPUT;
    if (cnt[ae::C_CAPPED]) return AE_ERR_NOCONV;
    return AE_OK;
}
