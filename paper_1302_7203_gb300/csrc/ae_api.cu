// ae_api.cu -- the extern "C" entry points declared in include/arrowhead.h.
// Argument checking, option defaults, scratch allocation (stream-ordered) and
// the optional synchronising summary; all arithmetic is in the kernels.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "ae_internal.h"

namespace {

thread_local char g_err[256] = "";

int cuda_fail(cudaError_t e) {
    snprintf(g_err, sizeof(g_err), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    return AE_ERR_CUDA;
}

// keep freed stream-ordered allocations in the device's pool so repeated
// calls do not return memory to the driver at every synchronisation
void keep_pool_warm() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    static int done_mask = 0;
    if (dev < 31 && (done_mask & (1 << dev))) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        unsigned long long thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    if (dev < 31) done_mask |= 1 << dev;
}


// events for opts->profile; destroyed after the synchronising summary
struct Prof {
    bool on = false;
    cudaEvent_t ev[5] = {};
    ~Prof() {
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
    }
    cudaError_t init(ae::RunOpts &ro) {
        on = true;
        for (int i = 0; i < 5; ++i) {
            cudaError_t e = cudaEventCreate(&ev[i]);
            if (e != cudaSuccess) return e;
            ro.ev[i] = ev[i];
        }
        return cudaSuccess;
    }
};

double bits_to_double(unsigned long long u) {
    double v;
    memcpy(&v, &u, sizeof(v));
    return v;
}

}  // namespace

namespace ae {
void record_cuda_error(cudaError_t e) { cuda_fail(e); }

int resolve_opts(const ae_opts *o, RunOpts &ro) {
    ae_opts def;
    ae_default_opts(&def);
    if (!o) o = &def;
    if (o->precision != AE_FP64 && o->precision != AE_FP32_BRACKET) return 1;
    if (o->finish != AE_FINISH_BISECT && o->finish != AE_FINISH_NEWTON) return 1;
    if (o->bgate != 0 && o->bgate != 1) return 1;
    ro.precision = o->precision;
    ro.finish = o->finish;
    ro.bgate = o->bgate;
    ro.kb_max = o->kb_max > 0.0 ? o->kb_max : def.kb_max;
    ro.knu_max = o->knu_max > 0.0 ? o->knu_max : def.knu_max;
    ro.max_iter = o->max_iter > 0 ? o->max_iter : def.max_iter;
    ro.fixup = o->fixup ? 1 : 0;
    for (int i = 0; i < 5; ++i) ro.ev[i] = nullptr;
    return 0;
}
}  // namespace ae

extern "C" {

void ae_default_opts(ae_opts *opts) {
    if (!opts) return;
    opts->precision = AE_FP64;
    opts->knu_max = 10.0;
    opts->max_iter = 2200;
    opts->fixup = 1;
    opts->profile = 0;
    opts->finish = AE_FINISH_BISECT;
    opts->bgate = 0;
    opts->kb_max = 10.0;
}

const char *ae_status_string(int status) {
    if (status == AE_OK) return "ok";
    if (status < 0) return "invalid argument";
    switch (status) {
        case AE_ERR_CUDA: return "CUDA error";
        case AE_ERR_INPUT: return "non-finite input";
        case AE_ERR_NOCONV: return "iteration cap reached";
        case AE_EAGAIN: return "queue full or result not ready (try again)";
        case AE_ERR_TOO_LARGE:
            return "too large: n beyond the static scratch of arrow_eig_noalloc "
                   "(AE_NOALLOC_SCRATCH_BYTES), or a part's items beyond the room "
                   "given to arrow_eig_part";
        default: return "unknown status";
    }
}

const char *ae_last_cuda_error(void) { return g_err; }

// One part of a split arrow_eig (arrow_eig_part): which part, the room the
// caller's outputs have, and where the part's first output position and item
// count go.
struct PartSpec {
    int part, nparts, cap;
    int *pos0, *count;
};

// Shared by arrow_eig, dpr1_eig and tri_arrow_svd: scratch, launch, optional
// synchronising summary.
static int solve_common(ae::Kind kind, int n, const double *d, const double *z, double alpha,
                        double rho, const ae::Outputs &out, const ae_opts *opts, ae_info *info,
                        void *stream, const double *zrow = nullptr,
                        const PartSpec *part = nullptr) {
    ae::RunOpts ro;
    if (ae::resolve_opts(opts, ro)) return -10;
    cudaStream_t st = (cudaStream_t)stream;
    keep_pool_warm();
    Prof prof;
    if (opts && opts->profile && info) {
        cudaError_t pe = prof.init(ro);
        if (pe != cudaSuccess) return cuda_fail(pe);
    }
    void *base = nullptr;
    cudaError_t e = cudaMallocAsync(&base, ae::arrow_scratch_bytes(n), st);
    if (e != cudaSuccess) return cuda_fail(e);
    ae::Scratch S = ae::carve_scratch(base, n);
    // one slice of n stored (delta_j, c_j) pairs per warp of the eigenvalue kernel
    void *wb = nullptr;
    const long long wstride = ((long long)n + 1) & ~1LL;
    e = cudaMallocAsync(&wb, sizeof(double2) * wstride * ae::eig_grid_warps(n), st);
    if (e != cudaSuccess) {
        cudaFreeAsync(base, st);
        return cuda_fail(e);
    }
    S.wbuf = (double2 *)wb;
    S.wstride = wstride;
    int status = AE_OK;
    bool solved = true;
    if (part) {
        e = ae::launch_arrow_part(n, d, z, alpha, part->part, part->nparts, part->cap, out, ro,
                                  S, st, part->pos0, part->count);
        solved = out.lambda && *part->count <= part->cap;
        if (e == cudaSuccess && out.lambda && !solved) status = AE_ERR_TOO_LARGE;
    } else {
        e = ae::launch_solve(kind, n, d, z, alpha, rho, out, ro, S, st, zrow);
    }
    if (e != cudaSuccess) status = cuda_fail(e);
    if (info && status == AE_OK && solved) {
        int cnt[ae::C_COUNT];
        unsigned long long c64[ae::C64_COUNT];
        e = cudaMemcpyAsync(cnt, S.cnt, sizeof(cnt), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c64, S.cnt64, sizeof(c64), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            status = cuda_fail(e);
        } else {
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
            info->max_Kb = bits_to_double(c64[ae::C64_MAXKB]);
            info->max_Knu = bits_to_double(c64[ae::C64_MAXKNU]);
            info->n_ddb = cnt[ae::C_DDB];
            info->n_mid64 = cnt[ae::C_MID64];
            info->total_deriv = (long long)c64[ae::C64_DERIV];
            info->n_f32_passes = (long long)c64[ae::C64_F32];
            info->n_df_passes = (long long)c64[ae::C64_DF];
            if (prof.on) {
                cudaEventElapsedTime(&info->ms_reduce, prof.ev[0], prof.ev[1]);
                cudaEventElapsedTime(&info->ms_eig, prof.ev[1], prof.ev[2]);
                cudaEventElapsedTime(&info->ms_fix, prof.ev[2], prof.ev[3]);
                cudaEventElapsedTime(&info->ms_vectors, prof.ev[3], prof.ev[4]);
            }
            if (cnt[ae::C_FLAGS] & ae::CF_BAD) status = AE_ERR_INPUT;
            else if (cnt[ae::C_CAPPED]) status = AE_ERR_NOCONV;
        }
    }
    e = cudaFreeAsync(wb, st);
    if (e != cudaSuccess && status == AE_OK) status = cuda_fail(e);
    e = cudaFreeAsync(base, st);
    if (e != cudaSuccess && status == AE_OK) status = cuda_fail(e);
    return status;
}

static ae::Outputs make_outputs(double *lambda, double *V, int ldv, double *U, int ldu,
                                double *shift, double *mu, const ae_diag *diag) {
    ae::Outputs out;
    out.lambda = lambda;
    out.V = V;
    out.ldv = ldv;
    out.U = U;
    out.ldu = ldu;
    out.shift = shift;
    out.mu = mu;
    out.dg_b = diag ? diag->b : nullptr;
    out.dg_Kb = diag ? diag->Kb : nullptr;
    out.dg_Knu = diag ? diag->Knu : nullptr;
    out.dg_iters = diag ? diag->iters : nullptr;
    out.dg_flags = diag ? diag->flags : nullptr;
    return out;
}

int arrow_eig(int n, const double *d, const double *z, double alpha, double *lambda,
              double *V, int ldv, double *shift, double *mu, const ae_opts *opts,
              ae_info *info, const ae_diag *diag, void *stream) {
    if (n < 1) return -1;
    if (n > 1 && !d) return -2;
    if (n > 1 && !z) return -3;
    if (!isfinite(alpha)) return -4;
    if (!lambda) return -5;
    if (V && ldv < n) return -7;
    const ae::Outputs out = make_outputs(lambda, V, ldv, nullptr, 0, shift, mu, diag);
    return solve_common(ae::KIND_ARROW, n, d, z, alpha, 0.0, out, opts, info, stream);
}

int arrow_eig_part(int n, const double *d, const double *z, double alpha, int part, int nparts,
                   double *lambda, double *V, int ldv, int cap, int *pos0, int *count,
                   const ae_opts *opts, ae_info *info, void *stream) {
    if (n < 1) return -1;
    if (n > 1 && !d) return -2;
    if (n > 1 && !z) return -3;
    if (!isfinite(alpha)) return -4;
    if (nparts < 1) return -6;
    if (part < 0 || part >= nparts) return -5;
    if (!lambda) return -7;
    if (V && ldv < n) return -9;
    if (cap < 0) return -10;
    if (!pos0) return -11;
    if (!count) return -12;
    const ae::Outputs out = make_outputs(lambda, V, ldv, nullptr, 0, nullptr, nullptr, nullptr);
    const PartSpec ps{part, nparts, cap, pos0, count};
    return solve_common(ae::KIND_ARROW, n, d, z, alpha, 0.0, out, opts, info, stream, nullptr,
                        &ps);
}

int arrow_eig_part_size(int n, const double *d, const double *z, int part, int nparts,
                        int *pos0, int *count, void *stream) {
    if (n < 1) return -1;
    if (n > 1 && !d) return -2;
    if (n > 1 && !z) return -3;
    if (part < 0 || part >= nparts) return -4;
    if (nparts < 1) return -5;
    if (!pos0) return -6;
    if (!count) return -7;
    const ae::Outputs out = make_outputs(nullptr, nullptr, n, nullptr, 0, nullptr, nullptr,
                                         nullptr);
    const PartSpec ps{part, nparts, 0, pos0, count};
    return solve_common(ae::KIND_ARROW, n, d, z, 0.0, 0.0, out, nullptr, nullptr, stream,
                        nullptr, &ps);
}

int dpr1_eig(int n, const double *d, const double *u, double rho, double *lambda, double *Q,
             int ldq, const ae_opts *opts, ae_info *info, const ae_diag *diag, void *stream) {
    if (n < 1) return -1;
    if (!d) return -2;
    if (!u) return -3;
    if (!isfinite(rho)) return -4;
    if (!lambda) return -5;
    if (Q && ldq < n) return -7;
    const ae::Outputs out = make_outputs(lambda, Q, ldq, nullptr, 0, nullptr, nullptr, diag);
    // rho = 0 is D itself: every row deflates (the spikes are scaled by rho)
    return solve_common(ae::KIND_DPR1, n, d, u, 0.0, rho, out, opts, info, stream);
}

int tri_arrow_svd(int n, const double *d, const double *z, double alpha, double *sigma,
                  double *U, int ldu, double *V, int ldv, const ae_opts *opts, ae_info *info,
                  const ae_diag *diag, void *stream) {
    if (n < 1) return -1;
    if (n > 1 && !d) return -2;
    if (n > 1 && !z) return -3;
    if (!isfinite(alpha) || alpha == 0.0) return -4;
    if (!sigma) return -5;
    if (U && ldu < n) return -7;
    if (V && ldv < n) return -9;
    if (U && !V) return -8;
    const ae::Outputs out = make_outputs(sigma, V, ldv, U, ldu, nullptr, nullptr, diag);
    return solve_common(ae::KIND_TSVD, n, d, z, alpha, 0.0, out, opts, info, stream);
}

int herm_arrow_eig(int n, const double *d, const double *z, double alpha, double *lambda,
                   double *U, int ldu, double *shift, double *mu, const ae_opts *opts,
                   ae_info *info, const ae_diag *diag, void *stream) {
    if (n < 1) return -1;
    if (n > 1 && !d) return -2;
    if (n > 1 && !z) return -3;
    if (!isfinite(alpha)) return -4;
    if (!lambda) return -5;
    if (U && ldu < n) return -7;
    // complex columns: ldu complex entries = 2 ldu doubles
    const ae::Outputs out = make_outputs(lambda, U, 2 * ldu, nullptr, 0, shift, mu, diag);
    return solve_common(ae::KIND_HERM, n, d, z, alpha, 0.0, out, opts, info, stream);
}

int nsym_arrow_eig(int n, const double *d, const double *zc, const double *zr, double alpha,
                   double *lambda, double *X, int ldx, double *Y, int ldy, double *shift,
                   double *mu, const ae_opts *opts, ae_info *info, const ae_diag *diag,
                   void *stream) {
    if (n < 1) return -1;
    if (n > 1 && !d) return -2;
    if (n > 1 && (!zc || !zr)) return -3;
    if (!isfinite(alpha)) return -4;
    if (!lambda) return -5;
    if (X && ldx < n) return -7;
    if (Y && !X) return -8;
    if (Y && ldy < n) return -9;
    const ae::Outputs out = make_outputs(lambda, X, ldx, Y, ldy, shift, mu, diag);
    return solve_common(ae::KIND_NSYM, n, d, zc, alpha, 0.0, out, opts, info, stream, zr);
}

int arrow_eig_host(int n, const double *d_host, const double *z_host, double alpha,
                   double *lambda_host, double *V_host, double *shift_host, double *mu_host,
                   const ae_opts *opts, ae_info *info, void *stream) {
    if (n < 1) return -1;
    if (n > 1 && !d_host) return -2;
    if (n > 1 && !z_host) return -3;
    if (!isfinite(alpha)) return -4;
    if (!lambda_host) return -5;
    cudaStream_t st = (cudaStream_t)stream;
    keep_pool_warm();
    const size_t n1 = (size_t)(n - 1);
    // V_host in page-locked memory the device can address (cudaHostAlloc /
    // cudaHostRegister): the solver writes the columns there itself, over the
    // host link while it computes, instead of a copy after the solve
    double *V_direct = nullptr;
    if (V_host) {
        cudaPointerAttributes pa;
        if (cudaPointerGetAttributes(&pa, V_host) == cudaSuccess &&
            pa.type == cudaMemoryTypeHost && pa.devicePointer)
            V_direct = (double *)pa.devicePointer;
        else
            cudaGetLastError();     // not registered: clear the lookup's error
    }
    const size_t vbytes = (V_host && !V_direct) ? sizeof(double) * (size_t)n * (size_t)n : 0;
    const size_t bytes = 256 * 6 + sizeof(double) * (2 * n1 + 3 * (size_t)n) + vbytes;
    void *base = nullptr;
    cudaError_t e = cudaMallocAsync(&base, bytes, st);
    if (e != cudaSuccess) return cuda_fail(e);
    char *p = (char *)base;
    auto take = [&](size_t b) {
        char *q = p;
        p += (b + 255) & ~(size_t)255;
        return (double *)q;
    };
    double *dd_ = take(sizeof(double) * (n1 ? n1 : 1));
    double *dz = take(sizeof(double) * (n1 ? n1 : 1));
    double *dl = take(sizeof(double) * n);
    double *ds = shift_host ? take(sizeof(double) * n) : nullptr;
    double *dm = mu_host ? take(sizeof(double) * n) : nullptr;
    double *dV = V_direct ? V_direct : (V_host ? take(vbytes) : nullptr);
    int status = AE_OK;
    if (n1) {
        e = cudaMemcpyAsync(dd_, d_host, sizeof(double) * n1, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dz, z_host, sizeof(double) * n1, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) status = cuda_fail(e);
    }
    if (status == AE_OK)
        status = arrow_eig(n, dd_, dz, alpha, dl, dV, n, ds, dm, opts, info, nullptr, stream);
    if (status == AE_OK) {
        e = cudaMemcpyAsync(lambda_host, dl, sizeof(double) * n, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && dV && !V_direct)
            e = cudaMemcpyAsync(V_host, dV, vbytes, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && ds)
            e = cudaMemcpyAsync(shift_host, ds, sizeof(double) * n, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && dm)
            e = cudaMemcpyAsync(mu_host, dm, sizeof(double) * n, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) status = cuda_fail(e);
    }
    cudaError_t e2 = cudaFreeAsync(base, st);
    cudaError_t e3 = cudaStreamSynchronize(st);
    if (status == AE_OK && e2 != cudaSuccess) status = cuda_fail(e2);
    if (status == AE_OK && e3 != cudaSuccess) status = cuda_fail(e3);
    return status;
}

int ae_fma_peaks(double *fp64_tflops, double *fp32_tflops, void *stream) {
    if (!fp64_tflops && !fp32_tflops) return -1;
    cudaError_t e = ae::probe_fma_rates(fp64_tflops, fp32_tflops, (cudaStream_t)stream);
    return e == cudaSuccess ? AE_OK : cuda_fail(e);
}

int ae_debug_rcp(int n, const double *x, double *y, void *stream) {
    if (n < 0) return -1;
    if (n > 0 && !x) return -2;
    if (n > 0 && !y) return -3;
    cudaError_t e = ae::launch_debug_rcp(n, x, y, (cudaStream_t)stream);
    return e == cudaSuccess ? AE_OK : cuda_fail(e);
}

int ae_debug_newton(int m, const double *delta, const double *cj, double b, double c, int side,
                    double pole, double left, double right, double x0, double dF0, double xdF0,
                    double rel0, int max_iter, double *out, void *stream) {
    if (m < 0) return -1;
    if (m > 0 && !delta) return -2;
    if (m > 0 && !cj) return -3;
    if (!(c > 0.0) || !isfinite(b)) return -4;
    if (side != 1 && side != -1) return -6;
    if (!(left < right)) return -8;
    if (max_iter < 1) return -14;
    if (!out) return -15;
    const ae::DebugNewton a{b, c, pole, left, right, x0, dF0, xdF0, rel0, side, max_iter};
    cudaError_t e = ae::launch_debug_newton(m, delta, cj, a, out, (cudaStream_t)stream);
    return e == cudaSuccess ? AE_OK : cuda_fail(e);
}

}  // extern "C"
