// ae_arrow.cu -- the eigen-solver pipeline on one stream, for the problem
// kinds that reduce to a real symmetric arrowhead (the kernels after the
// reduction are in ae_solve.cuh; this unit instantiates them for the
// arrowhead, ae_solve_*.cu for the other kinds):
//   ARROW  A = [diag(d) z; z^T alpha]                       (Sec. 1)
//   DPR1   M = diag(d) + rho u u^T, via A = L^{-1} M L        (Sec. 6.3)
//   SVD    B = [diag(d) z; 0 alpha], via A = B^T B            (Sec. 6.2)
//
//   k_check      validity / ordering flags; transformed keys and spikes
//   k_rank       stable descending order (ties: lower input row)   (Eq. order)
//   k_reduce     zero spikes deflated, equal poles folded, reduced poles
//                compacted (single CTA, block scans)               (Sec. 1)
//   k_post<K>    kind-specific arrowhead data (DPR1: spikes and corner of
//                L^{-1} M L; SVD: exact (d_j z_j)^2 and alpha^2 + z^T z), FP32 copies
//   k_eig<P>     one warp per eigenpair: Algorithm 1 shift, Algorithm 2 inverse
//                with b in double-double (Theorem 6), Algorithm 3 bisection
//   k_fix_decide / k_fix_solve<P>
//                Theorem C1 quotient > 3 -> Remark 1; K_nu (Eq. K0) above the
//                threshold -> Remark 2(a) other pole or 2(b) DPR1 shift; DPR1:
//                the last eigenvalue is re-solved next to the last pole
//   k_place      output positions (merge with deflated values)
//   k_vectors<K> one warp per column: v = x/||x|| (Eq. eigenvecAi / Algorithm 4),
//                DPR1 q ~ (D - lambda)^{-1} u, SVD right and left vectors
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "ae_internal.h"
#include "ae_pipeline.cuh"
#include "ae_solve.cuh"

namespace ae {

// ---------------------------------------------------------------------------
// input checks, transformed keys/spikes, ordering
// ---------------------------------------------------------------------------
// ARROW: key d, spike z.  DPR1: key sgn d (sgn = sign of rho), spike u.
// SVD: key d (> 0 required), spike d z.
// HERM: spike |zeta_r| of the complex (z[2r], z[2r+1]).  NSYM: spike
// sqrt(zc_r zr_r) of the pair (z[r], zrow[r]), which must share a sign or both
// be zero (the Remark of Sec. 6.1).
__global__ void k_check(Kind kind, int n1, const double *__restrict__ d,
                        const double *__restrict__ z, const double *__restrict__ zrow,
                        double sgn, Scratch S) {
    int flags = 0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n1; r += gridDim.x * blockDim.x) {
        const double dr = d[r];
        const double zr = kind == KIND_HERM ? z[2 * r] : z[r];
        if (!isfinite(dr) || !isfinite(zr)) flags |= CF_BAD;
        double key = dr, spk = zr;
        if (kind == KIND_DPR1) {
            key = sgn * dr;
            S.key[r] = key;
        } else if (kind == KIND_TSVD) {
            if (!(dr > 0.0)) flags |= CF_BAD;
            spk = dr * zr;
            S.spk[r] = spk;
        } else if (kind == KIND_HERM) {
            const double zi = z[2 * r + 1];
            if (!isfinite(zi)) flags |= CF_BAD;
            spk = hypot(zr, zi);
            S.spk[r] = spk;
        } else if (kind == KIND_NSYM) {
            const double zw = zrow[r];
            if (!isfinite(zw)) flags |= CF_BAD;
            if ((zr == 0.0) != (zw == 0.0) || (zr != 0.0 && (zr > 0.0) != (zw > 0.0)))
                flags |= CF_BAD;
            spk = sqrt(fabs(zr)) * sqrt(fabs(zw));
            S.spk[r] = spk;
        }
        if (spk == 0.0) flags |= CF_ZERO;
        if (key == 0.0) flags |= CF_ZEROPOLE;
        if (r + 1 < n1) {
            const double kn = kind == KIND_DPR1 ? sgn * d[r + 1] : d[r + 1];
            if (!(key > kn)) flags |= CF_UNSORTED;
        }
    }
    flags = __reduce_or_sync(FULL, flags);
    if ((threadIdx.x & 31) == 0 && flags) atomicOr(S.cnt + C_FLAGS, flags);
}

// perm[s] = input row at sorted position s (descending, ties by lower row)
__global__ void k_rank(int n1, const double *__restrict__ key, const int *cnt, int *perm) {
    __shared__ double tile[1024];
    const bool sorted = !(cnt[C_FLAGS] & CF_UNSORTED);
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (sorted) {
        if (r < n1) perm[r] = r;
        return;
    }
    // NaN compares as -inf here so that ranks always form a permutation (the
    // input is rejected later, but no index may leave its array meanwhile)
    const double dr = r < n1 ? (isnan(key[r]) ? -INFINITY : key[r]) : 0.0;
    int rank = 0;
    for (int base = 0; base < n1; base += 1024) {
        __syncthreads();
        for (int t = threadIdx.x; t < 1024; t += blockDim.x) {
            const double v = base + t < n1 ? key[base + t] : 0.0;
            tile[t] = isnan(v) ? -INFINITY : v;
        }
        __syncthreads();
        const int lim = min(1024, n1 - base);
        if (r < n1) {
            for (int t = 0; t < lim; ++t) {
                const double dq = tile[t];
                const int q = base + t;
                rank += (dq > dr) || (dq == dr && q < r);
            }
        }
    }
    if (r < n1) perm[rank] = r;
}

// Reduction (single CTA of 1024 threads) and the kind-specific arrowhead data.
__global__ void __launch_bounds__(1024) k_reduce(int n1, const double *__restrict__ key,
                                                 const double *__restrict__ spk,
                                                 const int *__restrict__ perm, Scratch S) {
    reduce_block(n1, key, spk, perm, S);
}

template <Kind K>
__global__ void __launch_bounds__(1024) k_post(int n1, const double *__restrict__ d,
                                               const double *__restrict__ z,
                                               const double *__restrict__ zrow, double alpha,
                                               double rho_abs, Scratch S) {
    post_block<K>(n1, d, z, zrow, alpha, rho_abs, S);
}

// One part of a split solve: its eigenpair range (an even split of the m + 1
// computed eigenpairs), its deflated rows and its first output position.
__global__ void k_part(Scratch S, int part, int nparts) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int nd = S.cnt[C_ND], ncomp = S.cnt[C_M] + 1;
    const int k0 = (int)((long long)part * ncomp / nparts);
    const int k1 = (int)((long long)(part + 1) * ncomp / nparts);
    // deflated values (non-increasing) in [p_{k1-1}, p_{k0-1})
    const int u0 = k0 == 0 ? 0 : count_ge(S.dval, nd, S.pv[k0 - 1], false);
    const int u1 = k1 == ncomp ? nd : (k1 == 0 ? 0 : count_ge(S.dval, nd, S.pv[k1 - 1], false));
    S.cnt[C_K0] = k0;
    S.cnt[C_K1] = k1;
    S.cnt[C_U0] = u0;
    S.cnt[C_U1] = u1 > u0 ? u1 : u0;
    S.cnt[C_POS0] = k0 + u0;
    S.cnt[C_WORK] = k0 > 0 ? k0 - 1 : 0;             // k_eig's first ticket
    S.cnt[C_KHI] = k1 < ncomp ? k1 + 1 : ncomp;
    S.cnt[C_PART] = 1;
}

__global__ void k_debug_rcp(int n, const double *x, double *y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = rcp(x[i]);
}

// The FP64 finish (newton_finish) on the shifted inverse's Pick function
// F(x) = (b - x) - c (sum_j cj_j / (1 - x delta_j) - 1/x), kappa = -1, from a
// caller's bracket, start and F' estimate; one thread.  out: nu (the right end
// of the final bracket), the FP64 evaluations, those with F'.
__global__ void k_debug_newton(int m, const double *__restrict__ delta,
                               const double *__restrict__ cj, DebugNewton a, double *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    auto FD = [&](double x, bool need_d, double &dF, double &err) {
        double S = 0.0, Sd = 0.0;
        for (int j = 0; j < m; ++j) {
            const double t = rcp(fma(-x, delta[j], 1.0));
            const double q = cj[j] * t;
            S += q;
            if (need_d) Sd = fma(q * delta[j], t, Sd);
        }
        const double rx = rcp(x);
        if (need_d) dF = -1.0 - a.c * fma(rx, rx, Sd);
        err = 0x1p-52 * (fabs(a.b) + fabs(x) + a.c * (fabs(S) + fabs(rx)));
        return (a.b - x) - a.c * (S - rx);
    };
    double left = a.left, right = a.right;
    bool fb;
    int itd = 0;
    const int it = newton_finish(FD, a.side, a.pole, -1.0, left, right, true, true, a.max_iter,
                                 left, right, fb, a.dF0, &itd, a.x0, a.c, a.xdF0, a.rel0);
    out[0] = right;
    out[1] = (double)it;
    out[2] = (double)itd;
}

// ---------------------------------------------------------------------------
// scratch layout
// ---------------------------------------------------------------------------
// One layout routine serves both sizing and carving, so they cannot disagree:
// every array starts on a 256-byte boundary.
static size_t layout(uintptr_t base, int n, Scratch *S) {
    const size_t n1 = n > 1 ? (size_t)n : 1;     // rows: n - 1 (arrowhead) or n (DPR1)
    const size_t nn = (size_t)n;
    uintptr_t p = (base + 255) & ~(uintptr_t)255;
    const uintptr_t start = base;
    auto take = [&](size_t bytes) {
        uintptr_t q = p;
        p += (bytes + 255) & ~(size_t)255;
        return (void *)q;
    };
    Scratch T;
    T.cnt = (int *)take(sizeof(int) * C_COUNT);
    T.cnt64 = (unsigned long long *)take(sizeof(unsigned long long) * C64_COUNT);
    T.prm = (double *)take(sizeof(double) * P_COUNT);
    T.perm = (int *)take(sizeof(int) * n1);
    T.spos = (int *)take(sizeof(int) * n1);
    T.kind = (int *)take(sizeof(int) * n1);
    T.run_s0 = (int *)take(sizeof(int) * n1);
    T.run_R = (double *)take(sizeof(double) * 2 * n1);
    T.key = (double *)take(sizeof(double) * n1);
    T.spk = (double *)take(sizeof(double) * n1);
    T.pd = (double *)take(sizeof(double) * n1);
    T.pz = (double *)take(sizeof(double) * n1);
    T.pz2 = (double *)take(sizeof(double) * n1);
    T.pz2lo = (double *)take(sizeof(double) * n1);
    T.pv = (double *)take(sizeof(double) * n1);
    T.pdh = (float *)take(sizeof(float) * n1);
    T.pdl = (float *)take(sizeof(float) * n1);
    T.pz2f = (float *)take(sizeof(float) * n1);
    T.prow = (int *)take(sizeof(int) * n1);
    T.drow = (int *)take(sizeof(int) * n1);
    T.dval = (double *)take(sizeof(double) * n1);
    T.es_sigma = (double *)take(sizeof(double) * nn);
    T.es_mu = (double *)take(sizeof(double) * nn);
    T.es_lam = (double *)take(sizeof(double) * nn);
    T.es_b = (double *)take(sizeof(double) * nn);
    T.es_Kb = (double *)take(sizeof(double) * nn);
    T.es_Knu = (double *)take(sizeof(double) * nn);
    T.es_fixshift = (double *)take(sizeof(double) * nn);
    T.es_pole = (int *)take(sizeof(int) * nn);
    T.es_iters = (int *)take(sizeof(int) * nn);
    T.es_flags = (int *)take(sizeof(int) * nn);
    T.es_fixpole = (int *)take(sizeof(int) * nn);
    T.fixlist = (int *)take(sizeof(int) * nn);
    T.pos = (int *)take(sizeof(int) * nn);
    T.pos0 = (int *)take(sizeof(int) * nn);
    T.wbuf = nullptr;
    T.wstride = 0;
    if (S) *S = T;
    return (size_t)(p - start);
}

// bytes to request: the layout from a 256-aligned base, plus room to align
size_t arrow_scratch_bytes(int n) { return layout(0, n, nullptr) + 256; }

Scratch carve_scratch(void *base, int n) {
    Scratch S;
    layout((uintptr_t)base, n, &S);
    return S;
}

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------
// CTAs of k_eig: enough for every eigenpair, at most what stays resident
// (every kind's k_eig has the same launch bounds, so the arrowhead's
// occupancy holds for all; the stored-pair slices are allocated for this grid)
static int eig_grid(int n) {
    static int per_sm = 0;
    if (!per_sm) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_eig<KIND_ARROW, KIND_ARROW>,
                                                      256, 0);
        if (per_sm <= 0) per_sm = 1;
    }
    const int want = (n + 7) / 8;
    const int cap = sm_count() * per_sm;
    return want < cap ? want : cap;
}

int eig_grid_warps(int n) { return eig_grid(n) * 8; }

cudaError_t launch_solve(Kind kind, int n, const double *d, const double *z, double alpha,
                         double rho, const Outputs &out, const RunOpts &ro, Scratch S,
                         cudaStream_t st, const double *zrow) {
    const int n1 = kind == KIND_DPR1 ? n : n - 1;
    const double sgn = (kind == KIND_DPR1 && rho < 0.0) ? -1.0 : 1.0;
    const double *key = (kind == KIND_DPR1 && sgn < 0.0) ? S.key : d;
    const bool rho0 = kind == KIND_DPR1 && rho == 0.0;   // M = D: every row deflates
    const bool own_spk = kind == KIND_TSVD || kind == KIND_HERM || kind == KIND_NSYM || rho0;
    const double *spk = own_spk ? S.spk : z;
    cudaError_t e;
    e = cudaMemsetAsync(S.cnt, 0, sizeof(int) * C_COUNT, st);
    if (e) return e;
    if (rho0 && n1 > 0) {
        e = cudaMemsetAsync(S.spk, 0, sizeof(double) * n1, st);
        if (e) return e;
    }
    e = cudaMemsetAsync(S.cnt64, 0, sizeof(unsigned long long) * C64_COUNT, st);
    if (e) return e;
    if (ro.ev[0]) cudaEventRecord(ro.ev[0], st);
    if (n1 > 0) {
        const int g = (n1 + 255) / 256;
        k_check<<<g, 256, 0, st>>>(kind, n1, d, z, zrow, sgn, S);
        k_rank<<<g, 256, 0, st>>>(n1, key, S.cnt, S.perm);
    }
    k_reduce<<<1, 1024, 0, st>>>(n1, key, spk, S.perm, S);
    SolveOpts so{ro.max_iter, ro.precision, ro.finish, ro.bgate, ro.kb_max};
    VecArgs va{n, n1, key, spk, z, zrow, alpha, sgn, out, (S.wbuf && out.V) ? 1 : 0};
    const int grid = eig_grid(n);
    switch (kind) {
        case KIND_ARROW:
            k_post<KIND_ARROW><<<1, 1024, 0, st>>>(n1, d, z, zrow, alpha, 0.0, S);
            launch_pipeline<KIND_ARROW, KIND_ARROW>(n, grid, S, so, ro, va, st);
            break;
        case KIND_DPR1:
            k_post<KIND_DPR1><<<1, 1024, 0, st>>>(n1, d, z, zrow, alpha, fabs(rho), S);
            launch_pipeline_dpr1(n, grid, S, so, ro, va, st);
            break;
        case KIND_TSVD:
            k_post<KIND_TSVD><<<1, 1024, 0, st>>>(n1, d, z, zrow, alpha, 0.0, S);
            launch_pipeline_tsvd(n, grid, S, so, ro, va, st);
            break;
        case KIND_HERM:
            k_post<KIND_HERM><<<1, 1024, 0, st>>>(n1, d, z, zrow, alpha, 0.0, S);
            launch_pipeline_herm(n, grid, S, so, ro, va, st);
            break;
        case KIND_NSYM:
            k_post<KIND_NSYM><<<1, 1024, 0, st>>>(n1, d, z, zrow, alpha, 0.0, S);
            launch_pipeline_nsym(n, grid, S, so, ro, va, st);
            break;
    }
    if (ro.ev[4]) cudaEventRecord(ro.ev[4], st);
    return cudaGetLastError();
}

cudaError_t launch_arrow_part(int n, const double *d, const double *z, double alpha, int part,
                              int nparts, int cap, const Outputs &out, const RunOpts &ro,
                              Scratch S, cudaStream_t st, int *pos0, int *count) {
    const int n1 = n - 1;
    cudaError_t e = cudaMemsetAsync(S.cnt, 0, sizeof(int) * C_COUNT, st);
    if (!e) e = cudaMemsetAsync(S.cnt64, 0, sizeof(unsigned long long) * C64_COUNT, st);
    if (e) return e;
    if (ro.ev[0]) cudaEventRecord(ro.ev[0], st);
    if (n1 > 0) {
        const int g = (n1 + 255) / 256;
        k_check<<<g, 256, 0, st>>>(KIND_ARROW, n1, d, z, nullptr, 1.0, S);
        k_rank<<<g, 256, 0, st>>>(n1, d, S.cnt, S.perm);
    }
    k_reduce<<<1, 1024, 0, st>>>(n1, d, z, S.perm, S);
    k_post<KIND_ARROW><<<1, 1024, 0, st>>>(n1, d, z, nullptr, alpha, 0.0, S);
    k_part<<<1, 32, 0, st>>>(S, part, nparts);
    int h[C_COUNT];
    e = cudaMemcpyAsync(h, S.cnt, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (e) return e;
    *pos0 = h[C_POS0];
    *count = (h[C_K1] - h[C_K0]) + (h[C_U1] - h[C_U0]);
    if (!out.lambda || *count > cap) return cudaSuccess;   // size query, or no room
    const SolveOpts so{ro.max_iter, ro.precision, ro.finish, ro.bgate, ro.kb_max};
    const VecArgs va{n, n1, d, z, z, nullptr, alpha, 1.0, out, (S.wbuf && out.V) ? 1 : 0};
    launch_pipeline<KIND_ARROW, KIND_ARROW>(n, eig_grid(n), S, so, ro, va, st);
    if (ro.ev[4]) cudaEventRecord(ro.ev[4], st);
    return cudaGetLastError();
}

cudaError_t launch_debug_rcp(int n, const double *x, double *y, cudaStream_t st) {
    if (n > 0) k_debug_rcp<<<(n + 255) / 256, 256, 0, st>>>(n, x, y);
    return cudaGetLastError();
}

cudaError_t launch_debug_newton(int m, const double *delta, const double *cj,
                                const DebugNewton &a, double *out, cudaStream_t st) {
    k_debug_newton<<<1, 32, 0, st>>>(m, delta, cj, a, out);
    return cudaGetLastError();
}

}  // namespace ae
