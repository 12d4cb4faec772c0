// ae_arrow.cu -- the arrowhead eigen-solver pipeline on one stream.
//
//   k_check     validity / ordering flags of the input            (Sec. 1)
//   k_rank      stable descending order (ties: lower input row)   (Sec. 1, Eq. order)
//   k_reduce    zero spikes deflated, equal poles folded, reduced
//               poles compacted (single CTA, block scans)         (Sec. 1)
//   k_eig       one warp per eigenpair: Algorithm 1 shift choice,
//               Algorithm 2 inverse with b in double-double
//               (Theorem 6), Algorithm 3 bisection, lambda = sigma + 1/nu
//   k_fix_decide / k_fix_solve
//               Theorem C1 quotient > 3 -> Remark 1; K_nu (Eq. K0) above
//               the threshold -> Remark 2(a) other pole or 2(b) DPR1 shift
//   k_place     output positions (merge with deflated values)
//   k_vectors   one warp per column: v = x/||x||, x = [(D-lambda)^{-1} z; -1]
//               (Eq. eigenvecAi / Algorithm 4), coalesced column writes
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "ae_internal.h"
#include "ae_solver.cuh"

namespace ae {

// ---------------------------------------------------------------------------
// input checks and ordering
// ---------------------------------------------------------------------------
__global__ void k_check(int n1, const double *__restrict__ d, const double *__restrict__ z,
                        int *cnt) {
    int flags = 0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n1; r += gridDim.x * blockDim.x) {
        const double dr = d[r], zr = z[r];
        if (!isfinite(dr) || !isfinite(zr)) flags |= CF_BAD;
        if (zr == 0.0) flags |= CF_ZERO;
        if (dr == 0.0) flags |= CF_ZEROPOLE;
        if (r + 1 < n1 && !(dr > d[r + 1])) flags |= CF_UNSORTED;
    }
    flags = __reduce_or_sync(FULL, flags);
    if ((threadIdx.x & 31) == 0 && flags) atomicOr(cnt + C_FLAGS, flags);
}

// perm[s] = input row at sorted position s (descending, ties by lower row)
__global__ void k_rank(int n1, const double *__restrict__ d, const int *cnt, int *perm) {
    __shared__ double tile[1024];
    const bool sorted = !(cnt[C_FLAGS] & CF_UNSORTED);
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (sorted) {
        if (r < n1) perm[r] = r;
        return;
    }
    // NaN compares as -inf here so that ranks always form a permutation (the
    // input is rejected later, but no index may leave its array meanwhile)
    const double dr = r < n1 ? (isnan(d[r]) ? -INFINITY : d[r]) : 0.0;
    int rank = 0;
    for (int base = 0; base < n1; base += 1024) {
        __syncthreads();
        for (int t = threadIdx.x; t < 1024; t += blockDim.x) {
            const double v = base + t < n1 ? d[base + t] : 0.0;
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

// block-wide exclusive scan of one int per thread (blockDim = 1024)
__device__ __forceinline__ int block_exscan(int v, int *warp_tot, int &total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int t = warp_tot[lane];
        int u = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(FULL, u, o);
            if (lane >= o) u += y;
        }
        warp_tot[lane] = u - t;       // exclusive prefix of warp totals
        if (lane == 31) warp_tot[32] = u;
    }
    __syncthreads();
    const int res = warp_tot[wid] + x - v;
    total = warp_tot[32];
    __syncthreads();
    return res;
}

// Reduction (single CTA of 1024 threads, loops over chunks of the sorted order).
__global__ void __launch_bounds__(1024) k_reduce(int n1, const double *__restrict__ d,
                                                 const double *__restrict__ z,
                                                 const int *__restrict__ perm, Scratch S) {
    __shared__ int wt[33];
    int carry_keep = 0, carry_defl = 0;
    for (int base = 0; base < n1; base += 1024) {
        const int s = base + threadIdx.x;
        int keep = 0, defl = 0;
        int r = -1;
        double dr = 0.0, zr = 0.0;
        bool zero = false, head = false;
        if (s < n1) {
            r = perm[s];
            dr = d[r];
            zr = z[r];
            zero = (zr == 0.0);
            if (!zero) {
                head = true;   // the first nonzero row of its run of equal poles
                for (int q = s - 1; q >= 0; --q) {
                    const int rq = perm[q];
                    if (d[rq] != dr) break;
                    if (z[rq] != 0.0) { head = false; break; }
                }
            }
            keep = head ? 1 : 0;
            defl = head ? 0 : 1;
        }
        int tk, td;
        const int jk = block_exscan(keep, wt, tk) + carry_keep;
        const int jd = block_exscan(defl, wt, td) + carry_defl;
        if (s < n1) {
            S.spos[r] = s;
            if (head) {
                // reduced spike: sqrt of the sum of squares over the run
                double acc = fabs(zr);
                for (int q = s + 1; q < n1; ++q) {
                    const int rq = perm[q];
                    if (d[rq] != dr) break;
                    acc = hypot(acc, z[rq]);
                }
                S.pd[jk] = dr;
                S.pz[jk] = acc;
                S.pz2[jk] = acc * acc;
                S.prow[jk] = r;
                S.kind[r] = 0;
            } else {
                S.kind[r] = zero ? 1 : 2;
                S.drow[jd] = r;
                S.dval[jd] = dr;
                if (!zero) {
                    // Helmert-type vector data: R_{m-1} over earlier nonzero
                    // members of the run, R_m including this row
                    double Rm1 = 0.0;
                    int q = s - 1;
                    for (; q >= 0; --q) {
                        const int rq = perm[q];
                        if (d[rq] != dr) break;
                        Rm1 = hypot(Rm1, z[rq]);
                    }
                    S.run_s0[r] = q + 1;
                    S.run_R[2 * r] = Rm1;
                    S.run_R[2 * r + 1] = hypot(Rm1, zr);
                }
            }
        }
        carry_keep += tk;
        carry_defl += td;
    }
    if (threadIdx.x == 0) {
        S.cnt[C_M] = carry_keep;
        S.cnt[C_ND] = carry_defl;
    }
    // FP32 copies for the opening bracket, scaled by powers of two so that the
    // largest |pole| and the largest spike^2 are O(1)
    __syncthreads();
    __shared__ double red[2][32];
    const int m = carry_keep;
    double mxd = 0.0, mxz = 0.0;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        mxd = fmax(mxd, fabs(S.pd[j]));
        mxz = fmax(mxz, S.pz2[j]);
    }
    mxd = warp_max(mxd);
    mxz = warp_max(mxz);
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = mxd;
        red[1][threadIdx.x >> 5] = mxz;
    }
    __syncthreads();
    mxd = 0.0;
    mxz = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        mxd = fmax(mxd, red[0][w]);
        mxz = fmax(mxz, red[1][w]);
    }
    const double ds = (mxd > 0.0 && isfinite(mxd)) ? ldexp(1.0, -ilogb(mxd)) : 1.0;
    const double zs = (mxz > 0.0 && isfinite(mxz)) ? ldexp(1.0, -ilogb(mxz)) : 1.0;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        const double v = S.pd[j] * ds;
        const float h = (float)v;
        S.pdh[j] = h;
        S.pdl[j] = (float)(v - (double)h);
        S.pz2f[j] = (float)(S.pz2[j] * zs);
    }
    if (threadIdx.x == 0) {
        S.fscale[0] = ds;
        S.fscale[1] = zs;
    }
}

// ---------------------------------------------------------------------------
// eigenpairs
// ---------------------------------------------------------------------------
__device__ __forceinline__ void store_result(const Scratch &S, int k, const EigResult &r) {
    S.es_sigma[k] = r.sigma;
    S.es_mu[k] = r.mu;
    S.es_lam[k] = r.lam;
    S.es_b[k] = r.b;
    S.es_Kb[k] = r.Kb;
    S.es_pole[k] = r.pole;
    S.es_iters[k] = r.iters;
}

__device__ __forceinline__ void record_stats(const Scratch &S, const EigResult &r,
                                             bool fix = false) {
    atomicAdd(S.cnt64 + C64_ITERS, (unsigned long long)r.iters);
    if (fix) atomicAdd(S.cnt64 + C64_ITERS_FIX, (unsigned long long)r.iters);
    atomicMax(S.cnt + C_MAXIT, r.iters);
    if (r.flags & AE_FLAG_CAPPED) atomicAdd(S.cnt + C_CAPPED, 1);
    if (r.flags & AE_FLAG_FP32_FALLBACK) atomicAdd(S.cnt + C_FP32FB, 1);
    if (isfinite(r.Kb)) atomic_max_nonneg(S.cnt64 + C64_MAXKB, r.Kb);
}

__global__ void __launch_bounds__(256) k_eig(double alpha, Scratch S, SolveOpts o) {
    const int lane = threadIdx.x & 31;
    const int m = S.cnt[C_M];
    const int ncomp = m + 1;
    const ArrowPoles R = {m,       S.pd,   S.pz,   S.pz2,          alpha,
                          S.pdh,   S.pdl,  S.pz2f, S.fscale[0],    S.fscale[1]};
    for (;;) {
        int k = 0;
        if (lane == 0) k = atomicAdd(S.cnt + C_WORK, 1);
        k = __shfl_sync(FULL, k, 0);
        if (k >= ncomp) break;
        EigResult res;
        if (m == 0) {
            res = {alpha, 0.0, alpha, NAN, 0.0, -1, 0, 0};
        } else {
            const WarpTeam T{lane};
            int i, side;
            select_shift(R, T, k, i, side);
            res = solve_shifted(R, T, i, side, o);
        }
        if (lane == 0) {
            store_result(S, k, res);
            S.es_flags[k] = res.flags;
            S.es_Knu[k] = 1.0;
            record_stats(S, res);
        }
    }
}

// Remedy decisions: one thread per eigenpair.
__global__ void k_fix_decide(Scratch S, double knu_max) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int m = S.cnt[C_M];
    if (k > m || m == 0) return;
    const double lam = S.es_lam[k], sig = S.es_sigma[k], mu = S.es_mu[k];
    const int i = S.es_pole[k];
    const double q = (fabs(sig) + fabs(mu)) / fabs(lam);
    int remedy = 0;
    double knu = 1.0;
    // Theorem C1 bounds the quotient by 3 except in the special cases (a)-(c);
    // Remark 1 needs D nonsingular.
    if (q > 3.0 && !(S.cnt[C_FLAGS] & CF_ZEROPOLE)) {
        remedy = AE_FLAG_NEARZERO;
    } else if (i >= 0) {
        // K_nu = |mu| / min(|mu|, |mu_o|), mu_o from the eigenvalue on the other
        // side of the shift pole
        const int kn = mu > 0.0 ? k + 1 : k - 1;
        if (kn >= 0 && kn <= m) {
            const double muo = (S.es_sigma[kn] - sig) + S.es_mu[kn];
            knu = fmax(1.0, fabs(mu) / fabs(muo));
        }
        if (knu > knu_max) {
            // Remark 2(a): the other pole of lambda's interval, if its K_nu is small
            const int io = mu > 0.0 ? i - 1 : i + 1;
            const int kn2 = mu > 0.0 ? k - 1 : k + 1;
            if (io >= 0 && io < m) {
                const double po = S.pd[io];
                const double mu2 = lam - po;
                double k2 = 1.0;
                if (kn2 >= 0 && kn2 <= m) {
                    const double muo2 = (S.es_sigma[kn2] - po) + S.es_mu[kn2];
                    k2 = fmax(1.0, fabs(mu2) / fabs(muo2));
                }
                if (k2 <= knu_max) {
                    remedy = AE_FLAG_OTHERPOLE;
                    S.es_fixpole[k] = io;
                }
            }
            if (!remedy) {
                // Remark 2(b): shift near lambda, inside its interval, not a pole
                double sh = lam;
                const double lo = k < m ? S.pd[k] : -INFINITY;
                const double hi = k > 0 ? S.pd[k - 1] : INFINITY;
                if (!(sh > lo)) sh = nextafter(lo, INFINITY);
                if (!(sh < hi)) sh = nextafter(hi, -INFINITY);
                S.es_fixshift[k] = sh;
                remedy = AE_FLAG_DPR1SHIFT;
            }
        }
    }
    S.es_Knu[k] = knu;
    atomic_max_nonneg(S.cnt64 + C64_MAXKNU, knu);
    if (remedy) {
        S.es_flags[k] |= remedy;
        const int slot = atomicAdd(S.cnt + C_NFIX, 1);
        S.fixlist[slot] = k;
        atomicAdd(S.cnt + (remedy == AE_FLAG_NEARZERO ? C_NEARZERO
                           : remedy == AE_FLAG_OTHERPOLE ? C_OTHERPOLE : C_DPR1), 1);
    }
}

// Remedy solves: one CTA (8 warps) per listed eigenpair, so that the few
// eigenpairs that need one still fill the GPU.
__global__ void __launch_bounds__(256) k_fix_solve(double alpha, Scratch S, SolveOpts o) {
    __shared__ double red[16];
    __shared__ int ticket;
    const int m = S.cnt[C_M];
    const int nfix = S.cnt[C_NFIX];
    const ArrowPoles R = {m,       S.pd,   S.pz,   S.pz2,          alpha,
                          S.pdh,   S.pdl,  S.pz2f, S.fscale[0],    S.fscale[1]};
    const CtaTeam<8> T{(int)threadIdx.x, red};
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) ticket = atomicAdd(S.cnt + C_WORK2, 1);
        __syncthreads();
        const int w = ticket;
        if (w >= nfix) break;
        const int k = S.fixlist[w];
        const int f = S.es_flags[k];
        EigResult res;
        if (f & AE_FLAG_NEARZERO) {
            res = solve_dpr1_shift(R, T, 0.0, o);
        } else if (f & AE_FLAG_OTHERPOLE) {
            const int io = S.es_fixpole[k];
            const int side = io < S.es_pole[k] ? -1 : +1;   // other pole above -> lambda below it
            res = solve_shifted(R, T, io, side, o);
        } else {
            res = solve_dpr1_shift(R, T, S.es_fixshift[k], o);
        }
        // the result must stay in the eigenvalue's interlacing interval
        const double lo = k < m ? R.pole(k) : -INFINITY;
        const double hi = k > 0 ? R.pole(k - 1) : INFINITY;
        const bool ok = (res.lam >= lo && res.lam <= hi) && isfinite(res.lam);
        if (threadIdx.x == 0) {
            if (ok) {
                // b and K_b stay those of Algorithm 1's shift pole
                res.b = S.es_b[k];
                res.Kb = S.es_Kb[k];
                store_result(S, k, res);
                S.es_flags[k] = f | res.flags;
                record_stats(S, res, true);
            } else {
                S.es_flags[k] = f & ~(AE_FLAG_NEARZERO | AE_FLAG_OTHERPOLE | AE_FLAG_DPR1SHIFT);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// output placement and vectors
// ---------------------------------------------------------------------------
// number of entries of a non-increasing array that are >= x (or > x)
__device__ __forceinline__ int count_ge(const double *a, int len, double x, bool strict) {
    int lo = 0, hi = len;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const bool in = strict ? (a[mid] > x) : (a[mid] >= x);
        if (in) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void k_place(Scratch S) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int m = S.cnt[C_M], nd = S.cnt[C_ND];
    const int ncomp = m + 1;
    if (t < ncomp) {
        S.pos[t] = nd ? t + count_ge(S.dval, nd, S.es_lam[t], false) : t;
    } else if (t < ncomp + nd) {
        const int u = t - ncomp;
        S.pos[t] = u + count_ge(S.es_lam, ncomp, S.dval[u], true);
    }
}

__global__ void __launch_bounds__(256) k_vectors(int n, const double *__restrict__ d,
                                                 const double *__restrict__ z, double alpha,
                                                 Scratch S, Outputs out) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int n1 = n - 1;
    const int m = S.cnt[C_M], nd = S.cnt[C_ND];
    const int ncomp = m + 1;
    for (int item = warp; item < ncomp + nd; item += nwarps) {
        const int pos = S.pos[item];
        double *col = out.V ? out.V + (size_t)pos * out.ldv : nullptr;
        if (item < ncomp) {
            const int k = item;
            const double sig = S.es_sigma[k], mu = S.es_mu[k];
            if (lane == 0) {
                out.lambda[pos] = S.es_lam[k];
                if (out.shift) out.shift[pos] = sig;
                if (out.mu) out.mu[pos] = mu;
                if (out.dg_b) out.dg_b[pos] = S.es_b[k];
                if (out.dg_Kb) out.dg_Kb[pos] = S.es_Kb[k];
                if (out.dg_Knu) out.dg_Knu[pos] = S.es_Knu[k];
                if (out.dg_iters) out.dg_iters[pos] = S.es_iters[k];
                if (out.dg_flags) out.dg_flags[pos] = S.es_flags[k];
            }
            if (!col) continue;
            // x_r = z_r / ((d_r - sigma) - mu) for every input row, x_{n-1} = -1.
            // Pass 1 stores x in the column and sums x^2 in sorted order (so the
            // norm does not depend on the order of the input rows); pass 2
            // scales the column in place.
            double s = 0.0;
            for (int q = lane; q < n1; q += 32) {
                const int r = S.perm[q];
                const double zr = z[r];
                const double x = zr == 0.0 ? 0.0 : zr * rcp((d[r] - sig) - mu);
                col[r] = x;
                s = fma(x, x, s);
            }
            s = warp_sum(s) + 1.0;
            if (isfinite(s)) {
                const double inv = 1.0 / sqrt(s);
                __syncwarp();
                for (int r = lane; r < n1; r += 32) col[r] *= inv;
                if (lane == 0) col[n1] = -inv;
                continue;
            }
            double scale = 1.0, inv;
            {
                // rescale by the largest component to avoid overflow
                double xm = 1.0;
                for (int r = lane; r < n1; r += 32) {
                    const double zr = z[r];
                    if (zr != 0.0) xm = fmax(xm, fabs(zr * rcp((d[r] - sig) - mu)));
                }
                xm = warp_max(xm);
                scale = 1.0 / xm;
                double s2 = 0.0;
                for (int q = lane; q < n1; q += 32) {
                    const int r = S.perm[q];
                    const double zr = z[r];
                    const double x = zr == 0.0 ? 0.0 : zr * rcp((d[r] - sig) - mu) * scale;
                    s2 = fma(x, x, s2);
                }
                s2 = warp_sum(s2) + scale * scale;
                inv = 1.0 / sqrt(s2);
            }
            for (int r = lane; r < n1; r += 32) {
                const double zr = z[r];
                const double x = zr == 0.0 ? 0.0 : zr * rcp((d[r] - sig) - mu) * scale;
                col[r] = x * inv;
            }
            if (lane == 0) col[n1] = -scale * inv;
        } else {
            const int u = item - ncomp;
            const int row = S.drow[u];
            if (lane == 0) {
                out.lambda[pos] = S.dval[u];
                if (out.shift) out.shift[pos] = S.dval[u];
                if (out.mu) out.mu[pos] = 0.0;
                if (out.dg_b) out.dg_b[pos] = NAN;
                if (out.dg_Kb) out.dg_Kb[pos] = 0.0;
                if (out.dg_Knu) out.dg_Knu[pos] = 1.0;
                if (out.dg_iters) out.dg_iters[pos] = 0;
                if (out.dg_flags) out.dg_flags[pos] = AE_FLAG_DEFLATED;
            }
            if (!col) continue;
            for (int r = lane; r < n; r += 32) col[r] = 0.0;
            __syncwarp();
            if (S.kind[row] == 1) {
                if (lane == 0) col[row] = 1.0;
            } else {
                // m-th later member q_m of a run of equal poles:
                // (-z_{q_m} sum_{l<m} z_{q_l} e_{q_l} + R_{m-1}^2 e_{q_m}) / (R_{m-1} R_m)
                const double Rm1 = S.run_R[2 * row], Rm = S.run_R[2 * row + 1];
                const double zq = z[row];
                const double den = Rm1 * Rm;
                const int s0 = S.run_s0[row], s1 = S.spos[row];
                for (int s = s0 + lane; s < s1; s += 32) {
                    const int rq = S.perm[s];
                    const double zl = z[rq];
                    if (zl != 0.0) col[rq] = -(zq * zl) / den;
                }
                if (lane == 0) col[row] = Rm1 / Rm;
            }
        }
    }
}

__global__ void k_debug_rcp(int n, const double *x, double *y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = rcp(x[i]);
}

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------
static int sm_count() {
    static int cached = 0;
    if (!cached) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&cached, cudaDevAttrMultiProcessorCount, dev);
        if (cached <= 0) cached = 1;
    }
    return cached;
}

// One layout routine serves both sizing and carving, so they cannot disagree:
// every array starts on a 256-byte boundary.
static size_t layout(uintptr_t base, int n, Scratch *S) {
    const size_t n1 = n > 1 ? (size_t)n - 1 : 1;
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
    T.perm = (int *)take(sizeof(int) * n1);
    T.spos = (int *)take(sizeof(int) * n1);
    T.kind = (int *)take(sizeof(int) * n1);
    T.run_s0 = (int *)take(sizeof(int) * n1);
    T.run_R = (double *)take(sizeof(double) * 2 * n1);
    T.pd = (double *)take(sizeof(double) * n1);
    T.pz = (double *)take(sizeof(double) * n1);
    T.pz2 = (double *)take(sizeof(double) * n1);
    T.pdh = (float *)take(sizeof(float) * n1);
    T.pdl = (float *)take(sizeof(float) * n1);
    T.pz2f = (float *)take(sizeof(float) * n1);
    T.fscale = (double *)take(sizeof(double) * 2);
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

// Issue the whole solve on `st`.  Scratch must hold arrow_scratch_bytes(n).
cudaError_t launch_arrow(int n, const double *d, const double *z, double alpha,
                         const Outputs &out, const RunOpts &ro, Scratch S, cudaStream_t st) {
    const int n1 = n - 1;
    cudaError_t e;
    e = cudaMemsetAsync(S.cnt, 0, sizeof(int) * C_COUNT, st);
    if (e) return e;
    e = cudaMemsetAsync(S.cnt64, 0, sizeof(unsigned long long) * C64_COUNT, st);
    if (e) return e;
    const int sms = sm_count();
    if (ro.ev[0]) cudaEventRecord(ro.ev[0], st);
    if (n1 > 0) {
        const int g = (n1 + 255) / 256;
        k_check<<<g, 256, 0, st>>>(n1, d, z, S.cnt);
        k_rank<<<g, 256, 0, st>>>(n1, d, S.cnt, S.perm);
    }
    k_reduce<<<1, 1024, 0, st>>>(n1, d, z, S.perm, S);
    SolveOpts so{ro.max_iter, ro.precision};
    const int warps = n;   // upper bound on eigenpairs
    int grid = (warps + 7) / 8;
    grid = grid < sms * 8 ? grid : sms * 8;
    if (ro.ev[1]) cudaEventRecord(ro.ev[1], st);
    k_eig<<<grid, 256, 0, st>>>(alpha, S, so);
    if (ro.ev[2]) cudaEventRecord(ro.ev[2], st);
    if (ro.fixup) {
        k_fix_decide<<<(n + 255) / 256, 256, 0, st>>>(S, ro.knu_max);
        int fgrid = n < sms * 4 ? n : sms * 4;
        k_fix_solve<<<fgrid, 256, 0, st>>>(alpha, S, so);
    }
    if (ro.ev[3]) cudaEventRecord(ro.ev[3], st);
    k_place<<<(n + 255) / 256, 256, 0, st>>>(S);
    int vgrid = (n + 7) / 8;
    vgrid = vgrid < sms * 16 ? vgrid : sms * 16;
    k_vectors<<<vgrid, 256, 0, st>>>(n, d, z, alpha, S, out);
    if (ro.ev[4]) cudaEventRecord(ro.ev[4], st);
    return cudaGetLastError();
}

cudaError_t launch_debug_rcp(int n, const double *x, double *y, cudaStream_t st) {
    if (n > 0) k_debug_rcp<<<(n + 255) / 256, 256, 0, st>>>(n, x, y);
    return cudaGetLastError();
}

}  // namespace ae
