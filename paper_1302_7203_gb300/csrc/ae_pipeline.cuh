// ae_pipeline.cuh -- the per-instance and per-eigenpair bodies of the solver
// pipeline, shared by the single-instance kernels (ae_arrow.cu) and the
// batched, persistent ones (ae_batch.cu).  Each function states which threads
// call it: a whole CTA of 1024 threads (the *_block functions), one thread, one
// warp, or one team.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "ae_internal.h"
#include "ae_solver.cuh"

namespace ae {

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
static __device__ void reduce_block(int n1, const double *__restrict__ key,
                             const double *__restrict__ spk, const int *__restrict__ perm,
                             const Scratch &S) {
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
            dr = key[r];
            zr = spk[r];
            zero = (zr == 0.0);
            if (!zero) {
                head = true;   // the first nonzero row of its run of equal poles
                for (int q = s - 1; q >= 0; --q) {
                    const int rq = perm[q];
                    if (key[rq] != dr) break;
                    if (spk[rq] != 0.0) { head = false; break; }
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
                    if (key[rq] != dr) break;
                    acc = hypot(acc, spk[rq]);
                }
                S.pd[jk] = dr;
                S.pv[jk] = dr;
                S.pz[jk] = acc;
                const double a2 = acc * acc;
                S.pz2[jk] = a2;
                S.pz2lo[jk] = fma(acc, acc, -a2);
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
                        if (key[rq] != dr) break;
                        Rm1 = hypot(Rm1, spk[rq]);
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
}

// block reductions for the single-CTA post kernel (blockDim = 1024)
__device__ __forceinline__ double block_max(double v, double *sh) {
    v = warp_max(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = sh[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, sh[w]);
        sh[0] = r;
    }
    __syncthreads();
    return sh[0];
}

// (the warp partials are combined by thread 0 alone and broadcast: on the one
// SM a single-CTA kernel runs on, every redundant FP64 instruction counts)
__device__ __forceinline__ dd block_sum_dd(dd v, double *sh) {
    v = warp_sum_dd(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        sh[threadIdx.x >> 5] = v.hi;
        sh[32 + (threadIdx.x >> 5)] = v.lo;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        dd r = {sh[0], sh[32]};
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = dd_add(r, dd{sh[w], sh[32 + w]});
        sh[0] = r.hi;
        sh[32] = r.lo;
    }
    __syncthreads();
    return dd{sh[0], sh[32]};
}

__device__ __forceinline__ double block_sum(double v, double *sh) {
    v = warp_sum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = sh[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r += sh[w];
        sh[0] = r;
    }
    __syncthreads();
    return sh[0];
}

// Kind-specific arrowhead data after the reduction, then the FP32 copies
// (single CTA of 1024 threads).
template <Kind K>
__device__ void post_block(int n1, const double *__restrict__ d, const double *__restrict__ z,
                           const double *__restrict__ zrow, double alpha, double rho_abs,
                           const Scratch &S) {
    __shared__ double sh[64];
    int m = S.cnt[C_M];
    dd al = {alpha, 0.0};
    if (K == KIND_DPR1) {
        // Sec. 6.3: the reduced DPR1 poles p_0 > ... > p_{m-1} with weights u'_j;
        // the arrowhead L^{-1} M L has poles p_0..p_{m-2}, spikes
        // zeta_j = u'_j sqrt(rho (p_j - p_{m-1})) and corner p_{m-1} + rho u'^T u'
        // (after u <- sqrt(rho) u); zeta_j^2 and the corner in double-double.
        dd uu = {0.0, 0.0};
        for (int j = threadIdx.x; j < m; j += blockDim.x) uu = dd_add_same(uu, two_prod(S.pz[j], S.pz[j]));
        uu = block_sum_dd(uu, sh);
        const double plast = m > 0 ? S.pd[m - 1] : 0.0;
        __syncthreads();
        for (int j = threadIdx.x; j < m - 1; j += blockDim.x) {
            const dd z2 = dd_mul(dd_mul_d(two_prod(S.pz[j], S.pz[j]), rho_abs),
                                 two_sum(S.pd[j], -plast));
            S.pz2[j] = z2.hi;
            S.pz2lo[j] = z2.lo;
            S.pz[j] = dd_sqrt(z2).hi;
        }
        al = dd_add(dd{plast, 0.0}, dd_mul_d(uu, rho_abs));
        if (threadIdx.x == 0) {
            S.prm[P_PLAST] = plast;
            S.cnt[C_M] = m - 1;      // arrowhead poles; m - 1 = -1: nothing to solve
        }
        m = m - 1;
    } else if (K == KIND_TSVD) {
        // Sec. 6.2: B^T B has poles d_j^2, spikes d_j z_j, corner alpha^2 + z^T z
        // (the corner over all rows; runs of equal d keep their folded spike).
        dd zz = {0.0, 0.0};
        for (int r = threadIdx.x; r < n1; r += blockDim.x) zz = dd_add_same(zz, two_prod(z[r], z[r]));
        zz = block_sum_dd(zz, sh);
        al = dd_add(two_prod(alpha, alpha), zz);
        __syncthreads();
        for (int j = threadIdx.x; j < m; j += blockDim.x) {
            const double dj = S.pd[j];
            S.pv[j] = dj * dj;
            const int r = S.prow[j];
            // a single-row pole: (d_j z_j)^2 exactly in double-double
            const bool single = (j + 1 == m || S.pd[j + 1] != dj) &&
                                S.pz[j] == fabs(S.spk[r]);
            if (single) {
                const dd dz = two_prod(dj, z[r]);
                const dd z2 = dd_mul(dz, dz);
                S.pz2[j] = z2.hi;
                S.pz2lo[j] = z2.lo;
            }
        }
        const int nd = S.cnt[C_ND];
        for (int t = threadIdx.x; t < nd; t += blockDim.x) S.dval[t] = S.dval[t] * S.dval[t];
    } else if (K == KIND_HERM || K == KIND_NSYM) {
        // a single-row pole's spike^2 exactly in double-double: |zeta|^2 =
        // re^2 + im^2 (Sec. 6.1), resp. zc zr (its Remark), as the paper asks
        // for the moduli in doubled precision when b is computed so
        for (int j = threadIdx.x; j < m; j += blockDim.x) {
            const int r = S.prow[j];
            if (S.pz[j] != S.spk[r]) continue;      // another row was folded in
            const dd z2 = K == KIND_HERM
                              ? dd_add(two_prod(z[2 * r], z[2 * r]),
                                       two_prod(z[2 * r + 1], z[2 * r + 1]))
                              : two_prod(z[r], zrow[r]);
            S.pz2[j] = z2.hi;
            S.pz2lo[j] = z2.lo;
            S.pz[j] = dd_sqrt(z2).hi;
        }
    }
    if (threadIdx.x == 0) {
        S.prm[P_ALPHA_HI] = al.hi;
        S.prm[P_ALPHA_LO] = al.lo;
    }
    // Algorithm 5's spike ratio needs sum_j |zeta_j| over the reduced poles
    __syncthreads();
    double zsum = 0.0;
    for (int j = threadIdx.x; j < m; j += blockDim.x) zsum += S.pz[j];
    zsum = block_sum(zsum, sh);
    if (threadIdx.x == 0) S.prm[P_ZSUM] = zsum;
    // FP32 copies: keys and spike^2 scaled by powers of two so that the
    // largest of each is O(1)
    double mxd = 0.0, mxz = 0.0;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        mxd = fmax(mxd, fabs(S.pd[j]));
        mxz = fmax(mxz, S.pz2[j]);
    }
    mxd = block_max(mxd, sh);
    mxz = block_max(mxz, sh);
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
        S.prm[P_DS] = ds;
        S.prm[P_ZS] = zs;
    }
}

template <Kind K>
struct PolesOf;
template <>
struct PolesOf<KIND_ARROW> {
    using type = ArrowPoles;
    __device__ static ArrowPoles make(const Scratch &S, int m) {
        return {m,      S.pd,  S.pz,  S.pz2,          S.pz2lo,        S.prm[P_ALPHA_HI],
                S.prm[P_ALPHA_LO], S.pdh, S.pdl,      S.pz2f,         S.prm[P_DS],
                S.prm[P_ZS],       S.prm[P_ZSUM]};
    }
};
template <>
struct PolesOf<KIND_DPR1> : PolesOf<KIND_ARROW> {};
template <>
struct PolesOf<KIND_HERM> : PolesOf<KIND_ARROW> {};
template <>
struct PolesOf<KIND_NSYM> : PolesOf<KIND_ARROW> {};
template <>
struct PolesOf<KIND_TSVD> {
    using type = TsvdPoles;
    __device__ static TsvdPoles make(const Scratch &S, int m) {
        return {m,     S.pd,     S.pv,              S.pz,  S.pz2, S.pz2lo,
                S.prm[P_ALPHA_HI], S.prm[P_ALPHA_LO], S.pdh, S.pdl, S.pz2f,
                S.prm[P_DS],       S.prm[P_ZS],       S.prm[P_ZSUM]};
    }
};

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
    if (r.iters_d && !fix) atomicAdd(S.cnt64 + C64_DERIV, (unsigned long long)r.iters_d);
    if (fix) atomicAdd(S.cnt64 + C64_ITERS_FIX, (unsigned long long)r.iters);
    if (r.f32p) atomicAdd(S.cnt64 + C64_F32, (unsigned long long)r.f32p);
    if (r.dfp) atomicAdd(S.cnt64 + C64_DF, (unsigned long long)r.dfp);
    atomicMax(S.cnt + C_MAXIT, r.iters);
    if (r.flags & AE_FLAG_CAPPED) atomicAdd(S.cnt + C_CAPPED, 1);
    if (r.flags & AE_FLAG_FP32_FALLBACK) atomicAdd(S.cnt + C_FP32FB, 1);
    if (r.flags & AE_FLAG_DDB) atomicAdd(S.cnt + C_DDB, 1);
    if (r.flags & AE_FLAG_MID64) atomicAdd(S.cnt + C_MID64, 1);
    if (isfinite(r.Kb)) atomic_max_nonneg(S.cnt64 + C64_MAXKB, r.Kb);
}

// Eigenpair k of the reduced arrowhead by one team; the team's rank-0 thread
// stores the result.
template <Kind K, class Team>
__device__ __forceinline__ void eig_item(const typename PolesOf<K>::type &R, const Team &T,
                                         const Scratch &S, int k, const SolveOpts &o,
                                         double2 *buf = nullptr) {
    const int m = R.m;
    EigResult res;
    if (m == 0) {
        const double a = S.prm[P_ALPHA_HI];
        res = {a, S.prm[P_ALPHA_LO], a, NAN, 0.0, -1, 0, 0};
    } else {
        int i, side;
        bool ran32 = false;
        const bool mid64 = select_shift(R, T, k, i, side, o.precision == 1, &ran32);
        res = solve_shifted(R, T, i, side, o, buf);
        if (mid64) res.flags |= AE_FLAG_MID64;
        if (ran32) ++res.f32p;
    }
    if (T.rank == 0) {
        store_result(S, k, res);
        S.es_flags[k] = res.flags;
        S.es_Knu[k] = 1.0;
        record_stats(S, res);
    }
}

// Remedy decision for eigenpair k; returns the AE_FLAG_* remedy (0: none).
static __device__ int fix_decide_item(Kind kind, const Scratch &S, int k, double knu_max) {
    const int m = S.cnt[C_M];
    if (k > m || m <= 0) return 0;
    const double lam = S.es_lam[k], sig = S.es_sigma[k], mu = S.es_mu[k];
    const int i = S.es_pole[k];
    const double q = (fabs(sig) + fabs(mu)) / fabs(lam);
    int remedy = 0;
    double knu = 1.0;
    if (kind == KIND_DPR1 && k == m &&
        fabs(lam - S.prm[P_PLAST]) < fabs(mu)) {
        // DPR1: the last eigenvalue lies between the last arrowhead pole and
        // the DPR1's last pole p_last, which is not a pole of the arrowhead; when
        // it is nearer p_last, re-solve from (A - p_last I)^{-1} so that
        // lambda - p_last (and the vector's last component) keep relative accuracy.
        S.es_fixshift[k] = S.prm[P_PLAST];
        remedy = AE_FLAG_DPR1SHIFT;
    } else if (q > 3.0 && !(S.cnt[C_FLAGS] & CF_ZEROPOLE)) {
        // Theorem C1 bounds the quotient by 3 except in the special cases
        // (a)-(c); Remark 1 needs D nonsingular.
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
                const double po = S.pv[io];
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
                const double lo = k < m ? S.pv[k] : -INFINITY;
                const double hi = k > 0 ? S.pv[k - 1] : INFINITY;
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
        atomicAdd(S.cnt + (remedy == AE_FLAG_NEARZERO ? C_NEARZERO
                           : remedy == AE_FLAG_OTHERPOLE ? C_OTHERPOLE : C_DPR1), 1);
    }
    return remedy;
}

// Remedy solve of eigenpair k by a team (a CTA in the single-instance pipeline,
// a warp in the batched one); all of its threads call it.
// buf: the team's slice of stored pairs (or null).
// Returns whether the remedy's result was kept (buf then holds its stored pairs).
template <Kind K, class Team>
__device__ bool fix_solve_item(const typename PolesOf<K>::type &R, const Team &T, const Scratch &S,
                               int k, const SolveOpts &o, double2 *buf = nullptr) {
    const int m = S.cnt[C_M];
    const int f = S.es_flags[k];
    EigResult res;
    if (f & AE_FLAG_NEARZERO) {
        res = solve_dpr1_shift(R, T, 0.0, o, buf);
    } else if (f & AE_FLAG_OTHERPOLE) {
        const int io = S.es_fixpole[k];
        const int side = io < S.es_pole[k] ? -1 : +1;   // other pole above -> lambda below it
        res = solve_shifted(R, T, io, side, o, buf);
    } else {
        res = solve_dpr1_shift(R, T, S.es_fixshift[k], o, buf);
    }
    // the result must stay in the eigenvalue's interlacing interval
    const double lo = k < m ? R.pole(k) : (K == KIND_DPR1 ? S.prm[P_PLAST] : -INFINITY);
    const double hi = k > 0 ? R.pole(k - 1) : INFINITY;
    const bool ok = (res.lam >= lo && res.lam <= hi) && isfinite(res.lam);
    if (T.rank == 0) {
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
    return ok;
}

// The items a solve writes: all of them, or one part of a split solve --
// computed eigenpairs [k0, k1) and the deflated rows [u0, u1) whose values
// lie in [p_{k1-1}, p_{k0-1}), which together hold the output positions
// [pos0, pos0 + (k1 - k0) + (u1 - u0)) of the whole decomposition.
struct PartRange {
    int k0, k1, u0, u1, pos0;
};

__device__ __forceinline__ PartRange part_range(const Scratch &S) {
    if (!S.cnt[C_PART]) return {0, S.cnt[C_M] + 1, 0, S.cnt[C_ND], 0};
    return {S.cnt[C_K0], S.cnt[C_K1], S.cnt[C_U0], S.cnt[C_U1], S.cnt[C_POS0]};
}

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

// output position of item t (computed eigenpairs first, then deflated rows).
// A deflated row's value v lies in its part's interval [p_{k1-1}, p_{k0-1}),
// so every computed eigenvalue before k0 exceeds it and none from k1 on does:
// only the part's own eigenvalues need comparing.
static __device__ void place_item(const Scratch &S, int t) {
    const int m = S.cnt[C_M], nd = S.cnt[C_ND];
    const int ncomp = m + 1;
    if (t < ncomp) {
        S.pos[t] = nd ? t + count_ge(S.dval, nd, S.es_lam[t], false) : t;
    } else if (t < ncomp + nd) {
        const int u = t - ncomp;
        const PartRange P = part_range(S);
        S.pos[t] = u + P.k0 + count_ge(S.es_lam + P.k0, P.k1 - P.k0, S.dval[u], true);
    }
}

// Helmert-type vector of a run-folded row:
// (-s_q sum_{l<m} s_l e_l + R_{m-1}^2 e_q) / (R_{m-1} R_m) with the run's spikes s
template <int STRIDE = 32>
__device__ __forceinline__ void run_column(const Scratch &S, const double *spk, int row, int lane,
                                           double *col, double sign) {
    const double Rm1 = S.run_R[2 * row], Rm = S.run_R[2 * row + 1];
    const double zq = spk[row];
    const double den = Rm1 * Rm;
    const int s0 = S.run_s0[row], s1 = S.spos[row];
    for (int s = s0 + lane; s < s1; s += STRIDE) {
        const int rq = S.perm[s];
        const double zl = spk[rq];
        if (zl != 0.0) col[rq] = sign * (-(zq * zl) / den);
    }
    if (lane == 0) col[row] = sign * (Rm1 / Rm);
}

// Output of item `item` (a computed eigenpair, or a deflated row) by one team:
// value, optional shift/mu/diagnostics, and its column(s).  `key`/`spk` are the
// transformed inputs the reduction saw; z is the caller's spike array (SVD:
// for the left vectors; HERM: the complex spikes; NSYM: the column spikes,
// zrow the row spikes).
// HERM writes U = Phi V (Sec. 6.1) as complex columns, row r at doubles 2r,
// 2r+1: u_r = zeta_r t_r / ||x|| with t_r = 1/((d_r - sigma) - mu), since
// Phi_r |zeta_r| = zeta_r.  NSYM writes the right vectors X = Psi V into V and
// the left ones Y = Psi^{-1} V into U: x_r = zc_r t_r / ||x||, y_r = zr_r t_r
// / ||x||, since Psi_r sqrt(zc_r zr_r) = zc_r; then y^T x = 1.
// stage: null (pass 1 keeps its values in the output column) or the team's
// scratch for RS * n1 doubles (the column is then written once, normalised --
// what an output in host memory needs).  columns = false writes the scalar
// outputs only.  pairs: stage is the team's stored-pair slice and still holds
// the (delta_j, zeta_j^2 / delta_j) of this item's final solve.
template <Kind K, class Team>
__device__ void vector_item(int n, int n1, const double *__restrict__ key,
                            const double *__restrict__ spk, const double *__restrict__ z,
                            const double *__restrict__ zrow, double alpha, double sgn,
                            const Scratch &S, const Outputs &out, int item, const Team &T,
                            double *stage = nullptr, bool columns = true,
                            bool pairs = false) {
    const int lane = T.rank;
    constexpr bool CPLX = K == KIND_HERM;
    constexpr bool TWO = K == KIND_NSYM;
    constexpr int RS = CPLX ? 2 : 1;           // doubles per row
    const int m = S.cnt[C_M];
    const int ncomp = m + 1;
    const bool last_row = K != KIND_DPR1;     // arrowhead rows have the x_n = -1 entry
    int pos = S.pos[item] - (S.cnt[C_PART] ? S.cnt[C_POS0] : 0);   // in this part's block
    if (K == KIND_DPR1 && sgn < 0.0) pos = n - 1 - pos;   // -M's order reversed
    double *col = (out.V && columns) ? out.V + (size_t)pos * out.ldv : nullptr;
    double *ucol = ((K == KIND_TSVD || TWO) && out.U && columns) ? out.U + (size_t)pos * out.ldu
                                                                   : nullptr;
    if (item < ncomp) {
        const int k = item;
        const double sig = S.es_sigma[k], mu = S.es_mu[k];
        const int pi = S.es_pole[k];
        double value = S.es_lam[k];
        double sv = 0.0;   // SVD: singular value
        if (K == KIND_TSVD) {
            // lambda = d_i^2 + mu (pole shift) or sigma + mu, in double-double
            dd l2;
            if (pi >= 0) {
                const double di = S.pd[pi];
                l2 = dd_add(two_prod(di, di), dd{mu, 0.0});
            } else {
                l2 = two_sum(sig, mu);
            }
            sv = dd_sqrt(l2).hi;
            value = sv;
        } else if (K == KIND_DPR1) {
            value = sgn * value;
        }
        if (lane == 0) {
            out.lambda[pos] = value;
            if (out.shift) out.shift[pos] = K == KIND_DPR1 ? sgn * sig : sig;
            if (out.mu) out.mu[pos] = K == KIND_DPR1 ? sgn * mu : mu;
            if (out.dg_b) out.dg_b[pos] = S.es_b[k];
            if (out.dg_Kb) out.dg_Kb[pos] = S.es_Kb[k];
            if (out.dg_Knu) out.dg_Knu[pos] = S.es_Knu[k];
            if (out.dg_iters) out.dg_iters[pos] = S.es_iters[k];
            if (out.dg_flags) out.dg_flags[pos] = S.es_flags[k];
        }
        if (!col) return;
        // 1/(shifted difference of row r - mu); 0 for a zero spike
        const double unit = unit_reg();
        auto recip = [&](int r) {
            if (spk[r] == 0.0) return 0.0;
            double del;
            if (K == KIND_TSVD) {
                const double dr = key[r];
                if (pi >= 0) {
                    const double di = S.pd[pi];
                    del = (dr - di) * (dr + di);
                } else {
                    del = fma(dr, dr, -sig);
                }
            } else {
                del = key[r] - sig;
            }
            return rcp_o(del - mu, unit);
        };
        // component of row r of x = [(D - lambda I)^{-1} spikes; -1]
        auto comp = [&](int r) { return spk[r] * recip(r); };
        // Pass 1 stores x (HERM, NSYM: the reciprocal t) in the column and sums
        // x^2 in sorted order (so the norm does not depend on the order of the
        // input rows); pass 2 scales in place.
        double *keep = stage ? stage : col;      // pass-1 values, RS doubles a row
        // two rows a lane at a time, two independent sums (the same order for
        // every kind, so that real spikes give the real solver's bits)
        auto one = [&](int r, double &acc) {
            if (CPLX || TWO) {
                const double t = recip(r);
                keep[RS * r] = t;
                const double x = spk[r] * t;
                acc = fma(x, x, acc);
            } else {
                const double x = comp(r);
                keep[r] = x;
                acc = fma(x, x, acc);
            }
        };
        double s = 0.0, s1 = 0.0;
        // Sorted input without deflation: row r is reduced pole r, and its
        // shifted difference d_r - sigma is the one the solve stored (0 for
        // the shift pole): the same double, loaded instead of recomputed.  The
        // staged values overwrite the stored pairs of rows up to r (a slot per
        // row, 2 per pair; the complex stage overwrites row r's own), so each
        // step's loads come before the team syncs and its stores after.
        const bool fast = pairs && stage && (K == KIND_ARROW || CPLX || TWO) && m == n1 &&
                          !(S.cnt[C_FLAGS] & CF_UNSORTED);
        if (fast) {
            const double2 *P = reinterpret_cast<const double2 *>(stage);
            auto one_d = [&](int r, double del, double &acc) {
                const double t = rcp_o(del - mu, unit);
                const double x = spk[r] * t;
                keep[RS * r] = (CPLX || TWO) ? t : x;
                acc = fma(x, x, acc);
            };
            for (int base = 0; base < n1; base += 2 * Team::size) {
                const int ra = base + lane, rb = ra + Team::size;
                const double da = ra < n1 ? P[ra].x : 0.0;
                const double db = rb < n1 ? P[rb].x : 0.0;
                T.sync();
                if (ra < n1) one_d(ra, da, s);
                if (rb < n1) one_d(rb, db, s1);
            }
        } else {
            int q0 = lane;
            for (; q0 + Team::size < n1; q0 += 2 * Team::size) {
                one(S.perm[q0], s);
                one(S.perm[q0 + Team::size], s1);
            }
            if (q0 < n1) one(S.perm[q0], s);
        }
        s += s1;
        s = T.sum(s) + (last_row ? 1.0 : 0.0);
        double inv, scale = 1.0;
        bool stored = true;
        if (isfinite(s) && s > 0x1p-960) {
            inv = 1.0 / sqrt(s);
        } else {
            // rescale by the largest component to avoid overflow/underflow
            stored = false;
            double xm = last_row ? 1.0 : 0.0;
            for (int r = lane; r < n1; r += Team::size) xm = fmax(xm, fabs(comp(r)));
            xm = T.max(xm);
            scale = 1.0 / xm;
            double s2 = 0.0;
            for (int q = lane; q < n1; q += Team::size) {
                const double x = comp(S.perm[q]) * scale;
                s2 = fma(x, x, s2);
            }
            s2 = T.sum(s2) + (last_row ? scale * scale : 0.0);
            inv = 1.0 / sqrt(s2);
        }
        // DPR1 with rho < 0 solved -M: q ~ (D - lambda)^{-1} u needs a sign flip
        const double vs = (K == KIND_DPR1 && sgn < 0.0) ? -1.0 : 1.0;
        T.sync();
        int r0 = lane;
        if (stored && !CPLX && !TWO) {
            // the common case, four rows a lane at a time so that four loads of
            // the pass-1 values are in flight (vs = +-1, so x (vs inv) is
            // bitwise vs x inv)
            const double f = vs * inv;
            constexpr int ST = Team::size;
            for (; r0 + 3 * ST < n1; r0 += 4 * ST) {
                const double x0 = keep[r0], x1 = keep[r0 + ST], x2 = keep[r0 + 2 * ST],
                             x3 = keep[r0 + 3 * ST];
                const double v0 = x0 * f, v1 = x1 * f, v2 = x2 * f, v3 = x3 * f;
                col[r0] = v0;
                col[r0 + ST] = v1;
                col[r0 + 2 * ST] = v2;
                col[r0 + 3 * ST] = v3;
                if (ucol) {
                    ucol[r0] = sv * v0 / key[r0];
                    ucol[r0 + ST] = sv * v1 / key[r0 + ST];
                    ucol[r0 + 2 * ST] = sv * v2 / key[r0 + 2 * ST];
                    ucol[r0 + 3 * ST] = sv * v3 / key[r0 + 3 * ST];
                }
            }
        }
        for (int r = r0; r < n1; r += Team::size) {
            if (CPLX) {
                const double t = (stored ? keep[2 * r] : recip(r) * scale) * inv;
                col[2 * r] = z[2 * r] * t;
                col[2 * r + 1] = z[2 * r + 1] * t;
            } else if (TWO) {
                const double t = (stored ? keep[r] : recip(r) * scale) * inv;
                col[r] = z[r] * t;
                if (ucol) ucol[r] = zrow[r] * t;
            } else {
                const double x = stored ? keep[r] : comp(r) * scale;
                const double v = vs * x * inv;
                col[r] = v;
                if (ucol) ucol[r] = sv * v / key[r];      // u_j = s v_j / d_j
            }
        }
        if (last_row && lane == 0) {
            const double vn = -scale * inv;
            col[RS * n1] = vn;
            if (CPLX) col[RS * n1 + 1] = 0.0;
            if (ucol) ucol[n1] = K == KIND_TSVD ? alpha * vn / sv : vn;   // SVD: u_n = alpha v_n / s
        }
    } else {
        const int u = item - ncomp;
        const int row = S.drow[u];
        const double kv = key[row];
        const double value = K == KIND_TSVD ? kv : (K == KIND_DPR1 ? sgn * kv : kv);
        if (lane == 0) {
            out.lambda[pos] = value;
            if (out.shift) out.shift[pos] = value;
            if (out.mu) out.mu[pos] = 0.0;
            if (out.dg_b) out.dg_b[pos] = NAN;
            if (out.dg_Kb) out.dg_Kb[pos] = 0.0;
            if (out.dg_Knu) out.dg_Knu[pos] = 1.0;
            if (out.dg_iters) out.dg_iters[pos] = 0;
            if (out.dg_flags) out.dg_flags[pos] = AE_FLAG_DEFLATED;
        }
        if (!col) return;
        for (int r = lane; r < RS * n; r += Team::size) col[r] = 0.0;
        if (TWO && ucol)
            for (int r = lane; r < n; r += Team::size) ucol[r] = 0.0;
        T.sync();
        if (S.kind[row] == 1) {
            if (lane == 0) {
                col[RS * row] = 1.0;
                if (TWO && ucol) ucol[row] = 1.0;
            }
        } else if (CPLX || TWO) {
            // Phi (resp. Psi, Psi^{-1}) times the real Helmert-type vector of
            // the moduli: rows l before `row` in its run get -|zeta_q| s_l /
            // (R_{m-1} R_m), the row itself (s_q / |zeta_q|) R_{m-1} / R_m, with
            // s the caller's spike (zeta, zc or zr)
            const double Rm1 = S.run_R[2 * row], Rm = S.run_R[2 * row + 1];
            const double zq = spk[row];
            const double f = -zq / (Rm1 * Rm);
            const int s0 = S.run_s0[row], s1 = S.spos[row];
            for (int q = s0 + lane; q < s1; q += Team::size) {
                const int rq = S.perm[q];
                if (spk[rq] == 0.0) continue;
                if (CPLX) {
                    col[2 * rq] = f * z[2 * rq];
                    col[2 * rq + 1] = f * z[2 * rq + 1];
                } else {
                    col[rq] = f * z[rq];
                    if (ucol) ucol[rq] = f * zrow[rq];
                }
            }
            if (lane == 0) {
                const double g = Rm1 / (Rm * zq);
                if (CPLX) {
                    col[2 * row] = g * z[2 * row];
                    col[2 * row + 1] = g * z[2 * row + 1];
                } else {
                    col[row] = g * z[row];
                    if (ucol) ucol[row] = g * zrow[row];
                }
            }
        } else {
            run_column<Team::size>(S, spk, row, lane, col, 1.0);
        }
        if (K == KIND_TSVD && ucol) {
            // B v = d_r v for a deflated right vector (its last entry is 0)
            T.sync();
            for (int r = lane; r < n; r += Team::size) ucol[r] = col[r];
        }
    }
}

}  // namespace ae
