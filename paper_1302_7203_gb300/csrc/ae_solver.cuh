// ae_solver.cuh -- one eigenpair per team (a warp, or a CTA of NW warps):
// shift selection (Algorithm 1; its midpoint test optionally in FP32 with an
// error bound), the inverse of the shifted arrowhead with its element b in
// double-double or, under Algorithm 5's gate, in standard precision
// (Algorithm 2, Eq. invAi / b_ob, Theorem 6), the inverse's extreme eigenvalue
// by bisection (Algorithm 3, optionally opened by an FP32 bracket) or by the
// bracketed Newton finish on the same function (optionally opened by FP32 and
// double-float model steps, closed by the local expansion of an FP64
// evaluation), and the Remark 1 / Remark 2(b) solve on the DPR1 inverse
// (A - sigma I)^{-1}.
//
// Notation (0-based): reduced poles p_0 > p_1 > ... > p_{m-1}, spikes
// zeta_j > 0, corner alpha; eigenvalue k (k = 0..m) lies in (p_k, p_{k-1}).
// With the shift sigma = p_i and delta_j = p_j - p_i, the inverse of the
// shifted matrix is the arrowhead (Eq. invAi)
//     diag(1/delta_j (j != i), 0),  spikes w_j = -zeta_j / (delta_j zeta_i),
//     w_zeta = 1/zeta_i,  corner b = (-a + sum_{j!=i} zeta_j^2/delta_j)/zeta_i^2.
// Its Pick function (Eq. Pick applied to it) is
//     F(x) = b - x - sum_{j!=i} w_j^2/(1/delta_j - x) - w_zeta^2/(0 - x).
// Each term is evaluated as w_j^2/(1/delta_j - x) = c zeta_j^2 / (delta_j (1 - x delta_j)),
// c = 1/zeta_i^2: the same value, with the same O(eps) relative error per
// term, but without materialising 1/delta_j and w_j (which would need O(n)
// storage per eigenpair).  So F(x) = (b - x) - c (S(x) - 1/x) with
//     S(x) = sum_{j!=i} zeta_j^2 / (delta_j (1 - x delta_j)).
// All terms of S(x) - 1/x have one sign on the side being searched, so the only
// cancellation is the final one, exactly as in the paper's evaluation.
//
// Every reduction has a fixed order, so a solve is bit-reproducible for a
// given team shape.
#pragma once
#include "ae_device.cuh"

namespace ae {

struct SolveOpts {
    int max_iter;
    int precision;
    int finish;     // 0: bisection (Algorithm 3); 1: bracketed Newton
    int bgate;      // 0: b always double-double; 1: Algorithm 5's gates
    double kb_max;  // the gate's "K_b >> 1" threshold
};

struct EigResult {
    double sigma;   // shift value (a pole, or a non-pole shift for remedies)
    double mu;      // lambda = sigma + mu
    double lam;
    double b;       // element b of the shifted inverse (NaN for DPR1 solves)
    double Kb;      // K_b of Eq. (K2)
    int pole;       // reduced pole index of the shift, -1 if none
    int iters;      // FP64 evaluations (bisection steps or Newton evaluations)
    int flags;
    int iters_d;    // of those, Newton evaluations that also formed F'
    int f32p;       // O(n) passes in FP32 (midpoint test, model steps, bracket)
    int dfp;        // O(n) passes in double-float (model steps)
};

// ---------------------------------------------------------------------------
// teams
// ---------------------------------------------------------------------------
struct WarpTeam {
    int rank;                       // lane
    static constexpr int size = 32;
    __device__ __forceinline__ double sum(double v) const { return warp_sum(v); }
    __device__ __forceinline__ float sumf(float v) const {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
        return v;
    }
    __device__ __forceinline__ dd sum(dd v) const { return warp_sum_dd(v); }
    __device__ __forceinline__ double max(double v) const { return warp_max(v); }
    __device__ __forceinline__ double min(double v) const { return warp_min(v); }
    __device__ __forceinline__ void sync() const { __syncwarp(); }
};

// NW consecutive warps of a CTA (the whole CTA when NW warps are all of it);
// `red` points at 2*NW doubles of shared memory of this team alone, and the
// team synchronises on its own named barrier `bar` (0: the CTA's barrier,
// which then must be the whole CTA), so several teams can share a CTA.
template <int NW>
struct CtaTeam {
    int rank;                       // thread index within the team
    double *red;
    int bar = 0;
    static constexpr int size = 32 * NW;
    __device__ __forceinline__ void bsync() const {
        asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(size) : "memory");
    }
    __device__ __forceinline__ double sum(double v) const {
        v = warp_sum(v);
        bsync();
        if ((rank & 31) == 0) red[rank >> 5] = v;
        bsync();
        double r = red[0];
#pragma unroll
        for (int w = 1; w < NW; ++w) r += red[w];
        return r;
    }
    // (sum() reduces within the warp itself: pass the per-thread value)
    __device__ __forceinline__ float sumf(float v) const { return (float)sum((double)v); }
    __device__ __forceinline__ dd sum(dd v) const {
        v = warp_sum_dd(v);
        bsync();
        if ((rank & 31) == 0) {
            red[rank >> 5] = v.hi;
            red[NW + (rank >> 5)] = v.lo;
        }
        bsync();
        dd r = {red[0], red[NW]};
#pragma unroll
        for (int w = 1; w < NW; ++w) r = dd_add(r, dd{red[w], red[NW + w]});
        return r;
    }
    __device__ __forceinline__ double max(double v) const {
        v = warp_max(v);
        bsync();
        if ((rank & 31) == 0) red[rank >> 5] = v;
        bsync();
        double r = red[0];
#pragma unroll
        for (int w = 1; w < NW; ++w) r = fmax(r, red[w]);
        return r;
    }
    __device__ __forceinline__ double min(double v) const {
        v = warp_min(v);
        bsync();
        if ((rank & 31) == 0) red[rank >> 5] = v;
        bsync();
        double r = red[0];
#pragma unroll
        for (int w = 1; w < NW; ++w) r = fmin(r, red[w]);
        return r;
    }
    __device__ __forceinline__ void sync() const { bsync(); }
};

// ---------------------------------------------------------------------------
// poles and spikes of a reduced arrowhead held in device memory
// ---------------------------------------------------------------------------
struct ArrowPoles {
    int m;
    const double *__restrict__ pd;   // poles, strictly decreasing
    const double *__restrict__ pz;   // zeta_j > 0
    const double *__restrict__ pz2;  // zeta_j^2 = pz2 + pz2lo
    const double *__restrict__ pz2lo;
    double alpha, alpha_lo;          // corner (double-double)
    // FP32 copies for the opening bracket: poles split hi + lo after scaling
    // by ds, and zeta^2 scaled by zs (ds, zs powers of two); null when absent
    const float *__restrict__ pdh;
    const float *__restrict__ pdl;
    const float *__restrict__ pz2f;
    double ds, zs;
    double zsum;                     // sum of zeta_j (Algorithm 5's spike ratio)

    __device__ __forceinline__ double pole(int j) const { return __ldg(pd + j); }
    // p_j - shift in double; `i` is the shift's pole index (-1: not a pole)
    __device__ __forceinline__ double shifted(int j, double shift, int) const {
        return __ldg(pd + j) - shift;
    }
    __device__ __forceinline__ dd shifted_dd(int j, double shift, int) const {
        return two_sum_ord(__ldg(pd + j), -shift);
    }
    __device__ __forceinline__ double z2(int j) const { return __ldg(pz2 + j); }
    __device__ __forceinline__ double zabs(int j) const { return __ldg(pz + j); }
    __device__ __forceinline__ dd z2_dd(int j) const { return {__ldg(pz2 + j), __ldg(pz2lo + j)}; }
    // a = alpha - shift, exact for a double alpha
    __device__ __forceinline__ dd a_dd(double shift, int) const {
        return dd_add(two_sum(alpha, -shift), dd{alpha_lo, 0.0});
    }
    // FP32: the shift split hi + lo after scaling, and the scaled difference
    __device__ __forceinline__ void f32_shift(double shift, int, float &sh, float &sl) const {
        const double ss = shift * ds;
        sh = (float)ss;
        sl = (float)(ss - (double)sh);
    }
    __device__ __forceinline__ float shifted_f32(int j, float sh, float sl) const {
        return (__ldg(pdh + j) - sh) + (__ldg(pdl + j) - sl);
    }
    // the same, and a magnitude g with |error| <= 2 u |result| + 2^-45 g + 2^-147
    // (u = 2^-24; the hi + lo splits are exact to 2^-48 relative)
    __device__ __forceinline__ float shifted_f32_mag(int j, float sh, float sl, float &g) const {
        const float h = __ldg(pdh + j);
        g = fabsf(h) + fabsf(sh);
        return (h - sh) + (__ldg(pdl + j) - sl);
    }
    __device__ __forceinline__ double f32_scale() const { return ds; }
    __device__ __forceinline__ float z2f(int j) const { return __ldg(pz2f + j); }
    __device__ __forceinline__ bool has_f32() const { return pdh != nullptr; }
};

// The arrowhead B^T B of the triangular arrowhead B = [D z; 0 alpha] (Sec. 6.2):
// poles d_j^2, spikes d_j z_j, corner alpha^2 + z^T z.  Shifted differences to
// a pole use the paper's (d_j - d_i)(d_j + d_i); to any other shift, one fused
// d_j d_j - shift.
struct TsvdPoles {
    int m;
    const double *__restrict__ pd;   // d_j > 0, strictly decreasing
    const double *__restrict__ pv;   // fl(d_j^2)
    const double *__restrict__ pz;   // |d_j z_j|
    const double *__restrict__ pz2;  // (d_j z_j)^2 = pz2 + pz2lo
    const double *__restrict__ pz2lo;
    double alpha, alpha_lo;          // alpha^2 + z^T z (double-double)
    const float *__restrict__ pdh;   // d_j * ds split hi + lo
    const float *__restrict__ pdl;
    const float *__restrict__ pz2f;
    double ds, zs;
    double zsum;                     // sum of |d_j z_j|

    __device__ __forceinline__ double pole(int j) const { return __ldg(pv + j); }
    __device__ __forceinline__ double shifted(int j, double shift, int i) const {
        const double dj = __ldg(pd + j);
        if (i >= 0) {
            const double di = __ldg(pd + i);
            return (dj - di) * (dj + di);
        }
        return fma(dj, dj, -shift);
    }
    __device__ __forceinline__ dd shifted_dd(int j, double shift, int i) const {
        const double dj = __ldg(pd + j);
        if (i >= 0) {
            const double di = __ldg(pd + i);
            return dd_mul(two_sum_ord(dj, -di), two_sum_ord(dj, di));
        }
        return dd_add(two_prod(dj, dj), dd{-shift, 0.0});
    }
    __device__ __forceinline__ double z2(int j) const { return __ldg(pz2 + j); }
    __device__ __forceinline__ double zabs(int j) const { return __ldg(pz + j); }
    __device__ __forceinline__ dd z2_dd(int j) const { return {__ldg(pz2 + j), __ldg(pz2lo + j)}; }
    __device__ __forceinline__ dd a_dd(double shift, int i) const {
        const dd al = {alpha, alpha_lo};
        if (i >= 0) {
            const double di = __ldg(pd + i);
            return dd_add(al, dd_neg(two_prod(di, di)));
        }
        return dd_add(al, dd{-shift, 0.0});
    }
    // FP32 only for pole shifts: split d_i; differences (d_j - d_i)(d_j + d_i) ds^2
    __device__ __forceinline__ void f32_shift(double, int i, float &sh, float &sl) const {
        const double ss = __ldg(pd + (i >= 0 ? i : 0)) * ds;
        sh = (float)ss;
        sl = (float)(ss - (double)sh);
    }
    __device__ __forceinline__ float shifted_f32(int j, float sh, float sl) const {
        const float h = __ldg(pdh + j), l = __ldg(pdl + j);
        return ((h - sh) + (l - sl)) * ((h + sh) + (l + sl));
    }
    // with g = (d_j + d_i)^2 (scaled): |error| <= 6 u |result| + 2^-44 g + 2^-145
    __device__ __forceinline__ float shifted_f32_mag(int j, float sh, float sl, float &g) const {
        const float h = __ldg(pdh + j), l = __ldg(pdl + j);
        const float s = (h + sh) + (l + sl);
        g = s * s;
        return ((h - sh) + (l - sl)) * s;
    }
    __device__ __forceinline__ double f32_scale() const { return ds * ds; }
    __device__ __forceinline__ float z2f(int j) const { return __ldg(pz2f + j); }
    __device__ __forceinline__ bool has_f32() const { return pdh != nullptr; }
};

__device__ __forceinline__ float rcp_f32(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// v 2^k as an unevaluated float pair hi + lo with |v 2^k - hi - lo| <= 2^-46 |v 2^k|,
// formed by integer operations on v's bits (no FP64 instruction): hi takes the
// top 24 bits of the significand (truncated), lo the next 23.  A scaled
// exponent below -100 gives 0, one above 100 gives +-2^100 (callers use this
// only where such terms are negligible).
__device__ __forceinline__ void split_df(double v, int k, float &hi, float &lo) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned bh = (unsigned)(b >> 32), bl = (unsigned)b;
    const unsigned sgn = bh & 0x80000000u;
    const int e = (int)((bh >> 20) & 0x7ffu) - 1023 + k;
    if (e < -100) {
        hi = 0.f;
        lo = 0.f;
    } else if (e > 100) {
        hi = __uint_as_float(sgn | (227u << 23));
        lo = 0.f;
    } else {
        hi = __uint_as_float(sgn | ((unsigned)(e + 127) << 23) | ((bh & 0xfffffu) << 3) |
                             (bl >> 29));
        const unsigned eb = sgn | ((unsigned)(e + 104) << 23);   // 2^(e - 23)
        lo = __uint_as_float(eb | ((bl >> 6) & 0x7fffffu)) - __uint_as_float(eb);
    }
}

// ---------------------------------------------------------------------------
// O(n) passes
// ---------------------------------------------------------------------------
// S(x) = sum_{j != skip} zeta_j^2 / (delta_j (1 - x delta_j)), delta_j = p_j - shift
template <class P, class Team>
__device__ __forceinline__ double secular_sum(const P &R, const Team &T, double shift, int skip,
                                              double x) {
    double acc0 = 0.0, acc1 = 0.0;
    const double one = unit_reg();
    int j = T.rank;
    for (; j + Team::size < R.m; j += 2 * Team::size) {
        if (j != skip) {
            const double dj = R.shifted(j, shift, skip);
            const double t = fma(-x, dj, one);
            acc0 = fma(R.z2(j), rcp_o(dj * t, one), acc0);
        }
        const int j2 = j + Team::size;
        if (j2 != skip) {
            const double dj = R.shifted(j2, shift, skip);
            const double t = fma(-x, dj, one);
            acc1 = fma(R.z2(j2), rcp_o(dj * t, one), acc1);
        }
    }
    if (j < R.m && j != skip) {
        const double dj = R.shifted(j, shift, skip);
        const double t = fma(-x, dj, one);
        acc0 = fma(R.z2(j), rcp_o(dj * t, one), acc0);
    }
    return T.sum(acc0 + acc1);
}

// The same S(x) from per-eigenpair stored (delta_j, c_j = zeta_j^2 / delta_j):
// S(x) = sum_j c_j / (1 - x delta_j); the shift's own slot holds (0, 0).  The
// buffer is written by the same threads earlier in the solve (plain loads).
template <class Team>
__device__ __forceinline__ double secular_sum_stored(const double2 *buf, int m, const Team &T,
                                                     double x) {
    double acc0 = 0.0, acc1 = 0.0;
    const double one = unit_reg();
    int j = T.rank;
    for (; j + Team::size < m; j += 2 * Team::size) {
        const double2 a = buf[j];
        const double2 b = buf[j + Team::size];
        acc0 = fma(a.y, rcp_o(fma(-x, a.x, one), one), acc0);
        acc1 = fma(b.y, rcp_o(fma(-x, b.x, one), one), acc1);
    }
    if (j < m) {
        const double2 a = buf[j];
        acc0 = fma(a.y, rcp_o(fma(-x, a.x, one), one), acc0);
    }
    return T.sum(acc0 + acc1);
}

// S(x) and S'(x) = sum_{j != skip} zeta_j^2 / (1 - x delta_j)^2 together, for the
// Newton finish.  Stored pairs: with r_j = 1/(1 - x delta_j) and q_j = c_j r_j,
// S = sum q_j and S' = sum q_j (delta_j r_j), since c_j delta_j = zeta_j^2.
template <class Team>
__device__ __forceinline__ double2 secular_sum_d_stored(const double2 *buf, int m,
                                                        const Team &T, double x) {
    double s0 = 0.0, s1 = 0.0, d0 = 0.0, d1 = 0.0;
    const double one = unit_reg();
    int j = T.rank;
    for (; j + Team::size < m; j += 2 * Team::size) {
        const double2 a = buf[j];
        const double2 b = buf[j + Team::size];
        const double ra = rcp_o(fma(-x, a.x, one), one);
        const double rb = rcp_o(fma(-x, b.x, one), one);
        const double qa = a.y * ra, qb = b.y * rb;
        s0 += qa;
        s1 += qb;
        d0 = fma(qa, a.x * ra, d0);
        d1 = fma(qb, b.x * rb, d1);
    }
    if (j < m) {
        const double2 a = buf[j];
        const double ra = rcp_o(fma(-x, a.x, one), one);
        const double qa = a.y * ra;
        s0 += qa;
        d0 = fma(qa, a.x * ra, d0);
    }
    return make_double2(T.sum(s0 + s1), T.sum(d0 + d1));
}

// S(x) in double-float and S'(x) in compensated FP32 from the stored pairs:
// the trial point that opens the Newton finish (no FP64 instruction per
// term).  Scaled so that x 2^-kx lies in [1, 2) (delta_j 2^kx, leaving
// x delta_j unchanged) and c_j 2^-kc <= 2.  Each term: t = 1 - x delta_j
// (exact product and TwoSum), r = 1/t (FP32 seed and one correction), q = c_j r
// (relative error ~2^-44), added to a Neumaier sum; S' adds q (delta_j r), all
// of one sign, with Kahan compensation (relative error below 2^-20).  Terms
// whose scaled delta_j or c_j falls outside 2^+-100 contribute below 2^-99
// each to either sum (near the zero |x delta_j r_j| <= 2).  Returns (S, S')
// unscaled; `ok` is false when a result is not finite or either scaled sum is
// below (m + 1) 2^-78, where those contributions could exceed 2^-21 of it.
// one term of secular_sum_df_stored, added to (sh + sl) and (dh - dc)
__device__ __forceinline__ void df_term(double2 a, float xh, float xl, int kx, int kc, float &sh,
                                        float &sl, float &dh, float &dc) {
    float Dh, Dl, ch, cl;
    split_df(a.x, kx, Dh, Dl);
    split_df(a.y, -kc, ch, cl);
    // t = 1 - x D = (1 - ph) - pl, ph + pl = x D
    const float ph = xh * Dh;
    const float pl = fmaf(xh, Dl, fmaf(xl, Dh, fmaf(xh, Dh, -ph)));
    const float s1 = 1.f - ph;
    const float bb = s1 - 1.f;
    const float th = s1;
    const float tl = ((1.f - (s1 - bb)) + (-ph - bb)) - pl;
    // r = 1/t
    const float r0 = rcp_f32(th);
    const float e = fmaf(-tl, r0, fmaf(-th, r0, 1.f));
    const float rh = fmaf(r0, e, r0);
    const float rl = fmaf(r0, e, r0 - rh);
    // q = c r
    const float qh = ch * rh;
    const float ql = fmaf(ch, rl, fmaf(cl, rh, fmaf(ch, rh, -qh)));
    // S += q (Neumaier)
    const float u = sh + qh;
    sl += (fabsf(sh) >= fabsf(qh) ? (sh - u) + qh : (qh - u) + sh) + ql;
    sh = u;
    // S' += q D r (Kahan)
    const float y = fmaf(qh, Dh * rh, -dc);
    const float w = dh + y;
    dc = (w - dh) - y;
    dh = w;
}

template <class Team>
__device__ __forceinline__ double2 secular_sum_df_stored(const double2 *buf, int m,
                                                         const Team &T, double x, int kx,
                                                         int kc, bool &ok) {
    const double xs = ldexp(x, -kx);
    const float xh = (float)xs;
    const float xl = (float)(xs - (double)xh);
    float sh0 = 0.f, sl0 = 0.f, dh0 = 0.f, dc0 = 0.f;
    float sh1 = 0.f, sl1 = 0.f, dh1 = 0.f, dc1 = 0.f;
    int j = T.rank;
    for (; j + Team::size < m; j += 2 * Team::size) {
        const double2 a = buf[j];
        const double2 b = buf[j + Team::size];
        df_term(a, xh, xl, kx, kc, sh0, sl0, dh0, dc0);
        df_term(b, xh, xl, kx, kc, sh1, sl1, dh1, dc1);
    }
    if (j < m) df_term(buf[j], xh, xl, kx, kc, sh0, sl0, dh0, dc0);
    const double S = T.sum(((double)sh0 + (double)sl0) + ((double)sh1 + (double)sl1));
    const double Sd = T.sum(((double)dh0 - (double)dc0) + ((double)dh1 - (double)dc1));
    const double floor = (double)(m + 1) * 0x1p-78;   // n terms of 2^-99: 2^-21 relative
    ok = isfinite(S) && isfinite(Sd) && fabs(S) >= floor && fabs(Sd) >= floor;
    return make_double2(ldexp(S, kc), ldexp(Sd, kc - kx));
}

// The same pair from the poles (no stored buffer): with r_j = 1/(delta_j t_j),
// the term is q_j = zeta_j^2 r_j and its derivative zeta_j^2/t_j^2 = q_j (delta_j r_j) delta_j.
template <class P, class Team>
__device__ __forceinline__ double2 secular_sum_d(const P &R, const Team &T, double shift,
                                                 int skip, double x) {
    double s0 = 0.0, d0 = 0.0;
    for (int j = T.rank; j < R.m; j += Team::size) {
        if (j == skip) continue;
        const double dj = R.shifted(j, shift, skip);
        const double r = rcp(dj * fma(-x, dj, 1.0));
        const double q = R.z2(j) * r;
        s0 += q;
        d0 = fma(q * (dj * r), dj, d0);
    }
    return make_double2(T.sum(s0), T.sum(d0));
}

// FP32 analogue on scaled data:
// T(y) = sum_{j != skip} zz_j / (D_j (1 - y D_j)),  D_j = (p_j - shift) ds sc,
// zz_j = zeta_j^2 zs.  With x = s y and s = ds sc:  S(x) = s T(y) / zs.
template <class P, class Team>
__device__ __forceinline__ float secular_sum_f32(const P &R, const Team &T, float sh, float sl,
                                                 float sc, int skip, float y) {
    float acc0 = 0.f, acc1 = 0.f;
    int j = T.rank;
    for (; j + Team::size < R.m; j += 2 * Team::size) {
        if (j != skip) {
            const float D = R.shifted_f32(j, sh, sl) * sc;
            const float t = fmaf(-y, D, 1.f);
            acc0 = fmaf(R.z2f(j), rcp_f32(D * t), acc0);
        }
        const int j2 = j + Team::size;
        if (j2 != skip) {
            const float D = R.shifted_f32(j2, sh, sl) * sc;
            const float t = fmaf(-y, D, 1.f);
            acc1 = fmaf(R.z2f(j2), rcp_f32(D * t), acc1);
        }
    }
    if (j < R.m && j != skip) {
        const float D = R.shifted_f32(j, sh, sl) * sc;
        const float t = fmaf(-y, D, 1.f);
        acc0 = fmaf(R.z2f(j), rcp_f32(D * t), acc0);
    }
    return T.sumf(acc0 + acc1);
}

// T(y) and T'(y) = sum_{j != skip} zz_j / (1 - y D_j)^2 together (the FP32
// model steps that open the Newton finish); same scaled data as above.
template <class P, class Team>
__device__ __forceinline__ float2 secular_sum_f32_d(const P &R, const Team &T, float sh,
                                                    float sl, float sc, int skip, float y) {
    float a0 = 0.f, d0 = 0.f;
    for (int j = T.rank; j < R.m; j += Team::size) {
        if (j == skip) continue;
        const float D = R.shifted_f32(j, sh, sl) * sc;
        const float rt = rcp_f32(fmaf(-y, D, 1.f));           // 1 / (1 - y D)
        const float q = R.z2f(j) * rcp_f32(D) * rt;            // zz / (D (1 - y D))
        a0 += q;
        d0 = fmaf(q * D, rt, d0);                              // zz / (1 - y D)^2
    }
    return make_float2(T.sumf(a0), T.sumf(d0));
}

// Algorithm 1, first part: the shift pole i and the side (+1: lambda > p_i).
// The test is the sign of F at the midpoint x = p_k + middle of lambda's
// interval, F(x) = (alpha - p_k - middle) - sum_j zeta_j^2 / ((p_j - p_k) - middle).
// With f32 set it is first evaluated in FP32 on the scaled copies, with a
// bound on its error; when that bound, plus a bound on the error of the FP64
// evaluation, leaves the sign in no doubt, the FP64 sign is known and its pass
// is skipped, so the chosen shift is the one the FP64 test gives.  Returns true
// when the FP64 pass ran in that mode.
//
// The bound.  Every pole lies at least |middle| from x (the nearest two sit at
// +-middle), so |p_j - p_k| <= 2 |D_j| with D_j = (p_j - p_k) - middle.  In FP32
// (unit u = 2^-24) the scaled D_j is computed with error below
// 14 u |D_j| + 2^-44 g_j + 2^-145 (shifted_f32_mag, doubled by the factor 2,
// plus the roundings of middle and of the subtraction), so below 16 u |D_j|
// once |D_j| >= 2^-20 g_j + 2^-100 (else the FP64 pass runs).  The approximate
// reciprocal (one ulp) and the spike and product roundings bring each term to
// 20 u |t_j|, plus 2^-150 (|r_j| + 1) where they are subnormal.  Summation over
// L terms per thread and a butterfly adds (L + 4) u sum |t_j| (a CTA team sums
// its warps' FP32 partials in double).  So |T - T_exact| <= (L + 24) u A' +
// 2^-150 (B + m), with A' = sum |t_j| below 2 A and B below 2 B' (A, B' the FP32
// sums of |t_j| and |r_j|).  The FP64 pass errs by at most (L + 16) 2^-52 A64 on
// the same scale, far below the slack the margin keeps for it.
template <class P, class Team>
__device__ __forceinline__ bool select_shift(const P &R, const Team &T, int k, int &i,
                                             int &side, bool f32 = false,
                                             bool *ran32 = nullptr) {
    const int m = R.m;
    if (k == 0) {
        i = 0; side = +1;
        return false;
    }
    if (k == m) {
        i = m - 1; side = -1;
        return false;
    }
    const double sk = R.pole(k);
    const double middle = 0.5 * R.shifted(k - 1, sk, k);
    const dd a = R.a_dd(sk, k);
    const double am = a.hi - middle;
    const double L = (double)((m + Team::size - 1) / Team::size);
    int sgn = 0;
    if (f32 && R.has_f32() && L < 0x1p16) {
        if (ran32) *ran32 = true;
        float sh, sl;
        R.f32_shift(sk, k, sh, sl);
        const double sc = R.f32_scale();
        const float mf = (float)(middle * sc);
        float tf = 0.f, af = 0.f, bf = 0.f;
        bool bad = false;
        for (int j = T.rank; j < m; j += Team::size) {
            float g;
            const float D = R.shifted_f32_mag(j, sh, sl, g) - mf;
            bad |= !(fabsf(D) >= fmaf(g, 0x1p-20f, 0x1p-100f));
            const float r = rcp_f32(D);
            const float t = R.z2f(j) * r;
            tf += t;
            af += fabsf(t);
            bf += fabsf(r);
        }
        if (bad) bf = INFINITY;
        tf = T.sumf(tf);
        af = T.sumf(af);
        bf = T.sumf(bf);
        // S = (sc / zs) T with the power-of-two scalings of the copies
        const double f = sc / R.zs;
        const double F32 = am - f * (double)tf;
        const double ET = 2.0 * (L + 24.0) * 0x1p-24 * (2.0 * (double)af) +
                          0x1p-148 * ((double)bf + (double)m);   // doubled again
        const double M = f * ET * (1.0 + 0x1p-20) + (L + 16.0) * 0x1p-52 * fabs(am);
        if (isfinite(F32) && fabs(F32) > M * (1.0 + 0x1p-40)) sgn = F32 > 0.0 ? 1 : -1;
    }
    const bool ran64 = sgn == 0;
    if (ran64) {
        double acc = 0.0;
        for (int j = T.rank; j < m; j += Team::size)
            acc = fma(R.z2(j), rcp(R.shifted(j, sk, k) - middle), acc);
        const double F = am - T.sum(acc);
        sgn = F < 0.0 ? -1 : 1;
    }
    if (sgn < 0) { i = k; side = +1; }
    else { i = k - 1; side = -1; }
    return f32 && ran64;
}

// T(shift, skip) = -(alpha - shift) + sum_{j != skip} zeta_j^2 / (p_j - shift) in
// double-double, split into its nonnegative parts P - Q as Theorem 6 does
// (shifted differences exact by TwoSum, zeta_j^2 exact by TwoProd).  The same
// O(n) pass collects what the brackets need: with wscale = 1/zeta_i the
// Gershgorin intervals 1/delta_j -+ |w_j|, |w_j| = |zeta_j/delta_j| wscale.
struct PassA {
    dd P, Q;            // T = P - Q, P, Q >= 0
    double pmax;        // max over j != skip of 1/delta_j (or -inf)
    double pmin;        // min over j != skip of 1/delta_j (or +inf)
    double up;          // max of 1/delta_j + |w_j|
    double lo;          // min of 1/delta_j - |w_j|
    double wsum;        // sum |zeta_j / delta_j|
    double usq;         // sum zeta_j^2 / delta_j^2
    double cabs;        // sum |zeta_j^2 / delta_j| (bounds every |c_j|)
};

// GERSH = false skips the Gershgorin quantities (pmax, pmin, up, lo, wsum),
// which the Newton finish does not use.
// Each t_j = zeta_j^2 / delta_j is formed as two partial quotients q1 + q2
// (q1 within an ulp of the quotient, q2 from the FMA residual) and added to
// its sign's compensated sum (csum_add, renormalised every 16 terms).  With a
// pole shift (skip >= 0) and poles sorted decreasingly, delta_j > 0 exactly
// for j < skip, so the two sums come from two branch-free index ranges.  The
// stored pair is (delta_j, q1).
// DD = false (Algorithm 5's standard precision): plain double differences,
// quotients and sums, 7 instead of ~21 FP64 instructions a term; the stored
// pairs are the same values.
// For a shift that is not a pole (skip < 0), q >= 0 is the number of poles
// above it, which splits the index range the same way.
template <bool GERSH = true, bool DD = true, class P, class Team>
__device__ __forceinline__ PassA pass_a(const P &R, const Team &T, double shift, int skip,
                                        double wscale, double2 *buf = nullptr, int q = -1) {
    dd s1 = {0.0, 0.0}, s2 = {0.0, 0.0};
    int c1 = 0, c2 = 0;
    const double one = unit_reg();
    double pmax = -INFINITY, pmin = INFINITY, up = -INFINITY, lo = INFINITY, wsum = 0.0,
           usq = 0.0;
    auto term = [&](int j, double &dhi, double &uacc) -> dd {
        dd del;
        double q1, q2 = 0.0, p;
        if (DD) {
            del = R.shifted_dd(j, shift, skip);
            const dd z2 = R.z2_dd(j);
            p = rcp_o(del.hi, one);
            q1 = z2.hi * p;
            const double res = fma(-q1, del.lo, fma(-q1, del.hi, z2.hi) + z2.lo);
            q2 = res * p;
        } else {
            del = dd{R.shifted(j, shift, skip), 0.0};
            p = rcp_o(del.hi, one);
            q1 = R.z2(j) * p;
        }
        if (buf) buf[j] = make_double2(del.hi, q1);   // (delta_j, zeta_j^2 / delta_j)
        if (GERSH) {
            const double aw = R.zabs(j) * fabs(p);
            pmax = fmax(pmax, p);
            pmin = fmin(pmin, p);
            up = fmax(up, fma(aw, wscale, p));
            lo = fmin(lo, fma(-aw, wscale, p));
            wsum += aw;
        }
        uacc = fma(q1, p, uacc);                        // zeta_j^2 / delta_j^2
        dhi = del.hi;
        return dd{q1, q2};
    };
    auto add = [](dd &acc, int &cnt, dd t) {
        if (!DD) {
            acc.hi += t.hi;
            return;
        }
        csum_add(acc, t);
        if (++cnt == 16) {
            acc = fast_two_sum(acc.hi, acc.lo);
            cnt = 0;
        }
    };
    double dhi;
    if (!DD && (skip >= 0 || q >= 0)) {
        // standard precision: two interleaved accumulators per range, so that
        // consecutive terms are independent
        const int e1 = skip >= 0 ? skip : q, b2 = skip >= 0 ? skip + 1 : q;
        double a0 = 0.0, a1 = 0.0, u1 = 0.0;
        int j = T.rank;
        for (; j + Team::size < e1; j += 2 * Team::size) {
            a0 += term(j, dhi, usq).hi;
            a1 += term(j + Team::size, dhi, u1).hi;
        }
        if (j < e1) a0 += term(j, dhi, usq).hi;
        s1.hi = a0 + a1;
        a0 = a1 = 0.0;
        j = b2 + ((T.rank - b2) % Team::size + Team::size) % Team::size;
        for (; j + Team::size < R.m; j += 2 * Team::size) {
            a0 += term(j, dhi, usq).hi;
            a1 += term(j + Team::size, dhi, u1).hi;
        }
        if (j < R.m) a0 += term(j, dhi, usq).hi;
        s2.hi = a0 + a1;
        usq += u1;
        if (buf && skip >= 0 && skip % Team::size == T.rank) buf[skip] = make_double2(0.0, 0.0);
    } else if (skip >= 0 || q >= 0) {
        const int e1 = skip >= 0 ? skip : q, b2 = skip >= 0 ? skip + 1 : q;
        for (int j = T.rank; j < e1; j += Team::size) add(s1, c1, term(j, dhi, usq));
        int j = b2 + ((T.rank - b2) % Team::size + Team::size) % Team::size;
        for (; j < R.m; j += Team::size) add(s2, c2, term(j, dhi, usq));
        if (buf && skip >= 0 && skip % Team::size == T.rank) buf[skip] = make_double2(0.0, 0.0);
    } else {
        for (int j = T.rank; j < R.m; j += Team::size) {
            const dd t = term(j, dhi, usq);
            if (dhi > 0.0) add(s1, c1, t);
            else add(s2, c2, t);
        }
    }
    if (DD) {
        s1 = fast_two_sum(s1.hi, s1.lo);
        s2 = fast_two_sum(s2.hi, s2.lo);
        s1 = T.sum(s1);
        s2 = T.sum(s2);
    } else {
        // standard precision: every thread's partial is one double (lo = 0), so
        // the team adds doubles too -- five more roundings on top of the L per
        // thread, where a double-double reduction costs ~100 FP64 instructions
        s1 = dd{T.sum(s1.hi), 0.0};
        s2 = dd{T.sum(s2.hi), 0.0};
    }
    PassA A;
    if (GERSH) {
        A.pmax = T.max(pmax);
        A.pmin = T.min(pmin);
        A.up = T.max(up);
        A.lo = T.min(lo);
        A.wsum = T.sum(wsum);
    } else {
        A.pmax = A.pmin = A.up = A.lo = A.wsum = NAN;
    }
    A.usq = T.sum(usq);
    A.cabs = s1.hi - s2.hi;             // s1 >= 0 >= s2
    const dd a = R.a_dd(shift, skip);   // alpha - shift
    if (a.hi < 0.0) {                   // -a > 0: P = -a + S1, Q = -S2
        A.P = dd_add_same(dd_neg(a), s1);
        A.Q = dd_neg(s2);
    } else {                            // P = S1, Q = a - S2
        A.P = s1;
        A.Q = dd_add_same(a, dd_neg(s2));
    }
    return A;
}

// Roots xs <= xb of (B - x)(x - P) + Wq = 0 with Wq > 0 (so xs < min(B, P) and
// xb > max(B, P)), without cancellation: the root away from zero by the
// formula, the other from the product of the roots, B P - Wq.
__device__ __forceinline__ void quad_roots(double B, double P, double Wq, double &xs,
                                           double &xb) {
    // sqrt((B - P)^2 + 4 Wq) with one square root: both terms scaled by 2^-k,
    // k from the larger one's exponent, so that nothing overflows and the
    // result scales exactly with the problem (a power-of-two scaling of A
    // moves k and nothing else)
    const double u = B - P, w = 4.0 * Wq;
    const int eu = (int)((__double_as_longlong(u) >> 52) & 0x7ff);   // biased exponents
    const int ew = (int)((__double_as_longlong(w) >> 52) & 0x7ff);
    const int k = max(eu, 1023 + ((ew - 1023) >> 1)) - 1023;
    double sq;
    if (eu > 0 && eu < 2047 && ew > 0 && ew < 2047 && k < 1023) {     // normal, finite
        // 2^-k and 2^k from their bits (-1022 <= -k, k <= 1022): exact scalings
        const double si = __longlong_as_double((long long)(1023 - k) << 52);
        const double so = __longlong_as_double((long long)(1023 + k) << 52);
        const double us = u * si, ws = (w * si) * si;
        sq = sqrt(fma(us, us, ws)) * so;
    } else {
        sq = hypot(u, 2.0 * sqrt(Wq));
    }
    const double s = B + P;
    if (s >= 0.0) {
        xb = 0.5 * (s + sq);
        xs = (B * P - Wq) / xb;
    } else {
        xs = 0.5 * (s - sq);
        xb = (B * P - Wq) / xs;
    }
}

// ---------------------------------------------------------------------------
// FP32 opening bracket
// ---------------------------------------------------------------------------
// Narrow [left, right] (which holds the zero of a function Phi) with FP32
// bisection into [l, r].  Phi(x) = G(x) - K T(y), x = s y, where G is the FP64
// part (shift, b, the 1/x term) and T the FP32 sum, K = K_over_s * s / zs.
// `dir` = +1 when Phi > 0 below the zero, -1 when above.  Returns false when
// the FP32 data cannot represent the problem ([l, r] is then [left, right]).
// The new ends are NOT verified here.
template <class P, class Team, class G64>
__device__ bool fp32_narrow(const P &R, const Team &T, double shift, int skip, double K_over_s,
                            int dir, G64 g64, double left, double right, double &l, double &r,
                            int &passes) {
    l = left;
    r = right;
    const double big = fmax(fabs(left), fabs(right));
    if (!(big > 0.0) || !isfinite(big)) return false;
    const double s = ldexp(1.0, ilogb(big));          // x = s y, |y| <= 2
    const double scd = s / R.f32_scale();               // D_j = scaled difference * scd
    if (!(scd > 0x1p-120 && scd < 0x1p120)) return false;
    float sh, sl;
    R.f32_shift(shift, skip, sh, sl);
    if (!isfinite(sh)) return false;
    const float sc = (float)scd;
    const double K = K_over_s * s / R.zs;
    for (int it = 0; it < 80; ++it) {
        const double mid = 0.5 * (l + r);
        if (r - l <= 0x1p-21 * fabs(mid)) break;
        const float y = (float)(mid / s);
        const double x = s * (double)y;                 // the point actually evaluated
        if (!(x > l && x < r)) break;
        const float Tf = secular_sum_f32(R, T, sh, sl, sc, skip, y);
        ++passes;
        const double KT = K * (double)Tf;
        const double phi = g64(x) - KT;
        if (!(fabs(phi) > 0x1p-24 * fabs(KT))) break;   // below FP32 resolution
        if ((phi > 0.0) == (dir > 0)) l = x;
        else r = x;
    }
    return true;
}

// Check the narrowed ends [l, r] of a bracket [left, right] in FP64 and move
// [left, right] in to them.  Each end gets one FP64 evaluation; an end that
// fails is moved out by 16x the width (twice at most) and otherwise left where
// it was.  Returns false when an end had to be given up.
template <class F64>
__device__ bool fp32_verify(int dir, F64 f64, double l, double r, double &left, double &right) {
    const double w = r - l;
    bool ok = true;
    // left end: Phi must say "below the zero"
    if (l > left) {
        double off = w, L = left;
        bool good = false;
        for (int t = 0; t < 3 && !good; ++t, off *= 16.0) {
            L = fmax(left, l - off);
            if (L == left) { good = true; break; }
            const double fl = f64(L);
            good = fl != 0.0 && ((fl > 0.0) == (dir > 0));
        }
        if (good) left = L;
        else ok = false;
    }
    // right end: Phi must not say "below the zero"
    if (r < right) {
        double off = w, Rr = right;
        bool good = false;
        for (int t = 0; t < 3 && !good; ++t, off *= 16.0) {
            Rr = fmin(right, r + off);
            if (Rr == right) { good = true; break; }
            const double fr = f64(Rr);
            good = fr == 0.0 || ((fr > 0.0) != (dir > 0));
        }
        if (good) right = Rr;
        else ok = false;
    }
    return ok;
}

// ---------------------------------------------------------------------------
// Bracketed Newton finish (not in the paper; a faster way to Algorithm 3's
// answer).  F is strictly decreasing on the bracket (F' <= -1) and has one
// curvature sign there: convex when the zero lies right of all of F's poles
// (side > 0), concave when left of them.  `pole` is F's pole nearest the
// bracket (its largest pole for side > 0, smallest for side < 0).
// [left, right] holds the zero; gl <= left, right <= gr are known-good ends.
// Every trial point lies strictly inside the current bracket, each evaluation
// moves the end on its side (F > 0: left) exactly as bisection does, and the
// loop stops on Algorithm 3's test right - left <= 2 eps |mid|, so nu = right
// is the right end of a bracket of the computed F of bisection's final width.
// Trial points, in order of preference:
//  * after a step that was lengthened to tol and did not change sides, F is
//    rounding noise there: a jump of twice the estimated noise width
//    (err / |F'|) towards the zero, growing 4x while it does not change sides,
//    then midpoints only;
//  * the zero of the one-pole model  a + kappa x + beta / (x - pole)  that
//    matches F and F' at x (kappa = -1 for the shifted inverse's Pick
//    function, 0 for the DPR1 secular function): the Newton step of a function
//    dominated by its nearest pole, exact for a 2 x 2 arrowhead; when the
//    Newton step -F/F' is shorter than 2^-30 |x - pole|, that step instead
//    (the two agree to that order, and the model's formula loses so short a
//    step in rounding); either lengthened to tol = 2^-52 |x| when shorter
//    (which closes the bracket from the other side once the zero is that near);
//  * when that leaves the bracket, the last such point taken from the side
//    whose steps do not overshoot, else the midpoint.  The model puts all of
//    F' beyond kappa on the nearest pole, so near x it is more convex than F:
//    from the pole's side of the zero (F > 0 for side > 0) its zero lies past
//    F's, from the far side (F < 0 for side > 0) short of it.
// Ends lv / rv not yet evaluated in FP64 (from the FP32 phase) are checked
// after the loop; a failed check is itself a good end on the other side, and
// the search resumes from the known-good end.  Returns the number of FP64
// evaluations; `fell_back` reports a failed check.
// ---------------------------------------------------------------------------
// F' is evaluated (3 more FP64 instructions a term) only when the last step
// was longer than 2^-26 rho, rho = |x - pole| the distance to F's nearest
// pole (F' = kappa - sum_k W_k / (x - p_k)^2 changes by a factor within
// 1 +- 2 |h| / rho over a step h): after a shorter one the previous F' is
// within 2^-25 relative of the current one, enough for a step whose own
// length is below 2^-26 rho.  (A bound relative to |x| instead lets a stale F'
// from nearer the pole, where |F'| is larger, shorten every step below the
// bound, so that F' is never re-evaluated and the bracket creeps.)  dF0
// (finite): an estimate of F' at the start that is that good already (the
// caller's bracket is that tight), so the first evaluation skips F' too.
//
// Local expansion (ca finite).  Both functions searched here have the form
// F(x) = kappa x + const + K (S(x) - 1/x) with the terms q_j = c_j / (1 - x delta_j)
// of S all of one sign beyond the poles (the shifted inverse's Pick function:
// kappa = -1, K = -c; the DPR1 function: kappa = 0, K = sign * rho); ca = -K.
// S(x + h) = S(x) + h S'(x) + sum_j q_j e_j^2 / (1 - e_j), e_j = h delta_j /
// (1 - x delta_j), |e_j| <= |h| / rho where rho = |x - pole| is the distance to
// F's nearest pole other than 0.  So
//     F(x + h) = F(x) + h F'(x) + ca h^2 / (x^2 (x + h))          (1/x term exact)
// up to |K S| (h/rho)^2 (1 + ...) from the remainder and |h| |K dS'| from an
// error dS' in S'.  For |h| <= Ha = min(2^-27 rho, err / (4 drel |K S'|)), drel
// a bound on the relative error of the S' in hand, both stay below a quarter
// of the rounding bound err of the FP64 evaluation at x (which includes
// 2^-52 |K S|), so the expansion is an evaluation of F with the same O(eps)
// error per term.  After each FP64
// evaluation the loop keeps that expansion (the anchor) and evaluates trial
// points within Ha of it from it, at scalar cost; those are not counted as
// FP64 evaluations.  The S' in hand is the one formed at xs (the last FP64
// evaluation with F', or dF0's point xdF0 with relative error rel0), moved to
// x with relative error at most 4 |x - xs| / rho while |x - xs| <= rho / 8.
template <class FD>
__device__ __forceinline__ int newton_finish(FD fd, int side, double pole, double kappa,
                                             double gl, double gr, bool lv, bool rv,
                                             int max_iter, double &left, double &right,
                                             bool &fell_back, double dF0 = NAN,
                                             int *nderiv = nullptr, double x0 = NAN,
                                             double ca = NAN, double xdF0 = NAN,
                                             double rel0 = INFINITY) {
    int it = 0, itd = 0, itl = 0;
    fell_back = false;
    bool need_d = !isfinite(dF0);
    double dF = need_d ? -1.0 : dF0;
    double xsrc = xdF0, rsrc = need_d ? INFINITY : rel0;
    double KSs = need_d ? 0.0 : dF0 - kappa + ca / xdF0 / xdF0;   // K S' at xsrc
    double xa = NAN, Fa = 0.0, dFa = 0.0, Ha = -1.0;
    for (;;) {
        // the first trial point: x0 when the caller has one inside the bracket
        double x = (x0 > left && x0 < right) ? x0 : 0.5 * (left + right);
        x0 = NAN;
        double pend = NAN;          // last model point from the good side
        double jump = 0.0;
        bool nudged = false, noisy = false, jumping = false, pside = false;
        double err = 0.0;
        while (right - left > TWO_EPS * fabs(0.5 * (left + right)) && it < max_iter) {
            double F;
            if (fabs(x - xa) <= Ha && itl < 64) {
                const double h = x - xa;
                const double ixa = rcp(xa);
                F = Fa + h * (dFa + (ca * ixa) * (h * ixa) * rcp(x));   // (no overflow)
                dF = dFa;
                ++itl;
            } else {
                F = fd(x, need_d, dF, err);
                ++it;
                itd += need_d ? 1 : 0;
                // (reciprocals, not divisions, in this scalar bookkeeping: a
                // few ulps here move no bound by more than its slack)
                const double ix = rcp(x);
                const double cxx = (ca * ix) * ix;              // ca / x^2
                if (need_d) {
                    xsrc = x;
                    rsrc = 0x1p-40;
                    KSs = dF - kappa + cxx;
                }
                Ha = -1.0;
                if (isfinite(ca) && isfinite(rsrc)) {
                    const double rho = fabs(x - pole);
                    const double dist = fabs(x - xsrc);
                    const double drel = rsrc + 4.0 * dist * rcp(rho);
                    double H = 0x1p-27 * rho;
                    if (fabs(KSs) > 0.0) H = fmin(H, 0.25 * err * rcp(drel * fabs(KSs)));
                    if (dist <= 0.125 * rho && H > 0.0) {
                        xa = x;
                        Fa = F;
                        dFa = kappa + KSs - cxx;
                        dF = dFa;
                        Ha = H;
                    }
                }
            }
            const bool pos = F > 0.0;
            if (pos) { left = x; lv = true; }
            else { right = x; rv = true; }
            const double mid = 0.5 * (left + right);
            const double towards = pos ? 1.0 : -1.0;    // direction of the zero from x
            const double tol = 0x1p-52 * fabs(x);
            double xn;
            bool nudge = false;
            if (noisy) {
                if (jumping && pos == pside) {          // the jump stayed on one side
                    jump *= 4.0;
                    xn = x + towards * jump;
                } else {
                    jumping = false;
                    xn = mid;
                }
            } else if (nudged && pos == pside) {        // the lengthened step stayed on one side
                noisy = true;
                jumping = true;
                jump = fmax(2.0 * err / fabs(dF), 2.0 * tol);
                xn = x + towards * jump;
            } else {
                const double d0 = fabs(x - pole);
                const double hN = -F * rcp(dF);          // the Newton step (F' < 0)
                if (fabs(hN) < 0x1p-30 * d0) {
                    // a step this short agrees with the model's to 2^-30 of its
                    // length, and the model's formula (differences of terms as
                    // large as |x| and beta / d0) would lose it in rounding and
                    // could point the wrong way
                    xn = x + hN;
                } else {
                    // one-pole model a + kappa x + beta / (x - pole) through
                    // (x, F, F'): beta = (kappa - F') (x - pole)^2 >= 0
                    const double beta = (kappa - dF) * d0 * d0;
                    const double a = F - kappa * x + (side > 0 ? -beta : beta) * rcp(d0);
                    if (kappa == 0.0) {
                        xn = pole - beta / a;
                    } else {                             // kappa = -1
                        double xs, xb;
                        quad_roots(a, pole, beta, xs, xb);
                        xn = side > 0 ? xb : xs;
                    }
                }
                if (fabs(xn - x) < tol) {
                    xn = x + towards * tol;
                    nudge = true;
                } else if (pos != (side > 0)) {
                    pend = xn;
                }
            }
            if (!(xn > left && xn < right)) {
                nudge = false;
                jumping = false;
                xn = (!noisy && pend > left && pend < right) ? pend : mid;
            }
            nudged = nudge;
            pside = pos;
            need_d = !(fabs(xn - x) < 0x1p-26 * fabs(x - pole));
            x = xn;
        }
        need_d = true;
        if (lv && rv) break;
        if (!lv) {
            ++it;
            if (fd(left, false, dF, err) > 0.0) lv = true;
            else { right = left; left = gl; lv = rv = true; fell_back = true; }
        }
        if (!rv) {
            ++it;
            if (!(fd(right, false, dF, err) > 0.0)) rv = true;
            else { left = right; right = gr; lv = rv = true; fell_back = true; }
        }
    }
    if (nderiv) *nderiv = itd;
    return it;
}

// ---------------------------------------------------------------------------
// Algorithm 2 + 3 for the shift pole i on `side`, then lambda = sigma + 1/nu.
// ---------------------------------------------------------------------------
template <class P, class Team>
__device__ EigResult solve_shifted(const P &R, const Team &T, int i, int side,
                                   const SolveOpts &o, double2 *buf = nullptr) {
    EigResult res;
    res.flags = 0;
    res.f32p = 0;
    res.dfp = 0;
    const double sigma = R.pole(i);
    const double zi = R.zabs(i);
    const double wz = 1.0 / zi;         // w_zeta
    const double c = wz * wz;           // 1/zeta_i^2
    const bool newton = o.finish == 1;
    PassA A;
    if (o.bgate) {
        // Algorithm 5: b in standard precision unless both C2 (i) and C2 (ii)
        // fail -- the spike ratio sum_{j != i} |zeta_j| / |zeta_i| exceeds the
        // order n and K_b of Eq. (K2) from the standard sums exceeds kb_max --
        // then P and Q again in double-double (Theorem 6)
        A = newton ? pass_a<false, false>(R, T, sigma, i, wz, buf)
                   : pass_a<true, false>(R, T, sigma, i, wz, buf);
        // (both tests multiplied out: ratio = (zsum - zeta_i) / zeta_i > m + 1
        // and K_b0 = (P + Q) / |P - Q| > kb_max, NaN or a zero P - Q included)
        if (R.zsum - zi > (double)(R.m + 1) * zi &&
            !(A.P.hi + A.Q.hi <= o.kb_max * fabs(A.P.hi - A.Q.hi))) {
            const PassA D = pass_a<false, true>(R, T, sigma, i, wz);
            A.P = D.P;
            A.Q = D.Q;
            res.flags |= 128;                  // AE_FLAG_DDB
        }
    } else {
        A = newton ? pass_a<false>(R, T, sigma, i, wz, buf)
                   : pass_a<true>(R, T, sigma, i, wz, buf);
    }
    // b = (P - Q) / zeta_i^2 in double-double (Theorem 6), rounded once
    const dd num = dd_add(A.P, dd_neg(A.Q));
    const double b = dd_div(num, two_prod(zi, zi)).hi;
    res.Kb = (A.P.hi + A.Q.hi) / fabs(num.hi);
    res.b = b;
    // with a buffer, each term is c_j / (1 - x delta_j) from the stored pair
    // (5 FP64 instructions instead of 7); the value is the same S(x)
    auto F64 = [&](double x) {
        const double S = buf ? secular_sum_stored(buf, R.m, T, x)
                             : secular_sum(R, T, sigma, i, x);
        return (b - x) - c * (S - rcp(x));
    };
    // F = (b - x) + c/x - c S(x),  c S(x) = (c s / zs) T(y) in the FP32 phase
    auto G = [&](double x) { return (b - x) + c * rcp(x); };
    const bool f32 = o.precision == 1 && R.has_f32();
    double left, right;
    int it = 0, itd = 0;
    if (newton) {
        // F's poles are 1/delta_j (j != i) and 0; the one nearest the searched
        // side is 1/delta_{i-1} (side > 0, i > 0) or 1/delta_{i+1} (side < 0,
        // i < m-1), else 0.  For x beyond all poles F(x) = b - x + sum_k W_k/(x - p_k)
        // (side > 0), W_k > 0 with sum W = c (sum_j zeta_j^2/delta_j^2 + 1); moving
        // all weight onto the nearest pole bounds F from one side and keeping
        // only that pole's weight from the other, so the zeros of the two
        // one-pole quadratics bracket the zero of F (widened by 2^-30 relative
        // for the rounding of the weights).
        const int jn = side > 0 ? i - 1 : i + 1;
        double pole = 0.0, Wn = c;
        if (jn >= 0 && jn < R.m) {
            const double pn = rcp(R.shifted_dd(jn, sigma, i).hi);
            if (side > 0 ? pn > 0.0 : pn < 0.0) {
                pole = pn;
                Wn = c * R.z2(jn) * pn * pn;
            }
        }
        double xs, xb, ys, yb;
        quad_roots(b, pole, c * (A.usq + 1.0), xs, xb);
        quad_roots(b, pole, Wn, ys, yb);
        if (side > 0) {
            left = fmax(pole, yb - 0x1p-30 * fabs(yb));
            right = xb + 0x1p-30 * fabs(xb);
        } else {
            left = xs - 0x1p-30 * fabs(xs);
            right = fmin(pole, ys + 0x1p-30 * fabs(ys));
        }
        if (!(isfinite(left) && isfinite(right) && left < right)) {
            // out of range for the quadratic bounds: Gershgorin, as bisection uses
            const PassA Gb = pass_a<true>(R, T, sigma, i, wz);
            const double norm1 = fma(Gb.wsum, wz, wz);
            if (side > 0) {
                left = fmax(Gb.pmax, 0.0);
                right = fmax(fmax(Gb.up, wz), b + norm1);
            } else {
                right = fmin(Gb.pmin, 0.0);
                left = fmin(fmin(Gb.lo, -wz), b - norm1);
            }
        }
        // F and F' = -1 - c (S'(x) + 1/x^2) in one pass, and a bound on the
        // rounding error of F (the terms of S share one sign on this side)
        auto FD = [&](double x, bool need_d, double &dF, double &err) {
            double2 S;
            if (need_d) {
                S = buf ? secular_sum_d_stored(buf, R.m, T, x) : secular_sum_d(R, T, sigma, i, x);
            } else {
                S.x = buf ? secular_sum_stored(buf, R.m, T, x) : secular_sum(R, T, sigma, i, x);
                S.y = 0.0;
            }
            const double rx = rcp(x);
            if (need_d) dF = -1.0 - c * fma(rx, rx, S.y);
            err = 0x1p-52 * (fabs(b) + fabs(x) + c * (fabs(S.x) + fabs(rx)));
            return (b - x) - c * (S.x - rx);
        };
        const double gl = left, gr = right;
        const bool lv = true, rv = true;
        // FP32 opening for the Newton finish: one-pole model steps on the
        // rescaled FP32 copy (F and F' with c S(x) = K T(y)) give the first
        // FP64 trial point; they move no bracket end (unverified)
        double x0 = NAN, dF0 = NAN;
        // a bracket already narrower than 2^-26 relative needs no FP32 steps:
        // the double-float step below starts from its middle
        const bool tight = right - left < 0x1p-26 * fabs(0.5 * (left + right));
        if (f32 && tight) {
            x0 = 0.5 * (left + right);
        } else if (f32) {
            const double big = fmax(fabs(left), fabs(right));
            const double s = ldexp(1.0, ilogb(big));
            const double scd = s / R.f32_scale();
            float sh = 0.f, sl = 0.f;
            R.f32_shift(sigma, i, sh, sl);
            if (big > 0.0 && isfinite(big) && scd > 0x1p-120 && scd < 0x1p120 && isfinite(sh)) {
                const float sc = (float)scd;
                const double K = c * s / R.zs;
                const double sinv = ldexp(1.0, -ilogb(big));   // 1/s, exact
                double x = 0.5 * (left + right);
                double dF32 = NAN, step = INFINITY;
                // up to 8 steps, until one is shorter than FP32 can resolve
                // (2^-20 of the distance to the nearest pole): far from the
                // zero, where a bracket spans orders of magnitude, each step
                // only about halves the distance, and an FP32 step costs the
                // FP64 pipe ~1/50 of an FP64 evaluation
                for (int t = 0; t < 8; ++t) {
                    const float y = (float)(x * sinv);
                    const double xe = s * (double)y;
                    const float2 Tf = secular_sum_f32_d(R, T, sh, sl, sc, i, y);
                    ++res.f32p;
                    const double rx = rcp(xe);
                    const double F = (b - xe) + c * rx - K * (double)Tf.x;
                    const double dF = -1.0 - c * rx * rx - K * (double)Tf.y * sinv;
                    const double d0 = fabs(xe - pole);
                    const double beta = (-1.0 - dF) * d0 * d0;
                    const double a = F + xe + (side > 0 ? -beta : beta) * rcp(d0);
                    double xs, xb;
                    quad_roots(a, pole, beta, xs, xb);
                    const double xn = side > 0 ? xb : xs;
                    if (!(xn > left && xn < right)) break;
                    step = fabs(xn - x);
                    dF32 = dF;
                    x = xn;
                    if (!(step > 0x1p-20 * fabs(x - pole))) break;
                }
                x0 = x;
                // an FP32 step that short (against the distance to the nearest
                // pole) leaves F' known to FP32 accuracy, which serves as the
                // first FP64 evaluation's F'
                if (step < 0x1p-20 * fabs(x0 - pole)) dF0 = dF32;
            } else {
                res.flags |= 64;
            }
        }
        // a bracket this tight means all of F's weight sits at its nearest pole
        // to that accuracy: F'(x) = -1 - W / (x - pole)^2 is the first F'
        const double xm = 0.5 * (left + right);
        if (right - left < 0x1p-26 * fabs(xm)) {
            const double dx = xm - pole;
            dF0 = -1.0 - c * (A.usq + 1.0) / (dx * dx);
        }
        // one more model step from the FP32 point with S in double-float and
        // S' in compensated FP32 on the stored pairs: the first FP64 trial
        // point lands within ~2^-40 relative of the zero, where the local
        // expansion of that one FP64 evaluation closes the bracket; its S'
        // (relative error below 2^-18 here) seeds the expansion
        double xdF0 = NAN, rel0 = INFINITY;
        if (f32 && buf && A.cabs > 0.0 && isfinite(A.cabs) && x0 > left && x0 < right &&
            x0 != 0.0) {
            bool ok;
            const double2 Sd =
                secular_sum_df_stored(buf, R.m, T, x0, ilogb(x0), ilogb(A.cabs), ok);
            ++res.dfp;
            if (ok) {
                const double rx = rcp(x0);
                const double F = (b - x0) - c * (Sd.x - rx);
                const double dF = -1.0 - c * fma(rx, rx, Sd.y);
                const double d0 = fabs(x0 - pole);
                const double beta = (-1.0 - dF) * d0 * d0;
                const double a = F + x0 + (side > 0 ? -beta : beta) * rcp(d0);
                double xs, xb;
                quad_roots(a, pole, beta, xs, xb);
                const double xn = side > 0 ? xb : xs;
                if (xn > left && xn < right && fabs(xn - x0) <= 0x1p-8 * d0) {
                    xdF0 = x0;
                    dF0 = dF;
                    rel0 = 0x1p-18;
                    x0 = xn;
                }
            }
        }
        bool fb;
        it = newton_finish(FD, side, pole, -1.0, gl, gr, lv, rv, o.max_iter, left, right, fb,
                           dF0, &itd, x0, c, xdF0, rel0);
        if (fb) res.flags |= 64;
    } else {
        // Gershgorin bracket of Algorithm 3 for the inverse: diagonal {1/delta_j, 0},
        // spikes {w_j, w_zeta}, corner b.
        const double norm1 = fma(A.wsum, wz, wz);
        if (side > 0) {
            left = fmax(A.pmax, 0.0);
            right = fmax(fmax(A.up, wz), b + norm1);
        } else {
            right = fmin(A.pmin, 0.0);
            left = fmin(fmin(A.lo, -wz), b - norm1);
        }
        if (f32) {
            double l, r;
            if (!fp32_narrow(R, T, sigma, i, c, +1, G, left, right, l, r, res.f32p) ||
                !fp32_verify(+1, F64, l, r, left, right))
                res.flags |= 64;
        }
        double mid = 0.5 * (left + right);
        while (right - left > TWO_EPS * fabs(mid) && it < o.max_iter) {
            const double F = F64(mid);
            if (F > 0.0) left = mid;
            else right = mid;
            mid = 0.5 * (left + right);
            ++it;
        }
    }
    const double nu = right;            // Algorithm 3 returns the right end
    res.sigma = sigma;
    res.mu = 1.0 / nu;
    res.lam = sigma + res.mu;
    res.pole = i;
    res.iters = it;
    res.iters_d = itd;
    res.flags |= (it >= o.max_iter) ? 16 : 0;
    return res;
}

// Remark 1 (shift = 0) and Remark 2(b) (shift near lambda, not a pole):
// (A - shift I)^{-1} = diag((D - shift I)^{-1}, 0) + rho u u^T with
// u = [(D - shift I)^{-1} z; -1] and rho = 1/(a - z^T (D - shift I)^{-1} z),
// whose denominator is computed in double-double.  Its eigenvalues are the
// zeros of phi(x) = 1 + rho sum_j u_j^2 / (p_j - x) (p_n = 0, u_n = -1), i.e.
// phi(x) = 1 + rho (S(x) - 1/x) with S over all poles.  The eigenvalue of A
// closest to the shift on the side sign(rho) gives the extreme zero nu of
// phi on that side; lambda = shift + 1/nu.
template <class P, class Team>
__device__ EigResult solve_dpr1_shift(const P &R, const Team &T, double shift,
                                      const SolveOpts &o, double2 *buf = nullptr) {
    EigResult res;
    res.sigma = shift;
    res.pole = -1;
    res.b = NAN;
    res.flags = 0;
    res.f32p = 0;
    res.dfp = 0;
    res.iters_d = 0;
    // q = number of poles above the shift: delta_j > 0 exactly for j < q, so
    // the largest 1/delta_j is 1/delta_{q-1} and the smallest 1/delta_q (the
    // poles are sorted and the shift is none of them)
    int q = 0;
    {
        int hi = R.m;
        while (q < hi) {
            const int mid = (q + hi) >> 1;
            if (R.pole(mid) > shift) q = mid + 1;
            else hi = mid;
        }
    }
    const PassA A = pass_a<false>(R, T, shift, -1, 1.0, buf, q);
    const double pmax = q > 0 ? rcp(R.shifted_dd(q - 1, shift, -1).hi)
                              : (R.m > 0 ? rcp(R.shifted_dd(R.m - 1, shift, -1).hi) : -INFINITY);
    const double pmin = q < R.m ? rcp(R.shifted_dd(q, shift, -1).hi)
                                : (R.m > 0 ? rcp(R.shifted_dd(0, shift, -1).hi) : INFINITY);
    const dd Tn = dd_add(A.P, dd_neg(A.Q));   // a - z^T (D - shift)^{-1} z = -Tn
    res.Kb = (A.P.hi + A.Q.hi) / fabs(Tn.hi);
    if (Tn.hi == 0.0) {                       // numerically singular: lambda = shift
        res.mu = 0.0;
        res.lam = shift;
        res.iters = 0;
        res.flags = 32;
        return res;
    }
    const double rho = -1.0 / Tn.hi;
    const double usq = A.usq + 1.0;          // ||u||^2
    // the zero lies within rho ||u||^2 of the outermost pole; when the rank-one
    // term dominates it sits right at that bound, so the computed bound is
    // widened by 2^-30 relative for its rounding
    double left, right;
    if (rho > 0.0) {
        left = fmax(pmax, 0.0);
        right = fma(rho, usq, left);
        right += 0x1p-30 * fabs(right);
    } else {
        right = fmin(pmin, 0.0);
        left = fma(rho, usq, right);
        left -= 0x1p-30 * fabs(left);
    }
    // rho > 0: phi increases through the zero (phi < 0 below it); rho < 0: phi > 0 below
    const int dir = rho > 0.0 ? -1 : +1;
    auto S0 = [&](double x) {
        return buf ? secular_sum_stored(buf, R.m, T, x) : secular_sum(R, T, shift, -1, x);
    };
    auto PHI = [&](double x) { return fma(rho, S0(x) - rcp(x), 1.0); };
    // (no FP32 bracket here: with a shift next to lambda, nu ~ 1/(lambda - shift)
    // is far outside what a power-of-two rescaled FP32 copy can represent; the
    // double-float steps below scale per evaluation instead)
    int it = 0, itd = 0;
    if (o.finish == 1) {
        // the Newton finish on dir * phi, which decreases through the zero; the
        // zero lies beyond all poles {1/delta_j, 0} on the side sign(rho), where
        // phi is concave (rho > 0) or convex (rho < 0)
        const int side = rho > 0.0 ? +1 : -1;
        const double pole = rho > 0.0 ? left : right;
        const double sg = (double)dir;
        auto FD = [&](double x, bool need_d, double &dF, double &err) {
            double2 S;
            if (need_d) {
                S = buf ? secular_sum_d_stored(buf, R.m, T, x) : secular_sum_d(R, T, shift, -1, x);
            } else {
                S.x = S0(x);
                S.y = 0.0;
            }
            const double rx = rcp(x);
            if (need_d) dF = sg * rho * fma(rx, rx, S.y);
            err = 0x1p-52 * (1.0 + fabs(rho) * (fabs(S.x) + fabs(rx)));
            return sg * fma(rho, S.x - rx, 1.0);
        };
        // under AE_FP32_BRACKET, model steps with S in double-float and S' in
        // compensated FP32 on the stored pairs (no FP32 copy of this problem
        // is needed) choose the first FP64 trial point, from the middle of the
        // bracket, and seed the local expansion (K = sign rho, so ca = -sign rho)
        double x0 = NAN, dF0 = NAN, xdF0 = NAN, rel0 = INFINITY;
        if (o.precision == 1 && buf && A.cabs > 0.0 && isfinite(A.cabs)) {
            const int kc = ilogb(A.cabs);
            double x = 0.5 * (left + right);
            for (int t = 0; t < 3 && x != 0.0 && isfinite(x); ++t) {
                bool ok;
                const double2 Sd = secular_sum_df_stored(buf, R.m, T, x, ilogb(x), kc, ok);
                ++res.dfp;
                if (!ok) break;
                const double rx = rcp(x);
                const double F = sg * fma(rho, Sd.x - rx, 1.0);
                const double dF = sg * rho * fma(rx, rx, Sd.y);
                const double d0 = fabs(x - pole);
                const double beta = -dF * d0 * d0;
                const double a = F + (side > 0 ? -beta : beta) * rcp(d0);
                const double xn = pole - beta / a;
                if (!(xn > left && xn < right)) break;
                xdF0 = x;
                dF0 = dF;
                rel0 = 0x1p-18;
                x0 = xn;
                const double step = fabs(xn - x);
                x = xn;
                if (step < 0x1p-30 * fabs(x)) break;
            }
        }
        bool fb;
        it = newton_finish(FD, side, pole, 0.0, left, right, true, true, o.max_iter, left, right,
                           fb, dF0, &itd, x0, -sg * rho, xdF0, rel0);
    } else {
        double mid = 0.5 * (left + right);
        while (right - left > TWO_EPS * fabs(mid) && it < o.max_iter) {
            const double phi = PHI(mid);
            if ((phi > 0.0) == (dir > 0)) left = mid;
            else right = mid;
            mid = 0.5 * (left + right);
            ++it;
        }
    }
    const double nu = right;
    res.mu = 1.0 / nu;
    res.lam = shift + res.mu;
    res.iters = it;
    res.iters_d = itd;
    res.flags |= (it >= o.max_iter) ? 16 : 0;
    return res;
}

}  // namespace ae
