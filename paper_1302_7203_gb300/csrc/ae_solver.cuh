// ae_solver.cuh -- one eigenpair per warp: shift selection (Algorithm 1),
// the inverse of the shifted arrowhead with its element b in double-double
// (Algorithm 2, Eq. invAi / b_ob, Theorem 6), bisection for the inverse's
// extreme eigenvalue (Algorithm 3) and the Remark 1 / Remark 2(b) solve on a
// DPR1 inverse (A - sigma I)^{-1}.
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
#pragma once
#include "ae_device.cuh"

namespace ae {

struct SolveOpts {
    int max_iter;
    int precision;
};

struct EigResult {
    double sigma;   // shift value (a pole, or a non-pole shift for remedies)
    double mu;      // lambda = sigma + mu
    double lam;
    double b;       // element b of the shifted inverse (NaN for DPR1 solves)
    double Kb;      // K_b of Eq. (K2)
    int pole;       // reduced pole index of the shift, -1 if none
    int iters;      // FP64 bisection steps
    int flags;
};

// Poles and spikes of a reduced arrowhead held in device memory.
struct ArrowPoles {
    int m;
    const double *__restrict__ pd;   // poles, strictly decreasing
    const double *__restrict__ pz;   // zeta_j > 0
    const double *__restrict__ pz2;  // fl(zeta_j^2)
    double alpha;
    // FP32 copies for the opening bracket: poles split hi + lo after scaling
    // by ds, and zeta^2 scaled by zs (ds, zs powers of two); null when absent
    const float *__restrict__ pdh;
    const float *__restrict__ pdl;
    const float *__restrict__ pz2f;
    double ds, zs;

    __device__ __forceinline__ double pole(int j) const { return __ldg(pd + j); }
    // p_j - shift in double; `i` is the shift's pole index (-1: not a pole)
    __device__ __forceinline__ double shifted(int j, double shift, int) const {
        return __ldg(pd + j) - shift;
    }
    __device__ __forceinline__ dd shifted_dd(int j, double shift, int) const {
        return two_sum(__ldg(pd + j), -shift);
    }
    __device__ __forceinline__ double z2(int j) const { return __ldg(pz2 + j); }
    __device__ __forceinline__ double zabs(int j) const { return __ldg(pz + j); }
    __device__ __forceinline__ dd z2_dd(int j) const {
        double z = __ldg(pz + j);
        return two_prod(z, z);
    }
    // a = alpha - shift, exact
    __device__ __forceinline__ dd a_dd(double shift, int) const { return two_sum(alpha, -shift); }
    // scaled shifted difference (p_j - shift) * ds in FP32 from the hi/lo split
    __device__ __forceinline__ float shifted_f32(int j, float sh, float sl) const {
        return (__ldg(pdh + j) - sh) + (__ldg(pdl + j) - sl);
    }
    __device__ __forceinline__ float z2f(int j) const { return __ldg(pz2f + j); }
    __device__ __forceinline__ bool has_f32() const { return pdh != nullptr; }
};

__device__ __forceinline__ float rcp_f32(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// FP32 analogue of secular_sum on scaled data:
// T(y) = sum_{j != skip} zz_j / (D_j (1 - y D_j)),  D_j = (p_j - shift) ds sc,
// zz_j = zeta_j^2 zs.  With x = s y and s = ds sc:  S(x) = s T(y) / zs.
template <class P>
__device__ __forceinline__ float secular_sum_f32(const P &R, float sh, float sl, float sc,
                                                 int skip, float y, int lane) {
    float acc0 = 0.f, acc1 = 0.f;
    int j = lane;
    for (; j + 32 < R.m; j += 64) {
        if (j != skip) {
            const float D = R.shifted_f32(j, sh, sl) * sc;
            const float t = fmaf(-y, D, 1.f);
            acc0 = fmaf(R.z2f(j), rcp_f32(D * t), acc0);
        }
        const int j2 = j + 32;
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
    float v = acc0 + acc1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// S(x) = sum_{j != skip} zeta_j^2 / (delta_j (1 - x delta_j)), delta_j = p_j - shift
template <class P>
__device__ __forceinline__ double secular_sum(const P &R, double shift, int skip, double x,
                                              int lane) {
    double acc0 = 0.0, acc1 = 0.0;
    int j = lane;
    for (; j + 32 < R.m; j += 64) {
        if (j != skip) {
            double dj = R.shifted(j, shift, skip);
            double t = fma(-x, dj, 1.0);
            acc0 = fma(R.z2(j), rcp(dj * t), acc0);
        }
        int j2 = j + 32;
        if (j2 != skip) {
            double dj = R.shifted(j2, shift, skip);
            double t = fma(-x, dj, 1.0);
            acc1 = fma(R.z2(j2), rcp(dj * t), acc1);
        }
    }
    if (j < R.m && j != skip) {
        double dj = R.shifted(j, shift, skip);
        double t = fma(-x, dj, 1.0);
        acc0 = fma(R.z2(j), rcp(dj * t), acc0);
    }
    return warp_sum(acc0 + acc1);
}

// Algorithm 1, first part: the shift pole i and the side (+1: lambda > p_i).
template <class P>
__device__ __forceinline__ void select_shift(const P &R, int k, int lane, int &i, int &side) {
    const int m = R.m;
    if (k == 0) {
        i = 0; side = +1;
    } else if (k == m) {
        i = m - 1; side = -1;
    } else {
        const double sk = R.pole(k);
        const double middle = 0.5 * R.shifted(k - 1, sk, k);
        const dd a = R.a_dd(sk, k);
        double acc = 0.0;
        for (int j = lane; j < m; j += 32)
            acc = fma(R.z2(j), rcp(R.shifted(j, sk, k) - middle), acc);
        const double F = (a.hi - middle) - warp_sum(acc);
        if (F < 0.0) { i = k; side = +1; }
        else { i = k - 1; side = -1; }
    }
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
};

template <class P>
__device__ __forceinline__ PassA pass_a(const P &R, double shift, int skip, double wscale,
                                        int lane) {
    dd s1 = {0.0, 0.0}, s2 = {0.0, 0.0};
    double pmax = -INFINITY, pmin = INFINITY, up = -INFINITY, lo = INFINITY, wsum = 0.0,
           usq = 0.0;
    for (int j = lane; j < R.m; j += 32) {
        if (j == skip) continue;
        const dd del = R.shifted_dd(j, shift, skip);
        const dd t = dd_div(R.z2_dd(j), del);
        if (del.hi > 0.0) s1 = dd_add_same(s1, t);
        else s2 = dd_add_same(s2, t);
        const double p = rcp(del.hi);
        const double aw = R.zabs(j) * fabs(p);
        pmax = fmax(pmax, p);
        pmin = fmin(pmin, p);
        up = fmax(up, fma(aw, wscale, p));
        lo = fmin(lo, fma(-aw, wscale, p));
        wsum += aw;
        usq = fma(aw, aw, usq);
    }
    s1 = warp_sum_dd(s1);
    s2 = warp_sum_dd(s2);
    PassA A;
    A.pmax = warp_max(pmax);
    A.pmin = warp_min(pmin);
    A.up = warp_max(up);
    A.lo = warp_min(lo);
    A.wsum = warp_sum(wsum);
    A.usq = warp_sum(usq);
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

// F(x) of the inverse's Pick function in FP64 (one evaluation, all terms)
template <class P>
__device__ __forceinline__ double pick_inverse_f64(const P &R, double sigma, int i, double b,
                                                   double c, double x, int lane) {
    const double S = secular_sum(R, sigma, i, x, lane);
    return (b - x) - c * (S - rcp(x));
}

// Narrow [left, right] (which holds the zero nu of F) with FP32 bisection, then
// verify the new ends in FP64: F(l) > 0 >= F(r).  Returns false (bracket
// unchanged) when the FP32 data cannot represent the problem or the check fails.
template <class P>
__device__ bool fp32_bracket(const P &R, double sigma, int i, double b, double c, double &left,
                             double &right, int lane) {
    const double big = fmax(fabs(left), fabs(right));
    if (!(big > 0.0) || !isfinite(big)) return false;
    const double s = ldexp(1.0, ilogb(big));          // x = s y, |y| <= 2
    const double scd = s / R.ds;                        // D_j = (p_j - sigma) ds * scd
    if (!(scd > 0x1p-120 && scd < 0x1p120)) return false;
    const double ss = sigma * R.ds;
    const float sh = (float)ss;
    const float sl = (float)(ss - (double)sh);
    if (!isfinite(sh)) return false;
    const float sc = (float)scd;
    const double K = c * s / R.zs;                      // F = G(x) - K T(y)
    double l = left, r = right;
    for (int it = 0; it < 80; ++it) {
        const double mid = 0.5 * (l + r);
        if (r - l <= 0x1p-20 * fabs(mid)) break;
        const float y = (float)(mid / s);
        const double x = s * (double)y;                 // the point actually evaluated
        if (!(x > l && x < r)) break;
        const float T = secular_sum_f32(R, sh, sl, sc, i, y, lane);
        const double F = (b - x) + c * rcp(x) - K * (double)T;
        if (F > 0.0) l = x;
        else r = x;
    }
    // widen by the bracket width and check both ends in FP64
    const double w = r - l;
    const double L = fmax(left, l - w), Rr = fmin(right, r + w);
    if (L > left && !(pick_inverse_f64(R, sigma, i, b, c, L, lane) > 0.0)) return false;
    if (Rr < right && !(pick_inverse_f64(R, sigma, i, b, c, Rr, lane) <= 0.0)) return false;
    left = L;
    right = Rr;
    return true;
}

// Algorithm 2 + 3 for the shift pole i on `side`, then lambda = sigma + 1/nu.
template <class P>
__device__ EigResult solve_shifted(const P &R, int i, int side, const SolveOpts &o, int lane) {
    EigResult res;
    const double sigma = R.pole(i);
    const double zi = R.zabs(i);
    const double wz = 1.0 / zi;         // w_zeta
    const double c = wz * wz;           // 1/zeta_i^2
    const PassA A = pass_a(R, sigma, i, wz, lane);
    // b = (P - Q) / zeta_i^2 in double-double (Theorem 6), rounded once
    const dd num = dd_add(A.P, dd_neg(A.Q));
    const double b = dd_div(num, two_prod(zi, zi)).hi;
    res.Kb = (A.P.hi + A.Q.hi) / fabs(num.hi);
    res.b = b;
    // Gershgorin bracket of Algorithm 3 for the inverse: diagonal {1/delta_j, 0},
    // spikes {w_j, w_zeta}, corner b.
    const double norm1 = fma(A.wsum, wz, wz);
    double left, right;
    if (side > 0) {
        left = fmax(A.pmax, 0.0);
        right = fmax(fmax(A.up, wz), b + norm1);
    } else {
        right = fmin(A.pmin, 0.0);
        left = fmin(fmin(A.lo, -wz), b - norm1);
    }
    if (o.precision == 1 && R.has_f32()) {
        // FP32 opening bracket on a power-of-two rescaled copy (x = s y), then
        // an FP64 check of both ends; on failure keep the Gershgorin bracket.
        res.flags = 0;
        if (!fp32_bracket(R, sigma, i, b, c, left, right, lane)) res.flags = 64;
    } else {
        res.flags = 0;
    }
    int it = 0;
    double mid = 0.5 * (left + right);
    while (right - left > TWO_EPS * fabs(mid) && it < o.max_iter) {
        const double S = secular_sum(R, sigma, i, mid, lane);
        const double F = (b - mid) - c * (S - rcp(mid));
        if (F > 0.0) left = mid;
        else right = mid;
        mid = 0.5 * (left + right);
        ++it;
    }
    const double nu = right;            // Algorithm 3 returns the right end
    res.sigma = sigma;
    res.mu = 1.0 / nu;
    res.lam = sigma + res.mu;
    res.pole = i;
    res.iters = it;
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
template <class P>
__device__ EigResult solve_dpr1_shift(const P &R, double shift, const SolveOpts &o, int lane) {
    EigResult res;
    res.sigma = shift;
    res.pole = -1;
    res.b = NAN;
    res.flags = 0;
    const PassA A = pass_a(R, shift, -1, 1.0, lane);
    const dd T = dd_add(A.P, dd_neg(A.Q));   // a - z^T (D - shift)^{-1} z = -T
    res.Kb = (A.P.hi + A.Q.hi) / fabs(T.hi);
    if (T.hi == 0.0) {                       // numerically singular: lambda = shift
        res.mu = 0.0;
        res.lam = shift;
        res.iters = 0;
        res.flags = 32;
        return res;
    }
    const double rho = -1.0 / T.hi;
    const double usq = A.usq + 1.0;          // ||u||^2
    double left, right;
    if (rho > 0.0) {
        left = fmax(A.pmax, 0.0);
        right = fma(rho, usq, left);
    } else {
        right = fmin(A.pmin, 0.0);
        left = fma(rho, usq, right);
    }
    int it = 0;
    double mid = 0.5 * (left + right);
    while (right - left > TWO_EPS * fabs(mid) && it < o.max_iter) {
        const double S = secular_sum(R, shift, -1, mid, lane);
        const double phi = fma(rho, S - rcp(mid), 1.0);
        // rho > 0: phi increases through the zero; rho < 0: it decreases
        if ((phi > 0.0) == (rho > 0.0)) right = mid;
        else left = mid;
        mid = 0.5 * (left + right);
        ++it;
    }
    const double nu = right;
    res.mu = 1.0 / nu;
    res.lam = shift + res.mu;
    res.iters = it;
    res.flags = (it >= o.max_iter) ? 16 : 0;
    return res;
}

}  // namespace ae
