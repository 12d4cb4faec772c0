/*
 * arrow_oracle.c -- CPU oracle for the arrowhead eigen-solver.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load or call this library.
 * It shares no code with the CUDA path (no headers, helpers or constants):
 * it is a plain, slow, independent statement of WHAT the method computes.
 *
 * What it computes (Jakovcevic Stor, Slapnicar, Barlow, "Accurate eigenvalue
 * decomposition of arrowhead matrices and applications"):
 *
 *  - Reduction (Sec. 1): rows with zeta == 0 are deflated (d_i, e_i); rows
 *    with exactly equal d are folded by rotations in their plane (the run's
 *    first row keeps zeta' = sqrt(sum zeta^2), the others are deflated);
 *    the rest are ordered d_1 > d_2 > ... (stable: ties by original index).
 *  - Eigenvalues of the reduced matrix: the zeros of the Pick function
 *        f(l) = alpha - l - sum_j zeta_j^2 / (d_j - l)            (Eq. Pick)
 *    one in each interval given by the interlacing property (Eq. interlace),
 *    the exterior ones inside Gershgorin's bounds (as in Algorithm 3).
 *  - Eigenvectors v = x / ||x||, x = [(D - l I)^{-1} z ; -1]    (Eq. Aeigenvec)
 *    with the caller's signed z, so sign normalisation is implicit.
 *  - DPR1  M = D + rho u u^T (Sec. 6.3): zeros of 1 + rho sum u_j^2/(d_j - l),
 *    vectors q ~ (D - l I)^{-1} u, solved directly (not through the
 *    arrowhead reduction the method uses).
 *  - Hermitian arrowhead [D z; z^* alpha] (Sec. 6.1) and the non-symmetric
 *    [D zc; zr^T alpha] (the Remark of Sec. 6.1): zeros of the same Pick
 *    function with weights |zeta|^2, resp. zc zr, exact in double-double;
 *    vectors from the rows of (C - l I) u = 0 directly.
 *  - SVD of B = [D z; 0 alpha] (Sec. 6.2): eigen-decomposition of the
 *    arrowhead B^T B = [D^2, D z; z^T D, alpha^2 + z^T z], singular values
 *    sqrt(l), right vectors v, left vectors u_j = s v_j / d_j, u_n = alpha v_n / s.
 *
 * How: every zero is found by bisection in double-double arithmetic on the
 * ORIGINAL secular function, written in coordinates shifted to the nearer end
 * of its interval so that each shifted difference d_j - sigma is exact
 * (TwoSum).  Each evaluation carries a running error bound; bisection stops
 * when the bracket reaches ~2^-103 relative or the sign is no longer certain,
 * and the final bracket width is reported as the oracle's own error bound.
 * It never forms the inverse of the shifted matrix and never computes the
 * element b, unlike the method it checks (except oracle_inverse_element,
 * which evaluates that element by its definition for pinning).
 *
 * Brute force for tiny inputs: cyclic Jacobi (symmetric) and one-sided
 * Jacobi (SVD) in IEEE binary128 (Golub & Van Loan, Sec. 8.5).
 *
 * Double-double building blocks: TwoSum (Knuth, TAOCP vol. 2, 4.2.2),
 * FastTwoSum (Dekker 1971), TwoProd via fused multiply-add.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* double-double arithmetic                                            */
/* ------------------------------------------------------------------ */
typedef struct { double hi, lo; } dd;

static dd dd_from(double a) { dd r = {a, 0.0}; return r; }

static dd two_sum(double a, double b) {
    double s = a + b;
    double bb = s - a;
    double e = (a - (s - bb)) + (b - bb);
    dd r = {s, e};
    return r;
}

static dd fast_two_sum(double a, double b) {
    double s = a + b;
    double e = b - (s - a);
    dd r = {s, e};
    return r;
}

static dd two_prod(double a, double b) {
    double p = a * b;
    double e = fma(a, b, -p);
    dd r = {p, e};
    return r;
}

static dd dd_add(dd x, dd y) {
    dd s = two_sum(x.hi, y.hi);
    dd t = two_sum(x.lo, y.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}

static dd dd_neg(dd x) { dd r = {-x.hi, -x.lo}; return r; }
static dd dd_sub(dd x, dd y) { return dd_add(x, dd_neg(y)); }

static dd dd_mul(dd x, dd y) {
    dd p = two_prod(x.hi, y.hi);
    p.lo += x.hi * y.lo + x.lo * y.hi;
    return fast_two_sum(p.hi, p.lo);
}

static dd dd_mul_d(dd x, double b) {
    dd p = two_prod(x.hi, b);
    p.lo += x.lo * b;
    return fast_two_sum(p.hi, p.lo);
}

/* long division: three partial quotients */
static dd dd_div(dd x, dd y) {
    double q1 = x.hi / y.hi;
    dd r = dd_sub(x, dd_mul_d(y, q1));
    double q2 = r.hi / y.hi;
    r = dd_sub(r, dd_mul_d(y, q2));
    double q3 = r.hi / y.hi;
    dd q = fast_two_sum(q1, q2);
    return dd_add(q, dd_from(q3));
}

static dd dd_sqrt(dd x) {
    if (x.hi <= 0.0) return dd_from(0.0);
    double s = sqrt(x.hi);
    dd r = dd_sub(x, two_prod(s, s));
    return fast_two_sum(s, r.hi / (2.0 * s));
}

static dd dd_abs(dd x) { return x.hi < 0.0 ? dd_neg(x) : x; }
static dd dd_half(dd x) { dd r = {0.5 * x.hi, 0.5 * x.lo}; return r; }
static int dd_lt(dd x, dd y) { return x.hi < y.hi || (x.hi == y.hi && x.lo < y.lo); }
static int dd_le(dd x, dd y) { return x.hi < y.hi || (x.hi == y.hi && x.lo <= y.lo); }

/* unit roundoff of double and a safe per-operation bound for dd results */
#define U53 1.1102230246251565e-16  /* 2^-53 */
#define U2 (U53 * U53)

/* ------------------------------------------------------------------ */
/* reduction of an arrowhead (or DPR1) input, Sec. 1                  */
/* ------------------------------------------------------------------ */
typedef struct {
    int n1;          /* number of rows of D (n-1 for an arrowhead, n for DPR1) */
    int m;           /* number of reduced poles */
    int ndefl;       /* number of deflated rows */
    int *order;      /* sorted position -> original row (d desc, index asc) */
    int *kind;       /* per original row: 0 pole head, 1 zero-deflated, 2 run-deflated */
    int *run_head;   /* per original row (kind 0/2): original row of the run's head */
    int *run_pos;    /* per original row (kind 0/2): position in its run */
    int *pole_row;   /* reduced pole j -> original row of its head */
    double *pole_d;  /* reduced pole values, strictly decreasing */
    dd *pole_c;      /* reduced zeta'^2 = sum of zeta^2 over the run (dd) */
    int *defl_row;   /* deflated rows, in sorted order */
} reduction;

static const double *g_sort_key;
static int cmp_desc(const void *a, const void *b) {
    int i = *(const int *)a, j = *(const int *)b;
    double x = g_sort_key[i], y = g_sort_key[j];
    if (x > y) return -1;
    if (x < y) return 1;
    return (i > j) - (i < j);
}

static void free_reduction(reduction *R) {
    free(R->order); free(R->kind); free(R->run_head); free(R->run_pos);
    free(R->pole_row); free(R->pole_d); free(R->pole_c); free(R->defl_row);
}

/* key[] are the pole values used for ordering and equality; z[] the spikes
   (|zeta| for the Hermitian and non-symmetric forms).  z2[], when given, are
   the exact squares zeta_r^2 in double-double (|zeta|^2 of a complex spike,
   or the product of a non-symmetric pair); else zeta_r^2 = TwoProd(z_r, z_r). */
static int reduce2(int n1, const double *key, const double *z, const dd *z2, reduction *R) {
    memset(R, 0, sizeof(*R));
    R->n1 = n1;
    int cap = n1 > 0 ? n1 : 1;
    R->order = malloc(sizeof(int) * cap);
    R->kind = malloc(sizeof(int) * cap);
    R->run_head = malloc(sizeof(int) * cap);
    R->run_pos = malloc(sizeof(int) * cap);
    R->pole_row = malloc(sizeof(int) * cap);
    R->pole_d = malloc(sizeof(double) * cap);
    R->pole_c = malloc(sizeof(dd) * cap);
    R->defl_row = malloc(sizeof(int) * cap);
    for (int r = 0; r < n1; r++) R->order[r] = r;
    g_sort_key = key;
    qsort(R->order, n1, sizeof(int), cmp_desc);
    int m = 0, nd = 0;
    int last_head = -1;       /* sorted run head (original row) */
    int run_len = 0;
    for (int s = 0; s < n1; s++) {
        int r = R->order[s];
        R->run_head[r] = -1;
        R->run_pos[r] = 0;
        if (z[r] == 0.0) {            /* +0.0 and -0.0 alike */
            R->kind[r] = 1;
            R->defl_row[nd++] = r;
            continue;
        }
        dd sq = z2 ? z2[r] : two_prod(z[r], z[r]);
        if (last_head >= 0 && key[r] == key[last_head]) {
            R->kind[r] = 2;
            R->run_head[r] = last_head;
            R->run_pos[r] = run_len++;
            R->defl_row[nd++] = r;
            R->pole_c[m - 1] = dd_add(R->pole_c[m - 1], sq);
        } else {
            R->kind[r] = 0;
            R->run_head[r] = r;
            R->run_pos[r] = 0;
            run_len = 1;
            last_head = r;
            R->pole_row[m] = r;
            R->pole_d[m] = key[r];
            R->pole_c[m] = sq;
            m++;
        }
    }
    R->m = m;
    R->ndefl = nd;
    return 0;
}

static int reduce(int n1, const double *key, const double *z, reduction *R) {
    return reduce2(n1, key, z, NULL, R);
}

/* ------------------------------------------------------------------ */
/* secular functions in shifted coordinates                           */
/* ------------------------------------------------------------------ */
/*
 * A secular problem: poles p_j (reduced, decreasing), weights c_j >= 0 (dd),
 * and the form of the function:
 *   ARROW:  f(mu) = a - mu - sum_j c_j/(delta_j - mu)     (decreasing in mu)
 *   DPR1:   f(mu) = 1 + rho * sum_j c_j/(delta_j - mu)    (monotone, sign(rho))
 * with delta_j = p_j - sigma exact (dd) and a = alpha - sigma (dd).
 */
enum { KIND_ARROW = 0, KIND_DPR1 = 1 };

typedef struct {
    int kind;
    int m;
    const dd *delta;   /* shifted poles, exact */
    const dd *c;       /* weights */
    dd a;              /* ARROW: alpha - sigma */
    double rho;        /* DPR1 */
} secular;

/* value at mu and a bound on its absolute rounding error */
static dd secular_eval(const secular *S, dd mu, double *bound) {
    dd sum = dd_from(0.0);
    double mag = 0.0;
    for (int j = 0; j < S->m; j++) {
        dd den = dd_sub(S->delta[j], mu);
        dd t = dd_div(S->c[j], den);
        sum = dd_add(sum, t);
        mag += fabs(t.hi);
    }
    double safety = (32.0 + 8.0 * (S->m + 2)) * U2;
    if (S->kind == KIND_ARROW) {
        dd f = dd_sub(dd_sub(S->a, mu), sum);
        *bound = safety * (fabs(S->a.hi) + fabs(mu.hi) + mag) * 1.0000001;
        return f;
    } else {
        dd f = dd_add(dd_from(1.0), dd_mul_d(sum, S->rho));
        *bound = safety * (1.0 + fabs(S->rho) * mag) * 1.0000001;
        return f;
    }
}

/* +1 when the function decreases in mu, -1 when it increases */
static int secular_dir(const secular *S) {
    if (S->kind == KIND_ARROW) return 1;
    return S->rho > 0 ? -1 : 1;
}

/*
 * Find the zero mu = sgn * t, t in (0, T], of a secular function that is
 * infinite with the "far" sign at t -> 0+ (a pole at mu = 0) and has the
 * opposite sign at t = T.  G(t) := sgn * dir * f(sgn*t) > 0 below the zero.
 * Returns mu and a relative error bound on it.
 */
static dd bisect_zero(const secular *S, int sgn, dd T, double *relerr, int *iters) {
    int dir = secular_dir(S);
    double bound;
    int it = 0;
    dd hi = T;
    /* make sure G(T) <= 0; widen if the caller's bound was not safe */
    for (int guard = 0; guard < 64; guard++) {
        dd mu = sgn > 0 ? hi : dd_neg(hi);
        dd f = secular_eval(S, mu, &bound);
        it++;
        double G = sgn * dir * f.hi;
        if (G <= 0.0) break;
        if (!isfinite(G)) { *relerr = INFINITY; if (iters) *iters = it; return mu; }
        hi = dd_mul_d(hi, 2.0);
    }
    /* geometric phase from a tiny positive lower end, chosen so that no
       term c_j / (delta_j - mu) can overflow */
    double cmax = 0.0;
    for (int j = 0; j < S->m; j++) if (S->c[j].hi > cmax) cmax = S->c[j].hi;
    double lo0 = ldexp(1.0, -1020);
    if (ldexp(cmax, -1000) > lo0) lo0 = ldexp(cmax, -1000);
    if (ldexp(hi.hi, -1000) > lo0) lo0 = ldexp(hi.hi, -1000);
    dd lo = dd_from(lo0);
    {
        dd mu = sgn > 0 ? lo : dd_neg(lo);
        dd f = secular_eval(S, mu, &bound);
        it++;
        double G = sgn * dir * f.hi;
        if (!(G > 0.0)) { /* zero below the representable search range */
            *relerr = INFINITY;
            if (iters) *iters = it;
            return mu;
        }
    }
    while (hi.hi > 4.0 * lo.hi) {
        int e = (ilogb(lo.hi) + ilogb(hi.hi)) / 2;
        dd mid = dd_from(ldexp(1.0, e));
        if (!dd_lt(lo, mid) || !dd_lt(mid, hi)) break;
        dd mu = sgn > 0 ? mid : dd_neg(mid);
        dd f = secular_eval(S, mu, &bound);
        it++;
        double G = sgn * dir * f.hi;
        if (fabs(f.hi) <= bound) { /* undecidable: keep the bracket */
            *relerr = (hi.hi - lo.hi) / lo.hi;
            if (iters) *iters = it;
            return mu;
        }
        if (G > 0.0) lo = mid; else hi = mid;
    }
    /* arithmetic phase */
    dd mid = dd_half(dd_add(lo, hi));
    for (int k = 0; k < 400; k++) {
        dd w = dd_sub(hi, lo);
        if (w.hi <= ldexp(mid.hi, -103)) break;
        if (!dd_lt(lo, mid) || !dd_lt(mid, hi)) break;
        dd mu = sgn > 0 ? mid : dd_neg(mid);
        dd f = secular_eval(S, mu, &bound);
        it++;
        if (fabs(f.hi) <= bound) break;
        double G = sgn * dir * f.hi;
        if (G > 0.0) lo = mid; else hi = mid;
        mid = dd_half(dd_add(lo, hi));
    }
    *relerr = dd_sub(hi, lo).hi / lo.hi;
    if (iters) *iters = it;
    return sgn > 0 ? mid : dd_neg(mid);
}

/*
 * Plain bisection on [lo, hi] for a secular function whose zero lies inside:
 * G(x) := dir * f(x) > 0 below the zero.  Used to refine a zero in unshifted
 * coordinates when the shifted value sigma + mu cancels (an eigenvalue near 0,
 * the cases singled out after Theorem C1).  On exit [lo, hi] still contains
 * the zero; returns the midpoint.
 */
static dd bisect_interval(const secular *S, dd lo, dd hi, double *width) {
    int dir = secular_dir(S);
    double bound;
    dd mid = dd_half(dd_add(lo, hi));
    for (int k = 0; k < 600; k++) {
        dd w = dd_sub(hi, lo);
        double scale = fmax(fabs(lo.hi), fabs(hi.hi));
        if (w.hi <= ldexp(scale, -104)) break;
        if (!dd_lt(lo, mid) || !dd_lt(mid, hi)) break;
        dd f = secular_eval(S, mid, &bound);
        if (fabs(f.hi) <= bound) break;
        if (dir * f.hi > 0.0) lo = mid; else hi = mid;
        mid = dd_half(dd_add(lo, hi));
    }
    *width = dd_sub(hi, lo).hi;
    return mid;
}

/* G at x for a secular function, with the sign certainty flag */
static int secular_side(const secular *S, dd x) {
    double bound;
    dd f = secular_eval(S, x, &bound);
    int dir = secular_dir(S);
    if (fabs(f.hi) <= bound) return 0;
    return dir * f.hi > 0.0 ? 1 : -1;   /* +1: x below the zero */
}

/* ------------------------------------------------------------------ */
/* one eigenvalue of a reduced secular problem                        */
/* ------------------------------------------------------------------ */
typedef struct {
    int pole;        /* index of the shift pole in the reduced list, -1 if none */
    double sigma;    /* the shift (a pole value, or 0 after refinement) */
    dd mu;           /* zero in shifted coordinates: lambda = sigma + mu */
    double relerr;   /* bound on |lambda error| / |lambda| */
    double abserr;   /* bound on |lambda error| */
    int iters;
} zero_info;

/*
 * If sigma + mu cancels, (|sigma| + |mu|) / |lambda| > 3 (Theorem C1 bounds this
 * quotient by 3 otherwise), find the zero again in unshifted coordinates,
 * delta_j = p_j, inside the bracket the shifted solve guarantees.
 * `unshifted` holds delta_j = p_j (exact) and a = alpha.
 */
static void refine_if_cancelled(zero_info *Z, const secular *unshifted, dd lim_lo, dd lim_hi) {
    dd lam = dd_add(dd_from(Z->sigma), Z->mu);
    double q = (fabs(Z->sigma) + fabs(Z->mu.hi)) / fabs(lam.hi);
    double abserr = (fabs(Z->sigma) + fabs(Z->mu.hi)) * Z->relerr + 4 * U2 * fabs(lam.hi);
    Z->abserr = abserr;
    Z->relerr = (lam.hi == 0.0) ? INFINITY : abserr / fabs(lam.hi);
    if (!(q > 3.0) || !isfinite(abserr)) return;
    double w = 4.0 * abserr + 1e-300;
    dd lo, hi;
    for (int tries = 0; tries < 200; tries++, w *= 4.0) {
        lo = dd_sub(lam, dd_from(w));
        hi = dd_add(lam, dd_from(w));
        if (dd_lt(lo, lim_lo)) lo = lim_lo;
        if (dd_lt(lim_hi, hi)) hi = lim_hi;
        int sl = secular_side(unshifted, lo), sh = secular_side(unshifted, hi);
        if (sl > 0 && sh < 0) break;
    }
    double width;
    dd l2 = bisect_interval(unshifted, lo, hi, &width);
    Z->sigma = 0.0;
    Z->mu = l2;
    Z->pole = -1;
    Z->abserr = width + 4 * U2 * fabs(l2.hi);
    Z->relerr = (l2.hi == 0.0) ? INFINITY : Z->abserr / fabs(l2.hi);
}

/*
 * Interval of zero k:
 *   ARROW (m poles, m+1 zeros, f decreasing): zero k in (p_k, p_{k-1}),
 *     with p_{-1} = +Gershgorin bound and p_m = -Gershgorin bound.
 *   DPR1 rho>0 (m zeros): zero k in (p_k, p_{k-1}), p_{-1} = p_0 + rho*sum c.
 *   DPR1 rho<0: zero k in (p_{k+1}, p_k), p_m = p_{m-1} + rho*sum c.
 * The nearer end is chosen by the sign of f at the midpoint (dd).
 */
static zero_info solve_zero(int kind, int m, const double *p, const dd *c, dd alpha,
                            double rho, int k, dd *delta_buf) {
    zero_info Z;
    memset(&Z, 0, sizeof(Z));
    secular S;
    S.kind = kind; S.m = m; S.c = c; S.rho = rho; S.delta = delta_buf;
    int upper, lower;   /* pole indices bounding the interval, -1 = none */
    if (kind == KIND_ARROW || rho > 0) {
        upper = k - 1;             /* p_{k-1} */
        lower = k < m ? k : -1;    /* p_k */
    } else {
        upper = k;                 /* p_k */
        lower = k + 1 < m ? k + 1 : -1;
    }
    double sumc = 0.0, maxc = 0.0;
    for (int j = 0; j < m; j++) { sumc += c[j].hi; }
    (void)maxc;
    int sgn;
    int pole;
    dd T;
    if (upper >= 0 && lower >= 0) {
        /* interior: midpoint test in coordinates shifted to the lower pole */
        double pl = p[lower], pu = p[upper];
        for (int j = 0; j < m; j++) delta_buf[j] = two_sum(p[j], -pl);
        S.a = dd_sub(alpha, dd_from(pl));
        dd gap = two_sum(pu, -pl);
        dd h = dd_half(gap);
        double bound;
        dd f = secular_eval(&S, h, &bound);
        int dir = secular_dir(&S);
        /* G(h) < 0 (for t measured up from the lower pole) => zero below h */
        double G = dir * f.hi;
        if (fabs(f.hi) > bound && G < 0.0) {
            pole = lower; sgn = +1; T = h;
        } else if (fabs(f.hi) > bound) {
            pole = upper; sgn = -1; T = h;
        } else {
            /* tie (the zero is at the midpoint within rounding): the upper
               pole, with a bracket reaching three quarters of the gap */
            pole = upper; sgn = -1; T = dd_add(h, dd_half(h));
        }
    } else if (lower >= 0) {
        /* zero above the top pole */
        pole = lower; sgn = +1;
        double pl = p[lower];
        double t = 0.0;
        if (kind == KIND_ARROW) {
            double a = alpha.hi - pl;
            double r = 0.0;
            for (int j = 0; j < m; j++) {
                double dj = p[j] - pl + sqrt(c[j].hi);
                if (dj > t) t = dj;
                r += sqrt(c[j].hi);
            }
            if (a + r > t) t = a + r;
        } else {
            t = fabs(rho) * sumc;
        }
        t = t * (1.0 + 1e-9) + ldexp(fabs(pl), -40) + 1e-300;
        T = dd_from(t);
    } else {
        /* zero below the bottom pole */
        pole = upper; sgn = -1;
        double pu = p[upper];
        double t = 0.0;
        if (kind == KIND_ARROW) {
            double a = alpha.hi - pu;
            double r = 0.0;
            for (int j = 0; j < m; j++) {
                double dj = sqrt(c[j].hi) - (p[j] - pu);
                if (dj > t) t = dj;
                r += sqrt(c[j].hi);
            }
            if (r - a > t) t = r - a;
        } else {
            t = fabs(rho) * sumc;
        }
        t = t * (1.0 + 1e-9) + ldexp(fabs(pu), -40) + 1e-300;
        T = dd_from(t);
    }
    double sigma = p[pole];
    for (int j = 0; j < m; j++) delta_buf[j] = two_sum(p[j], -sigma);
    S.a = dd_sub(alpha, dd_from(sigma));
    Z.pole = pole;
    Z.sigma = sigma;
    Z.mu = bisect_zero(&S, sgn, T, &Z.relerr, &Z.iters);
    /* refinement in unshifted coordinates when sigma + mu cancels; the
       zero stays inside its interlacing interval */
    for (int j = 0; j < m; j++) delta_buf[j] = dd_from(p[j]);
    secular U0 = S;
    U0.a = alpha;
    double big = 0.0;
    for (int j = 0; j < m; j++) big = fmax(big, fabs(p[j]));
    big = (big + fabs(alpha.hi) + fabs(rho) * sumc + 1.0) * 1e30;
    dd lim_lo = lower >= 0 ? dd_from(p[lower]) : dd_from(-big);
    dd lim_hi = upper >= 0 ? dd_from(p[upper]) : dd_from(big);
    refine_if_cancelled(&Z, &U0, lim_lo, lim_hi);
    return Z;
}

/* ------------------------------------------------------------------ */
/* output assembly: merge computed and deflated eigenvalues           */
/* ------------------------------------------------------------------ */
/* slot[pos] = k >= 0 : computed zero k ; slot[pos] = -1 - t : deflated row t */
static void merge_order(int ncomp, const double *lam_comp, int ndefl,
                        const double *lam_defl, int *slot) {
    int a = 0, b = 0, pos = 0;
    while (a < ncomp || b < ndefl) {
        if (b < ndefl && (a >= ncomp || lam_defl[b] >= lam_comp[a])) {
            slot[pos++] = -1 - b; b++;
        } else {
            slot[pos++] = a; a++;
        }
    }
}

/* Helmert-type vector of a run-deflated row (signed z): rows of its run
   before it get -z_q z_l / (R_{m-1} R_m), the row itself R_{m-1}/R_m. */
static void run_vector(const reduction *R, const double *z, int row, int nrows,
                       double *col) {
    for (int r = 0; r < nrows; r++) col[r] = 0.0;
    int head = R->run_head[row];
    int pos = R->run_pos[row];
    /* members of the run in sorted order up to `row` */
    dd prev = dd_from(0.0);
    int s0 = 0;
    while (R->order[s0] != head) s0++;
    int cnt = 0;
    for (int s = s0; s < R->n1 && cnt < pos; s++) {
        int r = R->order[s];
        if (R->kind[r] == 1) continue;
        if (R->run_head[r] != head) break;
        prev = dd_add(prev, two_prod(z[r], z[r]));
        cnt++;
    }
    dd Rm1 = dd_sqrt(prev);
    dd Rm = dd_sqrt(dd_add(prev, two_prod(z[row], z[row])));
    dd den = dd_mul(Rm1, Rm);
    cnt = 0;
    for (int s = s0; s < R->n1 && cnt < pos; s++) {
        int r = R->order[s];
        if (R->kind[r] == 1) continue;
        if (R->run_head[r] != head) break;
        dd num = dd_neg(two_prod(z[row], z[r]));
        col[r] = dd_div(num, den).hi;
        cnt++;
    }
    col[row] = dd_div(Rm1, Rm).hi;
}

/* ------------------------------------------------------------------ */
/* the zeros of a reduced arrowhead and their output order            */
/* ------------------------------------------------------------------ */
typedef struct {
    reduction R;
    int n1, ncomp;
    dd *c;            /* pole weights zeta'_j^2 */
    zero_info *Z;     /* computed zeros (those wanted) */
    int *slot;        /* output position -> computed k, or -1 - t for deflated row t */
} arrow_sol;

static void arrow_sol_free(arrow_sol *A) {
    free(A->slot); free(A->Z); free(A->c);
    free_reduction(&A->R);
}

/* d, zabs: n-1 rows (zabs only decides zero spikes and, without z2, gives the
   weights); z2: exact zeta^2 (dd) or NULL.  Positions ks[0..nk) (all if NULL). */
static void arrow_solve(int n, const double *d, const double *zabs, const dd *z2, double alpha,
                        const int *ks, int nk, int nthreads, arrow_sol *A) {
    int n1 = n - 1;
    A->n1 = n1;
    reduce2(n1, d, zabs, z2, &A->R);
    int m = A->R.m;
    A->c = malloc(sizeof(dd) * (m > 0 ? m : 1));
    for (int j = 0; j < m; j++) A->c[j] = A->R.pole_c[j];
    int ncomp = m + 1;
    A->ncomp = ncomp;
    int all = (ks == NULL);
    if (all) nk = n;
    int need_all_comp = all || A->R.ndefl > 0;
    A->Z = calloc(ncomp, sizeof(zero_info));
    char *want = calloc(ncomp, 1);
    if (need_all_comp) {
        memset(want, 1, ncomp);
    } else {
        for (int i = 0; i < nk; i++) want[ks[i]] = 1;
    }
    zero_info *Z = A->Z;
    const dd *c = A->c;
    const reduction *R = &A->R;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        dd *buf = malloc(sizeof(dd) * (m > 0 ? m : 1));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int k = 0; k < ncomp; k++) {
            if (!want[k]) continue;
            if (m == 0) {
                Z[k].pole = -1; Z[k].sigma = alpha; Z[k].mu = dd_from(0.0);
                Z[k].relerr = 0.0; Z[k].abserr = 0.0;
            } else {
                Z[k] = solve_zero(KIND_ARROW, m, R->pole_d, c, dd_from(alpha), 0.0, k, buf);
            }
        }
        free(buf);
    }
    A->slot = malloc(sizeof(int) * n);
    if (need_all_comp) {
        double *lam_comp = malloc(sizeof(double) * ncomp);
        for (int k = 0; k < ncomp; k++) lam_comp[k] = dd_add(dd_from(Z[k].sigma), Z[k].mu).hi;
        double *lam_defl = malloc(sizeof(double) * (R->ndefl > 0 ? R->ndefl : 1));
        for (int t = 0; t < R->ndefl; t++) lam_defl[t] = d[R->defl_row[t]];
        merge_order(ncomp, lam_comp, R->ndefl, lam_defl, A->slot);
        free(lam_comp); free(lam_defl);
    } else {
        for (int i = 0; i < n; i++) A->slot[i] = i;
    }
    free(want);
}

/* the scalar outputs of position `pos` into entry i of the output arrays;
   returns the computed zero (or NULL for a deflated row, *row set) */
static const zero_info *arrow_scalars(const arrow_sol *A, const double *d, int pos, int i,
                                      double *lam, double *lam_lo, double *sigma_out,
                                      double *mu_hi, double *mu_lo, double *relerr,
                                      double *abserr, int *row) {
    int s = A->slot[pos];
    if (s >= 0) {
        const zero_info *zi = &A->Z[s];
        dd l = dd_add(dd_from(zi->sigma), zi->mu);
        lam[i] = l.hi;
        if (lam_lo) lam_lo[i] = l.lo;
        if (sigma_out) sigma_out[i] = zi->sigma;
        if (mu_hi) mu_hi[i] = zi->mu.hi;
        if (mu_lo) mu_lo[i] = zi->mu.lo;
        if (relerr) relerr[i] = zi->relerr;
        if (abserr) abserr[i] = zi->abserr;
        return zi;
    }
    int t = -1 - s;
    *row = A->R.defl_row[t];
    lam[i] = d[*row];
    if (lam_lo) lam_lo[i] = 0.0;
    if (sigma_out) sigma_out[i] = d[*row];
    if (mu_hi) mu_hi[i] = 0.0;
    if (mu_lo) mu_lo[i] = 0.0;
    if (relerr) relerr[i] = 0.0;
    if (abserr) abserr[i] = 0.0;
    return NULL;
}

/* the denominators (d_r - sigma) - mu of Eq. (Aeigenvec) in double-double */
static dd vec_den(const double *d, int r, const zero_info *zi) {
    return dd_sub(two_sum(d[r], -zi->sigma), zi->mu);
}

/* the run data of a run-deflated row: Rm1 = |zeta'| of the rows before it,
   Rm including it (dd), over the exact squares sq() */
static void run_norms(const reduction *R, const dd *sq, int row, dd *Rm1, dd *Rm, int *s0) {
    int head = R->run_head[row];
    int pos = R->run_pos[row];
    int s = 0;
    while (R->order[s] != head) s++;
    *s0 = s;
    dd prev = dd_from(0.0);
    int cnt = 0;
    for (; s < R->n1 && cnt < pos; s++) {
        int r = R->order[s];
        if (R->kind[r] == 1) continue;
        if (R->run_head[r] != head) break;
        prev = dd_add(prev, sq[r]);
        cnt++;
    }
    *Rm1 = dd_sqrt(prev);
    *Rm = dd_sqrt(dd_add(prev, sq[row]));
}

/* ------------------------------------------------------------------ */
/* public: arrowhead eigen-decomposition                              */
/* ------------------------------------------------------------------ */
/*
 * n: matrix order (d, z have n-1 entries).  Outputs at final positions
 * ks[0..nk) (all n if ks == NULL):
 *   lam[i], lam_lo[i] : eigenvalue as double and its dd tail
 *   sigma[i], mu_hi[i], mu_lo[i] : shift representation lam = sigma + mu
 *   relerr[i], abserr[i] : the oracle's own error bounds for lam
 *   V (n x nk, column-major, may be NULL) : eigenvectors, rows in input order
 * Returns 0, or -1 on invalid input.
 */
int oracle_arrow_eig(int n, const double *d, const double *z, double alpha,
                     const int *ks, int nk, double *lam, double *lam_lo,
                     double *sigma_out, double *mu_hi, double *mu_lo,
                     double *relerr, double *abserr, double *V, int nthreads) {
    if (n < 1) return -1;
    for (int r = 0; r < n - 1; r++)
        if (!isfinite(d[r]) || !isfinite(z[r])) return -1;
    if (!isfinite(alpha)) return -1;
    int n1 = n - 1;
    arrow_sol A;
    arrow_solve(n, d, z, NULL, alpha, ks, nk, nthreads, &A);
    int all = (ks == NULL);
    if (all) nk = n;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int i = 0; i < nk; i++) {
        int pos = all ? i : ks[i];
        int row = -1;
        const zero_info *zi = arrow_scalars(&A, d, pos, i, lam, lam_lo, sigma_out, mu_hi,
                                            mu_lo, relerr, abserr, &row);
        double *col = V ? V + (size_t)i * n : NULL;
        if (!col) continue;
        if (zi) {
            /* x_r = z_r / ((d_r - sigma) - mu), x_last = -1 */
            dd *x = malloc(sizeof(dd) * n);
            dd ss = dd_from(1.0);
            for (int r = 0; r < n1; r++) {
                if (z[r] == 0.0) { x[r] = dd_from(0.0); continue; }
                x[r] = dd_div(dd_from(z[r]), vec_den(d, r, zi));
                ss = dd_add(ss, dd_mul(x[r], x[r]));
            }
            x[n1] = dd_from(-1.0);
            dd nrm = dd_sqrt(ss);
            for (int r = 0; r < n; r++) col[r] = dd_div(x[r], nrm).hi;
            free(x);
        } else if (A.R.kind[row] == 1) {
            for (int r = 0; r < n; r++) col[r] = 0.0;
            col[row] = 1.0;
        } else {
            run_vector(&A.R, z, row, n, col);
        }
    }
    arrow_sol_free(&A);
    return 0;
}

/*
 * Hermitian arrowhead C = [D z; z^* alpha] (Sec. 6.1): z complex, given as
 * (zre, zim), n-1 entries; the column above the corner holds zeta_r.  The
 * eigenvalues of C are the zeros of f(l) = alpha - l - sum |zeta_r|^2/(d_r - l),
 * with |zeta_r|^2 = zre^2 + zim^2 exactly in double-double, and the
 * eigenvectors u = x/||x||, x_r = zeta_r/(d_r - l), x_n = -1 (C u = l u row by
 * row).  Deflated rows: e_r for zeta_r = 0; a run of equal d gives the real
 * Helmert-type vector of the moduli, with each row r scaled by the phase
 * zeta_r/|zeta_r| (the unitary Phi of Sec. 6.1).  U is column-major n x nk,
 * real and imaginary parts in Ure, Uim (either pair may be NULL).
 */
int oracle_herm_eig(int n, const double *d, const double *zre, const double *zim,
                    double alpha, const int *ks, int nk, double *lam, double *lam_lo,
                    double *sigma_out, double *mu_hi, double *mu_lo, double *relerr,
                    double *abserr, double *Ure, double *Uim, int nthreads) {
    if (n < 1) return -1;
    int n1 = n - 1;
    for (int r = 0; r < n1; r++)
        if (!isfinite(d[r]) || !isfinite(zre[r]) || !isfinite(zim[r])) return -1;
    if (!isfinite(alpha)) return -1;
    double *za = malloc(sizeof(double) * (n1 > 0 ? n1 : 1));
    dd *z2 = malloc(sizeof(dd) * (n1 > 0 ? n1 : 1));
    for (int r = 0; r < n1; r++) {
        z2[r] = dd_add(two_prod(zre[r], zre[r]), two_prod(zim[r], zim[r]));
        za[r] = dd_sqrt(z2[r]).hi;
    }
    arrow_sol A;
    arrow_solve(n, d, za, z2, alpha, ks, nk, nthreads, &A);
    int all = (ks == NULL);
    if (all) nk = n;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int i = 0; i < nk; i++) {
        int pos = all ? i : ks[i];
        int row = -1;
        const zero_info *zi = arrow_scalars(&A, d, pos, i, lam, lam_lo, sigma_out, mu_hi,
                                            mu_lo, relerr, abserr, &row);
        if (!Ure || !Uim) continue;
        double *cr = Ure + (size_t)i * n, *ci = Uim + (size_t)i * n;
        for (int r = 0; r < n; r++) { cr[r] = 0.0; ci[r] = 0.0; }
        if (zi) {
            dd *t = malloc(sizeof(dd) * n);     /* 1/((d_r - sigma) - mu) */
            dd ss = dd_from(1.0);
            for (int r = 0; r < n1; r++) {
                if (za[r] == 0.0) { t[r] = dd_from(0.0); continue; }
                t[r] = dd_div(dd_from(1.0), vec_den(d, r, zi));
                ss = dd_add(ss, dd_mul(z2[r], dd_mul(t[r], t[r])));
            }
            dd nrm = dd_sqrt(ss);
            for (int r = 0; r < n1; r++) {
                dd tr = dd_div(t[r], nrm);
                cr[r] = dd_mul_d(tr, zre[r]).hi;
                ci[r] = dd_mul_d(tr, zim[r]).hi;
            }
            cr[n1] = dd_div(dd_from(-1.0), nrm).hi;
            free(t);
        } else if (A.R.kind[row] == 1) {
            cr[row] = 1.0;
        } else {
            /* Phi times the real run vector of the moduli: rows l before `row`
               in its run get -|zeta_q| zeta_l / (R_{m-1} R_m), the row itself
               (zeta_q/|zeta_q|) R_{m-1}/R_m */
            dd Rm1, Rm;
            int s0;
            run_norms(&A.R, z2, row, &Rm1, &Rm, &s0);
            dd den = dd_mul(Rm1, Rm);
            dd zq = dd_sqrt(z2[row]);
            int cnt = 0, head = A.R.run_head[row], p = A.R.run_pos[row];
            for (int s = s0; s < n1 && cnt < p; s++) {
                int r = A.R.order[s];
                if (A.R.kind[r] == 1) continue;
                if (A.R.run_head[r] != head) break;
                dd f = dd_neg(dd_div(zq, den));
                cr[r] = dd_mul_d(f, zre[r]).hi;
                ci[r] = dd_mul_d(f, zim[r]).hi;
                cnt++;
            }
            dd g = dd_div(Rm1, dd_mul(Rm, zq));
            cr[row] = dd_mul_d(g, zre[row]).hi;
            ci[row] = dd_mul_d(g, zim[row]).hi;
        }
    }
    arrow_sol_free(&A);
    free(za); free(z2);
    return 0;
}

/*
 * Non-symmetric arrowhead G = [D zc; zr^T alpha] (Remark in Sec. 6.1) with
 * zc_r zr_r > 0, or zc_r = zr_r = 0.  Its eigenvalues are the zeros of
 * f(l) = alpha - l - sum zc_r zr_r/(d_r - l) (zc_r zr_r exactly in
 * double-double); right eigenvectors x_r = zc_r/(d_r - l), left
 * y_r = zr_r/(d_r - l), x_n = y_n = -1 (G x = l x and y^T G = l y^T row by
 * row), both divided by sqrt(1 + sum zc_r zr_r/(d_r - l)^2) so that
 * y^T x = 1.  Deflated rows: e_r for both; a run of equal d gives the Helmert-
 * type vector v of the symmetric arrowhead with zeta_r = sqrt(zc_r zr_r),
 * mapped by x_r = (zc_r/zeta_r) v_r and y_r = (zr_r/zeta_r) v_r.  X, Y:
 * column-major n x nk (either may be NULL).  Returns -1 when a pair has
 * opposite signs or only one zero.
 */
int oracle_nsym_eig(int n, const double *d, const double *zc, const double *zr, double alpha,
                    const int *ks, int nk, double *lam, double *lam_lo, double *sigma_out,
                    double *mu_hi, double *mu_lo, double *relerr, double *abserr, double *X,
                    double *Y, int nthreads) {
    if (n < 1) return -1;
    int n1 = n - 1;
    for (int r = 0; r < n1; r++) {
        if (!isfinite(d[r]) || !isfinite(zc[r]) || !isfinite(zr[r])) return -1;
        if ((zc[r] == 0.0) != (zr[r] == 0.0)) return -1;
        if (zc[r] != 0.0 && (zc[r] > 0.0) != (zr[r] > 0.0)) return -1;
    }
    if (!isfinite(alpha)) return -1;
    double *za = malloc(sizeof(double) * (n1 > 0 ? n1 : 1));
    dd *z2 = malloc(sizeof(dd) * (n1 > 0 ? n1 : 1));
    for (int r = 0; r < n1; r++) {
        z2[r] = two_prod(zc[r], zr[r]);
        za[r] = dd_sqrt(z2[r]).hi;
    }
    arrow_sol A;
    arrow_solve(n, d, za, z2, alpha, ks, nk, nthreads, &A);
    int all = (ks == NULL);
    if (all) nk = n;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int i = 0; i < nk; i++) {
        int pos = all ? i : ks[i];
        int row = -1;
        const zero_info *zi = arrow_scalars(&A, d, pos, i, lam, lam_lo, sigma_out, mu_hi,
                                            mu_lo, relerr, abserr, &row);
        double *cx = X ? X + (size_t)i * n : NULL, *cy = Y ? Y + (size_t)i * n : NULL;
        if (!cx && !cy) continue;
        for (int r = 0; r < n; r++) {
            if (cx) cx[r] = 0.0;
            if (cy) cy[r] = 0.0;
        }
        if (zi) {
            dd *t = malloc(sizeof(dd) * n);
            dd ss = dd_from(1.0);
            for (int r = 0; r < n1; r++) {
                if (za[r] == 0.0) { t[r] = dd_from(0.0); continue; }
                t[r] = dd_div(dd_from(1.0), vec_den(d, r, zi));
                ss = dd_add(ss, dd_mul(z2[r], dd_mul(t[r], t[r])));
            }
            dd nrm = dd_sqrt(ss);
            for (int r = 0; r < n1; r++) {
                dd tr = dd_div(t[r], nrm);
                if (cx) cx[r] = dd_mul_d(tr, zc[r]).hi;
                if (cy) cy[r] = dd_mul_d(tr, zr[r]).hi;
            }
            double last = dd_div(dd_from(-1.0), nrm).hi;
            if (cx) cx[n1] = last;
            if (cy) cy[n1] = last;
            free(t);
        } else if (A.R.kind[row] == 1) {
            if (cx) cx[row] = 1.0;
            if (cy) cy[row] = 1.0;
        } else {
            dd Rm1, Rm;
            int s0;
            run_norms(&A.R, z2, row, &Rm1, &Rm, &s0);
            dd den = dd_mul(Rm1, Rm);
            dd zq = dd_sqrt(z2[row]);
            int cnt = 0, head = A.R.run_head[row], p = A.R.run_pos[row];
            for (int s = s0; s < n1 && cnt < p; s++) {
                int r = A.R.order[s];
                if (A.R.kind[r] == 1) continue;
                if (A.R.run_head[r] != head) break;
                dd f = dd_neg(dd_div(zq, den));
                if (cx) cx[r] = dd_mul_d(f, zc[r]).hi;
                if (cy) cy[r] = dd_mul_d(f, zr[r]).hi;
                cnt++;
            }
            dd g = dd_div(Rm1, dd_mul(Rm, zq));
            if (cx) cx[row] = dd_mul_d(g, zc[row]).hi;
            if (cy) cy[row] = dd_mul_d(g, zr[row]).hi;
        }
    }
    arrow_sol_free(&A);
    free(za); free(z2);
    return 0;
}

/*
 * The reduction decisions alone (bit-exact contract): order[s] = original
 * row at sorted position s; kind[r] in {0 pole, 1 zero-deflated,
 * 2 run-deflated}; head[r] = original row of r's run head (-1 if kind 1).
 * Returns the number of reduced poles.
 */
int oracle_reduce(int n1, const double *d, const double *z, int *order, int *kind,
                  int *head) {
    reduction R;
    reduce(n1, d, z, &R);
    for (int s = 0; s < n1; s++) order[s] = R.order[s];
    for (int r = 0; r < n1; r++) { kind[r] = R.kind[r]; head[r] = R.run_head[r]; }
    int m = R.m;
    free_reduction(&R);
    return m;
}

/*
 * The element b = [(A - d_i I)^{-1}]_{ii} of Eq. (invAi)/(b_ob), by its
 * definition f_bar(d_i)/zeta_i^2 (the Pick function of A without row i,
 * evaluated at d_i), in dd.  i is a row of the (already reduced) input.
 * Also returns K_b of Eq. (K2).
 */
int oracle_inverse_element(int n, const double *d, const double *z, double alpha,
                           int i, double *b_hi, double *b_lo, double *Kb) {
    int n1 = n - 1;
    if (i < 0 || i >= n1) return -1;
    dd a = dd_sub(dd_from(alpha), dd_from(d[i]));
    dd s1 = dd_from(0.0), s2 = dd_from(0.0);
    for (int j = 0; j < n1; j++) {
        if (j == i) continue;
        dd del = two_sum(d[j], -d[i]);
        dd t = dd_div(two_prod(z[j], z[j]), del);
        if (del.hi > 0) s1 = dd_add(s1, t); else s2 = dd_add(s2, t);
    }
    dd num = dd_add(dd_neg(a), dd_add(s1, s2));
    dd bb = dd_div(num, two_prod(z[i], z[i]));
    *b_hi = bb.hi;
    if (b_lo) *b_lo = bb.lo;
    if (Kb) *Kb = (fabs(a.hi) + fabs(s1.hi) + fabs(s2.hi)) / fabs(num.hi);
    return 0;
}

/* ------------------------------------------------------------------ */
/* public: DPR1  M = D + rho u u^T                                    */
/* ------------------------------------------------------------------ */
int oracle_dpr1_eig(int n, const double *d, const double *u, double rho,
                    const int *ks, int nk, double *lam, double *relerr,
                    double *Q, int nthreads) {
    if (n < 1 || !isfinite(rho)) return -1;
    for (int r = 0; r < n; r++)
        if (!isfinite(d[r]) || !isfinite(u[r])) return -1;
    reduction R;
    reduce(n, d, u, &R);
    int m = R.m;
    dd *c = malloc(sizeof(dd) * (m > 0 ? m : 1));
    for (int j = 0; j < m; j++) c[j] = R.pole_c[j];
    int ncomp = (rho == 0.0) ? 0 : m;
    int ndefl = R.ndefl;
    /* with rho == 0 every pole is an eigenvalue with a unit vector */
    int all = (ks == NULL);
    if (all) nk = n;
    zero_info *Z = calloc(ncomp > 0 ? ncomp : 1, sizeof(zero_info));
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        dd *buf = malloc(sizeof(dd) * (m > 0 ? m : 1));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int k = 0; k < ncomp; k++)
            Z[k] = solve_zero(KIND_DPR1, m, R.pole_d, c, dd_from(0.0), rho, k, buf);
        free(buf);
    }
    double *lam_comp = malloc(sizeof(double) * (ncomp > 0 ? ncomp : 1));
    for (int k = 0; k < ncomp; k++) lam_comp[k] = dd_add(dd_from(Z[k].sigma), Z[k].mu).hi;
    /* rho == 0: all rows behave as deflated with their unit vectors */
    int nd2 = (rho == 0.0) ? n : ndefl;
    int *drows = malloc(sizeof(int) * (nd2 > 0 ? nd2 : 1));
    if (rho == 0.0) { for (int s = 0; s < n; s++) drows[s] = R.order[s]; }
    else { for (int t = 0; t < ndefl; t++) drows[t] = R.defl_row[t]; }
    double *lam_defl = malloc(sizeof(double) * (nd2 > 0 ? nd2 : 1));
    for (int t = 0; t < nd2; t++) lam_defl[t] = d[drows[t]];
    int *slot = malloc(sizeof(int) * n);
    merge_order(ncomp, lam_comp, nd2, lam_defl, slot);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int i = 0; i < nk; i++) {
        int pos = all ? i : ks[i];
        int s = slot[pos];
        double *col = Q ? Q + (size_t)i * n : NULL;
        if (s >= 0) {
            zero_info *zi = &Z[s];
            dd l = dd_add(dd_from(zi->sigma), zi->mu);
            lam[i] = l.hi;
            if (relerr) relerr[i] = zi->relerr;
            if (col) {
                dd *x = malloc(sizeof(dd) * n);
                dd ss = dd_from(0.0);
                for (int r = 0; r < n; r++) {
                    if (u[r] == 0.0) { x[r] = dd_from(0.0); continue; }
                    dd den = dd_sub(two_sum(d[r], -zi->sigma), zi->mu);
                    x[r] = dd_div(dd_from(u[r]), den);
                    ss = dd_add(ss, dd_mul(x[r], x[r]));
                }
                dd nrm = dd_sqrt(ss);
                for (int r = 0; r < n; r++) col[r] = dd_div(x[r], nrm).hi;
                free(x);
            }
        } else {
            int row = drows[-1 - s];
            lam[i] = d[row];
            if (relerr) relerr[i] = 0.0;
            if (col) {
                if (rho == 0.0 || R.kind[row] == 1) {
                    for (int r = 0; r < n; r++) col[r] = 0.0;
                    col[row] = 1.0;
                } else {
                    run_vector(&R, u, row, n, col);
                }
            }
        }
    }
    free(slot); free(lam_defl); free(drows); free(lam_comp); free(Z); free(c);
    free_reduction(&R);
    return 0;
}

/* ------------------------------------------------------------------ */
/* public: SVD of the upper triangular arrowhead B = [D z; 0 alpha]   */
/* ------------------------------------------------------------------ */
/*
 * Requires d_j > 0 and distinct, z_j != 0 (an irreducible B with positive
 * diagonal, as Sec. 6.2 assumes), alpha != 0.  The arrowhead B^T B has poles
 * d_j^2, spikes d_j z_j and corner alpha^2 + z^T z; its shifted differences
 * (d_j - d_i)(d_j + d_i) are formed from exact dd sums.
 */
int oracle_tsvd(int n, const double *d, const double *z, double alpha,
                const int *ks, int nk, double *sv, double *relerr, double *U,
                double *V, int nthreads) {
    int n1 = n - 1;
    if (n < 2 || !isfinite(alpha) || alpha == 0.0) return -1;
    for (int r = 0; r < n1; r++) {
        if (!isfinite(d[r]) || !isfinite(z[r]) || !(d[r] > 0.0) || z[r] == 0.0) return -1;
        if (r > 0 && !(d[r] < d[r - 1])) return -1;
    }
    /* corner alpha^2 + z^T z in dd */
    dd corner = two_prod(alpha, alpha);
    for (int j = 0; j < n1; j++) corner = dd_add(corner, two_prod(z[j], z[j]));
    /* weights (d_j z_j)^2 in dd */
    dd *c = malloc(sizeof(dd) * n1);
    for (int j = 0; j < n1; j++) {
        dd dz = two_prod(d[j], z[j]);
        c[j] = dd_mul(dz, dz);
    }
    int all = (ks == NULL);
    if (all) nk = n;
    int ncomp = n;
    zero_info *Z = calloc(ncomp, sizeof(zero_info));
    char *want = calloc(ncomp, 1);
    if (all) memset(want, 1, ncomp); else for (int i = 0; i < nk; i++) want[ks[i]] = 1;
    /* Poles p_j = d_j^2 are not exact in double; the zero search below uses
       exact dd shifted differences (d_j - d_i)(d_j + d_i) directly. */
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        dd *delta = malloc(sizeof(dd) * n1);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int k = 0; k < ncomp; k++) {
            if (!want[k]) continue;
            int upper = k - 1, lower = k < n1 ? k : -1;
            secular S;
            S.kind = KIND_ARROW; S.m = n1; S.c = c; S.rho = 0.0; S.delta = delta;
            int pole, sgn;
            dd T;
            if (upper >= 0 && lower >= 0) {
                int i = lower;
                for (int j = 0; j < n1; j++)
                    delta[j] = dd_mul(two_sum(d[j], -d[i]), two_sum(d[j], d[i]));
                S.a = dd_sub(corner, two_prod(d[i], d[i]));
                dd gap = dd_mul(two_sum(d[upper], -d[i]), two_sum(d[upper], d[i]));
                dd h = dd_half(gap);
                double bound;
                dd f = secular_eval(&S, h, &bound);
                if (fabs(f.hi) > bound && f.hi < 0.0) { pole = lower; sgn = 1; T = h; }
                else if (fabs(f.hi) > bound) { pole = upper; sgn = -1; T = h; }
                else { pole = upper; sgn = -1; T = dd_add(h, dd_half(h)); }
            } else if (lower >= 0) {
                pole = lower; sgn = 1;
                /* Gershgorin on B^T B relative to d_0^2 */
                double t = corner.hi + 2.0 * fabs(d[0] * z[0]) * n1;
                for (int j = 0; j < n1; j++) t += fabs(d[j] * z[j]);
                T = dd_from(t * (1 + 1e-9));
            } else {
                pole = upper; sgn = -1;
                dd d2 = two_prod(d[upper], d[upper]);
                T = dd_mul_d(d2, 1.0);   /* singular values are >= 0 */
            }
            int i = pole;
            for (int j = 0; j < n1; j++)
                delta[j] = dd_mul(two_sum(d[j], -d[i]), two_sum(d[j], d[i]));
            S.a = dd_sub(corner, two_prod(d[i], d[i]));
            Z[k].pole = i;
            Z[k].sigma = d[i];  /* the shift in B^T B is d_i^2 */
            Z[k].mu = bisect_zero(&S, sgn, T, &Z[k].relerr, &Z[k].iters);
            /* eigenvalue of B^T B: d_i^2 + mu; refine unshifted if it cancels */
            dd d2 = two_prod(d[i], d[i]);
            dd lam = dd_add(d2, Z[k].mu);
            double q = (d2.hi + fabs(Z[k].mu.hi)) / fabs(lam.hi);
            double abserr = (d2.hi + fabs(Z[k].mu.hi)) * Z[k].relerr + 4 * U2 * fabs(lam.hi);
            Z[k].abserr = abserr;
            Z[k].relerr = abserr / fabs(lam.hi);
            if (q > 3.0 && isfinite(abserr)) {
                for (int j = 0; j < n1; j++) delta[j] = two_prod(d[j], d[j]);
                secular U0 = S;
                U0.a = corner;
                dd lim_lo = lower >= 0 ? two_prod(d[lower], d[lower]) : dd_from(0.0);
                dd lim_hi = upper >= 0 ? two_prod(d[upper], d[upper]) : dd_from(1e300);
                double w = 4.0 * abserr + 1e-300;
                dd lo = lim_lo, hi = lim_hi;
                for (int tries = 0; tries < 200; tries++, w *= 4.0) {
                    lo = dd_sub(lam, dd_from(w));
                    hi = dd_add(lam, dd_from(w));
                    if (dd_lt(lo, lim_lo)) lo = lim_lo;
                    if (dd_lt(lim_hi, hi)) hi = lim_hi;
                    if (secular_side(&U0, lo) > 0 && secular_side(&U0, hi) < 0) break;
                }
                double width;
                dd l2 = bisect_interval(&U0, lo, hi, &width);
                Z[k].pole = -1;
                Z[k].mu = l2;
                Z[k].abserr = width + 4 * U2 * fabs(l2.hi);
                Z[k].relerr = Z[k].abserr / fabs(l2.hi);
            }
        }
        free(delta);
    }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int q = 0; q < nk; q++) {
        int k = all ? q : ks[q];
        zero_info *zi = &Z[k];
        int i = zi->pole;
        dd lam = i >= 0 ? dd_add(two_prod(d[i], d[i]), zi->mu) : zi->mu;
        dd s = dd_sqrt(lam);
        sv[q] = s.hi;
        if (relerr) relerr[q] = 0.5 * zi->relerr + 4 * U2;
        if (U || V) {
            dd *x = malloc(sizeof(dd) * n);
            dd ss = dd_from(1.0);
            for (int r = 0; r < n1; r++) {
                dd del = i >= 0 ? dd_mul(two_sum(d[r], -d[i]), two_sum(d[r], d[i]))
                                : two_prod(d[r], d[r]);
                dd den = dd_sub(del, zi->mu);
                x[r] = dd_div(two_prod(d[r], z[r]), den);
                ss = dd_add(ss, dd_mul(x[r], x[r]));
            }
            x[n1] = dd_from(-1.0);
            dd nrm = dd_sqrt(ss);
            for (int r = 0; r < n; r++) x[r] = dd_div(x[r], nrm);
            if (V) for (int r = 0; r < n; r++) V[(size_t)q * n + r] = x[r].hi;
            if (U) {
                for (int r = 0; r < n1; r++)
                    U[(size_t)q * n + r] = dd_div(dd_mul(s, x[r]), dd_from(d[r])).hi;
                U[(size_t)q * n + n1] = dd_div(dd_mul_d(x[n1], alpha), s).hi;
            }
            free(x);
        }
    }
    free(want); free(Z); free(c);
    return 0;
}

/* ------------------------------------------------------------------ */
/* brute force: Jacobi in IEEE binary128                              */
/* ------------------------------------------------------------------ */
#if defined(__aarch64__)
typedef long double qd_t;          /* binary128 on AArch64 Linux */
#define QSQRT sqrtl
#define QFABS fabsl
#else
#include <quadmath.h>
typedef __float128 qd_t;
#define QSQRT sqrtq
#define QFABS fabsq
#endif

static void q_to_dd(qd_t q, double *hi, double *lo) {
    double h = (double)q;
    *hi = h;
    if (lo) *lo = (double)(q - (qd_t)h);
}

/*
 * Cyclic Jacobi for a symmetric n x n matrix A (column-major doubles).
 * Returns eigenvalues (hi, lo parts, unsorted order of the diagonal) and
 * eigenvectors (columns).  Rotations as in Golub & Van Loan, Alg. 8.5.2.
 */
int oracle_jacobi_sym(int n, const double *A, double *lam_hi, double *lam_lo,
                      double *Vout, int max_sweeps) {
    qd_t *a = malloc(sizeof(qd_t) * n * n);
    qd_t *v = malloc(sizeof(qd_t) * n * n);
    for (int i = 0; i < n * n; i++) a[i] = A[i];
    for (int i = 0; i < n * n; i++) v[i] = 0;
    for (int i = 0; i < n; i++) v[i * n + i] = 1;
#define AQ(i, j) a[(size_t)(j) * n + (i)]
#define VQ(i, j) v[(size_t)(j) * n + (i)]
    int sweeps = 0;
    for (; sweeps < max_sweeps; sweeps++) {
        qd_t off = 0, tot = 0;
        for (int j = 0; j < n; j++)
            for (int i = 0; i < n; i++) {
                qd_t x = AQ(i, j) * AQ(i, j);
                tot += x;
                if (i != j) off += x;
            }
        if (off == 0 || off <= tot * (qd_t)1e-66) break;
        for (int p = 0; p < n - 1; p++)
            for (int q = p + 1; q < n; q++) {
                qd_t apq = AQ(p, q);
                if (apq == 0) continue;
                qd_t app = AQ(p, p), aqq = AQ(q, q);
                qd_t tau = (aqq - app) / (2 * apq);
                qd_t t = (tau >= 0 ? 1 : -1) / (QFABS(tau) + QSQRT(1 + tau * tau));
                qd_t cs = 1 / QSQRT(1 + t * t), sn = t * cs;
                for (int k = 0; k < n; k++) {      /* A <- A J */
                    qd_t akp = AQ(k, p), akq = AQ(k, q);
                    AQ(k, p) = cs * akp - sn * akq;
                    AQ(k, q) = sn * akp + cs * akq;
                }
                for (int k = 0; k < n; k++) {      /* A <- J^T A */
                    qd_t apk = AQ(p, k), aqk = AQ(q, k);
                    AQ(p, k) = cs * apk - sn * aqk;
                    AQ(q, k) = sn * apk + cs * aqk;
                }
                for (int k = 0; k < n; k++) {      /* V <- V J */
                    qd_t vkp = VQ(k, p), vkq = VQ(k, q);
                    VQ(k, p) = cs * vkp - sn * vkq;
                    VQ(k, q) = sn * vkp + cs * vkq;
                }
            }
    }
    for (int i = 0; i < n; i++) q_to_dd(AQ(i, i), &lam_hi[i], lam_lo ? &lam_lo[i] : NULL);
    if (Vout) for (int i = 0; i < n * n; i++) Vout[i] = (double)v[i];
#undef AQ
#undef VQ
    free(a); free(v);
    return sweeps;
}

/*
 * One-sided (Hestenes) Jacobi SVD of a square n x n matrix B (column-major):
 * B J_1 J_2 ... = W with orthogonal columns; singular values are the column
 * norms, V = J_1 J_2 ..., U = W diag(1/s).  Output unsorted.
 */
int oracle_jacobi_svd(int n, const double *B, double *s_hi, double *Uout,
                      double *Vout, int max_sweeps) {
    qd_t *w = malloc(sizeof(qd_t) * n * n);
    qd_t *v = malloc(sizeof(qd_t) * n * n);
    for (int i = 0; i < n * n; i++) w[i] = B[i];
    for (int i = 0; i < n * n; i++) v[i] = 0;
    for (int i = 0; i < n; i++) v[i * n + i] = 1;
#define WQ(i, j) w[(size_t)(j) * n + (i)]
#define VQ(i, j) v[(size_t)(j) * n + (i)]
    int sweeps = 0;
    for (; sweeps < max_sweeps; sweeps++) {
        int rotated = 0;
        for (int p = 0; p < n - 1; p++)
            for (int q = p + 1; q < n; q++) {
                qd_t alpha = 0, beta = 0, gamma = 0;
                for (int k = 0; k < n; k++) {
                    alpha += WQ(k, p) * WQ(k, p);
                    beta += WQ(k, q) * WQ(k, q);
                    gamma += WQ(k, p) * WQ(k, q);
                }
                if (gamma == 0 || QFABS(gamma) <= (qd_t)1e-33 * QSQRT(alpha * beta)) continue;
                rotated = 1;
                qd_t zeta = (beta - alpha) / (2 * gamma);
                qd_t t = (zeta >= 0 ? 1 : -1) / (QFABS(zeta) + QSQRT(1 + zeta * zeta));
                qd_t cs = 1 / QSQRT(1 + t * t), sn = cs * t;
                for (int k = 0; k < n; k++) {
                    qd_t a1 = WQ(k, p), a2 = WQ(k, q);
                    WQ(k, p) = cs * a1 - sn * a2;
                    WQ(k, q) = sn * a1 + cs * a2;
                    qd_t v1 = VQ(k, p), v2 = VQ(k, q);
                    VQ(k, p) = cs * v1 - sn * v2;
                    VQ(k, q) = sn * v1 + cs * v2;
                }
            }
        if (!rotated) break;
    }
    for (int j = 0; j < n; j++) {
        qd_t nr = 0;
        for (int k = 0; k < n; k++) nr += WQ(k, j) * WQ(k, j);
        nr = QSQRT(nr);
        s_hi[j] = (double)nr;
        if (Uout) for (int k = 0; k < n; k++) Uout[(size_t)j * n + k] = nr > 0 ? (double)(WQ(k, j) / nr) : 0.0;
    }
    if (Vout) for (int i = 0; i < n * n; i++) Vout[i] = (double)v[i];
#undef WQ
#undef VQ
    free(w); free(v);
    return sweeps;
}

/* the dd primitives, exposed so that tests can pin them against binary128 */
void oracle_dd_ops(double ah, double al, double bh, double bl, double *out) {
    dd a = {ah, al}, b = {bh, bl};
    dd r;
    r = dd_add(a, b); out[0] = r.hi; out[1] = r.lo;
    r = dd_mul(a, b); out[2] = r.hi; out[3] = r.lo;
    r = dd_div(a, b); out[4] = r.hi; out[5] = r.lo;
    r = dd_sqrt(dd_abs(a)); out[6] = r.hi; out[7] = r.lo;
}

int oracle_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
