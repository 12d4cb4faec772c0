/*
 * arrowhead.h -- C ABI of the GB300 arrowhead eigen-solver library
 * (libarrowhead.so, built for sm_103a).
 *
 * Method: Jakovcevic Stor, Slapnicar & Barlow, "Accurate eigenvalue
 * decomposition of arrowhead matrices and applications".  For each eigenvalue
 * the solver shifts to the nearest pole d_i (Algorithm 1), forms the inverse of
 * the shifted arrowhead (Eq. invAi) with its one cancellation-prone element b
 * (Eq. b_ob) in double-double arithmetic (Theorem 6), finds that inverse's
 * extreme eigenvalue nu by bisection (Algorithm 3, or a bracketed Newton
 * finish on the same function; ae_opts.finish), and returns
 * lambda = d_i + 1/nu with the eigenvector of Eq. (eigenvecAi) / Algorithm 4.
 * Eigenvalues whose shifted value cancels (the special cases after Theorem C1)
 * are recomputed from the inverse of A (Remark 1); eigenvalues with a large
 * K_nu (Eq. K0) are recomputed from another pole or a DPR1 inverse (Remark 2).
 *
 * Conventions shared by every entry point:
 *  - All array arguments are DEVICE pointers (cudaMalloc'd, managed or
 *    device-accessible), owned by the caller, unless the name ends in _host.
 *  - All work is issued on `stream` (a cudaStream_t passed as void*; NULL is
 *    the legacy default stream) and is asynchronous: outputs are valid once
 *    the stream has completed.  Inputs must stay unchanged until then.
 *  - Matrices are column-major with a leading dimension; column k pairs with
 *    the k-th eigen/singular value.  Rows are in the caller's input order.
 *  - The library allocates its O(n) scratch with cudaMallocAsync on `stream`
 *    and frees it the same way; nothing is kept between calls.
 *  - Return value: AE_OK (0); -k when argument k (1-based) is invalid
 *    (LAPACK convention); AE_ERR_* (> 1000) for CUDA or device-side failures.
 *    When `info` is non-NULL the call waits for the stream and fills it, and
 *    device-side conditions (non-finite input, iteration cap reached) are
 *    reported in the return value as well; with info == NULL the call does
 *    not synchronise and such conditions show up only as NaN outputs.
 *  - No C++ exception crosses this interface.
 *  - Range: the solve squares spikes and shifted differences in double
 *    precision, so entries must lie between about 2^-500 and 2^500 in
 *    magnitude; scale A by a power of two first when they do not (exact).
 */
#ifndef ARROWHEAD_H
#define ARROWHEAD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AE_OK 0
#define AE_ERR_CUDA 1001      /* a CUDA runtime call failed (see ae_last_cuda_error) */
#define AE_ERR_INPUT 1002     /* device-side check: non-finite d, z or alpha */
#define AE_ERR_NOCONV 1003    /* some eigenpair reached opts->max_iter */
#define AE_ERR_TOO_LARGE 1004 /* arrow_eig_noalloc: n exceeds its static scratch;
                                 arrow_eig_part: the part's items exceed cap */

/* precision of the bisection (see ae_opts.precision) */
#define AE_FP64 0             /* all-FP64 bisection from the Gershgorin bracket */
#define AE_FP32_BRACKET 1     /* FP32 opening bracket, verified and finished in FP64 */

/* how the FP64 finish locates the zero (see ae_opts.finish) */
#define AE_FINISH_BISECT 0    /* bisection, Algorithm 3 (default) */
#define AE_FINISH_NEWTON 1    /* bracketed Newton on the same function, same stop test */

/* per-eigenpair flag bits reported through ae_diag.flags */
#define AE_FLAG_DEFLATED 1    /* deflated by the reduction (zero spike / equal pole) */
#define AE_FLAG_NEARZERO 2    /* recomputed from A^{-1} (Remark 1) */
#define AE_FLAG_OTHERPOLE 4   /* recomputed shifted to the other pole (Remark 2a) */
#define AE_FLAG_DPR1SHIFT 8   /* recomputed from (A - sigma I)^{-1} (Remark 2b) */
#define AE_FLAG_CAPPED 16     /* bisection stopped at max_iter */
#define AE_FLAG_SINGULAR 32   /* remedy found a zero denominator: lambda = sigma */
#define AE_FLAG_FP32_FALLBACK 64 /* FP32 bracket failed its FP64 check */
#define AE_FLAG_DDB 128       /* with opts->bgate: b recomputed in double-double */
#define AE_FLAG_MID64 256     /* with AE_FP32_BRACKET: Algorithm 1's midpoint test was
                                 not settled by its FP32 evaluation and ran in FP64 */

typedef struct ae_opts {
    int precision;     /* AE_FP64 (default): every step in FP64 (double-double
                          where the paper asks).  AE_FP32_BRACKET: FP32 where its
                          result is certified or only picks trial points --
                          Algorithm 1's midpoint test in FP32 with an error
                          bound (FP64 where the bound leaves the sign open, flag
                          AE_FLAG_MID64), bisection's opening bracket in FP32
                          with both ends checked in FP64, and the Newton
                          finish's first trial point from FP32 and double-float
                          model steps.  Bracket ends are always FP64 evaluations. */
    double knu_max;    /* K_nu above which Remark 2 is applied; default 10 */
    int max_iter;      /* bisection iteration cap per eigenpair; default 2200 */
    int fixup;         /* 1 (default): Remarks 1 and 2; 0: Algorithm 1 only */
    int profile;       /* 1: time the phases with CUDA events recorded on the
                          call's stream; the times land in ae_info (default 0) */
    int finish;        /* AE_FINISH_BISECT (default) or AE_FINISH_NEWTON.  Newton
                          keeps a sign-change bracket of the same Pick function,
                          every trial point inside it, and Algorithm 3's stop test
                          (right - left <= 2 eps |mid|, nu = right); trial points
                          come from a one-pole model of the function, and points
                          within a certified radius of an FP64 evaluation are
                          evaluated from its local expansion F(x) + h F'(x) at
                          the same error bound.  Not in the paper: a faster finish
                          to the same tolerance, for the remedies too. */
    int bgate;         /* 0 (default): the element b of Eq. (b_ob) always in
                          double-double.  1: Algorithm 5's gates -- b in
                          standard precision unless the spike ratio
                          sum_{j != i} |zeta_j| / |zeta_i| exceeds n (C2 (ii)
                          fails) and K_b of Eq. (K2) exceeds kb_max (C2 (i)
                          fails); then in double-double (flag AE_FLAG_DDB) */
    double kb_max;     /* K_b above which the gate asks for double-double;
                          default 10 */
} ae_opts;

/* Summary counters, filled on the host when passed (forces a stream sync). */
typedef struct ae_info {
    int n_reduced;        /* eigenpairs solved by bisection (m + 1 for arrow_eig) */
    int n_deflated;       /* eigenpairs returned by the reduction */
    int n_nearzero;       /* Remark 1 recomputations */
    int n_otherpole;      /* Remark 2(a) recomputations */
    int n_dpr1shift;      /* Remark 2(b) recomputations */
    int n_capped;         /* eigenpairs that hit max_iter */
    int n_fp32_fallback;  /* FP32 brackets rejected by the FP64 check */
    int max_iter_used;    /* largest FP64 step count (bisection or Newton) of any eigenpair */
    long long total_iter; /* sum of FP64 step counts (FP64 evaluations of the zero finder) */
    long long fix_iter;   /* the part of total_iter spent in remedies */
    double max_Kb;        /* largest K_b of Eq. (K2) met */
    double max_Knu;       /* largest K_nu of Eq. (K0) met (before remedies) */
    float ms_reduce;      /* with opts->profile: checks, ordering, reduction */
    float ms_eig;         /* eigenvalue kernel (shift, b, bisection) */
    float ms_fix;         /* remedy decisions and recomputations */
    float ms_vectors;     /* placement and eigenvector columns */
    int n_ddb;            /* with opts->bgate: eigenpairs whose b was recomputed in
                             double-double */
    long long total_deriv; /* Newton finish: the evaluations of total_iter - fix_iter
                              (the solves of Algorithm 1's shift) that also formed
                              the derivative */
    int n_mid64;          /* with AE_FP32_BRACKET: midpoint tests (Algorithm 1) that
                             needed their FP64 pass (flag AE_FLAG_MID64) */
    long long n_f32_passes; /* with AE_FP32_BRACKET: O(n) passes evaluated in FP32
                             (midpoint tests, model steps, bracket bisection) */
    long long n_df_passes;  /* with AE_FP32_BRACKET: O(n) passes in double-float
                             (the Newton finish's opening model steps) */
} ae_info;

/* Optional per-eigenpair diagnostics (device arrays of length n, any may be
   NULL), indexed like the returned eigenvalues. */
typedef struct ae_diag {
    double *b;       /* element b of Eq. (b_ob) for Algorithm 1's shift pole (NaN if none),
                        also when a remedy recomputed the eigenvalue */
    double *Kb;      /* K_b of Eq. (K2) for that shift pole */
    double *Knu;     /* K_nu of Eq. (K0) estimated from the neighbouring eigenvalues */
    int *iters;      /* FP64 bisection steps of the final solve */
    int *flags;      /* AE_FLAG_* bits */
} ae_diag;

/* Fill *opts with the defaults above. */
void ae_default_opts(ae_opts *opts);

/* Human-readable text for a return code. */
const char *ae_status_string(int status);

/* Text of the last CUDA error seen by the library in this thread. */
const char *ae_last_cuda_error(void);

/*
 * arrow_eig -- all eigenpairs of the real symmetric arrowhead matrix
 *     A = [diag(d) z; z^T alpha]                         (Sec. 1, Eq. A)
 * of order n (d and z have n - 1 entries).
 *
 *  n       matrix order, n >= 1                                        (arg 1)
 *  d, z    device, n-1 doubles each: poles and spikes in ANY order and sign;
 *          zero spikes (+0 or -0) and exactly equal poles are deflated
 *          (Sec. 1): stable descending sort (ties by lower input index),
 *          zero-spike rows return (d_r, e_r), equal-pole rows are folded
 *          into the first of their run by rotations              (args 2, 3)
 *  alpha   the corner element                                          (arg 4)
 *  lambda  device, n doubles out: eigenvalues in descending order; ties
 *          between a deflated and a computed value put the deflated first (5)
 *  V       device, ldv*n doubles out or NULL: column k is the unit
 *          eigenvector of lambda[k].  A computed eigenpair has
 *          v = x/||x||, x = [(D - lambda I)^{-1} z ; -1] (Eq. Aeigenvec), so its
 *          last component is negative.  A zero-spike row r gives e_r; the
 *          m-th later member q_m of a run of equal poles (nonzero spikes
 *          z_{q_0..q_t} in input order) gives
 *          (-z_{q_m} sum_{l<m} z_{q_l} e_{q_l} + R_{m-1}^2 e_{q_m}) / (R_{m-1} R_m),
 *          R_m^2 = sum_{l<=m} z_{q_l}^2                                (arg 6)
 *  ldv     leading dimension of V, >= n                                (arg 7)
 *  shift, mu  device, n doubles out or NULL: lambda[k] = shift[k] + mu[k]
 *          with shift[k] the pole used (Remark 1a), or the non-pole shift of
 *          Remarks 1/2(b); deflated values have mu = 0           (args 8, 9)
 *  opts    NULL for defaults                                          (arg 10)
 *  info    host, NULL or filled (synchronises)                        (arg 11)
 *  diag    host struct of optional device arrays, or NULL              (arg 12)
 *  stream  cudaStream_t                                               (arg 13)
 */
int arrow_eig(int n, const double *d, const double *z, double alpha,
              double *lambda, double *V, int ldv, double *shift, double *mu,
              const ae_opts *opts, ae_info *info, const ae_diag *diag, void *stream);

/*
 * arrow_eig_part -- one part of arrow_eig split across devices or calls.
 * Eigenpairs are independent once the reduction is done (Sec. 1: each comes
 * from the shifted inverse of its own nearest pole, O(n) work apiece), so one
 * instance splits by eigenpair ranges with nothing exchanged: every part
 * repeats the O(n log n) reduction of the whole input (Sec. 1: order, zero
 * spikes, equal poles) and then solves
 *   - the computed eigenpairs k in [k0, k1) of the reduced arrowhead with
 *     m + 1 computed eigenvalues, k0 = part (m + 1) / nparts and
 *     k1 = (part + 1) (m + 1) / nparts (integer division), and
 *   - the deflated rows whose values lie in [p_{k1-1}, p_{k0-1}) (reduced
 *     poles p; p_{-1} = +inf, p_m = -inf),
 * which hold the contiguous output positions [*pos0, *pos0 + *count) of the
 * whole decomposition, in the same descending order.  The remedy decision of
 * Eq. (K0) for an eigenpair needs the eigenvalues on both sides of it: each
 * part also solves the eigenpair just outside each end of its range (Algorithm
 * 1's solve only, which gives the bits the owning part computes), so the
 * parts' results put side by side equal arrow_eig's, except that a remedied
 * eigenpair (Remarks 1, 2) may be re-solved by a team of another width and so
 * agree within the tolerance rather than bit for bit.  The solver's counters
 * in info include the two edge solves.
 *
 *  n, d, z, alpha  the whole arrowhead, as arrow_eig                (args 1-4)
 *  part, nparts    this part, 0 <= part < nparts                     (args 5, 6)
 *  lambda  device, cap doubles out: the part's eigenvalues, descending    (7)
 *  V, ldv  device, ldv*cap doubles out or NULL: their eigenvectors (full
 *          length n, rows in the caller's input order), ldv >= n     (8, 9)
 *  cap     room of lambda and V in items; a part with more items returns
 *          AE_ERR_TOO_LARGE before it solves (arrow_eig_part_size gives the
 *          count)                                                       (10)
 *  pos0, count  host out: the part's first output position and item count
 *          (the call synchronises `stream` after the reduction)  (args 11, 12)
 *  opts, info, stream: as arrow_eig                           (args 13-15)
 */
int arrow_eig_part(int n, const double *d, const double *z, double alpha, int part, int nparts,
                   double *lambda, double *V, int ldv, int cap, int *pos0, int *count,
                   const ae_opts *opts, ae_info *info, void *stream);

/* The first output position and item count of part `part` of `nparts` of
   the arrowhead (d, z) (the reduction only; synchronises `stream`).
   Arguments as arrow_eig_part: n 1, d 2, z 3, part 4, nparts 5, pos0 6,
   count 7 (host), stream 8. */
int arrow_eig_part_size(int n, const double *d, const double *z, int part, int nparts,
                        int *pos0, int *count, void *stream);

/*
 * dpr1_eig -- all eigenpairs of the diagonal-plus-rank-one matrix
 *     M = diag(d) + rho u u^T                                  (Sec. 6.3)
 * of order n, through the paper's reduction to the arrowhead A = L^{-1} M L:
 * after ordering d_1 > ... > d_n (and folding as below), A has poles
 * d_1..d_{n-1}, spikes zeta_j = u_j sqrt(rho (d_j - d_n)) and corner
 * d_n + rho u^T u, the last two in double-double.  rho < 0 is solved as
 * -M = -diag(d) + |rho| u u^T.  The eigenvalue in (d_n, d_{n-1}) is re-solved
 * from (A - d_n I)^{-1} (Remark 2(b)'s DPR1 inverse) when it is nearer d_n,
 * so that lambda - d_n keeps its relative accuracy.
 *
 *  n       matrix order, n >= 1                                        (arg 1)
 *  d, u    device, n doubles each, any order and sign; u_r = +-0 deflates
 *          (d_r, e_r); exactly equal d fold like arrow_eig's equal poles (2, 3)
 *  rho     the rank-one weight; rho = 0 returns sorted d and unit vectors (4)
 *  lambda  device, n doubles out, descending                            (5)
 *  Q       device, ldq*n doubles out or NULL: column k is the unit eigenvector
 *          q ~ (diag(d) - lambda_k I)^{-1} u with a positive factor; deflated
 *          columns as in arrow_eig (unit vectors, rotation vectors of runs) (6)
 *  ldq     >= n                                                         (7)
 *  opts, info, diag, stream: as arrow_eig                      (args 8-11)
 */
int dpr1_eig(int n, const double *d, const double *u, double rho, double *lambda, double *Q,
             int ldq, const ae_opts *opts, ae_info *info, const ae_diag *diag, void *stream);

/*
 * tri_arrow_svd -- singular value decomposition B = U diag(sigma) V^T of the
 * upper triangular arrowhead
 *     B = [diag(d) z; 0 alpha]                                 (Sec. 6.2)
 * of order n (d, z have n-1 entries), through the arrowhead B^T B with poles
 * d_j^2, spikes d_j z_j and corner alpha^2 + z^T z (both in double-double);
 * shifted differences to a pole are (d_j - d_i)(d_j + d_i).  sigma = sqrt(lambda),
 * v the eigenvector of B^T B, u_j = sigma v_j / d_j, u_n = alpha v_n / sigma.
 *
 *  n       order, n >= 1                                               (arg 1)
 *  d       device, n-1 doubles, each > 0 (any order); a d_r <= 0 is reported as
 *          AE_ERR_INPUT (with info) -- flip row r of B to make it positive (2)
 *  z       device, n-1 doubles; z_r = 0 deflates (d_r, e_r, e_r)            (3)
 *  alpha   the corner, nonzero                                          (4)
 *  sigma   device, n doubles out, descending                            (5)
 *  U, ldu  device, ldu*n doubles out or NULL: left singular vectors (6, 7)
 *  V, ldv  device, ldv*n doubles out or NULL (required when U is given):
 *          right singular vectors, last component negative (x_n = -1 of
 *          Eq. Aeigenvec applied to B^T B)                            (8, 9)
 *  opts, info, diag, stream: as arrow_eig (diag refers to B^T B)  (args 10-13)
 */
int tri_arrow_svd(int n, const double *d, const double *z, double alpha, double *sigma,
                  double *U, int ldu, double *V, int ldv, const ae_opts *opts, ae_info *info,
                  const ae_diag *diag, void *stream);

/*
 * herm_arrow_eig -- all eigenpairs of the Hermitian arrowhead
 *     C = [diag(d) z; z^* alpha]                              (Sec. 6.1)
 * of order n, z complex: z_r = zeta_r is the column above the real corner.
 * The diagonal unitary similarity Phi = diag(zeta_r/|zeta_r|, 1) gives the
 * real arrowhead A = Phi^* C Phi = [diag(d) |z|; |z|^T alpha] (Eq. cc), solved
 * as arrow_eig solves it, with each |zeta_r|^2 = re^2 + im^2 in double-double
 * (the paper asks for the moduli in doubled precision when b is); then
 * U = Phi V, i.e. u_r = zeta_r / ((d_r - sigma) - mu) / ||x||, u_n = -1/||x||.
 *
 *  n       order, n >= 1                                               (arg 1)
 *  d       device, n-1 doubles, any order                               (2)
 *  z       device, n-1 complex numbers as 2(n-1) doubles (re, im interleaved,
 *          the layout of cuDoubleComplex / complex128); zeta_r = 0 deflates
 *          (d_r, e_r)                                                   (3)
 *  alpha   the real corner                                              (4)
 *  lambda  device, n doubles out, descending                            (5)
 *  U, ldu  device, column-major complex n x n (column k at U + 2*ldu*k
 *          doubles, row r at doubles 2r, 2r+1) out, or NULL; ldu >= n
 *          complex entries.  A run of equal d gives Phi times the real
 *          vector arrow_eig gives for the moduli                    (6, 7)
 *  shift, mu, opts, info, diag, stream: as arrow_eig (diag refers to A)
 *                                                               (args 8-13)
 * Returns as arrow_eig.
 */
int herm_arrow_eig(int n, const double *d, const double *z, double alpha, double *lambda,
                   double *U, int ldu, double *shift, double *mu, const ae_opts *opts,
                   ae_info *info, const ae_diag *diag, void *stream);

/*
 * nsym_arrow_eig -- all eigenpairs of the non-symmetric arrowhead
 *     G = [diag(d) zc; zr^T alpha]               (Remark of Sec. 6.1)
 * of order n with zc_r zr_r > 0 (each pair of one sign), or zc_r = zr_r = 0.
 * The diagonal similarity Psi = diag(sign(zr_r) sqrt(zc_r / zr_r), 1) gives
 * the symmetric arrowhead A = Psi^{-1} G Psi with zeta_r = sqrt(zc_r zr_r)
 * (zeta_r^2 = zc_r zr_r exactly in double-double); G has A's eigenvalues, right
 * eigenvectors X = Psi V and left eigenvectors Y = Psi^{-1} V, so that
 * x_r = zc_r t_r, y_r = zr_r t_r with t_r = 1/((d_r - sigma) - mu)/||x||,
 * x_n = y_n = -1/||x||, and Y^T X = I.  (The printed Psi has the ratio
 * inverted; this one makes Psi^{-1} G Psi symmetric.)
 *
 *  n       order, n >= 1                                               (arg 1)
 *  d       device, n-1 doubles, any order                               (2)
 *  zc, zr  device, n-1 doubles each: the column above the corner and the
 *          row left of it; a pair of opposite signs, or with exactly one
 *          zero, is reported as AE_ERR_INPUT (with info)            (3, 4)
 *  alpha   the corner                                                   (5)
 *  lambda  device, n doubles out, descending                            (6)
 *  X, ldx  device, ldx*n doubles out or NULL: right eigenvectors    (7, 8)
 *  Y, ldy  device, ldy*n doubles out or NULL (requires X): left
 *          eigenvectors                                            (9, 10)
 *  shift, mu, opts, info, diag, stream: as arrow_eig (diag refers to A)
 *                                                              (args 11-16)
 * Returns as arrow_eig.
 */
int nsym_arrow_eig(int n, const double *d, const double *zc, const double *zr, double alpha,
                   double *lambda, double *X, int ldx, double *Y, int ldy, double *shift,
                   double *mu, const ae_opts *opts, ae_info *info, const ae_diag *diag,
                   void *stream);

/*
 * Batched arrowheads: `count` independent instances of orders n_i >= 1, solved
 * together -- each stage of the arrow_eig pipeline is one persistent launch
 * over all instances (eigenpairs of every instance share one work queue and
 * are solved by teams of W = 8, 16 or 32 lanes, W chosen per order bucket by
 * ae_autotune and cached).  The method per instance is that of arrow_eig
 * (Algorithms 1-3, Theorem 6, Remarks 1-2); the batching is this library's.
 *
 * Layout (all device arrays except n_off / v_off, which are HOST arrays of
 * count + 1 int64 prefix sums):
 *   n_off[i]       sum of n_j for j < i (n_off[0] = 0, n_off[count] = total)
 *   d_all, z_all   instance i's n_i - 1 poles / spikes start at n_off[i] - i
 *   alpha_all[i]   corner of instance i
 *   lambda_all     instance i's eigenvalues (descending) start at n_off[i]
 *   V_all          NULL, or instance i's n_i x n_i column-major eigenvectors
 *                  (ld = n_i) start at v_off[i] (v_off NULL: packed, the prefix
 *                  sums of n_i^2)
 *   status_all     NULL, or per-instance AE_OK / AE_ERR_INPUT / AE_ERR_NOCONV
 * Conventions per instance are those of arrow_eig.  Returns -k for argument k.
 */
typedef struct ae_batch ae_batch;

/* One-shot batched solve on `stream` (synchronises before returning, since it
   frees its scratch).  info, if given, sums the per-instance counters. */
int arrow_eig_batched(int count, const long long *n_off, const long long *v_off,
                      const double *d_all, const double *z_all, const double *alpha_all,
                      double *lambda_all, double *V_all, int *status_all, const ae_opts *opts,
                      ae_info *info, void *stream);

/* A reusable plan for repeated solves of the same shapes and buffers: builds
   the descriptor table and all scratch (cudaMalloc), and captures the whole
   solve in a CUDA graph.  The plan keeps the buffer addresses: change their
   contents, not the buffers, between runs.  Arguments as arrow_eig_batched
   (plan is arg 1, count arg 2 ...). */
int ae_batch_create(ae_batch **plan, int count, const long long *n_off,
                    const long long *v_off, const double *d_all, const double *z_all,
                    const double *alpha_all, double *lambda_all, double *V_all,
                    int *status_all, const ae_opts *opts, void *stream);
/* Replay the captured solve on `stream` (asynchronous). */
int ae_batch_run(ae_batch *plan, void *stream);
/* Counters of the last run, summed over instances (synchronises `stream`). */
int ae_batch_info(ae_batch *plan, ae_info *info, void *stream);
/* Free the plan (waits for the device). */
void ae_batch_destroy(ae_batch *plan);

/* Time team widths 8, 16, 32 on synthetic instances for order buckets
   32..256 (larger buckets use 32) and store the fastest per bucket in the JSON
   cache $AE_TUNE_CACHE (default ~/.cache/arrowhead_tune.json), keyed by the
   device name and the library build.  Plans created afterwards use it. */
int ae_autotune(int n_max, void *stream);
/* The team width the batched solver uses for an instance of order n. */
int ae_team_width(int n);

/*
 * Serving: a request loop with continuous batching.  A worker thread keeps
 * `max_inflight` CUDA streams; each tick it retires finished requests and
 * admits queued ones (FIFO) while a stream is free and the device-memory budget
 * covers the request's scratch and results.  Admitted requests of any kind and
 * size run concurrently on their streams; results stay on the device, owned by
 * the server, until released.  Latency is submit -> observed completion.
 * The solves are those of arrow_eig / dpr1_eig / tri_arrow_svd.  Arrowhead
 * requests of order <= 1024 waiting among the first 1024 of the queue (up to
 * 256, in queue order, all with or all without vectors) are admitted together,
 * ahead of the larger requests between them: one pass of the batched stages
 * (one 32-lane team per eigenpair) on one stream solves them all, each into
 * its own result buffers; their results have the bits arrow_eig gives, except
 * remedied eigenpairs (Remarks 1, 2), which agree within the tolerance.
 */
#define AE_KIND_ARROW 0
#define AE_KIND_DPR1 1
#define AE_KIND_SVD 2
#define AE_EAGAIN 1005        /* queue full (submit), or result not ready */
#define AE_REQ_QUEUED 0
#define AE_REQ_RUNNING 1
#define AE_REQ_DONE 2
#define AE_REQ_ERROR 3

typedef struct ae_request {
    int kind;            /* AE_KIND_* */
    int n;               /* matrix order */
    const double *d;     /* device: poles (n-1; DPR1: n), caller-owned until DONE/ERROR */
    const double *z;     /* device: spikes (n-1), DPR1: u (n) */
    double alpha;        /* corner (arrow, SVD) or rho (DPR1) */
    int want_vectors;    /* 1: V (and U for SVD) as well */
} ae_request;

typedef struct ae_serve_stats_t {
    long long submitted, admitted, completed, rejected, failed, queued, running;
    size_t bytes_in_use;
    long long eigenpairs;       /* completed eigen/singular pairs */
    double p50_s, p99_s, max_s; /* latency percentiles of completed requests */
    double eigenpairs_per_s;    /* completed pairs / (last completion - first submit) */
    int cuda_error;             /* a CUDA error the worker met, else 0 */
    long long merged;           /* requests admitted in merged batched passes */
} ae_serve_stats_t;

typedef struct ae_server ae_server;
/* budget: bytes of device memory for scratch + held results; queue_cap: bound
   on waiting requests (submit returns AE_EAGAIN beyond it). */
int ae_serve_create(ae_server **srv, size_t hbm_budget_bytes, int max_inflight, int queue_cap,
                    const ae_opts *opts);
int ae_serve_submit(ae_server *srv, const ae_request *req, unsigned long long *ticket);
/* state: AE_REQ_*; latency_s of a finished request, else -1.  Returns the
   request's error status when state is AE_REQ_ERROR. */
int ae_serve_poll(ae_server *srv, unsigned long long ticket, int *state, double *latency_s);
/* Device pointers to a DONE request's results (lambda / sigma, V or Q, U);
   valid until ae_serve_release. */
int ae_serve_result(ae_server *srv, unsigned long long ticket, const double **lambda,
                    const double **V, const double **U);
/* Free a finished request and its results (AE_EAGAIN while it runs). */
int ae_serve_release(ae_server *srv, unsigned long long ticket);
int ae_serve_stats(ae_server *srv, ae_serve_stats_t *stats);
/* Stop the worker, wait for running requests, free everything. */
int ae_serve_destroy(ae_server *srv);

/*
 * arrow_eig_host -- arrow_eig on HOST buffers: copies d and z to the device,
 * solves, and copies lambda (and V, shift, mu when non-NULL) back, all on
 * `stream`, then synchronises.  Host buffers should be pinned for full
 * copy bandwidth.  When V is page-locked memory the device can address
 * (cudaHostAlloc, cudaHostRegister), the solver writes the eigenvector columns
 * into it directly while it computes (each column staged on the device and
 * written once), so the 8 n^2-byte transfer overlaps the solve; otherwise V is
 * computed on the device and copied back after it.  Arguments as arrow_eig;
 * V is n x n with ldv = n.
 */
int arrow_eig_host(int n, const double *d_host, const double *z_host, double alpha,
                   double *lambda_host, double *V_host, double *shift_host,
                   double *mu_host, const ae_opts *opts, ae_info *info, void *stream);

/*
 * arrow_eig_noalloc -- arrow_eig that allocates nothing.  The paper has no
 * counterpart: this is an interface for callers that cannot allocate device
 * memory while they run, e.g. an application that reserves all GPU memory up
 * front and hands the library only its input and output buffers, or a
 * latency-critical loop where an allocation could block, fail under memory
 * pressure or fragment a reserved pool.
 *
 * Arguments, outputs and return codes are those of arrow_eig (opts->profile is
 * ignored).  The solve's scratch lives in one static device array of
 * AE_NOALLOC_SCRATCH_BYTES (4 MiB) that every GPU loading the library holds
 * until the process exits; n is limited to what fits, n <= 20928 (larger n
 * returns AE_ERR_TOO_LARGE without touching the GPU).  The call issues no
 * cudaMalloc/cudaFree and no allocating library routine.
 *  - Its first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress, with that device current) and, with CUDA's
 *    default lazy module loading, is when the array and the solver's kernels
 *    are loaded onto that device, which takes device memory.  So make one
 *    call on each device (an n = 1 call will do) before reserving the rest of
 *    the device's memory and before any stream capture; later calls take none.
 *  - The looked-up address is kept for the life of the process: after a
 *    cudaDeviceReset the entry point must not be called again on that device.
 *  - All calls on a device share the one array: calls that may overlap on the
 *    GPU (different streams, or different host threads) race and corrupt each
 *    other's results.  Serialise them, e.g. on one stream.
 */
#define AE_NOALLOC_SCRATCH_BYTES (4u << 20)
int arrow_eig_noalloc(int n, const double *d, const double *z, double alpha,
                      double *lambda, double *V, int ldv, double *shift, double *mu,
                      const ae_opts *opts, ae_info *info, const ae_diag *diag, void *stream);

/*
 * ae_fma_peaks -- measured fused multiply-add throughput of this GPU's FP64
 * and FP32 pipes in TFLOP/s (2 flops per FMA), the denominators of the
 * solver's roofline.  The paper has no counterpart: it is a measurement aid.
 * A grid that fills every SM runs independent FMA chains (8 per thread, all
 * operands in registers); each rate is the best of three CUDA-event-timed
 * launches after a warm-up
 * (about 0.1 s for FP64, 0.04 s for FP32) on `stream`, which the call
 * synchronises.  Either output pointer (host) may be NULL, not both (-1).
 */
int ae_fma_peaks(double *fp64_tflops, double *fp32_tflops, void *stream);

/*
 * ae_debug_rcp -- the solver's FP64 reciprocal (Newton-Raphson refinement of
 * the hardware approximation) applied to x[0..n) into y, for testing against
 * IEEE division.  Device pointers.
 */
int ae_debug_rcp(int n, const double *x, double *y, void *stream);

/*
 * ae_debug_newton -- the solver's bracketed FP64 finish (the Newton
 * alternative to Algorithm 3's bisection) on one shifted inverse's Pick
 * function F(x) = (b - x) - c (sum_j cj[j] / (1 - x delta[j]) - 1/x), for
 * testing its termination and result from a given start.
 *   m, delta, cj  the m shifted differences delta_j = d_j - sigma (j != i) and
 *                 cj_j = zeta_j^2 / delta_j (device arrays)
 *   b, c          the inverse's element b and c = 1 / zeta_i^2 (> 0)
 *   side          +1: the zero lies right of all poles, -1: left (-6 else)
 *   pole          F's pole nearest that side (1/delta_{i-+1}, or 0)
 *   left < right  a bracket of the zero (-8 else)
 *   x0            first trial point (NaN: the bracket's middle)
 *   dF0, xdF0, rel0  an F' estimate (NaN: none), the point it was taken at
 *                 (NaN: unknown) and its relative error bound (INFINITY: none)
 *   max_iter      cap on FP64 evaluations (>= 1)
 *   out           device double[3]: nu (the final bracket's right end), the
 *                 FP64 evaluations, those that also formed F'
 * Runs on one thread; returns AE_OK, -k for argument k, or AE_ERR_CUDA.
 */
int ae_debug_newton(int m, const double *delta, const double *cj, double b, double c, int side,
                    double pole, double left, double right, double x0, double dF0, double xdF0,
                    double rel0, int max_iter, double *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* ARROWHEAD_H */
