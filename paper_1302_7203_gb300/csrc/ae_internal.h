// ae_internal.h -- types shared by the library's translation units (not part
// of the public C ABI, which is include/arrowhead.h).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "arrowhead.h"

namespace ae {

// slots of the int counter block
enum {
    C_M = 0,          // number of reduced poles m
    C_ND = 1,         // number of deflated rows
    C_FLAGS = 2,      // CF_* bits from k_check
    C_WORK = 3,       // work ticket of k_eig
    C_NFIX = 4,       // remedies listed from the front of the remedy list
    C_NFIX2 = 5,      // remedies listed from the back of the remedy list
    C_NEARZERO = 6,
    C_OTHERPOLE = 7,
    C_DPR1 = 8,
    C_CAPPED = 9,
    C_MAXIT = 10,
    C_FP32FB = 11,
    C_DDB = 12,       // b recomputed in double-double under the Algorithm 5 gate
    C_MID64 = 13,     // FP32 midpoint tests that needed the FP64 pass
    // one part of a split solve (arrow_eig_part); C_PART = 0: the whole problem
    C_PART = 14,
    C_K0 = 15,        // computed eigenpairs [k0, k1) of the reduced arrowhead
    C_K1 = 16,
    C_U0 = 17,        // deflated rows [u0, u1) (in sorted order)
    C_U1 = 18,
    C_POS0 = 19,      // output position of the part's first item
    C_KHI = 20,       // end of the eigenpairs k_eig solves (the part's range and its edges)
    C_COUNT = 21
};
enum { C64_ITERS = 0, C64_MAXKB = 1, C64_MAXKNU = 2, C64_ITERS_FIX = 3, C64_DERIV = 4,
       C64_F32 = 5,     // O(n) passes in FP32 (midpoint tests, FP32 steps and brackets)
       C64_DF = 6,      // O(n) passes in double-float (opening model steps)
       C64_COUNT = 7 };

// k_check flag bits
enum { CF_UNSORTED = 1, CF_ZERO = 2, CF_BAD = 4, CF_ZEROPOLE = 8 };

// problem kinds sharing the pipeline
// (HERM and NSYM are solved as the real arrowhead with spikes |zeta_r|, resp.
// sqrt(zc_r zr_r), and exact double-double squares; they differ only in the
// input check, the squares and the vector epilogue)
enum Kind { KIND_ARROW = 0, KIND_DPR1 = 1, KIND_TSVD = 2, KIND_HERM = 3, KIND_NSYM = 4 };

// slots of the per-solve double parameters
enum {
    P_ALPHA_HI = 0,   // corner of the arrowhead solved (double-double)
    P_ALPHA_LO = 1,
    P_PLAST = 2,      // DPR1: the last reduced pole (not an arrowhead pole)
    P_DS = 3,         // FP32 copies: pole scale
    P_ZS = 4,         // FP32 copies: spike^2 scale
    P_ZSUM = 5,       // sum of the reduced |zeta_j| (Algorithm 5's spike ratio)
    P_COUNT = 8
};

struct Scratch {
    int *cnt;
    unsigned long long *cnt64;
    int *perm;      // sorted position -> input row
    int *spos;      // input row -> sorted position
    int *kind;      // input row: 0 pole head, 1 zero spike, 2 folded into a run
    int *run_s0;    // folded row: sorted position where its run starts
    double *run_R;  // folded row: R_{m-1}, R_m
    double *key, *spk;      // transformed inputs (DPR1 with rho < 0: -d; SVD: d z)
    double *pd, *pz, *pz2;  // reduced keys (poles; SVD: d_j) / spikes / fl(spike^2)
    double *pz2lo;          // spike^2 = pz2 + pz2lo (double-double)
    double *pv;             // pole values (SVD: fl(d_j^2); else = pd)
    float *pdh, *pdl, *pz2f;  // FP32 copies: key*ds split hi+lo, spike^2*zs
    double *prm;              // P_* parameters
    int *prow;      // reduced pole -> input row of its head
    int *drow;      // deflated rows in sorted order
    double *dval;   // their pole values
    double *es_sigma, *es_mu, *es_lam, *es_b, *es_Kb, *es_Knu, *es_fixshift;
    int *es_pole, *es_iters, *es_flags, *es_fixpole, *fixlist;
    int *pos;       // output position of computed (first m+1) and deflated items
    int *pos0;      // computed item: the position its column was first written at
    double2 *wbuf;  // optional: one (delta_j, c_j) slice per eig team, wstride apart
    long long wstride;
};

struct Outputs {
    double *lambda;     // eigenvalues (SVD: singular values)
    double *V;          // eigenvectors (DPR1: Q; SVD: right singular vectors)
    long long ldv;
    double *U;          // SVD: left singular vectors
    long long ldu;
    double *shift, *mu;
    double *dg_b, *dg_Kb, *dg_Knu;
    int *dg_iters, *dg_flags;
};

// What the eigenvector epilogue needs (the transformed inputs the reduction
// saw, the caller's spikes, the outputs).  fused != 0: the eigenvalue kernel
// writes each column as soon as its eigenvalue is known, staged in the warp's
// stored-pair slice, and the vector kernel later only rewrites the columns
// that the remedies or the final placement changed (and the deflated ones).
struct VecArgs {
    int n, n1;
    const double *key, *spk, *z, *zrow;
    double alpha, sgn;
    Outputs out;
    int fused;
};

struct RunOpts {
    int precision;
    double knu_max;
    int max_iter;
    int fixup;
    int finish;
    int bgate;
    double kb_max;
    cudaEvent_t ev[5];   // phase boundaries when profiling (else null)
};

// Validate *o (null: the defaults) into ro; nonzero when a field is out of range.
int resolve_opts(const ae_opts *o, RunOpts &ro);

size_t arrow_scratch_bytes(int n);
// warps of the eigenvalue kernel for order n (the stored-pair buffer holds one
// slice of n pairs per warp)
int eig_grid_warps(int n);
Scratch carve_scratch(void *base, int n);
// Issue a whole solve on `st`.  ARROW: d, z have n-1 entries; DPR1: d, u (in z)
// have n entries and rho is used; SVD: d, z have n-1 entries; HERM: z holds n-1
// complex spikes (re, im interleaved), out.V is complex (ldv in doubles); NSYM:
// z the column spikes, zrow the row spikes, out.V / out.U the right / left
// vectors.
cudaError_t launch_solve(Kind kind, int n, const double *d, const double *z, double alpha,
                         double rho, const Outputs &out, const RunOpts &ro, Scratch S,
                         cudaStream_t st, const double *zrow = nullptr);
inline cudaError_t launch_arrow(int n, const double *d, const double *z, double alpha,
                                const Outputs &out, const RunOpts &ro, Scratch S,
                                cudaStream_t st) {
    return launch_solve(KIND_ARROW, n, d, z, alpha, 0.0, out, ro, S, st);
}
// One part of a split arrow_eig (see arrow_eig_part): the reduction, then
// (after a synchronisation that returns the part's first output position and
// item count) the pipeline on the part's items, unless out.lambda is null or
// the count exceeds cap.
cudaError_t launch_arrow_part(int n, const double *d, const double *z, double alpha, int part,
                              int nparts, int cap, const Outputs &out, const RunOpts &ro,
                              Scratch S, cudaStream_t st, int *pos0, int *count);
cudaError_t launch_debug_rcp(int n, const double *x, double *y, cudaStream_t st);
// arguments of the FP64-finish test hook (ae_debug_newton)
struct DebugNewton {
    double b, c, pole, left, right, x0, dF0, xdF0, rel0;
    int side, max_iter;
};
cudaError_t launch_debug_newton(int m, const double *delta, const double *cj,
                                const DebugNewton &a, double *out, cudaStream_t st);
// Requests of the serving loop solved together by the batched stages (see
// ae_batch.cu): the device block they need, and the launch.
size_t req_batch_bytes(int count, const int *ns);
cudaError_t launch_req_batch(int count, const int *ns, const double *const *d,
                             const double *const *z, const double *alpha, double *const *lam,
                             double *const *V, void *block, const RunOpts &ro, cudaStream_t st,
                             const int **cnt);
// FMA throughput of the FP64 and FP32 pipes (TFLOP/s), either pointer may be null
cudaError_t probe_fma_rates(double *fp64_tflops, double *fp32_tflops, cudaStream_t st);
// remember a CUDA error for ae_last_cuda_error()
void record_cuda_error(cudaError_t e);

}  // namespace ae
