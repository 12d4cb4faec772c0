// ae_solve.cuh -- the pipeline after the reduction, as templates over the
// problem kind: one warp per eigenpair (Algorithm 1's shift, Algorithm 2's
// inverse with b by Theorem 6 under Algorithm 5's gate, Algorithm 3's
// bisection or the bracketed Newton finish, the column of Eq. (eigenvecAi)),
// the remedies of Theorem C1 and Remarks 1-2, output placement and the
// remaining columns.  ae_arrow.cu instantiates it for the arrowhead itself;
// each other kind has a translation unit of its own (ae_solve_*.cu), so that
// the kinds compile in parallel.
#pragma once

#include <cuda_runtime.h>

#include "ae_internal.h"
#include "ae_pipeline.cuh"

namespace ae {

// ---------------------------------------------------------------------------
// eigenpairs
// ---------------------------------------------------------------------------
// With va.fused, each warp writes eigenpair k's column right after solving it
// (pass 1 staged in its stored-pair slice, which the solve no longer needs), at
// the position k + #(deflated values >= lambda_k) that the placement gives.
template <Kind K, Kind VK>
__global__ void __launch_bounds__(256, 3) k_eig(Scratch S, SolveOpts o, VecArgs va) {
    const int lane = threadIdx.x & 31;
    const int m = S.cnt[C_M];
    const auto R = PolesOf<K>::make(S, m);
    const WarpTeam T{lane};
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    double2 *buf = S.wbuf ? S.wbuf + gw * S.wstride : nullptr;
    // a part also solves the eigenpair on each side of its range (Algorithm
    // 1's solve only, the same bits its owner computes): the remedy decision
    // of Eq. (K0) needs both neighbours.  Its tickets start at its first such
    // eigenpair (k_part sets the counter); the range is re-read per item
    // rather than held in registers across the solve.
    const int k_hi = S.cnt[C_PART] ? S.cnt[C_KHI] : m + 1;
    for (;;) {
        int k = 0;
        if (lane == 0) k = atomicAdd(S.cnt + C_WORK, 1);
        k = __shfl_sync(FULL, k, 0);
        if (k >= k_hi) break;
        eig_item<K>(R, T, S, k, o, buf);
        if (va.fused && (!__ldcg(S.cnt + C_PART) ||
                         (k >= __ldcg(S.cnt + C_K0) && k < __ldcg(S.cnt + C_K1)))) {
            __syncwarp();
            if (lane == 0) {
                place_item(S, k);
                S.pos0[k] = S.pos[k];
            }
            __syncwarp();
            vector_item<VK>(va.n, va.n1, va.key, va.spk, va.z, va.zrow, va.alpha, va.sgn, S,
                            va.out, k, T, (double *)buf, true, true);
        }
    }
}

// Remedy decisions: one thread per eigenpair (of the part).  The solves on a
// DPR1 inverse (Remarks 1, 2(b)), which add a double-double pass, are listed
// from the front of the n-entry list and the others from its back, so that
// the remedy kernel deals the costlier ones out first, one per SM in turn.
static __global__ void k_fix_decide(Kind kind, Scratch S, double knu_max, int n) {
    const PartRange P = part_range(S);
    const int k = P.k0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P.k1) return;
    const int r = fix_decide_item(kind, S, k, knu_max);
    if (r == AE_FLAG_OTHERPOLE) S.fixlist[n - 1 - atomicAdd(S.cnt + C_NFIX2, 1)] = k;
    else if (r) S.fixlist[atomicAdd(S.cnt + C_NFIX, 1)] = k;
}

// remedy w of the list k_fix_decide wrote (front part first, then the back)
__device__ __forceinline__ int fix_at(const Scratch &S, long long w, int n) {
    const int nf = S.cnt[C_NFIX];
    return w < nf ? S.fixlist[w] : S.fixlist[n - 1 - (int)(w - nf)];
}

// Remedy solves by teams of NW warps (NW = 8, 4 or 2) that share their CTA:
// team g of CTA b takes remedies w = g * grid + b, then w + teams, ... (so that
// consecutive remedies land on different SMs), each on the stored-pair slice
// of the team's first warp (the grid never exceeds k_eig's, so the slices
// exist).  With va.fused the same team rewrites the remedied eigenpair's
// column (its position recorded in pos0, as k_eig does).
template <Kind K, Kind VK, int NW>
__device__ __forceinline__ void fix_solve_teams(const Scratch &S, const SolveOpts &o,
                                                const VecArgs &va, int nfix, double *red) {
    constexpr int TPC = 8 / NW;                  // teams per CTA of 8 warps
    const int m = S.cnt[C_M];
    const auto R = PolesOf<K>::make(S, m);
    const int g = (int)(threadIdx.x >> 5) / NW;
    const CtaTeam<NW> T{(int)threadIdx.x - g * 32 * NW, red + 2 * NW * g, NW == 8 ? 0 : 1 + g};
    const long long w0 = (long long)blockIdx.x * 8 + (long long)g * NW;
    double2 *buf = S.wbuf ? S.wbuf + w0 * S.wstride : nullptr;
    for (long long w = (long long)g * gridDim.x + blockIdx.x; w < nfix;
         w += (long long)TPC * gridDim.x) {
        const int k = fix_at(S, w, va.n);
        const bool kept = fix_solve_item<K>(R, T, S, k, o, buf);
        if (va.fused) {
            T.sync();
            if (T.rank == 0) {
                place_item(S, k);
                S.pos0[k] = S.pos[k];
            }
            T.sync();
            vector_item<VK>(va.n, va.n1, va.key, va.spk, va.z, va.zrow, va.alpha, va.sgn, S,
                            va.out, k, T, (double *)buf, true, kept);
        }
        T.sync();                                // before buf and red are reused
    }
}

// Remedy solves.  The team size is the largest of 8, 4, 2 warps that still
// gives every listed eigenpair a team of its own (one wave over the grid);
// with more remedies than half the grid's warps, one warp each, remedy w on
// warp w / CTAs of CTA w mod CTAs: spread over all SMs.
template <Kind K, Kind VK>
__global__ void __launch_bounds__(256) k_fix_solve(Scratch S, SolveOpts o, VecArgs va) {
    __shared__ double red[16];
    const int nfix = S.cnt[C_NFIX] + S.cnt[C_NFIX2];
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    if (nfix == 0) return;
    if (nwarps / 8 >= nfix) {
        fix_solve_teams<K, VK, 8>(S, o, va, nfix, red);
    } else if (nwarps / 4 >= nfix) {
        fix_solve_teams<K, VK, 4>(S, o, va, nfix, red);
    } else if (nwarps / 2 >= nfix) {
        fix_solve_teams<K, VK, 2>(S, o, va, nfix, red);
    } else {
        const int m = S.cnt[C_M];
        const auto R = PolesOf<K>::make(S, m);
        const int lane = threadIdx.x & 31;
        const WarpTeam T{lane};
        const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        double2 *buf = S.wbuf ? S.wbuf + gw * S.wstride : nullptr;
        // (tickets would hand consecutive remedies to the warps of the first
        // CTAs to arrive, on a few SMs)
        const int wi = threadIdx.x >> 5;
        for (long long w = (long long)wi * gridDim.x + blockIdx.x; w < nfix;
             w += (long long)(blockDim.x >> 5) * gridDim.x) {
            const int k = fix_at(S, w, va.n);
            const bool kept = fix_solve_item<K>(R, T, S, k, o, buf);
            if (va.fused) {
                __syncwarp();
                if (lane == 0) {
                    place_item(S, k);
                    S.pos0[k] = S.pos[k];
                }
                __syncwarp();
                vector_item<VK>(va.n, va.n1, va.key, va.spk, va.z, va.zrow, va.alpha, va.sgn,
                                S, va.out, k, T, (double *)buf, true, kept);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// output placement and vectors
// ---------------------------------------------------------------------------
static __global__ void k_place(Scratch S) {
    const PartRange P = part_range(S);
    const int ncomp = S.cnt[C_M] + 1;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int nk = P.k1 - P.k0;
    if (i < nk) place_item(S, P.k0 + i);
    else if (i < nk + P.u1 - P.u0) place_item(S, ncomp + P.u0 + (i - nk));
}

// All columns, or with va.fused (k_eig and k_fix_solve wrote the computed
// ones) only those whose final position differs from the one used then, and
// the deflated ones; the scalar outputs of every item (K_nu and the remedy
// flags are known only now).  Staged in the warps' stored-pair slices when
// there are enough of them.
template <Kind K>
__global__ void __launch_bounds__(256) k_vectors(VecArgs va, Scratch S) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int ncomp = S.cnt[C_M] + 1;
    const PartRange P = part_range(S);
    const int nk = P.k1 - P.k0;
    const int nitems = nk + P.u1 - P.u0;
    const WarpTeam T{lane};
    double *stage = (S.wbuf && va.fused) ? (double *)(S.wbuf + (long long)warp * S.wstride)
                                         : nullptr;
    for (int i = warp; i < nitems; i += nwarps) {
        const int item = i < nk ? P.k0 + i : ncomp + P.u0 + (i - nk);
        const bool cols = !(va.fused && item < ncomp) || S.pos[item] != S.pos0[item];
        vector_item<K>(va.n, va.n1, va.key, va.spk, va.z, va.zrow, va.alpha, va.sgn, S, va.out,
                       item, T, stage, cols);
    }
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

// K: the arrowhead the kernels solve; VK: the kind of the vector epilogue
// (Hermitian and non-symmetric inputs solve the real arrowhead of their moduli).
// grid: k_eig's CTAs, no more than the stored-pair slices allocated (8 a CTA).
template <Kind K, Kind VK>
static void launch_pipeline(int n, int grid, Scratch S, const SolveOpts &so,
                            const RunOpts &ro, const VecArgs &va, cudaStream_t st) {
    const int sms = sm_count();
    if (ro.ev[1]) cudaEventRecord(ro.ev[1], st);
    k_eig<K, VK><<<grid, 256, 0, st>>>(S, so, va);
    if (ro.ev[2]) cudaEventRecord(ro.ev[2], st);
    if (ro.fixup) {
        k_fix_decide<<<(n + 255) / 256, 256, 0, st>>>(K, S, ro.knu_max, n);
        // every CTA resident at once (the remedies are assigned statically)
        static int fix_per_sm = 0;
        if (!fix_per_sm) {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fix_per_sm, k_fix_solve<K, VK>, 256, 0);
            if (fix_per_sm <= 0) fix_per_sm = 1;
        }
        int fgrid = sms * fix_per_sm;
        fgrid = fgrid < grid ? fgrid : grid;
        fgrid = n < fgrid ? n : fgrid;
        k_fix_solve<K, VK><<<fgrid, 256, 0, st>>>(S, so, va);
    }
    if (ro.ev[3]) cudaEventRecord(ro.ev[3], st);
    k_place<<<(n + 255) / 256, 256, 0, st>>>(S);
    // fused: one warp per stored-pair slice, so every warp can stage
    int vgrid = (n + 7) / 8;
    const int vcap = va.fused ? grid : sms * 16;
    vgrid = vgrid < vcap ? vgrid : vcap;
    k_vectors<VK><<<vgrid, 256, 0, st>>>(va, S);
}

// The pipeline for each kind other than the arrowhead, one translation unit
// each (ae_solve_dpr1.cu, ae_solve_svd.cu, ae_solve_herm.cu, ae_solve_nsym.cu).
void launch_pipeline_dpr1(int n, int grid, Scratch S, const SolveOpts &so, const RunOpts &ro,
                          const VecArgs &va, cudaStream_t st);
void launch_pipeline_tsvd(int n, int grid, Scratch S, const SolveOpts &so, const RunOpts &ro,
                          const VecArgs &va, cudaStream_t st);
void launch_pipeline_herm(int n, int grid, Scratch S, const SolveOpts &so, const RunOpts &ro,
                          const VecArgs &va, cudaStream_t st);
void launch_pipeline_nsym(int n, int grid, Scratch S, const SolveOpts &so, const RunOpts &ro,
                          const VecArgs &va, cudaStream_t st);

}  // namespace ae
