// ae_batch.cu -- many arrowheads of uneven order solved together.
//
// All instances go through the same pipeline as arrow_eig, but each stage is
// ONE persistent launch over every instance:
//   k_batch_prep      one CTA per instance: checks, order, reduction, FP32 copies
//   k_batch_eig       global work queue of (instance, eigenpair) units; a unit
//                     is 32/W eigenpairs of one instance solved by W-lane teams
//                     (W = 8, 16 or 32, chosen per order bucket by the tuner)
//   k_batch_fix_*     remedy decisions over all eigenpairs, one CTA per remedy
//   k_batch_place / k_batch_vectors / k_batch_status
// A plan (ae_batch_create) owns the descriptor table and the scratch of every
// instance and captures the whole sequence in a CUDA graph that
// ae_batch_run replays.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <sys/stat.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "ae_pipeline.cuh"

namespace ae {

// ---------------------------------------------------------------------------
// sub-warp teams: W consecutive lanes of a warp share one eigenpair
// ---------------------------------------------------------------------------
template <int W>
struct SubWarpTeam {
    int rank;        // lane within the team
    unsigned mask;   // the team's lanes
    static constexpr int size = W;
    __device__ __forceinline__ double sum(double v) const {
#pragma unroll
        for (int o = W / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
        return v;
    }
    __device__ __forceinline__ float sumf(float v) const {
#pragma unroll
        for (int o = W / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
        return v;
    }
    __device__ __forceinline__ dd sum(dd v) const {
#pragma unroll
        for (int o = W / 2; o > 0; o >>= 1) {
            dd w = {__shfl_xor_sync(mask, v.hi, o), __shfl_xor_sync(mask, v.lo, o)};
            v = dd_add(v, w);
        }
        return v;
    }
    __device__ __forceinline__ double max(double v) const {
#pragma unroll
        for (int o = W / 2; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(mask, v, o));
        return v;
    }
    __device__ __forceinline__ double min(double v) const {
#pragma unroll
        for (int o = W / 2; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(mask, v, o));
        return v;
    }
    __device__ __forceinline__ void sync() const { __syncwarp(mask); }
};

struct BatchInst {
    int n, n1;
    const double *d, *z, *alpha;   // device inputs of this instance
    Scratch S;
    Outputs out;
    int team;                      // eigenpair team width W
};

struct BatchCtl {
    int tick_eig, tick_fix, nfix, tick_vec;
};

// index i with off[i] <= t < off[i+1]
__device__ __forceinline__ int find_inst(const long long *off, int count, long long t) {
    int lo = 0, hi = count;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_batch_prep(const BatchInst *__restrict__ I,
                                                     BatchCtl *ctl) {
    __shared__ double tile[1024];
    __shared__ int sflags;
    const BatchInst &B = I[blockIdx.x];
    const Scratch &S = B.S;
    const int n1 = B.n1;
    if (blockIdx.x == 0 && threadIdx.x == 0) *ctl = BatchCtl{0, 0, 0, 0};
    if (threadIdx.x < C_COUNT) S.cnt[threadIdx.x] = 0;
    if (threadIdx.x < C64_COUNT) S.cnt64[threadIdx.x] = 0ull;
    if (threadIdx.x == 0) sflags = 0;
    // -1: no column written by the remedy pass (see k_batch_fix_solve)
    for (int k = threadIdx.x; k < B.n; k += blockDim.x) S.pos0[k] = -1;
    __syncthreads();
    int flags = 0;
    for (int r = threadIdx.x; r < n1; r += blockDim.x) {
        const double dr = B.d[r], zr = B.z[r];
        if (!isfinite(dr) || !isfinite(zr)) flags |= CF_BAD;
        if (zr == 0.0) flags |= CF_ZERO;
        if (dr == 0.0) flags |= CF_ZEROPOLE;
        if (r + 1 < n1 && !(dr > B.d[r + 1])) flags |= CF_UNSORTED;
    }
    flags = __reduce_or_sync(FULL, flags);
    if ((threadIdx.x & 31) == 0 && flags) atomicOr(&sflags, flags);
    __syncthreads();
    flags = sflags;
    if (threadIdx.x == 0) S.cnt[C_FLAGS] = flags;
    // order: identity when sorted, else ranks counted against tiles of the poles
    if (!(flags & CF_UNSORTED)) {
        for (int r = threadIdx.x; r < n1; r += blockDim.x) S.perm[r] = r;
    } else {
        for (int rb = 0; rb < n1; rb += blockDim.x) {
            const int r = rb + threadIdx.x;
            const double dr = r < n1 ? (isnan(B.d[r]) ? -INFINITY : B.d[r]) : 0.0;
            int rank = 0;
            for (int base = 0; base < n1; base += 1024) {
                __syncthreads();
                const double v = base + (int)threadIdx.x < n1 ? B.d[base + threadIdx.x] : 0.0;
                tile[threadIdx.x] = isnan(v) ? -INFINITY : v;
                __syncthreads();
                const int lim = min(1024, n1 - base);
                if (r < n1)
                    for (int t = 0; t < lim; ++t) {
                        const double dq = tile[t];
                        rank += (dq > dr) || (dq == dr && base + t < r);
                    }
            }
            if (r < n1) S.perm[rank] = r;
        }
    }
    __syncthreads();
    reduce_block(n1, B.d, B.z, S.perm, S);
    __syncthreads();
    post_block<KIND_ARROW>(n1, B.d, B.z, nullptr, *B.alpha, 0.0, S);
}

// buf: this warp's 4 slices of stored (delta_j, c_j) pairs, `stride` apart
template <int W>
__device__ __forceinline__ void batch_unit(const BatchInst &B, long long unit_in_inst, int lane,
                                           const SolveOpts &o, double2 *buf, long long stride) {
    constexpr int EPW = 32 / W;
    const int m = B.S.cnt[C_M];
    const int g = lane / W;
    const int k = (int)(unit_in_inst * EPW) + g;
    const auto R = PolesOf<KIND_ARROW>::make(B.S, m);
    double2 *tb = buf ? buf + g * stride : nullptr;
    // the solve, then (with vectors and a stored-pair slice) the column at its
    // position as the single-instance k_eig writes it
    auto run = [&](const auto &T) {
        eig_item<KIND_ARROW>(R, T, B.S, k, o, tb);
        if (B.out.V && tb) {
            T.sync();
            if (T.rank == 0) {
                place_item(B.S, k);
                B.S.pos0[k] = B.S.pos[k];
            }
            T.sync();
            // (the stored differences only for whole-warp teams: narrower ones
            // would add a sync per step to the divergent teams of one warp)
            vector_item<KIND_ARROW>(B.n, B.n1, B.d, B.z, B.z, nullptr, *B.alpha, 1.0, B.S,
                                    B.out, k, T, (double *)tb, true, W == 32);
        }
    };
    if constexpr (W == 32) {
        if (k <= m) run(WarpTeam{lane});
    } else {
        const unsigned mask = ((1u << W) - 1u) << (lane & ~(W - 1));
        if (k <= m) run(SubWarpTeam<W>{lane & (W - 1), mask});
    }
}

__global__ void __launch_bounds__(256, 3) k_batch_eig(const BatchInst *__restrict__ I, int count,
                                                   const long long *__restrict__ uoff,
                                                   BatchCtl *ctl, SolveOpts o, double2 *wbuf,
                                                   long long wstride) {
    const int lane = threadIdx.x & 31;
    const long long total = uoff[count];
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    double2 *buf = wbuf ? wbuf + gw * 4 * wstride : nullptr;
    for (;;) {
        long long u = 0;
        if (lane == 0) u = atomicAdd(&ctl->tick_eig, 1);
        u = __shfl_sync(FULL, u, 0);
        if (u >= total) break;
        const int i = find_inst(uoff, count, u);
        const BatchInst &B = I[i];
        const long long ui = u - uoff[i];
        switch (B.team) {
            case 8: batch_unit<8>(B, ui, lane, o, buf, wstride); break;
            case 16: batch_unit<16>(B, ui, lane, o, buf, wstride); break;
            default: batch_unit<32>(B, ui, lane, o, buf, wstride); break;
        }
        __syncwarp();
    }
}

__global__ void k_batch_fix_decide(const BatchInst *__restrict__ I, int count,
                                   const long long *__restrict__ eoff, int2 *fixlist,
                                   BatchCtl *ctl, double knu_max) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= eoff[count]) return;
    const int i = find_inst(eoff, count, t);
    const int k = (int)(t - eoff[i]);
    if (fix_decide_item(KIND_ARROW, I[i].S, k, knu_max)) fixlist[atomicAdd(&ctl->nfix, 1)] = {i, k};
}

// One warp per remedied eigenpair (remedies are many in a batch of small
// instances), on the warp's first stored-pair slice; the warp also rewrites the
// remedied column, which k_batch_vectors then skips unless the final placement
// moved it.
__global__ void __launch_bounds__(256) k_batch_fix_solve(const BatchInst *__restrict__ I,
                                                         const int2 *fixlist, BatchCtl *ctl,
                                                         SolveOpts o, double2 *wbuf,
                                                         long long wstride) {
    const int lane = threadIdx.x & 31;
    const WarpTeam T{lane};
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    double2 *buf = wbuf ? wbuf + gw * 4 * wstride : nullptr;
    for (;;) {
        int w = 0;
        if (lane == 0) w = atomicAdd(&ctl->tick_fix, 1);
        w = __shfl_sync(FULL, w, 0);
        if (w >= ctl->nfix) break;
        const int2 ik = fixlist[w];
        const BatchInst &B = I[ik.x];
        const Scratch &S = B.S;
        const auto R = PolesOf<KIND_ARROW>::make(S, S.cnt[C_M]);
        const bool kept = fix_solve_item<KIND_ARROW>(R, T, S, ik.y, o, buf);
        __syncwarp();
        if (B.out.V && buf) {
            if (lane == 0) {
                place_item(S, ik.y);
                S.pos0[ik.y] = S.pos[ik.y];
            }
            __syncwarp();
            vector_item<KIND_ARROW>(B.n, B.n1, B.d, B.z, B.z, nullptr, *B.alpha, 1.0, S, B.out,
                                    ik.y, T, (double *)buf, true, kept);
        }
        __syncwarp();
    }
}

__global__ void k_batch_place(const BatchInst *__restrict__ I, int count,
                              const long long *__restrict__ eoff) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= eoff[count]) return;
    const int i = find_inst(eoff, count, t);
    place_item(I[i].S, (int)(t - eoff[i]));
}

__global__ void __launch_bounds__(256) k_batch_vectors(const BatchInst *__restrict__ I, int count,
                                                       const long long *__restrict__ eoff,
                                                       BatchCtl *ctl) {
    const int lane = threadIdx.x & 31;
    const long long total = eoff[count];
    for (;;) {
        long long t = 0;
        if (lane == 0) t = atomicAdd(&ctl->tick_vec, 1);
        t = __shfl_sync(FULL, t, 0);
        if (t >= total) break;
        const int i = find_inst(eoff, count, t);
        const BatchInst &B = I[i];
        const int item = (int)(t - eoff[i]);
        const bool cols = !(item <= B.S.cnt[C_M] && B.S.pos0[item] >= 0 &&
                            B.S.pos[item] == B.S.pos0[item]);
        vector_item<KIND_ARROW>(B.n, B.n1, B.d, B.z, B.z, nullptr, *B.alpha, 1.0, B.S, B.out,
                                item, WarpTeam{lane}, nullptr, cols);
        __syncwarp();
    }
}

__global__ void k_batch_status(const BatchInst *__restrict__ I, int count, int *status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int *c = I[i].S.cnt;
    status[i] = (c[C_FLAGS] & CF_BAD) ? AE_ERR_INPUT : (c[C_CAPPED] ? AE_ERR_NOCONV : AE_OK);
}

// ---------------------------------------------------------------------------
// tuner: eigenpair team width per order bucket, cached as JSON
// ---------------------------------------------------------------------------
static std::mutex g_tune_mu;
static std::map<int, int> g_tune;          // bucket -> W
static bool g_tune_loaded = false;

static const char *build_tag() { return __DATE__ " " __TIME__; }

static int bucket_of(int n) {
    int b = 32;
    while (b < n && b < (1 << 24)) b <<= 1;
    return b;
}

static int default_team(int n) { return n <= 48 ? 8 : (n <= 160 ? 16 : 32); }

static std::string device_key() {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
    return std::string(p.name) + "|" + build_tag();
}

static std::string cache_path() {
    const char *e = getenv("AE_TUNE_CACHE");
    if (e && *e) return e;
    const char *h = getenv("HOME");
    return std::string(h ? h : "/tmp") + "/.cache/arrowhead_tune.json";
}

// file format: {"key": "<device>|<build>", "team": {"32": 8, "64": 16, ...}}
static void load_cache_locked() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    FILE *f = fopen(cache_path().c_str(), "r");
    if (!f) return;
    std::string s;
    char buf[4096];
    size_t k;
    while ((k = fread(buf, 1, sizeof buf, f)) > 0) s.append(buf, k);
    fclose(f);
    const std::string want = "\"key\": \"" + device_key() + "\"";
    if (s.find(want) == std::string::npos) return;   // another device or build
    size_t p = s.find("\"team\"");
    if (p == std::string::npos) return;
    p = s.find('{', p);
    while (p != std::string::npos) {
        const size_t q = s.find('"', p + 1);
        if (q == std::string::npos) break;
        const size_t r = s.find('"', q + 1);
        const size_t c = s.find(':', r);
        if (r == std::string::npos || c == std::string::npos) break;
        const int b = atoi(s.substr(q + 1, r - q - 1).c_str());
        const int w = atoi(s.c_str() + c + 1);
        if (b > 0 && (w == 8 || w == 16 || w == 32)) g_tune[b] = w;
        p = s.find(',', c);
    }
}

static void save_cache_locked() {
    const std::string path = cache_path();
    const size_t slash = path.rfind('/');
    if (slash != std::string::npos) {
        const std::string dir = path.substr(0, slash);
        for (size_t i = 1; i <= dir.size(); ++i)
            if (i == dir.size() || dir[i] == '/') mkdir(dir.substr(0, i).c_str(), 0755);
    }
    FILE *f = fopen(path.c_str(), "w");
    if (!f) return;
    fprintf(f, "{\"key\": \"%s\", \"team\": {", device_key().c_str());
    bool first = true;
    for (auto &kv : g_tune) {
        fprintf(f, "%s\"%d\": %d", first ? "" : ", ", kv.first, kv.second);
        first = false;
    }
    fprintf(f, "}}\n");
    fclose(f);
}

int team_for(int n) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    load_cache_locked();
    auto it = g_tune.find(bucket_of(n));
    return it != g_tune.end() ? it->second : default_team(n);
}


// ---------------------------------------------------------------------------
// plans
// ---------------------------------------------------------------------------
static int sm_count_b() {
    int dev = 0, c = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
    return c > 0 ? c : 1;
}

static int batch_eig_grid() {
    static int per_sm = 0;
    if (!per_sm) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_eig, 256, 0);
        if (per_sm <= 0) per_sm = 1;
    }
    return sm_count_b() * per_sm;
}

struct Plan {
    int count = 0;
    long long total_n = 0;
    double2 *wbuf = nullptr;     // 4 slices of stored pairs per warp of k_batch_eig
    long long wstride = 0;
    BatchInst *d_inst = nullptr;
    long long *d_eoff = nullptr, *d_uoff = nullptr;
    int2 *d_fix = nullptr;
    BatchCtl *d_ctl = nullptr;
    void *scratch = nullptr;
    int *status = nullptr;
    SolveOpts so{};
    RunOpts ro{};
    cudaGraphExec_t exec = nullptr;
    std::vector<BatchInst> host;
};

static void enqueue(const Plan &P, cudaStream_t st) {
    const int sms = sm_count_b();
    k_batch_prep<<<P.count, 1024, 0, st>>>(P.d_inst, P.d_ctl);
    k_batch_eig<<<batch_eig_grid(), 256, 0, st>>>(P.d_inst, P.count, P.d_uoff, P.d_ctl, P.so,
                                                  P.wbuf, P.wstride);
    const unsigned g = (unsigned)((P.total_n + 255) / 256);
    if (P.ro.fixup) {
        k_batch_fix_decide<<<g, 256, 0, st>>>(P.d_inst, P.count, P.d_eoff, P.d_fix, P.d_ctl,
                                              P.ro.knu_max);
        k_batch_fix_solve<<<batch_eig_grid(), 256, 0, st>>>(P.d_inst, P.d_fix, P.d_ctl, P.so,
                                                             P.wbuf, P.wstride);
    }
    k_batch_place<<<g, 256, 0, st>>>(P.d_inst, P.count, P.d_eoff);
    k_batch_vectors<<<sms * 16, 256, 0, st>>>(P.d_inst, P.count, P.d_eoff, P.d_ctl);
    if (P.status) k_batch_status<<<(P.count + 255) / 256, 256, 0, st>>>(P.d_inst, P.count, P.status);
}

static void free_plan(Plan *P) {
    if (!P) return;
    if (P->exec) cudaGraphExecDestroy(P->exec);
    cudaFree(P->d_inst);
    cudaFree(P->d_eoff);
    cudaFree(P->d_uoff);
    cudaFree(P->d_fix);
    cudaFree(P->d_ctl);
    cudaFree(P->scratch);
    cudaFree(P->wbuf);
    delete P;
}

// Build the descriptor table and scratch; `force_team` > 0 overrides the tuner.
static cudaError_t build_plan(Plan *P, int count, const long long *n_off, const long long *v_off,
                              const double *d_all, const double *z_all, const double *alpha_all,
                              double *lambda_all, double *V_all, int *status_all,
                              const RunOpts &ro, int force_team, cudaStream_t st) {
    P->count = count;
    P->status = status_all;
    P->ro = ro;
    P->so = SolveOpts{ro.max_iter, ro.precision, ro.finish, ro.bgate, ro.kb_max};
    std::vector<size_t> soff(count + 1, 0);
    for (int i = 0; i < count; ++i) {
        const int n = (int)(n_off[i + 1] - n_off[i]);
        soff[i + 1] = soff[i] + ((arrow_scratch_bytes(n) + 255) & ~(size_t)255);
    }
    P->total_n = n_off[count];
    cudaError_t e;
    if ((e = cudaMalloc(&P->scratch, soff[count] + 256))) return e;
    if ((e = cudaMalloc(&P->d_inst, sizeof(BatchInst) * count))) return e;
    if ((e = cudaMalloc(&P->d_eoff, sizeof(long long) * (count + 1)))) return e;
    if ((e = cudaMalloc(&P->d_uoff, sizeof(long long) * (count + 1)))) return e;
    if ((e = cudaMalloc(&P->d_fix, sizeof(int2) * (size_t)(P->total_n > 0 ? P->total_n : 1))))
        return e;
    if ((e = cudaMalloc(&P->d_ctl, sizeof(BatchCtl)))) return e;
    long long nmax = 1;
    for (int i = 0; i < count; ++i) nmax = std::max(nmax, n_off[i + 1] - n_off[i]);
    P->wstride = (nmax + 1) & ~1LL;
    if ((e = cudaMalloc(&P->wbuf, sizeof(double2) * P->wstride * 4 *
                                      (size_t)batch_eig_grid() * 8)))
        return e;
    P->host.resize(count);
    std::vector<long long> uoff(count + 1, 0);
    long long vo = 0;
    for (int i = 0; i < count; ++i) {
        const int n = (int)(n_off[i + 1] - n_off[i]);
        BatchInst &B = P->host[i];
        B.n = n;
        B.n1 = n - 1;
        B.d = d_all + (n_off[i] - i);
        B.z = z_all + (n_off[i] - i);
        B.alpha = alpha_all + i;
        B.S = carve_scratch((char *)P->scratch + soff[i], n);
        B.out.lambda = lambda_all + n_off[i];
        const long long vi = v_off ? v_off[i] : vo;
        B.out.V = V_all ? V_all + vi : nullptr;
        B.out.ldv = n;
        B.out.U = nullptr;
        B.out.ldu = 0;
        B.out.shift = B.out.mu = nullptr;
        B.out.dg_b = B.out.dg_Kb = B.out.dg_Knu = nullptr;
        B.out.dg_iters = B.out.dg_flags = nullptr;
        B.team = force_team > 0 ? force_team : team_for(n);
        vo += (long long)n * n;
        uoff[i + 1] = uoff[i] + (n + (32 / B.team) - 1) / (32 / B.team);
    }
    if ((e = cudaMemcpyAsync(P->d_inst, P->host.data(), sizeof(BatchInst) * count,
                             cudaMemcpyHostToDevice, st)))
        return e;
    if ((e = cudaMemcpyAsync(P->d_eoff, n_off, sizeof(long long) * (count + 1),
                             cudaMemcpyHostToDevice, st)))
        return e;
    if ((e = cudaMemcpyAsync(P->d_uoff, uoff.data(), sizeof(long long) * (count + 1),
                             cudaMemcpyHostToDevice, st)))
        return e;
    return cudaStreamSynchronize(st);
}

// ---------------------------------------------------------------------------
// a batch of separate requests (the serving loop): instances with their own
// input and output buffers, solved by one pass of the batched stages
// ---------------------------------------------------------------------------
// Layout of the one device block a request batch needs: descriptors, prefix
// tables, remedy list, control block, corners, per-instance scratch and the
// stored-pair slices; every part 256-byte aligned.
struct ReqBatchLayout {
    size_t inst, eoff, uoff, fix, ctl, alpha, scratch, wbuf, total;
    long long wstride;
    std::vector<size_t> soff;
};

static ReqBatchLayout req_batch_layout(int count, const int *ns) {
    ReqBatchLayout L;
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    long long total_n = 0, nmax = 1;
    L.soff.assign(count + 1, 0);
    for (int i = 0; i < count; ++i) {
        total_n += ns[i];
        nmax = std::max<long long>(nmax, ns[i]);
        L.soff[i + 1] = L.soff[i] + up(arrow_scratch_bytes(ns[i]));
    }
    L.wstride = (nmax + 1) & ~1LL;
    size_t p = 0;
    L.inst = p; p += up(sizeof(BatchInst) * count);
    L.eoff = p; p += up(sizeof(long long) * (count + 1));
    L.uoff = p; p += up(sizeof(long long) * (count + 1));
    L.fix = p;  p += up(sizeof(int2) * (size_t)(total_n > 0 ? total_n : 1));
    L.ctl = p;  p += up(sizeof(BatchCtl));
    L.alpha = p; p += up(sizeof(double) * count);
    L.scratch = p; p += L.soff[count];
    L.wbuf = p; p += sizeof(double2) * (size_t)L.wstride * 4 * (size_t)batch_eig_grid() * 8;
    L.total = p + 256;
    return L;
}

size_t req_batch_bytes(int count, const int *ns) { return req_batch_layout(count, ns).total; }

// Solve `count` arrowhead requests (orders ns, inputs d[i], z[i] with corner
// alpha[i], outputs lam[i] and V[i] with ld = n) with the batched stages on
// `st`, using the device block `block` of req_batch_bytes() bytes.  Every
// eigenpair is solved by a 32-lane team, so each result has the bits the
// single-instance solve gives (remedies, solved by a warp here and by a team
// as wide as one wave allows there, agree within the tolerance).  cnt[i]
// receives the device address of instance i's counters (C_COUNT ints).
cudaError_t launch_req_batch(int count, const int *ns, const double *const *d,
                             const double *const *z, const double *alpha, double *const *lam,
                             double *const *V, void *block, const RunOpts &ro, cudaStream_t st,
                             const int **cnt) {
    const ReqBatchLayout L = req_batch_layout(count, ns);
    char *b = (char *)(((uintptr_t)block + 255) & ~(uintptr_t)255);
    Plan P;
    P.count = count;
    P.ro = ro;
    P.so = SolveOpts{ro.max_iter, ro.precision, ro.finish, ro.bgate, ro.kb_max};
    P.d_inst = (BatchInst *)(b + L.inst);
    P.d_eoff = (long long *)(b + L.eoff);
    P.d_uoff = (long long *)(b + L.uoff);
    P.d_fix = (int2 *)(b + L.fix);
    P.d_ctl = (BatchCtl *)(b + L.ctl);
    P.wbuf = (double2 *)(b + L.wbuf);
    P.wstride = L.wstride;
    double *d_alpha = (double *)(b + L.alpha);
    std::vector<BatchInst> host(count);
    std::vector<long long> eoff(count + 1, 0), uoff(count + 1, 0);
    for (int i = 0; i < count; ++i) {
        BatchInst &B = host[i];
        B.n = ns[i];
        B.n1 = ns[i] - 1;
        B.d = d[i];
        B.z = z[i];
        B.alpha = d_alpha + i;
        B.S = carve_scratch(b + L.scratch + L.soff[i], ns[i]);
        B.out = Outputs{};
        B.out.lambda = lam[i];
        B.out.V = V ? V[i] : nullptr;
        B.out.ldv = ns[i];
        B.team = 32;
        eoff[i + 1] = eoff[i] + ns[i];
        uoff[i + 1] = uoff[i] + ns[i];
        cnt[i] = B.S.cnt;
    }
    P.total_n = eoff[count];
    // (pageable sources: each copy is staged before the call returns)
    cudaError_t e = cudaMemcpyAsync(P.d_inst, host.data(), sizeof(BatchInst) * count,
                                    cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemcpyAsync(P.d_eoff, eoff.data(), sizeof(long long) * (count + 1),
                                cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemcpyAsync(P.d_uoff, uoff.data(), sizeof(long long) * (count + 1),
                                cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemcpyAsync(d_alpha, alpha, sizeof(double) * count, cudaMemcpyHostToDevice,
                                st);
    if (e) return e;
    enqueue(P, st);
    return cudaGetLastError();
}

static cudaError_t capture_plan(Plan *P) {
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e) return e;
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (!e) {
        enqueue(*P, cs);
        e = cudaStreamEndCapture(cs, &g);
    }
    if (!e) e = cudaGraphInstantiate(&P->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    return e;
}

static cudaError_t plan_info(const Plan &P, ae_info *info, cudaStream_t st) {
    std::vector<int> cnt((size_t)P.count * C_COUNT);
    std::vector<unsigned long long> c64((size_t)P.count * C64_COUNT);
    for (int i = 0; i < P.count; ++i) {
        cudaError_t e = cudaMemcpyAsync(&cnt[(size_t)i * C_COUNT], P.host[i].S.cnt,
                                        sizeof(int) * C_COUNT, cudaMemcpyDeviceToHost, st);
        if (!e) e = cudaMemcpyAsync(&c64[(size_t)i * C64_COUNT], P.host[i].S.cnt64,
                                    sizeof(unsigned long long) * C64_COUNT,
                                    cudaMemcpyDeviceToHost, st);
        if (e) return e;
    }
    cudaError_t e = cudaStreamSynchronize(st);
    if (e) return e;
    memset(info, 0, sizeof(*info));
    for (int i = 0; i < P.count; ++i) {
        const int *c = &cnt[(size_t)i * C_COUNT];
        const unsigned long long *u = &c64[(size_t)i * C64_COUNT];
        info->n_reduced += c[C_M] + 1;
        info->n_deflated += c[C_ND];
        info->n_nearzero += c[C_NEARZERO];
        info->n_otherpole += c[C_OTHERPOLE];
        info->n_dpr1shift += c[C_DPR1];
        info->n_capped += c[C_CAPPED];
        info->n_fp32_fallback += c[C_FP32FB];
        info->n_ddb += c[C_DDB];
        info->n_mid64 += c[C_MID64];
        info->total_deriv += (long long)u[C64_DERIV];
        info->n_f32_passes += (long long)u[C64_F32];
        info->n_df_passes += (long long)u[C64_DF];
        if (c[C_MAXIT] > info->max_iter_used) info->max_iter_used = c[C_MAXIT];
        info->total_iter += (long long)u[C64_ITERS];
        info->fix_iter += (long long)u[C64_ITERS_FIX];
        double kb, kn;
        memcpy(&kb, &u[C64_MAXKB], sizeof kb);
        memcpy(&kn, &u[C64_MAXKNU], sizeof kn);
        if (kb > info->max_Kb) info->max_Kb = kb;
        if (kn > info->max_Knu) info->max_Knu = kn;
    }
    return cudaSuccess;
}

// synthetic instances for the tuner's timing runs (not part of any solve):
// d_r strictly decreasing in [-10, 10], z_r in (0, 1], alpha in [-1, 1]
__device__ __forceinline__ double hash01(unsigned long long x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x ^= x >> 31;
    return (double)(x >> 11) * 0x1p-53;
}

__global__ void k_gen_uniform(int count, int n, double *d, double *z, double *alpha) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long rows = (long long)count * (n - 1);
    if (t < rows) {
        const int r = (int)(t % (n - 1));
        d[t] = 10.0 - 20.0 * (r + 0.25 + 0.5 * hash01(2 * t)) / (n - 1);
        z[t] = 1.0 - 0.95 * hash01(2 * t + 1);
    }
    if (t < count) alpha[t] = 2.0 * hash01(~t) - 1.0;
}

static cudaError_t time_team(int n, int W, float *ms, cudaStream_t st) {
    const int count = (int)std::max(2LL, std::min(4096LL, (1LL << 19) / n));
    std::vector<long long> n_off(count + 1);
    for (int i = 0; i <= count; ++i) n_off[i] = (long long)i * n;
    double *buf = nullptr;
    const size_t rows = (size_t)count * (n - 1);
    cudaError_t e = cudaMalloc(&buf, sizeof(double) * (2 * rows + count + (size_t)count * n));
    if (e) return e;
    double *d = buf, *z = buf + rows, *al = z + rows, *lam = al + count;
    k_gen_uniform<<<(unsigned)((rows + 255) / 256) + 1, 256, 0, st>>>(count, n, d, z, al);
    Plan *P = new Plan();
    RunOpts ro{};
    resolve_opts(nullptr, ro);
    ro.precision = AE_FP32_BRACKET;
    e = build_plan(P, count, n_off.data(), nullptr, d, z, al, lam, nullptr, nullptr, ro, W, st);
    cudaEvent_t a = nullptr, b = nullptr;
    if (!e) e = cudaEventCreate(&a);
    if (!e) e = cudaEventCreate(&b);
    if (!e) {
        enqueue(*P, st);   // warm-up
        cudaEventRecord(a, st);
        for (int r = 0; r < 2; ++r) enqueue(*P, st);
        cudaEventRecord(b, st);
        e = cudaEventSynchronize(b);
        if (!e) e = cudaEventElapsedTime(ms, a, b);
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    free_plan(P);
    cudaFree(buf);
    return e;
}

}  // namespace ae

struct ae_batch {
    ae::Plan *p;
};

namespace {
int batch_args(int count, const long long *n_off, const double *d_all, const double *z_all,
               const double *alpha_all, const double *lambda_all) {
    if (count < 1) return -2;
    if (!n_off || n_off[0] != 0) return -3;
    for (int i = 0; i < count; ++i)
        if (n_off[i + 1] - n_off[i] < 1 || n_off[i + 1] - n_off[i] > (1 << 30)) return -3;
    if (n_off[count] > count && (!d_all || !z_all)) return -5;
    if (!alpha_all) return -7;
    if (!lambda_all) return -8;
    return 0;
}

int resolve(const ae_opts *o, ae::RunOpts &ro) { return ae::resolve_opts(o, ro); }

int fail(cudaError_t e) {
    ae::record_cuda_error(e);
    return AE_ERR_CUDA;
}
}  // namespace

extern "C" {

int ae_batch_create(ae_batch **plan, int count, const long long *n_off, const long long *v_off,
                    const double *d_all, const double *z_all, const double *alpha_all,
                    double *lambda_all, double *V_all, int *status_all, const ae_opts *opts,
                    void *stream) {
    if (!plan) return -1;
    *plan = nullptr;
    const int a = batch_args(count, n_off, d_all, z_all, alpha_all, lambda_all);
    if (a) return a;
    ae::RunOpts ro;
    if (resolve(opts, ro)) return -11;
    ae::Plan *P = new ae::Plan();
    cudaError_t e = ae::build_plan(P, count, n_off, v_off, d_all, z_all, alpha_all, lambda_all,
                                   V_all, status_all, ro, 0, (cudaStream_t)stream);
    if (!e) e = ae::capture_plan(P);
    if (e) {
        ae::free_plan(P);
        return fail(e);
    }
    *plan = new ae_batch{P};
    return AE_OK;
}

int ae_batch_run(ae_batch *plan, void *stream) {
    if (!plan || !plan->p) return -1;
    cudaError_t e = cudaGraphLaunch(plan->p->exec, (cudaStream_t)stream);
    return e ? fail(e) : AE_OK;
}

int ae_batch_info(ae_batch *plan, ae_info *info, void *stream) {
    if (!plan || !plan->p) return -1;
    if (!info) return -2;
    cudaError_t e = ae::plan_info(*plan->p, info, (cudaStream_t)stream);
    if (e) return fail(e);
    return AE_OK;
}

void ae_batch_destroy(ae_batch *plan) {
    if (!plan) return;
    cudaDeviceSynchronize();
    ae::free_plan(plan->p);
    delete plan;
}

int arrow_eig_batched(int count, const long long *n_off, const long long *v_off,
                      const double *d_all, const double *z_all, const double *alpha_all,
                      double *lambda_all, double *V_all, int *status_all, const ae_opts *opts,
                      ae_info *info, void *stream) {
    const int a = batch_args(count, n_off, d_all, z_all, alpha_all, lambda_all);
    if (a) return a;
    ae::RunOpts ro;
    if (resolve(opts, ro)) return -10;
    cudaStream_t st = (cudaStream_t)stream;
    ae::Plan *P = new ae::Plan();
    cudaError_t e = ae::build_plan(P, count, n_off, v_off, d_all, z_all, alpha_all, lambda_all,
                                   V_all, status_all, ro, 0, st);
    if (!e) {
        ae::enqueue(*P, st);
        e = cudaGetLastError();
    }
    int status = AE_OK;
    if (!e && info) {
        e = ae::plan_info(*P, info, st);
        if (!e && info->n_capped) status = AE_ERR_NOCONV;
    }
    if (!e) e = cudaStreamSynchronize(st);   // the plan's buffers are freed below
    ae::free_plan(P);
    return e ? fail(e) : status;
}

int ae_autotune(int n_max, void *stream) {
    if (n_max < 2) return -1;
    cudaStream_t st = (cudaStream_t)stream;
    std::map<int, int> found;
    for (int b = 32; b <= 256 && b <= std::max(32, n_max); b <<= 1) {
        int best = 32;
        float best_ms = 0.f;
        for (int W : {8, 16, 32}) {
            float ms = 0.f;
            cudaError_t e = ae::time_team(b, W, &ms, st);
            if (e) return fail(e);
            if (W == 8 || ms < best_ms) {
                best = W;
                best_ms = ms;
            }
        }
        found[b] = best;
    }
    for (int b = 512; b <= n_max && b <= (1 << 24); b <<= 1) found[b] = 32;
    std::lock_guard<std::mutex> lk(ae::g_tune_mu);
    ae::load_cache_locked();
    for (auto &kv : found) ae::g_tune[kv.first] = kv.second;
    ae::save_cache_locked();
    return AE_OK;
}

int ae_team_width(int n) { return n < 1 ? -1 : ae::team_for(n); }

}  // extern "C"
