// ae_serve.cu -- a request loop over the solver: continuous batching of
// arrowhead / DPR1 / triangular-arrowhead-SVD solves of any size.
//
// A worker thread owns `max_inflight` CUDA streams ("slots").  Each tick it
//   1. retires finished requests (their completion event has fired): records
//      the latency (submit -> observed completion), reads the request's
//      counters, frees its scratch, and frees the slot;
//   2. admits queued requests in FIFO order while a slot is free and the
//      device-memory budget covers the request's scratch and results
//      (results stay on the device, owned by the server, until released).
// An admitted request runs the same pipeline as arrow_eig / dpr1_eig /
// tri_arrow_svd on its slot's stream, so requests admitted while others run
// overlap on the GPU.  Small arrowhead requests waiting among the first
// kScan of the queue (order at most kSmallN, up to kMergeMax of them, in
// their queue order, ahead of the larger requests between them) are admitted
// as one: a single pass of the batched stages on one slot solves them all,
// one 32-lane team per eigenpair, so that their results carry the
// single-instance solve's bits (remedied eigenpairs agree within the
// tolerance), while each keeps its own result buffers and completion.
// Nothing on the device waits for the host.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "ae_internal.h"

namespace {

using clk = std::chrono::steady_clock;

struct Req {
    unsigned long long id = 0;
    ae_request in{};
    int state = AE_REQ_QUEUED;
    int status = AE_OK;
    size_t bytes = 0;           // scratch + results charged to the budget
    bool charged = false;       // bytes are counted in in_use
    void *scratch = nullptr;
    void *wbuf = nullptr;       // stored (delta_j, c_j) pairs of the eigenvalue kernel
    double *result = nullptr;   // lambda | V | U in one block
    double *lam = nullptr, *V = nullptr, *U = nullptr;
    int slot = -1;
    cudaEvent_t done = nullptr;
    int *cnt_host = nullptr;    // pinned copy of the solve's counters
    clk::time_point t_submit, t_done;
};

size_t wbuf_bytes(int n) {
    return sizeof(double2) * (size_t)((n + 1) & ~1) * (size_t)ae::eig_grid_warps(n);
}

constexpr int kSmallN = 1024;     // orders merged into one batched pass
constexpr int kMergeMax = 256;    // requests per merged pass
constexpr int kScan = 1024;       // queue entries searched for them

bool mergeable(const ae_request &r) {
    return r.kind == AE_KIND_ARROW && r.n >= 2 && r.n <= kSmallN;
}

size_t result_doubles(const ae_request &r) {
    const size_t n = (size_t)r.n;
    size_t k = n;                                          // eigen/singular values
    if (r.want_vectors) k += n * n * (r.kind == AE_KIND_SVD ? 2 : 1);
    return k;
}

}  // namespace

struct ae_server {
    int dev = 0;
    size_t budget = 0, in_use = 0;
    int max_inflight = 0, queue_cap = 0;
    ae::RunOpts ro{};
    std::vector<cudaStream_t> streams;
    std::vector<int> slot_busy;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Req *> queue;
    std::map<unsigned long long, Req *> reqs;
    std::vector<Req *> inflight;
    unsigned long long next_id = 1;
    std::atomic<bool> stop{false};
    std::thread worker;
    // statistics
    long long submitted = 0, admitted = 0, completed = 0, rejected = 0, failed = 0;
    long long eigenpairs = 0;
    std::vector<double> lat;
    bool started = false;
    clk::time_point t_first, t_last;
    int worker_error = cudaSuccess;

    long long merged = 0;             // requests solved in merged batched passes

    void loop();
    bool admit_locked(Req *r);
    int admit_merged_locked();
    void retire_locked(Req *r);
};

// Admit the small arrowhead requests among the first kScan of the queue (all
// with the want_vectors of the first of them) as one batched pass on one free
// slot; returns how many were admitted (0: fewer than two waiting, or no slot
// or memory now).
int ae_server::admit_merged_locked() {
    std::vector<int> at;              // their queue positions, in order
    int want = -1;
    for (int q = 0; q < (int)queue.size() && q < kScan && (int)at.size() < kMergeMax; ++q) {
        const ae_request &r = queue[q]->in;
        if (!mergeable(r) || (want >= 0 && r.want_vectors != want)) continue;
        want = r.want_vectors;
        at.push_back(q);
    }
    const int cnt = (int)at.size();
    if (cnt < 2) return 0;
    int slot = -1;
    for (int s = 0; s < max_inflight; ++s)
        if (!slot_busy[s]) { slot = s; break; }
    if (slot < 0) return 0;
    std::vector<int> ns(cnt);
    std::vector<Req *> rs(cnt);
    size_t res_bytes = 0;
    for (int i = 0; i < cnt; ++i) {
        rs[i] = queue[at[i]];
        ns[i] = rs[i]->in.n;
        res_bytes += sizeof(double) * result_doubles(rs[i]->in);
    }
    const size_t block_bytes = ae::req_batch_bytes(cnt, ns.data());
    if (in_use + res_bytes + block_bytes > budget && !(inflight.empty() && in_use == 0))
        return 0;
    cudaStream_t st = streams[slot];
    void *block = nullptr;
    cudaError_t e = cudaMallocAsync(&block, block_bytes, st);
    int got = 0;
    for (; !e && got < cnt; ++got)
        e = cudaMallocAsync((void **)&rs[got]->result,
                            sizeof(double) * result_doubles(rs[got]->in), st);
    if (e) {                        // out of device memory now: retry later
        for (int i = 0; i < got; ++i) {
            cudaFreeAsync(rs[i]->result, st);
            rs[i]->result = nullptr;
        }
        if (block) cudaFreeAsync(block, st);
        cudaGetLastError();
        return 0;
    }
    std::vector<const double *> d(cnt), z(cnt);
    std::vector<double> alpha(cnt);
    std::vector<double *> lam(cnt), V(cnt);
    std::vector<const int *> cntp(cnt);
    for (int i = 0; i < cnt; ++i) {
        Req *r = rs[i];
        const size_t n = (size_t)r->in.n;
        r->lam = r->result;
        r->V = r->in.want_vectors ? r->result + n : nullptr;
        r->U = nullptr;
        d[i] = r->in.d;
        z[i] = r->in.z;
        alpha[i] = r->in.alpha;
        lam[i] = r->lam;
        V[i] = r->V;
    }
    // (the run shares want_vectors, so a pass writes columns for all or none)
    e = ae::launch_req_batch(cnt, ns.data(), d.data(), z.data(), alpha.data(), lam.data(),
                             V.data(), block, ro, st, cntp.data());
    for (int i = 0; i < cnt && !e; ++i)
        e = cudaMemcpyAsync(rs[i]->cnt_host, cntp[i], sizeof(int) * ae::C_COUNT,
                            cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaFreeAsync(block, st);
    for (int i = 0; i < cnt && !e; ++i) e = cudaEventRecord(rs[i]->done, st);
    const size_t share = block_bytes / cnt;
    for (int i = cnt - 1; i >= 0; --i) queue.erase(queue.begin() + at[i]);
    for (int i = 0; i < cnt; ++i) {
        Req *r = rs[i];
        if (e) {
            r->state = AE_REQ_ERROR;
            r->status = AE_ERR_CUDA;
            continue;
        }
        r->slot = slot;
        r->state = AE_REQ_RUNNING;
        r->bytes = sizeof(double) * result_doubles(r->in) + share;
        in_use += r->bytes;
        r->charged = true;
        inflight.push_back(r);
        ++admitted;
        ++merged;
    }
    if (e) {
        worker_error = e;
        return cnt;
    }
    slot_busy[slot] = cnt;          // freed as its requests retire
    return cnt;
}

bool ae_server::admit_locked(Req *r) {
    int slot = -1;
    for (int s = 0; s < max_inflight; ++s)
        if (!slot_busy[s]) { slot = s; break; }
    if (slot < 0) return false;
    if (in_use + r->bytes > budget && !(inflight.empty() && in_use == 0)) return false;
    cudaStream_t st = streams[slot];
    const ae_request &q = r->in;
    const ae::Kind kind = q.kind == AE_KIND_DPR1 ? ae::KIND_DPR1
                        : q.kind == AE_KIND_SVD ? ae::KIND_TSVD : ae::KIND_ARROW;
    const long long wstride = ((long long)q.n + 1) & ~1LL;
    cudaError_t e = cudaMallocAsync(&r->scratch, ae::arrow_scratch_bytes(q.n), st);
    if (!e) e = cudaMallocAsync(&r->wbuf, wbuf_bytes(q.n), st);
    if (!e) e = cudaMallocAsync((void **)&r->result, sizeof(double) * result_doubles(q), st);
    if (e) {                       // out of device memory now: retry later
        if (r->scratch) cudaFreeAsync(r->scratch, st);
        if (r->wbuf) cudaFreeAsync(r->wbuf, st);
        r->scratch = nullptr;
        r->wbuf = nullptr;
        r->result = nullptr;
        cudaGetLastError();
        return false;
    }
    const size_t n = (size_t)q.n;
    r->lam = r->result;
    r->V = q.want_vectors ? r->result + n : nullptr;
    r->U = (q.want_vectors && q.kind == AE_KIND_SVD) ? r->result + n + n * n : nullptr;
    ae::Scratch S = ae::carve_scratch(r->scratch, q.n);
    S.wbuf = (double2 *)r->wbuf;
    S.wstride = wstride;
    ae::Outputs out{};
    out.lambda = r->lam;
    out.V = r->V;
    out.ldv = q.n;
    out.U = r->U;
    out.ldu = q.n;
    e = ae::launch_solve(kind, q.n, q.d, q.z, q.kind == AE_KIND_DPR1 ? 0.0 : q.alpha,
                         q.kind == AE_KIND_DPR1 ? q.alpha : 0.0, out, ro, S, st);
    if (!e) e = cudaMemcpyAsync(r->cnt_host, S.cnt, sizeof(int) * ae::C_COUNT,
                                cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaFreeAsync(r->scratch, st);
    if (!e) e = cudaFreeAsync(r->wbuf, st);
    if (!e) e = cudaEventRecord(r->done, st);
    r->scratch = nullptr;
    r->wbuf = nullptr;
    if (e) {
        r->state = AE_REQ_ERROR;
        r->status = AE_ERR_CUDA;
        worker_error = e;
        return true;
    }
    slot_busy[slot] = 1;
    r->slot = slot;
    r->state = AE_REQ_RUNNING;
    in_use += r->bytes;
    r->charged = true;
    inflight.push_back(r);
    ++admitted;
    return true;
}

void ae_server::retire_locked(Req *r) {
    r->t_done = clk::now();
    if (slot_busy[r->slot] > 0) --slot_busy[r->slot];
    const int *c = r->cnt_host;
    if (c[ae::C_FLAGS] & ae::CF_BAD) r->status = AE_ERR_INPUT;
    else if (c[ae::C_CAPPED]) r->status = AE_ERR_NOCONV;
    r->state = r->status == AE_OK ? AE_REQ_DONE : AE_REQ_ERROR;
    const double l = std::chrono::duration<double>(r->t_done - r->t_submit).count();
    lat.push_back(l);
    ++completed;
    if (r->status != AE_OK) ++failed;
    eigenpairs += r->in.n;
    t_last = r->t_done;
}

void ae_server::loop() {
    cudaSetDevice(dev);
    std::unique_lock<std::mutex> lk(mu);
    while (!stop.load()) {
        // 1. retire
        for (size_t i = 0; i < inflight.size();) {
            Req *r = inflight[i];
            const cudaError_t q = cudaEventQuery(r->done);
            if (q == cudaSuccess) {
                retire_locked(r);
                inflight[i] = inflight.back();
                inflight.pop_back();
            } else {
                if (q != cudaErrorNotReady) worker_error = q;
                ++i;
            }
        }
        // 2. admit in FIFO order (a run of small arrowheads at the head as one)
        while (!queue.empty()) {
            if (admit_merged_locked() > 0) continue;
            if (!admit_locked(queue.front())) break;
            queue.pop_front();
        }
        if (inflight.empty() && queue.empty()) {
            cv.wait_for(lk, std::chrono::milliseconds(5));
        } else {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        }
    }
}

extern "C" {

int ae_serve_create(ae_server **srv, size_t hbm_budget_bytes, int max_inflight, int queue_cap,
                    const ae_opts *opts) {
    if (!srv) return -1;
    *srv = nullptr;
    if (max_inflight < 1 || max_inflight > 256) return -3;
    if (queue_cap < 1) return -4;
    ae::RunOpts ro;
    if (ae::resolve_opts(opts, ro)) return -5;
    ae_server *s = new ae_server();
    cudaGetDevice(&s->dev);
    s->budget = hbm_budget_bytes;
    s->max_inflight = max_inflight;
    s->queue_cap = queue_cap;
    s->ro = ro;
    s->streams.resize(max_inflight);
    s->slot_busy.assign(max_inflight, 0);
    for (auto &st : s->streams) {
        cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e) {
            ae::record_cuda_error(e);
            delete s;
            return AE_ERR_CUDA;
        }
    }
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, s->dev) == cudaSuccess) {
        unsigned long long thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    s->worker = std::thread([s] { s->loop(); });
    *srv = s;
    return AE_OK;
}

int ae_serve_submit(ae_server *s, const ae_request *req, unsigned long long *ticket) {
    if (!s) return -1;
    if (!req) return -2;
    if (!ticket) return -3;
    const ae_request &q = *req;
    if (q.kind != AE_KIND_ARROW && q.kind != AE_KIND_DPR1 && q.kind != AE_KIND_SVD) return -2;
    if (q.n < 1) return -2;
    const int rows = q.kind == AE_KIND_DPR1 ? q.n : q.n - 1;
    if (rows > 0 && (!q.d || !q.z)) return -2;
    if (!isfinite(q.alpha) || (q.kind == AE_KIND_SVD && q.alpha == 0.0)) return -2;
    Req *r = new Req();
    r->in = q;
    r->bytes = ae::arrow_scratch_bytes(q.n) + wbuf_bytes(q.n) + sizeof(double) * result_doubles(q);
    if (cudaEventCreateWithFlags(&r->done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost((void **)&r->cnt_host, sizeof(int) * ae::C_COUNT) != cudaSuccess) {
        if (r->done) cudaEventDestroy(r->done);
        delete r;
        return AE_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if ((int)s->queue.size() >= s->queue_cap) {
        ++s->rejected;
        cudaEventDestroy(r->done);
        cudaFreeHost(r->cnt_host);
        delete r;
        return AE_EAGAIN;
    }
    r->id = s->next_id++;
    r->t_submit = clk::now();
    if (!s->started) {
        s->started = true;
        s->t_first = r->t_submit;
    }
    s->reqs[r->id] = r;
    s->queue.push_back(r);
    ++s->submitted;
    *ticket = r->id;
    s->cv.notify_one();
    return AE_OK;
}

int ae_serve_poll(ae_server *s, unsigned long long ticket, int *state, double *latency_s) {
    if (!s) return -1;
    if (!state) return -3;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return -2;
    Req *r = it->second;
    *state = r->state;
    if (latency_s)
        *latency_s = (r->state == AE_REQ_DONE || r->state == AE_REQ_ERROR)
                         ? std::chrono::duration<double>(r->t_done - r->t_submit).count()
                         : -1.0;
    return r->state == AE_REQ_ERROR ? r->status : AE_OK;
}

int ae_serve_result(ae_server *s, unsigned long long ticket, const double **lambda,
                    const double **V, const double **U) {
    if (!s) return -1;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return -2;
    Req *r = it->second;
    if (r->state != AE_REQ_DONE) return r->state == AE_REQ_ERROR ? r->status : AE_EAGAIN;
    if (lambda) *lambda = r->lam;
    if (V) *V = r->V;
    if (U) *U = r->U;
    return AE_OK;
}

int ae_serve_release(ae_server *s, unsigned long long ticket) {
    if (!s) return -1;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return -2;
    Req *r = it->second;
    if (r->state == AE_REQ_QUEUED || r->state == AE_REQ_RUNNING) return AE_EAGAIN;
    if (r->result) cudaFreeAsync(r->result, s->streams[r->slot >= 0 ? r->slot : 0]);
    if (r->charged) s->in_use -= r->bytes;
    cudaEventDestroy(r->done);
    cudaFreeHost(r->cnt_host);
    s->reqs.erase(it);
    delete r;
    s->cv.notify_one();
    return AE_OK;
}

int ae_serve_stats(ae_server *s, ae_serve_stats_t *st) {
    if (!s) return -1;
    if (!st) return -2;
    std::lock_guard<std::mutex> lk(s->mu);
    memset(st, 0, sizeof(*st));
    st->submitted = s->submitted;
    st->admitted = s->admitted;
    st->completed = s->completed;
    st->rejected = s->rejected;
    st->failed = s->failed;
    st->queued = (long long)s->queue.size();
    st->running = (long long)s->inflight.size();
    st->bytes_in_use = s->in_use;
    st->eigenpairs = s->eigenpairs;
    if (!s->lat.empty()) {
        std::vector<double> v = s->lat;
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) {
            const size_t k = (size_t)std::min<double>(v.size() - 1, floor(p * (v.size() - 1) + 0.5));
            return v[k];
        };
        st->p50_s = pct(0.50);
        st->p99_s = pct(0.99);
        st->max_s = v.back();
        const double span = std::chrono::duration<double>(s->t_last - s->t_first).count();
        st->eigenpairs_per_s = span > 0 ? s->eigenpairs / span : 0.0;
    }
    st->cuda_error = s->worker_error;
    st->merged = s->merged;
    return AE_OK;
}

int ae_serve_destroy(ae_server *s) {
    if (!s) return -1;
    s->stop.store(true);
    s->cv.notify_one();
    if (s->worker.joinable()) s->worker.join();
    for (auto st : s->streams) cudaStreamSynchronize(st);
    for (auto &kv : s->reqs) {
        Req *r = kv.second;
        if (r->result) cudaFree(r->result);
        if (r->done) cudaEventDestroy(r->done);
        if (r->cnt_host) cudaFreeHost(r->cnt_host);
        delete r;
    }
    for (auto st : s->streams) cudaStreamDestroy(st);
    delete s;
    return AE_OK;
}

}  // extern "C"
