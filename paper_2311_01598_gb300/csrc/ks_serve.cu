// ks_serve.cu -- key-switch serving engine with continuous batching.
//
// Requests (params, key, level, device buffers) are queued by ks_server_submit
// from any thread.  One scheduler thread:
//   * admits queued requests in arrival order while a slot is free and the
//     request's scratch fits in the HBM budget (a pool carved out of one
//     allocation made at creation, first-fit with coalescing);
//   * groups the admitted requests that share a parameter set (up to
//     max_batch) and launches them as one Output-Centric batch on the next
//     stream lane, so batches on different lanes overlap on the device;
//   * retires finished batches (CUDA event query), releasing slots and
//     scratch, and records completion times.
// Requests that arrive while batches run join the next batch as soon as
// slots and memory free up (continuous batching).  Keys stay resident: the
// server only refers to keys the caller created.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ks_internal.h"
#include "ks_launch.h"

namespace ks {

using Clock = std::chrono::steady_clock;

struct Req {
    const ks_params *P;
    const ks_key *K;
    uint32_t nact;
    const u64 *d;
    u64 *o0, *o1;
    double t_arrive = 0, t_admit = 0, t_done = 0;
    size_t off = 0, bytes = 0;
    int state = 0;  // 0 queued, 1 on the device, 2 done
    int status = KS_OK;
};

struct Batch {
    std::vector<uint64_t> tickets;
    cudaEvent_t ev = nullptr;
    size_t lane = 0;
};

// Batches queued on one lane at most: a further batch would only wait behind
// them, so requests stay in the server's queue and join a larger batch once
// a lane frees up (at low load every lane is idle and requests launch at
// once).
constexpr int kLaneDepth = 2;

// First-fit allocator over [0, size) with coalescing free list.
class Pool {
  public:
    void init(size_t size) { free_[0] = size; }
    bool alloc(size_t bytes, size_t *off)
    {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }

  private:
    std::map<size_t, size_t> free_;
};

}  // namespace ks

struct ks_server {
    ks_server_config cfg{};
    int device = 0;
    unsigned char *pool_mem = nullptr;
    ks::Pool pool;
    std::vector<cudaStream_t> lanes;
    std::vector<int> lane_batches;  // batches in flight per lane
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, ks::Req> reqs;
    uint64_t next_ticket = 1;
    std::vector<ks::Batch> inflight;
    uint32_t inflight_jobs = 0;
    std::thread worker;
    bool stop = false;
    ks::Clock::time_point t0;
    // statistics
    uint64_t n_done = 0, n_batches = 0, max_batch_seen = 0;
};

namespace ks {

static double now_s(const ks_server *S) { return std::chrono::duration<double>(Clock::now() - S->t0).count(); }

static size_t req_bytes(const Req &r) { return oc_scratch_words(r.P->tables, (int)r.nact) * sizeof(u64); }

// Scheduler: runs until stop is set and all work is finished.
static void scheduler(ks_server *S)
{
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        bool progress = false;
        // 1. retire finished batches
        for (size_t b = 0; b < S->inflight.size();) {
            cudaError_t q = cudaEventQuery(S->inflight[b].ev);
            if (q == cudaErrorNotReady) {
                ++b;
                continue;
            }
            const double t = now_s(S);
            for (uint64_t tk : S->inflight[b].tickets) {
                Req &r = S->reqs[tk];
                r.t_done = t;
                r.state = 2;
                if (q != cudaSuccess) r.status = KS_ECUDA;
                S->pool.release(r.off, r.bytes);
                S->inflight_jobs -= 1;
                S->n_done += 1;
            }
            if (q != cudaSuccess) cudaGetLastError();
            cudaEventDestroy(S->inflight[b].ev);
            S->lane_batches[S->inflight[b].lane] -= 1;
            S->inflight.erase(S->inflight.begin() + (long)b);
            progress = true;
        }
        if (progress) S->cv_done.notify_all();
        // 2. admit and launch batches, oldest request first
        while (!S->queue.empty() && S->inflight_jobs < S->cfg.max_inflight_jobs) {
            // the least loaded lane, if any lane has room for another batch
            size_t li = 0;
            for (size_t l = 1; l < S->lanes.size(); ++l)
                if (S->lane_batches[l] < S->lane_batches[li]) li = l;
            if (S->lane_batches[li] >= kLaneDepth) break;
            const ks_params *P0 = S->reqs[S->queue.front()].P;
            std::vector<uint64_t> take;
            for (auto it = S->queue.begin(); it != S->queue.end();) {
                Req &r = S->reqs[*it];
                if (take.size() >= S->cfg.max_batch || S->inflight_jobs + take.size() >= S->cfg.max_inflight_jobs)
                    break;
                if (r.P != P0) {
                    ++it;
                    continue;
                }
                r.bytes = (req_bytes(r) + 255) & ~(size_t)255;
                if (!S->pool.alloc(r.bytes, &r.off)) break;  // HBM budget full: wait for completions
                take.push_back(*it);
                it = S->queue.erase(it);
            }
            if (take.empty()) break;
            std::vector<OcJob> jobs(take.size());
            const double t = now_s(S);
            for (size_t i = 0; i < take.size(); ++i) {
                Req &r = S->reqs[take[i]];
                r.state = 1;
                r.t_admit = t;
                const int nact = (int)r.nact;
                const int nd = (nact + P0->alpha - 1) / P0->alpha;
                OcJob &J = jobs[i];
                J.d = r.d;
                J.out0 = r.o0;
                J.out1 = r.o1;
                J.key = key_view(r.K);
                J.y = (u64 *)(S->pool_mem + r.off);
                J.tmp = J.y + (size_t)nact * P0->N;
                J.cp = J.tmp + ((size_t)nd * (nact + P0->kp) + 2 * (size_t)nact) * P0->N;
                J.pre = P0->d_up_pre_lvl + (size_t)(nact - 1) * P0->nq;
                J.nact = nact;
                J.nd = nd;
            }
            S->inflight_jobs += (uint32_t)take.size();
            cudaStream_t lane = S->lanes[li];
            lk.unlock();
            int rc = launch_oc(P0->tables, (int)jobs.size(), jobs.data(), P0->sched.oc_variant, lane);
            Batch bt;
            bt.tickets = take;
            bt.lane = li;
            if (cudaEventCreateWithFlags(&bt.ev, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventRecord(bt.ev, lane) != cudaSuccess) {
                cudaGetLastError();
                rc = KS_ECUDA;
            }
            lk.lock();
            if (rc != KS_OK) {  // fail the requests once nothing of theirs can still run
                cudaStreamSynchronize(lane);
                cudaGetLastError();
                if (bt.ev) cudaEventDestroy(bt.ev);
                for (uint64_t tk : take) {
                    Req &r = S->reqs[tk];
                    r.state = 2;
                    r.status = rc;
                    r.t_done = now_s(S);
                    S->pool.release(r.off, r.bytes);
                    S->inflight_jobs -= 1;
                }
                S->cv_done.notify_all();
                continue;
            }
            S->n_batches += 1;
            S->max_batch_seen = std::max<uint64_t>(S->max_batch_seen, take.size());
            S->lane_batches[li] += 1;
            S->inflight.push_back(bt);
            progress = true;
        }
        if (S->stop && S->queue.empty() && S->inflight.empty()) break;
        if (!progress) {
            if (S->inflight.empty())
                S->cv_work.wait_for(lk, std::chrono::milliseconds(2));
            else
                S->cv_work.wait_for(lk, std::chrono::microseconds(20));
        }
    }
}

}  // namespace ks

using namespace ks;

extern "C" {

int ks_server_create(const ks_server_config *cfg, ks_server **out)
{
    if (!cfg || !out) return fail(KS_EINVAL, "NULL argument");
    *out = nullptr;
    if (cfg->max_inflight_jobs < 1 || cfg->max_batch < 1 || cfg->max_batch > (uint32_t)kMaxBatch ||
        cfg->n_streams < 1 || cfg->n_streams > 16 || cfg->hbm_budget_bytes < (1u << 20))
        return fail(KS_EINVAL, "server config: slots >= 1, batch 1..64, streams 1..16, budget >= 1 MiB");
    ks_server *S = new ks_server();
    S->cfg = *cfg;
    if (cudaGetDevice(&S->device) != cudaSuccess ||
        cudaMalloc((void **)&S->pool_mem, cfg->hbm_budget_bytes) != cudaSuccess) {
        cudaGetLastError();
        delete S;
        return fail(KS_ENOMEM, "server scratch pool allocation failed");
    }
    S->pool.init(cfg->hbm_budget_bytes);
    for (uint32_t i = 0; i < cfg->n_streams; ++i) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            for (cudaStream_t s : S->lanes) cudaStreamDestroy(s);
            cudaFree(S->pool_mem);
            delete S;
            return fail(KS_ECUDA, "server stream creation failed");
        }
        S->lanes.push_back(st);
    }
    S->lane_batches.assign(S->lanes.size(), 0);
    S->t0 = Clock::now();
    S->worker = std::thread(scheduler, S);
    *out = S;
    return KS_OK;
}

void ks_server_destroy(ks_server *S)
{
    if (!S) return;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    S->worker.join();
    cudaSetDevice(S->device);
    for (cudaStream_t s : S->lanes) cudaStreamDestroy(s);
    cudaFree(S->pool_mem);
    delete S;
}

int ks_server_submit(ks_server *S, const ks_request *req, uint64_t *ticket)
{
    if (!S || !req || !ticket) return fail(KS_EINVAL, "NULL argument");
    const ks_params *P = req->params;
    if (!P || !req->key || req->key->params != P) return fail(KS_EINVAL, "request key/params mismatch");
    if (req->key->shard) return fail(KS_EINVAL, "request key is a tower shard");
    if (req->level_towers < 1 || req->level_towers > (uint32_t)P->nq) return fail(KS_EINVAL, "bad level");
    if (!req->d_in || !req->d_out0 || !req->d_out1) return fail(KS_EINVAL, "NULL data pointer");
    // the combine kernels move two words at a time
    if (((uintptr_t)req->d_in | (uintptr_t)req->d_out0 | (uintptr_t)req->d_out1) & 15)
        return fail(KS_EINVAL, "d_in, d_out0 and d_out1 must be 16-byte aligned");
    {
        const size_t len = (size_t)req->level_towers * P->N * sizeof(u64);
        auto overlap = [len](const void *a, const void *b) {
            const char *x = (const char *)a, *y = (const char *)b;
            return x < y + len && y < x + len;
        };
        if (overlap(req->d_in, req->d_out0) || overlap(req->d_in, req->d_out1) || overlap(req->d_out0, req->d_out1))
            return fail(KS_EINVAL, "d_in, d_out0, d_out1 overlap");
    }
    if (P->device != S->device) return fail(KS_EINVAL, "params on another device");
    Req r;
    r.P = P;
    r.K = req->key;
    r.nact = req->level_towers;
    r.d = req->d_in;
    r.o0 = req->d_out0;
    r.o1 = req->d_out1;
    const size_t bytes = (oc_scratch_words(P->tables, (int)r.nact) * sizeof(u64) + 255) & ~(size_t)255;
    if (bytes > S->cfg.hbm_budget_bytes) return fail(KS_EINVAL, "request needs more scratch than the whole budget");
    {
        std::lock_guard<std::mutex> g(S->mu);
        if (S->stop) return fail(KS_EINVAL, "server is stopping");
        r.t_arrive = now_s(S);
        *ticket = S->next_ticket++;
        S->reqs.emplace(*ticket, r);
        S->queue.push_back(*ticket);
    }
    S->cv_work.notify_one();
    return KS_OK;
}

int ks_server_wait(ks_server *S, uint64_t ticket, uint32_t timeout_ms)
{
    if (!S) return fail(KS_EINVAL, "NULL server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(KS_EINVAL, "unknown ticket");
    const bool ok = S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                        [&] { return S->reqs[ticket].state == 2; });
    if (!ok) return fail(KS_ETIMEOUT, "request not finished before the timeout");
    return S->reqs[ticket].status;
}

int ks_server_times(ks_server *S, uint64_t ticket, double *t_arrive, double *t_admit, double *t_done)
{
    if (!S) return fail(KS_EINVAL, "NULL server");
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(KS_EINVAL, "unknown ticket");
    if (t_arrive) *t_arrive = it->second.t_arrive;
    if (t_admit) *t_admit = it->second.t_admit;
    if (t_done) *t_done = it->second.t_done;
    return it->second.state == 2 ? KS_OK : fail(KS_ETIMEOUT, "request not finished");
}

int ks_server_stats(ks_server *S, uint64_t *n_done, uint64_t *n_batches, uint64_t *max_batch)
{
    if (!S) return fail(KS_EINVAL, "NULL server");
    std::lock_guard<std::mutex> g(S->mu);
    if (n_done) *n_done = S->n_done;
    if (n_batches) *n_batches = S->n_batches;
    if (max_batch) *max_batch = S->max_batch_seen;
    return KS_OK;
}

int ks_server_run_trace(ks_server *S, uint32_t n, const ks_request *reqs, const double *arrival_s,
                        double *latency_s, uint32_t timeout_ms)
{
    if (!S || (n > 0 && (!reqs || !arrival_s))) return fail(KS_EINVAL, "NULL argument");
    std::vector<uint64_t> tk(n);
    const Clock::time_point start = Clock::now();
    for (uint32_t i = 0; i < n; ++i) {
        const auto due = start + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(arrival_s[i]));
        while (Clock::now() < due) {  // precise arrival: sleep coarsely, then spin
            const auto left = due - Clock::now();
            if (left > std::chrono::microseconds(200)) std::this_thread::sleep_for(left - std::chrono::microseconds(150));
        }
        int rc = ks_server_submit(S, &reqs[i], &tk[i]);
        if (rc) return rc;
    }
    int status = KS_OK;
    for (uint32_t i = 0; i < n; ++i) {
        int rc = ks_server_wait(S, tk[i], timeout_ms);
        if (rc && status == KS_OK) status = rc;
        double a = 0, d = 0;
        ks_server_times(S, tk[i], &a, nullptr, &d);
        if (latency_s) latency_s[i] = d - a;
    }
    return status;
}

}  // extern "C"
