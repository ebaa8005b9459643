// server.cu -- the request loop: continuous batching over a resident store.
//
// Requests (epsilon-join or top-k query sets) arrive one at a time through
// dl_submit. A scheduler thread keeps up to `slots` batches in flight, each on
// its own CUDA stream and worker thread: whenever a slot is free it takes
// queued requests in arrival order, as many as fit the row limit and the
// memory budget (admission by memory: the budget given at creation, and the
// device's free memory at that moment), and hands them to a worker that runs
// them as one dl_batch_join. Requests that arrive while batches are on the GPU
// wait only for the next free slot, and batches on different streams overlap
// on the device. A finished batch is split into one result per request; dl_poll
// returns it. Latency is measured from dl_submit to the result being ready.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <thread>
#include <vector>

#include "kernels.h"

namespace dl {

using Clock = std::chrono::steady_clock;

struct Req {
    uint64_t ticket;
    int32_t kind;
    int32_t k;
    double eps;
    int64_t nq;
    std::vector<int64_t> ids;
    std::vector<float> feats;
    int64_t est_bytes;
    Clock::time_point t_submit;
    int status = DL_EAGAIN;      // DL_EAGAIN while queued or running
    bool canceled = false;
    dl_result *result = nullptr;
    double latency_ms = 0.0;
};

struct Server {
    const dl_store *S = nullptr;
    int device = 0;
    int64_t budget = 0;
    int slots = 2;
    int64_t max_rows = 65536;
    dl_join_opts opts{};
    std::mutex mu;
    std::condition_variable cv_sched;   // scheduler: new request, or a slot freed
    std::condition_variable cv_done;    // pollers: a request finished
    std::deque<std::shared_ptr<Req>> queue;
    std::map<uint64_t, std::shared_ptr<Req>> all;
    uint64_t next_ticket = 1;
    int busy = 0;
    int64_t inflight_bytes = 0;
    bool stop = false;
    std::thread sched;
    std::vector<std::thread> workers;                     // one persistent worker per slot
    std::vector<cudaStream_t> streams;
    std::vector<bool> stream_busy;
    std::vector<std::vector<std::shared_ptr<Req>>> jobs;  // per slot: the batch handed over
    std::condition_variable cv_work;
    // statistics
    std::vector<double> lat_ms;
    int64_t done = 0, failed = 0, batches = 0, batched_requests = 0, admit_waits = 0;
};

// Device-memory estimate of one request inside a batch (queries, output, workspace).
static int64_t estimate_bytes(const dl_store *S, int32_t kind, int64_t nq, int32_t k)
{
    const int64_t d = S->d, dp = S->dp;
    int64_t b = nq * (d * 4 + dp * 2 + 64) * 2;           // uploaded + internal query store
    if (kind == DL_REQ_TOPK) {
        const int64_t cap = std::max<int64_t>(64, 4 * k);
        b += nq * k * 16 + nq * 16 * (k * 4 + cap * 8);    // output + heaps + candidate lists (<= 16 slots)
    } else {
        b += nq * 16 * 1024 + (1 << 20);                   // output / candidates, grown on demand
    }
    return b;
}

static void finish(Server *sv, const std::vector<std::shared_ptr<Req>> &reqs, dl_result *batch, int rc,
                   cudaStream_t st)
{
    std::vector<dl_result *> outs(reqs.size(), nullptr);
    if (rc == DL_OK) {
        // split the batch result into one result per request (device-to-device copies)
        for (size_t i = 0; i < reqs.size() && rc == DL_OK; ++i) {
            dl_result *r = new dl_result();
            r->device = sv->device;
            r->stream = st;
            r->stats = batch->stats;
            if (reqs[i]->kind == DL_REQ_EPS) {
                const int64_t o = batch->pair_off[i], n = batch->pair_off[i + 1] - o;
                r->kind = 0;
                r->count = n;
                r->cap = n;
                void *blk = nullptr;
                rc = dev_alloc(&blk, std::max<int64_t>(n, 1) * 16, st);
                if (!rc && n > 0) {
                    r->d_r = (int64_t *)blk;
                    r->d_s = r->d_r + n;
                    cudaMemcpyAsync(r->d_r, batch->d_r + o, n * 8, cudaMemcpyDeviceToDevice, st);
                    cudaMemcpyAsync(r->d_s, batch->d_s + o, n * 8, cudaMemcpyDeviceToDevice, st);
                } else if (!rc) {
                    r->d_r = (int64_t *)blk;
                    r->d_s = r->d_r;
                }
                r->stats.pairs_out = n;
            } else {
                const int64_t o = batch->topk_off[i], n = reqs[i]->nq * reqs[i]->k;
                r->kind = 1;
                r->k = reqs[i]->k;
                r->nq = reqs[i]->nq;
                void *blk = nullptr;
                rc = dev_alloc(&blk, std::max<int64_t>(n, 1) * 16, st);
                if (!rc) {
                    r->d_ids = (int64_t *)blk;
                    r->d_d2 = (double *)(r->d_ids + n);
                    if (n > 0) {
                        cudaMemcpyAsync(r->d_ids, batch->d_ids + o, n * 8, cudaMemcpyDeviceToDevice, st);
                        cudaMemcpyAsync(r->d_d2, batch->d_d2 + o, n * 8, cudaMemcpyDeviceToDevice, st);
                    }
                }
            }
            outs[i] = r;
        }
        if (rc == DL_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = DL_ECUDA;
    }
    dl_result_free(batch);
    const auto now = Clock::now();
    std::lock_guard<std::mutex> lk(sv->mu);
    for (size_t i = 0; i < reqs.size(); ++i) {
        auto &q = reqs[i];
        if (rc == DL_OK) {
            q->result = outs[i];
            q->status = DL_OK;
            q->latency_ms = std::chrono::duration<double, std::milli>(now - q->t_submit).count();
            sv->lat_ms.push_back(q->latency_ms);
            sv->done++;
        } else {
            if (outs[i]) dl_result_free(outs[i]);
            q->status = DL_EFAILED;
            sv->failed++;
        }
        sv->inflight_bytes -= q->est_bytes;
    }
}

static void run_batch(Server *sv, int slot, std::vector<std::shared_ptr<Req>> reqs)
{
    NvtxScope nvtx_scope("dl_server batch");
    cudaStream_t st = sv->streams[slot];
    int64_t total = 0;
    for (auto &q : reqs) total += q->nq;
    std::vector<int64_t> ids((size_t)total);
    std::vector<float> feats((size_t)total * sv->S->d);
    std::vector<dl_request> rq(reqs.size());
    int64_t off = 0;
    for (size_t i = 0; i < reqs.size(); ++i) {
        auto &q = reqs[i];
        std::memcpy(ids.data() + off, q->ids.data(), q->nq * 8);
        std::memcpy(feats.data() + off * sv->S->d, q->feats.data(), q->nq * sv->S->d * 4);
        rq[i].kind = q->kind;
        rq[i].k = q->k;
        rq[i].eps = q->eps;
        rq[i].q_begin = off;
        rq[i].nq = q->nq;
        off += q->nq;
    }
    dl_join_opts o = sv->opts;
    o.cuda_stream = st;
    dl_result *batch = nullptr;
    const int rc = dl_batch_join(sv->S, ids.data(), feats.data(), total, sv->S->d, DL_MEM_HOST, rq.data(),
                                 (int32_t)rq.size(), &o, &batch);
    finish(sv, reqs, batch, rc, st);
}

// Persistent worker of one slot: runs each batch the scheduler hands it.
static void worker(Server *sv, int slot)
{
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    while (true) {
        sv->cv_work.wait(lk, [&] { return sv->stop || !sv->jobs[slot].empty(); });
        if (sv->jobs[slot].empty() && sv->stop) break;
        std::vector<std::shared_ptr<Req>> reqs;
        reqs.swap(sv->jobs[slot]);
        lk.unlock();
        run_batch(sv, slot, std::move(reqs));
        lk.lock();
        sv->stream_busy[slot] = false;
        sv->busy--;
        sv->cv_sched.notify_all();
        sv->cv_done.notify_all();
    }
}

static void scheduler(Server *sv)
{
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    while (true) {
        sv->cv_sched.wait(lk, [&] { return sv->stop || (!sv->queue.empty() && sv->busy < sv->slots); });
        if (sv->stop) break;
        // admission: rows, budget and the device's free memory
        size_t free_b = 0, total_b = 0;
        lk.unlock();
        cudaMemGetInfo(&free_b, &total_b);
        lk.lock();
        const int64_t room = std::min<int64_t>(sv->budget - sv->inflight_bytes, (int64_t)free_b - (int64_t)(256 << 20));
        std::vector<std::shared_ptr<Req>> take;
        int64_t rows = 0, bytes = 0;
        while (!sv->queue.empty()) {
            auto &q = sv->queue.front();
            if (q->canceled) {
                sv->queue.pop_front();
                continue;
            }
            if (!take.empty() && (rows + q->nq > sv->max_rows || bytes + q->est_bytes > room)) break;
            if (take.empty() && q->est_bytes > room && sv->busy > 0) break;   // wait for memory to free up
            take.push_back(q);
            rows += q->nq;
            bytes += q->est_bytes;
            sv->queue.pop_front();
        }
        if (take.empty()) {
            sv->admit_waits++;
            sv->cv_sched.wait_for(lk, std::chrono::milliseconds(1));
            continue;
        }
        int slot = 0;
        while (sv->stream_busy[slot]) ++slot;
        sv->stream_busy[slot] = true;
        sv->busy++;
        sv->inflight_bytes += bytes;
        sv->batches++;
        sv->batched_requests += (int64_t)take.size();
        sv->jobs[slot] = std::move(take);
        sv->cv_work.notify_all();
    }
}

}  // namespace dl

struct dl_server : public dl::Server {};

using namespace dl;

extern "C" {

int dl_server_create(dl_server **out, const dl_store *S, int64_t mem_budget_bytes, int32_t slots, int64_t max_batch_rows,
                     const dl_join_opts *opts)
{
    clear_error();
    if (!out || !S || mem_budget_bytes <= 0 || slots < 1 || slots > 8 || max_batch_rows < 1) {
        set_error("dl_server_create: bad arguments");
        return DL_EINVAL;
    }
    *out = nullptr;
    dl_server *sv = new dl_server();
    sv->S = S;
    sv->device = S->device;
    sv->budget = mem_budget_bytes;
    sv->slots = slots;
    sv->max_rows = max_batch_rows;
    if (opts)
        sv->opts = *opts;
    else
        dl_join_opts_default(&sv->opts);
    cudaSetDevice(sv->device);
    sv->streams.resize(slots);
    sv->stream_busy.assign(slots, false);
    sv->jobs.resize(slots);
    for (int i = 0; i < slots; ++i) {
        cudaError_t e = cudaStreamCreateWithFlags(&sv->streams[i], cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            for (int j = 0; j < i; ++j) cudaStreamDestroy(sv->streams[j]);
            delete sv;
            return cuda_fail(e, "dl_server_create stream");
        }
    }
    for (int i = 0; i < slots; ++i) sv->workers.emplace_back(worker, sv, i);
    sv->sched = std::thread(scheduler, sv);
    *out = sv;
    return DL_OK;
}

int dl_submit(dl_server *sv, const int64_t *q_ids, const float *q_feats, int64_t nq, int32_t kind, double eps,
              int32_t k, uint64_t *ticket)
{
    clear_error();
    if (!sv || !ticket || nq < 0 || (nq > 0 && (!q_ids || !q_feats))) {
        set_error("dl_submit: bad arguments");
        return DL_EINVAL;
    }
    if (kind == DL_REQ_EPS && (std::isnan(eps) || eps < 0.0)) {
        set_error("dl_submit: eps must be >= 0");
        return DL_EINVAL;
    }
    if (kind == DL_REQ_TOPK && (k < 1 || k > 1024)) {
        set_error("dl_submit: k out of range");
        return DL_EINVAL;
    }
    if (kind != DL_REQ_EPS && kind != DL_REQ_TOPK) {
        set_error("dl_submit: bad kind %d", kind);
        return DL_EINVAL;
    }
    if (nq > sv->max_rows) {
        set_error("dl_submit: %lld query rows exceed the server's batch row limit %lld", (long long)nq,
                  (long long)sv->max_rows);
        return DL_ENOMEM_ADMIT;
    }
    auto q = std::make_shared<Req>();
    q->kind = kind;
    q->k = kind == DL_REQ_TOPK ? k : 0;
    q->eps = eps;
    q->nq = nq;
    q->ids.assign(q_ids, q_ids + nq);
    q->feats.assign(q_feats, q_feats + nq * sv->S->d);
    q->est_bytes = estimate_bytes(sv->S, kind, nq, q->k);
    if (q->est_bytes > sv->budget) {
        set_error("dl_submit: request needs ~%lld bytes, more than the server budget %lld",
                  (long long)q->est_bytes, (long long)sv->budget);
        return DL_ENOMEM_ADMIT;
    }
    q->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        q->ticket = sv->next_ticket++;
        sv->all[q->ticket] = q;
        sv->queue.push_back(q);
        *ticket = q->ticket;
    }
    sv->cv_sched.notify_one();
    return DL_OK;
}

int dl_poll(dl_server *sv, uint64_t ticket, int64_t timeout_us, dl_result **out)
{
    clear_error();
    if (!sv || !out) {
        set_error("dl_poll: bad arguments");
        return DL_EINVAL;
    }
    *out = nullptr;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) {
        set_error("dl_poll: unknown ticket %llu", (unsigned long long)ticket);
        return DL_EINVAL;
    }
    auto q = it->second;
    if (q->status == DL_EAGAIN && !q->canceled && timeout_us > 0)
        sv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us),
                             [&] { return q->status != DL_EAGAIN || q->canceled; });
    if (q->canceled) {
        sv->all.erase(ticket);
        return DL_ECANCELED;
    }
    if (q->status == DL_EAGAIN) return timeout_us > 0 ? DL_ETIMEOUT : DL_EAGAIN;
    const int st = q->status;
    if (st == DL_OK) *out = q->result;
    q->result = nullptr;
    sv->all.erase(ticket);
    if (st != DL_OK) set_error("dl_poll: request failed; it may be resubmitted");
    return st;
}

int dl_cancel(dl_server *sv, uint64_t ticket)
{
    if (!sv) return DL_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) return DL_EINVAL;
    auto q = it->second;
    for (auto qi = sv->queue.begin(); qi != sv->queue.end(); ++qi)
        if ((*qi)->ticket == ticket) {   // still queued: drop it
            sv->queue.erase(qi);
            q->canceled = true;
            sv->cv_done.notify_all();
            return DL_OK;
        }
    set_error("dl_cancel: request already running or finished");
    return DL_EAGAIN;
}

int dl_server_get_stats(dl_server *sv, dl_server_stats *st)
{
    if (!sv || !st) return DL_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    std::memset(st, 0, sizeof *st);
    st->completed = sv->done;
    st->failed = sv->failed;
    st->batches = sv->batches;
    st->queued = (int64_t)sv->queue.size();
    st->in_flight_batches = sv->busy;
    st->admission_waits = sv->admit_waits;
    if (!sv->lat_ms.empty()) {
        std::vector<double> v = sv->lat_ms;
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) { return v[std::min(v.size() - 1, (size_t)(p * (v.size() - 1) + 0.5))]; };
        st->p50_ms = pct(0.50);
        st->p99_ms = pct(0.99);
        st->max_ms = v.back();
        double s = 0;
        for (double x : v) s += x;
        st->mean_ms = s / v.size();
    }
    st->mean_batch_requests = sv->batches ? (double)sv->batched_requests / sv->batches : 0.0;
    return DL_OK;
}

int dl_server_destroy(dl_server *sv)
{
    if (!sv) return DL_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;   // queued requests are dropped; batches already handed over finish
    }
    sv->cv_sched.notify_all();
    sv->cv_work.notify_all();
    if (sv->sched.joinable()) sv->sched.join();
    for (auto &w : sv->workers)
        if (w.joinable()) w.join();
    for (auto &kv : sv->all)
        if (kv.second->result) dl_result_free(kv.second->result);
    for (auto s : sv->streams) cudaStreamDestroy(s);
    delete sv;
    return DL_OK;
}

}  // extern "C"
