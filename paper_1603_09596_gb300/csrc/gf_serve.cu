// gf_serve.cu -- continuous-batching request loop over several resident forests.
//
// Requests (one query vector each, for one of the server's forests) are queued per forest.  A
// dispatcher thread forms a batch from the forest whose oldest request has waited longest and
// launches it on a free slot.  A slot owns a CUDA stream and every buffer a batch needs (pinned
// host staging, device queries / results, the streaming kernel's workspace), reserved at creation
// within the HBM budget, so a batch is admitted exactly when a slot -- and its memory -- is free.
// Batches on different slots overlap on the device; requests that arrive while others run are
// picked up by the next free slot.  A completion thread polls the slots' events, hands results to
// their requests and records the latency from submission to completion.
//
// Every wait is bounded: gf_server_poll returns GF_ETIMEOUT after its timeout and the server's own
// threads re-check their stop flag at least every millisecond.
#include "gf_internal.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <random>
#include <thread>
#include <unordered_map>
#include <vector>

using Clock = std::chrono::steady_clock;

namespace {

struct Request {
    uint64_t ticket;
    int forest;
    int k;
    std::vector<float> q;
    Clock::time_point t0;
    // result
    std::vector<int64_t> ids;
    std::vector<float> dists;
    int status = GF_OK;
    bool done = false;
    double latency_ms = 0.0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    float *q_host = nullptr;
    int64_t *ids_host = nullptr;
    float *d_host = nullptr;
    float *q_dev = nullptr;
    int64_t *ids_dev = nullptr;
    float *d_dev = nullptr;
    void *ws = nullptr;
    int64_t ws_bytes = 0;
    bool busy = false;
    bool inflight = false;
    int status = GF_OK;
    int k = 0;
    int algo = GF_ALGO_STREAM;  // the kernel path of the batch in flight
    std::vector<Request *> batch;
};

}  // namespace

struct gf_server {
    std::vector<gf_forest *> forests;
    gf_server_opts opts;
    int dmax = 0;
    std::mutex mu;
    std::condition_variable cv_work;   // dispatcher: new request or a free slot
    std::condition_variable cv_done;   // pollers: a request finished
    std::condition_variable cv_inflight;  // completer: a batch was launched
    std::vector<std::deque<Request *>> queues;
    std::unordered_map<uint64_t, Request *> requests;
    std::vector<Slot> slots;
    std::thread dispatcher, completer;
    bool stop = false;
    uint64_t next_ticket = 1;
    // statistics
    std::vector<double> lat_ms;
    uint64_t batches = 0, batched_queries = 0, completed = 0, leaf_batches = 0;
    Clock::time_point t_first, t_last;
    bool any = false;
};

static void release_slot_memory(Slot &s) {
    if (s.stream) cudaStreamSynchronize(s.stream);
    cudaFreeHost(s.q_host);
    cudaFreeHost(s.ids_host);
    cudaFreeHost(s.d_host);
    cudaFree(s.q_dev);
    cudaFree(s.ids_dev);
    cudaFree(s.d_dev);
    cudaFree(s.ws);
    if (s.ev) cudaEventDestroy(s.ev);
    if (s.stream) cudaStreamDestroy(s.stream);
    s = Slot();
}

// The kernel of a batch of m queries on F: the leaf-major path when the server allows it and the
// batch shares leaves enough for it to pay (the rule of GF_ALGO_AUTO), else the streaming kernel.
static int32_t batch_algo(const gf_server *S, const gf_forest *F, int64_t m, int32_t k) {
    if (S->opts.algo == GF_ALGO_STREAM) return GF_ALGO_STREAM;
    const int p = S->opts.precision;
    const int R = S->opts.rerank_R > 0 ? S->opts.rerank_R : F->tune_R[p];
    QueryExtra x;
    x.leaf_budget = leaf_budget_of(F, S->opts.checks, S->opts.eps);
    return gf_leaf_preferred(F, m, k, p, R, x) ? GF_ALGO_LEAF : GF_ALGO_STREAM;
}

// Launch one batch on slot s (called by the dispatcher without the lock held).
static int launch_batch(gf_server *S, Slot &s, int f) {
    gf_forest *F = S->forests[f];
    const int m = (int)s.batch.size(), d = F->d, k = s.k;
    for (int i = 0; i < m; ++i) std::memcpy(s.q_host + (size_t)i * d, s.batch[i]->q.data(), (size_t)d * 4);
    GF_CUDA_TRY(cudaMemcpyAsync(s.q_dev, s.q_host, (size_t)m * d * 4, cudaMemcpyHostToDevice, s.stream));
    gf_query_opts o;
    gf_query_opts_default(&o);
    o.precision = S->opts.precision;
    o.rerank_R = S->opts.rerank_R;
    o.checks = S->opts.checks;
    o.eps = S->opts.eps;
    o.stream = s.stream;
    o.algo = batch_algo(S, F, m, k);
    s.algo = o.algo;
    o.workspace = s.ws;
    o.workspace_bytes = s.ws_bytes;
    int r = gf_query_ex(F, s.q_dev, m, k, &o, s.ids_dev, s.d_dev);
    if (r) return r;
    GF_CUDA_TRY(cudaMemcpyAsync(s.ids_host, s.ids_dev, (size_t)m * k * 8, cudaMemcpyDeviceToHost, s.stream));
    GF_CUDA_TRY(cudaMemcpyAsync(s.d_host, s.d_dev, (size_t)m * k * 4, cudaMemcpyDeviceToHost, s.stream));
    GF_CUDA_TRY(cudaEventRecord(s.ev, s.stream));
    return GF_OK;
}

static void dispatcher_loop(gf_server *S, int device) {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        // wait for work and a free slot (bounded, re-checking the stop flag)
        int slot = -1, f = -1;
        while (true) {
            if (S->stop) return;
            slot = -1;
            for (size_t i = 0; i < S->slots.size(); ++i)
                if (!S->slots[i].busy) { slot = (int)i; break; }
            f = -1;
            for (size_t i = 0; i < S->queues.size(); ++i)
                if (!S->queues[i].empty() && (f < 0 || S->queues[i].front()->t0 < S->queues[f].front()->t0)) f = (int)i;
            if (slot >= 0 && f >= 0) break;
            S->cv_work.wait_for(lk, std::chrono::milliseconds(1));
        }
        Slot &s = S->slots[slot];
        s.busy = true;
        s.batch.clear();
        s.k = 0;
        auto &q = S->queues[f];
        while (!q.empty() && (int)s.batch.size() < S->opts.max_batch) {
            s.batch.push_back(q.front());
            s.k = std::max(s.k, q.front()->k);
            q.pop_front();
        }
        lk.unlock();
        const int r = launch_batch(S, s, f);
        lk.lock();
        s.status = r;
        s.inflight = true;
        S->batches++;
        S->leaf_batches += s.algo == GF_ALGO_LEAF;
        S->batched_queries += s.batch.size();
        S->cv_inflight.notify_one();
    }
}

static void completer_loop(gf_server *S, int device) {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        bool any_inflight = false, progressed = false;
        for (auto &s : S->slots) {
            if (!s.inflight) continue;
            any_inflight = true;
            // a failed launch completes at once; otherwise wait for the slot's event
            const bool ready = s.status != GF_OK || cudaEventQuery(s.ev) == cudaSuccess;
            if (!ready) continue;
            const auto now = Clock::now();
            for (size_t i = 0; i < s.batch.size(); ++i) {
                Request *rq = s.batch[i];
                rq->status = s.status;
                if (s.status == GF_OK) {
                    rq->ids.assign(s.ids_host + i * s.k, s.ids_host + i * s.k + rq->k);
                    rq->dists.assign(s.d_host + i * s.k, s.d_host + i * s.k + rq->k);
                }
                rq->latency_ms = std::chrono::duration<double, std::milli>(now - rq->t0).count();
                rq->done = true;
                S->lat_ms.push_back(rq->latency_ms);
                S->completed++;
                if (!S->any) { S->t_first = rq->t0; S->any = true; }
                S->t_last = now;
            }
            s.batch.clear();
            s.inflight = false;
            s.busy = false;
            progressed = true;
        }
        if (progressed) {
            S->cv_done.notify_all();
            S->cv_work.notify_one();
            continue;
        }
        if (S->stop && !any_inflight) return;
        if (any_inflight) {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        } else {
            S->cv_inflight.wait_for(lk, std::chrono::milliseconds(1));
        }
    }
}

extern "C" void gf_server_opts_default(gf_server_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->max_batch = 1024;
    o->slots = 4;
    o->hbm_budget_bytes = (int64_t)4 << 30;
    o->k_max = 10;
    o->precision = GF_FP32;
}

extern "C" int gf_server_create(gf_forest *const *forests, int32_t nforests, const gf_server_opts *opts,
                                gf_server **out) {
    if (!out) return gf_fail(GF_EINVAL, "out is null");
    *out = nullptr;
    if (!forests || nforests < 1) return gf_fail(GF_EINVAL, "no forests");
    gf_server_opts o;
    gf_server_opts_default(&o);
    if (opts) o = *opts;
    if (o.max_batch < 1 || o.slots < 1 || o.k_max < 1 || o.hbm_budget_bytes <= 0 ||
        (o.algo != GF_ALGO_AUTO && o.algo != GF_ALGO_STREAM))
        return gf_fail(GF_EINVAL, "bad server options");
    if (o.precision != GF_FP32 && o.k_max > (o.rerank_R > 0 ? o.rerank_R : 64))
        return gf_fail(GF_EINVAL, "k_max exceeds the shortlist");
    auto *S = new gf_server();
    S->opts = o;
    int64_t ws_max = 0;
    for (int i = 0; i < nforests; ++i) {
        if (!forests[i]) { delete S; return gf_fail(GF_EINVAL, "forest %d is null", i); }
        if (o.precision == GF_BF16_RERANK && !forests[i]->xb) { delete S; return gf_fail(GF_EINVAL, "forest %d has no bf16 copy", i); }
        if (o.precision == GF_FP8_RERANK && !forests[i]->x8) { delete S; return gf_fail(GF_EINVAL, "forest %d has no fp8 copy", i); }
        S->forests.push_back(forests[i]);
        S->dmax = std::max(S->dmax, forests[i]->d);
        gf_query_opts qo;
        gf_query_opts_default(&qo);
        qo.precision = o.precision;
        qo.rerank_R = o.rerank_R;
        qo.checks = o.checks;
        qo.eps = o.eps;
        qo.algo = GF_ALGO_STREAM;  // the streaming kernel, for any batch
        int64_t b = 0;
        int r = gf_query_workspace_size(forests[i], o.max_batch, &qo, &b);
        if (r) { delete S; return r; }
        ws_max = std::max(ws_max, b);
        // the leaf-major path, for a full batch if it would take one (its scratch grows with m)
        if (batch_algo(S, forests[i], o.max_batch, 1) == GF_ALGO_LEAF) {
            qo.algo = GF_ALGO_LEAF;
            if ((r = gf_query_workspace_size(forests[i], o.max_batch, &qo, &b))) { delete S; return r; }
            ws_max = std::max(ws_max, b);
        }
    }
    const int64_t per_slot = (int64_t)o.max_batch * S->dmax * 4 + (int64_t)o.max_batch * o.k_max * 12 + ws_max;
    const int nslots = (int)std::min<int64_t>(o.slots, o.hbm_budget_bytes / per_slot);
    if (nslots < 1) {
        delete S;
        return gf_fail(GF_ENOMEM, "HBM budget %lld B holds no batch slot (%lld B each)", (long long)o.hbm_budget_bytes,
                       (long long)per_slot);
    }
    S->queues.resize(nforests);
    S->slots.resize(nslots);
    int device = 0;
    cudaGetDevice(&device);
    for (auto &s : S->slots) {
        cudaError_t e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost(&s.q_host, (size_t)o.max_batch * S->dmax * 4);
        if (e == cudaSuccess) e = cudaMallocHost(&s.ids_host, (size_t)o.max_batch * o.k_max * 8);
        if (e == cudaSuccess) e = cudaMallocHost(&s.d_host, (size_t)o.max_batch * o.k_max * 4);
        if (e == cudaSuccess) e = cudaMalloc(&s.q_dev, (size_t)o.max_batch * S->dmax * 4);
        if (e == cudaSuccess) e = cudaMalloc(&s.ids_dev, (size_t)o.max_batch * o.k_max * 8);
        if (e == cudaSuccess) e = cudaMalloc(&s.d_dev, (size_t)o.max_batch * o.k_max * 4);
        if (e == cudaSuccess && ws_max > 0) e = cudaMalloc(&s.ws, (size_t)ws_max);
        if (e == cudaSuccess && ws_max > 0) e = cudaMemset(s.ws, 0, (size_t)ws_max);
        s.ws_bytes = ws_max;
        if (e != cudaSuccess) {
            cudaGetLastError();
            for (auto &t : S->slots) release_slot_memory(t);
            delete S;
            return gf_cuda_fail(e, "server slot allocation");
        }
    }
    S->dispatcher = std::thread(dispatcher_loop, S, device);
    S->completer = std::thread(completer_loop, S, device);
    *out = S;
    return GF_OK;
}

extern "C" int gf_server_slots(const gf_server *S) { return S ? (int)S->slots.size() : 0; }

extern "C" int gf_server_submit(gf_server *S, int32_t forest, const float *q_host, int32_t k, uint64_t *ticket) {
    if (!S || !q_host || !ticket) return gf_fail(GF_EINVAL, "null argument");
    if (forest < 0 || forest >= (int)S->forests.size()) return gf_fail(GF_EINVAL, "forest %d out of range", forest);
    if (k < 1 || k > S->opts.k_max) return gf_fail(GF_EINVAL, "k=%d outside [1, %d]", k, S->opts.k_max);
    auto *rq = new Request();
    rq->forest = forest;
    rq->k = k;
    rq->q.assign(q_host, q_host + S->forests[forest]->d);
    rq->t0 = Clock::now();
    {
        std::lock_guard<std::mutex> g(S->mu);
        if (S->stop) { delete rq; return gf_fail(GF_EINVAL, "server is stopping"); }
        rq->ticket = S->next_ticket++;
        S->requests[rq->ticket] = rq;
        S->queues[forest].push_back(rq);
        *ticket = rq->ticket;
    }
    S->cv_work.notify_one();
    return GF_OK;
}

extern "C" int gf_server_poll(gf_server *S, uint64_t ticket, int64_t *ids_host, float *dists_host,
                              int32_t timeout_us) {
    if (!S) return gf_fail(GF_EINVAL, "null server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->requests.find(ticket);
    if (it == S->requests.end()) return gf_fail(GF_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    Request *rq = it->second;
    const auto deadline = Clock::now() + std::chrono::microseconds(std::max(0, timeout_us));
    while (!rq->done) {
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !rq->done)
            return gf_fail(GF_ETIMEOUT, "request %llu not finished", (unsigned long long)ticket);
    }
    const int st = rq->status;
    if (st == GF_OK) {
        if (ids_host) std::memcpy(ids_host, rq->ids.data(), rq->ids.size() * 8);
        if (dists_host) std::memcpy(dists_host, rq->dists.data(), rq->dists.size() * 4);
    }
    S->requests.erase(it);
    delete rq;
    return st;
}

static double percentile(std::vector<double> v, double p) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = p * (v.size() - 1);
    const size_t i = (size_t)pos;
    const double f = pos - i;
    return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

extern "C" int gf_server_get_stats(gf_server *S, gf_server_stats *st) {
    if (!S || !st) return gf_fail(GF_EINVAL, "null argument");
    std::lock_guard<std::mutex> g(S->mu);
    std::memset(st, 0, sizeof *st);
    st->completed = (int64_t)S->completed;
    st->batches = (int64_t)S->batches;
    st->mean_batch = S->batches ? (double)S->batched_queries / S->batches : 0.0;
    st->p50_ms = percentile(S->lat_ms, 0.50);
    st->p99_ms = percentile(S->lat_ms, 0.99);
    st->max_ms = S->lat_ms.empty() ? 0.0 : *std::max_element(S->lat_ms.begin(), S->lat_ms.end());
    st->span_s = S->any ? std::chrono::duration<double>(S->t_last - S->t_first).count() : 0.0;
    st->qps = st->span_s > 0 ? st->completed / st->span_s : 0.0;
    st->slots = (int32_t)S->slots.size();
    st->leaf_batches = (int32_t)std::min<uint64_t>(S->leaf_batches, INT32_MAX);
    return GF_OK;
}

extern "C" int gf_server_reset_stats(gf_server *S) {
    if (!S) return gf_fail(GF_EINVAL, "null server");
    std::lock_guard<std::mutex> g(S->mu);
    S->lat_ms.clear();
    S->batches = S->batched_queries = S->completed = S->leaf_batches = 0;
    S->any = false;
    return GF_OK;
}

extern "C" int gf_server_destroy(gf_server *S) {
    if (!S) return GF_OK;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    S->cv_inflight.notify_all();
    if (S->dispatcher.joinable()) S->dispatcher.join();
    if (S->completer.joinable()) S->completer.join();
    for (auto &s : S->slots) release_slot_memory(s);
    for (auto &kv : S->requests) delete kv.second;
    for (auto &q : S->queues) q.clear();
    delete S;
    return GF_OK;
}

// Open-loop load: Poisson arrivals at `rate_qps` for `duration_s`, each request for a forest drawn
// uniformly, its query taken round-robin from that forest's host query set; waits (bounded) for
// every request, then fills `st`.
extern "C" int gf_server_run_poisson(gf_server *S, const float *const *queries_host, const int64_t *nq,
                                     double rate_qps, double duration_s, int32_t k, uint64_t seed,
                                     int32_t timeout_ms, gf_server_stats *st) {
    if (!S || !queries_host || !nq || rate_qps <= 0 || duration_s <= 0)
        return gf_fail(GF_EINVAL, "bad load arguments");
    const int nf = (int)S->forests.size();
    for (int f = 0; f < nf; ++f)
        if (!queries_host[f] || nq[f] < 1) return gf_fail(GF_EINVAL, "forest %d has no queries", f);
    gf_server_reset_stats(S);
    std::mt19937_64 rng(seed);
    std::exponential_distribution<double> gap(rate_qps);
    std::uniform_int_distribution<int> pick(0, nf - 1);
    std::vector<int64_t> next(nf, 0);
    std::vector<uint64_t> tickets;
    const auto t0 = Clock::now();
    double t = 0.0;
    while (t < duration_s) {
        t += gap(rng);
        const auto due = t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(t));
        std::this_thread::sleep_until(due);
        const int f = pick(rng);
        const float *q = queries_host[f] + (size_t)(next[f] % nq[f]) * S->forests[f]->d;
        next[f]++;
        uint64_t tk = 0;
        int r = gf_server_submit(S, f, q, k, &tk);
        if (r) return r;
        tickets.push_back(tk);
    }
    int worst = GF_OK;
    for (uint64_t tk : tickets) {
        int r = gf_server_poll(S, tk, nullptr, nullptr, timeout_ms * 1000);
        if (r && !worst) worst = r;
    }
    if (st) gf_server_get_stats(S, st);
    return worst;
}
