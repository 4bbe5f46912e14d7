// Serving layer: asynchronous requests with continuous batching.
//
// aidw_submit queues a request and returns a handle. A worker thread owned by the context
// admits queued requests in arrival order while their device footprint (batch scratch plus
// staging of host arrays) fits the serving budget, packs them into one persistent batch launch
// (batched.cu) on one of several streams, and goes on admitting newly arrived requests into the
// next launch on another stream while earlier launches still run, so their work overlaps on the
// device. Completion is observed with events; the footprint is then returned to the budget.
// FP32 requests without a kNN output go through the batch kernel, whose per-item result does
// not depend on the batch composition; FP64 requests and requests asking for neighbour indices
// run alone through the one-shot path.
//
// A large FP32 request is cut into chunks of contiguous queries of about kChunkPairs
// pair-evaluations each (the cut depends on the request's own sizes only, so its result is the
// same alone and in any mix), and a flight takes at most one chunk of each queued request, in
// arrival order, up to about kFlightPairs pair-evaluations in all. A launch then lasts tens of
// milliseconds at most, and a small request arriving behind a large one waits for one flight
// instead of the whole large request (a persistent batch kernel holds every SM until its work
// runs out, so a launch on the other stream cannot start earlier).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "aidw_internal.cuh"
#include "aidw_runtime.h"

namespace aidw {

namespace {

using Clock = std::chrono::steady_clock;

inline size_t align256(size_t b)
{
    return (b + 255) & ~static_cast<size_t>(255);
}

// Chunking of large requests and the work cap of one flight (pair-evaluations; about 14 ms and
// 35 ms of the GPU at the batch kernel's rate). Measured on the served workload (64 datasets,
// 256-262,144 queries a request) against no chunking: p99 80 against 99 ms at half the
// capacity and 427 against 515 ms at 0.8 of it, throughput at 7x overload 2.63e12 against
// 2.71e12 pair-evals/s; caps of 1.6e10 / 3.2e10 made flights so short (1.5 requests a launch)
// that throughput at overload fell to 2.34e12 without a better p99.
constexpr double kChunkPairs = 4e10;
constexpr double kFlightPairs = 1e11;

// Express lane: requests of at most kExpressPairs pair-evaluations (about 1-2 ms on one CTA per
// SM) may also go to a launch of their own, one persistent CTA per SM, taken out of arrival
// order; the other launches leave one CTA slot per SM free for it, so that a small request
// starts at once instead of waiting for a large launch to release the SMs (measured cost for a
// large batch: 72.3 against 70.9 ms with 7 instead of 8 CTAs per SM).
constexpr double kExpressPairs = 5e8;
constexpr double kExpressFlightPairs = 2e9;
constexpr size_t kExpressScan = 256;  // queued requests the express lane looks at

struct Request {
    int64_t ds = 0;
    const void *qx = nullptr, *qy = nullptr;
    int64_t m = 0;
    aidw_params p{};
    void *out = nullptr;
    float *out_alpha = nullptr;
    int32_t *out_knn = nullptr;
    bool host_qx = false, host_qy = false, host_out = false, host_alpha = false;
    bool solo = false;  // FP64 or kNN output: runs through the one-shot path
    int64_t n_pad = 0;  // the dataset's padded size (chunk footprints)
    int64_t n = 0;      // the dataset's size (chunk work)
    int64_t chunk_m = 0;  // queries per chunk (the last one may hold fewer)
    int32_t nchunks = 1, next_chunk = 0, chunks_done = 0;
    size_t footprint = 0;  // of the largest chunk
    int status = AIDW_PENDING;
    bool done = false;
    Clock::time_point t_submit, t_done;
};

// One chunk of a request in a flight: queries [begin, end) of request id.
struct Piece {
    int64_t id;
    int64_t begin, end;
};

struct Flight {
    bool busy = false;
    bool express = false;  // the express lane (one persistent CTA per SM)
    std::vector<Piece> pieces;
    cudaEvent_t done_ev = nullptr;
    cudaStream_t stream = nullptr;
    void *pinned = nullptr;  // host staging (pinned), grown on demand
    size_t pinned_bytes = 0;
    size_t footprint = 0;
    // Host copies to perform when the launch completes: (dst user pointer, src pinned, bytes).
    struct CopyOut {
        void *dst;
        const void *src;
        size_t bytes;
    };
    std::vector<CopyOut> copy_out;
};

}  // namespace

struct ServingRuntime {
    aidw_ctx *ctx = nullptr;
    aidw_tune_config cfg{};  // kernel shape: the context's when the runtime started
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<int64_t> queue;
    std::unordered_map<int64_t, Request> reqs;
    int64_t next_id = 1;
    size_t max_queue = 4096;
    size_t budget = size_t(8) << 30;  // device bytes in flight
    size_t in_flight = 0;
    int max_items = 256;
    int n_slots = 2;           // launches at once, besides the express lane
    bool express_lane = true;  // flights.back() is the express lane
    std::vector<Flight> flights;
    bool stop = false;
    std::thread worker;
    aidw_serving_stats stats{};
};

namespace {

// Device bytes of `m` queries of request r in a flight: batch scratch plus host staging.
size_t request_footprint(const Request &r, int64_t m_chunk, int64_t n_pad,
                         const aidw_tune_config &cfg)
{
    size_t b = batch_item_bytes(n_pad, m_chunk, r.p.k, cfg) + 4096;
    const size_t m = static_cast<size_t>(m_chunk);
    if (r.host_qx)
        b += align256(4 * m);
    if (r.host_qy)
        b += align256(4 * m);
    if (r.host_out)
        b += align256(4 * m);
    if (r.host_alpha)
        b += align256(4 * m);
    return b;
}

// Completes a whole request (status, time, statistics).
void finish_request(ServingRuntime *rt, Request &r, int status, Clock::time_point now)
{
    if (r.status == AIDW_PENDING)
        r.status = status;
    r.done = true;
    r.t_done = now;
    if (r.status == AIDW_OK)
        ++rt->stats.completed;
    else
        ++rt->stats.failed;
}

void finish(ServingRuntime *rt, const std::vector<int64_t> &ids, int status)
{
    const auto now = Clock::now();
    for (int64_t id : ids)
        finish_request(rt, rt->reqs[id], status, now);
}

// One launch's chunks have finished: a request is done once all its chunks are (its status is
// its first error, if any).
void finish_pieces(ServingRuntime *rt, const std::vector<Piece> &pieces, int status)
{
    const auto now = Clock::now();
    for (const Piece &pc : pieces) {
        Request &r = rt->reqs[pc.id];
        if (status != AIDW_OK && r.status == AIDW_PENDING)
            r.status = status;
        if (++r.chunks_done == r.nchunks)
            finish_request(rt, r, AIDW_OK, now);
    }
}

// Admission of the next chunk of a queued request into the flight being assembled (pure host
// logic; aidw_debug_admission runs it without a GPU). Queued requests are visited in arrival
// order, one chunk each per flight: a chunk that does not fit stops the flight (no overtaking),
// as does one that would take the flight's work above max_flight_pairs (unless the flight is
// empty: a flight always takes its first chunk); a request that could never fit the budget
// fails with OOM, and FP64 / kNN-output requests run alone.
enum class Admit { kTake, kSolo, kRejectOom, kStop };

Admit admission_step(bool solo, size_t footprint, size_t budget, size_t in_flight,
                     size_t flight_bytes, size_t flight_count, int max_items, double pairs,
                     double flight_pairs, double max_flight_pairs)
{
    if (static_cast<int64_t>(flight_count) >= max_items)
        return Admit::kStop;
    if (solo)
        return flight_count == 0 ? Admit::kSolo : Admit::kStop;
    if (footprint > budget)
        return Admit::kRejectOom;
    if (in_flight + flight_bytes + footprint > budget)
        return Admit::kStop;
    if (flight_count > 0 && max_flight_pairs > 0.0 && flight_pairs + pairs > max_flight_pairs)
        return Admit::kStop;
    return Admit::kTake;
}

bool ensure_pinned(Flight &f, size_t bytes)
{
    if (f.pinned_bytes >= bytes)
        return true;
    if (f.pinned)
        cudaFreeHost(f.pinned);
    f.pinned = nullptr;
    f.pinned_bytes = 0;
    size_t cap = bytes + bytes / 2 + (1 << 20);
    if (cudaHostAlloc(&f.pinned, cap, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    f.pinned_bytes = cap;
    return true;
}

// Launches the batch of request chunks `pc` (rq[i] owns pc[i]) on flight slot f. Called without
// the runtime lock; the chunks are owned by this launch until completion.
int launch_flight(ServingRuntime *rt, Flight &f, const std::vector<Request *> &rq,
                  const std::vector<Piece> &pc)
{
    NvtxScope range("aidw serving flight");
    aidw_ctx *ctx = rt->ctx;
    cudaStream_t st = f.stream;
    // Staging sizes.
    size_t host_bytes = 0, dev_bytes = 0;
    for (size_t i = 0; i < rq.size(); ++i) {
        const Request *r = rq[i];
        const size_t b = align256(4 * static_cast<size_t>(pc[i].end - pc[i].begin));
        const size_t h = (r->host_qx ? b : 0) + (r->host_qy ? b : 0) + (r->host_out ? b : 0) +
                         (r->host_alpha ? b : 0);
        host_bytes += h;
        dev_bytes += h;
    }
    f.copy_out.clear();
    if (host_bytes && !ensure_pinned(f, host_bytes))
        return AIDW_ERR_OOM;
    void *dstage = nullptr;
    int rc = ctx_alloc(ctx, dev_bytes, st, &dstage);
    if (rc)
        return rc;
    std::vector<aidw_batch_item> items(rq.size());
    char *hp = static_cast<char *>(f.pinned);
    char *dp = static_cast<char *>(dstage);
    bool ok = true;
    for (size_t i = 0; i < rq.size(); ++i) {
        const Request &r = *rq[i];
        const int64_t b0 = pc[i].begin;
        const size_t bytes = 4 * static_cast<size_t>(pc[i].end - b0), b = align256(bytes);
        aidw_batch_item &it = items[i];
        it.ds = r.ds;
        it.m = pc[i].end - b0;
        it.params = r.p;
        it.qx = static_cast<const float *>(r.qx) + b0;
        it.qy = static_cast<const float *>(r.qy) + b0;
        it.out = static_cast<float *>(r.out) + b0;
        it.out_alpha = r.out_alpha ? r.out_alpha + b0 : nullptr;
        auto stage_in = [&](const float *src, const float **dst) {
            std::memcpy(hp, src, bytes);
            ok &= cudaMemcpyAsync(dp, hp, bytes, cudaMemcpyHostToDevice, st) == cudaSuccess;
            *dst = reinterpret_cast<const float *>(dp);
            hp += b;
            dp += b;
        };
        auto stage_out = [&](float *user, float **dst) {
            *dst = reinterpret_cast<float *>(dp);
            f.copy_out.push_back({user, hp, bytes});
            hp += b;
            dp += b;
        };
        if (r.host_qx)
            stage_in(it.qx, &it.qx);
        if (r.host_qy)
            stage_in(it.qy, &it.qy);
        if (r.host_out)
            stage_out(it.out, &it.out);
        if (r.host_alpha)
            stage_out(it.out_alpha, &it.out_alpha);
    }
    if (!ok) {
        ctx_free(ctx, dstage, dev_bytes, st);
        return AIDW_ERR_CUDA;
    }
    BatchState bs{};
    aidw_tune_config cfg = rt->cfg;
    int reserve = 0;
    if (f.express)
        cfg.ctas_per_sm = 1;
    else if (rt->express_lane)
        reserve = 1;
    rc = batch_build(ctx, items.data(), static_cast<int32_t>(items.size()), st, &bs, cfg,
                     reserve);
    if (rc == AIDW_OK)
        rc = batch_enqueue(ctx, bs, st);
    if (rc == AIDW_OK) {
        // Device staging of outputs -> pinned host staging, in the same order as copy_out.
        char *d = static_cast<char *>(dstage);
        char *h = static_cast<char *>(f.pinned);
        for (size_t i = 0; i < rq.size(); ++i) {
            const Request &r = *rq[i];
            const size_t bytes = 4 * static_cast<size_t>(pc[i].end - pc[i].begin);
            const size_t b = align256(bytes);
            if (r.host_qx)
                d += b, h += b;
            if (r.host_qy)
                d += b, h += b;
            if (r.host_out) {
                cudaMemcpyAsync(h, d, bytes, cudaMemcpyDeviceToHost, st);
                d += b, h += b;
            }
            if (r.host_alpha) {
                cudaMemcpyAsync(h, d, bytes, cudaMemcpyDeviceToHost, st);
                d += b, h += b;
            }
        }
    }
    if (bs.block)
        batch_release(ctx, &bs, st);
    ctx_free(ctx, dstage, dev_bytes, st);
    if (rc == AIDW_OK && cudaEventRecord(f.done_ev, st) != cudaSuccess)
        rc = AIDW_ERR_CUDA;
    return rc;
}

void worker_main(ServingRuntime *rt)
{
    cudaSetDevice(ctx_device(rt->ctx));
    std::unique_lock<std::mutex> g(rt->mu);
    for (;;) {
        // 1. Completions.
        bool any_busy = false;
        for (Flight &f : rt->flights) {
            if (!f.busy)
                continue;
            const cudaError_t q = cudaEventQuery(f.done_ev);
            if (q == cudaErrorNotReady) {
                any_busy = true;
                continue;
            }
            int status = q == cudaSuccess ? AIDW_OK : AIDW_ERR_CUDA;
            if (q != cudaSuccess)
                cudaGetLastError();
            for (const Flight::CopyOut &c : f.copy_out)
                std::memcpy(c.dst, c.src, c.bytes);
            f.copy_out.clear();
            finish_pieces(rt, f.pieces, status);
            rt->in_flight -= f.footprint;
            f.footprint = 0;
            f.pieces.clear();
            f.busy = false;
            rt->cv_done.notify_all();
        }
        if (rt->stop && rt->queue.empty() && !any_busy)
            break;
        // 2. Admission into every free slot: one chunk of each queued request at most, in
        // arrival order.
        for (Flight &f : rt->flights) {
            if (f.busy || rt->queue.empty())
                continue;
            std::vector<Piece> pieces;
            std::vector<Request *> rq;
            size_t fp = 0;
            double fpairs = 0.0;
            if (f.express) {
                // Small whole requests from the first kExpressScan queued, out of order.
                for (size_t qi = 0; qi < rt->queue.size() && qi < kExpressScan;) {
                    const int64_t id = rt->queue[qi];
                    Request &r = rt->reqs[id];
                    const double pairs = static_cast<double>(r.m) * static_cast<double>(r.n);
                    const bool small = !r.solo && r.nchunks == 1 && pairs <= kExpressPairs;
                    if (!small || admission_step(false, r.footprint, rt->budget, rt->in_flight,
                                                 fp, pieces.size(), rt->max_items, pairs,
                                                 fpairs, kExpressFlightPairs) != Admit::kTake) {
                        ++qi;
                        continue;
                    }
                    rt->queue.erase(rt->queue.begin() + static_cast<std::ptrdiff_t>(qi));
                    pieces.push_back({id, 0, r.m});
                    rq.push_back(&r);
                    fp += r.footprint;
                    fpairs += pairs;
                    r.next_chunk = 1;
                    ++rt->stats.batched_requests;
                }
            }
            for (size_t qi = 0; !f.express && qi < rt->queue.size();) {
                const int64_t id = rt->queue[qi];
                Request &r = rt->reqs[id];
                const int64_t b = static_cast<int64_t>(r.next_chunk) * r.chunk_m;
                const int64_t e = std::min<int64_t>(b + r.chunk_m, r.m);
                const double pairs = static_cast<double>(e - b) * static_cast<double>(r.n);
                const Admit a = admission_step(r.solo, r.footprint, rt->budget, rt->in_flight, fp,
                                               pieces.size(), rt->max_items, pairs, fpairs,
                                               kFlightPairs);
                if (a == Admit::kStop)
                    break;  // the rest waits for the next flight or for memory to free up
                if (a == Admit::kSolo) {
                    rt->queue.erase(rt->queue.begin() + static_cast<std::ptrdiff_t>(qi));
                    g.unlock();
                    int rc = interpolate_impl(rt->ctx, r.ds, r.qx, r.qy, r.m, &r.p, r.out,
                                              r.out_alpha, r.out_knn, f.stream, 0, 0);
                    if (rc == AIDW_OK && cudaStreamSynchronize(f.stream) != cudaSuccess)
                        rc = AIDW_ERR_CUDA;
                    g.lock();
                    finish(rt, {id}, rc);
                    ++rt->stats.launches;
                    rt->cv_done.notify_all();
                    continue;
                }
                if (a == Admit::kRejectOom) {
                    rt->queue.erase(rt->queue.begin() + static_cast<std::ptrdiff_t>(qi));
                    finish(rt, {id}, AIDW_ERR_OOM);
                    rt->cv_done.notify_all();
                    continue;
                }
                pieces.push_back({id, b, e});
                rq.push_back(&r);
                fp += r.footprint;
                fpairs += pairs;
                if (++r.next_chunk == r.nchunks) {
                    rt->queue.erase(rt->queue.begin() + static_cast<std::ptrdiff_t>(qi));
                    ++rt->stats.batched_requests;
                } else {
                    ++qi;
                }
            }
            if (pieces.empty())
                continue;
            f.busy = true;
            f.pieces = pieces;
            f.footprint = fp;
            rt->in_flight += fp;
            ++rt->stats.launches;
            int live = 0;
            for (const Flight &o : rt->flights)
                live += o.busy ? 1 : 0;
            if (live > rt->stats.max_concurrent_launches)
                rt->stats.max_concurrent_launches = live;
            g.unlock();
            const int rc = launch_flight(rt, f, rq, pieces);
            g.lock();
            if (rc != AIDW_OK) {
                finish_pieces(rt, f.pieces, rc);
                rt->in_flight -= f.footprint;
                f.footprint = 0;
                f.pieces.clear();
                f.busy = false;
                f.copy_out.clear();
                rt->cv_done.notify_all();
            } else {
                any_busy = true;
            }
        }
        // 3. Sleep until new work or a completion is likely.
        if (any_busy)
            rt->cv_work.wait_for(g, std::chrono::microseconds(20));
        else if (rt->queue.empty() && !rt->stop)
            rt->cv_work.wait(g, [&] { return rt->stop || !rt->queue.empty(); });
    }
}

// The launch slots: n_slots regular ones, then the express lane.
void create_flights(ServingRuntime *rt)
{
    rt->flights.resize(rt->n_slots + (rt->express_lane ? 1 : 0));
    for (Flight &f : rt->flights) {
        cudaStreamCreateWithFlags(&f.stream, cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&f.done_ev, cudaEventDisableTiming);
    }
    if (rt->express_lane)
        rt->flights.back().express = true;
}

ServingRuntime *ensure_serving(aidw_ctx *ctx)
{
    const size_t left = ctx_budget_left(ctx);
    const aidw_tune_config cfg = ctx_tune(ctx);
    std::lock_guard<std::mutex> g(ctx_mutex(ctx));
    ServingRuntime *&rt = ctx_serving(ctx);
    if (!rt) {
        rt = new ServingRuntime();
        rt->ctx = ctx;
        rt->cfg = cfg;
        rt->max_queue = static_cast<size_t>(ctx_serving_queue_limit(ctx));
        if (left != SIZE_MAX)
            rt->budget = left / 2;
        cudaSetDevice(ctx_device(ctx));
        create_flights(rt);
        rt->worker = std::thread(worker_main, rt);
    }
    return rt;
}

}  // namespace

void serving_stop(ServingRuntime *rt)
{
    if (!rt)
        return;
    {
        std::lock_guard<std::mutex> g(rt->mu);
        rt->stop = true;
    }
    rt->cv_work.notify_all();
    if (rt->worker.joinable())
        rt->worker.join();
    for (Flight &f : rt->flights) {
        if (f.stream)
            cudaStreamSynchronize(f.stream);
        if (f.pinned)
            cudaFreeHost(f.pinned);
        if (f.done_ev)
            cudaEventDestroy(f.done_ev);
        if (f.stream)
            cudaStreamDestroy(f.stream);
    }
    delete rt;
}

}  // namespace aidw

using namespace aidw;

extern "C" {

// Test hook (not in the public header): runs the serving runtime's admission of one flight over
// a queue of `count` chunks, one per queued request (solo flags, device footprints, nullable
// pair-evaluations) against `budget` with `in_flight` bytes already running and a flight work
// cap of max_flight_pairs (0: none), and writes each chunk's action: 0 taken into the flight,
// 1 run alone, 2 failed with OOM, 3 left in the queue. Host only.
int aidw_debug_admission(int64_t count, const int32_t *solo, const uint64_t *footprint,
                         uint64_t budget, uint64_t in_flight, int32_t max_items,
                         const double *pairs, double max_flight_pairs, int32_t *action)
{
    if (count < 0 || max_items < 1 || (count > 0 && (!solo || !footprint || !action)))
        return AIDW_ERR_INVALID_ARG;
    size_t fp = 0, n = 0;
    double fpairs = 0.0;
    bool stopped = false;
    for (int64_t i = 0; i < count; ++i) {
        if (stopped) {
            action[i] = 3;
            continue;
        }
        const double pr = pairs ? pairs[i] : 0.0;
        switch (admission_step(solo[i] != 0, footprint[i], budget, in_flight, fp, n, max_items,
                               pr, fpairs, max_flight_pairs)) {
        case Admit::kTake:
            action[i] = 0;
            fp += footprint[i];
            fpairs += pr;
            ++n;
            break;
        case Admit::kSolo:
            action[i] = 1;
            break;
        case Admit::kRejectOom:
            action[i] = 2;
            break;
        case Admit::kStop:
            action[i] = 3;
            stopped = true;
            break;
        }
    }
    return AIDW_OK;
}

int aidw_serving_configure(aidw_ctx *ctx, size_t inflight_bytes, int32_t max_batch_requests,
                           int32_t streams, int64_t max_queued)
{
    if (!ctx || max_batch_requests < 0 || streams < 0 || streams > 8 || max_queued < 0)
        return AIDW_ERR_INVALID_ARG;
    const aidw_tune_config cfg = ctx_tune(ctx);
    {
        // The check and the creation in one critical section: a submit on another thread
        // creates the default runtime under the same lock.
        std::lock_guard<std::mutex> g(ctx_mutex(ctx));
        if (ctx_serving(ctx))
            return AIDW_ERR_INVALID_ARG;  // configure before the first submit
        ServingRuntime *rt = new ServingRuntime();
        rt->ctx = ctx;
        rt->cfg = cfg;
        if (max_queued)
            ctx_serving_queue_limit(ctx) = max_queued;
        rt->max_queue = static_cast<size_t>(ctx_serving_queue_limit(ctx));
        if (inflight_bytes)
            rt->budget = inflight_bytes;
        if (max_batch_requests)
            rt->max_items = max_batch_requests;
        if (streams)
            rt->n_slots = streams;
        cudaSetDevice(ctx_device(ctx));
        create_flights(rt);
        rt->worker = std::thread(worker_main, rt);
        ctx_serving(ctx) = rt;
    }
    return AIDW_OK;
}

int aidw_serving_set_queue_limit(aidw_ctx *ctx, int64_t max_queued)
{
    if (!ctx || max_queued < 1)
        return AIDW_ERR_INVALID_ARG;
    ServingRuntime *rt;
    {
        std::lock_guard<std::mutex> g(ctx_mutex(ctx));
        ctx_serving_queue_limit(ctx) = max_queued;
        rt = ctx_serving(ctx);
    }
    if (rt) {
        std::lock_guard<std::mutex> g(rt->mu);
        rt->max_queue = static_cast<size_t>(max_queued);
    }
    return AIDW_OK;
}

int aidw_submit(aidw_ctx *ctx, aidw_dataset ds, const void *qx, const void *qy, int64_t m,
                const aidw_params *p, void *out, float *out_alpha, int32_t *out_knn,
                aidw_request *out_id)
{
    if (!ctx || !out_id || !p)
        return AIDW_ERR_INVALID_ARG;
    *out_id = 0;
    DatasetDev dev;
    double r_exp;
    if (!dataset_lookup(ctx, ds, &dev, &r_exp))
        return AIDW_ERR_NOT_FOUND;
    int rc = validate_params(p, dev.n);
    if (rc)
        return rc;
    if (m < 0 || m > (int64_t(1) << 31) || (m > 0 && (!qx || !qy || !out)))
        return AIDW_ERR_INVALID_ARG;
    const int device = ctx_device(ctx);
    Request r;
    r.ds = ds;
    r.qx = qx;
    r.qy = qy;
    r.m = m;
    r.p = *p;
    r.out = out;
    r.out_alpha = out_alpha;
    r.out_knn = out_knn;
    const int kq = pointer_kind(qx, device), kqy = pointer_kind(qy, device);
    const int ko = pointer_kind(out, device), ka = pointer_kind(out_alpha, device);
    if (kq < 0 || kqy < 0 || ko < 0 || ka < 0 || pointer_kind(out_knn, device) < 0)
        return AIDW_ERR_INVALID_ARG;
    r.host_qx = kq == 0;
    r.host_qy = kqy == 0;
    r.host_out = ko == 0;
    r.host_alpha = out_alpha && ka == 0;
    r.solo = p->precision != AIDW_F32C || out_knn != nullptr;
    ServingRuntime *rt = ensure_serving(ctx);
    {
        // Refuse early when the queue is full, before the O(m) scan of host inputs below (the
        // decisive check is repeated under the same lock when the request is queued).
        std::lock_guard<std::mutex> g(rt->mu);
        if (rt->queue.size() >= rt->max_queue) {
            ++rt->stats.rejected_again;
            return AIDW_ERR_AGAIN;
        }
    }
    if (r.host_qx || r.host_qy) {
        for (int64_t i = 0; i < m; ++i) {
            const float a = static_cast<const float *>(qx)[i];
            const float b = static_cast<const float *>(qy)[i];
            if (!r.solo && !(std::isfinite(a) && std::isfinite(b)))
                return AIDW_ERR_INVALID_ARG;
        }
    }
    r.n = dev.n;
    r.n_pad = dev.n_pad;
    r.chunk_m = m;
    if (!r.solo && m > 0) {
        // Chunks of whole 256-query blocks, about kChunkPairs pair-evaluations each.
        const double per = std::floor(kChunkPairs / static_cast<double>(dev.n) / 256.0) * 256.0;
        r.chunk_m = std::max<int64_t>(256, static_cast<int64_t>(std::min(per, 1e15)));
        if (r.chunk_m >= m)
            r.chunk_m = m;
        r.nchunks = static_cast<int32_t>((m + r.chunk_m - 1) / r.chunk_m);
    }
    r.footprint = request_footprint(r, r.chunk_m, dev.n_pad, rt->cfg);
    {
        std::lock_guard<std::mutex> g(rt->mu);
        if (rt->queue.size() >= rt->max_queue) {
            ++rt->stats.rejected_again;
            return AIDW_ERR_AGAIN;
        }
        const int64_t id = rt->next_id++;
        r.t_submit = Clock::now();
        if (m == 0) {
            r.status = AIDW_OK;
            r.done = true;
            r.t_done = r.t_submit;
            rt->reqs.emplace(id, r);
            *out_id = id;
            return AIDW_OK;
        }
        rt->reqs.emplace(id, r);
        rt->queue.push_back(id);
        ++rt->stats.submitted;
        *out_id = id;
    }
    rt->cv_work.notify_one();
    return AIDW_OK;
}

int aidw_poll(aidw_ctx *ctx, aidw_request id, int32_t *done)
{
    if (!ctx || !done)
        return AIDW_ERR_INVALID_ARG;
    *done = 0;
    ServingRuntime *rt = ctx_serving(ctx);
    if (!rt)
        return AIDW_ERR_NOT_FOUND;
    std::lock_guard<std::mutex> g(rt->mu);
    auto it = rt->reqs.find(id);
    if (it == rt->reqs.end())
        return AIDW_ERR_NOT_FOUND;
    if (!it->second.done)
        return AIDW_PENDING;
    *done = 1;
    return it->second.status;
}

int aidw_wait(aidw_ctx *ctx, aidw_request id, int64_t timeout_us)
{
    if (!ctx)
        return AIDW_ERR_INVALID_ARG;
    ServingRuntime *rt = ctx_serving(ctx);
    if (!rt)
        return AIDW_ERR_NOT_FOUND;
    std::unique_lock<std::mutex> g(rt->mu);
    auto it = rt->reqs.find(id);
    if (it == rt->reqs.end())
        return AIDW_ERR_NOT_FOUND;
    Request *r = &it->second;
    auto pred = [&] { return r->done; };
    if (timeout_us < 0)
        rt->cv_done.wait(g, pred);
    else if (!rt->cv_done.wait_for(g, std::chrono::microseconds(timeout_us), pred))
        return AIDW_ERR_TIMEOUT;
    return r->status;
}

int aidw_request_latency_us(aidw_ctx *ctx, aidw_request id, double *latency_us)
{
    if (!ctx || !latency_us)
        return AIDW_ERR_INVALID_ARG;
    ServingRuntime *rt = ctx_serving(ctx);
    if (!rt)
        return AIDW_ERR_NOT_FOUND;
    std::lock_guard<std::mutex> g(rt->mu);
    auto it = rt->reqs.find(id);
    if (it == rt->reqs.end())
        return AIDW_ERR_NOT_FOUND;
    if (!it->second.done)
        return AIDW_PENDING;
    *latency_us =
        std::chrono::duration<double, std::micro>(it->second.t_done - it->second.t_submit)
            .count();
    return AIDW_OK;
}

int aidw_release_request(aidw_ctx *ctx, aidw_request id)
{
    if (!ctx)
        return AIDW_ERR_INVALID_ARG;
    ServingRuntime *rt = ctx_serving(ctx);
    if (!rt)
        return AIDW_ERR_NOT_FOUND;
    std::lock_guard<std::mutex> g(rt->mu);
    auto it = rt->reqs.find(id);
    if (it == rt->reqs.end())
        return AIDW_ERR_NOT_FOUND;
    if (!it->second.done)
        return AIDW_PENDING;
    rt->reqs.erase(it);
    return AIDW_OK;
}

int aidw_serving_get_stats(aidw_ctx *ctx, aidw_serving_stats *out)
{
    if (!ctx || !out)
        return AIDW_ERR_INVALID_ARG;
    ServingRuntime *rt = ctx_serving(ctx);
    if (!rt) {
        std::memset(out, 0, sizeof(*out));
        return AIDW_OK;
    }
    std::lock_guard<std::mutex> g(rt->mu);
    *out = rt->stats;
    out->queued = static_cast<int64_t>(rt->queue.size());
    out->in_flight_bytes = rt->in_flight;
    out->budget_bytes = rt->budget;
    return AIDW_OK;
}

}  // extern "C"
