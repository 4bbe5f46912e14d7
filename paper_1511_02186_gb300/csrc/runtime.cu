// Batching and serving layer over the one-shot interpolation path.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "aidw_internal.cuh"
#include "aidw_runtime.h"

namespace aidw {

struct Request {
    int64_t ds;
    const void *qx, *qy;
    int64_t m;
    aidw_params p;
    void *out;
    float *out_alpha;
    int32_t *out_knn;
    int status = AIDW_PENDING;
    bool done = false;
    std::chrono::steady_clock::time_point t_submit, t_done;
};

struct ServingRuntime {
    aidw_ctx *ctx = nullptr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<int64_t> queue;
    std::unordered_map<int64_t, Request> reqs;
    int64_t next_id = 1;
    size_t max_queue = 4096;
    bool stop = false;
    std::thread worker;
    cudaStream_t stream = nullptr;
};

namespace {

void worker_main(ServingRuntime *rt)
{
    cudaSetDevice(ctx_device(rt->ctx));
    for (;;) {
        int64_t id;
        Request r;
        {
            std::unique_lock<std::mutex> g(rt->mu);
            rt->cv_work.wait(g, [&] { return rt->stop || !rt->queue.empty(); });
            if (rt->queue.empty())
                return;
            id = rt->queue.front();
            rt->queue.pop_front();
            r = rt->reqs[id];
        }
        int rc = interpolate_impl(rt->ctx, r.ds, r.qx, r.qy, r.m, &r.p, r.out, r.out_alpha,
                                  r.out_knn, rt->stream, 0, 0);
        if (rc == AIDW_OK && cudaStreamSynchronize(rt->stream) != cudaSuccess)
            rc = AIDW_ERR_CUDA;
        {
            std::lock_guard<std::mutex> g(rt->mu);
            Request &q = rt->reqs[id];
            q.status = rc;
            q.done = true;
            q.t_done = std::chrono::steady_clock::now();
        }
        rt->cv_done.notify_all();
    }
}

ServingRuntime *ensure_serving(aidw_ctx *ctx)
{
    std::lock_guard<std::mutex> g(ctx_mutex(ctx));
    ServingRuntime *&rt = ctx_serving(ctx);
    if (!rt) {
        rt = new ServingRuntime();
        rt->ctx = ctx;
        cudaSetDevice(ctx_device(ctx));
        cudaStreamCreateWithFlags(&rt->stream, cudaStreamNonBlocking);
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
    if (rt->stream)
        cudaStreamDestroy(rt->stream);
    delete rt;
}

}  // namespace aidw

using namespace aidw;

extern "C" {

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
    if (m < 0 || (m > 0 && (!qx || !qy || !out)))
        return AIDW_ERR_INVALID_ARG;
    ServingRuntime *rt = ensure_serving(ctx);
    {
        std::lock_guard<std::mutex> g(rt->mu);
        if (rt->queue.size() >= rt->max_queue)
            return AIDW_ERR_AGAIN;
        const int64_t id = rt->next_id++;
        Request r;
        r.ds = ds;
        r.qx = qx;
        r.qy = qy;
        r.m = m;
        r.p = *p;
        r.out = out;
        r.out_alpha = out_alpha;
        r.out_knn = out_knn;
        r.t_submit = std::chrono::steady_clock::now();
        rt->reqs.emplace(id, r);
        rt->queue.push_back(id);
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
    auto pred = [&] { return rt->reqs[id].done; };
    if (timeout_us < 0)
        rt->cv_done.wait(g, pred);
    else if (!rt->cv_done.wait_for(g, std::chrono::microseconds(timeout_us), pred))
        return AIDW_ERR_TIMEOUT;
    return rt->reqs[id].status;
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
    *latency_us = std::chrono::duration<double, std::micro>(it->second.t_done -
                                                            it->second.t_submit)
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

}  // extern "C"
