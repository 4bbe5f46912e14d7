// Batched AIDW: many independent (dataset, query set) items in one persistent work-queue
// kernel, launched through a captured CUDA graph.
//
// Every item is cut into units that depend only on the item itself (never on what else is in
// the batch), so an item's result is bit-identical whether it runs alone or in any mix:
//   KNN     (item, query block, split)  phase-1 scan of one data split       (no wait)
//   SELECT  (item, query block)         merge + Eq. 2-6 for 512 queries      waits for the
//                                                                            block's KNN splits
//   WEIGHTS (item, query block, split)  phase-2 scan of one data split       waits for all of
//                                                                            the item's SELECTs
//   FINAL   (item, query block)         split merge + Eq. 1 ratio            waits for the
//                                                                            block's WEIGHTS
// The work list holds all KNN units, then all SELECT, WEIGHTS and FINAL units, each phase in
// decreasing item size; CTAs take units in list order from one atomic counter. A unit only
// waits on units earlier in the list, which running CTAs have already taken and never block
// on later ones, so the waits end; each wait is still bounded and raises the error word if it
// runs out. Producers publish with a fence and an atomic add; consumers read counters with
// acquire loads and results with L2 loads.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "aidw_runtime.h"
#include "f32_device.cuh"

namespace aidw {

namespace {

using namespace f32dev;

enum UnitType : int32_t { kUnitKnn = 0, kUnitSelect = 1, kUnitWeights = 2, kUnitFinal = 3 };

// Data-split lengths of the batched plan (points). A phase-1 split restarts the neighbour lists,
// so phase-1 splits are longer.
constexpr int64_t kBatchKnnSplit = 262144;
constexpr int64_t kBatchWSplit = 65536;
constexpr uint32_t kMaxWaitPolls = 1u << 26;  // x >= 256 ns sleep: tens of seconds at most

struct BatchItemDev {
    DatasetDev ds;
    const float *qx, *qy;
    float *out, *out_alpha;
    int64_t m;
    int32_t k, kp;
    double r_exp;
    AlphaMap am;
    PassPlan knn, w;
    float *part_d2;
    QParamF32 *qparam;
    float *part_sum;
    uint32_t *cnt_knn;  // [knn.qblocks] finished phase-1 splits per query block
    uint32_t *cnt_sel;  // [1] finished SELECT units
    uint32_t *cnt_w;    // [w.qblocks] finished phase-2 splits per query block
};

struct WorkUnit {
    int32_t item, qblock, split, type;
};

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Thread 0 waits (bounded) until *p >= target; the verdict is shared through `flag`.
__device__ __forceinline__ bool cta_wait_count(const uint32_t *p, uint32_t target, int *flag)
{
    if (threadIdx.x == 0) {
        bool ok = false;
        for (uint32_t i = 0; i < kMaxWaitPolls; ++i) {
            if (ld_acquire(p) >= target) {
                ok = true;
                break;
            }
            __nanosleep(256);
        }
        *flag = ok ? 1 : 0;
    }
    __syncthreads();
    const bool ok = *flag != 0;
    __syncthreads();
    return ok;
}

// Every thread's results are made visible at GPU scope before thread 0 counts the unit done.
__device__ __forceinline__ void cta_publish(uint32_t *counter)
{
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0)
        atomicAdd(counter, 1u);
}

__global__ void __launch_bounds__(kThreads, 4)
f32_batch_kernel(const BatchItemDev *__restrict__ items, const WorkUnit *__restrict__ units,
                 int n_units, uint32_t *next, int *err)
{
    __shared__ __align__(128) float4 ktile[2][kTileF32Knn];
    __shared__ __align__(128) float4 txy[2][kTileF32W];
    __shared__ __align__(128) float2 tz[2][kTileF32W];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int s_unit, s_flag;
    init_tile_barriers(bar);
    TileSeq ts{bar, 0u};
    const int tid = threadIdx.x;

    for (;;) {
        if (tid == 0)
            s_unit = static_cast<int>(atomicAdd(next, 1u));
        __syncthreads();
        const int u = s_unit;
        __syncthreads();
        if (u >= n_units)
            break;
        const WorkUnit wu = units[u];
        const BatchItemDev &it = items[wu.item];
        bool ok = true;
        if (wu.type == kUnitKnn) {
            const int64_t qbase = static_cast<int64_t>(wu.qblock) * it.knn.q_per_block;
            const int64_t p0 = static_cast<int64_t>(wu.split) * it.knn.split_len;
            const int64_t p1 = min(p0 + it.knn.split_len, it.ds.n_pad);
            switch (it.kp) {
            case 8:
                ok = knn_unit<8, 4, false>(it.ds, it.m, qbase, p0, p1, it.qx, it.qy, it.k,
                                           wu.split, it.part_d2, nullptr, err, ktile, ts,
                                           nullptr);
                break;
            case 12:
                ok = knn_unit<12, 4, false>(it.ds, it.m, qbase, p0, p1, it.qx, it.qy, it.k,
                                            wu.split, it.part_d2, nullptr, err, ktile, ts,
                                            nullptr);
                break;
            case 16:
                ok = knn_unit<16, 4, false>(it.ds, it.m, qbase, p0, p1, it.qx, it.qy, it.k,
                                            wu.split, it.part_d2, nullptr, err, ktile, ts,
                                            nullptr);
                break;
            default:
                ok = knn_unit<32, 2, false>(it.ds, it.m, qbase, p0, p1, it.qx, it.qy, it.k,
                                            wu.split, it.part_d2, nullptr, err, ktile, ts,
                                            nullptr);
                break;
            }
            if (ok)
                cta_publish(&it.cnt_knn[wu.qblock]);
        } else if (wu.type == kUnitSelect) {
            ok = cta_wait_count(&it.cnt_knn[wu.qblock], it.knn.splits, &s_flag);
            if (ok) {
                const int64_t qbase = static_cast<int64_t>(wu.qblock) * it.knn.q_per_block;
                const int64_t qend = min(qbase + it.knn.q_per_block, it.m);
                for (int64_t q = qbase + tid; q < qend; q += kThreads)
                    select_query(q, it.m, it.knn.splits, it.k, it.r_exp, it.am, it.part_d2,
                                 nullptr, it.qparam, it.out_alpha, nullptr);
                cta_publish(it.cnt_sel);
            }
        } else if (wu.type == kUnitWeights) {
            ok = cta_wait_count(it.cnt_sel, it.knn.qblocks, &s_flag);
            if (ok) {
                const int64_t qbase = static_cast<int64_t>(wu.qblock) * it.w.q_per_block;
                const int64_t p0 = static_cast<int64_t>(wu.split) * it.w.split_len;
                const int64_t p1 = min(p0 + it.w.split_len, it.ds.n_pad);
                ok = weights_unit<kQW32>(it.ds, it.m, qbase, p0, p1, it.qx, it.qy, it.qparam,
                                         wu.split, it.part_sum, err, txy, tz, ts);
                if (ok)
                    cta_publish(&it.cnt_w[wu.qblock]);
            }
        } else {
            ok = cta_wait_count(&it.cnt_w[wu.qblock], it.w.splits, &s_flag);
            if (ok) {
                const int64_t qbase = static_cast<int64_t>(wu.qblock) * it.w.q_per_block;
                const int64_t qend = min(qbase + it.w.q_per_block, it.m);
                for (int64_t q = qbase + tid; q < qend; q += kThreads)
                    it.out[q] = finalize_query(q, it.m, it.w.splits, it.part_sum);
            }
        }
        if (!ok) {
            if (tid == 0)
                atomicOr(err, kErrTimeout);
            break;
        }
    }
}

inline size_t align256(size_t b)
{
    return (b + 255) & ~static_cast<size_t>(255);
}

PassPlan batch_pass(int64_t m, int64_t n_pad, int qpb, int64_t target)
{
    PassPlan pp{};
    pp.q_per_block = qpb;
    pp.qblocks = static_cast<int>((m + qpb - 1) / qpb);
    const int64_t G = n_pad / kPadPoints;
    int64_t S = (n_pad + target - 1) / target;
    S = std::max<int64_t>(1, std::min<int64_t>(S, std::min<int64_t>(G, kMaxSplits)));
    const int64_t per = (G + S - 1) / S;
    pp.splits = static_cast<int>((G + per - 1) / per);
    pp.split_len = per * kPadPoints;
    return pp;
}

int batch_grid(int sm_count)
{
    static int per_sm = 0;
    if (!per_sm) {
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f32_batch_kernel, kThreads, 0);
        per_sm = n > 0 ? n : 1;
    }
    return per_sm * sm_count;
}

}  // namespace

size_t batch_item_bytes(int64_t n_pad, int64_t m, int k)
{
    const int kp = kp_for(k);
    const PassPlan pk = batch_pass(m, n_pad, kThreads * (kp <= 16 ? 4 : 2), kBatchKnnSplit);
    const PassPlan pw = batch_pass(m, n_pad, kThreads * kQW32, kBatchWSplit);
    const size_t mm = static_cast<size_t>(m);
    return align256(pk.splits * static_cast<size_t>(k) * mm * sizeof(float)) +
           align256(mm * sizeof(QParamF32)) + align256(pw.splits * 4 * mm * sizeof(float)) +
           sizeof(uint32_t) * (pk.qblocks + 1 + pw.qblocks) + sizeof(BatchItemDev) +
           sizeof(WorkUnit) * (pk.qblocks * (pk.splits + 1) + pw.qblocks * (pw.splits + 1));
}

// Validates the items and builds the device tables of a batch in library memory.
int batch_build(aidw_ctx *ctx, const aidw_batch_item *items, int32_t count, cudaStream_t st,
                BatchState *bs)
{
    if (count < 0 || (count > 0 && !items))
        return AIDW_ERR_INVALID_ARG;
    const int device = ctx_device(ctx);
    std::vector<BatchItemDev> h(count);
    std::vector<size_t> scratch_off(count), cnt_off(count);
    size_t scratch_total = 0, cnt_total = sizeof(uint32_t);  // slot 0: the work counter
    for (int32_t i = 0; i < count; ++i) {
        const aidw_batch_item &b = items[i];
        DatasetDev dev;
        double r_exp;
        if (!dataset_lookup(ctx, b.ds, &dev, &r_exp))
            return AIDW_ERR_NOT_FOUND;
        int rc = validate_params(&b.params, dev.n);
        if (rc)
            return rc;
        if (b.params.precision != AIDW_F32C || b.m < 0 || b.m > (int64_t(1) << 31))
            return AIDW_ERR_INVALID_ARG;
        if (b.m > 0 && (pointer_kind(b.qx, device) != 1 || pointer_kind(b.qy, device) != 1 ||
                        pointer_kind(b.out, device) != 1 ||
                        (b.out_alpha && pointer_kind(b.out_alpha, device) != 1)))
            return AIDW_ERR_INVALID_ARG;
        BatchItemDev &d = h[i];
        std::memset(&d, 0, sizeof(d));
        d.ds = dev;
        d.qx = b.qx;
        d.qy = b.qy;
        d.out = b.out;
        d.out_alpha = b.out_alpha;
        d.m = b.m;
        d.k = b.params.k;
        d.kp = kp_for(b.params.k);
        d.r_exp = r_exp;
        d.am = alpha_map(b.params);
        const int qk = kThreads * (d.kp <= 16 ? 4 : 2);
        d.knn = batch_pass(b.m, dev.n_pad, qk, kBatchKnnSplit);
        d.w = batch_pass(b.m, dev.n_pad, kThreads * kQW32, kBatchWSplit);
        const size_t m = static_cast<size_t>(b.m);
        scratch_off[i] = scratch_total;
        scratch_total += align256(d.knn.splits * static_cast<size_t>(d.k) * m * sizeof(float)) +
                         align256(m * sizeof(QParamF32)) +
                         align256(d.w.splits * 4 * m * sizeof(float));
        cnt_off[i] = cnt_total;
        cnt_total += sizeof(uint32_t) * (d.knn.qblocks + 1 + d.w.qblocks);
    }
    // Units: phases in order, items in decreasing size within each phase.
    std::vector<int32_t> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        return static_cast<double>(h[a].m) * h[a].ds.n_pad >
               static_cast<double>(h[b].m) * h[b].ds.n_pad;
    });
    std::vector<WorkUnit> u;
    for (int32_t i : order)
        for (int qb = 0; qb < h[i].knn.qblocks; ++qb)
            for (int s = 0; s < h[i].knn.splits; ++s)
                u.push_back({i, qb, s, kUnitKnn});
    for (int32_t i : order)
        for (int qb = 0; qb < h[i].knn.qblocks; ++qb)
            u.push_back({i, qb, 0, kUnitSelect});
    for (int32_t i : order)
        for (int qb = 0; qb < h[i].w.qblocks; ++qb)
            for (int s = 0; s < h[i].w.splits; ++s)
                u.push_back({i, qb, s, kUnitWeights});
    for (int32_t i : order)
        for (int qb = 0; qb < h[i].w.qblocks; ++qb)
            u.push_back({i, qb, 0, kUnitFinal});

    const size_t b_items = align256(sizeof(BatchItemDev) * std::max<int32_t>(count, 1));
    const size_t b_units = align256(sizeof(WorkUnit) * std::max<size_t>(u.size(), 1));
    const size_t b_cnt = align256(cnt_total);
    bs->bytes = b_items + b_units + b_cnt + scratch_total;
    int rc = ctx_alloc(ctx, bs->bytes, st, &bs->block);
    if (rc)
        return rc;
    char *base = static_cast<char *>(bs->block);
    bs->d_items = base;
    bs->d_units = base + b_items;
    bs->d_counters = reinterpret_cast<uint32_t *>(base + b_items + b_units);
    bs->counter_bytes = cnt_total;
    char *scratch = base + b_items + b_units + b_cnt;
    for (int32_t i = 0; i < count; ++i) {
        BatchItemDev &d = h[i];
        const size_t m = static_cast<size_t>(d.m);
        char *p = scratch + scratch_off[i];
        d.part_d2 = reinterpret_cast<float *>(p);
        p += align256(d.knn.splits * static_cast<size_t>(d.k) * m * sizeof(float));
        d.qparam = reinterpret_cast<QParamF32 *>(p);
        p += align256(m * sizeof(QParamF32));
        d.part_sum = reinterpret_cast<float *>(p);
        uint32_t *c = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(bs->d_counters) +
                                                   cnt_off[i]);
        d.cnt_knn = c;
        d.cnt_sel = c + d.knn.qblocks;
        d.cnt_w = c + d.knn.qblocks + 1;
    }
    bs->n_units = static_cast<int>(u.size());
    bs->grid = batch_grid(ctx_sm_count(ctx));
    bool ok = true;
    if (count > 0)
        ok &= cudaMemcpyAsync(bs->d_items, h.data(), sizeof(BatchItemDev) * count,
                              cudaMemcpyHostToDevice, st) == cudaSuccess;
    if (!u.empty())
        ok &= cudaMemcpyAsync(bs->d_units, u.data(), sizeof(WorkUnit) * u.size(),
                              cudaMemcpyHostToDevice, st) == cudaSuccess;
    // Pageable sources: the copies have completed when cudaMemcpyAsync returns for the host
    // side, but the device side is ordered on `st` before the kernel.
    if (!ok) {
        ctx_free(ctx, bs->block, bs->bytes, st);
        bs->block = nullptr;
        return AIDW_ERR_CUDA;
    }
    return AIDW_OK;
}

// Stream-ordered: zero the counters, run the persistent kernel.
int batch_enqueue(aidw_ctx *ctx, const BatchState &bs, cudaStream_t st)
{
    if (bs.n_units == 0)
        return AIDW_OK;
    if (cudaMemsetAsync(bs.d_counters, 0, bs.counter_bytes, st) != cudaSuccess)
        return AIDW_ERR_CUDA;
    f32_batch_kernel<<<bs.grid, kThreads, 0, st>>>(
        static_cast<const BatchItemDev *>(bs.d_items), static_cast<const WorkUnit *>(bs.d_units),
        bs.n_units, bs.d_counters, ctx_err_word(ctx));
    return cudaGetLastError() == cudaSuccess ? AIDW_OK : AIDW_ERR_CUDA;
}

void batch_release(aidw_ctx *ctx, BatchState *bs, cudaStream_t st)
{
    if (bs->graph)
        cudaGraphExecDestroy(bs->graph);
    bs->graph = nullptr;
    ctx_free(ctx, bs->block, bs->bytes, st);
    bs->block = nullptr;
}

}  // namespace aidw

using namespace aidw;

struct aidw_batch {
    BatchState st;
};

extern "C" {

int aidw_interpolate_batch(aidw_ctx *ctx, const aidw_batch_item *items, int32_t count,
                           void *stream)
{
    if (!ctx)
        return AIDW_ERR_INVALID_ARG;
    if (cudaSetDevice(ctx_device(ctx)) != cudaSuccess)
        return AIDW_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    BatchState bs;
    int rc = batch_build(ctx, items, count, st, &bs);
    if (rc)
        return rc;
    rc = batch_enqueue(ctx, bs, st);
    batch_release(ctx, &bs, st);
    return rc;
}

int aidw_batch_create(aidw_ctx *ctx, const aidw_batch_item *items, int32_t count,
                      aidw_batch **out)
{
    if (!ctx || !out)
        return AIDW_ERR_INVALID_ARG;
    *out = nullptr;
    if (cudaSetDevice(ctx_device(ctx)) != cudaSuccess)
        return AIDW_ERR_CUDA;
    cudaStream_t cap;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess)
        return AIDW_ERR_CUDA;
    aidw_batch *b = new aidw_batch();
    int rc = batch_build(ctx, items, count, cap, &b->st);
    if (rc == AIDW_OK && cudaStreamSynchronize(cap) != cudaSuccess)
        rc = AIDW_ERR_CUDA;
    if (rc == AIDW_OK) {
        // Capture the counter reset and the persistent kernel as one graph.
        cudaGraph_t g = nullptr;
        bool ok = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            const int erc = batch_enqueue(ctx, b->st, cap);
            ok = cudaStreamEndCapture(cap, &g) == cudaSuccess && erc == AIDW_OK;
        }
        ok = ok && cudaGraphInstantiate(&b->st.graph, g, 0) == cudaSuccess;
        if (g)
            cudaGraphDestroy(g);
        if (!ok) {
            cudaGetLastError();
            rc = AIDW_ERR_CUDA;
        }
    }
    if (rc != AIDW_OK) {
        if (b->st.block)
            batch_release(ctx, &b->st, cap);
        cudaStreamSynchronize(cap);
        cudaStreamDestroy(cap);
        delete b;
        return rc;
    }
    cudaStreamDestroy(cap);
    *out = b;
    return AIDW_OK;
}

int aidw_batch_launch(aidw_ctx *ctx, aidw_batch *b, void *stream)
{
    if (!ctx || !b)
        return AIDW_ERR_INVALID_ARG;
    if (b->st.n_units == 0)
        return AIDW_OK;
    return cudaGraphLaunch(b->st.graph, static_cast<cudaStream_t>(stream)) == cudaSuccess
               ? AIDW_OK
               : AIDW_ERR_CUDA;
}

int aidw_batch_destroy(aidw_ctx *ctx, aidw_batch *b)
{
    if (!ctx || !b)
        return AIDW_ERR_INVALID_ARG;
    cudaSetDevice(ctx_device(ctx));
    cudaDeviceSynchronize();
    batch_release(ctx, &b->st, 0);
    cudaStreamSynchronize(0);
    delete b;
    return AIDW_OK;
}

}  // extern "C"
