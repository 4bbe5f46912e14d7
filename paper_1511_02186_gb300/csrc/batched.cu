// Batched AIDW: many independent (dataset, query set) items in one persistent work-queue
// kernel, launched through a captured CUDA graph.
//
// Every item is cut into units that depend only on the item itself (never on what else is in
// the batch), so an item's result is bit-identical whether it runs alone or in any mix:
//   KNN     (item, query block)         pruned phase-1 scan of Z-ordered      (no wait)
//                                       queries (nearest data tiles first)
//   SELECT  (item, query block)         merge + Eq. 2-6 for the block        waits for the
//                                                                            block's KNN splits
//   WEIGHTS (item, query block, split)  phase-2 scan of one data split       waits for all of
//                                                                            the item's SELECTs
//   FINAL   (item, query block)         split merge + Eq. 1 ratio            waits for the
//                                                                            block's WEIGHTS
// Before the persistent kernel, the queries of all items are put in Z-order item by item (Morton
// keys over each item's dataset box, a stable radix sort by key, then a stable sort by item) so
// that each KNN unit's block is compact; results go back to the caller's order.
// The work list holds all KNN units, then all SELECT, WEIGHTS and FINAL units, each phase in
// decreasing item size (or, with the shape's interleaved unit order, each item's SELECT and
// WEIGHTS units placed after the KNN units of items further down, so that both phases share
// the SMs, and the FINAL units last); CTAs take units in list order from one atomic counter.
// A unit only waits on units earlier in the list, which running CTAs have already taken and
// never block on later ones, so the waits end; each wait is still bounded and raises the error
// word if it runs out. Producers publish with a fence and an atomic add; consumers read counters with
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

// Data-split length of the batched phase-1 plan (points) for datasets too large to prune; a
// phase-1 split restarts the neighbour lists, so these splits are long. The phase-2 split
// length is a tuning field (aidw_tune_config.split_points).
constexpr int64_t kBatchKnnSplit = 262144;

struct BatchItemDev {
    DatasetDev ds;
    const float *qx, *qy;
    float *out, *out_alpha;
    int64_t m;
    int32_t k, kp, kq;  // kq: queries per thread of the pruned phase-1 units
    double r_exp;
    AlphaMap am;
    PassPlan knn, w;
    float *part_d2;
    QParamF32 *qparam;
    float *part_sum;
    const float *sqx, *sqy;  // the item's queries in Z-order
    const uint32_t *perm;    // Z-order position -> caller's query index
    int64_t qoff;            // offset of the item in the batch-wide query arrays
    int32_t ntiles, ntiles_p2;
    uint32_t *cnt_knn;  // [knn.qblocks] finished phase-1 units per query block
    uint32_t *cnt_sel;  // [1] finished SELECT units
    uint32_t *cnt_w;    // [w.qblocks] finished phase-2 splits per query block
};

struct WorkUnit {
    int32_t item, qblock, split, type;
};

// Every thread's results are made visible at GPU scope before thread 0 counts the unit done.
__device__ __forceinline__ void cta_publish(uint32_t *counter)
{
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0)
        atomicAdd(counter, 1u);
}

// QW: phase-2 queries per thread; tw: phase-2 tile points (256 or 512).
template <int QW>
__global__ void __launch_bounds__(kThreads, 4)
f32_batch_kernel(const BatchItemDev *__restrict__ items, const WorkUnit *__restrict__ units,
                 int n_units, uint32_t *next, int *err, int tw)
{
    extern __shared__ unsigned long long order[];  // tile order of a KNN unit
    __shared__ CullShared cs;
    // Phase-1 and phase-2 units take turns on the same coordinate tile buffers.
    static_assert(kTileF32Knn == kTileF32W, "shared tile buffers");
    __shared__ __align__(128) float4 txy[2][kTileF32W];
    float4(*ktile)[kTileF32Knn] = txy;
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
        if (wu.type == kUnitKnn && it.ntiles_p2 == 0) {
            // Dataset too large for the shared-memory tile order: split scan.
            const int64_t qbase = static_cast<int64_t>(wu.qblock) * it.knn.q_per_block;
            const int64_t p0 = static_cast<int64_t>(wu.split) * it.knn.split_len;
            const int64_t p1 = min(p0 + it.knn.split_len, it.ds.n_pad);
            switch (it.kp) {
            case 8:
                ok = knn_unit<8, 4, false>(it.ds, it.m, qbase, p0, p1, it.sqx, it.sqy, it.k,
                                           wu.split, it.part_d2, nullptr, err, ktile, ts,
                                           nullptr);
                break;
            case 12:
                ok = knn_unit<12, 4, false>(it.ds, it.m, qbase, p0, p1, it.sqx, it.sqy, it.k,
                                            wu.split, it.part_d2, nullptr, err, ktile, ts,
                                            nullptr);
                break;
            case 16:
                ok = knn_unit<16, 4, false>(it.ds, it.m, qbase, p0, p1, it.sqx, it.sqy, it.k,
                                            wu.split, it.part_d2, nullptr, err, ktile, ts,
                                            nullptr);
                break;
            default:
                ok = knn_unit<32, 2, false>(it.ds, it.m, qbase, p0, p1, it.sqx, it.sqy, it.k,
                                            wu.split, it.part_d2, nullptr, err, ktile, ts,
                                            nullptr);
                break;
            }
            if (ok)
                cta_publish(&it.cnt_knn[wu.qblock]);
        } else if (wu.type == kUnitKnn) {
            const int64_t qbase = static_cast<int64_t>(wu.qblock) * it.knn.q_per_block;
#define AIDW_CULL_UNIT(KP, Q)                                                                  \
    ok = knn_cull_unit<KP, Q, false>(it.ds, it.m, qbase, it.ntiles, it.ntiles_p2, it.sqx, it.sqy, \
                                     it.k, it.part_d2, nullptr, err, ktile, ts, order, nullptr,  \
                                     cs)
            const bool q2 = it.kq == 2;
            switch (it.kp) {
            case 8:
                if (q2)
                    AIDW_CULL_UNIT(8, 2);
                else
                    AIDW_CULL_UNIT(8, 4);
                break;
            case 12:
                if (q2)
                    AIDW_CULL_UNIT(12, 2);
                else
                    AIDW_CULL_UNIT(12, 4);
                break;
            case 16:
                if (q2)
                    AIDW_CULL_UNIT(16, 2);
                else
                    AIDW_CULL_UNIT(16, 4);
                break;
            default:
                AIDW_CULL_UNIT(32, 2);
                break;
            }
#undef AIDW_CULL_UNIT
            if (ok)
                cta_publish(&it.cnt_knn[wu.qblock]);
        } else if (wu.type == kUnitSelect) {
            ok = cta_wait_count(&it.cnt_knn[wu.qblock], it.knn.splits, &s_flag);
            if (ok) {
                const int64_t qbase = static_cast<int64_t>(wu.qblock) * it.knn.q_per_block;
                const int64_t qend = min(qbase + it.knn.q_per_block, it.m);
                for (int64_t q = qbase + tid; q < qend; q += kThreads)
                    select_query(q, it.m, it.knn.splits, it.k, it.r_exp, it.am, it.part_d2,
                                 nullptr, it.qparam, it.out_alpha, nullptr, it.perm);
                cta_publish(it.cnt_sel);
            }
        } else if (wu.type == kUnitWeights) {
            ok = cta_wait_count(it.cnt_sel, it.knn.qblocks, &s_flag);
            if (ok) {
                const int64_t qbase = static_cast<int64_t>(wu.qblock) * it.w.q_per_block;
                const int64_t p0 = static_cast<int64_t>(wu.split) * it.w.split_len;
                const int64_t p1 = min(p0 + it.w.split_len, it.ds.n_pad);
                if (tw == 256)
                    ok = weights_unit<QW, 256>(
                        it.ds, it.m, qbase, p0, p1, it.sqx, it.sqy, it.qparam, wu.split,
                        it.part_sum, err, reinterpret_cast<float4(*)[256]>(&txy[0][0]),
                        reinterpret_cast<float2(*)[256]>(&tz[0][0]), ts);
                else
                    ok = weights_unit<QW, kTileF32W>(it.ds, it.m, qbase, p0, p1, it.sqx, it.sqy,
                                                     it.qparam, wu.split, it.part_sum, err, txy,
                                                     tz, ts);
                if (ok)
                    cta_publish(&it.cnt_w[wu.qblock]);
            }
        } else {
            ok = cta_wait_count(&it.cnt_w[wu.qblock], it.w.splits, &s_flag);
            if (ok) {
                const int64_t qbase = static_cast<int64_t>(wu.qblock) * it.w.q_per_block;
                const int64_t qend = min(qbase + it.w.q_per_block, it.m);
                for (int64_t q = qbase + tid; q < qend; q += kThreads)
                    it.out[it.perm[q]] = finalize_query(q, it.m, it.w.splits, it.part_sum);
            }
        }
        if (!ok) {
            if (tid == 0)
                atomicOr(err, kErrTimeout);
            break;
        }
    }
}

// Batch-wide query ordering, step 1: Morton key of every query over its item's dataset box;
// values are batch-wide positions, and the item of every position is recorded.
__global__ void batch_keys_kernel(const BatchItemDev *__restrict__ items, uint32_t *keys,
                                  uint32_t *vals, uint32_t *item_of)
{
    const BatchItemDev &it = items[blockIdx.y];
    const float4 box = *it.ds.box;
    for (int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < it.m;
         q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t g = it.qoff + q;
        keys[g] = morton_of(it.qx[q], it.qy[q], box);
        vals[g] = static_cast<uint32_t>(g);
        item_of[g] = blockIdx.y;
    }
}

// Step 2 (after the sort by key): the item of each sorted entry, as the key of a second,
// stable sort that groups the items while keeping each item's Z-order.
__global__ void batch_item_keys_kernel(const uint32_t *__restrict__ vals,
                                       const uint32_t *__restrict__ item_of, int64_t total,
                                       uint32_t *keys)
{
    for (int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; j < total;
         j += static_cast<int64_t>(gridDim.x) * blockDim.x)
        keys[j] = item_of[vals[j]];
}

// Step 3: ordered coordinates and the caller's index of every ordered query.
__global__ void batch_gather_kernel(const BatchItemDev *__restrict__ items,
                                    const uint32_t *__restrict__ vals,
                                    const uint32_t *__restrict__ item_of, int64_t total,
                                    float *sqx, float *sqy, uint32_t *perm)
{
    for (int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; j < total;
         j += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const uint32_t g = vals[j];
        const BatchItemDev &it = items[item_of[g]];
        const int64_t q = static_cast<int64_t>(g) - it.qoff;
        sqx[j] = it.qx[q];
        sqy[j] = it.qy[q];
        perm[j] = static_cast<uint32_t>(q);
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

using BatchKernel = void (*)(const BatchItemDev *, const WorkUnit *, int, uint32_t *, int *,
                            int);

BatchKernel batch_kernel_for(int qw)
{
    return qw == 2 ? f32_batch_kernel<2> : (qw == 8 ? f32_batch_kernel<8> : f32_batch_kernel<4>);
}

// Persistent grid: CTAs per SM as occupancy allows, or fewer if the shape asks for it.
int batch_grid(int sm_count, size_t dyn, int qw, int ctas_per_sm)
{
    const BatchKernel fn = batch_kernel_for(qw);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(dyn));
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, kThreads, dyn);
    n = n > 0 ? n : 1;
    if (ctas_per_sm > 0 && ctas_per_sm < n)
        n = ctas_per_sm;
    return n * sm_count;
}

}  // namespace

// Phase-1 plan of a batch item: one pruned unit per query block when the dataset's tile order
// fits in shared memory and the item has enough queries, else split scans. A pruned unit visits
// the tiles near its block's queries; with few queries spread over the data that is most of
// the tiles, scanned by one CTA (m = 256 against 800,000 points: 19 ms as one pruned unit, 5 ms
// as split scans), so an item with fewer than kBatchCullMinQueries queries scans instead, its
// data cut into enough splits for about kBatchKnnUnits units in all. Above that the pruned
// units do several times less work than a scan of every pair, which a batch's throughput
// needs (the 256-dataset batch: 80.5 ms with the pruned units from 1,024 queries on, 83.5 ms
// from 4,096 on).
constexpr int64_t kBatchCullMinQueries = 1024;
constexpr int64_t kBatchKnnUnits = 128;

// Phase-2 plan of a batch item: data splits of at most split_points points, and, for an item
// with few queries, enough of them for about kBatchMinWeightUnits units of 256 queries, so
// that an item alone (a lightly loaded server's flight) still spreads over every SM (a request
// of 8,192 queries against 231,679 points with 65,536-point splits: 128 units for 608 resident
// CTAs; served in 5.3 ms, with the extra splits in 2.7 ms, the one-shot call 2.5 ms). The split
// length depends on the item's sizes and split_points only (not on the rest of the batch, nor
// on the arithmetic-neutral shape fields).
constexpr int64_t kBatchMinWeightUnits = 1024;

PassPlan batch_w_plan(int64_t m, int64_t n_pad, int qpb, int64_t split_points)
{
    const int64_t blocks256 = std::max<int64_t>(1, (m + 255) / 256);
    const int64_t want = (kBatchMinWeightUnits + blocks256 - 1) / blocks256;
    const int64_t target = std::max<int64_t>(kPadPoints, (n_pad + want - 1) / want);
    return batch_pass(m, n_pad, qpb, std::min<int64_t>(split_points, target));
}

PassPlan batch_knn_plan(int64_t m, int64_t n_pad, int kp, int kq, bool *cull)
{
    *cull = n_pad / kTileF32Knn <= kMaxCullTiles && m >= kBatchCullMinQueries;
    const int qk = kThreads * (*cull ? kq : (kp <= 16 ? 4 : 2));
    if (*cull)
        return batch_pass(m, n_pad, qk, n_pad);
    const int64_t qblocks = std::max<int64_t>(1, (m + qk - 1) / qk);
    const int64_t splits = std::max<int64_t>(1, kBatchKnnUnits / qblocks);
    const int64_t target = std::max<int64_t>(kPadPoints, (n_pad + splits - 1) / splits);
    return batch_pass(m, n_pad, qk, std::min<int64_t>(target, kBatchKnnSplit));
}

size_t batch_item_bytes(int64_t n_pad, int64_t m, int k, const aidw_tune_config &cfg)
{
    bool cull;
    const int kp = kp_for(k, cfg.knn_list);
    const PassPlan pk = batch_knn_plan(m, n_pad, kp, cull_queries_per_thread(kp,
                                       cfg.knn_queries_per_thread), &cull);
    const PassPlan pw = batch_w_plan(m, n_pad, kThreads * cfg.queries_per_thread,
                                     cfg.split_points);
    const size_t mm = static_cast<size_t>(m);
    return align256(pk.splits * static_cast<size_t>(k) * mm * sizeof(float)) +
           align256(mm * sizeof(QParamF32)) + align256(pw.splits * 4 * mm * sizeof(float)) +
           sizeof(uint32_t) * (pk.qblocks + 1 + pw.qblocks) + sizeof(BatchItemDev) +
           sizeof(WorkUnit) * (pk.qblocks * (pk.splits + 1) + pw.qblocks * (pw.splits + 1)) +
           mm * (6 * sizeof(uint32_t)) + radix_scratch_bytes(m);
}

// Validates the items and builds the device tables of a batch in library memory.
int batch_build(aidw_ctx *ctx, const aidw_batch_item *items, int32_t count, cudaStream_t st,
                BatchState *bs, const aidw_tune_config &cfg)
{
    if (!tune_valid(cfg))
        return AIDW_ERR_INVALID_ARG;
    if (count < 0 || count > 65535 || (count > 0 && !items))
        return AIDW_ERR_INVALID_ARG;
    const int device = ctx_device(ctx);
    std::vector<BatchItemDev> h(count);
    std::vector<size_t> scratch_off(count), cnt_off(count);
    size_t scratch_total = 0, cnt_total = sizeof(uint32_t);  // slot 0: the work counter
    int64_t total_q = 0, max_m = 0;
    int max_p2 = 0;
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
        d.kp = kp_for(b.params.k, cfg.knn_list);
        d.kq = cull_queries_per_thread(d.kp, cfg.knn_queries_per_thread);
        d.r_exp = r_exp;
        d.am = alpha_map(b.params);
        bool cull;
        d.knn = batch_knn_plan(b.m, dev.n_pad, d.kp, d.kq, &cull);
        d.w = batch_w_plan(b.m, dev.n_pad, kThreads * cfg.queries_per_thread, cfg.split_points);
        d.ntiles = static_cast<int32_t>(dev.n_pad / kTileF32Knn);
        int p2 = 1;
        while (p2 < d.ntiles)
            p2 <<= 1;
        d.ntiles_p2 = cull ? p2 : 0;
        if (cull && b.m > 0)
            max_p2 = std::max(max_p2, p2);
        d.qoff = total_q;
        total_q += b.m;
        max_m = std::max<int64_t>(max_m, b.m);
        const size_t m = static_cast<size_t>(b.m);
        scratch_off[i] = scratch_total;
        scratch_total += align256(d.knn.splits * static_cast<size_t>(d.k) * m * sizeof(float)) +
                         align256(m * sizeof(QParamF32)) +
                         align256(d.w.splits * 4 * m * sizeof(float));
        cnt_off[i] = cnt_total;
        cnt_total += sizeof(uint32_t) * (d.knn.qblocks + 1 + d.w.qblocks);
    }
    // Units: items in decreasing size within each phase; phase by phase, or interleaved.
    std::vector<int32_t> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        return static_cast<double>(h[a].m) * h[a].ds.n_pad >
               static_cast<double>(h[b].m) * h[b].ds.n_pad;
    });
    std::vector<WorkUnit> u;
    auto knn_units = [&](int32_t i) {
        for (int qb = 0; qb < h[i].knn.qblocks; ++qb)
            for (int s = 0; s < h[i].knn.splits; ++s)
                u.push_back({i, qb, s, kUnitKnn});
    };
    auto select_units = [&](int32_t i) {
        for (int qb = 0; qb < h[i].knn.qblocks; ++qb)
            u.push_back({i, qb, 0, kUnitSelect});
    };
    auto weight_units = [&](int32_t i) {
        for (int qb = 0; qb < h[i].w.qblocks; ++qb)
            for (int s = 0; s < h[i].w.splits; ++s)
                u.push_back({i, qb, s, kUnitWeights});
    };
    if (cfg.unit_order == 1) {
        // Interleaved: phase-1 units run ahead by about two waves of CTAs; each item's SELECT
        // and WEIGHTS units follow once its phase-1 units are that far back in the list, with
        // the phase-1 units of the next item after them, so both phases share the SMs.
        const size_t lead = static_cast<size_t>(2 * 4 * ctx_sm_count(ctx));
        size_t queued = 0;
        int32_t next = 0;
        while (next < count && queued < lead) {
            queued += static_cast<size_t>(h[order[next]].knn.qblocks) * h[order[next]].knn.splits;
            knn_units(order[next++]);
        }
        for (int32_t ii = 0; ii < count; ++ii) {
            while (next <= ii)
                knn_units(order[next++]);
            select_units(order[ii]);
            weight_units(order[ii]);
            if (next < count)
                knn_units(order[next++]);
        }
    } else {
        for (int32_t i : order)
            knn_units(i);
        for (int32_t i : order)
            select_units(i);
        for (int32_t i : order)
            weight_units(i);
    }
    // FINAL units last: each waits for its block's WEIGHTS units, all taken long before.
    for (int32_t i : order)
        for (int qb = 0; qb < h[i].w.qblocks; ++qb)
            u.push_back({i, qb, 0, kUnitFinal});

    const size_t tq = static_cast<size_t>(std::max<int64_t>(total_q, 1));
    const size_t b_items = align256(sizeof(BatchItemDev) * std::max<int32_t>(count, 1));
    const size_t b_units = align256(sizeof(WorkUnit) * std::max<size_t>(u.size(), 1));
    const size_t b_cnt = align256(cnt_total);
    const size_t b_q = align256(tq * sizeof(uint32_t));
    const size_t b_order = 6 * b_q + align256(radix_scratch_bytes(static_cast<int64_t>(tq)));
    bs->bytes = b_items + b_units + b_cnt + b_order + scratch_total;
    int rc = ctx_alloc(ctx, bs->bytes, st, &bs->block);
    if (rc)
        return rc;
    char *base = static_cast<char *>(bs->block);
    bs->d_items = base;
    bs->d_units = base + b_items;
    bs->d_counters = reinterpret_cast<uint32_t *>(base + b_items + b_units);
    bs->counter_bytes = cnt_total;
    char *ord = base + b_items + b_units + b_cnt;
    bs->keys = reinterpret_cast<uint32_t *>(ord);
    bs->vals = reinterpret_cast<uint32_t *>(ord + b_q);
    bs->item_of = reinterpret_cast<uint32_t *>(ord + 2 * b_q);
    bs->perm = reinterpret_cast<uint32_t *>(ord + 3 * b_q);
    bs->sqx = reinterpret_cast<float *>(ord + 4 * b_q);
    bs->sqy = reinterpret_cast<float *>(ord + 5 * b_q);
    bs->sort_tmp = ord + 6 * b_q;
    char *scratch = ord + b_order;
    for (int32_t i = 0; i < count; ++i) {
        BatchItemDev &d = h[i];
        const size_t m = static_cast<size_t>(d.m);
        char *p = scratch + scratch_off[i];
        d.part_d2 = reinterpret_cast<float *>(p);
        p += align256(d.knn.splits * static_cast<size_t>(d.k) * m * sizeof(float));
        d.qparam = reinterpret_cast<QParamF32 *>(p);
        p += align256(m * sizeof(QParamF32));
        d.part_sum = reinterpret_cast<float *>(p);
        d.sqx = bs->sqx + d.qoff;
        d.sqy = bs->sqy + d.qoff;
        d.perm = bs->perm + d.qoff;
        uint32_t *c = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(bs->d_counters) +
                                                   cnt_off[i]);
        d.cnt_knn = c;
        d.cnt_sel = c + d.knn.qblocks;
        d.cnt_w = c + d.knn.qblocks + 1;
    }
    bs->count = count;
    bs->total_q = total_q;
    bs->max_m = max_m;
    bs->dyn_smem = sizeof(unsigned long long) * static_cast<size_t>(std::max(max_p2, 1));
    bs->n_units = static_cast<int>(u.size());
    bs->cfg = cfg;
    bs->grid = batch_grid(ctx_sm_count(ctx), bs->dyn_smem, cfg.queries_per_thread,
                          cfg.ctas_per_sm);
    bool ok = true;
    if (count > 0)
        ok &= cudaMemcpyAsync(bs->d_items, h.data(), sizeof(BatchItemDev) * count,
                              cudaMemcpyHostToDevice, st) == cudaSuccess;
    if (!u.empty())
        ok &= cudaMemcpyAsync(bs->d_units, u.data(), sizeof(WorkUnit) * u.size(),
                              cudaMemcpyHostToDevice, st) == cudaSuccess;
    // The copies read pageable host memory: they are staged before cudaMemcpyAsync returns,
    // and ordered on `st` before the kernels.
    if (!ok) {
        ctx_free(ctx, bs->block, bs->bytes, st);
        bs->block = nullptr;
        return AIDW_ERR_CUDA;
    }
    return AIDW_OK;
}

// Stream-ordered: order the queries, zero the counters, run the persistent kernel.
int batch_enqueue(aidw_ctx *ctx, const BatchState &bs, cudaStream_t st)
{
    if (bs.n_units == 0)
        return AIDW_OK;
    NvtxScope range("aidw batch");
    const BatchItemDev *items = static_cast<const BatchItemDev *>(bs.d_items);
    const int64_t tq = bs.total_q;
    const unsigned gx = static_cast<unsigned>(std::min<int64_t>((bs.max_m + 255) / 256, 64));
    batch_keys_kernel<<<dim3(std::max(gx, 1u), bs.count), 256, 0, st>>>(items, bs.keys, bs.vals,
                                                                         bs.item_of);
    if (cudaGetLastError() != cudaSuccess ||
        radix_sort_pairs(bs.keys, bs.vals, tq, bs.sort_tmp, st, 32) != cudaSuccess)
        return AIDW_ERR_CUDA;
    const unsigned g1 = static_cast<unsigned>(std::min<int64_t>((tq + 255) / 256, 4096));
    batch_item_keys_kernel<<<std::max(g1, 1u), 256, 0, st>>>(bs.vals, bs.item_of, tq, bs.keys);
    if (cudaGetLastError() != cudaSuccess ||
        radix_sort_pairs(bs.keys, bs.vals, tq, bs.sort_tmp, st, 16) != cudaSuccess)
        return AIDW_ERR_CUDA;
    batch_gather_kernel<<<std::max(g1, 1u), 256, 0, st>>>(items, bs.vals, bs.item_of, tq,
                                                          bs.sqx, bs.sqy, bs.perm);
    if (cudaMemsetAsync(bs.d_counters, 0, bs.counter_bytes, st) != cudaSuccess)
        return AIDW_ERR_CUDA;
    batch_kernel_for(bs.cfg.queries_per_thread)<<<bs.grid, kThreads, bs.dyn_smem, st>>>(
        items, static_cast<const WorkUnit *>(bs.d_units), bs.n_units, bs.d_counters,
        ctx_err_word(ctx), bs.cfg.tile_points);
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

// (Re)builds a prepared batch under `cfg`: the tables on a private stream, then the query
// ordering, the counter reset and the persistent kernel captured as one graph. Earlier launches
// of the batch are waited for first. On failure the batch is rebuilt with its previous shape.
int batch_prepare(aidw_ctx *ctx, aidw_batch *b, const aidw_tune_config &cfg)
{
    if (!tune_valid(cfg))
        return AIDW_ERR_INVALID_ARG;
    if (cudaSetDevice(ctx_device(ctx)) != cudaSuccess)
        return AIDW_ERR_CUDA;
    cudaStream_t cap;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess)
        return AIDW_ERR_CUDA;
    const bool had = b->st.block != nullptr || b->st.graph != nullptr;
    const aidw_tune_config old = b->st.cfg;
    if (had) {
        cudaDeviceSynchronize();
        batch_release(ctx, &b->st, cap);
        b->st = BatchState{};
    }
    auto attempt = [&](const aidw_tune_config &c) {
        BatchState fresh;
        int rc = batch_build(ctx, b->items.data(), static_cast<int32_t>(b->items.size()), cap,
                             &fresh, c);
        if (rc == AIDW_OK && cudaStreamSynchronize(cap) != cudaSuccess)
            rc = AIDW_ERR_CUDA;
        if (rc == AIDW_OK) {
            cudaGraph_t g = nullptr;
            bool ok = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                const int erc = batch_enqueue(ctx, fresh, cap);
                ok = cudaStreamEndCapture(cap, &g) == cudaSuccess && erc == AIDW_OK;
            }
            ok = ok && cudaGraphInstantiate(&fresh.graph, g, 0) == cudaSuccess;
            if (g)
                cudaGraphDestroy(g);
            if (!ok) {
                cudaGetLastError();
                rc = AIDW_ERR_CUDA;
            }
        }
        if (rc != AIDW_OK) {
            if (fresh.block)
                batch_release(ctx, &fresh, cap);
            cudaStreamSynchronize(cap);
            return rc;
        }
        b->st = fresh;
        return AIDW_OK;
    };
    int rc = attempt(cfg);
    if (rc != AIDW_OK && had)
        attempt(old);
    cudaStreamDestroy(cap);
    return rc;
}

}  // namespace aidw

using namespace aidw;

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
    int rc = batch_build(ctx, items, count, st, &bs, ctx_tune(ctx));
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
    if (count < 0 || count > 65535 || (count > 0 && !items))
        return AIDW_ERR_INVALID_ARG;
    aidw_batch *b = new aidw_batch();
    b->items.assign(items, items + count);
    const int rc = batch_prepare(ctx, b, ctx_tune(ctx));
    if (rc != AIDW_OK) {
        delete b;
        return rc;
    }
    *out = b;
    return AIDW_OK;
}

int aidw_batch_set_config(aidw_ctx *ctx, aidw_batch *b, const aidw_tune_config *cfg)
{
    if (!ctx || !b || !cfg)
        return AIDW_ERR_INVALID_ARG;
    return batch_prepare(ctx, b, *cfg);
}

int aidw_batch_get_config(aidw_ctx *ctx, aidw_batch *b, aidw_tune_config *out)
{
    if (!ctx || !b || !out)
        return AIDW_ERR_INVALID_ARG;
    *out = b->st.cfg;
    return AIDW_OK;
}

int aidw_batch_launch(aidw_ctx *ctx, aidw_batch *b, void *stream)
{
    if (!ctx || !b)
        return AIDW_ERR_INVALID_ARG;
    if (b->st.n_units == 0)
        return AIDW_OK;
    NvtxScope range("aidw batch");
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
