// Batched AIDW: many independent (dataset, query set) items in one persistent work-queue
// kernel, launched through a captured CUDA graph.
//
// Every item is cut into units that depend only on the item itself (never on what else is in
// the batch), so an item's result is bit-identical whether it runs alone or in any mix:
//   phase-1 list
//     KNN     (item, query block)         pruned phase-1 scan of Z-ordered queries (nearest
//                                         data tiles first) with the selection (Eq. 3-6)
//                                         fused: the block's phase-2 parameters are ready
//             (item, query block, split)  split scan for items too large to prune or with
//                                         few queries
//     SELECT  (item, query block)         merge of a split-scan block's lists + Eq. 3-6; waits
//                                         for the block's KNN units (earlier in the list)
//   phase-2 list
//     WEIGHTS (item, query block, split)  phase-2 scan of one data split; needs every query
//                                         block of its item through selection
//     FINAL   (item, query block)         split merge + Eq. 1 ratio; waits for the block's
//                                         WEIGHTS units (earlier in the list)
// Before the persistent kernel, the queries of all items are put in Z-order item by item (one
// radix sort of keys made of the item's index and the query's Morton cell in its dataset's
// box) so that each KNN unit's block is compact; results go back to the caller's order.
// Both lists hold the items in decreasing size; CTAs take units from them through two atomic
// counters, preferring a phase-2 unit whose inputs are complete and taking phase-1 units
// otherwise, so that phase 1 (ALU and latency bound) shares the SMs with phase 2 (MUFU bound)
// instead of running before it (see f32_batch_kernel). Producers publish with a fence and an
// atomic add; consumers read counters with acquire loads and results with L2 loads.
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

// Queries per thread of the batch's split-scan phase-1 units (every list length).
constexpr int kBatchSplitQ = 2;

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
    uint32_t *cnt_knn;   // [knn.qblocks] finished split-scan phase-1 units per query block
    uint32_t *cnt_ready; // [1] query blocks through selection (pruned KNN or SELECT units)
    uint32_t *cnt_w;     // [w.qblocks] finished phase-2 splits per query block
};

struct WorkUnit {
    int32_t item, qblock, split, type;
    // Phase-2 units: the counter that completes their inputs and its target value (read by the
    // scheduler without touching the item table).
    uint32_t target, reserved;
    const uint32_t *counter;
};

// Every thread's results are made visible at GPU scope before thread 0 counts the unit done.
__device__ __forceinline__ void cta_publish(uint32_t *counter)
{
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0)
        atomicAdd(counter, 1u);
}

// The persistent kernel's tile buffers and their barriers, at file scope so that the phase-2
// unit below, compiled as a function of its own, addresses them as shared memory directly.
__shared__ __align__(128) float4 g_txy[2][kTileF32W];
__shared__ __align__(128) float2 g_tz[2][kTileF32W];
__shared__ __align__(8) uint64_t g_bar[2];

// A WEIGHTS unit as an out-of-line function: inlined into the persistent kernel, the phase-2
// loop was scheduled worse than in the one-shot kernel (measured on a one-item batch of 1M
// points x 65,536 queries: 29 % more instructions per pair, the XU pipe busy 73 % of the time
// instead of 92 %). The tiles consumed (whole tiles of the split) are counted by the caller.
template <int QW, int TW>
__device__ __noinline__ bool batch_weights_unit(const BatchItemDev *itp, int qblock, int split,
                                                int *err, uint32_t seq)
{
    const BatchItemDev &it = *itp;
    const int64_t qbase = static_cast<int64_t>(qblock) * it.w.q_per_block;
    const int64_t p0 = static_cast<int64_t>(split) * it.w.split_len;
    const int64_t p1 = min(p0 + it.w.split_len, it.ds.n_pad);
    TileSeq ts{g_bar, seq};
    return weights_unit<QW, TW>(it.ds, it.m, qbase, p0, p1, it.sqx, it.sqy, it.qparam, split,
                                it.part_sum, err,
                                reinterpret_cast<float4(*)[TW]>(&g_txy[0][0]),
                                reinterpret_cast<float2(*)[TW]>(&g_tz[0][0]), ts);
}

// Largest tile count whose pruned-scan tile order (8 bytes a tile) fits in g_tz.
constexpr int kOrderInTz = static_cast<int>(sizeof(g_tz) / sizeof(unsigned long long));

// Whether a phase-2 unit's inputs are complete (thread 0; an acquire load, so that the CTA reads
// the producers' results after the following barrier): a WEIGHTS unit needs its item's phase 1
// (every query block selected), a FINAL unit the WEIGHTS units of its query block.
__device__ __forceinline__ bool p2_ready(const WorkUnit &wu)
{
    return ld_acquire(wu.counter) >= wu.target;
}

// What a CTA does next (decided by thread 0, shared through shared memory).
enum NextKind : int32_t { kExit = 0, kRunP1 = 1, kRunP2 = 2, kWaitP2 = 3 };

// The persistent batch kernel. Units come from two lists: phase 1 (KNN units, with the
// selection fused into pruned ones, and SELECT units after the split-scan KNN units of their
// query block) and phase 2 (WEIGHTS units, then FINAL units), both in decreasing item size,
// each with its own counter. A CTA takes the next phase-2 unit when its inputs are complete
// and a phase-1 unit otherwise; a phase-2 unit taken before its inputs are complete is held
// while the CTA runs phase-1 units, and waited for (bounded) once none are left. With
// p1_every > 0, every p1_every-th CTA takes phase-1 units first, so phase 1 runs ahead of
// phase 2 on part of the SMs while the rest run phase 2. A unit only ever waits for units
// that running CTAs have already taken (phase-1 units never wait for phase 2, a SELECT unit
// only for earlier phase-1 units, a FINAL unit for WEIGHTS units, all earlier in their list),
// so every wait ends; each is still bounded and raises the error word if it runs out. Which
// CTA runs a unit never changes its arithmetic.
// QW: phase-2 queries per thread; tw: phase-2 tile points (256 or 512). LEAN: the variant for
// batches whose items all have k <= 16 and whose pruned phase-1 units take 2 queries per
// thread, compiled for 64 registers (8 CTAs per SM instead of 4; the MUFU-bound phase-2 units
// need the warps) with only those phase-1 units built in.
template <int QW, bool LEAN>
__global__ void __launch_bounds__(kThreads, LEAN ? 8 : 4)
f32_batch_kernel(const BatchItemDev *__restrict__ items, const WorkUnit *__restrict__ units,
                 int n1, int n2, uint32_t *next, int *err, int tw, int p1_every,
                 bool dyn_order_in_tz)
{
    // Tile order of a pruned KNN unit: in the phase-2 value buffers (unused by phase-1 units)
    // when the batch's datasets have at most kOrderInTz tiles, else in dynamic shared memory.
    extern __shared__ unsigned long long dyn_order[];
    unsigned long long *order =
        dyn_order_in_tz ? reinterpret_cast<unsigned long long *>(&g_tz[0][0]) : dyn_order;
    __shared__ CullShared cs;
    // Phase-1 and phase-2 units take turns on the same coordinate tile buffers.
    static_assert(kTileF32Knn == kTileF32W, "shared tile buffers");
    float4(*ktile)[kTileF32Knn] = g_txy;
    __shared__ int s_kind, s_unit, s_flag;
    init_tile_barriers(g_bar);
    TileSeq ts{g_bar, 0u};
    const int tid = threadIdx.x;
    const WorkUnit *units2 = units + n1;
    uint32_t *next1 = next, *next2 = next + 1;
    // Thread 0's scheduling state.
    int pending = -1;  // phase-2 unit taken, inputs not yet complete
    bool p1_done = false;
    const bool p1_first = p1_every > 0 && (blockIdx.x % p1_every) == 0;

    for (;;) {
        if (tid == 0) {
            int kind = kExit, unit = -1;
            auto take_p1 = [&]() {
                if (p1_done)
                    return false;
                const int u = static_cast<int>(atomicAdd(next1, 1u));
                if (u < n1) {
                    kind = kRunP1;
                    unit = u;
                    return true;
                }
                p1_done = true;
                return false;
            };
            if (pending < 0) {
                bool p2 = !p1_first;
                if (p2) {
                    // Peek at the next phase-2 unit; phase 1 while it cannot run yet.
                    const int h = static_cast<int>(*reinterpret_cast<volatile uint32_t *>(next2));
                    p2 = h >= n2 || p2_ready(units2[h]);
                }
                if (!p2 && !take_p1())
                    p2 = true;
                if (p2) {
                    const int u = static_cast<int>(atomicAdd(next2, 1u));
                    if (u < n2)
                        pending = u;
                }
            }
            if (pending >= 0) {
                if (p2_ready(units2[pending])) {
                    kind = kRunP2;
                    unit = pending;
                    pending = -1;
                } else if (!take_p1()) {
                    kind = kWaitP2;
                    unit = pending;
                    pending = -1;
                }
            }
            s_kind = kind;
            s_unit = unit;
        }
        __syncthreads();
        int kind = s_kind;
        const int uidx = s_unit;
        __syncthreads();
        if (kind == kExit)
            break;
        // The previous unit's generic accesses to the tile buffers (and the tile order kept in
        // g_tz) are ordered before this unit's bulk copies into them.
        if (tid == 0)
            fence_proxy_async_smem();
        bool ok = true;
        if (kind == kWaitP2) {
            // Every phase-1 unit has been taken: the inputs are being computed by running CTAs.
            const WorkUnit &w2 = units2[uidx];
            if (tid == 0) {
                bool got = false;
                for (uint32_t i = 0; i < kMaxWaitPolls; ++i) {
                    if (p2_ready(w2)) {
                        got = true;
                        break;
                    }
                    __nanosleep(256);
                }
                s_flag = got ? 1 : 0;
            }
            __syncthreads();
            ok = s_flag != 0;
            __syncthreads();
            kind = kRunP2;
        }
        const WorkUnit wu = kind == kRunP1 ? units[uidx] : units2[uidx];
        const BatchItemDev &it = items[wu.item];
        if (!ok) {
            // fall through to the error exit below
        } else if (wu.type == kUnitKnn && it.ntiles_p2 == 0) {
            // Dataset too large for the shared-memory tile order: split scan.
            const int64_t qbase = static_cast<int64_t>(wu.qblock) * it.knn.q_per_block;
            const int64_t p0 = static_cast<int64_t>(wu.split) * it.knn.split_len;
            const int64_t p1 = min(p0 + it.knn.split_len, it.ds.n_pad);
#define AIDW_SPLIT_UNIT(KP)                                                                    \
    ok = knn_unit<KP, kBatchSplitQ, false>(it.ds, it.m, qbase, p0, p1, it.sqx, it.sqy, it.k,     \
                                           wu.split, it.part_d2, nullptr, err, ktile, ts, nullptr)
            switch (it.kp) {
            case 8:
                AIDW_SPLIT_UNIT(8);
                break;
            case 12:
                AIDW_SPLIT_UNIT(12);
                break;
            case 16:
                AIDW_SPLIT_UNIT(16);
                break;
            default:
                if constexpr (!LEAN)
                    AIDW_SPLIT_UNIT(32);
                break;
            }
#undef AIDW_SPLIT_UNIT
            if (ok)
                cta_publish(&it.cnt_knn[wu.qblock]);
        } else if (wu.type == kUnitKnn) {
            // Pruned scan with the selection fused: the query block is complete afterwards.
            const int64_t qbase = static_cast<int64_t>(wu.qblock) * it.knn.q_per_block;
            const FusedSelect fsel{it.r_exp, it.am, it.qparam, it.out_alpha, it.perm};
#define AIDW_CULL_UNIT(KP, Q)                                                                  \
    ok = knn_cull_unit<KP, Q, false>(it.ds, it.m, qbase, it.ntiles, it.ntiles_p2, it.sqx, it.sqy, \
                                     it.k, it.part_d2, nullptr, err, ktile, ts, order, nullptr,  \
                                     cs, &fsel)
            const bool q2 = LEAN || it.kq == 2;
            switch (it.kp) {
            case 8:
                if (q2)
                    AIDW_CULL_UNIT(8, 2);
                else if constexpr (!LEAN)
                    AIDW_CULL_UNIT(8, 4);
                break;
            case 12:
                if (q2)
                    AIDW_CULL_UNIT(12, 2);
                else if constexpr (!LEAN)
                    AIDW_CULL_UNIT(12, 4);
                break;
            case 16:
                if (q2)
                    AIDW_CULL_UNIT(16, 2);
                else if constexpr (!LEAN)
                    AIDW_CULL_UNIT(16, 4);
                break;
            default:
                if constexpr (!LEAN)
                    AIDW_CULL_UNIT(32, 2);
                break;
            }
#undef AIDW_CULL_UNIT
            if (ok)
                cta_publish(it.cnt_ready);
        } else if (wu.type == kUnitSelect) {
            ok = cta_wait_count(&it.cnt_knn[wu.qblock], it.knn.splits, &s_flag);
            if (ok) {
                const int64_t qbase = static_cast<int64_t>(wu.qblock) * it.knn.q_per_block;
                const int64_t qend = min(qbase + it.knn.q_per_block, it.m);
                for (int64_t q = qbase + tid; q < qend; q += kThreads)
                    select_query(q, it.m, it.knn.splits, it.k, it.r_exp, it.am, it.part_d2,
                                 nullptr, it.qparam, it.out_alpha, nullptr, it.perm);
                cta_publish(it.cnt_ready);
            }
        } else if (wu.type == kUnitWeights) {
            const int64_t p0 = static_cast<int64_t>(wu.split) * it.w.split_len;
            const int64_t p1 = min(p0 + it.w.split_len, it.ds.n_pad);
            if (tw == 256) {
                ok = batch_weights_unit<QW, 256>(&it, wu.qblock, wu.split, err, ts.seq);
                ts.seq += static_cast<uint32_t>(weights_tiles<256>(it.ds, p0, p1));
            } else {
                ok = batch_weights_unit<QW, kTileF32W>(&it, wu.qblock, wu.split, err, ts.seq);
                ts.seq += static_cast<uint32_t>(weights_tiles<kTileF32W>(it.ds, p0, p1));
            }
            if (ok)
                cta_publish(&it.cnt_w[wu.qblock]);
        } else {
            const int64_t qbase = static_cast<int64_t>(wu.qblock) * it.w.q_per_block;
            const int64_t qend = min(qbase + it.w.q_per_block, it.m);
            for (int64_t q = qbase + tid; q < qend; q += kThreads)
                it.out[it.perm[q]] = finalize_query(q, it.m, it.w.splits, it.part_sum);
        }
        if (!ok) {
            if (tid == 0)
                atomicOr(err, kErrTimeout);
            break;
        }
    }
}

// Batch-wide query ordering, step 1: one 32-bit key per query, the item's index in the high
// item_bits bits and the top bits of the query's Morton key over its item's dataset box below
// (2^(32 - item_bits) cells: at least 256 x 256 per item), so that one radix sort groups the
// items and puts each item's queries in Z-order; values are batch-wide positions, and the item
// of every position is recorded.
__global__ void batch_keys_kernel(const BatchItemDev *__restrict__ items, int item_bits,
                                  uint32_t *keys, uint32_t *vals, uint32_t *item_of)
{
    const BatchItemDev &it = items[blockIdx.y];
    const float4 box = *it.ds.box;
    const uint32_t hi = item_bits > 0 ? (blockIdx.y << (32 - item_bits)) : 0u;
    for (int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < it.m;
         q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t g = it.qoff + q;
        keys[g] = hi | (morton_of(it.qx[q], it.qy[q], box) >> item_bits);
        vals[g] = static_cast<uint32_t>(g);
        item_of[g] = blockIdx.y;
    }
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

using BatchKernel = void (*)(const BatchItemDev *, const WorkUnit *, int, int, uint32_t *,
                            int *, int, int, bool);

BatchKernel batch_kernel_for(int qw, bool lean)
{
    if (lean)
        return f32_batch_kernel<2, true>;
    return qw == 2 ? f32_batch_kernel<2, false>
                   : (qw == 8 ? f32_batch_kernel<8, false> : f32_batch_kernel<4, false>);
}

// Shape field unit_order = 1: every kBatchP1Every-th persistent CTA takes phase-1 units first.
constexpr int kBatchP1Every = 4;

// Persistent grid: CTAs per SM as occupancy allows, or fewer if the shape asks for it, less
// `reserve` per SM (left free for another launch; at least one CTA per SM remains).
int batch_grid(int sm_count, size_t dyn, int qw, bool lean, int ctas_per_sm, int reserve)
{
    const BatchKernel fn = batch_kernel_for(qw, lean);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(dyn));
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, kThreads, dyn);
    n = n > 0 ? n : 1;
    if (ctas_per_sm > 0 && ctas_per_sm < n)
        n = ctas_per_sm;
    n = n - reserve > 0 ? n - reserve : 1;
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
// of 8,192 queries against 231,679 points with 65,536-point splits: 128 units; served in 5.3 ms,
// with the extra splits in 2.7 ms, the one-shot call 2.5 ms). 512 units keep at least 3-4 CTAs
// busy on every SM and make fewer, longer units than 1,024 (the 256-dataset batch: 70.7 against
// 71.3 ms). The split length depends on the item's sizes and split_points only (not on the rest
// of the batch, nor on the arithmetic-neutral shape fields).
constexpr int64_t kBatchMinWeightUnits = 512;

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
    const int qk = kThreads * (*cull ? kq : kBatchSplitQ);
    if (*cull)
        return batch_pass(m, n_pad, qk, n_pad);
    const int64_t qblocks = std::max<int64_t>(1, (m + qk - 1) / qk);
    const int64_t splits = std::max<int64_t>(1, kBatchKnnUnits / qblocks);
    const int64_t target = std::max<int64_t>(kPadPoints, (n_pad + splits - 1) / splits);
    return batch_pass(m, n_pad, qk, std::min<int64_t>(target, kBatchKnnSplit));
}

// Phase-1 scratch of an item: split lists [S][k][m] for split-scan items; pruned items select
// inside their KNN units and keep no lists.
size_t batch_lists_bytes(const PassPlan &pk, bool cull, int k, int64_t m)
{
    return cull ? 0
                : align256(pk.splits * static_cast<size_t>(k) * static_cast<size_t>(m) *
                           sizeof(float));
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
    return batch_lists_bytes(pk, cull, k, m) + align256(mm * sizeof(QParamF32)) +
           align256(pw.splits * 4 * mm * sizeof(float)) +
           sizeof(uint32_t) * (pk.qblocks + 1 + pw.qblocks) + sizeof(BatchItemDev) +
           sizeof(WorkUnit) * (pk.qblocks * (pk.splits + 1) + pw.qblocks * (pw.splits + 1)) +
           mm * (6 * sizeof(uint32_t)) + radix_scratch_bytes(m);
}

// Validates the items and builds the device tables of a batch in library memory.
int batch_build(aidw_ctx *ctx, const aidw_batch_item *items, int32_t count, cudaStream_t st,
                BatchState *bs, const aidw_tune_config &cfg, int reserve_ctas_per_sm)
{
    if (!tune_valid(cfg))
        return AIDW_ERR_INVALID_ARG;
    if (count < 0 || count > 65535 || (count > 0 && !items))
        return AIDW_ERR_INVALID_ARG;
    const int device = ctx_device(ctx);
    std::vector<BatchItemDev> h(count);
    std::vector<size_t> scratch_off(count), cnt_off(count);
    // Slots 0 and 1: the counters of the phase-1 and phase-2 work lists.
    size_t scratch_total = 0, cnt_total = 2 * sizeof(uint32_t);
    int64_t total_q = 0, max_m = 0;
    int max_p2 = 0;
    // The 64-register kernel serves the batch if every item fits its built-in phase-1 units.
    bool lean = cfg.queries_per_thread == 2;
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
        if (b.m > 0 && (d.kp > 16 || (cull && d.kq != 2)))
            lean = false;
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
        scratch_total += batch_lists_bytes(d.knn, cull, d.k, b.m) +
                         align256(m * sizeof(QParamF32)) +
                         align256(d.w.splits * 4 * m * sizeof(float));
        cnt_off[i] = cnt_total;
        cnt_total += sizeof(uint32_t) * (d.knn.qblocks + 1 + d.w.qblocks);
    }
    // Two work lists, items in decreasing size in both: phase 1 (the KNN units of an item, and
    // for a split-scan item the SELECT unit of each query block after them) and phase 2 (all
    // WEIGHTS units, then all FINAL units: a FINAL unit waits for its block's WEIGHTS units,
    // which are all taken before it).
    std::vector<int32_t> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        return static_cast<double>(h[a].m) * h[a].ds.n_pad >
               static_cast<double>(h[b].m) * h[b].ds.n_pad;
    });
    std::vector<WorkUnit> u;
    for (int32_t i : order) {
        for (int qb = 0; qb < h[i].knn.qblocks; ++qb)
            for (int sp = 0; sp < h[i].knn.splits; ++sp)
                u.push_back({i, qb, sp, kUnitKnn});
        if (h[i].ntiles_p2 == 0)
            for (int qb = 0; qb < h[i].knn.qblocks; ++qb)
                u.push_back({i, qb, 0, kUnitSelect});
    }
    const size_t n1 = u.size();
    for (int32_t i : order)
        for (int qb = 0; qb < h[i].w.qblocks; ++qb)
            for (int sp = 0; sp < h[i].w.splits; ++sp)
                u.push_back({i, qb, sp, kUnitWeights});
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
        p += batch_lists_bytes(d.knn, d.ntiles_p2 != 0, d.k, d.m);
        d.qparam = reinterpret_cast<QParamF32 *>(p);
        p += align256(m * sizeof(QParamF32));
        d.part_sum = reinterpret_cast<float *>(p);
        d.sqx = bs->sqx + d.qoff;
        d.sqy = bs->sqy + d.qoff;
        d.perm = bs->perm + d.qoff;
        uint32_t *c = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(bs->d_counters) +
                                                   cnt_off[i]);
        d.cnt_knn = c;
        d.cnt_ready = c + d.knn.qblocks;
        d.cnt_w = c + d.knn.qblocks + 1;
    }
    for (size_t j = n1; j < u.size(); ++j) {
        WorkUnit &w = u[j];
        const BatchItemDev &d = h[w.item];
        if (w.type == kUnitWeights) {
            w.counter = d.cnt_ready;
            w.target = static_cast<uint32_t>(d.knn.qblocks);
        } else {
            w.counter = d.cnt_w + w.qblock;
            w.target = static_cast<uint32_t>(d.w.splits);
        }
    }
    bs->count = count;
    bs->total_q = total_q;
    bs->max_m = max_m;
    // Up to kOrderInTz tiles the tile order lives in the phase-2 value buffers: no dynamic
    // shared memory, so 8 CTAs of the 64-register kernel fit on an SM.
    bs->order_in_tz = max_p2 <= kOrderInTz;
    bs->dyn_smem = bs->order_in_tz
                       ? 0
                       : sizeof(unsigned long long) * static_cast<size_t>(std::max(max_p2, 1));
    bs->n_units = static_cast<int>(u.size());
    bs->n_units1 = static_cast<int>(n1);
    bs->cfg = cfg;
    bs->lean = lean;
    bs->grid = batch_grid(ctx_sm_count(ctx), bs->dyn_smem, cfg.queries_per_thread, lean,
                          cfg.ctas_per_sm, reserve_ctas_per_sm);
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
    // Bits for the item index (even, so that the Morton part keeps whole cells), at most 16.
    int item_bits = 0;
    while ((int64_t(1) << item_bits) < bs.count)
        ++item_bits;
    item_bits = (item_bits + 1) & ~1;
    batch_keys_kernel<<<dim3(std::max(gx, 1u), bs.count), 256, 0, st>>>(
        items, item_bits, bs.keys, bs.vals, bs.item_of);
    if (cudaGetLastError() != cudaSuccess ||
        radix_sort_pairs(bs.keys, bs.vals, tq, bs.sort_tmp, st, 32) != cudaSuccess)
        return AIDW_ERR_CUDA;
    const unsigned g1 = static_cast<unsigned>(std::min<int64_t>((tq + 255) / 256, 4096));
    batch_gather_kernel<<<std::max(g1, 1u), 256, 0, st>>>(items, bs.vals, bs.item_of, tq,
                                                          bs.sqx, bs.sqy, bs.perm);
    if (cudaMemsetAsync(bs.d_counters, 0, bs.counter_bytes, st) != cudaSuccess)
        return AIDW_ERR_CUDA;
    batch_kernel_for(bs.cfg.queries_per_thread, bs.lean)<<<bs.grid, kThreads, bs.dyn_smem, st>>>(
        items, static_cast<const WorkUnit *>(bs.d_units), bs.n_units1,
        bs.n_units - bs.n_units1, bs.d_counters, ctx_err_word(ctx), bs.cfg.tile_points,
        bs.cfg.unit_order == 1 ? kBatchP1Every : 0, bs.order_in_tz);
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
