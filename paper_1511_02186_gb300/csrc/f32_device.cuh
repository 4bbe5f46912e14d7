// Device-side building blocks of the FP32 ("F32C") path, shared by the per-call grid kernels
// (kernels_f32.cu) and the persistent batched kernel (batched.cu).
//
// Phase 1 (Sec. 2.2 Step 1; kNN procedure of Sec. 3.1.2) and phase 2 (Eq. 1 over all data
// points, Sec. 3.2.1) are two all-pairs scans of the data points against blocks of queries. A
// unit of work is one (query block, data split): 128 threads, each holding Q queries in
// registers as Q/2 packed pairs, stream the split's data tiles through shared memory (one TMA
// bulk copy per tile into a double buffer completed on an mbarrier) and read every data point
// as a broadcast.
#pragma once

#include <math_constants.h>

#include "aidw_internal.cuh"
#include "warp_knn.cuh"

namespace aidw {
namespace f32dev {

constexpr int kChunkKnn = 8;  // points between neighbour-list threshold checks
constexpr int kChunkW = 32;   // points summed in plain FP32 before a Kahan merge
constexpr float kFilterMargin = 1.0f + 9.5367431640625e-07f;  // 1 + 2^-20
constexpr float kBoundShrink = 1.0f - 9.5367431640625e-07f;   // 1 - 2^-20, box bounds

// Squared distance from negated data coordinates: q + (-p) is exactly q - p.
__device__ __forceinline__ float dist2_neg(float qx, float qy, float npx, float npy)
{
    const float dx = __fadd_rn(qx, npx);
    const float dy = __fadd_rn(qy, npy);
    return __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, kEpsF32));
}

// Inserts v (< L[KP-1]) into the ascending register list L, after any equal entries.
template <int KP>
__device__ __forceinline__ void list_insert(float (&L)[KP], float v)
{
    L[KP - 1] = v;
#pragma unroll
    for (int i = KP - 1; i > 0; --i) {
        const float a = L[i - 1], b = L[i];
        L[i - 1] = fminf(a, b);
        L[i] = fmaxf(a, b);
    }
}

// Shared-memory index list of one query of one thread: entry i at base[i * kThreads].
// Moves entries [pos, KP-1) up by one and writes id at pos, where pos is the number of
// current entries (before insertion) not greater than v among the first KP-1.
template <int KP>
__device__ __forceinline__ void index_insert(const float (&L)[KP], int32_t *base, float v,
                                             int32_t id)
{
    int pos = 0;
#pragma unroll
    for (int i = 0; i < KP - 1; ++i)
        pos += (L[i] <= v) ? 1 : 0;
    for (int i = KP - 1; i > pos; --i)
        base[i * kThreads] = base[(i - 1) * kThreads];
    base[pos * kThreads] = id;
}

__device__ __forceinline__ float neg_filter_threshold(float kth)
{
    return -(kth * kFilterMargin);
}

__device__ __forceinline__ uint32_t sign_or3(uint32_t acc, float a, float b)
{
    return acc | __float_as_uint(a) | __float_as_uint(b);
}

// A CTA's tile stream: two shared-memory buffers with one mbarrier each. `seq` counts the
// tiles consumed since the barriers were initialised, so the tile with sequence number s lands
// in buffer s & 1 and completes phase (s >> 1) & 1 of that buffer's barrier. Every unit drains
// its own tiles before it returns, so units can follow one another on the same barriers.
struct TileSeq {
    uint64_t *bar;
    uint32_t seq;
};

// Bounded wait for the tiles still in flight after an abandoned scan (tiles t, t+1).
__device__ __forceinline__ void drain(TileSeq &ts, int t, int ntiles)
{
    for (int u = t; u < ntiles && u < t + 2; ++u) {
        const uint32_t sq = ts.seq + u;
        (void)mbar_wait(&ts.bar[sq & 1], (sq >> 1) & 1);
    }
}

// One tile of kTileF32Knn points (stored positions pbase..) through the phase-1 filter and,
// where a sign bit fires, the exact insertion (see knn_unit). With `sub` (the tile's 64-point
// sub-tile boxes) the warp skips a sub-tile when, for every one of its queries, the box bound
// (shrunk by 2^-20 for rounding, as for tiles) exceeds the query's current k-th distance.
template <int KP, int Q, bool IDX>
__device__ __forceinline__ void knn_tile(const float4 *tb, int64_t pbase, float2 (&qxp)[Q / 2],
                                         float2 (&qyp)[Q / 2], float2 (&nthr)[Q / 2],
                                         float (&L)[Q][KP], int32_t *idx_smem,
                                         const float4 *__restrict__ sub = nullptr)
{
    constexpr int H = Q / 2;
    static_assert(kSubTile % kChunkKnn == 0 && kTileF32Knn % kSubTile == 0, "whole sub-tiles");
    const int tid = threadIdx.x;
    for (int c = 0; c < kTileF32Knn; c += kChunkKnn) {
        if (sub && (c % kSubTile) == 0) {
            const float4 sb = sub[c / kSubTile];
            bool need = false;
#pragma unroll
            for (int j = 0; j < Q; ++j) {
                const float qx = (j & 1) ? qxp[j / 2].y : qxp[j / 2].x;
                const float qy = (j & 1) ? qyp[j / 2].y : qyp[j / 2].x;
                const float dx = fmaxf(0.0f, fmaxf(sb.x - qx, qx - sb.z));
                const float dy = fmaxf(0.0f, fmaxf(sb.y - qy, qy - sb.w));
                const float lb = __fmul_rn(__fmaf_rn(dx, dx, __fmul_rn(dy, dy)), kBoundShrink);
                need |= !(lb > L[j][KP - 1]);
            }
            if (!__any_sync(0xffffffffu, need)) {
                c += kSubTile - kChunkKnn;  // the loop adds the last chunk
                continue;
            }
        }
        uint32_t acc[Q];
#pragma unroll
        for (int j = 0; j < Q; ++j)
            acc[j] = 0u;
#pragma unroll
        for (int u = 0; u < kChunkKnn; u += 2) {
            const float4 pa = tb[c + u];
            const float4 pb = tb[c + u + 1];
#pragma unroll
            for (int h = 0; h < H; ++h) {
                const float2 dxa = __fadd2_rn(qxp[h], make_float2(pa.x, pa.y));
                const float2 dya = __fadd2_rn(qyp[h], make_float2(pa.z, pa.w));
                const float2 va = __ffma2_rn(dxa, dxa, __ffma2_rn(dya, dya, nthr[h]));
                const float2 dxb = __fadd2_rn(qxp[h], make_float2(pb.x, pb.y));
                const float2 dyb = __fadd2_rn(qyp[h], make_float2(pb.z, pb.w));
                const float2 vb = __ffma2_rn(dxb, dxb, __ffma2_rn(dyb, dyb, nthr[h]));
                acc[2 * h] = sign_or3(acc[2 * h], va.x, vb.x);
                acc[2 * h + 1] = sign_or3(acc[2 * h + 1], va.y, vb.y);
            }
        }
        uint32_t any = 0u;
#pragma unroll
        for (int j = 0; j < Q; ++j)
            any |= acc[j];
        if (static_cast<int32_t>(any) < 0) {
#pragma unroll
            for (int j = 0; j < Q; ++j) {
                if (static_cast<int32_t>(acc[j]) < 0) {
                    const float qxj = (j & 1) ? qxp[j / 2].y : qxp[j / 2].x;
                    const float qyj = (j & 1) ? qyp[j / 2].y : qyp[j / 2].x;
#pragma unroll 1
                    for (int u = 0; u < kChunkKnn; ++u) {
                        const float4 p = tb[c + u];
                        const float d = dist2_neg(qxj, qyj, p.x, p.z);
                        if (d < L[j][KP - 1]) {
                            if (IDX)
                                index_insert<KP>(L[j], idx_smem + j * KP * kThreads + tid,
                                                 d, static_cast<int32_t>(pbase + c + u));
                            list_insert<KP>(L[j], d);
                        }
                    }
                    const float nt = neg_filter_threshold(L[j][KP - 1]);
                    if (j & 1)
                        nthr[j / 2].y = nt;
                    else
                        nthr[j / 2].x = nt;
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------------------------
// Phase 1 unit: neighbour lists of Q * kThreads queries over data points [p_begin, p_end).
//
// The hot loop evaluates, with FP32x2 instructions, v = dx^2 + (dy^2 - T') for two queries at a
// time, where T' is the query's current k-th squared distance enlarged by 2^-20 (relative), and
// ORs the sign bits of v per query over an 8-point chunk. A negative v is necessary for a point
// to enter the list: if the exact FP32 distance d2 = fl(dx^2 + fl(dy^2)) is below T then the
// real dx^2 + dy^2 is below T (1 + 2^-23), and v, computed with at most u T' of rounding error
// (u = 2^-24), stays negative. Only for a query whose sign bit is set is the chunk rescanned
// with the exact distance, which alone decides insertion; the lists are therefore exactly those
// of the plain scan. Returns false if a tile wait timed out (the error word is then set).
// ---------------------------------------------------------------------------------------------
template <int KP, int Q, bool IDX>
__device__ __forceinline__ bool knn_unit(const DatasetDev &ds, int64_t m, int64_t qbase,
                                         int64_t p_begin, int64_t p_end,
                                         const float *__restrict__ qx,
                                         const float *__restrict__ qy, int k, int s,
                                         float *__restrict__ part_d2,
                                         int32_t *__restrict__ part_idx, int *__restrict__ err,
                                         float4 (*tile)[kTileF32Knn], TileSeq &ts,
                                         int32_t *idx_smem)
{
    static_assert(Q % 2 == 0, "queries are processed in packed pairs");
    constexpr int H = Q / 2;
    const int tid = threadIdx.x;
    const int ntiles = static_cast<int>((p_end - p_begin) / kTileF32Knn);

    float2 qxp[H], qyp[H], nthr[H];
    float L[Q][KP];
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const int64_t q = min(qbase + j * kThreads + tid, m - 1);
        const float a = qx[q], b = qy[q];
        if (j & 1) {
            qxp[j / 2].y = a;
            qyp[j / 2].y = b;
        } else {
            qxp[j / 2].x = a;
            qyp[j / 2].x = b;
        }
#pragma unroll
        for (int i = 0; i < KP; ++i)
            L[j][i] = (i < KP - k) ? -CUDART_INF_F : CUDART_INF_F;
        if (IDX) {
#pragma unroll
            for (int i = 0; i < KP; ++i)
                idx_smem[(j * KP + i) * kThreads + tid] = -1;
        }
    }
#pragma unroll
    for (int h = 0; h < H; ++h)
        nthr[h] = make_float2(-CUDART_INF_F, -CUDART_INF_F);

    constexpr uint32_t kBytes = kTileF32Knn * sizeof(float4);
    if (tid == 0) {
        for (int t = 0; t < 2 && t < ntiles; ++t) {
            const uint32_t b = (ts.seq + t) & 1;
            mbar_arrive_expect_tx(&ts.bar[b], kBytes);
            tma_load_1d(tile[b], ds.nxy2 + p_begin + static_cast<int64_t>(t) * kTileF32Knn,
                        kBytes, &ts.bar[b]);
        }
    }

    for (int t = 0; t < ntiles; ++t) {
        const uint32_t sq = ts.seq + t;
        const int b = sq & 1;
        const bool got = mbar_wait(&ts.bar[b], (sq >> 1) & 1);
        if (!__syncthreads_and(got)) {
            if (tid == 0) {
                atomicOr(err, kErrTimeout);
                drain(ts, t, ntiles);
            }
            ts.seq += ntiles;
            return false;
        }
        const int64_t pbase = p_begin + static_cast<int64_t>(t) * kTileF32Knn;
        knn_tile<KP, Q, IDX>(tile[b], pbase, qxp, qyp, nthr, L, idx_smem);
        __syncthreads();
        if (tid == 0 && t + 2 < ntiles) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&ts.bar[b], kBytes);
            tma_load_1d(tile[b], ds.nxy2 + pbase + 2 * kTileF32Knn, kBytes, &ts.bar[b]);
        }
    }
    ts.seq += ntiles;

#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const int64_t q = qbase + j * kThreads + tid;
        if (q >= m)
            continue;
#pragma unroll
        for (int i = 0; i < KP; ++i) {
            const int r = i - (KP - k);
            if (r >= 0) {
                const int64_t o = (static_cast<int64_t>(s) * k + r) * m + q;
                part_d2[o] = L[j][i];
                if (IDX) {
                    const int32_t v = idx_smem[(j * KP + i) * kThreads + tid];
                    part_idx[o] = v >= 0 ? ds.orig[v] : -1;
                }
            }
        }
    }
    return true;
}

// ---------------------------------------------------------------------------------------------
// Phase 1 over Z-ordered queries, one CTA per query block and no data splits. The CTA takes the
// bounding box of its queries, computes for every data tile a lower bound of the squared
// distance between the two boxes, sorts the tiles by it and, among equal bounds, by the distance
// between the box centres (bitonic sort in shared memory), and visits them in that order. After
// each tile it takes T = the largest k-th squared distance of its queries; it stops at the first
// tile whose bound exceeds T. Each warp (32 Q consecutive queries) also skips a tile whose bound
// to the warp's own box exceeds the warp's largest k-th distance, and, inside a tile, every
// 64-point sub-tile whose bound exceeds the k-th distance of each of its queries (knn_tile). No
// skipped point could enter a list: its exact FP32 distance is at least the box bound (the
// bound is shrunk by 2^-20 to cover rounding), which exceeds every affected query's current
// k-th distance.
// ---------------------------------------------------------------------------------------------

// Eq. 3-6 and the phase-2 parameters of one query from its k nearest squared distances d[0..k)
// (ascending, each offset by kEpsF32): r_obs as an FP32 pairwise sum of the distances, R, mu and
// alpha in FP64. Writes alpha to *alpha.
__device__ __forceinline__ QParamF32 select_params(const float *d, int k, double r_exp,
                                                   const AlphaMap &am, double *alpha_out)
{
    const float d1 = d[0];
    // Eq. 3: mean of the k distances; sqrt of (d2 - eps) undoes the coincidence offset.
    float v[AIDW_MAX_K];
    for (int r = 0; r < k; ++r)
        v[r] = __fsqrt_rn(__fsub_rn(d[r], kEpsF32));
    for (int stride = 1; stride < k; stride *= 2)
        for (int i = 0; i + stride < k; i += 2 * stride)
            v[i] = __fadd_rn(v[i], v[i + stride]);
    const double r_obs = static_cast<double>(v[0]) / k;
    const double R = r_obs / r_exp;           // Eq. 4
    const double mu = membership_eq5(R, am);  // Eq. 5
    const double alpha = alpha_eq6(mu, am);   // Eq. 6

    const float L1 = lg2_approx(d1);
    QParamF32 o;
    if (d1 == kEpsF32) {
        // Coincident query: weight 1 on every coincident point, 0 elsewhere.
        o.neg_s = -kCoincScaleF32;
        o.c = kCoincScaleF32 * L1;
    } else {
        const float sh = static_cast<float>(0.5 * alpha);
        o.neg_s = -sh;
        o.c = sh * L1;
    }
    *alpha_out = alpha;
    return o;
}

// Selection fused into a pruned phase-1 unit (one unit holds every list of its queries, so
// no merge is needed): Eq. 3-6 straight from the register lists, the phase-2 parameters to
// qparam[q] and alpha to out_alpha[perm[q]] (nullable); the lists themselves are not stored.
struct FusedSelect {
    double r_exp;
    AlphaMap am;
    QParamF32 *qparam;
    float *out_alpha;
    const uint32_t *perm;  // Z-order position -> caller's query index
};

// One query of a fused selection (kept out of line: it runs once per query, and inlined into
// the scan it would lengthen the scan's register life ranges).
static __device__ __noinline__ void fused_select_query(const float *d, int k,
                                                       const FusedSelect *fs, int64_t q)
{
    double alpha;
    fs->qparam[q] = select_params(d, k, fs->r_exp, fs->am, &alpha);
    if (fs->out_alpha)
        fs->out_alpha[fs->perm[q]] = static_cast<float>(alpha);
}

// ---------------------------------------------------------------------------------------------
// Phase 1 with one warp per query. A block of queries scans the data tiles near all of its
// queries together (knn_cull_unit); when the queries lie far apart compared with the data points
// (few queries, or many fewer queries than points) the block shares little, its warps scan the
// union of what each query needs, and a call with few queries leaves most SMs idle. Here a warp
// serves one query at a time: its 32 lanes hold the 32 smallest squared distances seen so far
// as a list sorted across the lanes (lane j the j-th smallest, with the point's stored
// position), scan 32 points per step with one point per lane, and take the points closer than
// the k-th entry: a few by shifting the larger entries up one lane each, more by a bitonic sort
// of the step's candidates and a bitonic merge with the list.
// The points are visited through the dataset's box hierarchy (warp_visit_boxes: 32-tile
// super-tiles, 512-point tiles, 64-point sub-tiles), nearest box first at every level, skipping
// every box whose bound exceeds the current k-th distance. The bounds are shrunk by 2^-20 for
// rounding as in knn_cull_unit, so no skipped point could enter the list: the k smallest values
// are those of a full scan. k <= 32.
// ---------------------------------------------------------------------------------------------
// Up to this many candidates in a step are inserted one at a time; more are sorted and merged.
constexpr int kWarpInsertMax = 6;

// Squared-distance lower bound from (qx, qy) to a box (xmin, ymin, xmax, ymax), shrunk for
// rounding; +inf for an empty box.
__device__ __forceinline__ float box_bound(float qx, float qy, float4 b)
{
    const float dx = fmaxf(0.0f, fmaxf(b.x - qx, qx - b.z));
    const float dy = fmaxf(0.0f, fmaxf(b.y - qy, qy - b.w));
    return __fmul_rn(__fmaf_rn(dx, dx, __fmul_rn(dy, dy)), kBoundShrink);
}

// Compare-exchange of a bitonic network across lanes: in an ascending run (up) the lower lane
// of each pair keeps the smaller entry. Equal entries stay where they are.
__device__ __forceinline__ void warp_cx(float &v, int32_t &i, int stride, bool up)
{
    const float ov = __shfl_xor_sync(kFullMask, v, stride);
    const int32_t oi = __shfl_xor_sync(kFullMask, i, stride);
    const bool lower = (threadIdx.x & stride) == 0;
    const bool take = (lower == up) ? (ov < v) : (ov > v);
    if (take) {
        v = ov;
        i = oi;
    }
}

// Points [p, p + 32) of the Z-ordered copy, one per lane, against the warp's list (ld, li) and
// its k-th entry thr (warp-uniform, updated).
__device__ __forceinline__ void warp_scan32(const float4 *__restrict__ nxy2, int64_t p, float qx,
                                            float qy, int k, float &ld, int32_t &li, float &thr)
{
    const int lane = threadIdx.x & 31;
    const float4 pt = nxy2[p + lane];
    const float d = dist2_neg(qx, qy, pt.x, pt.z);
    unsigned cand = __ballot_sync(kFullMask, d < thr);
    if (!cand)
        return;
    if (__popc(cand) <= kWarpInsertMax) {
        // Few candidates: each is inserted in turn by shifting the larger entries up one lane.
        while (cand) {
            const int src = __ffs(cand) - 1;
            cand &= cand - 1;
            const float c = __shfl_sync(kFullMask, d, src);
            if (!(c < thr))
                continue;
            const int32_t ci = static_cast<int32_t>(p + src);
            const float up = __shfl_up_sync(kFullMask, ld, 1);
            const int32_t upi = __shfl_up_sync(kFullMask, li, 1);
            if (!(ld <= c)) {
                const bool here = lane == 0 || up <= c;
                ld = here ? c : up;
                li = here ? ci : upi;
            }
            thr = __shfl_sync(kFullMask, ld, k - 1);
        }
        return;
    }
    const bool is_cand = (cand >> lane) & 1u;
    float v = is_cand ? d : CUDART_INF_F;
    int32_t vi = is_cand ? static_cast<int32_t>(p + lane) : -1;
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1)
            warp_cx(v, vi, stride, (lane & size) == 0);
    }
    // The 32 smallest of the two sorted lists, as a bitonic sequence, then sorted.
    const float rv = __shfl_sync(kFullMask, v, 31 - lane);
    const int32_t ri = __shfl_sync(kFullMask, vi, 31 - lane);
    if (rv < ld) {
        ld = rv;
        li = ri;
    }
#pragma unroll
    for (int stride = 16; stride > 0; stride >>= 1)
        warp_cx(ld, li, stride, true);
    thr = __shfl_sync(kFullMask, ld, k - 1);
}

// Visit key of a box for an FP32 query (make_visit_key); ~0 for an empty box.
__device__ __forceinline__ unsigned long long box_key(float qx, float qy, float4 b)
{
    const float cx = 0.5f * (b.x + b.z) - qx, cy = 0.5f * (b.y + b.w) - qy;
    return make_visit_key(box_bound(qx, qy, b), fmaf(cx, cx, cy * cy));
}

// The FP32 visitor of warp_visit_boxes: the warp's list (ld, li) and its k-th entry thr.
struct WarpKnnF32 {
    const float4 *nxy2;
    float qx, qy;
    int k;
    float ld;
    int32_t li;
    float thr;

    __device__ __forceinline__ unsigned long long key(float4 b) const
    {
        return box_key(qx, qy, b);
    }
    // A box may hold an entering point unless its bound exceeds the k-th distance.
    __device__ __forceinline__ bool open(unsigned long long key) const
    {
        return key != ~0ull && !(visit_key_bound(key) > thr);
    }
    __device__ __forceinline__ void scan(int64_t p)
    {
#pragma unroll
        for (int u = 0; u < kSubTile; u += 32)
            warp_scan32(nxy2, p + u, qx, qy, k, ld, li, thr);
    }
};

// The k nearest stored points of (qx, qy) by one warp: lanes 0..k-1 end holding the k smallest
// squared distances in ascending order (ld) and the points' stored positions (li).
__device__ __forceinline__ void warp_knn(const DatasetDev &ds, float qx, float qy, int k,
                                         float &ld, int32_t &li)
{
    WarpKnnF32 v{ds.nxy2, qx, qy, k, CUDART_INF_F, -1, CUDART_INF_F};
    warp_visit_boxes(ds, v);
    ld = v.ld;
    li = v.li;
}

// Shared-memory scratch of a pruned phase-1 unit.
struct CullShared {
    float red[4][kThreads / 32];
    float4 box;
    float thr;
    int issued;
};

// Phase-1 unit over one block of Z-ordered queries (qbase..), all data tiles, pruned as above.
// `order` holds ntiles_p2 (a power of two >= ntiles) 64-bit keys in shared memory. Returns false
// if a tile wait timed out (the error word is then set).
template <int KP, int Q, bool IDX>
__device__ __forceinline__ bool knn_cull_unit(const DatasetDev &ds, int64_t m, int64_t qbase,
                                              int ntiles, int ntiles_p2,
                                              const float *__restrict__ sqx,
                                              const float *__restrict__ sqy, int k,
                                              float *__restrict__ part_d2,
                                              int32_t *__restrict__ part_idx,
                                              int *__restrict__ err,
                                              float4 (*tile)[kTileF32Knn], TileSeq &ts,
                                              unsigned long long *order, int32_t *idx_smem,
                                              CullShared &cs,
                                              const FusedSelect *fsel = nullptr)
{
    constexpr int H = Q / 2;
    constexpr int W = kThreads / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float (*red)[W] = cs.red;

    float2 qxp[H], qyp[H], nthr[H];
    float L[Q][KP];
    float bx0 = CUDART_INF_F, by0 = CUDART_INF_F, bx1 = -CUDART_INF_F, by1 = -CUDART_INF_F;
    // Each warp takes 32 Q consecutive Z-ordered queries, so its queries have a compact box.
    const int64_t wbase = qbase + static_cast<int64_t>(warp) * 32 * Q + lane;
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const int64_t q = min(wbase + j * 32, m - 1);
        const float a = sqx[q], b = sqy[q];
        bx0 = fminf(bx0, a);
        by0 = fminf(by0, b);
        bx1 = fmaxf(bx1, a);
        by1 = fmaxf(by1, b);
        if (j & 1) {
            qxp[j / 2].y = a;
            qyp[j / 2].y = b;
        } else {
            qxp[j / 2].x = a;
            qyp[j / 2].x = b;
        }
#pragma unroll
        for (int i = 0; i < KP; ++i)
            L[j][i] = (i < KP - k) ? -CUDART_INF_F : CUDART_INF_F;
        if (IDX) {
#pragma unroll
            for (int i = 0; i < KP; ++i)
                idx_smem[(j * KP + i) * kThreads + tid] = -1;
        }
    }
#pragma unroll
    for (int h = 0; h < H; ++h)
        nthr[h] = make_float2(-CUDART_INF_F, -CUDART_INF_F);
    for (int o = 16; o > 0; o >>= 1) {
        bx0 = fminf(bx0, __shfl_xor_sync(0xffffffffu, bx0, o));
        by0 = fminf(by0, __shfl_xor_sync(0xffffffffu, by0, o));
        bx1 = fmaxf(bx1, __shfl_xor_sync(0xffffffffu, bx1, o));
        by1 = fmaxf(by1, __shfl_xor_sync(0xffffffffu, by1, o));
    }
    const float4 wb = make_float4(bx0, by0, bx1, by1);  // the warp's query box
    float wthr = CUDART_INF_F;                          // the warp's largest k-th distance
    if (lane == 0) {
        red[0][warp] = bx0;
        red[1][warp] = by0;
        red[2][warp] = bx1;
        red[3][warp] = by1;
    }
    __syncthreads();
    if (tid == 0) {
        float4 b = make_float4(red[0][0], red[1][0], red[2][0], red[3][0]);
        for (int w = 1; w < W; ++w) {
            b.x = fminf(b.x, red[0][w]);
            b.y = fminf(b.y, red[1][w]);
            b.z = fmaxf(b.z, red[2][w]);
            b.w = fmaxf(b.w, red[3][w]);
        }
        cs.box = b;
        cs.thr = CUDART_INF_F;
    }
    __syncthreads();
    const float4 qb = cs.box;
    const float qcx = 0.5f * (qb.x + qb.z), qcy = 0.5f * (qb.y + qb.w);
    // Lower bounds of the box-to-box squared distance, keyed for an ascending sort; among tiles
    // with equal bounds (in particular every tile that overlaps the query box, bound 0) the one
    // whose centre is nearest the query box's centre comes first, so the lists fill with near
    // points early and later tiles rarely insert. Key: bound (32 bits), centre distance
    // (the top 19 bits of its FP32 encoding), tile (13 bits).
    static_assert(kMaxCullTiles <= 8192, "13-bit tile field");
    for (int t = tid; t < ntiles_p2; t += kThreads) {
        unsigned long long key = ~0ull;
        if (t < ntiles) {
            const float4 tb = ds.tile_box[t];
            const float dx = fmaxf(0.0f, fmaxf(tb.x - qb.z, qb.x - tb.z));
            const float dy = fmaxf(0.0f, fmaxf(tb.y - qb.w, qb.y - tb.w));
            const float lb = __fmul_rn(__fmaf_rn(dx, dx, __fmul_rn(dy, dy)), kBoundShrink);
            const float cx = 0.5f * (tb.x + tb.z) - qcx, cy = 0.5f * (tb.y + tb.w) - qcy;
            const float cd = fminf(fmaf(cx, cx, cy * cy), 3.0e38f);  // finite, >= 0
            key = (static_cast<unsigned long long>(__float_as_uint(lb)) << 32) |
                  (static_cast<unsigned long long>(__float_as_uint(cd) >> 13) << 13) |
                  static_cast<unsigned long long>(t);
        }
        order[t] = key;
    }
    __syncthreads();
    for (int kk = 2; kk <= ntiles_p2; kk <<= 1) {
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < ntiles_p2; i += kThreads) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const unsigned long long a = order[i], b = order[ixj];
                    const bool up = (i & kk) == 0;
                    if ((a > b) == up) {
                        order[i] = b;
                        order[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }

    constexpr uint32_t kBytes = kTileF32Knn * sizeof(float4);
    if (tid == 0) {
        int issued = 0;
        for (; issued < 2 && issued < ntiles; ++issued) {
            const int64_t t = static_cast<int64_t>(order[issued] & 0x1fffull);
            const uint32_t b = (ts.seq + issued) & 1;
            mbar_arrive_expect_tx(&ts.bar[b], kBytes);
            tma_load_1d(tile[b], ds.nxy2 + t * kTileF32Knn, kBytes, &ts.bar[b]);
        }
        cs.issued = issued;
    }
    __syncthreads();
    int i = 0;
    bool ok = true;
    for (; i < ntiles; ++i) {
        const unsigned long long key = order[i];
        if (__uint_as_float(static_cast<uint32_t>(key >> 32)) > cs.thr)
            break;
        const uint32_t sq = ts.seq + i;
        const int b = sq & 1;
        const bool got = mbar_wait(&ts.bar[b], (sq >> 1) & 1);
        if (!__syncthreads_and(got)) {
            ok = false;
            break;
        }
        const int64_t t = static_cast<int64_t>(key & 0x1fffull);
        // A warp skips a tile that cannot reach any of its queries: the same bound as the
        // block's, from the warp's own box against its own k-th distances (warp-uniform).
        const float4 tb = ds.tile_box[t];
        const float wdx = fmaxf(0.0f, fmaxf(tb.x - wb.z, wb.x - tb.z));
        const float wdy = fmaxf(0.0f, fmaxf(tb.y - wb.w, wb.y - tb.w));
        const float wlb = __fmul_rn(__fmaf_rn(wdx, wdx, __fmul_rn(wdy, wdy)), kBoundShrink);
        if (!(wlb > wthr))
            knn_tile<KP, Q, IDX>(tile[b], t * kTileF32Knn, qxp, qyp, nthr, L, idx_smem,
                                 ds.sub_box + t * (kTileF32Knn / kSubTile));
        float mx = -CUDART_INF_F;
#pragma unroll
        for (int j = 0; j < Q; ++j)
            mx = fmaxf(mx, L[j][KP - 1]);
        for (int o = 16; o > 0; o >>= 1)
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        wthr = mx;
        if (lane == 0)
            red[0][warp] = mx;
        __syncthreads();
        if (tid == 0) {
            float v = red[0][0];
            for (int w = 1; w < W; ++w)
                v = fmaxf(v, red[0][w]);
            cs.thr = v;
            const int nx = i + 2;
            if (nx < ntiles &&
                __uint_as_float(static_cast<uint32_t>(order[nx] >> 32)) <= v) {
                const int64_t tn = static_cast<int64_t>(order[nx] & 0x1fffull);
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&ts.bar[b], kBytes);
                tma_load_1d(tile[b], ds.nxy2 + tn * kTileF32Knn, kBytes, &ts.bar[b]);
                cs.issued = nx + 1;
            }
        }
        __syncthreads();
    }
    // Wait (bounded) for tiles issued but not consumed before leaving.
    const int issued = cs.issued;
    if (tid == 0) {
        for (int u = i; u < issued; ++u) {
            const uint32_t sq = ts.seq + u;
            (void)mbar_wait(&ts.bar[sq & 1], (sq >> 1) & 1);
        }
        if (!ok)
            atomicOr(err, kErrTimeout);
    }
    ts.seq += issued;
    __syncthreads();
    if (!ok)
        return false;
    if (!IDX && fsel) {
        // The same k values, in the same order, as a one-split merge would read back.
        float d[Q][AIDW_MAX_K];
#pragma unroll
        for (int j = 0; j < Q; ++j) {
#pragma unroll
            for (int r0 = 0; r0 < KP; ++r0) {
                const int r = r0 - (KP - k);
                if (r >= 0)
                    d[j][r] = L[j][r0];
            }
        }
#pragma unroll 1
        for (int j = 0; j < Q; ++j) {
            const int64_t q = wbase + j * 32;
            if (q >= m)
                continue;
            fused_select_query(d[j], k, fsel, q);
        }
        return true;
    }
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const int64_t q = wbase + j * 32;
        if (q >= m)
            continue;
#pragma unroll
        for (int r0 = 0; r0 < KP; ++r0) {
            const int r = r0 - (KP - k);
            if (r >= 0) {
                const int64_t o = static_cast<int64_t>(r) * m + q;
                part_d2[o] = L[j][r0];
                if (IDX) {
                    const int32_t v = idx_smem[(j * KP + r0) * kThreads + tid];
                    part_idx[o] = v >= 0 ? ds.orig[v] : -1;
                }
            }
        }
    }
    return true;
}

// ---------------------------------------------------------------------------------------------
// Selection of one query: merge the S split lists (ties to the lower index), r_obs (Eq. 3) as an
// FP32 pairwise sum of the k distances, R (Eq. 4 with r_exp of Eq. 2), mu (Eq. 5) and alpha
// (Eq. 6) in FP64, then the phase-2 parameters. Split lists are read with L2-coherent loads so
// that a consumer on another SM sees a producer's results after the counter handshake.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void select_query(int64_t q, int64_t m, int S, int k, double r_exp,
                                             const AlphaMap &am, const float *part_d2,
                                             const int32_t *part_idx, QParamF32 *qp,
                                             float *out_alpha, int32_t *out_knn,
                                             const uint32_t *perm = nullptr)
{
    const int64_t qo = perm ? static_cast<int64_t>(perm[q]) : q;  // caller's query index
    int cur[kMaxSplits];
    float hd[kMaxSplits];
    int32_t hi[kMaxSplits];
    for (int s = 0; s < S; ++s) {
        cur[s] = 0;
        const int64_t o = static_cast<int64_t>(s) * k * m + q;
        hd[s] = __ldcg(part_d2 + o);
        hi[s] = part_idx ? __ldcg(part_idx + o) : 0;
    }
    float d[AIDW_MAX_K];
    for (int r = 0; r < k; ++r) {
        int bs = 0;
        for (int s = 1; s < S; ++s)
            if (hd[s] < hd[bs] || (hd[s] == hd[bs] && hi[s] < hi[bs]))
                bs = s;
        d[r] = hd[bs];
        if (out_knn)
            out_knn[qo * k + r] = hi[bs];
        if (++cur[bs] < k) {
            const int64_t o = (static_cast<int64_t>(bs) * k + cur[bs]) * m + q;
            hd[bs] = __ldcg(part_d2 + o);
            hi[bs] = part_idx ? __ldcg(part_idx + o) : 0;
        } else {
            hd[bs] = CUDART_INF_F;
            hi[bs] = INT32_MAX;
        }
    }
    double alpha;
    qp[q] = select_params(d, k, r_exp, am, &alpha);
    if (out_alpha)
        out_alpha[qo] = static_cast<float>(alpha);
}

// ---------------------------------------------------------------------------------------------
// Phase 2 unit: compensated sums of w and w z for Q * kThreads queries over [p_begin, p_end).
// Distances, power scale and both sums run as FP32x2 instructions on query pairs; lg2 and ex2
// run on the MUFU. w = 2^(s (L1 - log2 d2)) with s = alpha/2 and L1 = log2 of the nearest
// squared distance, i.e. (d1/d)^alpha <= 1: the ratio of Eq. 1 is unchanged and nothing
// overflows. Each thread sums kChunkW points per query in plain FP32 and merges the chunk sums
// by Kahan steps; the partial sums of the split go to part_sum[s][0..3][q]. Tiles of TW points
// hold whole chunks, so neither Q nor TW changes any query's sequence of operations. Chunks
// that hold only padding (from the first multiple of kChunkW at or above n) are not summed:
// they would add weights of exactly 0; tiles made of them are not loaded.
// ---------------------------------------------------------------------------------------------

// End of the summed chunks of a split [p_begin, p_end): the dataset's last real point rounded
// up to a whole chunk.
__device__ __forceinline__ int64_t weights_end(const DatasetDev &ds, int64_t p_end)
{
    return min(p_end, (ds.n + kChunkW - 1) / kChunkW * kChunkW);
}

// Tiles of TW points a phase-2 unit over [p_begin, p_end) loads.
template <int TW>
__device__ __forceinline__ int weights_tiles(const DatasetDev &ds, int64_t p_begin,
                                             int64_t p_end)
{
    const int64_t e = weights_end(ds, p_end);
    return e > p_begin ? static_cast<int>((e - p_begin + TW - 1) / TW) : 0;
}

template <int Q, int TW>
__device__ __forceinline__ bool weights_unit(const DatasetDev &ds, int64_t m, int64_t qbase,
                                             int64_t p_begin, int64_t p_end,
                                             const float *__restrict__ qx,
                                             const float *__restrict__ qy,
                                             const QParamF32 *qp, int s,
                                             float *__restrict__ part_sum,
                                             int *__restrict__ err,
                                             float4 (*txy)[TW],
                                             float2 (*tz)[TW], TileSeq &ts)
{
    static_assert(Q % 2 == 0, "queries are processed in packed pairs");
    static_assert(TW % kChunkW == 0 && kPadPoints % TW == 0, "whole chunks, whole tiles");
    constexpr int H = Q / 2;
    const int tid = threadIdx.x;
    const int ntiles = weights_tiles<TW>(ds, p_begin, p_end);
    const int64_t p_sum = weights_end(ds, p_end);

    float2 qxp[H], qyp[H], nsp[H], ccp[H];
    float hw[Q], cw[Q], hz[Q], cz[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const int64_t q = min(qbase + j * kThreads + tid, m - 1);
        const float2 o = __ldcg(reinterpret_cast<const float2 *>(qp + q));
        const float a = qx[q], b = qy[q];
        if (j & 1) {
            qxp[j / 2].y = a;
            qyp[j / 2].y = b;
            nsp[j / 2].y = o.x;
            ccp[j / 2].y = o.y;
        } else {
            qxp[j / 2].x = a;
            qyp[j / 2].x = b;
            nsp[j / 2].x = o.x;
            ccp[j / 2].x = o.y;
        }
        hw[j] = cw[j] = hz[j] = cz[j] = 0.0f;
    }
    const float2 eps2 = make_float2(kEpsF32, kEpsF32);

    constexpr uint32_t kBxy = TW * sizeof(float4);
    constexpr uint32_t kBz = TW * sizeof(float2);
    if (tid == 0) {
        for (int t = 0; t < 2 && t < ntiles; ++t) {
            const uint32_t b = (ts.seq + t) & 1;
            const int64_t o = p_begin + static_cast<int64_t>(t) * TW;
            mbar_arrive_expect_tx(&ts.bar[b], kBxy + kBz);
            tma_load_1d(txy[b], ds.nxy2 + o, kBxy, &ts.bar[b]);
            tma_load_1d(tz[b], ds.zz + o, kBz, &ts.bar[b]);
        }
    }

    for (int t = 0; t < ntiles; ++t) {
        const uint32_t sq = ts.seq + t;
        const int b = sq & 1;
        const bool got = mbar_wait(&ts.bar[b], (sq >> 1) & 1);
        if (!__syncthreads_and(got)) {
            if (tid == 0) {
                atomicOr(err, kErrTimeout);
                drain(ts, t, ntiles);
            }
            ts.seq += ntiles;
            return false;
        }
        const int64_t t0 = p_begin + static_cast<int64_t>(t) * TW;
        const int cend = static_cast<int>(min(static_cast<int64_t>(TW), p_sum - t0));
        for (int c = 0; c < cend; c += kChunkW) {
            float2 sw[H], sz[H];
#pragma unroll
            for (int h = 0; h < H; ++h)
                sw[h] = sz[h] = make_float2(0.0f, 0.0f);
            // The whole chunk unrolled (measured: 355 ms at 1M x 1M against 357-359 ms for
            // steps of 4, 8 or 16 points, with 70 registers instead of 80).
#pragma unroll
            for (int u = 0; u < kChunkW; ++u) {
                const float4 p = txy[b][c + u];
                const float2 zz = tz[b][c + u];
#pragma unroll
                for (int h = 0; h < H; ++h) {
                    const float2 dx = __fadd2_rn(qxp[h], make_float2(p.x, p.y));
                    const float2 dy = __fadd2_rn(qyp[h], make_float2(p.z, p.w));
                    const float2 d2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, eps2));
                    const float2 lg = make_float2(lg2_approx(d2.x), lg2_approx(d2.y));
                    const float2 e = __ffma2_rn(lg, nsp[h], ccp[h]);
                    const float2 w = make_float2(ex2_approx(e.x), ex2_approx(e.y));
                    sw[h] = __fadd2_rn(sw[h], w);
                    sz[h] = __ffma2_rn(w, zz, sz[h]);
                }
            }
#pragma unroll
            for (int h = 0; h < H; ++h) {
                kahan_add(hw[2 * h], cw[2 * h], sw[h].x);
                kahan_add(hw[2 * h + 1], cw[2 * h + 1], sw[h].y);
                kahan_add(hz[2 * h], cz[2 * h], sz[h].x);
                kahan_add(hz[2 * h + 1], cz[2 * h + 1], sz[h].y);
            }
        }
        __syncthreads();
        if (tid == 0 && t + 2 < ntiles) {
            fence_proxy_async_smem();
            const int64_t o = p_begin + static_cast<int64_t>(t + 2) * TW;
            mbar_arrive_expect_tx(&ts.bar[b], kBxy + kBz);
            tma_load_1d(txy[b], ds.nxy2 + o, kBxy, &ts.bar[b]);
            tma_load_1d(tz[b], ds.zz + o, kBz, &ts.bar[b]);
        }
    }
    ts.seq += ntiles;
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const int64_t q = qbase + j * kThreads + tid;
        if (q >= m)
            continue;
        float *o = part_sum + static_cast<int64_t>(s) * 4 * m + q;
        o[0] = hw[j];
        o[m] = -cw[j];
        o[2 * m] = hz[j];
        o[3 * m] = -cz[j];
    }
    return true;
}

// Eq. 1 for one query: merge the S splits' compensated sums in FP64 and divide.
__device__ __forceinline__ float finalize_query(int64_t q, int64_t m, int S,
                                                const float *part_sum)
{
    double W = 0.0, WZ = 0.0;
    for (int s = 0; s < S; ++s) {
        const float *o = part_sum + static_cast<int64_t>(s) * 4 * m + q;
        W += static_cast<double>(__ldcg(o)) + static_cast<double>(__ldcg(o + m));
        WZ += static_cast<double>(__ldcg(o + 2 * m)) + static_cast<double>(__ldcg(o + 3 * m));
    }
    return static_cast<float>(WZ / W);
}

// Shared-memory barrier set-up common to every kernel that streams tiles.
__device__ __forceinline__ void init_tile_barriers(uint64_t *bar)
{
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
}

template <int KP>
constexpr int knn_q()
{
    return KP <= 16 ? 4 : 2;
}

// Register list length for k: the smallest of 8, 12, 16, 32 that holds k and kp_min.
__host__ __device__ inline int kp_for(int k, int kp_min = 0)
{
    const int v = k > kp_min ? k : kp_min;
    return v <= 8 ? 8 : (v <= 12 ? 12 : (v <= 16 ? 16 : 32));
}

}  // namespace f32dev
}  // namespace aidw
