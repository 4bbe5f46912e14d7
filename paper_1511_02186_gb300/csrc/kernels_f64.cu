// FP64 kernels of the AIDW hot path for sm_103a: the same two scans as the FP32 path with
// every step at double precision or finer (Sec. 3.2.1 builds its kernels for float and double
// alike; phase 2's log2, exp2 and sum of the weights run in 62-bit fixed point, f64_math.cuh).
// Squared distances of phase 1 are formed as dx*dx + dy*dy with each product and sum rounded
// separately, so neighbour lists agree bit for bit with a reference that evaluates the same
// expression in IEEE double without fused multiply-add. Ties go to the lower index. Both
// phase-1 scans put an FP32 prefilter in front of those exact distances (prefilter_thr): a
// 16-point chunk is scanned exactly only when one of its FP32 distances could be within the
// query's k-th distance, which keeps the lists exact while most pairs cost FP32 work only.
#include <math_constants.h>

#include <algorithm>

#include "aidw_internal.cuh"
#include "f64_math.cuh"
#include "warp_knn.cuh"

namespace aidw {
namespace {

constexpr int kChunkKnn = 16;
constexpr int kChunkW = 32;
// FP64 phase-2 queries per thread (8,192 x 1M with 256-thread CTAs: 104.6 ms with 2, 109.0 ms
// with 4, 161.8 ms with 8)
constexpr int kQW64 = 2;
constexpr int kTileW64 = 256;  // FP64 phase-2 tile (points), beside 72 KB of tables
// FP64 phase-2 CTA: 16 warps share one copy of the tables, one CTA per SM by registers (72 a
// thread): the integer steps of log2 / exp2 are long dependent chains that need the warps
// (8,192 x 1M: 101.7 ms; two CTAs of 256 threads per SM 104.6 ms, one of 768 threads 109.6 ms).
constexpr int kThreadsW64 = 512;

__device__ __forceinline__ double dist2_exact(double qx, double qy, double px, double py)
{
    const double dx = __dsub_rn(qx, px);
    const double dy = __dsub_rn(qy, py);
    return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
}

__device__ __forceinline__ double dist2_eps(double qx, double qy, double px, double py)
{
    const double dx = __dsub_rn(qx, px);
    const double dy = __dsub_rn(qy, py);
    return __fma_rn(dx, dx, __fma_rn(dy, dy, kEpsF64));
}

template <int KP>
__device__ __forceinline__ void list_insert(double (&L)[KP], double v)
{
    L[KP - 1] = v;
#pragma unroll
    for (int i = KP - 1; i > 0; --i) {
        const double a = L[i - 1], b = L[i];
        L[i - 1] = fmin(a, b);
        L[i] = fmax(a, b);
    }
}

template <int KP>
__device__ __forceinline__ void index_insert(const double (&L)[KP], int32_t *base, double v,
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

__device__ __forceinline__ void drain(uint64_t *bar, int t, int ntiles)
{
    for (int u = t; u < ntiles && u < t + 2; ++u)
        (void)mbar_wait(&bar[u & 1], (u >> 1) & 1);
}

// FP32 prefilter of the exact FP64 phase-1 scans. Coordinates are taken relative to a centre c
// and rounded to float. With a = q - c and d the exact distance, the FP32 distance d_f of the
// rounded coordinates is at least d - 2^-22.5 d - 2^-22.9 |a| (two roundings of each coordinate,
// one of each difference, one of the sum of squares), so d <= sqrt(T) implies
// d_f^2 <= (sqrt(T) (1 + 2^-21) + |a| 2^-21)^2: a chunk whose FP32 distances all exceed that holds
// no point that could enter a list whose k-th squared distance is T, and skips the exact FP64
// distances (lists are unchanged).
__device__ __forceinline__ float prefilter_thr(double kth, double ra)
{
    const double b = fma(sqrt(kth), 1.0 + 0x1p-21, ra * 0x1p-21);
    return __double2float_ru(b * b);
}

template <int KP, int Q, bool IDX>
__global__ void __launch_bounds__(kThreads)
f64_knn_kernel(DatasetDev ds, int64_t m, PassPlan pp, const double *__restrict__ qx,
               const double *__restrict__ qy, int k, double *__restrict__ part_d2,
               int32_t *__restrict__ part_idx, int *__restrict__ err)
{
    __shared__ __align__(128) double2 tile[2][kTileF64Knn];
    __shared__ __align__(16) float2 tilef[kTileF64Knn];  // tile points - c, FP32 (prefilter)
    __shared__ __align__(8) uint64_t bar[2];
    extern __shared__ int32_t idx_smem[];

    const int tid = threadIdx.x;
    const int s = blockIdx.y;
    const int64_t qbase = static_cast<int64_t>(blockIdx.x) * pp.q_per_block;
    const int64_t p_begin = static_cast<int64_t>(s) * pp.split_len;
    const int64_t p_end = min(p_begin + pp.split_len, ds.n_pad);
    const int ntiles = static_cast<int>((p_end - p_begin) / kTileF64Knn);
    const float4 dbox = *ds.box;  // the prefilter's centre: the dataset box's
    const double ccx = 0.5 * (static_cast<double>(dbox.x) + static_cast<double>(dbox.z));
    const double ccy = 0.5 * (static_cast<double>(dbox.y) + static_cast<double>(dbox.w));

    double qxr[Q], qyr[Q], ra[Q];
    float2 qf[Q];
    float thr[Q];
    double L[Q][KP];
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const int64_t q = min(qbase + j * kThreads + tid, m - 1);
        qxr[j] = qx[q];
        qyr[j] = qy[q];
        const double ax = qxr[j] - ccx, ay = qyr[j] - ccy;
        qf[j] = make_float2(static_cast<float>(ax), static_cast<float>(ay));
        ra[j] = sqrt(ax * ax + ay * ay);
        thr[j] = CUDART_INF_F;
#pragma unroll
        for (int i = 0; i < KP; ++i)
            L[j][i] = (i < KP - k) ? -CUDART_INF : CUDART_INF;
        if (IDX) {
#pragma unroll
            for (int i = 0; i < KP; ++i)
                idx_smem[(j * KP + i) * kThreads + tid] = -1;
        }
    }
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    constexpr uint32_t kBytes = kTileF64Knn * sizeof(double2);
    if (tid == 0) {
        for (int t = 0; t < 2 && t < ntiles; ++t) {
            mbar_arrive_expect_tx(&bar[t], kBytes);
            tma_load_1d(tile[t], ds.xy64 + p_begin + static_cast<int64_t>(t) * kTileF64Knn,
                        kBytes, &bar[t]);
        }
    }
    bool ok = true;
    for (int t = 0; t < ntiles; ++t) {
        const int b = t & 1;
        const bool got = mbar_wait(&bar[b], (t >> 1) & 1);
        if (!__syncthreads_and(got)) {
            ok = false;
            if (tid == 0) {
                atomicOr(err, kErrTimeout);
                drain(bar, t, ntiles);
            }
            break;
        }
        const int64_t pbase = p_begin + static_cast<int64_t>(t) * kTileF64Knn;
        for (int u = tid; u < kTileF64Knn; u += kThreads) {
            const double2 p = tile[b][u];
            tilef[u] = make_float2(static_cast<float>(p.x - ccx), static_cast<float>(p.y - ccy));
        }
        __syncthreads();
        for (int c = 0; c < kTileF64Knn; c += kChunkKnn) {
            float mn[Q];
#pragma unroll
            for (int j = 0; j < Q; ++j)
                mn[j] = CUDART_INF_F;
#pragma unroll
            for (int u = 0; u < kChunkKnn; ++u) {
                const float2 p = tilef[c + u];
#pragma unroll
                for (int j = 0; j < Q; ++j) {
                    const float dx = qf[j].x - p.x, dy = qf[j].y - p.y;
                    mn[j] = fminf(mn[j], fmaf(dx, dx, dy * dy));
                }
            }
#pragma unroll
            for (int j = 0; j < Q; ++j) {
                if (!(mn[j] <= thr[j]))  // (a padding point's FP32 distance is +inf)
                    continue;
                bool changed = false;
#pragma unroll 1
                for (int u = 0; u < kChunkKnn; ++u) {
                    const double2 p = tile[b][c + u];
                    const double d = dist2_exact(qxr[j], qyr[j], p.x, p.y);
                    if (d < L[j][KP - 1]) {
                        if (IDX)
                            index_insert<KP>(L[j], idx_smem + j * KP * kThreads + tid, d,
                                             static_cast<int32_t>(pbase + c + u));
                        list_insert<KP>(L[j], d);
                        changed = true;
                    }
                }
                if (changed)
                    thr[j] = prefilter_thr(L[j][KP - 1], ra[j]);
            }
        }
        __syncthreads();
        if (tid == 0 && t + 2 < ntiles) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bar[b], kBytes);
            tma_load_1d(tile[b], ds.xy64 + pbase + 2 * kTileF64Knn, kBytes, &bar[b]);
        }
    }
    if (!ok)
        return;
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
                if (IDX)
                    part_idx[o] = idx_smem[(j * KP + i) * kThreads + tid];
            }
        }
    }
}

// ---------------------------------------------------------------------------------------------
// Phase 1 over Z-ordered FP64 queries, pruned as the FP32 path's (one CTA per query block, data
// tiles visited in order of a lower bound of the box-to-box distance, nearest centre first among
// equal bounds, the block stopping at the first tile beyond its queries' largest k-th distance,
// each warp skipping tiles beyond its own). Without the kNN output it keeps distances only (the
// k nearest distances, and so r_obs, do not depend on which of two tied points is kept); with
// it, it keeps the k smallest pairs (distance, caller index), i.e. ties to the lower index as
// the caller-order scan with strict "<" has them. A tile's points are gathered from
// the caller-order FP64 copy through the Z-order map. The tile boxes hold the FP32 coordinates;
// widened by 2^-23 of their largest magnitude they contain the FP64 points (FP32 rounding moves a
// coordinate by at most 2^-24 of it), and the bound is shrunk by 2^-50 to cover its own rounding
// and that of the exact distance, so no skipped point could have entered a list. Inside a
// visited tile the FP32 prefilter (centre: the block's query box) decides which chunks get the
// exact distances.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ double box_bound64(float4 tb, double qx0, double qy0, double qx1,
                                              double qy1)
{
    const double bx0 = tb.x, by0 = tb.y, bx1 = tb.z, by1 = tb.w;
    const double mag = fmax(fmax(fabs(bx0), fabs(bx1)), fmax(fabs(by0), fabs(by1)));
    const double d = mag * 0x1p-23 + 0x1p-140;
    const double dx = fmax(0.0, fmax((bx0 - d) - qx1, qx0 - (bx1 + d)));
    const double dy = fmax(0.0, fmax((by0 - d) - qy1, qy0 - (by1 + d)));
    return (dx * dx + dy * dy) * (1.0 - 0x1p-50);
}

// Lexicographic insertion of (v, vi) into the ascending (distance, index) register lists of one
// query: the k smallest pairs, so that ties go to the lower caller index as in the scan order.
template <int KP>
__device__ __forceinline__ void pair_insert(double (&L)[KP], int32_t (&I)[KP], double v,
                                            int32_t vi)
{
#pragma unroll
    for (int j = 0; j < KP; ++j) {
        const bool lt = v < L[j] || (v == L[j] && vi < I[j]);
        const double lo = lt ? v : L[j];
        const int32_t loi = lt ? vi : I[j];
        v = lt ? L[j] : v;
        vi = lt ? I[j] : vi;
        L[j] = lo;
        I[j] = loi;
    }
}

template <int KP, int Q, bool IDX>
__global__ void __launch_bounds__(kThreads)
f64_knn_cull_kernel(DatasetDev ds, int64_t m, int qpb, int ntiles, int ntiles_p2,
                    const double *__restrict__ sqx, const double *__restrict__ sqy, int k,
                    double *__restrict__ part_d2, int32_t *__restrict__ part_idx)
{
    extern __shared__ unsigned long long order[];  // [ntiles_p2] sort keys
    __shared__ __align__(16) double2 tile[kTileF32Knn];
    __shared__ __align__(16) float2 tilef[kTileF32Knn];  // tile points - block centre, FP32
    __shared__ int32_t tidx[IDX ? kTileF32Knn : 1];  // caller index of each tile point
    constexpr int W = kThreads / 32;
    __shared__ double red[4][W];
    __shared__ double sbox[4];
    __shared__ double sthr;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t qbase = static_cast<int64_t>(blockIdx.x) * qpb;
    const int64_t wbase = qbase + static_cast<int64_t>(warp) * 32 * Q + lane;

    double qxr[Q], qyr[Q];
    double L[Q][KP];
    int32_t I[Q][IDX ? KP : 1];
    double bx0 = CUDART_INF, by0 = CUDART_INF, bx1 = -CUDART_INF, by1 = -CUDART_INF;
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const int64_t q = min(wbase + j * 32, m - 1);
        qxr[j] = sqx[q];
        qyr[j] = sqy[q];
        bx0 = fmin(bx0, qxr[j]);
        by0 = fmin(by0, qyr[j]);
        bx1 = fmax(bx1, qxr[j]);
        by1 = fmax(by1, qyr[j]);
#pragma unroll
        for (int i = 0; i < KP; ++i) {
            L[j][i] = (i < KP - k) ? -CUDART_INF : CUDART_INF;
            if constexpr (IDX)
                I[j][i] = (i < KP - k) ? -1 : INT32_MAX;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        bx0 = fmin(bx0, __shfl_xor_sync(0xffffffffu, bx0, o));
        by0 = fmin(by0, __shfl_xor_sync(0xffffffffu, by0, o));
        bx1 = fmax(bx1, __shfl_xor_sync(0xffffffffu, bx1, o));
        by1 = fmax(by1, __shfl_xor_sync(0xffffffffu, by1, o));
    }
    const double wx0 = bx0, wy0 = by0, wx1 = bx1, wy1 = by1;  // the warp's query box
    double wthr = CUDART_INF;
    if (lane == 0) {
        red[0][warp] = bx0;
        red[1][warp] = by0;
        red[2][warp] = bx1;
        red[3][warp] = by1;
    }
    __syncthreads();
    if (tid == 0) {
        double b0 = red[0][0], b1 = red[1][0], b2 = red[2][0], b3 = red[3][0];
        for (int w = 1; w < W; ++w) {
            b0 = fmin(b0, red[0][w]);
            b1 = fmin(b1, red[1][w]);
            b2 = fmax(b2, red[2][w]);
            b3 = fmax(b3, red[3][w]);
        }
        sbox[0] = b0;
        sbox[1] = b1;
        sbox[2] = b2;
        sbox[3] = b3;
        sthr = CUDART_INF;
    }
    __syncthreads();
    const double qx0 = sbox[0], qy0 = sbox[1], qx1 = sbox[2], qy1 = sbox[3];
    const double ccx = 0.5 * (qx0 + qx1), ccy = 0.5 * (qy0 + qy1);
    const float qcx = static_cast<float>(ccx);
    const float qcy = static_cast<float>(ccy);
    // FP32 prefilter (prefilter_thr) with the block's centre as c.
    float2 qf[Q];
    double ra[Q];
    float thr[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const double ax = qxr[j] - ccx, ay = qyr[j] - ccy;
        qf[j] = make_float2(static_cast<float>(ax), static_cast<float>(ay));
        ra[j] = sqrt(ax * ax + ay * ay);
        thr[j] = CUDART_INF_F;
    }
    // Keys: bound rounded down to FP32 (32 bits), centre distance (19 bits), tile (13 bits).
    for (int t = tid; t < ntiles_p2; t += kThreads) {
        unsigned long long key = ~0ull;
        if (t < ntiles) {
            const float4 tb = ds.tile_box[t];
            const float lb = __double2float_rd(box_bound64(tb, qx0, qy0, qx1, qy1));
            const float cx = 0.5f * (tb.x + tb.z) - qcx, cy = 0.5f * (tb.y + tb.w) - qcy;
            const float cd = fminf(fmaf(cx, cx, cy * cy), 3.0e38f);
            key = (static_cast<unsigned long long>(__float_as_uint(fmaxf(lb, 0.0f))) << 32) |
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

    for (int i = 0; i < ntiles; ++i) {
        const unsigned long long key = order[i];
        if (static_cast<double>(__uint_as_float(static_cast<uint32_t>(key >> 32))) > sthr)
            break;
        const int64_t t = static_cast<int64_t>(key & 0x1fffull);
        for (int u = tid; u < kTileF32Knn; u += kThreads) {
            const int32_t o = ds.orig[t * kTileF32Knn + u];
            const double2 p = o >= 0 ? ds.xy64[o] : make_double2(CUDART_INF, CUDART_INF);
            tile[u] = p;
            tilef[u] = make_float2(static_cast<float>(p.x - ccx), static_cast<float>(p.y - ccy));
            if (IDX)
                tidx[u] = o;
        }
        __syncthreads();
        const double wlb = box_bound64(ds.tile_box[t], wx0, wy0, wx1, wy1);
        if (!(wlb > wthr)) {  // a tie needs d == wthr, and the bound is strictly below d
            for (int c = 0; c < kTileF32Knn; c += kChunkKnn) {
                float mn[Q];
#pragma unroll
                for (int j = 0; j < Q; ++j)
                    mn[j] = CUDART_INF_F;
#pragma unroll
                for (int u = 0; u < kChunkKnn; ++u) {
                    const float2 p = tilef[c + u];
#pragma unroll
                    for (int j = 0; j < Q; ++j) {
                        const float dx = qf[j].x - p.x, dy = qf[j].y - p.y;
                        mn[j] = fminf(mn[j], fmaf(dx, dx, dy * dy));
                    }
                }
#pragma unroll
                for (int j = 0; j < Q; ++j) {
                    if (!(mn[j] <= thr[j]))  // (a padding point's FP32 distance is +inf or NaN)
                        continue;
                    // The exact scan of the chunk; with indices a tie with the k-th distance may
                    // still enter (lower index).
                    bool changed = false;
#pragma unroll 1
                    for (int u = 0; u < kChunkKnn; ++u) {
                        const double2 p = tile[c + u];
                        const double d = dist2_exact(qxr[j], qyr[j], p.x, p.y);
                        if constexpr (IDX) {
                            const int32_t id = tidx[c + u];
                            if (d < L[j][KP - 1] || (d == L[j][KP - 1] && id < I[j][KP - 1])) {
                                pair_insert<KP>(L[j], I[j], d, id);
                                changed = true;
                            }
                        } else if (d < L[j][KP - 1]) {
                            list_insert<KP>(L[j], d);
                            changed = true;
                        }
                    }
                    if (changed)
                        thr[j] = prefilter_thr(L[j][KP - 1], ra[j]);
                }
            }
        }
        double mx = -CUDART_INF;
#pragma unroll
        for (int j = 0; j < Q; ++j)
            mx = fmax(mx, L[j][KP - 1]);
        for (int o = 16; o > 0; o >>= 1)
            mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        wthr = mx;
        if (lane == 0)
            red[0][warp] = mx;
        __syncthreads();
        if (tid == 0) {
            double v = red[0][0];
            for (int w = 1; w < W; ++w)
                v = fmax(v, red[0][w]);
            sthr = v;
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const int64_t q = wbase + j * 32;
        if (q >= m)
            continue;
#pragma unroll
        for (int i = 0; i < KP; ++i) {
            const int r = i - (KP - k);
            if (r >= 0) {
                part_d2[static_cast<int64_t>(r) * m + q] = L[j][i];
                if constexpr (IDX)
                    part_idx[static_cast<int64_t>(r) * m + q] = I[j][i];
            }
        }
    }
}

// ---------------------------------------------------------------------------------------------
// FP64 phase 1 with one warp per query (the FP32 form is in f32_device.cuh): the warp's lanes
// hold the k smallest (distance, caller index) pairs seen so far as a list sorted across the
// lanes, 32 points are scanned per step (one per lane, read from the FP64 copy through the
// Z-order map, exact distance as in the other FP64 scans), and the points that precede the k-th
// entry are inserted one at a time when they are few, else sorted and merged. The pairs order by
// distance, then caller index, so the lists are the k smallest pairs whatever the visit order:
// those of the caller-order scan, ties going to the lower index. Boxes are walked by
// warp_visit_boxes with FP64 bounds from the FP32 boxes widened for rounding (box_bound64).
// ---------------------------------------------------------------------------------------------
constexpr int kWarpInsertMax64 = 6;

// (a, ai) precedes (b, bi): smaller distance, or equal distance and lower caller index.
__device__ __forceinline__ bool pair_lt(double a, int32_t ai, double b, int32_t bi)
{
    return a < b || (a == b && ai < bi);
}

// Compare-exchange of a bitonic network across lanes on (distance, index) pairs.
__device__ __forceinline__ void warp_cx64(double &v, int32_t &i, int stride, bool up)
{
    const double ov = __shfl_xor_sync(kFullMask, v, stride);
    const int32_t oi = __shfl_xor_sync(kFullMask, i, stride);
    const bool lower = (threadIdx.x & stride) == 0;
    const bool take = (lower == up) ? pair_lt(ov, oi, v, i) : pair_lt(v, i, ov, oi);
    if (take) {
        v = ov;
        i = oi;
    }
}

// The FP64 visitor of warp_visit_boxes. Empty list entries and padding points are
// (+inf, INT32_MAX), which no pair precedes.
struct WarpKnnF64 {
    const int32_t *orig;
    const double2 *xy64;
    double qx, qy;
    float qxf, qyf;
    int k;
    double ld;     // this lane's list entry
    int32_t li;
    double thr;    // the k-th entry (warp-uniform)
    int32_t thi;

    __device__ __forceinline__ unsigned long long key(float4 b) const
    {
        if (!(b.x <= b.z))
            return ~0ull;  // empty box
        const float lb = __double2float_rd(box_bound64(b, qx, qy, qx, qy));
        const float cx = 0.5f * (b.x + b.z) - qxf, cy = 0.5f * (b.y + b.w) - qyf;
        return make_visit_key(lb, fmaf(cx, cx, cy * cy));
    }
    // The bound is below every distance in the box, so a box whose bound exceeds the k-th
    // distance holds no point that precedes the k-th pair, even at a tie.
    __device__ __forceinline__ bool open(unsigned long long key) const
    {
        return key != ~0ull && !(static_cast<double>(visit_key_bound(key)) > thr);
    }
    __device__ __forceinline__ void scan(int64_t p)
    {
#pragma unroll
        for (int u = 0; u < kSubTile; u += 32)
            scan32(p + u);
    }
    __device__ __forceinline__ void scan32(int64_t p)
    {
        const int lane = threadIdx.x & 31;
        const int32_t o = orig[p + lane];
        double d = CUDART_INF;
        int32_t id = INT32_MAX;
        if (o >= 0) {
            const double2 pt = xy64[o];
            d = dist2_exact(qx, qy, pt.x, pt.y);
            id = o;
        }
        unsigned cand = __ballot_sync(kFullMask, pair_lt(d, id, thr, thi));
        if (!cand)
            return;
        if (__popc(cand) <= kWarpInsertMax64) {
            while (cand) {
                const int src = __ffs(cand) - 1;
                cand &= cand - 1;
                const double c = __shfl_sync(kFullMask, d, src);
                const int32_t ci = __shfl_sync(kFullMask, id, src);
                if (!pair_lt(c, ci, thr, thi))
                    continue;
                const double up = __shfl_up_sync(kFullMask, ld, 1);
                const int32_t upi = __shfl_up_sync(kFullMask, li, 1);
                if (pair_lt(c, ci, ld, li)) {
                    const bool here = lane == 0 || pair_lt(up, upi, c, ci);
                    ld = here ? c : up;
                    li = here ? ci : upi;
                }
                thr = __shfl_sync(kFullMask, ld, k - 1);
                thi = __shfl_sync(kFullMask, li, k - 1);
            }
            return;
        }
        const bool is_cand = (cand >> lane) & 1u;
        double v = is_cand ? d : CUDART_INF;
        int32_t vi = is_cand ? id : INT32_MAX;
#pragma unroll
        for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
            for (int stride = size >> 1; stride > 0; stride >>= 1)
                warp_cx64(v, vi, stride, (lane & size) == 0);
        }
        // The 32 smallest of the two sorted lists, as a bitonic sequence, then sorted.
        const double rv = __shfl_sync(kFullMask, v, 31 - lane);
        const int32_t ri = __shfl_sync(kFullMask, vi, 31 - lane);
        if (pair_lt(rv, ri, ld, li)) {
            ld = rv;
            li = ri;
        }
#pragma unroll
        for (int stride = 16; stride > 0; stride >>= 1)
            warp_cx64(ld, li, stride, true);
        thr = __shfl_sync(kFullMask, ld, k - 1);
        thi = __shfl_sync(kFullMask, li, k - 1);
    }
};

// One warp per query (grid-stride over the queries, caller order); writes one split's lists
// [k][m] (distances, and caller indices when part_idx is not null) for f64_select_kernel.
__global__ void __launch_bounds__(kThreads)
f64_knn_warp_kernel(DatasetDev ds, int64_t m, const double *__restrict__ qx,
                    const double *__restrict__ qy, int k, double *__restrict__ part_d2,
                    int32_t *__restrict__ part_idx)
{
    constexpr int W = kThreads / 32;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = static_cast<int64_t>(gridDim.x) * W;
    for (int64_t q = static_cast<int64_t>(blockIdx.x) * W + (threadIdx.x >> 5); q < m;
         q += nwarps) {
        const double x = qx[q], y = qy[q];
        WarpKnnF64 v{ds.orig, ds.xy64, x, y, static_cast<float>(x), static_cast<float>(y), k,
                     CUDART_INF, INT32_MAX, CUDART_INF, INT32_MAX};
        warp_visit_boxes(ds, v);
        if (lane < k) {
            part_d2[static_cast<int64_t>(lane) * m + q] = v.ld;
            if (part_idx)
                part_idx[static_cast<int64_t>(lane) * m + q] = v.li;
        }
    }
}

__global__ void __launch_bounds__(256)
f64_select_kernel(int64_t m, int S, int k, double r_exp, AlphaMap am,
                  const double *__restrict__ part_d2, const int32_t *__restrict__ part_idx,
                  QParamF64 *__restrict__ qp, float *__restrict__ out_alpha,
                  int32_t *__restrict__ out_knn, const uint32_t *__restrict__ perm,
                  bool x_params)
{
    const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q >= m)
        return;
    int cur[kMaxSplits];
    double hd[kMaxSplits];
    int32_t hi[kMaxSplits];
    for (int s = 0; s < S; ++s) {
        cur[s] = 0;
        const int64_t o = static_cast<int64_t>(s) * k * m + q;
        hd[s] = part_d2[o];
        hi[s] = part_idx ? part_idx[o] : 0;
    }
    double r_sum = 0.0, d1 = 0.0;
    for (int r = 0; r < k; ++r) {
        int bs = 0;
        for (int s = 1; s < S; ++s)
            if (hd[s] < hd[bs] || (hd[s] == hd[bs] && hi[s] < hi[bs]))
                bs = s;
        if (r == 0)
            d1 = hd[bs];
        r_sum = __dadd_rn(r_sum, __dsqrt_rn(hd[bs]));  // Eq. 3, ascending order
        if (out_knn)
            out_knn[(perm ? static_cast<int64_t>(perm[q]) : q) * k + r] = hi[bs];
        if (++cur[bs] < k) {
            const int64_t o = (static_cast<int64_t>(bs) * k + cur[bs]) * m + q;
            hd[bs] = part_d2[o];
            hi[bs] = part_idx ? part_idx[o] : 0;
        } else {
            hd[bs] = CUDART_INF;
            hi[bs] = INT32_MAX;
        }
    }
    const double r_obs = r_sum / k;
    const double R = r_obs / r_exp;           // Eq. 4
    const double mu = membership_eq5(R, am);  // Eq. 5
    const double alpha = alpha_eq6(mu, am);   // Eq. 6
    if (out_alpha)
        out_alpha[perm ? perm[q] : q] = static_cast<float>(alpha);
    if (x_params) {
        // AIDW_F64X: kappa kept within [2^-100, 2^100] (beyond, the weights are those of the
        // bounds to far below the tolerance: all equal, or only the nearest points') and the
        // reference squared distance.
        QParamF64X x;
        x.kappa = d1 == 0.0 ? kCoincScaleDf
                            : fmax(fmin(0.5 * alpha, kCoincScaleDf), 1.0 / kCoincScaleDf);
        x.d1sq = __dadd_rn(d1, kEpsF64);
        reinterpret_cast<QParamF64X *>(qp)[q] = x;
        return;
    }
    QParamF64 o;
    if (d1 == 0.0) {
        o.neg_s = -kCoincScaleF64;
        o.c = kCoincScaleF64 * f64math::log2_c(kEpsF64);
    } else {
        const double sh = 0.5 * alpha;
        o.neg_s = -sh;
        o.c = sh * f64math::log2_c(__dadd_rn(d1, kEpsF64));
    }
    qp[q] = o;
}

// The sum of the weights of one query is kept as an unsigned fixed-point integer with 96
// fraction bits, accumulated exactly on the integer pipe from the weights exp2_t gives in that
// form (weights are at most 1 + a few ulps, the nearest point's being 1, so the sum of any
// n < 2^31 of them fits; each weight is truncated below 2^-96, at most n 2^-96 in all against a
// sum of at least 1).

// The fixed-point sum as two doubles whose sum is within 2^-100 of it, relative.
__device__ __forceinline__ void fixed_to_doubles(unsigned __int128 v, double &hi, double &lo)
{
    const unsigned long long A = static_cast<unsigned long long>(v >> 64);
    const unsigned long long B = static_cast<unsigned long long>(v);
    hi = __ull2double_rn(A) * 0x1p-32;
    const long long dA = static_cast<long long>(A - __double2ull_rn(hi * 0x1p32));  // exact
    lo = __ll2double_rn(dA) * 0x1p-32 + __ull2double_rn(B) * 0x1p-96;
}

// One CTA of 512 threads per SM (12 KB of 256-point tiles plus 72 KB of tables).
template <int Q>
__global__ void __launch_bounds__(kThreadsW64, 1)
f64_weights_kernel(DatasetDev ds, int64_t m, PassPlan pp, const double *__restrict__ qx,
                   const double *__restrict__ qy, const QParamF64 *__restrict__ qp,
                   double *__restrict__ part_sum, int *__restrict__ err)
{
    __shared__ __align__(128) double2 txy[2][kTileW64];
    __shared__ __align__(128) double tz[2][kTileW64];
    __shared__ __align__(8) uint64_t bar[2];
    extern __shared__ double2 f64_dyn[];  // f64math::Tables (kTablesBytes)
    f64math::Tables &tabs = *reinterpret_cast<f64math::Tables *>(f64_dyn);

    const int tid = threadIdx.x;
    const int s = blockIdx.y;
    f64math::load_tables(tabs);  // ordered before use by the barrier after the mbarrier set-up
    const int64_t qbase = static_cast<int64_t>(blockIdx.x) * pp.q_per_block;
    const int64_t p_begin = static_cast<int64_t>(s) * pp.split_len;
    const int64_t p_end = min(p_begin + pp.split_len, ds.n_pad);
    const int ntiles = static_cast<int>((p_end - p_begin) / kTileW64);

    double qxr[Q], qyr[Q], ns[Q], cc[Q], hz[Q], cz[Q];
    unsigned __int128 aw[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const int64_t q = min(qbase + j * kThreadsW64 + tid, m - 1);
        qxr[j] = qx[q];
        qyr[j] = qy[q];
        const QParamF64 o = qp[q];
        ns[j] = o.neg_s;
        cc[j] = o.c;
        hz[j] = cz[j] = 0.0;
        aw[j] = 0;
    }
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    constexpr uint32_t kBxy = kTileW64 * sizeof(double2);
    constexpr uint32_t kBz = kTileW64 * sizeof(double);
    if (tid == 0) {
        for (int t = 0; t < 2 && t < ntiles; ++t) {
            const int64_t o = p_begin + static_cast<int64_t>(t) * kTileW64;
            mbar_arrive_expect_tx(&bar[t], kBxy + kBz);
            tma_load_1d(txy[t], ds.xy64 + o, kBxy, &bar[t]);
            tma_load_1d(tz[t], ds.z64 + o, kBz, &bar[t]);
        }
    }
    bool ok = true;
    for (int t = 0; t < ntiles; ++t) {
        const int b = t & 1;
        const bool got = mbar_wait(&bar[b], (t >> 1) & 1);
        if (!__syncthreads_and(got)) {
            ok = false;
            if (tid == 0) {
                atomicOr(err, kErrTimeout);
                drain(bar, t, ntiles);
            }
            break;
        }
        for (int c = 0; c < kTileW64; c += kChunkW) {
            double sz[Q];
#pragma unroll
            for (int j = 0; j < Q; ++j)
                sz[j] = 0.0;
            // One point at a time (the Q queries' chains interleave): 109.1 ms on 8,192 x 1M
            // against 124.5 ms unrolled by 4 and 109.6 ms by 2.
#pragma unroll 1
            for (int u = 0; u < kChunkW; ++u) {
                const double2 p = txy[b][c + u];
                const double pz = tz[b][c + u];
#pragma unroll
                for (int j = 0; j < Q; ++j) {
                    const double d2 = dist2_eps(qxr[j], qyr[j], p.x, p.y);
                    unsigned __int128 w96;
                    const double w = f64math::exp2_t<true>(
                        __fma_rn(f64math::log2_t(d2, tabs), ns[j], cc[j]), tabs, &w96);
                    aw[j] += w96;
                    sz[j] = __fma_rn(w, pz, sz[j]);
                }
            }
#pragma unroll
            for (int j = 0; j < Q; ++j)
                kahan_add(hz[j], cz[j], sz[j]);
        }
        __syncthreads();
        if (tid == 0 && t + 2 < ntiles) {
            fence_proxy_async_smem();
            const int64_t o = p_begin + static_cast<int64_t>(t + 2) * kTileW64;
            mbar_arrive_expect_tx(&bar[b], kBxy + kBz);
            tma_load_1d(txy[b], ds.xy64 + o, kBxy, &bar[b]);
            tma_load_1d(tz[b], ds.z64 + o, kBz, &bar[b]);
        }
    }
    if (!ok)
        return;
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const int64_t q = qbase + j * kThreadsW64 + tid;
        if (q >= m)
            continue;
        double *o = part_sum + static_cast<int64_t>(s) * 4 * m + q;
        fixed_to_doubles(aw[j], o[0], o[m]);
        o[2 * m] = hz[j];
        o[3 * m] = -cz[j];
    }
}

__global__ void __launch_bounds__(256)
f64_finalize_kernel(int64_t m, int S, const double *__restrict__ part_sum,
                    double *__restrict__ out, const uint32_t *__restrict__ perm)
{
    const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q >= m)
        return;
    double W = 0.0, Wc = 0.0, WZ = 0.0, WZc = 0.0;
    for (int s = 0; s < S; ++s) {
        const double *o = part_sum + static_cast<int64_t>(s) * 4 * m + q;
        kahan_add(W, Wc, o[0]);
        kahan_add(W, Wc, o[m]);
        kahan_add(WZ, WZc, o[2 * m]);
        kahan_add(WZ, WZc, o[3 * m]);
    }
    out[perm ? perm[q] : q] = (WZ - WZc) / (W - Wc);  // Eq. 1
}

template <int KP>
constexpr int knn_q64()
{
    return KP <= 16 ? 2 : 1;
}

template <int KP, bool IDX>
cudaError_t launch_knn_t(const DatasetDev &ds, const Plan &pl, const double *qx,
                         const double *qy, int k, const Scratch &sc, int *err, cudaStream_t st)
{
    constexpr int Q = knn_q64<KP>();
    const size_t dyn = IDX ? sizeof(int32_t) * Q * KP * kThreads : 0;
    auto fn = f64_knn_kernel<KP, Q, IDX>;
    if (dyn > 0) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(dyn));
        if (e != cudaSuccess)
            return e;
    }
    dim3 grid(pl.knn.qblocks, pl.knn.splits);
    fn<<<grid, kThreads, dyn, st>>>(ds, pl.m, pl.knn, qx, qy, k,
                                    static_cast<double *>(sc.part_d2), sc.part_idx, err);
    return cudaGetLastError();
}

template <int KP>
int knn_slots_t(bool with_idx)
{
    constexpr int Q = knn_q64<KP>();
    int n = 0;
    if (with_idx) {
        const size_t dyn = sizeof(int32_t) * Q * KP * kThreads;
        cudaFuncSetAttribute(f64_knn_kernel<KP, Q, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(dyn));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f64_knn_kernel<KP, Q, true>, kThreads,
                                                      dyn);
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f64_knn_kernel<KP, Q, false>,
                                                      kThreads, 0);
    }
    return n > 0 ? n : 1;
}

}  // namespace

int f64_knn_queries_per_block(int k)
{
    return kThreads * (k <= 16 ? 2 : 1);
}

int f64_w_queries_per_block()
{
    return kThreadsW64 * kQW64;
}

int f64_knn_slots_per_sm(int k, bool with_idx)
{
    if (k <= 8)
        return knn_slots_t<8>(with_idx);
    if (k <= 16)
        return knn_slots_t<16>(with_idx);
    return knn_slots_t<32>(with_idx);
}

// The FP64 phase-2 kernel takes its log2 / exp2 tables in dynamic shared memory.
cudaError_t prepare_f64_weights()
{
    return cudaFuncSetAttribute(f64_weights_kernel<kQW64>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(f64math::kTablesBytes));
}

int f64_w_slots_per_sm()
{
    int n = 0;
    if (prepare_f64_weights() != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f64_weights_kernel<kQW64>, kThreadsW64,
                                                  f64math::kTablesBytes);
    return n > 0 ? n : 1;
}

cudaError_t launch_f64_knn(const DatasetDev &ds, const Plan &pl, const double *qx,
                           const double *qy, int k, const Scratch &sc, int *err,
                           cudaStream_t st)
{
    if (k <= 8)
        return pl.with_idx ? launch_knn_t<8, true>(ds, pl, qx, qy, k, sc, err, st)
                           : launch_knn_t<8, false>(ds, pl, qx, qy, k, sc, err, st);
    if (k <= 16)
        return pl.with_idx ? launch_knn_t<16, true>(ds, pl, qx, qy, k, sc, err, st)
                           : launch_knn_t<16, false>(ds, pl, qx, qy, k, sc, err, st);
    return pl.with_idx ? launch_knn_t<32, true>(ds, pl, qx, qy, k, sc, err, st)
                       : launch_knn_t<32, false>(ds, pl, qx, qy, k, sc, err, st);
}

cudaError_t launch_f64_select(const Plan &pl, int k, double r_exp, const AlphaMap &am,
                              const Scratch &sc, float *out_alpha, int32_t *out_knn,
                              cudaStream_t st, const uint32_t *perm, bool x_params)
{
    const int64_t blocks = (pl.m + 255) / 256;
    f64_select_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(
        pl.m, pl.knn.splits, k, r_exp, am, static_cast<const double *>(sc.part_d2),
        pl.with_idx ? sc.part_idx : nullptr, static_cast<QParamF64 *>(sc.qparam), out_alpha,
        out_knn, perm, x_params);
    return cudaGetLastError();
}

template <int KP, bool IDX>
cudaError_t launch_cull64_t(const DatasetDev &ds, const Plan &pl, const double *sqx,
                            const double *sqy, int k, const Scratch &sc, cudaStream_t st)
{
    constexpr int Q = knn_q64<KP>();
    const int ntiles = static_cast<int>(ds.n_pad / kTileF32Knn);
    int p2 = 1;
    while (p2 < ntiles)
        p2 <<= 1;
    const size_t dyn = sizeof(unsigned long long) * p2;
    auto fn = f64_knn_cull_kernel<KP, Q, IDX>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(dyn));
    if (e != cudaSuccess)
        return e;
    fn<<<pl.knn.qblocks, kThreads, dyn, st>>>(ds, pl.m, pl.knn.q_per_block, ntiles, p2, sqx,
                                              sqy, k, static_cast<double *>(sc.part_d2),
                                              sc.part_idx);
    return cudaGetLastError();
}

cudaError_t launch_f64_knn_cull(const DatasetDev &ds, const Plan &pl, const double *sqx,
                                const double *sqy, int k, const Scratch &sc, int *err,
                                cudaStream_t st)
{
    (void)err;  // no bounded waits: tiles are gathered with plain loads
    const bool idx = pl.with_idx;
    if (k <= 8)
        return idx ? launch_cull64_t<8, true>(ds, pl, sqx, sqy, k, sc, st)
                   : launch_cull64_t<8, false>(ds, pl, sqx, sqy, k, sc, st);
    if (k <= 16)
        return idx ? launch_cull64_t<16, true>(ds, pl, sqx, sqy, k, sc, st)
                   : launch_cull64_t<16, false>(ds, pl, sqx, sqy, k, sc, st);
    return idx ? launch_cull64_t<32, true>(ds, pl, sqx, sqy, k, sc, st)
               : launch_cull64_t<32, false>(ds, pl, sqx, sqy, k, sc, st);
}

cudaError_t launch_f64_knn_warp(const DatasetDev &ds, const Plan &pl, const double *qx,
                                const double *qy, int k, const Scratch &sc, int sm_count,
                                cudaStream_t st)
{
    constexpr int W = kThreads / 32;
    const int64_t want = (pl.m + W - 1) / W;
    const int64_t cap = static_cast<int64_t>(sm_count) * 16;
    const unsigned grid = static_cast<unsigned>(std::max<int64_t>(1, std::min(want, cap)));
    f64_knn_warp_kernel<<<grid, kThreads, 0, st>>>(ds, pl.m, qx, qy, k,
                                                   static_cast<double *>(sc.part_d2),
                                                   pl.with_idx ? sc.part_idx : nullptr);
    return cudaGetLastError();
}

cudaError_t launch_f64_weights(const DatasetDev &ds, const Plan &pl, const double *qx,
                               const double *qy, const Scratch &sc, int *err, cudaStream_t st)
{
    dim3 grid(pl.w.qblocks, pl.w.splits);
    const cudaError_t e = prepare_f64_weights();
    if (e != cudaSuccess)
        return e;
    f64_weights_kernel<kQW64><<<grid, kThreadsW64, f64math::kTablesBytes, st>>>(
        ds, pl.m, pl.w, qx, qy, static_cast<const QParamF64 *>(sc.qparam),
        static_cast<double *>(sc.part_sum), err);
    return cudaGetLastError();
}

cudaError_t launch_f64_finalize(const Plan &pl, const Scratch &sc, double *out,
                                cudaStream_t st, const uint32_t *perm)
{
    const int64_t blocks = (pl.m + 255) / 256;
    f64_finalize_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(
        pl.m, pl.w.splits, static_cast<const double *>(sc.part_sum), out, perm);
    return cudaGetLastError();
}

}  // namespace aidw

// Test hook: the FP64 path's log2 and exp2 evaluated elementwise on device arrays.
namespace aidw {
namespace {
__global__ void f64_math_probe_kernel(const double *__restrict__ x, const double *__restrict__ y,
                                      int64_t n, double *__restrict__ lx,
                                      double *__restrict__ ey)
{
    extern __shared__ double2 f64_dyn[];  // f64math::Tables (kTablesBytes)
    f64math::Tables &tabs = *reinterpret_cast<f64math::Tables *>(f64_dyn);
    f64math::load_tables(tabs);
    __syncthreads();
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        lx[i] = f64math::log2_t(x[i], tabs);
        ey[i] = f64math::exp2_t<false>(y[i], tabs, nullptr);
    }
}
}  // namespace
}  // namespace aidw

extern "C" int aidw_debug_f64_log2_exp2(const double *x, const double *y, int64_t n, double *lx,
                                        double *ey)
{
    if (n < 0 || (n > 0 && (!x || !y || !lx || !ey)))
        return AIDW_ERR_INVALID_ARG;
    if (n == 0)
        return AIDW_OK;
    const unsigned blocks = static_cast<unsigned>(n < 256 * 1024 ? (n + 255) / 256 : 1024);
    if (cudaFuncSetAttribute(aidw::f64_math_probe_kernel,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(aidw::f64math::kTablesBytes)) != cudaSuccess)
        return AIDW_ERR_CUDA;
    aidw::f64_math_probe_kernel<<<blocks, 256, aidw::f64math::kTablesBytes>>>(x, y, n, lx, ey);
    return cudaDeviceSynchronize() == cudaSuccess ? AIDW_OK : AIDW_ERR_CUDA;
}
