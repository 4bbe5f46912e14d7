// Spatial ordering helpers: Morton (Z-order) keys, a stable LSD radix sort of (key, value)
// pairs, gathers, bounding boxes.
//
// Data points are stored in Z-order so that each 512-point tile covers a compact region with a
// tight bounding box, and every call orders its queries the same way so that each query block
// is compact too. The phase-1 scan can then visit data tiles nearest-first and skip every tile
// whose box is provably farther than all of the block's current k-th neighbours. The order
// changes which tiles are read, never the result: the neighbour lists are exact.
#include <math_constants.h>

#include <cstdint>

#include "aidw_internal.cuh"

namespace aidw {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;  // keys per block and pass

// Order-preserving map of floats to unsigned integers (for atomic min / max).
__device__ __forceinline__ uint32_t f2ord(float f)
{
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ float ord2f(uint32_t u)
{
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

__global__ void bbox_kernel(const float2 *__restrict__ xy, int64_t n, uint32_t *ord4)
{
    float x0 = CUDART_INF_F, y0 = CUDART_INF_F, x1 = -CUDART_INF_F, y1 = -CUDART_INF_F;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float2 p = xy[i];
        x0 = fminf(x0, p.x);
        y0 = fminf(y0, p.y);
        x1 = fmaxf(x1, p.x);
        y1 = fmaxf(y1, p.y);
    }
    for (int o = 16; o > 0; o >>= 1) {
        x0 = fminf(x0, __shfl_xor_sync(0xffffffffu, x0, o));
        y0 = fminf(y0, __shfl_xor_sync(0xffffffffu, y0, o));
        x1 = fmaxf(x1, __shfl_xor_sync(0xffffffffu, x1, o));
        y1 = fmaxf(y1, __shfl_xor_sync(0xffffffffu, y1, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&ord4[0], f2ord(x0));
        atomicMin(&ord4[1], f2ord(y0));
        atomicMax(&ord4[2], f2ord(x1));
        atomicMax(&ord4[3], f2ord(y1));
    }
}

__global__ void bbox_finish_kernel(const uint32_t *ord4, float4 *box)
{
    *box = make_float4(ord2f(ord4[0]), ord2f(ord4[1]), ord2f(ord4[2]), ord2f(ord4[3]));
}

// Keys for points (x, y) given as separate float arrays or interleaved pairs; padding slots
// [n, n_total) get the largest key so they sort last.
__global__ void morton_keys_kernel(const float *__restrict__ x, const float *__restrict__ y,
                                   const float2 *__restrict__ xy, int64_t n, int64_t n_total,
                                   const float4 *__restrict__ box, uint32_t *keys,
                                   uint32_t *vals)
{
    const float4 b = *box;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n_total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        uint32_t key = 0xffffffffu;
        if (i < n) {
            const float px = xy ? xy[i].x : x[i];
            const float py = xy ? xy[i].y : y[i];
            key = morton_of(px, py, b);
        }
        keys[i] = key;
        vals[i] = static_cast<uint32_t>(i);
    }
}

__global__ void __launch_bounds__(kSortThreads)
radix_hist_kernel(const uint32_t *__restrict__ keys, int64_t n, int shift, uint32_t *counts,
                  int nblocks)
{
    __shared__ uint32_t h[256];
    const int tid = threadIdx.x;
    h[tid] = 0;
    __syncthreads();
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kSortTile;
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const int64_t i = base + j * kSortThreads + tid;
        if (i < n)
            atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    counts[static_cast<int64_t>(tid) * nblocks + blockIdx.x] = h[tid];
}

// Exclusive scan of the digit counts in two levels: segments of kScanSeg counts are scanned in
// place by one block each (segment-local prefixes), the segment totals by one block; the
// scatter adds the two. (One block scanning all counts sequentially took 0.4 ms per pass at
// 3.8M keys; most of a batch's query ordering.)
constexpr int kScanThreads = 1024;
constexpr int kScanSeg = 4 * kScanThreads;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *warp_tot,
                                                         uint32_t *total)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o)
            inc += t;
    }
    if (lane == 31)
        warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = lane < kScanThreads / 32 ? warp_tot[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o)
                wi += t;
        }
        if (lane < kScanThreads / 32)
            warp_tot[lane] = wi - w;
        if (lane == 31)
            *total = wi;
    }
    __syncthreads();
    return warp_tot[warp] + inc - v;
}

__global__ void __launch_bounds__(kScanThreads)
radix_scan_local_kernel(uint32_t *counts, int64_t total, uint32_t *seg_sums)
{
    __shared__ uint32_t warp_tot[32];
    __shared__ uint32_t seg_total;
    const int64_t i0 = static_cast<int64_t>(blockIdx.x) * kScanSeg + 4 * threadIdx.x;
    uint32_t c[4];
    uint32_t t = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        c[j] = i0 + j < total ? counts[i0 + j] : 0u;
        t += c[j];
    }
    uint32_t run = block_exclusive_scan(t, warp_tot, &seg_total);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (i0 + j < total)
            counts[i0 + j] = run;
        run += c[j];
    }
    if (threadIdx.x == 0)
        seg_sums[blockIdx.x] = seg_total;
}

// Exclusive scan of the segment totals in place, by one block.
__global__ void __launch_bounds__(kScanThreads) radix_scan_top_kernel(uint32_t *seg, int64_t n)
{
    __shared__ uint32_t warp_tot[32];
    __shared__ uint32_t chunk_total;
    uint32_t carry = 0;
    for (int64_t b = 0; b < n; b += kScanThreads) {
        const int64_t i = b + threadIdx.x;
        const uint32_t v = i < n ? seg[i] : 0u;
        const uint32_t ex = block_exclusive_scan(v, warp_tot, &chunk_total);
        if (i < n)
            seg[i] = carry + ex;
        carry += chunk_total;
        __syncthreads();
    }
}

// Stable scatter: keys of one block keep their input order within each digit.
__global__ void __launch_bounds__(kSortThreads)
radix_scatter_kernel(const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                     uint32_t *__restrict__ kout, uint32_t *__restrict__ vout, int64_t n,
                     int shift, const uint32_t *__restrict__ offsets,
                     const uint32_t *__restrict__ seg_offsets, int nblocks)
{
    constexpr int W = kSortThreads / 32;
    __shared__ uint32_t base_off[256];
    __shared__ uint32_t running[256];
    __shared__ uint32_t wcount[W][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t oi = static_cast<int64_t>(tid) * nblocks + blockIdx.x;
    base_off[tid] = offsets[oi] + seg_offsets[oi / kScanSeg];
    running[tid] = 0;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kSortTile;
    for (int j = 0; j < kSortItems; ++j) {
#pragma unroll
        for (int w = 0; w < W; ++w)
            wcount[w][tid] = 0;
        __syncthreads();
        const int64_t i = base + j * kSortThreads + tid;
        const bool valid = i < n;
        const uint32_t key = valid ? kin[i] : 0u;
        const uint32_t d = (key >> shift) & 255u;
        const uint32_t tag = valid ? d : (256u + lane);  // invalid lanes match nobody
        const uint32_t same = __match_any_sync(0xffffffffu, tag);
        const uint32_t rank = __popc(same & lt_mask);
        if (valid && lane == __ffs(same) - 1)
            wcount[warp][d] = __popc(same);
        __syncthreads();
        if (valid) {
            uint32_t prior = 0;
            for (int w = 0; w < warp; ++w)
                prior += wcount[w][d];
            const uint32_t pos = base_off[d] + running[d] + prior + rank;
            kout[pos] = key;
            vout[pos] = vin[i];
        }
        __syncthreads();
        uint32_t add = 0;
#pragma unroll
        for (int w = 0; w < W; ++w)
            add += wcount[w][tid];
        running[tid] += add;
        __syncthreads();
    }
}

// One warp per tile of kTileF32Knn sorted points: box of the finite points.
// Bounding box of the finite points of every group of G consecutive stored points (one warp
// per group).
template <int G>
__global__ void tile_box_kernel(const float4 *__restrict__ nxy2, int64_t ntiles, float4 *boxes)
{
    const int64_t t = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= ntiles)
        return;
    float x0 = CUDART_INF_F, y0 = CUDART_INF_F, x1 = -CUDART_INF_F, y1 = -CUDART_INF_F;
    for (int u = lane; u < G; u += 32) {
        const float4 p = nxy2[t * G + u];
        const float px = -p.x, py = -p.z;
        if (isfinite(px) && isfinite(py)) {
            x0 = fminf(x0, px);
            y0 = fminf(y0, py);
            x1 = fmaxf(x1, px);
            y1 = fmaxf(y1, py);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        x0 = fminf(x0, __shfl_xor_sync(0xffffffffu, x0, o));
        y0 = fminf(y0, __shfl_xor_sync(0xffffffffu, y0, o));
        x1 = fmaxf(x1, __shfl_xor_sync(0xffffffffu, x1, o));
        y1 = fmaxf(y1, __shfl_xor_sync(0xffffffffu, y1, o));
    }
    if (lane == 0)
        boxes[t] = make_float4(x0, y0, x1, y1);
}

// One warp per group of kSuperTiles tile boxes: their union (empty tiles hold an empty box,
// (+inf, +inf, -inf, -inf), which the union ignores).
__global__ void super_box_kernel(const float4 *__restrict__ tbox, int64_t ntiles,
                                 int64_t nsuper, float4 *boxes)
{
    const int64_t s = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (s >= nsuper)
        return;
    const int64_t t = s * kSuperTiles + lane;
    float4 b = make_float4(CUDART_INF_F, CUDART_INF_F, -CUDART_INF_F, -CUDART_INF_F);
    if (lane < kSuperTiles && t < ntiles)
        b = tbox[t];
    for (int o = 16; o > 0; o >>= 1) {
        b.x = fminf(b.x, __shfl_xor_sync(0xffffffffu, b.x, o));
        b.y = fminf(b.y, __shfl_xor_sync(0xffffffffu, b.y, o));
        b.z = fmaxf(b.z, __shfl_xor_sync(0xffffffffu, b.z, o));
        b.w = fmaxf(b.w, __shfl_xor_sync(0xffffffffu, b.w, o));
    }
    if (lane == 0)
        boxes[s] = b;
}

// Morton keys of FP64 query coordinates (rounded to FP32 for the key: the key only orders).
__global__ void morton_keys_f64_kernel(const double *__restrict__ x,
                                       const double *__restrict__ y, int64_t n,
                                       const float4 *__restrict__ box, uint32_t *keys,
                                       uint32_t *vals)
{
    const float4 b = *box;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        keys[i] = morton_of(static_cast<float>(x[i]), static_cast<float>(y[i]), b);
        vals[i] = static_cast<uint32_t>(i);
    }
}

template <typename T>
__global__ void gather_pairs_kernel(const T *__restrict__ x, const T *__restrict__ y,
                                    const uint32_t *__restrict__ perm, int64_t m, T *sx, T *sy)
{
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < m;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const uint32_t p = perm[i];
        sx[i] = x[p];
        sy[i] = y[p];
    }
}

inline unsigned grid_for(int64_t n, int threads, int cap)
{
    const int64_t b = (n + threads - 1) / threads;
    return static_cast<unsigned>(b < cap ? (b > 0 ? b : 1) : cap);
}

}  // namespace

size_t radix_scratch_bytes(int64_t n)
{
    const int64_t nblocks = (n + kSortTile - 1) / kSortTile;
    const int64_t nseg = (256 * nblocks + kScanSeg - 1) / kScanSeg;
    return sizeof(uint32_t) *
           (2 * static_cast<size_t>(n) + 256 * static_cast<size_t>(nblocks) +
            static_cast<size_t>(nseg));
}

// Sorts (keys, vals)[0..n) stably by the low `bits` bits of the key (rounded up to a multiple
// of 16, so that an even number of 8-bit passes leaves the result in place); tmp holds
// radix_scratch_bytes(n) bytes.
cudaError_t radix_sort_pairs(uint32_t *keys, uint32_t *vals, int64_t n, void *tmp,
                             cudaStream_t st, int bits)
{
    if (n <= 1)
        return cudaSuccess;
    const int nblocks = static_cast<int>((n + kSortTile - 1) / kSortTile);
    uint32_t *k2 = static_cast<uint32_t *>(tmp);
    uint32_t *v2 = k2 + n;
    uint32_t *counts = v2 + n;
    const int64_t ncounts = static_cast<int64_t>(nblocks) * 256;
    const int64_t nseg = (ncounts + kScanSeg - 1) / kScanSeg;
    uint32_t *seg = counts + ncounts;
    uint32_t *ka = keys, *va = vals, *kb = k2, *vb = v2;
    const int top = bits <= 16 ? 16 : 32;
    for (int shift = 0; shift < top; shift += 8) {
        radix_hist_kernel<<<nblocks, kSortThreads, 0, st>>>(ka, n, shift, counts, nblocks);
        radix_scan_local_kernel<<<static_cast<unsigned>(nseg), kScanThreads, 0, st>>>(
            counts, ncounts, seg);
        radix_scan_top_kernel<<<1, kScanThreads, 0, st>>>(seg, nseg);
        radix_scatter_kernel<<<nblocks, kSortThreads, 0, st>>>(ka, va, kb, vb, n, shift, counts,
                                                               seg, nblocks);
        uint32_t *t = ka;
        ka = kb;
        kb = t;
        t = va;
        va = vb;
        vb = t;
    }
    return cudaGetLastError();  // an even number of passes: the result is back in keys / vals
}

// Bounding box of n points of an interleaved array into *box (device), using 16 bytes of
// scratch.
cudaError_t bbox_of(const float2 *xy, int64_t n, uint32_t *scratch4, float4 *box,
                    cudaStream_t st)
{
    const uint32_t init[4] = {0xffffffffu, 0xffffffffu, 0u, 0u};
    cudaError_t e = cudaMemcpyAsync(scratch4, init, sizeof(init), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess)
        return e;
    bbox_kernel<<<grid_for(n, 256, 1024), 256, 0, st>>>(xy, n, scratch4);
    bbox_finish_kernel<<<1, 1, 0, st>>>(scratch4, box);
    return cudaGetLastError();
}

cudaError_t morton_keys(const float *x, const float *y, const float2 *xy, int64_t n,
                        int64_t n_total, const float4 *box, uint32_t *keys, uint32_t *vals,
                        cudaStream_t st)
{
    morton_keys_kernel<<<grid_for(n_total, 256, 4096), 256, 0, st>>>(x, y, xy, n, n_total, box,
                                                                     keys, vals);
    return cudaGetLastError();
}

cudaError_t tile_boxes(const float4 *nxy2, int64_t ntiles, float4 *boxes, cudaStream_t st)
{
    tile_box_kernel<kTileF32Knn>
        <<<grid_for(ntiles * 32, 256, 1 << 20), 256, 0, st>>>(nxy2, ntiles, boxes);
    return cudaGetLastError();
}

cudaError_t super_tile_boxes(const float4 *tile_boxes, int64_t ntiles, int64_t nsuper,
                             float4 *boxes, cudaStream_t st)
{
    static_assert(kSuperTiles == 32, "one lane per tile of a super-tile");
    super_box_kernel<<<grid_for(nsuper * 32, 256, 1 << 20), 256, 0, st>>>(tile_boxes, ntiles,
                                                                          nsuper, boxes);
    return cudaGetLastError();
}

cudaError_t sub_tile_boxes(const float4 *nxy2, int64_t nsub, float4 *boxes, cudaStream_t st)
{
    tile_box_kernel<kSubTile><<<grid_for(nsub * 32, 256, 1 << 20), 256, 0, st>>>(nxy2, nsub,
                                                                                 boxes);
    return cudaGetLastError();
}

cudaError_t gather_queries(const float *qx, const float *qy, const uint32_t *perm, int64_t m,
                           float *sqx, float *sqy, cudaStream_t st)
{
    gather_pairs_kernel<float><<<grid_for(m, 256, 4096), 256, 0, st>>>(qx, qy, perm, m, sqx,
                                                                       sqy);
    return cudaGetLastError();
}

cudaError_t morton_keys_f64(const double *x, const double *y, int64_t n, const float4 *box,
                            uint32_t *keys, uint32_t *vals, cudaStream_t st)
{
    morton_keys_f64_kernel<<<grid_for(n, 256, 4096), 256, 0, st>>>(x, y, n, box, keys, vals);
    return cudaGetLastError();
}

cudaError_t gather_queries_f64(const double *qx, const double *qy, const uint32_t *perm,
                               int64_t m, double *sqx, double *sqy, cudaStream_t st)
{
    gather_pairs_kernel<double><<<grid_for(m, 256, 4096), 256, 0, st>>>(qx, qy, perm, m, sqx,
                                                                        sqy);
    return cudaGetLastError();
}

}  // namespace aidw
