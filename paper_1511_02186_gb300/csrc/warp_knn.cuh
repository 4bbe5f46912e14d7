// The box-hierarchy walk of the one-warp-per-query phase-1 scans (FP32 in f32_device.cuh,
// FP64 in kernels_f64.cu).
//
// A warp serves one query. The dataset's Z-ordered points are grouped three ways, each with a
// bounding box: 32-tile super-tiles (16,384 points), 512-point tiles and 64-point sub-tiles.
// The walk is depth first: at each level every lane holds the visit key of one child box, a
// warp-wide minimum picks the next child, and the level ends when the smallest key's box is
// farther than the query's current k-th neighbour (the visitor decides, from its own list). A
// visit key holds the box's squared-distance lower bound in its high 32 bits (a non-negative
// float, whose bits order like its value) and the squared distance to the box centre below it,
// so that among the boxes a query lies in (bound 0) the one centred nearest comes first; the
// low 5 bits are left for the lane. The first sub-tiles scanned are therefore the nearest, the
// k-th distance falls early, and the rest of the walk is mostly pruned.
#pragma once

#include <math_constants.h>

#include "aidw_internal.cuh"

namespace aidw {

constexpr unsigned kFullMask = 0xffffffffu;

// Visit key from a box's lower bound (>= 0; +inf or NaN mean "never visit") and the squared
// distance to its centre (tie-break only).
__device__ __forceinline__ unsigned long long make_visit_key(float lb, float cd)
{
    if (!(lb < CUDART_INF_F))
        return ~0ull;
    cd = fminf(cd, 3.0e38f);
    return (static_cast<unsigned long long>(__float_as_uint(lb)) << 32) |
           (static_cast<unsigned long long>(__float_as_uint(cd) >> 5) << 5);
}

// The lower bound stored in a visit key.
__device__ __forceinline__ float visit_key_bound(unsigned long long key)
{
    return __uint_as_float(static_cast<uint32_t>(key >> 32));
}

// The smallest of the lanes' keys with its lane in the low 5 bits; ~0 if all are ~0.
__device__ __forceinline__ unsigned long long warp_min_key(unsigned long long key)
{
    const int lane = threadIdx.x & 31;
    if (key != ~0ull)
        key |= static_cast<unsigned long long>(lane);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(kFullMask, key, o);
        key = other < key ? other : key;
    }
    return key;
}

// Walks the boxes of `ds` for one warp. The visitor provides
//   unsigned long long key(float4 box)  the box's visit key (~0 for an empty box),
//   bool open(unsigned long long key)   whether the box may hold a point that enters the list
//                                       (false for ~0; warp-uniform),
//   void scan(int64_t p)                scan the 64 stored points [p, p + 64).
template <class Visitor>
__device__ __forceinline__ void warp_visit_boxes(const DatasetDev &ds, Visitor &v)
{
    constexpr int S = kTileF32Knn / kSubTile;  // 8 sub-tiles per tile
    const int lane = threadIdx.x & 31;
    const int64_t ntiles = ds.n_pad / kTileF32Knn;
    const int64_t nsuper = (ntiles + kSuperTiles - 1) / kSuperTiles;
    for (int64_t b = 0; b < nsuper; b += 32) {
        const int64_t s = b + lane;
        unsigned long long ks = s < nsuper ? v.key(ds.super_box[s]) : ~0ull;
        for (;;) {
            const unsigned long long ms = warp_min_key(ks);
            if (!v.open(ms))
                break;
            const int js = static_cast<int>(ms & 31ull);
            if (lane == js)
                ks = ~0ull;
            const int64_t t0 = (b + js) * kSuperTiles;
            const int64_t t = t0 + lane;
            unsigned long long kt =
                (lane < kSuperTiles && t < ntiles) ? v.key(ds.tile_box[t]) : ~0ull;
            for (;;) {
                const unsigned long long mt = warp_min_key(kt);
                if (!v.open(mt))
                    break;
                const int jt = static_cast<int>(mt & 31ull);
                if (lane == jt)
                    kt = ~0ull;
                const int64_t tt = t0 + jt;
                unsigned long long ku = lane < S ? v.key(ds.sub_box[tt * S + lane]) : ~0ull;
                for (;;) {
                    const unsigned long long mu = warp_min_key(ku);
                    if (!v.open(mu))
                        break;
                    const int ju = static_cast<int>(mu & 31ull);
                    if (lane == ju)
                        ku = ~0ull;
                    v.scan(tt * kTileF32Knn + static_cast<int64_t>(ju) * kSubTile);
                }
            }
        }
    }
}

}  // namespace aidw
