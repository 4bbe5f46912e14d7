// Internal declarations shared by the library's translation units: device-side dataset view,
// launch plans, Blackwell TMA/mbarrier helpers and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/aidw.h"

namespace aidw {

// Data points per shared-memory tile. Dataset arrays are padded to a multiple of
// kPadPoints with sentinel points at +infinity (value 0), which never enter a neighbour list
// and get weight 0, so every tile is full and every TMA copy has a whole-tile size.
constexpr int kTileF32Knn = 512;   // float4 (-x, -x, -y, -y): 8 KiB per buffer
constexpr int kTileF32W = 512;     // float4 (-x, -x, -y, -y) + float2 (z, z): 12 KiB per buffer
constexpr int kTileF64Knn = 512;   // double2 (x, y): 8 KiB per buffer
constexpr int kTileF64W = 512;     // double2 + double: 12 KiB per buffer
constexpr int kPadPoints = 2048;   // common multiple of every tile and split granule
constexpr int kSubTile = 64;       // points per sub-tile box (pruned phase 1)
constexpr int kSuperTiles = 32;    // tiles per super-tile box (the per-query phase 1)

// Added under the square of distances: it is absorbed (below half an ulp) for any distance
// above ~1e-15 of unit scale, and turns an exact coincidence (d2 == 0) into d2 == kEps so
// that log2 stays finite. FLT_MIN / DBL_MIN, the smallest normal numbers.
constexpr float kEpsF32 = 1.17549435e-38f;
constexpr double kEpsF64 = 2.2250738585072014e-308;
// Power scale used for coincident queries: w = 2^(kCoincScale (L1 - log2 d2)) is exactly 1 on
// a coincident point (d2 == eps) and underflows to 0 everywhere else.
constexpr float kCoincScaleF32 = 1.2676506e30f;  // 2^100
constexpr double kCoincScaleF64 = 8.452712498170644e270;  // 2^900
constexpr double kCoincScaleDf = 1.2676506002282294e30;   // 2^100 (AIDW_F64X: float range)

// Bounded waits: an mbarrier wait gives up after this many polls and raises the error word;
// a wait on another CTA's counter gives up after kMaxWaitPolls polls of at least 256 ns
// (tens of seconds at most).
constexpr uint32_t kMaxPolls = 1u << 26;
constexpr uint32_t kMaxWaitPolls = 1u << 26;
constexpr int kErrTimeout = 1;

// Kernel shape shared by every scan kernel.
constexpr int kThreads = 128;   // threads per CTA
constexpr int kMaxSplits = 64;  // data-range splits per pass

// Levels and bounds of Eq. 5 and Eq. 6, passed to kernels by value.
struct AlphaMap {
    double level[5];
    double r_min, r_max;
};

// FP32 copies are stored negated and duplicated, (-x, -x, -y, -y) and (z, z), so that one
// shared-memory load yields the register pairs that packed FP32x2 instructions operate on for
// two queries at once (q + (-x) is exactly q - x). They are kept in Z-order (Morton order of
// the points), with orig[] mapping a stored position back to the caller's index and one
// bounding box per 512-point tile. The FP64 copies keep the caller's order.
struct DatasetDev {
    const float4 *nxy2;     // [n_pad] (-x, -x, -y, -y), Z-order
    const float2 *zz;       // [n_pad] (z, z), Z-order
    const int32_t *orig;    // [n_pad] caller's index of each stored point, -1 for padding
    const float4 *tile_box; // [n_pad / kTileF32Knn] (xmin, ymin, xmax, ymax) of finite points
    const float4 *sub_box;  // [n_pad / kSubTile] the same per 64-point sub-tile
    const float4 *super_box; // [ceil(tiles / kSuperTiles)] the same per 32 tiles
    const float4 *box;      // [1] bounding box of all points
    const double2 *xy64;    // [n_pad] caller's order
    const double *z64;      // [n_pad] caller's order
    int64_t n;
    int64_t n_pad;
};

// How one scan pass is cut into work: query blocks (one CTA each) times data-range splits,
// each split a whole number of kPadPoints-point granules.
struct PassPlan {
    int q_per_block;   // queries handled by one CTA
    int qblocks;       // ceil(m / q_per_block)
    int splits;        // S: data-range splits, each scanned by its own CTA
    int64_t split_len; // points per split (multiple of kPadPoints)
};

struct Plan {
    int64_t m;
    PassPlan knn;  // phase 1 scan
    PassPlan w;    // phase 2 scan
    bool with_idx; // keep neighbour indices (needed for the kNN output)
    int kp;        // FP32 phase 1: register k-list length (8, 12, 16 or 32)
    int qw;        // FP32 phase 2: queries per thread (2, 4 or 8)
    int tw;        // FP32 phase 2: data points per shared-memory tile (256 or 512)
    int knn_slots; // phase-1 CTAs resident on the whole GPU (occupancy x SMs)
    int kq;        // pruned phase 1: queries per thread (2 or 4)
};

// Per-query parameters of phase 2 produced by the selection kernel.
//   F32: w = ex2(fma(log2(d2), neg_s, c)), neg_s = -alpha/2, c = alpha/2 * log2(d1^2)
//   F64: same with doubles.
struct QParamF32 {
    float neg_s;
    float c;
};
struct QParamF64 {
    double neg_s;
    double c;
};

// Per-query constants of the AIDW_F64X phase 2: kappa = alpha / 2 (the coincidence scale for a
// query on a data point) and the nearest squared distance the weights are relative to.
struct QParamF64X {
    double kappa;
    double d1sq;
};
static_assert(sizeof(QParamF64X) == sizeof(QParamF64), "shares the FP64 scratch layout");

// Scratch buffers of one interpolation (device memory owned by the library or by the
// caller of the allocation-free entry point).
struct Scratch {
    void *part_d2;     // [S_knn][k][m] float (F32) or double (F64): per-split sorted lists
    int32_t *part_idx; // [S_knn][k][m] or null when indices are not kept
    void *qparam;      // [m] QParamF32 / QParamF64
    void *part_sum;    // [S_w][4][m] float (w_hi, w_lo, wz_hi, wz_lo) or double
};

size_t scratch_bytes(int precision, const Plan &pl, int k);
void scratch_carve(void *base, int precision, const Plan &pl, int k, Scratch *s);

// ---- launchers (all stream-ordered, return cudaGetLastError()) --------------------------
cudaError_t launch_f32_knn(const DatasetDev &ds, const Plan &pl, const float *qx,
                           const float *qy, int k, const Scratch &sc, int *err,
                           cudaStream_t st);
cudaError_t launch_f32_select(const Plan &pl, int k, double r_exp, const AlphaMap &am,
                              const Scratch &sc, float *out_alpha, int32_t *out_knn,
                              cudaStream_t st, const uint32_t *perm = nullptr);
cudaError_t launch_f32_weights(const DatasetDev &ds, const Plan &pl, const float *qx,
                               const float *qy, const Scratch &sc, int *err, cudaStream_t st);
cudaError_t launch_f32_finalize(const Plan &pl, const Scratch &sc, float *out,
                                cudaStream_t st, const uint32_t *perm = nullptr);
// Phase 1 with one warp per query, in the caller's order (queries that lie far apart compared
// with the data points): one split's lists in sc.part_d2 (and sc.part_idx when non-null).
cudaError_t launch_f32_knn_warp(const DatasetDev &ds, int64_t m, const float *qx,
                                const float *qy, int k, const Scratch &sc, int sm_count,
                                cudaStream_t st);
// Phase 1 over Z-ordered queries with nearest-first tile visiting and bounding-box pruning
// (one split); sqx / sqy are the queries in Z-order.
constexpr int64_t kMaxCullTiles = 8192;
cudaError_t launch_f32_knn_cull(const DatasetDev &ds, const Plan &pl, const float *sqx,
                                const float *sqy, int k, const Scratch &sc, int *err,
                                cudaStream_t st);

// Spatial helpers (spatial.cu).
size_t radix_scratch_bytes(int64_t n);
cudaError_t radix_sort_pairs(uint32_t *keys, uint32_t *vals, int64_t n, void *tmp,
                             cudaStream_t st, int bits = 32);
cudaError_t bbox_of(const float2 *xy, int64_t n, uint32_t *scratch4, float4 *box,
                    cudaStream_t st);
cudaError_t morton_keys(const float *x, const float *y, const float2 *xy, int64_t n,
                        int64_t n_total, const float4 *box, uint32_t *keys, uint32_t *vals,
                        cudaStream_t st);
cudaError_t tile_boxes(const float4 *nxy2, int64_t ntiles, float4 *boxes, cudaStream_t st);
cudaError_t sub_tile_boxes(const float4 *nxy2, int64_t nsub, float4 *boxes, cudaStream_t st);
// Box of every group of kSuperTiles consecutive tile boxes (the last group may be shorter).
cudaError_t super_tile_boxes(const float4 *tile_boxes, int64_t ntiles, int64_t nsuper,
                             float4 *boxes, cudaStream_t st);
cudaError_t gather_queries(const float *qx, const float *qy, const uint32_t *perm, int64_t m,
                           float *sqx, float *sqy, cudaStream_t st);
cudaError_t morton_keys_f64(const double *x, const double *y, int64_t n, const float4 *box,
                            uint32_t *keys, uint32_t *vals, cudaStream_t st);
cudaError_t gather_queries_f64(const double *qx, const double *qy, const uint32_t *perm,
                               int64_t m, double *sqx, double *sqy, cudaStream_t st);

cudaError_t launch_f64_knn(const DatasetDev &ds, const Plan &pl, const double *qx,
                           const double *qy, int k, const Scratch &sc, int *err,
                           cudaStream_t st);
cudaError_t launch_f64_select(const Plan &pl, int k, double r_exp, const AlphaMap &am,
                              const Scratch &sc, float *out_alpha, int32_t *out_knn,
                              cudaStream_t st, const uint32_t *perm = nullptr,
                              bool x_params = false);
// Phase 1 over Z-ordered FP64 queries, pruned like launch_f32_knn_cull; with pl.with_idx the
// lists are the k smallest (distance, caller index) pairs, so ties go to the lower index as in
// the caller-order scan; sqx / sqy are the queries in Z-order and the dataset's points are read
// through its Z-order map.
cudaError_t launch_f64_knn_cull(const DatasetDev &ds, const Plan &pl, const double *sqx,
                                const double *sqy, int k, const Scratch &sc, int *err,
                                cudaStream_t st);
// Phase 1 with one warp per query in the caller's order (one split's lists [k][m]); with
// pl.with_idx the lists are the k smallest (distance, caller index) pairs, as above.
cudaError_t launch_f64_knn_warp(const DatasetDev &ds, const Plan &pl, const double *qx,
                                const double *qy, int k, const Scratch &sc, int sm_count,
                                cudaStream_t st);
cudaError_t launch_f64_weights(const DatasetDev &ds, const Plan &pl, const double *qx,
                               const double *qy, const Scratch &sc, int *err,
                               cudaStream_t st);
cudaError_t launch_f64_finalize(const Plan &pl, const Scratch &sc, double *out,
                                cudaStream_t st, const uint32_t *perm = nullptr);
// AIDW_F64X phase 2 (kernels_f64x.cu); reads QParamF64X written by launch_f64_select with
// x_params and leaves part_sum in the layout launch_f64_finalize reads.
cudaError_t launch_f64x_weights(const DatasetDev &ds, const Plan &pl, const double *qx,
                                const double *qy, const Scratch &sc, int *err,
                                cudaStream_t st);

// Shape of the kernels: queries per CTA of each scan and the CTA slots per SM that occupancy
// allows (used to cut splits into whole waves). FP32 shapes follow the tuning fields of
// aidw_tune_config (kp: k-list length, qw: phase-2 queries per thread, tw: tile points).
int f32_knn_queries_per_block(int kp);
int f32_w_queries_per_block(int qw);
int f32_knn_slots_per_sm(int kp, bool with_idx);
int f32_w_slots_per_sm(int qw, int tw);
// k-list length for k under a minimum (aidw_tune_config.knn_list).
int f32_list_length(int k, int kp_min);
// Queries per thread of the pruned phase 1 for list length kp under the shape's request
// (aidw_tune_config.knn_queries_per_thread; 0 = 4 for lists of up to 16, lists of 32 take 2).
inline int cull_queries_per_thread(int kp, int requested)
{
    return kp > 16 ? 2 : (requested == 2 ? 2 : 4);
}
// Built-in shape and the check of a caller's shape (autotune.cu).
aidw_tune_config tune_default();
bool tune_valid(const aidw_tune_config &c);
int f64_knn_queries_per_block(int k);
int f64_w_queries_per_block();
int f64_knn_slots_per_sm(int k, bool with_idx);
int f64_w_slots_per_sm();
int f64x_w_queries_per_block();
int f64x_w_slots_per_sm();

// Pipe-rate microbenchmarks (probe.cu).
cudaError_t run_pipe_probe(int sm_count, aidw_pipe_rates *out);

// ---- device helpers: Blackwell bulk-copy (TMA) and mbarrier ------------------------------
#if defined(__CUDACC__)

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// One-dimensional bulk copy global -> shared through the TMA unit; completion is signalled
// on `bar` as transaction bytes. dst, src and bytes must be multiples of 16.
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, uint32_t bytes,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Bounded wait for phase `parity` of `bar`. Returns false (and leaves the caller to raise
// the error word) if the phase did not complete within max_polls polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                          uint32_t max_polls = kMaxPolls)
{
    uint32_t addr = smem_addr(bar);
    for (uint32_t i = 0; i < max_polls; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done)
            return true;
    }
    return false;
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Thread 0 waits (bounded: max_polls acquire loads, 256 ns apart at least) until
// *p >= target; the outcome is shared with the CTA through the shared word `flag`.
__device__ __forceinline__ bool cta_wait_count(const uint32_t *p, uint32_t target, int *flag,
                                               uint32_t max_polls = kMaxWaitPolls)
{
    if (threadIdx.x == 0) {
        bool ok = false;
        for (uint32_t i = 0; i < max_polls; ++i) {
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

// MUFU approximations with flush-to-zero (single SFU instruction each).
__device__ __forceinline__ float lg2_approx(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Eq. 5 (Sec. 2.2 Step 2): fuzzy membership of the NN statistic, with pi / R_max as printed.
__device__ __forceinline__ double membership_eq5(double R, const AlphaMap &am)
{
    if (R <= am.r_min)
        return 0.0;
    if (R >= am.r_max)
        return 1.0;
    return 0.5 - 0.5 * cos((3.141592653589793 / am.r_max) * (R - am.r_min));
}

// Eq. 6 (Sec. 2.2 Step 3): alpha is alpha_1 up to mu = 0.1, alpha_5 from mu = 0.9, and in
// between runs linearly from alpha_s at mu = 0.1 + 0.2 (s - 1) to alpha_(s+1) 0.2 later.
__device__ __forceinline__ double alpha_eq6(double mu, const AlphaMap &am)
{
    if (mu <= 0.1)
        return am.level[0];
    if (mu >= 0.9)
        return am.level[4];
    int seg = static_cast<int>((mu - 0.1) * 5.0);
    seg = seg < 0 ? 0 : (seg > 3 ? 3 : seg);
    const double t = (mu - (0.1 + 0.2 * seg)) * 5.0;
    return am.level[seg] * (1.0 - t) + am.level[seg + 1] * t;
}

// Spreads the low 16 bits of v to the even bit positions.
__device__ __forceinline__ uint32_t spread16(uint32_t v)
{
    v &= 0xffffu;
    v = (v | (v << 8)) & 0x00ff00ffu;
    v = (v | (v << 4)) & 0x0f0f0f0fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

// Z-order (Morton) key of (x, y) on a 65536 x 65536 grid over `box` (xmin, ymin, xmax, ymax);
// points outside the box, or NaN, clamp to its edges.
__device__ __forceinline__ uint32_t morton_of(float x, float y, float4 box)
{
    const float sx = box.z > box.x ? 65535.0f / (box.z - box.x) : 0.0f;
    const float sy = box.w > box.y ? 65535.0f / (box.w - box.y) : 0.0f;
    const float fx = fminf(fmaxf((x - box.x) * sx, 0.0f), 65535.0f);
    const float fy = fminf(fmaxf((y - box.y) * sy, 0.0f), 65535.0f);
    return (spread16(static_cast<uint32_t>(fy)) << 1) | spread16(static_cast<uint32_t>(fx));
}

// Kahan step: adds v to the running sum h whose compensation (excess added so far) is c.
template <typename T>
__device__ __forceinline__ void kahan_add(T &h, T &c, T v)
{
    const T y = v - c;
    const T t = h + y;
    c = (t - h) - y;
    h = t;
}

#endif  // __CUDACC__

}  // namespace aidw
