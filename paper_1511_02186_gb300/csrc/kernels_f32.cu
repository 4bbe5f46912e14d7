// FP32 ("F32C") per-call kernels of the AIDW hot path for sm_103a.
//
//   f32_knn_kernel      grid (query blocks, data splits): phase-1 unit per CTA (neighbour lists)
//   f32_select_kernel   one thread per query: split merge, Eq. 2-6 -> phase-2 parameters
//   f32_weights_kernel  grid (query blocks, data splits): phase-2 unit per CTA (weighted sums)
//   f32_finalize_kernel one thread per query: split merge, Eq. 1 ratio in FP64
// The unit bodies live in f32_device.cuh and are shared with the persistent batched kernel.
#include <algorithm>

#include "f32_device.cuh"

namespace aidw {
namespace {

using namespace f32dev;

template <int KP, int Q, bool IDX>
__global__ void __launch_bounds__(kThreads)
f32_knn_kernel(DatasetDev ds, int64_t m, PassPlan pp, const float *__restrict__ qx,
               const float *__restrict__ qy, int k, float *__restrict__ part_d2,
               int32_t *__restrict__ part_idx, int *__restrict__ err)
{
    __shared__ __align__(128) float4 tile[2][kTileF32Knn];
    __shared__ __align__(8) uint64_t bar[2];
    extern __shared__ int32_t idx_smem[];  // [Q][KP][kThreads] when IDX
    init_tile_barriers(bar);
    TileSeq ts{bar, 0u};
    const int s = blockIdx.y;
    const int64_t p_begin = static_cast<int64_t>(s) * pp.split_len;
    const int64_t p_end = min(p_begin + pp.split_len, ds.n_pad);
    knn_unit<KP, Q, IDX>(ds, m, static_cast<int64_t>(blockIdx.x) * pp.q_per_block, p_begin,
                         p_end, qx, qy, k, s, part_d2, part_idx, err, tile, ts, idx_smem);
}

__global__ void __launch_bounds__(256)
f32_select_kernel(int64_t m, int S, int k, double r_exp, AlphaMap am,
                  const float *__restrict__ part_d2, const int32_t *__restrict__ part_idx,
                  QParamF32 *__restrict__ qp, float *__restrict__ out_alpha,
                  int32_t *__restrict__ out_knn, const uint32_t *__restrict__ perm)
{
    const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q < m)
        select_query(q, m, S, k, r_exp, am, part_d2, part_idx, qp, out_alpha, out_knn, perm);
}

// Phase 1 with one warp per query (warp_knn), in the caller's order: each query's k nearest
// squared distances (and stored positions mapped to caller indices when part_idx is non-null)
// as one split's lists [k][m], for the selection kernel, which amortises its FP64 work over a
// thread per query.
__global__ void __launch_bounds__(kThreads)
f32_knn_warp_kernel(DatasetDev ds, int64_t m, const float *__restrict__ qx,
                    const float *__restrict__ qy, int k, float *__restrict__ part_d2,
                    int32_t *__restrict__ part_idx)
{
    constexpr int W = kThreads / 32;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = static_cast<int64_t>(gridDim.x) * W;
    for (int64_t q = static_cast<int64_t>(blockIdx.x) * W + (threadIdx.x >> 5); q < m;
         q += nwarps) {
        float ld;
        int32_t li;
        warp_knn(ds, qx[q], qy[q], k, ld, li);
        if (lane < k) {
            part_d2[static_cast<int64_t>(lane) * m + q] = ld;
            if (part_idx)
                part_idx[static_cast<int64_t>(lane) * m + q] = li >= 0 ? ds.orig[li] : -1;
        }
    }
}

template <int KP, int Q, bool IDX>
__global__ void __launch_bounds__(kThreads)
f32_knn_cull_kernel(DatasetDev ds, int64_t m, int qpb, int ntiles, int ntiles_p2,
                    const float *__restrict__ sqx, const float *__restrict__ sqy, int k,
                    float *__restrict__ part_d2, int32_t *__restrict__ part_idx,
                    int *__restrict__ err)
{
    extern __shared__ unsigned long long order[];  // [ntiles_p2], then the index lists if IDX
    __shared__ __align__(128) float4 tile[2][kTileF32Knn];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ CullShared cs;
    init_tile_barriers(bar);
    TileSeq ts{bar, 0u};
    knn_cull_unit<KP, Q, IDX>(ds, m, static_cast<int64_t>(blockIdx.x) * qpb, ntiles, ntiles_p2,
                              sqx, sqy, k, part_d2, part_idx, err, tile, ts, order,
                              reinterpret_cast<int32_t *>(order + ntiles_p2), cs);
}

template <int Q, int TW>
__global__ void __launch_bounds__(kThreads)
f32_weights_kernel(DatasetDev ds, int64_t m, PassPlan pp, const float *__restrict__ qx,
                   const float *__restrict__ qy, const QParamF32 *__restrict__ qp,
                   float *__restrict__ part_sum, int *__restrict__ err)
{
    __shared__ __align__(128) float4 txy[2][TW];
    __shared__ __align__(128) float2 tz[2][TW];
    __shared__ __align__(8) uint64_t bar[2];
    init_tile_barriers(bar);
    TileSeq ts{bar, 0u};
    const int s = blockIdx.y;
    const int64_t p_begin = static_cast<int64_t>(s) * pp.split_len;
    const int64_t p_end = min(p_begin + pp.split_len, ds.n_pad);
    weights_unit<Q, TW>(ds, m, static_cast<int64_t>(blockIdx.x) * pp.q_per_block, p_begin,
                        p_end, qx, qy, qp, s, part_sum, err, txy, tz, ts);
}

__global__ void __launch_bounds__(256)
f32_finalize_kernel(int64_t m, int S, const float *__restrict__ part_sum,
                    float *__restrict__ out, const uint32_t *__restrict__ perm)
{
    const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q < m)
        out[perm ? perm[q] : q] = finalize_query(q, m, S, part_sum);
}

template <int KP, int Q, bool IDX>
cudaError_t launch_cull_t(const DatasetDev &ds, const Plan &pl, const float *sqx,
                          const float *sqy, int k, const Scratch &sc, int *err, cudaStream_t st)
{
    const int ntiles = static_cast<int>(ds.n_pad / kTileF32Knn);
    int p2 = 1;
    while (p2 < ntiles)
        p2 <<= 1;
    const size_t dyn = sizeof(unsigned long long) * p2 +
                       (IDX ? sizeof(int32_t) * Q * KP * kThreads : 0);
    auto fn = f32_knn_cull_kernel<KP, Q, IDX>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(dyn));
    if (e != cudaSuccess)
        return e;
    fn<<<pl.knn.qblocks, kThreads, dyn, st>>>(ds, pl.m, pl.knn.q_per_block, ntiles, p2, sqx,
                                              sqy, k, static_cast<float *>(sc.part_d2),
                                              sc.part_idx, err);
    return cudaGetLastError();
}

template <int KP, bool IDX>
cudaError_t launch_knn_t(const DatasetDev &ds, const Plan &pl, const float *qx,
                         const float *qy, int k, const Scratch &sc, int *err, cudaStream_t st)
{
    constexpr int Q = knn_q<KP>();
    const size_t dyn = IDX ? sizeof(int32_t) * Q * KP * kThreads : 0;
    auto fn = f32_knn_kernel<KP, Q, IDX>;
    if (dyn > 0) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(dyn));
        if (e != cudaSuccess)
            return e;
    }
    dim3 grid(pl.knn.qblocks, pl.knn.splits);
    fn<<<grid, kThreads, dyn, st>>>(ds, pl.m, pl.knn, qx, qy, k,
                                    static_cast<float *>(sc.part_d2), sc.part_idx, err);
    return cudaGetLastError();
}

template <int KP>
int knn_slots_t(bool with_idx)
{
    constexpr int Q = knn_q<KP>();
    int n = 0;
    if (with_idx) {
        const size_t dyn = sizeof(int32_t) * Q * KP * kThreads;
        cudaFuncSetAttribute(f32_knn_kernel<KP, Q, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(dyn));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f32_knn_kernel<KP, Q, true>, kThreads,
                                                      dyn);
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f32_knn_kernel<KP, Q, false>,
                                                      kThreads, 0);
    }
    return n > 0 ? n : 1;
}

}  // namespace

int f32_list_length(int k, int kp_min)
{
    return f32dev::kp_for(k, kp_min);
}

int f32_knn_queries_per_block(int kp)
{
    return kThreads * (kp <= 16 ? 4 : 2);
}

int f32_w_queries_per_block(int qw)
{
    return kThreads * qw;
}

int f32_knn_slots_per_sm(int kp, bool with_idx)
{
    switch (kp) {
    case 8: return knn_slots_t<8>(with_idx);
    case 12: return knn_slots_t<12>(with_idx);
    case 16: return knn_slots_t<16>(with_idx);
    default: return knn_slots_t<32>(with_idx);
    }
}

template <int Q, int TW>
int w_slots_t()
{
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f32_weights_kernel<Q, TW>, kThreads, 0);
    return n > 0 ? n : 1;
}

int f32_w_slots_per_sm(int qw, int tw)
{
    if (tw == 256)
        return qw == 2 ? w_slots_t<2, 256>()
                       : (qw == 8 ? w_slots_t<8, 256>() : w_slots_t<4, 256>());
    return qw == 2 ? w_slots_t<2, 512>() : (qw == 8 ? w_slots_t<8, 512>() : w_slots_t<4, 512>());
}

cudaError_t launch_f32_knn(const DatasetDev &ds, const Plan &pl, const float *qx,
                           const float *qy, int k, const Scratch &sc, int *err,
                           cudaStream_t st)
{
    switch (pl.kp) {
    case 8:
        return pl.with_idx ? launch_knn_t<8, true>(ds, pl, qx, qy, k, sc, err, st)
                           : launch_knn_t<8, false>(ds, pl, qx, qy, k, sc, err, st);
    case 12:
        return pl.with_idx ? launch_knn_t<12, true>(ds, pl, qx, qy, k, sc, err, st)
                           : launch_knn_t<12, false>(ds, pl, qx, qy, k, sc, err, st);
    case 16:
        return pl.with_idx ? launch_knn_t<16, true>(ds, pl, qx, qy, k, sc, err, st)
                           : launch_knn_t<16, false>(ds, pl, qx, qy, k, sc, err, st);
    default:
        return pl.with_idx ? launch_knn_t<32, true>(ds, pl, qx, qy, k, sc, err, st)
                           : launch_knn_t<32, false>(ds, pl, qx, qy, k, sc, err, st);
    }
}

cudaError_t launch_f32_select(const Plan &pl, int k, double r_exp, const AlphaMap &am,
                              const Scratch &sc, float *out_alpha, int32_t *out_knn,
                              cudaStream_t st, const uint32_t *perm)
{
    const int64_t blocks = (pl.m + 255) / 256;
    f32_select_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(
        pl.m, pl.knn.splits, k, r_exp, am, static_cast<const float *>(sc.part_d2),
        pl.with_idx ? sc.part_idx : nullptr, static_cast<QParamF32 *>(sc.qparam), out_alpha,
        out_knn, perm);
    return cudaGetLastError();
}

cudaError_t launch_f32_knn_warp(const DatasetDev &ds, int64_t m, const float *qx,
                                const float *qy, int k, const Scratch &sc, int sm_count,
                                cudaStream_t st)
{
    constexpr int W = kThreads / 32;
    const int64_t want = (m + W - 1) / W;
    const int64_t cap = static_cast<int64_t>(sm_count) * 16;
    const unsigned grid = static_cast<unsigned>(std::max<int64_t>(1, std::min(want, cap)));
    f32_knn_warp_kernel<<<grid, kThreads, 0, st>>>(ds, m, qx, qy, k,
                                                   static_cast<float *>(sc.part_d2),
                                                   sc.part_idx);
    return cudaGetLastError();
}

cudaError_t launch_f32_knn_cull(const DatasetDev &ds, const Plan &pl, const float *sqx,
                                const float *sqy, int k, const Scratch &sc, int *err,
                                cudaStream_t st)
{
    const bool q2 = pl.kq == 2;
#define AIDW_CULL(KP, Q)                                                                       \
    return pl.with_idx ? launch_cull_t<KP, Q, true>(ds, pl, sqx, sqy, k, sc, err, st)         \
                       : launch_cull_t<KP, Q, false>(ds, pl, sqx, sqy, k, sc, err, st)
    switch (pl.kp) {
    case 8:
        if (q2)
            AIDW_CULL(8, 2);
        AIDW_CULL(8, 4);
    case 12:
        if (q2)
            AIDW_CULL(12, 2);
        AIDW_CULL(12, 4);
    case 16:
        if (q2)
            AIDW_CULL(16, 2);
        AIDW_CULL(16, 4);
    default:
        AIDW_CULL(32, 2);
    }
#undef AIDW_CULL
}

cudaError_t launch_f32_weights(const DatasetDev &ds, const Plan &pl, const float *qx,
                               const float *qy, const Scratch &sc, int *err, cudaStream_t st)
{
    dim3 grid(pl.w.qblocks, pl.w.splits);
    auto fn = f32_weights_kernel<4, 512>;
    if (pl.tw == 256)
        fn = pl.qw == 2 ? f32_weights_kernel<2, 256>
                        : (pl.qw == 8 ? f32_weights_kernel<8, 256> : f32_weights_kernel<4, 256>);
    else
        fn = pl.qw == 2 ? f32_weights_kernel<2, 512>
                        : (pl.qw == 8 ? f32_weights_kernel<8, 512> : f32_weights_kernel<4, 512>);
    fn<<<grid, kThreads, 0, st>>>(ds, pl.m, pl.w, qx, qy,
                                  static_cast<const QParamF32 *>(sc.qparam),
                                  static_cast<float *>(sc.part_sum), err);
    return cudaGetLastError();
}

cudaError_t launch_f32_finalize(const Plan &pl, const Scratch &sc, float *out, cudaStream_t st,
                                const uint32_t *perm)
{
    const int64_t blocks = (pl.m + 255) / 256;
    f32_finalize_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(
        pl.m, pl.w.splits, static_cast<const float *>(sc.part_sum), out, perm);
    return cudaGetLastError();
}

}  // namespace aidw
