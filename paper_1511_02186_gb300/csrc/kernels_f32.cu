// FP32 ("F32C") per-call kernels of the AIDW hot path for sm_103a.
//
//   f32_knn_kernel      grid (query blocks, data splits): phase-1 unit per CTA (neighbour lists)
//   f32_select_kernel   one thread per query: split merge, Eq. 2-6 -> phase-2 parameters
//   f32_weights_kernel  grid (query blocks, data splits): phase-2 unit per CTA (weighted sums)
//   f32_finalize_kernel one thread per query: split merge, Eq. 1 ratio in FP64
// The unit bodies live in f32_device.cuh and are shared with the persistent batched kernel.
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

// ---------------------------------------------------------------------------------------------
// Phase 1 over Z-ordered queries, one CTA per query block and no data splits. The CTA takes the
// bounding box of its queries, computes for every data tile a lower bound of the squared
// distance between the two boxes, sorts the tiles by it (bitonic sort in shared memory) and
// visits them nearest first. After each tile it takes T = the largest k-th squared distance of
// its queries; it stops at the first tile whose bound exceeds T. No skipped point could enter a
// list: its exact FP32 distance is at least the box bound (the bound is shrunk by 2^-20 to
// cover rounding), which exceeds every query's current k-th distance.
// ---------------------------------------------------------------------------------------------
constexpr float kBoundShrink = 1.0f - 9.5367431640625e-07f;  // 1 - 2^-20

template <int KP, int Q, bool IDX>
__global__ void __launch_bounds__(kThreads)
f32_knn_cull_kernel(DatasetDev ds, int64_t m, int qpb, int ntiles, int ntiles_p2,
                    const float *__restrict__ sqx, const float *__restrict__ sqy, int k,
                    float *__restrict__ part_d2, int32_t *__restrict__ part_idx,
                    int *__restrict__ err)
{
    constexpr int H = Q / 2;
    constexpr int W = kThreads / 32;
    extern __shared__ unsigned long long order[];  // [ntiles_p2], then the index lists if IDX
    __shared__ __align__(128) float4 tile[2][kTileF32Knn];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ float red[4][W];
    __shared__ float4 s_box;
    __shared__ float s_thr;
    __shared__ int s_issued;
    int32_t *idx_smem = reinterpret_cast<int32_t *>(order + ntiles_p2);
    init_tile_barriers(bar);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t qbase = static_cast<int64_t>(blockIdx.x) * qpb;

    float2 qxp[H], qyp[H], nthr[H];
    float L[Q][KP];
    float bx0 = CUDART_INF_F, by0 = CUDART_INF_F, bx1 = -CUDART_INF_F, by1 = -CUDART_INF_F;
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const int64_t q = min(qbase + j * kThreads + tid, m - 1);
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
        s_box = b;
        s_thr = CUDART_INF_F;
    }
    __syncthreads();
    const float4 qb = s_box;
    // Lower bounds of the box-to-box squared distance, keyed for an ascending sort.
    for (int t = tid; t < ntiles_p2; t += kThreads) {
        unsigned long long key = ~0ull;
        if (t < ntiles) {
            const float4 tb = ds.tile_box[t];
            const float dx = fmaxf(0.0f, fmaxf(tb.x - qb.z, qb.x - tb.z));
            const float dy = fmaxf(0.0f, fmaxf(tb.y - qb.w, qb.y - tb.w));
            const float lb = __fmul_rn(__fmaf_rn(dx, dx, __fmul_rn(dy, dy)), kBoundShrink);
            key = (static_cast<unsigned long long>(__float_as_uint(lb)) << 32) |
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
            const int64_t t = static_cast<int64_t>(order[issued] & 0xffffffffull);
            mbar_arrive_expect_tx(&bar[issued], kBytes);
            tma_load_1d(tile[issued], ds.nxy2 + t * kTileF32Knn, kBytes, &bar[issued]);
        }
        s_issued = issued;
    }
    __syncthreads();
    int i = 0;
    bool ok = true;
    for (; i < ntiles; ++i) {
        const unsigned long long key = order[i];
        if (__uint_as_float(static_cast<uint32_t>(key >> 32)) > s_thr)
            break;
        const int b = i & 1;
        const bool got = mbar_wait(&bar[b], (i >> 1) & 1);
        if (!__syncthreads_and(got)) {
            ok = false;
            break;
        }
        const int64_t t = static_cast<int64_t>(key & 0xffffffffull);
        knn_tile<KP, Q, IDX>(tile[b], t * kTileF32Knn, qxp, qyp, nthr, L, idx_smem);
        float mx = -CUDART_INF_F;
#pragma unroll
        for (int j = 0; j < Q; ++j)
            mx = fmaxf(mx, L[j][KP - 1]);
        for (int o = 16; o > 0; o >>= 1)
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0)
            red[0][warp] = mx;
        __syncthreads();
        if (tid == 0) {
            float v = red[0][0];
            for (int w = 1; w < W; ++w)
                v = fmaxf(v, red[0][w]);
            s_thr = v;
            const int nx = i + 2;
            if (nx < ntiles &&
                __uint_as_float(static_cast<uint32_t>(order[nx] >> 32)) <= v) {
                const int64_t tn = static_cast<int64_t>(order[nx] & 0xffffffffull);
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&bar[b], kBytes);
                tma_load_1d(tile[b], ds.nxy2 + tn * kTileF32Knn, kBytes, &bar[b]);
                s_issued = nx + 1;
            }
        }
        __syncthreads();
    }
    // Wait (bounded) for tiles issued but not consumed before leaving.
    if (tid == 0) {
        for (int u = i; u < s_issued; ++u)
            (void)mbar_wait(&bar[u & 1], (u >> 1) & 1);
        if (!ok)
            atomicOr(err, kErrTimeout);
    }
    if (!ok)
        return;
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const int64_t q = qbase + j * kThreads + tid;
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
}

template <int Q>
__global__ void __launch_bounds__(kThreads)
f32_weights_kernel(DatasetDev ds, int64_t m, PassPlan pp, const float *__restrict__ qx,
                   const float *__restrict__ qy, const QParamF32 *__restrict__ qp,
                   float *__restrict__ part_sum, int *__restrict__ err)
{
    __shared__ __align__(128) float4 txy[2][kTileF32W];
    __shared__ __align__(128) float2 tz[2][kTileF32W];
    __shared__ __align__(8) uint64_t bar[2];
    init_tile_barriers(bar);
    TileSeq ts{bar, 0u};
    const int s = blockIdx.y;
    const int64_t p_begin = static_cast<int64_t>(s) * pp.split_len;
    const int64_t p_end = min(p_begin + pp.split_len, ds.n_pad);
    weights_unit<Q>(ds, m, static_cast<int64_t>(blockIdx.x) * pp.q_per_block, p_begin, p_end,
                    qx, qy, qp, s, part_sum, err, txy, tz, ts);
}

__global__ void __launch_bounds__(256)
f32_finalize_kernel(int64_t m, int S, const float *__restrict__ part_sum,
                    float *__restrict__ out, const uint32_t *__restrict__ perm)
{
    const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q < m)
        out[perm ? perm[q] : q] = finalize_query(q, m, S, part_sum);
}

template <int KP, bool IDX>
cudaError_t launch_cull_t(const DatasetDev &ds, const Plan &pl, const float *sqx,
                          const float *sqy, int k, const Scratch &sc, int *err, cudaStream_t st)
{
    constexpr int Q = knn_q<KP>();
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

int f32_knn_queries_per_block(int k)
{
    return kThreads * (f32dev::kp_for(k) <= 16 ? 4 : 2);
}

int f32_w_queries_per_block()
{
    return kThreads * f32dev::kQW32;
}

int f32_knn_slots_per_sm(int k, bool with_idx)
{
    switch (f32dev::kp_for(k)) {
    case 8: return knn_slots_t<8>(with_idx);
    case 12: return knn_slots_t<12>(with_idx);
    case 16: return knn_slots_t<16>(with_idx);
    default: return knn_slots_t<32>(with_idx);
    }
}

int f32_w_slots_per_sm()
{
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f32_weights_kernel<f32dev::kQW32>,
                                                  kThreads, 0);
    return n > 0 ? n : 1;
}

cudaError_t launch_f32_knn(const DatasetDev &ds, const Plan &pl, const float *qx,
                           const float *qy, int k, const Scratch &sc, int *err,
                           cudaStream_t st)
{
    switch (f32dev::kp_for(k)) {
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

cudaError_t launch_f32_knn_cull(const DatasetDev &ds, const Plan &pl, const float *sqx,
                                const float *sqy, int k, const Scratch &sc, int *err,
                                cudaStream_t st)
{
    switch (f32dev::kp_for(k)) {
    case 8:
        return pl.with_idx ? launch_cull_t<8, true>(ds, pl, sqx, sqy, k, sc, err, st)
                           : launch_cull_t<8, false>(ds, pl, sqx, sqy, k, sc, err, st);
    case 12:
        return pl.with_idx ? launch_cull_t<12, true>(ds, pl, sqx, sqy, k, sc, err, st)
                           : launch_cull_t<12, false>(ds, pl, sqx, sqy, k, sc, err, st);
    case 16:
        return pl.with_idx ? launch_cull_t<16, true>(ds, pl, sqx, sqy, k, sc, err, st)
                           : launch_cull_t<16, false>(ds, pl, sqx, sqy, k, sc, err, st);
    default:
        return pl.with_idx ? launch_cull_t<32, true>(ds, pl, sqx, sqy, k, sc, err, st)
                           : launch_cull_t<32, false>(ds, pl, sqx, sqy, k, sc, err, st);
    }
}

cudaError_t launch_f32_weights(const DatasetDev &ds, const Plan &pl, const float *qx,
                               const float *qy, const Scratch &sc, int *err, cudaStream_t st)
{
    dim3 grid(pl.w.qblocks, pl.w.splits);
    f32_weights_kernel<f32dev::kQW32><<<grid, kThreads, 0, st>>>(
        ds, pl.m, pl.w, qx, qy, static_cast<const QParamF32 *>(sc.qparam),
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
