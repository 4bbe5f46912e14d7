// FP32 ("F32C") kernels of the AIDW hot path for sm_103a.
//
// Phase 1 (Sec. 2.2 Step 1, kNN procedure of Sec. 3.1.2) and phase 2 (Eq. 1 over all data
// points, Sec. 3.2.1) are two all-pairs scans of the data points against blocks of queries:
//   f32_knn_kernel      per (query block, data split): per-query sorted list of the k smallest
//                       squared distances (and optionally their indices), in registers
//   f32_select_kernel   per query: merge the split lists, r_obs (Eq. 3, FP32 pairwise sum),
//                       R (Eq. 2, 4), mu (Eq. 5), alpha (Eq. 6) in FP64 -> phase-2 parameters
//   f32_weights_kernel  per (query block, data split): sum w and sum w z with
//                       w = d^-alpha (d1/d)^... normalised by the nearest distance, MUFU lg2/ex2,
//                       chunk sums merged by Kahan steps
//   f32_finalize_kernel per query: merge split sums in FP64, Z = sum(w z) / sum(w) (Eq. 1)
// Data tiles stream through shared memory with one-dimensional TMA bulk copies into a double
// buffer completed on mbarriers; every thread keeps Q queries in registers and reads each
// data point as a broadcast from shared memory.
#include <math_constants.h>

#include "aidw_internal.cuh"

namespace aidw {
namespace {

constexpr int kChunkKnn = 8;   // points between neighbour-list threshold checks
constexpr int kChunkW = 32;    // points summed in plain FP32 before a Kahan merge

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

// Bounded wait for both buffers' outstanding copies after an abandoned scan.
__device__ __forceinline__ void drain(uint64_t *bar, int t, int ntiles)
{
    for (int u = t; u < ntiles && u < t + 2; ++u)
        (void)mbar_wait(&bar[u & 1], (u >> 1) & 1);
}

// ---------------------------------------------------------------------------------------------
// Phase 1: per (query block, split) neighbour lists.
//
// Each thread owns Q queries, processed as Q/2 packed pairs. For every data point and pair the
// hot loop evaluates, with FP32x2 instructions, v = dx^2 + (dy^2 - T') where T' is the k-th
// squared distance enlarged by 2^-20 (relative); the sign bits of v are OR-ed per query over a
// 16-point chunk. A negative v is necessary for a point to enter the list: if the exact FP32
// distance d2 = fl(dx^2 + fl(dy^2)) is below T then the real dx^2 + dy^2 is below T(1 + 2^-23)
// and v, computed with at most u T' of error, stays below zero. Only for a query whose sign bit
// is set the chunk is rescanned with the exact distance, which alone decides insertion, so the
// neighbour lists are exactly those of the plain scan.
// ---------------------------------------------------------------------------------------------
constexpr float kFilterMargin = 1.0f + 9.5367431640625e-07f;  // 1 + 2^-20

__device__ __forceinline__ float neg_filter_threshold(float kth)
{
    return -(kth * kFilterMargin);
}

__device__ __forceinline__ uint32_t sign_or3(uint32_t acc, float a, float b)
{
    return acc | __float_as_uint(a) | __float_as_uint(b);
}

template <int KP, int Q, bool IDX>
__global__ void __launch_bounds__(kThreads)
f32_knn_kernel(DatasetDev ds, int64_t m, PassPlan pp, const float *__restrict__ qx,
               const float *__restrict__ qy, int k, float *__restrict__ part_d2,
               int32_t *__restrict__ part_idx, int *__restrict__ err)
{
    static_assert(Q % 2 == 0, "queries are processed in packed pairs");
    constexpr int H = Q / 2;
    __shared__ __align__(128) float4 tile[2][kTileF32Knn];
    __shared__ __align__(8) uint64_t bar[2];
    extern __shared__ int32_t idx_smem[];  // [Q][KP][kThreads] when IDX

    const int tid = threadIdx.x;
    const int s = blockIdx.y;
    const int64_t qbase = static_cast<int64_t>(blockIdx.x) * pp.q_per_block;
    const int64_t p_begin = static_cast<int64_t>(s) * pp.split_len;
    const int64_t p_end = min(p_begin + pp.split_len, ds.n_pad);
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

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    constexpr uint32_t kBytes = kTileF32Knn * sizeof(float4);
    if (tid == 0) {
        for (int t = 0; t < 2 && t < ntiles; ++t) {
            mbar_arrive_expect_tx(&bar[t], kBytes);
            tma_load_1d(tile[t], ds.nxy2 + p_begin + static_cast<int64_t>(t) * kTileF32Knn,
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
        const float4 *tb = tile[b];
        const int64_t pbase = p_begin + static_cast<int64_t>(t) * kTileF32Knn;
        for (int c = 0; c < kTileF32Knn; c += kChunkKnn) {
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
        __syncthreads();
        if (tid == 0 && t + 2 < ntiles) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bar[b], kBytes);
            tma_load_1d(tile[b], ds.nxy2 + pbase + 2 * kTileF32Knn, kBytes, &bar[b]);
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
// Selection: merge split lists, Eq. 3 (FP32 pairwise), Eq. 2/4/5/6 (FP64).
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
f32_select_kernel(int64_t m, int S, int k, double r_exp, AlphaMap am,
                  const float *__restrict__ part_d2, const int32_t *__restrict__ part_idx,
                  QParamF32 *__restrict__ qp, float *__restrict__ out_alpha,
                  int32_t *__restrict__ out_knn)
{
    const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q >= m)
        return;
    int cur[kMaxSplits];
    float hd[kMaxSplits];
    int32_t hi[kMaxSplits];
    for (int s = 0; s < S; ++s) {
        cur[s] = 0;
        const int64_t o = static_cast<int64_t>(s) * k * m + q;
        hd[s] = part_d2[o];
        hi[s] = part_idx ? part_idx[o] : 0;
    }
    float d[AIDW_MAX_K];
    for (int r = 0; r < k; ++r) {
        int bs = 0;
        for (int s = 1; s < S; ++s)
            if (hd[s] < hd[bs] || (hd[s] == hd[bs] && hi[s] < hi[bs]))
                bs = s;
        d[r] = hd[bs];
        if (out_knn)
            out_knn[q * k + r] = hi[bs];
        if (++cur[bs] < k) {
            const int64_t o = (static_cast<int64_t>(bs) * k + cur[bs]) * m + q;
            hd[bs] = part_d2[o];
            hi[bs] = part_idx ? part_idx[o] : 0;
        } else {
            hd[bs] = CUDART_INF_F;
            hi[bs] = INT32_MAX;
        }
    }
    const float d1 = d[0];
    // Eq. 3: mean of the k distances; sqrt of (d2 - eps) undoes the coincidence offset.
    float v[AIDW_MAX_K];
    for (int r = 0; r < k; ++r)
        v[r] = __fsqrt_rn(__fsub_rn(d[r], kEpsF32));
    for (int stride = 1; stride < k; stride *= 2)
        for (int i = 0; i + stride < k; i += 2 * stride)
            v[i] = __fadd_rn(v[i], v[i + stride]);
    const double r_obs = static_cast<double>(v[0]) / k;
    const double R = r_obs / r_exp;                  // Eq. 4
    const double mu = membership_eq5(R, am);         // Eq. 5
    const double alpha = alpha_eq6(mu, am);          // Eq. 6

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
    qp[q] = o;
    if (out_alpha)
        out_alpha[q] = static_cast<float>(alpha);
}

// ---------------------------------------------------------------------------------------------
// Phase 2: per (query block, split) weighted sums. Q queries per thread in packed pairs: the
// distance, power scale and both sums run as FP32x2 instructions, lg2 and ex2 on the MUFU.
// ---------------------------------------------------------------------------------------------
template <int Q>
__global__ void __launch_bounds__(kThreads)
f32_weights_kernel(DatasetDev ds, int64_t m, PassPlan pp, const float *__restrict__ qx,
                   const float *__restrict__ qy, const QParamF32 *__restrict__ qp,
                   float *__restrict__ part_sum, int *__restrict__ err)
{
    static_assert(Q % 2 == 0, "queries are processed in packed pairs");
    constexpr int H = Q / 2;
    __shared__ __align__(128) float4 txy[2][kTileF32W];
    __shared__ __align__(128) float2 tz[2][kTileF32W];
    __shared__ __align__(8) uint64_t bar[2];

    const int tid = threadIdx.x;
    const int s = blockIdx.y;
    const int64_t qbase = static_cast<int64_t>(blockIdx.x) * pp.q_per_block;
    const int64_t p_begin = static_cast<int64_t>(s) * pp.split_len;
    const int64_t p_end = min(p_begin + pp.split_len, ds.n_pad);
    const int ntiles = static_cast<int>((p_end - p_begin) / kTileF32W);

    float2 qxp[H], qyp[H], nsp[H], ccp[H];
    float hw[Q], cw[Q], hz[Q], cz[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const int64_t q = min(qbase + j * kThreads + tid, m - 1);
        const QParamF32 o = qp[q];
        const float a = qx[q], b = qy[q];
        if (j & 1) {
            qxp[j / 2].y = a;
            qyp[j / 2].y = b;
            nsp[j / 2].y = o.neg_s;
            ccp[j / 2].y = o.c;
        } else {
            qxp[j / 2].x = a;
            qyp[j / 2].x = b;
            nsp[j / 2].x = o.neg_s;
            ccp[j / 2].x = o.c;
        }
        hw[j] = cw[j] = hz[j] = cz[j] = 0.0f;
    }
    const float2 eps2 = make_float2(kEpsF32, kEpsF32);

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    constexpr uint32_t kBxy = kTileF32W * sizeof(float4);
    constexpr uint32_t kBz = kTileF32W * sizeof(float2);
    if (tid == 0) {
        for (int t = 0; t < 2 && t < ntiles; ++t) {
            const int64_t o = p_begin + static_cast<int64_t>(t) * kTileF32W;
            mbar_arrive_expect_tx(&bar[t], kBxy + kBz);
            tma_load_1d(txy[t], ds.nxy2 + o, kBxy, &bar[t]);
            tma_load_1d(tz[t], ds.zz + o, kBz, &bar[t]);
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
        for (int c = 0; c < kTileF32W; c += kChunkW) {
            float2 sw[H], sz[H];
#pragma unroll
            for (int h = 0; h < H; ++h)
                sw[h] = sz[h] = make_float2(0.0f, 0.0f);
#pragma unroll 4
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
            const int64_t o = p_begin + static_cast<int64_t>(t + 2) * kTileF32W;
            mbar_arrive_expect_tx(&bar[b], kBxy + kBz);
            tma_load_1d(txy[b], ds.nxy2 + o, kBxy, &bar[b]);
            tma_load_1d(tz[b], ds.zz + o, kBz, &bar[b]);
        }
    }
    if (!ok)
        return;
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
}

__global__ void __launch_bounds__(256)
f32_finalize_kernel(int64_t m, int S, const float *__restrict__ part_sum,
                    float *__restrict__ out)
{
    const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q >= m)
        return;
    double W = 0.0, WZ = 0.0;
    for (int s = 0; s < S; ++s) {
        const float *o = part_sum + static_cast<int64_t>(s) * 4 * m + q;
        W += static_cast<double>(o[0]) + static_cast<double>(o[m]);
        WZ += static_cast<double>(o[2 * m]) + static_cast<double>(o[3 * m]);
    }
    out[q] = static_cast<float>(WZ / W);  // Eq. 1
}

constexpr int kQW32 = 8;

template <int KP>
constexpr int knn_q()
{
    return KP <= 16 ? 4 : 2;
}

// Register list length for k: the smallest of 8, 12, 16, 32 that holds k.
inline int kp_for(int k)
{
    return k <= 8 ? 8 : (k <= 12 ? 12 : (k <= 16 ? 16 : 32));
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
    return kThreads * (k <= 16 ? 4 : 2);
}

int f32_w_queries_per_block()
{
    return kThreads * kQW32;
}

int f32_knn_slots_per_sm(int k, bool with_idx)
{
    switch (kp_for(k)) {
    case 8: return knn_slots_t<8>(with_idx);
    case 12: return knn_slots_t<12>(with_idx);
    case 16: return knn_slots_t<16>(with_idx);
    default: return knn_slots_t<32>(with_idx);
    }
}

int f32_w_slots_per_sm()
{
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f32_weights_kernel<kQW32>, kThreads, 0);
    return n > 0 ? n : 1;
}

cudaError_t launch_f32_knn(const DatasetDev &ds, const Plan &pl, const float *qx,
                           const float *qy, int k, const Scratch &sc, int *err,
                           cudaStream_t st)
{
    switch (kp_for(k)) {
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
                              cudaStream_t st)
{
    const int64_t blocks = (pl.m + 255) / 256;
    f32_select_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(
        pl.m, pl.knn.splits, k, r_exp, am, static_cast<const float *>(sc.part_d2),
        pl.with_idx ? sc.part_idx : nullptr, static_cast<QParamF32 *>(sc.qparam), out_alpha,
        out_knn);
    return cudaGetLastError();
}

cudaError_t launch_f32_weights(const DatasetDev &ds, const Plan &pl, const float *qx,
                               const float *qy, const Scratch &sc, int *err, cudaStream_t st)
{
    dim3 grid(pl.w.qblocks, pl.w.splits);
    f32_weights_kernel<kQW32><<<grid, kThreads, 0, st>>>(
        ds, pl.m, pl.w, qx, qy, static_cast<const QParamF32 *>(sc.qparam),
        static_cast<float *>(sc.part_sum), err);
    return cudaGetLastError();
}

cudaError_t launch_f32_finalize(const Plan &pl, const Scratch &sc, float *out, cudaStream_t st)
{
    const int64_t blocks = (pl.m + 255) / 256;
    f32_finalize_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(
        pl.m, pl.w.splits, static_cast<const float *>(sc.part_sum), out);
    return cudaGetLastError();
}

}  // namespace aidw
