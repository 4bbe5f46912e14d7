// AIDW_F64X phase 2 for sm_103a: Eq. 1 over all data points with FP64 inputs and output, the
// squared distance formed in FP64 exactly as the FP64 path forms it, and the rest of each pair's
// work (log2, the adaptive power, exp2, both weighted sums) in double-float arithmetic on the
// FP32 pipes (df_math.cuh). GB300 runs FP64 at 1/64 of its FP32 rate, so the four FP64
// operations of the distance bound this scan and the hundred-odd FP32 operations per pair run
// beside them. Phase 1, the selection of alpha (Eq. 2-6) and the final division stay the FP64
// path's kernels.
#include <math_constants.h>

#include "aidw_internal.cuh"
#include "df_math.cuh"

namespace aidw {
namespace {

constexpr int kQX = 2;       // queries per thread
constexpr int kChunkX = 16;  // points summed per double-float merge

__device__ __forceinline__ double dist2_eps_x(double qx, double qy, double px, double py)
{
    const double dx = __dsub_rn(qx, px);
    const double dy = __dsub_rn(qy, py);
    return __fma_rn(dx, dx, __fma_rn(dy, dy, kEpsF64));
}

__device__ __forceinline__ void drain_x(uint64_t *bar, int t, int ntiles)
{
    for (int u = t; u < ntiles && u < t + 2; ++u)
        (void)mbar_wait(&bar[u & 1], (u >> 1) & 1);
}

// One block of kThreads * Q queries against one data split; per query the two double-float
// sums (w, w z) go to part_sum as four doubles (sum of w hi, lo, sum of w z hi, lo), which the
// FP64 finalisation adds up.
template <int Q>
__global__ void __launch_bounds__(kThreads)
f64x_weights_kernel(DatasetDev ds, int64_t m, PassPlan pp, const double *__restrict__ qx,
                    const double *__restrict__ qy, const QParamF64X *__restrict__ qp,
                    double *__restrict__ part_sum, int *__restrict__ err)
{
    __shared__ __align__(128) double2 txy[2][kTileF64W];
    __shared__ __align__(128) double tz[2][kTileF64W];
    __shared__ __align__(16) float2 tzf[kTileF64W];  // z of the current tile, double-float
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ dfm::Tables tabs;

    const int tid = threadIdx.x;
    const int s = blockIdx.y;
    dfm::load_tables(tabs);  // ordered before use by the barrier after the mbarrier set-up
    const int64_t qbase = static_cast<int64_t>(blockIdx.x) * pp.q_per_block;
    const int64_t p_begin = static_cast<int64_t>(s) * pp.split_len;
    const int64_t p_end = min(p_begin + pp.split_len, ds.n_pad);
    const int ntiles = static_cast<int>((p_end - p_begin) / kTileF64W);

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    constexpr uint32_t kBxy = kTileF64W * sizeof(double2);
    constexpr uint32_t kBz = kTileF64W * sizeof(double);
    if (tid == 0) {
        for (int t = 0; t < 2 && t < ntiles; ++t) {
            const int64_t o = p_begin + static_cast<int64_t>(t) * kTileF64W;
            mbar_arrive_expect_tx(&bar[t], kBxy + kBz);
            tma_load_1d(txy[t], ds.xy64 + o, kBxy, &bar[t]);
            tma_load_1d(tz[t], ds.z64 + o, kBz, &bar[t]);
        }
    }

    double qxr[Q], qyr[Q];
    float kh[Q], kl[Q], Wh[Q], Wl[Q], Zh[Q], Zl[Q];
    dfm::RefLog ref[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const int64_t q = min(qbase + j * kThreads + tid, m - 1);
        qxr[j] = qx[q];
        qyr[j] = qy[q];
        const QParamF64X o = qp[q];
        kh[j] = __double2float_rn(o.kappa);
        kl[j] = __double2float_rn(o.kappa - static_cast<double>(kh[j]));
        ref[j] = dfm::ref_log(o.d1sq, tabs);
        Wh[j] = Wl[j] = Zh[j] = Zl[j] = 0.0f;
    }

    bool ok = true;
    for (int t = 0; t < ntiles; ++t) {
        const int b = t & 1;
        const bool got = mbar_wait(&bar[b], (t >> 1) & 1);
        if (!__syncthreads_and(got)) {
            ok = false;
            if (tid == 0) {
                atomicOr(err, kErrTimeout);
                drain_x(bar, t, ntiles);
            }
            break;
        }
        for (int i = tid; i < kTileF64W; i += kThreads) {
            const double z = tz[b][i];
            const float h = __double2float_rn(z);
            tzf[i] = make_float2(h, __double2float_rn(z - static_cast<double>(h)));
        }
        __syncthreads();
        for (int c = 0; c < kTileF64W; c += kChunkX) {
            float aw[Q], cw[Q], az[Q], cz[Q];
#pragma unroll
            for (int j = 0; j < Q; ++j)
                aw[j] = cw[j] = az[j] = cz[j] = 0.0f;
#pragma unroll 2
            for (int u = 0; u < kChunkX; ++u) {
                const double2 p = txy[b][c + u];
                const float2 pz = tzf[c + u];
#pragma unroll
                for (int j = 0; j < Q; ++j) {
                    const double d2 = dist2_eps_x(qxr[j], qyr[j], p.x, p.y);
                    float vh, vl, yh, yl, wh, wl, e, zh, zl;
                    dfm::log2_ratio(d2, ref[j], tabs, vh, vl);
                    dfm::mul(kh[j], kl[j], vh, vl, yh, yl);  // -y = kappa log2(d^2 / d1^2)
                    dfm::exp2_df(-yh, -yl, tabs, wh, wl);
                    dfm::two_sum(aw[j], wh, aw[j], e);
                    cw[j] = __fadd_rn(cw[j], __fadd_rn(e, wl));
                    dfm::mul(wh, wl, pz.x, pz.y, zh, zl);
                    dfm::two_sum(az[j], zh, az[j], e);
                    cz[j] = __fadd_rn(cz[j], __fadd_rn(e, zl));
                }
            }
#pragma unroll
            for (int j = 0; j < Q; ++j) {
                dfm::add(Wh[j], Wl[j], aw[j], cw[j]);
                dfm::add(Zh[j], Zl[j], az[j], cz[j]);
            }
        }
        __syncthreads();
        if (tid == 0 && t + 2 < ntiles) {
            fence_proxy_async_smem();
            const int64_t o = p_begin + static_cast<int64_t>(t + 2) * kTileF64W;
            mbar_arrive_expect_tx(&bar[b], kBxy + kBz);
            tma_load_1d(txy[b], ds.xy64 + o, kBxy, &bar[b]);
            tma_load_1d(tz[b], ds.z64 + o, kBz, &bar[b]);
        }
    }
    if (!ok)
        return;
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const int64_t q = qbase + j * kThreads + tid;
        if (q >= m)
            continue;
        double *o = part_sum + static_cast<int64_t>(s) * 4 * m + q;
        o[0] = Wh[j];
        o[m] = Wl[j];
        o[2 * m] = Zh[j];
        o[3 * m] = Zl[j];
    }
}

__global__ void df_weight_probe_kernel(const double *__restrict__ d2,
                                       const double *__restrict__ d1sq,
                                       const double *__restrict__ kappa, int64_t n,
                                       double *__restrict__ v, double *__restrict__ w)
{
    __shared__ dfm::Tables tabs;
    dfm::load_tables(tabs);
    __syncthreads();
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const dfm::RefLog ref = dfm::ref_log(d1sq[i], tabs);
        const float kh = __double2float_rn(kappa[i]);
        const float kl = __double2float_rn(kappa[i] - static_cast<double>(kh));
        float vh, vl, yh, yl, wh, wl;
        dfm::log2_ratio(d2[i], ref, tabs, vh, vl);
        dfm::mul(kh, kl, vh, vl, yh, yl);
        dfm::exp2_df(-yh, -yl, tabs, wh, wl);
        v[i] = static_cast<double>(vh) + static_cast<double>(vl);
        w[i] = static_cast<double>(wh) + static_cast<double>(wl);
    }
}

}  // namespace

int f64x_w_queries_per_block()
{
    return kThreads * kQX;
}

int f64x_w_slots_per_sm()
{
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f64x_weights_kernel<kQX>, kThreads, 0);
    return n > 0 ? n : 1;
}

cudaError_t launch_f64x_weights(const DatasetDev &ds, const Plan &pl, const double *qx,
                                const double *qy, const Scratch &sc, int *err, cudaStream_t st)
{
    dim3 grid(pl.w.qblocks, pl.w.splits);
    f64x_weights_kernel<kQX><<<grid, kThreads, 0, st>>>(
        ds, pl.m, pl.w, qx, qy, static_cast<const QParamF64X *>(sc.qparam),
        static_cast<double *>(sc.part_sum), err);
    return cudaGetLastError();
}

}  // namespace aidw

extern "C" int aidw_debug_df_weight(const double *d2, const double *d1sq, const double *kappa,
                                    int64_t n, double *v, double *w)
{
    if (n < 0 || (n > 0 && (!d2 || !d1sq || !kappa || !v || !w)))
        return AIDW_ERR_INVALID_ARG;
    if (n == 0)
        return AIDW_OK;
    const unsigned blocks = static_cast<unsigned>(n < 256 * 1024 ? (n + 255) / 256 : 1024);
    aidw::df_weight_probe_kernel<<<blocks, 256>>>(d2, d1sq, kappa, n, v, w);
    return cudaDeviceSynchronize() == cudaSuccess ? AIDW_OK : AIDW_ERR_CUDA;
}
