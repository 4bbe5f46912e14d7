// The paper's own kernel designs, rebuilt for sm_103a as a measured comparison beside the
// optimized path (Sec. 3.1, Sec. 4.2): one thread per query; the naive version reads every data
// point from global memory, the tiled version stages blocks of data points in shared memory
// for the whole thread block (Sec. 3.1.1); the data sit in structure-of-arrays form (x[], y[],
// z[]) or as an array of aligned structures ({x, y, z, 0}, Sec. 3.1.3). Both phases scan all n
// points in the caller's order: phase 1 keeps the k smallest squared distances (Sec. 3.1.2)
// for r_obs (Eq. 3), phase 2 forms the weights of Eq. 1 over all points.
//
// The arithmetic per pair is the optimized path's (weights normalised by the nearest distance
// through log2 / exp2, chunk sums merged by compensated steps; in FP64 with the CUDA library's
// log2 / exp2 where the optimized path has its own table-driven pair), so the four variants of
// one precision produce the same bits and the comparison isolates data layout and tiling.
#include <math_constants.h>

#include <algorithm>

#include "aidw_runtime.h"

namespace aidw {
namespace {

constexpr int kBlock = 256;  // threads per block, and data points per shared-memory tile
constexpr int kChunk = 32;   // points summed plainly before a compensated merge

template <typename T>
struct alignas(4 * sizeof(T)) Point4 {
    T x, y, z, pad;
};

template <typename T>
struct Num;

template <>
struct Num<float> {
    static constexpr float kEps = kEpsF32;
    static constexpr float kCoinc = kCoincScaleF32;
    __device__ static float sub(float a, float b) { return __fsub_rn(a, b); }
    __device__ static float mul(float a, float b) { return __fmul_rn(a, b); }
    __device__ static float add(float a, float b) { return __fadd_rn(a, b); }
    __device__ static float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    __device__ static float sqrt(float a) { return __fsqrt_rn(a); }
    __device__ static float lg2(float a) { return lg2_approx(a); }
    __device__ static float ex2(float a) { return ex2_approx(a); }
    // Hides a value from the compiler so that lg2 of it runs on the MUFU like the per-pair lg2
    // (a compile-time lg2 of a constant need not equal the MUFU result).
    __device__ static float opaque(float a)
    {
        asm volatile("" : "+f"(a));
        return a;
    }
};

template <>
struct Num<double> {
    static constexpr double kEps = kEpsF64;
    static constexpr double kCoinc = kCoincScaleF64;
    __device__ static double sub(double a, double b) { return __dsub_rn(a, b); }
    __device__ static double mul(double a, double b) { return __dmul_rn(a, b); }
    __device__ static double add(double a, double b) { return __dadd_rn(a, b); }
    __device__ static double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
    __device__ static double sqrt(double a) { return __dsqrt_rn(a); }
    __device__ static double lg2(double a) { return log2(a); }
    __device__ static double ex2(double a) { return exp2(a); }
    __device__ static double opaque(double a)
    {
        asm volatile("" : "+d"(a));
        return a;
    }
};

// The caller-order copies of one dataset in the layout under test.
template <typename T>
struct Layout {
    const T *x, *y, *z;      // SoA
    const Point4<T> *p;      // AoaS
    int64_t n;
};

template <typename T, bool AOAS>
__device__ __forceinline__ void load_xy(const Layout<T> &d, int64_t i, T &x, T &y)
{
    if (AOAS) {
        const Point4<T> p = d.p[i];
        x = p.x;
        y = p.y;
    } else {
        x = d.x[i];
        y = d.y[i];
    }
}

template <typename T, bool AOAS>
__device__ __forceinline__ void load_xyz(const Layout<T> &d, int64_t i, T &x, T &y, T &z)
{
    if (AOAS) {
        const Point4<T> p = d.p[i];
        x = p.x;
        y = p.y;
        z = p.z;
    } else {
        x = d.x[i];
        y = d.y[i];
        z = d.z[i];
    }
}

// Phase 1 step: d2 as the oracle forms it (each product and sum rounded), then insertion into
// the ascending register list L[0..KP). The first KP - k slots hold -inf and never move, so the
// k nearest squared distances are L[KP - k .. KP - 1] and the insertion threshold is L[KP - 1]
// (compile-time indices only: the list stays in registers). d1 tracks the nearest.
template <typename T, int KP>
__device__ __forceinline__ void knn_step(T qx, T qy, T px, T py, T (&L)[KP], T &d1)
{
    using N = Num<T>;
    const T dx = N::sub(qx, px), dy = N::sub(qy, py);
    const T d2 = N::add(N::mul(dx, dx), N::mul(dy, dy));
    if (d2 < L[KP - 1]) {  // strict: an equal distance does not displace an earlier point
        T v = d2;
#pragma unroll
        for (int j = 0; j < KP; ++j) {
            const T lo = L[j] < v ? L[j] : v;
            v = L[j] < v ? v : L[j];
            L[j] = lo;
        }
        d1 = d2 < d1 ? d2 : d1;
    }
}

// Phase 2 step: w = 2^(c - s log2(d2 + eps)), plain chunk sums.
template <typename T>
__device__ __forceinline__ void weight_step(T qx, T qy, T px, T py, T pz, T neg_s, T c, T &sw,
                                            T &sz)
{
    using N = Num<T>;
    const T dx = N::sub(qx, px), dy = N::sub(qy, py);
    const T d2 = N::fma(dx, dx, N::fma(dy, dy, N::kEps));
    const T w = N::ex2(N::fma(N::lg2(d2), neg_s, c));
    sw = N::add(sw, w);
    sz = N::fma(w, pz, sz);
}

template <typename T, bool TILED, bool AOAS, int KP>
__global__ void __launch_bounds__(kBlock)
paper_aidw_kernel(Layout<T> d, const T *__restrict__ qx, const T *__restrict__ qy, int64_t m,
                  int k, double r_exp, AlphaMap am, T *__restrict__ out,
                  float *__restrict__ out_alpha)
{
    using N = Num<T>;
    __shared__ T sx[TILED ? kBlock : 1], sy[TILED ? kBlock : 1], sz[TILED ? kBlock : 1];
    const int64_t q = static_cast<int64_t>(blockIdx.x) * kBlock + threadIdx.x;
    const bool active = q < m;
    const T x0 = qx[active ? q : m - 1], y0 = qy[active ? q : m - 1];
    const int64_t n = d.n;

    // ---- phase 1: the k smallest squared distances ----
    T L[KP];
#pragma unroll
    for (int j = 0; j < KP; ++j)
        L[j] = j < KP - k ? -CUDART_INF : CUDART_INF;
    T d1 = CUDART_INF;
    if (TILED) {
        for (int64_t base = 0; base < n; base += kBlock) {
            const int64_t i = base + threadIdx.x;
            T px = CUDART_INF, py = CUDART_INF;
            if (i < n)
                load_xy<T, AOAS>(d, i, px, py);
            __syncthreads();
            sx[threadIdx.x] = px;
            sy[threadIdx.x] = py;
            __syncthreads();
            const int cnt = n - base < kBlock ? static_cast<int>(n - base) : kBlock;
            for (int t = 0; t < cnt; ++t)
                knn_step<T, KP>(x0, y0, sx[t], sy[t], L, d1);
        }
    } else {
        for (int64_t i = 0; i < n; ++i) {
            T px, py;
            load_xy<T, AOAS>(d, i, px, py);
            knn_step<T, KP>(x0, y0, px, py, L, d1);
        }
    }

    // ---- Eq. 3-6 ----
    T r_sum = 0;
#pragma unroll
    for (int j = 0; j < KP; ++j)
        if (j >= KP - k)
            r_sum = N::add(r_sum, N::sqrt(L[j]));  // ascending order
    const double r_obs = static_cast<double>(r_sum) / k;
    const double R = r_obs / r_exp;           // Eq. 4
    const double mu = membership_eq5(R, am);  // Eq. 5
    const double alpha = alpha_eq6(mu, am);   // Eq. 6
    // L1 = log2(d1^2 + eps) through the same instruction as every pair's log2, so that a
    // coincident point (d2 == eps) gets exactly e = 0.
    const T L1 = N::lg2(N::opaque(N::add(d1, N::kEps)));
    T neg_s, c;
    if (d1 == T(0)) {
        // Coincident query: weight 1 on every coincident point, 0 elsewhere.
        neg_s = -N::kCoinc;
        c = N::kCoinc * L1;
    } else {
        const T sh = static_cast<T>(0.5 * alpha);
        neg_s = -sh;
        c = sh * L1;
    }

    // ---- phase 2: Eq. 1 over all points ----
    T hw = 0, cw = 0, hz = 0, cz = 0, sw = 0, szs = 0;
    int in_chunk = 0;
    if (TILED) {
        for (int64_t base = 0; base < n; base += kBlock) {
            const int64_t i = base + threadIdx.x;
            T px = CUDART_INF, py = CUDART_INF, pz = 0;
            if (i < n)
                load_xyz<T, AOAS>(d, i, px, py, pz);
            __syncthreads();
            sx[threadIdx.x] = px;
            sy[threadIdx.x] = py;
            sz[threadIdx.x] = pz;
            __syncthreads();
            const int cnt = n - base < kBlock ? static_cast<int>(n - base) : kBlock;
            for (int t = 0; t < cnt; ++t) {
                weight_step<T>(x0, y0, sx[t], sy[t], sz[t], neg_s, c, sw, szs);
                if (++in_chunk == kChunk) {
                    kahan_add(hw, cw, sw);
                    kahan_add(hz, cz, szs);
                    sw = szs = 0;
                    in_chunk = 0;
                }
            }
        }
    } else {
        for (int64_t i = 0; i < n; ++i) {
            T px, py, pz;
            load_xyz<T, AOAS>(d, i, px, py, pz);
            weight_step<T>(x0, y0, px, py, pz, neg_s, c, sw, szs);
            if (++in_chunk == kChunk) {
                kahan_add(hw, cw, sw);
                kahan_add(hz, cz, szs);
                sw = szs = 0;
                in_chunk = 0;
            }
        }
    }
    kahan_add(hw, cw, sw);
    kahan_add(hz, cz, szs);
    if (!active)
        return;
    const double W = static_cast<double>(hw) - static_cast<double>(cw);
    const double WZ = static_cast<double>(hz) - static_cast<double>(cz);
    out[q] = static_cast<T>(WZ / W);
    if (out_alpha)
        out_alpha[q] = static_cast<float>(alpha);
}

// Caller-order copies in the layout under test, from the dataset's FP64 arrays.
template <typename T>
__global__ void paper_layout_kernel(const double2 *__restrict__ xy, const double *__restrict__ z,
                                    int64_t n, T *x, T *y, T *zz, Point4<T> *p)
{
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const T a = static_cast<T>(xy[i].x), b = static_cast<T>(xy[i].y);
        const T c = static_cast<T>(z[i]);
        if (p) {
            p[i] = Point4<T>{a, b, c, T(0)};
        } else {
            x[i] = a;
            y[i] = b;
            zz[i] = c;
        }
    }
}

template <typename T, bool TILED, bool AOAS>
void launch_kp(int kp, unsigned blocks, const Layout<T> &d, const T *qx, const T *qy, int64_t m,
               int k, double r_exp, const AlphaMap &am, T *out, float *out_alpha,
               cudaStream_t st)
{
    if (kp == 8)
        paper_aidw_kernel<T, TILED, AOAS, 8>
            <<<blocks, kBlock, 0, st>>>(d, qx, qy, m, k, r_exp, am, out, out_alpha);
    else if (kp == 16)
        paper_aidw_kernel<T, TILED, AOAS, 16>
            <<<blocks, kBlock, 0, st>>>(d, qx, qy, m, k, r_exp, am, out, out_alpha);
    else
        paper_aidw_kernel<T, TILED, AOAS, 32>
            <<<blocks, kBlock, 0, st>>>(d, qx, qy, m, k, r_exp, am, out, out_alpha);
}

template <typename T>
int run_paper(aidw_ctx *ctx, const DatasetDev &ds, double r_exp, const aidw_params &p,
              const void *qx, const void *qy, int64_t m, void *out, float *out_alpha,
              int version, int layout, cudaStream_t st)
{
    const bool aoas = layout == AIDW_LAYOUT_AOAS;
    const size_t a = ((sizeof(T) * ds.n + 255) / 256) * 256;  // one SoA array
    const size_t bytes = aoas ? sizeof(Point4<T>) * ds.n : 3 * a;
    void *blk = nullptr;
    int rc = ctx_alloc(ctx, bytes, st, &blk);
    if (rc)
        return rc;
    Layout<T> d{};
    d.n = ds.n;
    T *x = nullptr, *y = nullptr, *z = nullptr;
    Point4<T> *pp = nullptr;
    if (aoas) {
        pp = static_cast<Point4<T> *>(blk);
    } else {
        x = static_cast<T *>(blk);
        y = reinterpret_cast<T *>(static_cast<char *>(blk) + a);
        z = reinterpret_cast<T *>(static_cast<char *>(blk) + 2 * a);
    }
    d.x = x;
    d.y = y;
    d.z = z;
    d.p = pp;
    const unsigned cb = static_cast<unsigned>(std::min<int64_t>((ds.n + 255) / 256, 4096));
    paper_layout_kernel<T><<<cb, 256, 0, st>>>(ds.xy64, ds.z64, ds.n, x, y, z, pp);
    const AlphaMap am = alpha_map(p);
    const int kp = p.k <= 8 ? 8 : (p.k <= 16 ? 16 : 32);
    const unsigned blocks = static_cast<unsigned>((m + kBlock - 1) / kBlock);
    const T *tqx = static_cast<const T *>(qx), *tqy = static_cast<const T *>(qy);
    T *tout = static_cast<T *>(out);
    if (version == AIDW_VERSION_TILED) {
        if (aoas)
            launch_kp<T, true, true>(kp, blocks, d, tqx, tqy, m, p.k, r_exp, am, tout,
                                     out_alpha, st);
        else
            launch_kp<T, true, false>(kp, blocks, d, tqx, tqy, m, p.k, r_exp, am, tout,
                                      out_alpha, st);
    } else {
        if (aoas)
            launch_kp<T, false, true>(kp, blocks, d, tqx, tqy, m, p.k, r_exp, am, tout,
                                      out_alpha, st);
        else
            launch_kp<T, false, false>(kp, blocks, d, tqx, tqy, m, p.k, r_exp, am, tout,
                                       out_alpha, st);
    }
    rc = cudaGetLastError() == cudaSuccess ? AIDW_OK : AIDW_ERR_CUDA;
    ctx_free(ctx, blk, bytes, st);
    return rc;
}

}  // namespace
}  // namespace aidw

using namespace aidw;

extern "C" int aidw_interpolate_paper(aidw_ctx *ctx, aidw_dataset ds, const void *qx,
                                      const void *qy, int64_t m, const aidw_params *p,
                                      void *out, float *out_alpha, int32_t version,
                                      int32_t layout, void *stream)
{
    if (!ctx || !p)
        return AIDW_ERR_INVALID_ARG;
    if ((version != AIDW_VERSION_NAIVE && version != AIDW_VERSION_TILED) ||
        (layout != AIDW_LAYOUT_SOA && layout != AIDW_LAYOUT_AOAS) ||
        p->precision == AIDW_F64X)  // the paper's designs come in FP32 and FP64 only
        return AIDW_ERR_INVALID_ARG;
    DatasetDev dev;
    double r_exp;
    if (!dataset_lookup(ctx, ds, &dev, &r_exp))
        return AIDW_ERR_NOT_FOUND;
    int rc = validate_params(p, dev.n);
    if (rc)
        return rc;
    if (m < 0 || m > (int64_t(1) << 31))
        return AIDW_ERR_INVALID_ARG;
    if (m == 0)
        return AIDW_OK;
    const int device = ctx_device(ctx);
    if (pointer_kind(qx, device) != 1 || pointer_kind(qy, device) != 1 ||
        pointer_kind(out, device) != 1 || (out_alpha && pointer_kind(out_alpha, device) != 1))
        return AIDW_ERR_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess)
        return AIDW_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return p->precision == AIDW_F64
               ? run_paper<double>(ctx, dev, r_exp, *p, qx, qy, m, out, out_alpha, version,
                                   layout, st)
               : run_paper<float>(ctx, dev, r_exp, *p, qx, qy, m, out, out_alpha, version,
                                  layout, st);
}
