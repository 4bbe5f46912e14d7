// C ABI of the library: context, dataset store, one-shot interpolation, diagnostics.
// The batched and serving entry points live in runtime.cu.
#include <math_constants.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "aidw_internal.cuh"
#include "aidw_runtime.h"

namespace aidw {

namespace {

inline size_t align256(size_t b)
{
    return (b + 255) & ~static_cast<size_t>(255);
}

// Converts caller arrays (float or double) into unsorted FP32 staging arrays and the padded
// FP64 layout, and counts non-finite inputs. FP64 padding points are +inf with value 0.
template <typename T>
__global__ void convert_dataset_kernel(const T *__restrict__ x, const T *__restrict__ y,
                                       const T *__restrict__ z, int64_t n, int64_t n_pad,
                                       float2 *xy32, float *z32, double2 *xy64, double *z64,
                                       unsigned long long *bad)
{
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    unsigned long long nb = 0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n_pad;
         i += stride) {
        double a, b, c;
        if (i < n) {
            a = static_cast<double>(x[i]);
            b = static_cast<double>(y[i]);
            c = static_cast<double>(z[i]);
            nb += (isfinite(a) && isfinite(b) && isfinite(c)) ? 0 : 1;
            const float fa = static_cast<float>(a), fb = static_cast<float>(b);
            const float fc = static_cast<float>(c);
            // FP32 copies must stay finite too (values beyond float range are rejected).
            if (!(isfinite(fa) && isfinite(fb) && isfinite(fc)))
                ++nb;
            xy32[i] = make_float2(fa, fb);
            z32[i] = fc;
        } else {
            a = b = CUDART_INF;
            c = 0.0;
        }
        xy64[i] = make_double2(a, b);
        z64[i] = c;
    }
    if (nb)
        atomicAdd(bad, nb);
}

// Writes the Z-ordered FP32 layout: stored position i holds caller point perm[i] (padding
// positions, perm[i] >= n, hold +inf points with value 0).
__global__ void gather_dataset_kernel(const float2 *__restrict__ xy32,
                                      const float *__restrict__ z32,
                                      const uint32_t *__restrict__ perm, int64_t n,
                                      int64_t n_pad, float4 *nxy2, float2 *zz, int32_t *orig)
{
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n_pad;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const uint32_t p = perm[i];
        if (p < n) {
            const float2 q = xy32[p];
            const float v = z32[p];
            nxy2[i] = make_float4(-q.x, -q.x, -q.y, -q.y);
            zz[i] = make_float2(v, v);
            orig[i] = static_cast<int32_t>(p);
        } else {
            nxy2[i] = make_float4(-CUDART_INF_F, -CUDART_INF_F, -CUDART_INF_F, -CUDART_INF_F);
            zz[i] = make_float2(0.0f, 0.0f);
            orig[i] = -1;
        }
    }
}

}  // namespace

}  // namespace aidw

using namespace aidw;

struct DatasetRec {
    DatasetDev dev;
    void *block = nullptr;
    size_t bytes = 0;
    double area = 0.0;
    double r_exp = 0.0;
};

struct aidw_ctx {
    int device = 0;
    int sm_count = 0;
    size_t budget = 0;
    size_t in_use = 0;
    int64_t fail_after = -1;
    int *d_err = nullptr;
    unsigned long long *d_bad = nullptr;
    cudaMemPool_t pool = nullptr;
    std::mutex mu;
    std::unordered_map<int64_t, DatasetRec> datasets;
    int64_t next_ds = 1;
    bool profiling = false;
    cudaEvent_t ev[5] = {};
    aidw_kernel_times last{};
    bool last_valid = false;
    int slots_cache[3][4][2] = {};  // [precision][kp bucket][with_idx] knn slots
    int wslots_cache[3][3][2] = {};  // [precision][queries per thread 2/4/8][tile 256/512]
    aidw_tune_config tune = aidw::tune_default();
    ServingRuntime *serving = nullptr;
    int64_t serving_queue_limit = 4096;  // requests waiting for admission at most
};

namespace aidw {

// ---- memory accounting --------------------------------------------------------------------

int ctx_alloc(aidw_ctx *ctx, size_t bytes, cudaStream_t st, void **p)
{
    *p = nullptr;
    if (bytes == 0)
        return AIDW_OK;
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        if (ctx->fail_after >= 0) {
            if (ctx->fail_after == 0) {
                ctx->fail_after = -1;
                return AIDW_ERR_OOM;
            }
            --ctx->fail_after;
        }
        if (ctx->budget && ctx->in_use + bytes > ctx->budget)
            return AIDW_ERR_OOM;
        ctx->in_use += bytes;
    }
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, ctx->pool, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        std::lock_guard<std::mutex> g(ctx->mu);
        ctx->in_use -= bytes;
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? AIDW_ERR_OOM : AIDW_ERR_CUDA;
    }
    return AIDW_OK;
}

void ctx_free(aidw_ctx *ctx, void *p, size_t bytes, cudaStream_t st)
{
    if (!p)
        return;
    cudaFreeAsync(p, st);
    std::lock_guard<std::mutex> g(ctx->mu);
    ctx->in_use -= bytes;
}

size_t ctx_budget_left(aidw_ctx *ctx)
{
    std::lock_guard<std::mutex> g(ctx->mu);
    if (!ctx->budget)
        return SIZE_MAX;
    return ctx->budget > ctx->in_use ? ctx->budget - ctx->in_use : 0;
}

int *ctx_err_word(aidw_ctx *ctx)
{
    return ctx->d_err;
}

int ctx_device(aidw_ctx *ctx)
{
    return ctx->device;
}

int ctx_sm_count(aidw_ctx *ctx)
{
    return ctx->sm_count;
}

// Copies a dataset's record while holding the context lock, so that a concurrent
// aidw_destroy_dataset (which erases the record under the same lock) cannot free it while it is
// read; no pointer into the table leaves the lock.
static bool ctx_dataset_copy(aidw_ctx *ctx, aidw_dataset id, DatasetRec *out)
{
    std::lock_guard<std::mutex> g(ctx->mu);
    auto it = ctx->datasets.find(id);
    if (it == ctx->datasets.end())
        return false;
    *out = it->second;
    return true;
}

bool dataset_lookup(aidw_ctx *ctx, aidw_dataset id, DatasetDev *dev, double *r_exp)
{
    DatasetRec r;
    if (!ctx_dataset_copy(ctx, id, &r))
        return false;
    *dev = r.dev;
    *r_exp = r.r_exp;
    return true;
}

// ---- pointers ----------------------------------------------------------------------------

// 1: device memory of `device`; 0: host memory; -1: device memory of another device.
int pointer_kind(const void *p, int device)
{
    if (!p)
        return 0;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)
        return a.device == device ? 1 : -1;
    return 0;
}

// ---- planning ------------------------------------------------------------------------------

static PassPlan plan_pass(int64_t m, int64_t n_pad, int qpb, int slots_total, int64_t fixed)
{
    PassPlan pp{};
    pp.q_per_block = qpb;
    pp.qblocks = static_cast<int>((m + qpb - 1) / qpb);
    const int64_t G = n_pad / kPadPoints;
    double best = 1e300;
    for (int S = 1; S <= kMaxSplits && S <= G; ++S) {
        const int64_t per = (G + S - 1) / S;
        const int64_t Se = (G + per - 1) / per;
        if (Se != S)
            continue;
        const int64_t items = static_cast<int64_t>(pp.qblocks) * Se;
        const int64_t waves = (items + slots_total - 1) / slots_total;
        const double cost = static_cast<double>(waves) * (per * kPadPoints + fixed);
        if (cost < best * (1.0 - 1e-9)) {
            best = cost;
            pp.splits = static_cast<int>(Se);
            pp.split_len = per * kPadPoints;
        }
    }
    return pp;
}

// AIDW_F64 and AIDW_F64X share the FP64 arrays, phase 1, selection and finalisation.
static bool f64_arrays(int precision)
{
    return precision == AIDW_F64 || precision == AIDW_F64X;
}

static int kp_bucket(int kp)
{
    return kp <= 8 ? 0 : (kp <= 12 ? 1 : (kp <= 16 ? 2 : 3));
}

Plan make_plan(aidw_ctx *ctx, int precision, int64_t n_pad, int64_t m, int k, bool with_idx,
               int force_knn_splits, int force_w_splits, const aidw_tune_config *cfg)
{
    const aidw_tune_config &tc = cfg ? *cfg : ctx->tune;
    const bool f64 = f64_arrays(precision);
    const bool x = precision == AIDW_F64X;
    Plan pl{};
    pl.m = m;
    pl.with_idx = with_idx;
    pl.kp = f32_list_length(k, tc.knn_list);
    pl.kq = f64 ? (k <= 16 ? 2 : 1) : cull_queries_per_thread(pl.kp, tc.knn_queries_per_thread);
    pl.qw = tc.queries_per_thread;
    pl.tw = tc.tile_points;
    int &ks = ctx->slots_cache[precision][kp_bucket(f64 ? k : pl.kp)][with_idx ? 1 : 0];
    if (!ks)
        ks = f64 ? f64_knn_slots_per_sm(k, with_idx) : f32_knn_slots_per_sm(pl.kp, with_idx);
    int &ws = ctx->wslots_cache[precision][pl.qw == 2 ? 0 : (pl.qw == 4 ? 1 : 2)]
                               [pl.tw == 256 ? 0 : 1];
    if (!ws)
        ws = x ? f64x_w_slots_per_sm()
               : (f64 ? f64_w_slots_per_sm() : f32_w_slots_per_sm(pl.qw, pl.tw));
    const int qk = f64 ? f64_knn_queries_per_block(k) : f32_knn_queries_per_block(pl.kp);
    const int qw = x ? f64x_w_queries_per_block()
                     : (f64 ? f64_w_queries_per_block() : f32_w_queries_per_block(pl.qw));
    // A split restarts its neighbour lists: about k (1 + ln(n_split / k)) insertions per query,
    // each a rescan of a chunk by a partly idle warp. Measured on GB300 at n = m = 2^20,
    // k = 10, every extra split costs about as much as scanning 100,000 more points.
    pl.knn_slots = ks * ctx->sm_count;
    // The FP64 scan is bound by its FP64 pipe (the exact rescans behind the FP32 prefilter),
    // which co-resident CTAs share: it is planned as one CTA per SM (measured at n = 1M,
    // 4,096 queries: 8 splits 24 ms, 37 splits 39 ms).
    pl.knn = plan_pass(m, n_pad, qk, (f64 ? 1 : ks) * ctx->sm_count, 10000 * k);
    pl.w = plan_pass(m, n_pad, qw, ws * ctx->sm_count, 1024);
    const int64_t G = n_pad / kPadPoints;
    auto force = [&](PassPlan &pp, int S) {
        if (S <= 0)
            return;
        S = static_cast<int>(S > G ? G : S);
        S = S > kMaxSplits ? kMaxSplits : S;
        const int64_t per = (G + S - 1) / S;
        pp.splits = static_cast<int>((G + per - 1) / per);
        pp.split_len = per * kPadPoints;
    };
    force(pl.knn, force_knn_splits);
    force(pl.w, force_w_splits);
    return pl;
}

aidw_tune_config ctx_tune(aidw_ctx *ctx)
{
    std::lock_guard<std::mutex> g(ctx->mu);
    return ctx->tune;
}

void ctx_set_tune(aidw_ctx *ctx, const aidw_tune_config &c)
{
    std::lock_guard<std::mutex> g(ctx->mu);
    ctx->tune = c;
}

size_t scratch_bytes(int precision, const Plan &pl, int k)
{
    const size_t es = f64_arrays(precision) ? sizeof(double) : sizeof(float);
    const size_t m = static_cast<size_t>(pl.m);
    size_t b = align256(pl.knn.splits * static_cast<size_t>(k) * m * es);
    if (pl.with_idx)
        b += align256(pl.knn.splits * static_cast<size_t>(k) * m * sizeof(int32_t));
    b += align256(m * (f64_arrays(precision) ? sizeof(QParamF64) : sizeof(QParamF32)));
    b += align256(pl.w.splits * 4 * m * es);
    return b;
}

void scratch_carve(void *base, int precision, const Plan &pl, int k, Scratch *s)
{
    const size_t es = f64_arrays(precision) ? sizeof(double) : sizeof(float);
    const size_t m = static_cast<size_t>(pl.m);
    char *p = static_cast<char *>(base);
    s->part_d2 = p;
    p += align256(pl.knn.splits * static_cast<size_t>(k) * m * es);
    s->part_idx = nullptr;
    if (pl.with_idx) {
        s->part_idx = reinterpret_cast<int32_t *>(p);
        p += align256(pl.knn.splits * static_cast<size_t>(k) * m * sizeof(int32_t));
    }
    s->qparam = p;
    p += align256(m * (f64_arrays(precision) ? sizeof(QParamF64) : sizeof(QParamF32)));
    s->part_sum = p;
}

int validate_params(const aidw_params *p, int64_t n)
{
    if (!p)
        return AIDW_ERR_INVALID_ARG;
    if (p->precision != AIDW_F32C && !f64_arrays(p->precision))
        return AIDW_ERR_INVALID_ARG;
    if (p->k < 1 || p->k > AIDW_MAX_K || p->k > n)
        return AIDW_ERR_INVALID_ARG;
    for (int i = 0; i < 5; ++i)
        if (!std::isfinite(p->alpha[i]) || !(p->alpha[i] > 0.0))
            return AIDW_ERR_INVALID_ARG;
    if (!std::isfinite(p->r_min) || !std::isfinite(p->r_max) || !(p->r_max > p->r_min) ||
        !(p->r_max > 0.0))
        return AIDW_ERR_INVALID_ARG;
    if (p->flags != 0 || p->reserved != 0)
        return AIDW_ERR_INVALID_ARG;
    return AIDW_OK;
}

AlphaMap alpha_map(const aidw_params &p)
{
    AlphaMap am;
    for (int i = 0; i < 5; ++i)
        am.level[i] = p.alpha[i];
    am.r_min = p.r_min;
    am.r_max = p.r_max;
    return am;
}

// Phase boundaries of one interpolation: the profiling events (when profiling is on) and NVTX
// ranges naming the phases, so that a profiler can attribute the kernels launched in each (for
// example `ncu --nvtx --nvtx-include "aidw phase 2/"`). The ranges span the host-side enqueue;
// without a tool attached the NVTX calls do nothing.
class PhaseMarks {
  public:
    PhaseMarks(aidw_ctx *ctx, cudaStream_t st, bool profile)
        : ctx_(ctx), st_(st), profile_(profile)
    {
    }
    PhaseMarks(const PhaseMarks &) = delete;
    PhaseMarks &operator=(const PhaseMarks &) = delete;
    ~PhaseMarks()
    {
        if (open_)
            nvtxRangePop();
    }
    // Boundary i: the start of phase i (0 phase 1, with the query ordering; 1 selection;
    // 2 phase 2; 3 finalisation), 4 the end.
    void at(int i)
    {
        static const char *const kNames[4] = {"aidw phase 1", "aidw select", "aidw phase 2",
                                              "aidw finalize"};
        if (profile_)
            cudaEventRecord(ctx_->ev[i], st_);
        if (open_)
            nvtxRangePop();
        open_ = i < 4;
        if (open_)
            nvtxRangePushA(kNames[i]);
    }

  private:
    aidw_ctx *ctx_;
    cudaStream_t st_;
    bool profile_;
    bool open_ = false;
};

// Enqueues the four kernels of one interpolation on `st` with device arrays only.
int enqueue_interpolation(aidw_ctx *ctx, const DatasetDev &ds, double r_exp, const Plan &pl,
                          const aidw_params &p, const void *qx, const void *qy,
                          const Scratch &sc, void *out, float *out_alpha, int32_t *out_knn,
                          cudaStream_t st, bool profile)
{
    const AlphaMap am = alpha_map(p);
    cudaError_t e;
    const bool f64 = f64_arrays(p.precision);
    const bool x = p.precision == AIDW_F64X;
    PhaseMarks marks(ctx, st, profile);
    marks.at(0);
    e = f64 ? launch_f64_knn(ds, pl, static_cast<const double *>(qx),
                             static_cast<const double *>(qy), p.k, sc, ctx->d_err, st)
            : launch_f32_knn(ds, pl, static_cast<const float *>(qx),
                             static_cast<const float *>(qy), p.k, sc, ctx->d_err, st);
    if (e != cudaSuccess)
        return AIDW_ERR_CUDA;
    marks.at(1);
    e = f64 ? launch_f64_select(pl, p.k, r_exp, am, sc, out_alpha, out_knn, st, nullptr, x)
            : launch_f32_select(pl, p.k, r_exp, am, sc, out_alpha, out_knn, st);
    if (e != cudaSuccess)
        return AIDW_ERR_CUDA;
    marks.at(2);
    e = x     ? launch_f64x_weights(ds, pl, static_cast<const double *>(qx),
                                    static_cast<const double *>(qy), sc, ctx->d_err, st)
        : f64 ? launch_f64_weights(ds, pl, static_cast<const double *>(qx),
                                   static_cast<const double *>(qy), sc, ctx->d_err, st)
              : launch_f32_weights(ds, pl, static_cast<const float *>(qx),
                                 static_cast<const float *>(qy), sc, ctx->d_err, st);
    if (e != cudaSuccess)
        return AIDW_ERR_CUDA;
    marks.at(3);
    e = f64 ? launch_f64_finalize(pl, sc, static_cast<double *>(out), st)
            : launch_f32_finalize(pl, sc, static_cast<float *>(out), st);
    if (e != cudaSuccess)
        return AIDW_ERR_CUDA;
    marks.at(4);
    if (profile) {
        ctx->last = aidw_kernel_times{};
        ctx->last.splits = pl.knn.splits;
        ctx->last.query_blocks = pl.knn.qblocks;
        ctx->last.launches = 4;
        ctx->last.weight_splits = pl.w.splits;
        ctx->last_valid = true;
    }
    return AIDW_OK;
}

// Queries below this count keep the plain split scan for phase 1 (ordering them would cost
// more than it saves).
constexpr int64_t kCullMinQueries = 2048;

// The pruned phase 1 serves every precision (FP64 lists with indices keep the oracle's tie
// order by ordering pairs (distance, caller index)) when there are enough queries: with m
// queries spread over the data, a block of q queries covers about q/m of the area, so each of
// the m/q blocks visits about n q / (512 m) tiles, and with fewer blocks than the GPU holds (P)
// the pruned scan takes about n q^2 P / m per-pair steps of one CTA against n m / P steps of
// each CTA for the split scan: the pruned scan wins when m > q sqrt(P). Measured at n = 1M
// with random queries: in FP32 the split scan is faster at m = 8,192 and the pruned scan at
// 32,768; in FP64 (both scans with the FP32 prefilter) the split scan at 8,192 (34 against
// 45 ms) and the pruned scan at 16,384 (38 against 66 ms), so FP64 takes twice the bound.
bool use_culled_knn(int precision, const DatasetDev &ds, int64_t m, bool with_idx,
                    const Plan &pl)
{
    (void)with_idx;
    const double need = kThreads * pl.kq * std::sqrt(static_cast<double>(pl.knn_slots)) *
                        (f64_arrays(precision) ? 2.0 : 1.0);
    return ds.n_pad / kTileF32Knn <= kMaxCullTiles && m >= kCullMinQueries &&
           static_cast<double>(m) >= need;
}

// Whether a call takes the per-query phase 1 (one warp per query). In FP32 its cost grows with
// the query count alone (about 25 ns of the GPU per query against 1M points, 13 ns against
// 65,536), while the block scans share their tiles among a block's queries and gain as the
// queries get denser. Measured phase 1 (ms, against 1M uniform points / 65,536 clustered
// points; block scans = the split scan below 12,600 queries, the pruned scan above):
//   queries        1,024   4,096   8,192   32,768   131,072
//   block scans    2.63    3.41    4.46    1.93     1.09     /  0.61  0.64  0.73  0.54  0.46
//   warp per query 0.24    0.25    0.34    0.99     3.24     /  0.13  0.14  0.19  0.49  1.67
// so FP32 calls of up to kWarpKnnMaxQueries take it. In FP64 and FP64X (exact FP64 distances
// per lane, read through the Z-order map) the block scans cost far more, measured phase 1 (ms):
//   queries        512    2,048  8,192  16,384  32,768  65,536  131,072  262,144
//   1M uniform:  split scan 10.9 17.5 32.4 45.2 60.8 114 198; pruned scan 141 92.0 58.0 39.3
//                24.3 15.4 13.1; warp per query 0.19 0.26 0.66 1.20 2.26 4.49 8.73
//   65,536 clustered: split 3.74 5.45 10.4 13.9 20.1 39.4 77.4 145; pruned 24.9 17.5 9.24
//                6.78 5.30 5.22 6.20 8.07; warp 0.11 0.14 0.35 0.62 1.20 2.32 4.58 9.06
// so FP64 calls of up to kWarpKnnMaxQueriesF64 take it.
constexpr int64_t kWarpKnnMaxQueries = 32768;
constexpr int64_t kWarpKnnMaxQueriesF64 = 131072;

bool use_warp_knn(int precision, const DatasetDev &ds, int64_t m, int sm_count)
{
    (void)ds;
    (void)sm_count;
    return m <= (precision == AIDW_F32C ? kWarpKnnMaxQueries : kWarpKnnMaxQueriesF64);
}

void plan_culled_knn(Plan *pl, int64_t n_pad)
{
    pl->knn.splits = 1;
    pl->knn.split_len = n_pad;
    pl->knn.q_per_block = kThreads * pl->kq;
    pl->knn.qblocks = static_cast<int>((pl->m + pl->knn.q_per_block - 1) / pl->knn.q_per_block);
}

size_t culled_extra_bytes(int64_t m, int precision)
{
    const size_t mm = static_cast<size_t>(m);
    const size_t es = f64_arrays(precision) ? sizeof(double) : sizeof(float);
    return 2 * align256(mm * sizeof(uint32_t)) + 2 * align256(mm * es) +
           align256(radix_scratch_bytes(m));
}

// Interpolation with Z-ordered queries and the pruned phase-1 scan: Morton keys of the queries
// over the dataset's box, stable radix sort, gather, phase 1 (pruned), selection and
// finalisation writing back to the caller's order; phase 2 runs on the ordered queries.
int enqueue_culled(aidw_ctx *ctx, const DatasetDev &ds, double r_exp, const Plan &pl,
                   const aidw_params &p, const void *qx, const void *qy, const Scratch &sc,
                   void *extra, void *out, float *out_alpha, int32_t *out_knn, cudaStream_t st,
                   bool profile)
{
    const AlphaMap am = alpha_map(p);
    const int64_t m = pl.m;
    const bool f64 = f64_arrays(p.precision);
    const bool xp = p.precision == AIDW_F64X;
    const size_t es = f64 ? sizeof(double) : sizeof(float);
    const size_t b4 = align256(static_cast<size_t>(m) * sizeof(uint32_t));
    const size_t bq = align256(static_cast<size_t>(m) * es);
    char *e = static_cast<char *>(extra);
    uint32_t *keys = reinterpret_cast<uint32_t *>(e);
    uint32_t *perm = reinterpret_cast<uint32_t *>(e + b4);
    void *sqx = e + 2 * b4;
    void *sqy = e + 2 * b4 + bq;
    void *sort_tmp = e + 2 * b4 + 2 * bq;
    PhaseMarks marks(ctx, st, profile);
    marks.at(0);
    bool ok;
    if (f64) {
        const double *x = static_cast<const double *>(qx), *y = static_cast<const double *>(qy);
        double *sx = static_cast<double *>(sqx), *sy = static_cast<double *>(sqy);
        ok = morton_keys_f64(x, y, m, ds.box, keys, perm, st) == cudaSuccess;
        ok = ok && radix_sort_pairs(keys, perm, m, sort_tmp, st) == cudaSuccess;
        ok = ok && gather_queries_f64(x, y, perm, m, sx, sy, st) == cudaSuccess;
        ok = ok && launch_f64_knn_cull(ds, pl, sx, sy, p.k, sc, ctx->d_err, st) == cudaSuccess;
        marks.at(1);
        ok = ok && launch_f64_select(pl, p.k, r_exp, am, sc, out_alpha, out_knn, st, perm,
                                     xp) == cudaSuccess;
        marks.at(2);
        ok = ok && (xp ? launch_f64x_weights(ds, pl, sx, sy, sc, ctx->d_err, st)
                       : launch_f64_weights(ds, pl, sx, sy, sc, ctx->d_err, st)) == cudaSuccess;
        marks.at(3);
        ok = ok && launch_f64_finalize(pl, sc, static_cast<double *>(out), st, perm) ==
                       cudaSuccess;
    } else {
        const float *x = static_cast<const float *>(qx), *y = static_cast<const float *>(qy);
        float *sx = static_cast<float *>(sqx), *sy = static_cast<float *>(sqy);
        ok = morton_keys(x, y, nullptr, m, m, ds.box, keys, perm, st) == cudaSuccess;
        ok = ok && radix_sort_pairs(keys, perm, m, sort_tmp, st) == cudaSuccess;
        ok = ok && gather_queries(x, y, perm, m, sx, sy, st) == cudaSuccess;
        ok = ok && launch_f32_knn_cull(ds, pl, sx, sy, p.k, sc, ctx->d_err, st) == cudaSuccess;
        marks.at(1);
        ok = ok && launch_f32_select(pl, p.k, r_exp, am, sc, out_alpha, out_knn, st, perm) ==
                       cudaSuccess;
        marks.at(2);
        ok = ok && launch_f32_weights(ds, pl, sx, sy, sc, ctx->d_err, st) == cudaSuccess;
        marks.at(3);
        ok = ok && launch_f32_finalize(pl, sc, static_cast<float *>(out), st, perm) ==
                       cudaSuccess;
    }
    if (!ok)
        return AIDW_ERR_CUDA;
    marks.at(4);
    if (profile) {
        ctx->last = aidw_kernel_times{};
        ctx->last.splits = pl.knn.splits;
        ctx->last.query_blocks = pl.knn.qblocks;
        ctx->last.launches = 4 + 14;  // + Morton keys, 12 radix-sort passes, gather
        ctx->last.weight_splits = pl.w.splits;
        ctx->last_valid = true;
    }
    return AIDW_OK;
}

// FP32 interpolation with the per-query (one warp per query) phase 1, in the caller's order:
// phase 1, selection, phase 2, finalisation (four launches, no query ordering).
int enqueue_warp(aidw_ctx *ctx, const DatasetDev &ds, double r_exp, const Plan &pl,
                 const aidw_params &p, const void *qx, const void *qy, const Scratch &sc,
                 void *out, float *out_alpha, int32_t *out_knn, cudaStream_t st, bool profile)
{
    PhaseMarks marks(ctx, st, profile);
    const AlphaMap am = alpha_map(p);
    bool ok;
    if (p.precision == AIDW_F32C) {
        const float *fx = static_cast<const float *>(qx), *fy = static_cast<const float *>(qy);
        marks.at(0);
        ok = launch_f32_knn_warp(ds, pl.m, fx, fy, p.k, sc, ctx->sm_count, st) == cudaSuccess;
        marks.at(1);
        ok = ok && launch_f32_select(pl, p.k, r_exp, am, sc, out_alpha, out_knn, st) ==
                       cudaSuccess;
        marks.at(2);
        ok = ok && launch_f32_weights(ds, pl, fx, fy, sc, ctx->d_err, st) == cudaSuccess;
        marks.at(3);
        ok = ok && launch_f32_finalize(pl, sc, static_cast<float *>(out), st) == cudaSuccess;
    } else {
        const bool x = p.precision == AIDW_F64X;
        const double *dx = static_cast<const double *>(qx), *dy = static_cast<const double *>(qy);
        marks.at(0);
        ok = launch_f64_knn_warp(ds, pl, dx, dy, p.k, sc, ctx->sm_count, st) == cudaSuccess;
        marks.at(1);
        ok = ok && launch_f64_select(pl, p.k, r_exp, am, sc, out_alpha, out_knn, st, nullptr,
                                     x) == cudaSuccess;
        marks.at(2);
        ok = ok && (x ? launch_f64x_weights(ds, pl, dx, dy, sc, ctx->d_err, st)
                      : launch_f64_weights(ds, pl, dx, dy, sc, ctx->d_err, st)) == cudaSuccess;
        marks.at(3);
        ok = ok && launch_f64_finalize(pl, sc, static_cast<double *>(out), st) == cudaSuccess;
    }
    if (!ok)
        return AIDW_ERR_CUDA;
    marks.at(4);
    if (profile) {
        ctx->last = aidw_kernel_times{};
        ctx->last.splits = 1;
        ctx->last.query_blocks = 0;
        ctx->last.launches = 4;
        ctx->last.weight_splits = pl.w.splits;
        ctx->last_valid = true;
    }
    return AIDW_OK;
}

// Reads and clears the on-device error word (synchronous).
int consume_device_error(aidw_ctx *ctx, cudaStream_t st)
{
    int h = 0;
    if (cudaMemcpyAsync(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return AIDW_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess)
        return AIDW_ERR_CUDA;
    if (h) {
        cudaMemsetAsync(ctx->d_err, 0, sizeof(int), st);
        cudaStreamSynchronize(st);
        return AIDW_ERR_TIMEOUT;
    }
    return AIDW_OK;
}

// Full interpolation, host or device arrays (see aidw.h). `force_*` override the split
// counts (used by the tests to exercise split merges); 0 means "plan".
int interpolate_impl(aidw_ctx *ctx, aidw_dataset dsid, const void *qx, const void *qy,
                     int64_t m, const aidw_params *p, void *out, float *out_alpha,
                     int32_t *out_knn, cudaStream_t st, int force_knn_splits,
                     int force_w_splits, const aidw_tune_config *cfg)
{
    DatasetDev ds;
    double r_exp;
    if (!dataset_lookup(ctx, dsid, &ds, &r_exp))
        return AIDW_ERR_NOT_FOUND;
    int rc = validate_params(p, ds.n);
    if (rc)
        return rc;
    if (m < 0 || m > (int64_t(1) << 31))
        return AIDW_ERR_INVALID_ARG;
    if (m == 0)
        return AIDW_OK;
    if (!qx || !qy || !out)
        return AIDW_ERR_INVALID_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess)
        return AIDW_ERR_CUDA;
    const bool f64 = f64_arrays(p->precision);
    const size_t es = f64 ? sizeof(double) : sizeof(float);
    const int kq = pointer_kind(qx, ctx->device), kqy = pointer_kind(qy, ctx->device);
    const int ko = pointer_kind(out, ctx->device);
    const int ka = pointer_kind(out_alpha, ctx->device);
    const int kn = pointer_kind(out_knn, ctx->device);
    if (kq < 0 || kqy < 0 || ko < 0 || ka < 0 || kn < 0)
        return AIDW_ERR_INVALID_ARG;
    const bool host_q = kq == 0 || kqy == 0;
    const bool host_any = host_q || ko == 0 || (out_alpha && ka == 0) || (out_knn && kn == 0);
    if (host_q) {
        for (int64_t i = 0; i < m; ++i) {
            const double a = f64 ? static_cast<const double *>(qx)[i]
                                 : static_cast<const float *>(qx)[i];
            const double b = f64 ? static_cast<const double *>(qy)[i]
                                 : static_cast<const float *>(qy)[i];
            if (!std::isfinite(a) || !std::isfinite(b))
                return AIDW_ERR_INVALID_ARG;
        }
    }

    // Tests force the phase-1 route: force_knn_splits -1 takes the per-query scan and -2 the
    // pruned scan (where the dataset's tile count allows it) whatever the sizes; > 0 the split
    // scan with that many splits.
    const bool force_cull =
        force_knn_splits == -2 && ds.n_pad / kTileF32Knn <= kMaxCullTiles;
    const bool warp = force_knn_splits == -1 ||
                      (force_knn_splits == 0 && use_warp_knn(p->precision, ds, m, ctx->sm_count));
    Plan pl = make_plan(ctx, p->precision, ds.n_pad, m, p->k, out_knn != nullptr,
                        force_knn_splits > 0 ? force_knn_splits : 0, force_w_splits, cfg);
    const bool cull = force_cull || (!warp && force_knn_splits == 0 &&
                                     use_culled_knn(p->precision, ds, m, out_knn != nullptr, pl));
    if (cull)
        plan_culled_knn(&pl, ds.n_pad);
    if (warp) {
        // One list per query, [k][m], for the selection kernel.
        pl.knn.splits = 1;
        pl.knn.split_len = ds.n_pad;
    }
    const size_t sb = scratch_bytes(p->precision, pl, p->k) +
                      (cull ? culled_extra_bytes(m, p->precision) : 0);
    // Staging for host arrays.
    const size_t b_q = (kq == 0 ? align256(m * es) : 0) + (kqy == 0 ? align256(m * es) : 0);
    const size_t b_o = ko == 0 ? align256(m * es) : 0;
    const size_t b_a = (out_alpha && ka == 0) ? align256(m * sizeof(float)) : 0;
    const size_t b_n = (out_knn && kn == 0) ? align256(m * p->k * sizeof(int32_t)) : 0;
    const size_t total = sb + b_q + b_o + b_a + b_n;
    void *blk = nullptr;
    rc = ctx_alloc(ctx, total, st, &blk);
    if (rc)
        return rc;
    Scratch sc;
    scratch_carve(blk, p->precision, pl, p->k, &sc);
    void *extra = static_cast<char *>(blk) + scratch_bytes(p->precision, pl, p->k);
    char *stage = static_cast<char *>(blk) + sb;
    const void *dqx = qx, *dqy = qy;
    void *dout = out;
    float *dalpha = out_alpha;
    int32_t *dknn = out_knn;
    bool ok = true;
    if (kq == 0) {
        ok &= cudaMemcpyAsync(stage, qx, m * es, cudaMemcpyHostToDevice, st) == cudaSuccess;
        dqx = stage;
        stage += align256(m * es);
    }
    if (kqy == 0) {
        ok &= cudaMemcpyAsync(stage, qy, m * es, cudaMemcpyHostToDevice, st) == cudaSuccess;
        dqy = stage;
        stage += align256(m * es);
    }
    if (ko == 0) {
        dout = stage;
        stage += b_o;
    }
    if (out_alpha && ka == 0) {
        dalpha = reinterpret_cast<float *>(stage);
        stage += b_a;
    }
    if (out_knn && kn == 0) {
        dknn = reinterpret_cast<int32_t *>(stage);
        stage += b_n;
    }
    if (!ok) {
        ctx_free(ctx, blk, total, st);
        return AIDW_ERR_CUDA;
    }
    rc = warp   ? enqueue_warp(ctx, ds, r_exp, pl, *p, dqx, dqy, sc, dout, dalpha, dknn, st,
                               ctx->profiling)
         : cull ? enqueue_culled(ctx, ds, r_exp, pl, *p, dqx, dqy, sc, extra, dout, dalpha, dknn,
                                 st, ctx->profiling)
                : enqueue_interpolation(ctx, ds, r_exp, pl, *p, dqx, dqy, sc, dout, dalpha, dknn,
                                        st, ctx->profiling);
    if (rc == AIDW_OK && host_any) {
        ok = true;
        if (ko == 0)
            ok &= cudaMemcpyAsync(out, dout, m * es, cudaMemcpyDeviceToHost, st) == cudaSuccess;
        if (out_alpha && ka == 0)
            ok &= cudaMemcpyAsync(out_alpha, dalpha, m * sizeof(float), cudaMemcpyDeviceToHost,
                                  st) == cudaSuccess;
        if (out_knn && kn == 0)
            ok &= cudaMemcpyAsync(out_knn, dknn, m * p->k * sizeof(int32_t),
                                  cudaMemcpyDeviceToHost, st) == cudaSuccess;
        if (!ok)
            rc = AIDW_ERR_CUDA;
    }
    ctx_free(ctx, blk, total, st);
    if (rc == AIDW_OK && host_any)
        rc = consume_device_error(ctx, st);
    return rc;
}

}  // namespace aidw

// =============================================================================================
// extern "C" entry points
// =============================================================================================

extern "C" {

void aidw_params_default(aidw_params *p)
{
    if (!p)
        return;
    std::memset(p, 0, sizeof(*p));
    p->k = 10;
    p->precision = AIDW_F32C;
    for (int i = 0; i < 5; ++i)
        p->alpha[i] = 1.0 + i;
    p->r_min = 0.0;
    p->r_max = 2.0;
}

const char *aidw_status_string(int s)
{
    switch (s) {
    case AIDW_OK: return "ok";
    case AIDW_PENDING: return "pending";
    case AIDW_ERR_INVALID_ARG: return "invalid argument";
    case AIDW_ERR_OOM: return "out of device memory or HBM budget";
    case AIDW_ERR_AGAIN: return "queue full, try again";
    case AIDW_ERR_TIMEOUT: return "timed out";
    case AIDW_ERR_CUDA: return "CUDA runtime error";
    case AIDW_ERR_NOT_FOUND: return "unknown handle";
    case AIDW_ERR_UNSUPPORTED: return "unsupported device or option";
    default: return "unknown status";
    }
}

int aidw_init(aidw_ctx **out, int device, size_t hbm_budget_bytes)
{
    if (!out)
        return AIDW_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return AIDW_ERR_INVALID_ARG;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess)
        return AIDW_ERR_CUDA;
    if (prop.major != 10 || prop.minor != 3)
        return AIDW_ERR_UNSUPPORTED;
    if (cudaSetDevice(device) != cudaSuccess)
        return AIDW_ERR_CUDA;
    aidw_ctx *ctx = new aidw_ctx();
    ctx->device = device;
    ctx->sm_count = prop.multiProcessorCount;
    ctx->budget = hbm_budget_bytes;
    cudaMemPoolProps pp;
    std::memset(&pp, 0, sizeof(pp));
    pp.allocType = cudaMemAllocationTypePinned;
    pp.handleTypes = cudaMemHandleTypeNone;
    pp.location.type = cudaMemLocationTypeDevice;
    pp.location.id = device;
    bool ok = cudaMemPoolCreate(&ctx->pool, &pp) == cudaSuccess;
    if (ok) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    ok = ok && cudaMalloc(&ctx->d_err, sizeof(int)) == cudaSuccess;
    ok = ok && cudaMalloc(&ctx->d_bad, sizeof(unsigned long long)) == cudaSuccess;
    ok = ok && cudaMemset(ctx->d_err, 0, sizeof(int)) == cudaSuccess;
    for (int i = 0; ok && i < 5; ++i)
        ok = cudaEventCreate(&ctx->ev[i]) == cudaSuccess;
    // Places aidw_interpolate_noalloc's fixed scratch array on the device now, at set-up, so
    // that its calls never load a module (and its 16 MiB) in the middle of a request.
    ok = ok && noalloc_prepare(device) == AIDW_OK;
    if (!ok) {
        cudaGetLastError();
        aidw_shutdown(ctx);
        return AIDW_ERR_CUDA;
    }
    *out = ctx;
    return AIDW_OK;
}

int aidw_shutdown(aidw_ctx *ctx)
{
    if (!ctx)
        return AIDW_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    serving_stop(ctx->serving);
    ctx->serving = nullptr;
    cudaDeviceSynchronize();
    for (auto &kv : ctx->datasets)
        cudaFree(kv.second.block);
    ctx->datasets.clear();
    if (ctx->d_err)
        cudaFree(ctx->d_err);
    if (ctx->d_bad)
        cudaFree(ctx->d_bad);
    for (int i = 0; i < 5; ++i)
        if (ctx->ev[i])
            cudaEventDestroy(ctx->ev[i]);
    if (ctx->pool)
        cudaMemPoolDestroy(ctx->pool);
    cudaGetLastError();
    delete ctx;
    return AIDW_OK;
}

int aidw_create_dataset(aidw_ctx *ctx, const void *x, const void *y, const void *z, int64_t n,
                        double area, int32_t dtype, aidw_dataset *out)
{
    if (!ctx || !x || !y || !z || !out)
        return AIDW_ERR_INVALID_ARG;
    *out = 0;
    if (n < 1 || n > (int64_t(1) << 31) - 2 * kPadPoints)
        return AIDW_ERR_INVALID_ARG;
    if (!std::isfinite(area) || !(area > 0.0))
        return AIDW_ERR_INVALID_ARG;
    if (dtype != AIDW_DTYPE_F32 && dtype != AIDW_DTYPE_F64)
        return AIDW_ERR_INVALID_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess)
        return AIDW_ERR_CUDA;
    const int kx = pointer_kind(x, ctx->device), ky = pointer_kind(y, ctx->device);
    const int kz = pointer_kind(z, ctx->device);
    if (kx < 0 || ky < 0 || kz < 0)
        return AIDW_ERR_INVALID_ARG;
    const size_t es = dtype == AIDW_DTYPE_F64 ? sizeof(double) : sizeof(float);
    const int64_t n_pad = (n + kPadPoints - 1) / kPadPoints * kPadPoints;
    const size_t np = static_cast<size_t>(n_pad);
    const int64_t ntiles = n_pad / kTileF32Knn;
    const int64_t nsub = n_pad / kSubTile;
    const int64_t nsuper = (ntiles + kSuperTiles - 1) / kSuperTiles;
    const size_t bytes = align256(np * sizeof(float4)) + align256(np * sizeof(float2)) +
                         align256(np * sizeof(int32_t)) + align256(np * sizeof(double2)) +
                         align256(np * sizeof(double)) + align256(ntiles * sizeof(float4)) +
                         align256(nsub * sizeof(float4)) + align256(nsuper * sizeof(float4)) +
                         align256(sizeof(float4));
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        if (ctx->fail_after >= 0) {
            if (ctx->fail_after == 0) {
                ctx->fail_after = -1;
                return AIDW_ERR_OOM;
            }
            --ctx->fail_after;
        }
        if (ctx->budget && ctx->in_use + bytes > ctx->budget)
            return AIDW_ERR_OOM;
        ctx->in_use += bytes;
    }
    auto unreserve = [&]() {
        std::lock_guard<std::mutex> g(ctx->mu);
        ctx->in_use -= bytes;
    };
    void *blk = nullptr;
    if (cudaMalloc(&blk, bytes) != cudaSuccess) {
        cudaGetLastError();
        unreserve();
        return AIDW_ERR_OOM;
    }
    // Temporary block: host-array staging (if any), unsorted FP32 copies, sort keys and values,
    // radix-sort scratch, bounding-box scratch.
    const size_t one = align256(static_cast<size_t>(n) * es);
    const bool stage_host = kx == 0 || ky == 0 || kz == 0;
    const size_t tmp_bytes = (stage_host ? 3 * one : 0) + align256(np * sizeof(float2)) +
                             align256(np * sizeof(float)) + 2 * align256(np * sizeof(uint32_t)) +
                             align256(radix_scratch_bytes(n_pad)) + 256;
    void *tmp = nullptr;
    if (cudaMalloc(&tmp, tmp_bytes) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(blk);
        unreserve();
        return AIDW_ERR_OOM;
    }
    char *t = static_cast<char *>(tmp);
    const void *sx = x, *sy = y, *sz = z;
    if (stage_host) {
        if (kx == 0) {
            cudaMemcpy(t, x, n * es, cudaMemcpyHostToDevice);
            sx = t;
        }
        if (ky == 0) {
            cudaMemcpy(t + one, y, n * es, cudaMemcpyHostToDevice);
            sy = t + one;
        }
        if (kz == 0) {
            cudaMemcpy(t + 2 * one, z, n * es, cudaMemcpyHostToDevice);
            sz = t + 2 * one;
        }
        t += 3 * one;
    }
    float2 *xy32 = reinterpret_cast<float2 *>(t);
    t += align256(np * sizeof(float2));
    float *z32 = reinterpret_cast<float *>(t);
    t += align256(np * sizeof(float));
    uint32_t *keys = reinterpret_cast<uint32_t *>(t);
    t += align256(np * sizeof(uint32_t));
    uint32_t *perm = reinterpret_cast<uint32_t *>(t);
    t += align256(np * sizeof(uint32_t));
    void *sort_tmp = t;
    t += align256(radix_scratch_bytes(n_pad));
    uint32_t *box_scratch = reinterpret_cast<uint32_t *>(t);

    char *b = static_cast<char *>(blk);
    float4 *nxy2 = reinterpret_cast<float4 *>(b);
    b += align256(np * sizeof(float4));
    float2 *zz = reinterpret_cast<float2 *>(b);
    b += align256(np * sizeof(float2));
    int32_t *orig = reinterpret_cast<int32_t *>(b);
    b += align256(np * sizeof(int32_t));
    double2 *xy64 = reinterpret_cast<double2 *>(b);
    b += align256(np * sizeof(double2));
    double *z64 = reinterpret_cast<double *>(b);
    b += align256(np * sizeof(double));
    float4 *tbox = reinterpret_cast<float4 *>(b);
    b += align256(ntiles * sizeof(float4));
    float4 *sbox = reinterpret_cast<float4 *>(b);
    b += align256(nsub * sizeof(float4));
    float4 *upbox = reinterpret_cast<float4 *>(b);
    b += align256(nsuper * sizeof(float4));
    float4 *box = reinterpret_cast<float4 *>(b);

    int rc = AIDW_OK;
    cudaMemset(ctx->d_bad, 0, sizeof(unsigned long long));
    const int threads = 256;
    const int blocks = static_cast<int>(std::min<int64_t>((n_pad + threads - 1) / threads,
                                                          ctx->sm_count * 8));
    if (dtype == AIDW_DTYPE_F64)
        convert_dataset_kernel<double><<<blocks, threads>>>(
            static_cast<const double *>(sx), static_cast<const double *>(sy),
            static_cast<const double *>(sz), n, n_pad, xy32, z32, xy64, z64, ctx->d_bad);
    else
        convert_dataset_kernel<float><<<blocks, threads>>>(
            static_cast<const float *>(sx), static_cast<const float *>(sy),
            static_cast<const float *>(sz), n, n_pad, xy32, z32, xy64, z64, ctx->d_bad);
    unsigned long long bad = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpy(&bad, ctx->d_bad, sizeof(bad), cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = AIDW_ERR_CUDA;
    else if (bad)
        rc = AIDW_ERR_INVALID_ARG;
    // Z-order the FP32 copy and box every tile.
    if (rc == AIDW_OK) {
        bool ok = bbox_of(xy32, n, box_scratch, box, 0) == cudaSuccess;
        ok = ok && morton_keys(nullptr, nullptr, xy32, n, n_pad, box, keys, perm, 0) ==
                       cudaSuccess;
        ok = ok && radix_sort_pairs(keys, perm, n_pad, sort_tmp, 0) == cudaSuccess;
        if (ok) {
            gather_dataset_kernel<<<blocks, threads>>>(xy32, z32, perm, n, n_pad, nxy2, zz, orig);
            ok = cudaGetLastError() == cudaSuccess;
        }
        ok = ok && tile_boxes(nxy2, ntiles, tbox, 0) == cudaSuccess;
        ok = ok && sub_tile_boxes(nxy2, nsub, sbox, 0) == cudaSuccess;
        ok = ok && super_tile_boxes(tbox, ntiles, nsuper, upbox, 0) == cudaSuccess;
        ok = ok && cudaDeviceSynchronize() == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            rc = AIDW_ERR_CUDA;
        }
    }
    cudaFree(tmp);
    if (rc) {
        cudaFree(blk);
        unreserve();
        return rc;
    }
    DatasetRec rec;
    rec.dev.nxy2 = nxy2;
    rec.dev.zz = zz;
    rec.dev.orig = orig;
    rec.dev.tile_box = tbox;
    rec.dev.sub_box = sbox;
    rec.dev.super_box = upbox;
    rec.dev.box = box;
    rec.dev.xy64 = xy64;
    rec.dev.z64 = z64;
    rec.dev.n = n;
    rec.dev.n_pad = n_pad;
    rec.block = blk;
    rec.bytes = bytes;
    rec.area = area;
    rec.r_exp = 1.0 / (2.0 * std::sqrt(static_cast<double>(n) / area));  // Eq. 2
    std::lock_guard<std::mutex> g(ctx->mu);
    const int64_t id = ctx->next_ds++;
    ctx->datasets.emplace(id, rec);
    *out = id;
    return AIDW_OK;
}

int aidw_destroy_dataset(aidw_ctx *ctx, aidw_dataset ds)
{
    if (!ctx)
        return AIDW_ERR_INVALID_ARG;
    DatasetRec rec;
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        auto it = ctx->datasets.find(ds);
        if (it == ctx->datasets.end())
            return AIDW_ERR_NOT_FOUND;
        rec = it->second;
        ctx->datasets.erase(it);
    }
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    cudaFree(rec.block);
    std::lock_guard<std::mutex> g(ctx->mu);
    ctx->in_use -= rec.bytes;
    return AIDW_OK;
}

int aidw_dataset_info(aidw_ctx *ctx, aidw_dataset ds, int64_t *n, size_t *device_bytes)
{
    if (!ctx)
        return AIDW_ERR_INVALID_ARG;
    DatasetRec r;
    if (!ctx_dataset_copy(ctx, ds, &r))
        return AIDW_ERR_NOT_FOUND;
    if (n)
        *n = r.dev.n;
    if (device_bytes)
        *device_bytes = r.bytes;
    return AIDW_OK;
}

int aidw_interpolate(aidw_ctx *ctx, aidw_dataset ds, const void *qx, const void *qy, int64_t m,
                     const aidw_params *p, void *out, float *out_alpha, int32_t *out_knn,
                     void *stream)
{
    if (!ctx)
        return AIDW_ERR_INVALID_ARG;
    return interpolate_impl(ctx, ds, qx, qy, m, p, out, out_alpha, out_knn,
                            static_cast<cudaStream_t>(stream), 0, 0);
}

// Test hook with forced split counts (not part of the public header's contract).
int aidw_debug_interpolate_splits(aidw_ctx *ctx, aidw_dataset ds, const void *qx,
                                  const void *qy, int64_t m, const aidw_params *p, void *out,
                                  float *out_alpha, int32_t *out_knn, void *stream,
                                  int32_t knn_splits, int32_t w_splits)
{
    if (!ctx)
        return AIDW_ERR_INVALID_ARG;
    return interpolate_impl(ctx, ds, qx, qy, m, p, out, out_alpha, out_knn,
                            static_cast<cudaStream_t>(stream), knn_splits, w_splits);
}

int aidw_idw(aidw_ctx *ctx, aidw_dataset ds, const void *qx, const void *qy, int64_t m,
             double alpha, int32_t precision, void *out, void *stream)
{
    if (!ctx)
        return AIDW_ERR_INVALID_ARG;
    // Standard IDW is AIDW with five equal levels: Eq. 6 then returns alpha whatever R is.
    // One neighbour is still found, to normalise the weights and to detect coincidence.
    aidw_params p;
    aidw_params_default(&p);
    p.k = 1;
    p.precision = precision;
    for (int i = 0; i < 5; ++i)
        p.alpha[i] = alpha;
    return interpolate_impl(ctx, ds, qx, qy, m, &p, out, nullptr, nullptr,
                            static_cast<cudaStream_t>(stream), 0, 0);
}

int aidw_check_device_errors(aidw_ctx *ctx)
{
    if (!ctx)
        return AIDW_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    if (cudaDeviceSynchronize() != cudaSuccess)
        return AIDW_ERR_CUDA;
    return consume_device_error(ctx, 0);
}

int aidw_set_profiling(aidw_ctx *ctx, int on)
{
    if (!ctx)
        return AIDW_ERR_INVALID_ARG;
    ctx->profiling = on != 0;
    ctx->last_valid = false;
    return AIDW_OK;
}

int aidw_last_kernel_times(aidw_ctx *ctx, aidw_kernel_times *out)
{
    if (!ctx || !out)
        return AIDW_ERR_INVALID_ARG;
    if (!ctx->last_valid)
        return AIDW_ERR_NOT_FOUND;
    if (cudaEventSynchronize(ctx->ev[4]) != cudaSuccess)
        return AIDW_ERR_CUDA;
    float t[4];
    for (int i = 0; i < 4; ++i)
        cudaEventElapsedTime(&t[i], ctx->ev[i], ctx->ev[i + 1]);
    ctx->last.knn_ms = t[0];
    ctx->last.select_ms = t[1];
    ctx->last.weights_ms = t[2];
    ctx->last.finalize_ms = t[3];
    *out = ctx->last;
    return AIDW_OK;
}

int aidw_measure_pipe_rates(aidw_ctx *ctx, aidw_pipe_rates *out)
{
    if (!ctx || !out)
        return AIDW_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    return run_pipe_probe(ctx->sm_count, out) == cudaSuccess ? AIDW_OK : AIDW_ERR_CUDA;
}

int aidw_debug_fail_alloc_after(aidw_ctx *ctx, int64_t after)
{
    if (!ctx)
        return AIDW_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(ctx->mu);
    ctx->fail_after = after < 0 ? -1 : after;
    return AIDW_OK;
}

}  // extern "C"

namespace aidw {
ServingRuntime *&ctx_serving(aidw_ctx *ctx)
{
    return ctx->serving;
}
std::mutex &ctx_mutex(aidw_ctx *ctx)
{
    return ctx->mu;
}
int64_t &ctx_serving_queue_limit(aidw_ctx *ctx)
{
    return ctx->serving_queue_limit;
}
}  // namespace aidw
