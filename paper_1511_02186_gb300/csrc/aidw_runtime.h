// Host-side runtime shared between the one-shot API (aidw_api.cu) and the batching / serving
// layer (runtime.cu).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <mutex>
#include <vector>

#include "aidw_internal.cuh"

struct aidw_ctx;

namespace aidw {

// NVTX range over a scope: names the host-side enqueue interval, to which a profiler attributes
// the kernels launched inside it; a no-op without a tool attached.
class NvtxScope {
  public:
    explicit NvtxScope(const char *name)
    {
        nvtxRangePushA(name);
    }
    ~NvtxScope()
    {
        nvtxRangePop();
    }
    NvtxScope(const NvtxScope &) = delete;
    NvtxScope &operator=(const NvtxScope &) = delete;
};

struct ServingRuntime;

// Device memory from the context's pool, charged to its HBM budget (stream-ordered).
int ctx_alloc(aidw_ctx *ctx, size_t bytes, cudaStream_t st, void **p);
void ctx_free(aidw_ctx *ctx, void *p, size_t bytes, cudaStream_t st);
size_t ctx_budget_left(aidw_ctx *ctx);
int *ctx_err_word(aidw_ctx *ctx);
int ctx_device(aidw_ctx *ctx);
int ctx_sm_count(aidw_ctx *ctx);
ServingRuntime *&ctx_serving(aidw_ctx *ctx);
std::mutex &ctx_mutex(aidw_ctx *ctx);
// Serving queue length (read and written under ctx_mutex).
int64_t &ctx_serving_queue_limit(aidw_ctx *ctx);

bool dataset_lookup(aidw_ctx *ctx, int64_t id, DatasetDev *dev, double *r_exp);
int pointer_kind(const void *p, int device);
int validate_params(const aidw_params *p, int64_t n);
AlphaMap alpha_map(const aidw_params &p);
// Shape from `cfg`, or from the context's shape when cfg is null.
Plan make_plan(aidw_ctx *ctx, int precision, int64_t n_pad, int64_t m, int k, bool with_idx,
               int force_knn_splits, int force_w_splits, const aidw_tune_config *cfg = nullptr);
aidw_tune_config ctx_tune(aidw_ctx *ctx);
void ctx_set_tune(aidw_ctx *ctx, const aidw_tune_config &c);
int interpolate_impl(aidw_ctx *ctx, int64_t dsid, const void *qx, const void *qy, int64_t m,
                     const aidw_params *p, void *out, float *out_alpha, int32_t *out_knn,
                     cudaStream_t st, int force_knn_splits, int force_w_splits,
                     const aidw_tune_config *cfg = nullptr);
int consume_device_error(aidw_ctx *ctx, cudaStream_t st);
int enqueue_interpolation(aidw_ctx *ctx, const DatasetDev &ds, double r_exp, const Plan &pl,
                          const aidw_params &p, const void *qx, const void *qy,
                          const Scratch &sc, void *out, float *out_alpha, int32_t *out_knn,
                          cudaStream_t st, bool profile);
// The pruned phase 1 (Z-ordered queries, nearest tiles first): whether a call takes it, the
// plan change it needs (one query block per CTA, no data splits), the scratch it needs beyond
// scratch_bytes (query ordering), and the enqueue.
bool use_culled_knn(int precision, const DatasetDev &ds, int64_t m, bool with_idx,
                    const Plan &pl);
void plan_culled_knn(Plan *pl, int64_t n_pad);
size_t culled_extra_bytes(int64_t m, int precision);
int enqueue_culled(aidw_ctx *ctx, const DatasetDev &ds, double r_exp, const Plan &pl,
                   const aidw_params &p, const void *qx, const void *qy, const Scratch &sc,
                   void *extra, void *out, float *out_alpha, int32_t *out_knn, cudaStream_t st,
                   bool profile);
// The per-query phase 1 (one warp per query, caller order): whether a call of `precision`
// takes it, and the enqueue (phase 1, selection, phase 2, finalisation; the plan keeps one list
// split). Query and output arrays are float for AIDW_F32C, double otherwise.
bool use_warp_knn(int precision, const DatasetDev &ds, int64_t m, int sm_count);
int enqueue_warp(aidw_ctx *ctx, const DatasetDev &ds, double r_exp, const Plan &pl,
                 const aidw_params &p, const void *qx, const void *qy, const Scratch &sc,
                 void *out, float *out_alpha, int32_t *out_knn, cudaStream_t st, bool profile);
// Resolves the device address of aidw_interpolate_noalloc's scratch array on `device` (made
// current by the caller); called once per context at aidw_init.
int noalloc_prepare(int device);

// Stops the serving thread (waits for admitted work) and frees its state; null is a no-op.
void serving_stop(ServingRuntime *rt);

// A built batch (batched.cu): device tables, work list, counters and scratch in one block.
struct BatchState {
    void *block = nullptr;
    size_t bytes = 0;
    void *d_items = nullptr;  // item table
    void *d_units = nullptr;  // work list
    uint32_t *d_counters = nullptr;  // [0] work counter, then per-item counters
    size_t counter_bytes = 0;
    int n_units = 0;   // phase-1 and phase-2 units
    int n_units1 = 0;  // phase-1 units (the first n_units1 of the work list)
    bool lean = false;  // the 64-register kernel variant serves this batch
    bool order_in_tz = false;  // pruned units keep their tile order in the phase-2 z buffers
    int grid = 0;
    cudaGraphExec_t graph = nullptr;
    // Batch-wide query ordering (Z-order within each item).
    int32_t count = 0;
    int64_t total_q = 0, max_m = 0;
    size_t dyn_smem = 0;
    uint32_t *keys = nullptr, *vals = nullptr, *item_of = nullptr, *perm = nullptr;
    float *sqx = nullptr, *sqy = nullptr;
    void *sort_tmp = nullptr;
    aidw_tune_config cfg{};  // shape the batch was built with
};
// reserve_ctas_per_sm: persistent CTAs per SM to leave free (for a concurrent launch).
int batch_build(aidw_ctx *ctx, const aidw_batch_item *items, int32_t count, cudaStream_t st,
                BatchState *bs, const aidw_tune_config &cfg, int reserve_ctas_per_sm = 0);
int batch_enqueue(aidw_ctx *ctx, const BatchState &bs, cudaStream_t st);
void batch_release(aidw_ctx *ctx, BatchState *bs, cudaStream_t st);
// Device bytes one batch item of m queries against n_pad points with k neighbours needs.
size_t batch_item_bytes(int64_t n_pad, int64_t m, int k, const aidw_tune_config &cfg);

}  // namespace aidw

// A prepared batch: its items (kept to rebuild it under another shape) and the built state.
struct aidw_batch {
    aidw::BatchState st;
    std::vector<aidw_batch_item> items;
};

namespace aidw {
int batch_prepare(aidw_ctx *ctx, aidw_batch *b, const aidw_tune_config &cfg);
}  // namespace aidw
