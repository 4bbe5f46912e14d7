/*
 * aidw.h -- C ABI of the GB300 (sm_103a) Adaptive Inverse Distance Weighting library.
 *
 * The method is AIDW as defined by Mei, Xu & Xu, "Accelerating Adaptive IDW Interpolation
 * Algorithm on a Single GPU" (arXiv 1511.02186):
 *   phase 1 (Sec. 2.2, Steps 1-3; kNN per Sec. 3.1.2): for every query point find its k nearest
 *           data points, form r_obs (Eq. 3) against r_exp (Eq. 2), the statistic R (Eq. 4), the
 *           fuzzy membership mu_R (Eq. 5) and the adaptive power alpha (Eq. 6);
 *   phase 2 (Sec. 2.1, Eq. 1; Sec. 3.2.1): Z = sum_i z_i d_i^-alpha / sum_i d_i^-alpha over ALL
 *           n data points.
 *
 * Conventions for every entry point:
 *   - Return value: AIDW_OK (0) or a negative AIDW_ERR_* status; no entry point throws, aborts
 *     or prints. aidw_status_string() names a status.
 *   - Notation: n data points, m query points, k neighbours, A the study area.
 *   - Pointers to caller arrays may be host memory (pageable or pinned) or device memory of the
 *     context's device; the library tells them apart with cudaPointerGetAttributes. A call that
 *     touches any host array copies through library-owned device buffers and returns only once
 *     its results are in the caller's host arrays. A call whose arrays are all on the device is
 *     stream-ordered: it returns after enqueuing its kernels on the given stream.
 *   - Caller arrays remain caller-owned; the library never frees them and keeps no reference to
 *     them after the call returns (asynchronous calls: after the stream reaches the work).
 *   - Datasets are copied into library-owned device memory at creation and stay resident until
 *     destroyed.
 *   - A context is not thread-safe: serialise calls on one context, or use one per thread.
 */
#ifndef AIDW_H
#define AIDW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes --------------------------------------------------------------------- */
#define AIDW_OK 0
#define AIDW_PENDING 1             /* request admitted, results not ready yet */
#define AIDW_ERR_INVALID_ARG (-1)  /* a size, parameter or input value is outside the domain */
#define AIDW_ERR_OOM (-2)          /* device memory or the context's HBM budget is exhausted */
#define AIDW_ERR_AGAIN (-3)        /* serving queue full: resubmit later */
#define AIDW_ERR_TIMEOUT (-4)      /* a bounded wait ran out (host wait or an on-device wait) */
#define AIDW_ERR_CUDA (-5)         /* a CUDA runtime call failed */
#define AIDW_ERR_NOT_FOUND (-6)    /* unknown dataset or request handle */
#define AIDW_ERR_UNSUPPORTED (-7)  /* device is not sm_103 or an option is not built */

/* ---- precisions and dtypes ------------------------------------------------------------ */
/* AIDW_F32C: distances, kNN selection and weights in FP32; the two weighted sums in FP32 with
 * Kahan-compensated merges; alpha mapping (Eq. 2, 4, 5, 6) and the final ratio in FP64.
 * Queries and the output are float arrays.
 * AIDW_F64: every step at double precision or finer: distances, kNN selection, alpha, the
 * power scale, the weighted sum of z and the final ratio in FP64; log2, exp2 and the sum of the
 * weights in 62-bit fixed point on the integer pipe (within about an ulp of the FP64 result).
 * Queries and the output are double arrays.
 * AIDW_F64X (the library's addition; the paper has FP32 and FP64 only): FP64 arrays and the
 * FP64 path's phase 1, neighbour lists and alpha; in phase 2 each pair's squared distance is
 * formed in FP64 and the rest of its work (log2, the power of Eq. 1, both weighted sums) runs
 * in double-float arithmetic (pairs of floats, about 48 bits) on the FP32 pipes, which on
 * GB300 run at 64 times the FP64 rate. Results agree with the FP64 path to about 1e-13
 * relative to max(|Z|, sum w|z| / sum w); weights below 2^-126 of the nearest point's are
 * dropped. */
#define AIDW_F32C 0
#define AIDW_F64 1
#define AIDW_F64X 2

#define AIDW_DTYPE_F32 0
#define AIDW_DTYPE_F64 1

/* Largest k supported by the kernels (the register-resident neighbour list holds 32). */
#define AIDW_MAX_K 32

typedef struct aidw_ctx aidw_ctx;
typedef int64_t aidw_dataset;
typedef int64_t aidw_request;

/* Parameters of one interpolation (Sec. 2.2). */
typedef struct aidw_params {
    int32_t k;         /* neighbours for r_obs (Eq. 3); 1 <= k <= min(n, AIDW_MAX_K) */
    int32_t precision; /* AIDW_F32C, AIDW_F64 or AIDW_F64X */
    double alpha[5];   /* the five levels alpha_1..alpha_5 of Eq. 6; finite, > 0 */
    double r_min;      /* R_min of Eq. 5 (the paper suggests 0.0) */
    double r_max;      /* R_max of Eq. 5 (the paper suggests 2.0); r_max > r_min, r_max > 0 */
    uint32_t flags;    /* reserved, must be 0 */
    int32_t reserved;  /* reserved, must be 0 */
} aidw_params;

/* Fills k = 10, precision = AIDW_F32C, alpha = {1,2,3,4,5}, r_min = 0, r_max = 2. The level
 * values are not given by the paper (Eq. 6 leaves them to the user); these are a default. */
void aidw_params_default(aidw_params *p);

/* ---- context -------------------------------------------------------------------------- */
/* Creates a context on CUDA device `device`. hbm_budget_bytes caps the device memory the
 * context holds at once (datasets + per-call scratch); 0 means "whatever the device has".
 * It also places aidw_interpolate_noalloc's 16 MiB scratch array on the device (once per
 * device and process; not charged to the budget).
 * Returns AIDW_ERR_UNSUPPORTED if the device is not compute capability 10.3. */
int aidw_init(aidw_ctx **out, int device, size_t hbm_budget_bytes);

/* Waits for the context's work, frees every dataset and buffer it owns, and the context. */
int aidw_shutdown(aidw_ctx *ctx);

/* ---- datasets (Sec. 3.2.1: the data points' coordinates and values) ------------------- */
/* Copies n data points (x[i], y[i]) with values z[i] into library-owned device memory, as
 * FP32 and FP64 structure-of-arrays copies padded to a tile multiple. `area` is the study
 * area A of Eq. 2 (the paper does not say how A is obtained, so the caller supplies it).
 * dtype is AIDW_DTYPE_F32 or AIDW_DTYPE_F64 for all three arrays.
 * Errors: INVALID_ARG if n < 1, n > 2^31 - 2048, area is not finite and > 0, or any x, y, z
 * is NaN or infinite (checked on the device after the copy); OOM if the memory or the budget
 * runs out. This call is synchronous. */
int aidw_create_dataset(aidw_ctx *ctx, const void *x, const void *y, const void *z, int64_t n,
                        double area, int32_t dtype, aidw_dataset *out);

/* Frees a dataset. Work already enqueued on it must have finished (the call synchronizes the
 * device before freeing). */
int aidw_destroy_dataset(aidw_ctx *ctx, aidw_dataset ds);

/* Number of points and device bytes held by a dataset. */
int aidw_dataset_info(aidw_ctx *ctx, aidw_dataset ds, int64_t *n, size_t *device_bytes);

/* ---- interpolation -------------------------------------------------------------------- */
/* AIDW at m query points (qx[j], qy[j]) against dataset ds.
 *   qx, qy   m coordinates, float for AIDW_F32C, double for AIDW_F64 and AIDW_F64X
 *   out      m predictions Z (Eq. 1), float for AIDW_F32C, double for AIDW_F64 and AIDW_F64X
 *   out_alpha  nullable; m adaptive powers alpha (Eq. 6) as float
 *   out_knn  nullable; m*k int32 data-point indices, row j holding query j's neighbours in
 *            ascending distance, ties to the lower index (Sec. 3.1.2 with strict "<")
 *   stream   cudaStream_t to order the work on (NULL: the legacy default stream)
 * A query that coincides exactly with data points returns the mean z of those points (the
 * limit of Eq. 1). m == 0 is a no-op. Errors: INVALID_ARG for a bad k, level, bound, size or
 * (for host arrays) a non-finite query coordinate; on device arrays a non-finite query gives a
 * NaN prediction instead. NOT_FOUND for an unknown dataset; OOM when scratch does not fit. */
int aidw_interpolate(aidw_ctx *ctx, aidw_dataset ds, const void *qx, const void *qy, int64_t m,
                     const aidw_params *p, void *out, float *out_alpha, int32_t *out_knn,
                     void *stream);

/* Standard IDW (Sec. 2.1, Eq. 1) with one constant power `alpha` for all queries: phase 2 of
 * AIDW alone. Same array conventions as aidw_interpolate; `precision` selects the path. */
int aidw_idw(aidw_ctx *ctx, aidw_dataset ds, const void *qx, const void *qy, int64_t m,
             double alpha, int32_t precision, void *out, void *stream);

/* Allocation-free variant of aidw_interpolate for AIDW_F32C (the paper has no counterpart:
 * it concerns how this library obtains memory, not the method). For callers that must not
 * allocate device memory while serving a call, e.g. a process whose device footprint is fixed
 * at start-up and may not grow or fail mid-request, or code that cannot accept the implicit
 * device synchronisation of cudaFree: this call performs no cudaMalloc, cudaFree or other
 * allocation. Its scratch is one 16 MiB __device__ array inside the library, held on every
 * GPU that loads the library until the process exits. The context and the dataset are
 * created beforehand (they allocate once, at set-up); aidw_init also places the array on the
 * context's device and looks up its address, so that under CUDA's lazy module loading the
 * array is committed at set-up and not by a call. Kernel code is a separate matter: under lazy
 * module loading the CUDA driver loads a kernel at its first launch, so a caller that may not
 * allocate at all after set-up makes one call of each size class it will serve during set-up
 * (or runs with CUDA_MODULE_LOADING=EAGER).
 *   qx, qy, out  DEVICE arrays of m floats on the context's device (host arrays are rejected)
 *   p            as for aidw_interpolate; p->precision must be AIDW_F32C
 * Phase 1 takes aidw_interpolate's route when its scratch fits the array: up to 32,768 queries
 * one warp per query (about m * (4k + 24) bytes), above that the pruned scan over queries put
 * in Z-order (about m * (4k + 49) bytes, m up to about 189,000 at k = 10); otherwise it scans
 * every (query, data point) pair in data splits, which for many queries costs far more (at
 * 131,072 queries x 1M points about 61 ms against 3.4 ms for the pruned scan; phase 2 is the
 * same either way). Limit: the split scan
 * needs about m * (4k + 24) bytes within 16 MiB (m <= 262,144 for k = 10, about 110,000 for
 * k = 32); larger calls return AIDW_ERR_INVALID_ARG. All calls share the one array and it keeps
 * the last call's contents (every element a call reads, it has written first): calls whose
 * work overlaps on the GPU (for example on two streams) race and must be serialised by the
 * caller. Stream-ordered on `stream`; kernel timeouts are reported by
 * aidw_check_device_errors. */
int aidw_interpolate_noalloc(aidw_ctx *ctx, aidw_dataset ds, const float *qx, const float *qy,
                             int64_t m, const aidw_params *p, float *out, void *stream);

/* ---- the paper's kernel designs, for comparison ------------------------------------------ */
/* AIDW computed by the paper's own GPU designs (Sec. 3.1), rebuilt for sm_103a as a measured
 * comparison beside aidw_interpolate: one thread per query scanning all n points twice (phase 1
 * keeps the k smallest squared distances, Sec. 3.1.2; phase 2 forms the weights of Eq. 1), with
 * version AIDW_VERSION_NAIVE (every data point read from global memory) or AIDW_VERSION_TILED
 * (blocks of 256 data points staged in shared memory for the thread block, Sec. 3.1.1), and the
 * data in layout AIDW_LAYOUT_SOA (x[], y[], z[]) or AIDW_LAYOUT_AOAS ({x, y, z, 0} aligned
 * structures, Sec. 3.1.3), copied from the dataset in the caller's order for the call. Precision
 * as p->precision (AIDW_F32C or AIDW_F64: float or double arrays). Per pair the FP32
 * arithmetic is aidw_interpolate's; in FP64 the weights use the CUDA library's log2 / exp2
 * (aidw_interpolate's FP64 path has its own table-driven pair). The four variants of one
 * precision give identical results. Device arrays only; stream-ordered.
 * Errors: INVALID_ARG (bad version, layout, size or a host array), NOT_FOUND, OOM. */
#define AIDW_VERSION_NAIVE 0
#define AIDW_VERSION_TILED 1
#define AIDW_LAYOUT_SOA 0
#define AIDW_LAYOUT_AOAS 1
int aidw_interpolate_paper(aidw_ctx *ctx, aidw_dataset ds, const void *qx, const void *qy,
                           int64_t m, const aidw_params *p, void *out, float *out_alpha,
                           int32_t version, int32_t layout, void *stream);

/* ---- batched launch (many datasets in one persistent kernel) -------------------------- */
/* The paper interpolates one dataset per launch; batching independent problems (Sec. 3.1.1:
 * every query is independent, so every item is too) is this library's addition.
 * One entry of a batch: a dataset, its queries and outputs (all DEVICE arrays of the context's
 * device, float) and its parameters (precision must be AIDW_F32C; k and levels may differ per
 * item). The kNN index output is not available in batches. */
typedef struct aidw_batch_item {
    aidw_dataset ds;
    const float *qx, *qy;
    int64_t m;
    aidw_params params;
    float *out;
    float *out_alpha; /* nullable */
} aidw_batch_item;

/* Runs every item through one persistent work-queue kernel on `stream` (stream-ordered; the
 * item arrays must stay valid until the stream reaches the work). Items are cut into units
 * that depend only on the item, so each item's result is bit-identical whatever else is in the
 * batch, and equal to aidw_interpolate's within the FP32 tolerance. Errors: INVALID_ARG (bad
 * item, host array), NOT_FOUND (dataset), OOM (scratch). */
int aidw_interpolate_batch(aidw_ctx *ctx, const aidw_batch_item *items, int32_t count,
                           void *stream);

/* A prepared batch: the item table, work list and scratch are built once and the counter reset
 * plus the persistent kernel are captured as one CUDA graph; aidw_batch_launch replays it (the
 * caller may rewrite query contents in place between launches). aidw_batch_destroy waits for
 * the device and frees the batch. */
typedef struct aidw_batch aidw_batch;
int aidw_batch_create(aidw_ctx *ctx, const aidw_batch_item *items, int32_t count,
                      aidw_batch **out);
int aidw_batch_launch(aidw_ctx *ctx, aidw_batch *batch, void *stream);
int aidw_batch_destroy(aidw_ctx *ctx, aidw_batch *batch);

/* ---- kernel shapes and the autotuner ---------------------------------------------------- */
/* The shape of the FP32 kernels (the paper fixes none: Sec. 3.1.1 tiles data through shared
 * memory for a block of queries; sizes are the implementation's). Every field except
 * split_points is arithmetic-neutral: the per-query operations and their order do not depend
 * on it, so results are bit-identical across its values. split_points (and, in aidw_interpolate,
 * the phase-2 split count that occupancy picks for a query-block size) regroups the FP32 partial
 * sums of Eq. 1, which changes results only within the FP32 tolerance. */
typedef struct aidw_tune_config {
    int32_t queries_per_thread; /* phase 2: 2, 4 or 8 queries per thread (query block 128x) */
    int32_t tile_points;        /* phase 2: data points per shared-memory tile, 256 or 512 */
    int32_t knn_list;           /* phase 1: k-list register length at least this: 0 (the
                                 * smallest of 8, 12, 16, 32 that holds k), 16 or 32 */
    int32_t split_points;       /* batches: data points per phase-2 work unit, a multiple of
                                 * 2,048 in [2,048, 4,194,304] */
    int32_t ctas_per_sm;        /* batches: persistent CTAs per SM, 0 = as many as fit */
    int32_t knn_queries_per_thread; /* pruned phase 1: 2 or 4 queries per thread (query block
                                 * 128x), 0 = 4 for lists of up to 16, else 2; lists of 32
                                 * always take 2 */
    int32_t unit_order;         /* batches: which units a persistent CTA takes first.
                                 * 0 = every CTA takes the next phase-2 unit as soon as its
                                 * inputs are complete, phase-1 units while they are not;
                                 * 1 = the same, except that one CTA in four takes phase-1
                                 * units first (phase 1 runs ahead on part of the SMs) */
    int32_t reserved;           /* zero */
} aidw_tune_config;

/* Fills the built-in shape: 2 queries per thread in both phases, 512-point tiles, the smallest
 * list, 65,536 points per batch work unit, full occupancy, unit order 0. */
int aidw_tune_config_default(aidw_tune_config *out);
/* AIDW_OK if every field is one of the values above, else AIDW_ERR_INVALID_ARG. */
int aidw_tune_config_check(const aidw_tune_config *cfg);

/* The context's shape, used by aidw_interpolate (FP32), aidw_interpolate_noalloc,
 * aidw_interpolate_batch and new prepared batches; the serving runtime keeps the shape the
 * context had when it started. Set it between calls, not while work is queued. */
int aidw_set_tune_config(aidw_ctx *ctx, const aidw_tune_config *cfg);
int aidw_get_tune_config(aidw_ctx *ctx, aidw_tune_config *out);

/* Autotuner flags. AIDW_TUNE_CACHE: look the workload's key up in the process-wide tuning cache
 * first (a hit is used without timing: *best_ms = -1, one untimed run for
 * aidw_autotune_interpolate, none for batches) and store the winner under it.
 * AIDW_TUNE_APPLY (aidw_autotune_interpolate): make the winner the context's shape. */
#define AIDW_TUNE_CACHE 1u
#define AIDW_TUNE_APPLY 2u

/* Times an FP32 interpolation (arguments as aidw_interpolate, device arrays only) under
 * candidate shapes by coordinate search from the context's shape (queries per thread, tile
 * points, k-list length, phase-1 queries per thread; each candidate run `reps` times after one
 * warm-up, fastest run counts) and returns the fastest in *best with its time in *best_ms.
 * `out` receives the results of the last run. Synchronous. Errors: as aidw_interpolate;
 * INVALID_ARG for host arrays, F64 or reps < 1. */
int aidw_autotune_interpolate(aidw_ctx *ctx, aidw_dataset ds, const void *qx, const void *qy,
                              int64_t m, const aidw_params *p, void *out, int32_t reps,
                              uint32_t flags, aidw_tune_config *best, double *best_ms);

/* Rebuilds a prepared batch under `cfg` (work list, scratch and graph). */
int aidw_batch_set_config(aidw_ctx *ctx, aidw_batch *batch, const aidw_tune_config *cfg);
int aidw_batch_get_config(aidw_ctx *ctx, aidw_batch *batch, aidw_tune_config *out);

/* Times the prepared batch under candidate shapes by coordinate search from its current one
 * (queries per thread, tile points, k-list length, phase-1 queries per thread, points per work
 * unit, CTAs per SM, unit order; each
 * candidate launched `reps` times after one warm-up, fastest launch counts), leaves the batch
 * prepared with the fastest and returns it. Synchronous; after a search the batch's outputs
 * hold the winner's results. Errors: INVALID_ARG, NOT_FOUND (a dataset was destroyed), OOM,
 * CUDA, TIMEOUT (an on-device wait ran out). */
int aidw_batch_autotune(aidw_ctx *ctx, aidw_batch *batch, int32_t reps, uint32_t flags,
                        aidw_tune_config *best, double *best_ms);

/* Process-wide tuning cache: workload keys (printable ASCII without '"' or '\\', at most 255
 * characters; the autotuner's keys name the device and the workload's size class) mapped to
 * shapes. Files hold one JSON object per line:
 *   {"key": "...", "queries_per_thread": 4, "tile_points": 512, "knn_list": 0,
 *    "split_points": 65536, "ctas_per_sm": 0, "knn_queries_per_thread": 0, "unit_order": 0,
 *    "ms": 91.5}
 * _load merges a file into the cache (INVALID_ARG on a malformed line, NOT_FOUND if the file
 * cannot be opened; nothing is merged on error); _save writes the whole cache; _get returns
 * NOT_FOUND for an unknown key. Host only: usable without a GPU. */
int aidw_tune_cache_put(const char *key, const aidw_tune_config *cfg, double ms);
int aidw_tune_cache_get(const char *key, aidw_tune_config *out, double *ms);
int aidw_tune_cache_clear(void);
int aidw_tune_cache_size(void);
int aidw_tune_cache_save(const char *path);
int aidw_tune_cache_load(const char *path);

/* ---- serving: asynchronous requests with continuous batching --------------------------- */
/* Serving has no counterpart in the paper; each request is one interpolation as above.
 * Enqueues one interpolation request (same arguments as aidw_interpolate; arrays may be host
 * or device and must stay valid until aidw_poll/aidw_wait report completion). The context's
 * serving thread, started on first use, admits queued requests in arrival order while their
 * device footprint fits the serving budget and packs them into persistent batch launches
 * (continuous batching: a new launch starts on another stream while earlier ones still run).
 * A large FP32 request is cut into chunks of whole 256-query blocks served by successive
 * launches, one chunk per queued request per launch, and small requests may also take an
 * express launch slot out of arrival order. An FP32 request's result does not depend on what
 * it was batched with. FP64 requests and requests with a kNN output run alone. Returns
 * AIDW_ERR_AGAIN if the queue (4,096 requests unless configured otherwise) is full: the request
 * was not accepted, and the caller resubmits later or sheds it; a request larger than the
 * whole budget finishes with AIDW_ERR_OOM. */
int aidw_submit(aidw_ctx *ctx, aidw_dataset ds, const void *qx, const void *qy, int64_t m,
                const aidw_params *p, void *out, float *out_alpha, int32_t *out_knn,
                aidw_request *out_id);

/* *done = 1 when the request has finished (its status is returned), else 0 and AIDW_PENDING. */
int aidw_poll(aidw_ctx *ctx, aidw_request id, int32_t *done);

/* Waits up to timeout_us microseconds (< 0: no limit) for a request; returns its status, or
 * AIDW_ERR_TIMEOUT. */
int aidw_wait(aidw_ctx *ctx, aidw_request id, int64_t timeout_us);

/* Submit -> completion latency of a finished request in microseconds. */
int aidw_request_latency_us(aidw_ctx *ctx, aidw_request id, double *latency_us);

/* Forgets a finished request (its handle becomes unknown); AIDW_PENDING if not finished. */
int aidw_release_request(aidw_ctx *ctx, aidw_request id);

/* Shapes the serving runtime; call before the first aidw_submit (INVALID_ARG afterwards).
 * inflight_bytes: device memory that admitted requests may hold at once (0: half of the
 * context's budget, or 8 GiB without one); max_batch_requests: requests per launch (0: 256);
 * streams: launches that may run at once (0: 2, at most 8); max_queued: requests that may wait
 * for admission at once (0: the context's current limit, 4,096 unless changed by
 * aidw_serving_set_queue_limit), beyond which aidw_submit returns AIDW_ERR_AGAIN. */
int aidw_serving_configure(aidw_ctx *ctx, size_t inflight_bytes, int32_t max_batch_requests,
                           int32_t streams, int64_t max_queued);

/* Changes the serving queue's length (requests waiting for admission; >= 1) at any time,
 * before or after the first aidw_submit: later submits see the new limit, requests already
 * queued stay queued (a shorter limit only refuses new ones). INVALID_ARG for max_queued < 1. */
int aidw_serving_set_queue_limit(aidw_ctx *ctx, int64_t max_queued);

typedef struct aidw_serving_stats {
    int64_t submitted;       /* requests accepted by aidw_submit */
    int64_t completed;       /* finished with AIDW_OK */
    int64_t failed;          /* finished with an error status */
    int64_t rejected_again;  /* aidw_submit calls refused with AIDW_ERR_AGAIN */
    int64_t launches;        /* device launches (batches and lone requests) */
    int64_t batched_requests;        /* requests that went through batch launches */
    int32_t max_concurrent_launches; /* most launches in flight at once */
    int32_t reserved;
    int64_t queued;          /* requests waiting for admission now */
    size_t in_flight_bytes;  /* device bytes held by admitted requests now */
    size_t budget_bytes;     /* admission budget */
} aidw_serving_stats;

int aidw_serving_get_stats(aidw_ctx *ctx, aidw_serving_stats *out);

/* ---- diagnostics (the library's own; no counterpart in the paper) ------------------------ */
/* Names a status code ("unknown status" for any other value); the string is static. */
const char *aidw_status_string(int status);

/* Checks the context's on-device error word (set by a bounded wait inside a kernel that ran
 * out) after synchronizing the device; returns AIDW_OK or AIDW_ERR_TIMEOUT and clears it. */
int aidw_check_device_errors(aidw_ctx *ctx);

/* Per-kernel device times of the most recent aidw_interpolate on this context, measured with
 * CUDA events on the call's stream when profiling is on (aidw_set_profiling). */
typedef struct aidw_kernel_times {
    double knn_ms;      /* phase 1 distance scan and neighbour lists */
    double select_ms;   /* neighbour-list merge and Eq. 2-6 */
    double weights_ms;  /* phase 2 distance scan and weighted sums */
    double finalize_ms; /* split merge and the ratio of Eq. 1 */
    int32_t splits;     /* data-range splits of the phase-1 scan */
    int32_t query_blocks;
    int32_t launches;   /* kernels launched by the call */
    int32_t weight_splits; /* data-range splits of the phase-2 scan */
} aidw_kernel_times;

int aidw_set_profiling(aidw_ctx *ctx, int on);
int aidw_last_kernel_times(aidw_ctx *ctx, aidw_kernel_times *out);

/* Measured issue rates of the pipes that bound the kernels, for roofline denominators:
 * FP32 FFMA, MUFU ex2/lg2 and FP64 DFMA results per clock per SM, timed by microbenchmark
 * kernels on the context's device, plus the SM count and the SM clock the driver reports. */
typedef struct aidw_pipe_rates {
    double ffma_per_clk_sm;
    double ex2_per_clk_sm;
    double lg2_per_clk_sm;
    double fmnmx_per_clk_sm;
    double sm_clock_mhz; /* clock observed during the microbenchmarks */
    int32_t sm_count;
    int32_t reserved;
    double dfma_per_clk_sm; /* FP64 fused multiply-adds per clock per SM */
} aidw_pipe_rates;

int aidw_measure_pipe_rates(aidw_ctx *ctx, aidw_pipe_rates *out);

/* Test hook (host-side fault injection): the `after`-th device allocation from now fails with
 * AIDW_ERR_OOM; after < 0 disables it. */
int aidw_debug_fail_alloc_after(aidw_ctx *ctx, int64_t after);

/* Test hook for the bounded on-device waits: runs one CTA that waits, with the scans' own wait
 * code and a limit of `polls` polls (1 .. 2^20), on something that never completes (which = 0:
 * an mbarrier tile wait with no arrival; which = 1: another CTA's counter that is never
 * incremented). The wait runs out, the kernel raises the context's error word and returns, so
 * the next aidw_check_device_errors (or synchronous call) returns AIDW_ERR_TIMEOUT and the
 * context stays usable. Synchronous; returns AIDW_OK once the kernel has finished. */
int aidw_debug_expire_wait(aidw_ctx *ctx, int32_t which, uint32_t polls);

/* Test hooks for the phase-2 arithmetic, evaluated on the current device (synchronous; DEVICE
 * arrays of n doubles; INVALID_ARG for n < 0 or a null array, CUDA on a launch error).
 * aidw_debug_f64_log2_exp2: lx[i] = log2(x[i]) and ey[i] = 2^y[i] by the AIDW_F64 scan's
 *   table-driven FP64 functions (x positive or +inf).
 * aidw_debug_df_weight: the AIDW_F64X scan's double-float weight of one pair: v[i] =
 *   log2(d2[i] / d1sq[i]) and w[i] = 2^(-kappa[i] v[i]), each returned as hi + lo rounded to
 *   double (d2 and d1sq positive normal, kappa > 0). */
int aidw_debug_f64_log2_exp2(const double *x, const double *y, int64_t n, double *lx,
                             double *ey);
int aidw_debug_df_weight(const double *d2, const double *d1sq, const double *kappa, int64_t n,
                         double *v, double *w);

#ifdef __cplusplus
}
#endif

#endif /* AIDW_H */
