// Allocation-free variant of the FP32 interpolation (aidw_interpolate_noalloc).
//
// Who needs it: callers that must not allocate device memory while they serve a call, e.g.
// a process that reserves its whole device footprint at start-up and may not grow it or risk
// an out-of-memory failure in the middle of a request, or code for which the implicit device
// synchronisation that cudaFree (and possibly cudaMalloc) performs is not acceptable.
// aidw_interpolate takes its per-call scratch from a stream-ordered pool, which can allocate;
// this entry point instead uses one fixed scratch area that is part of the library image.
//
// The scratch area is a file-scope __device__ array of kNoAllocScratchBytes. Every GPU that
// loads the library holds it until the process exits. Host code cannot use the array's name
// as a device address (in host code it names a host-side stand-in), so the device address is
// looked up with cudaGetSymbolAddress once per device, with that device current. aidw_init does
// this when it creates a context: under CUDA's lazy module loading the lookup is what places
// this file's module, and with it the array, on the device, so it belongs at set-up and not in
// the middle of a request.
//
// The call takes the same phase-1 route as aidw_interpolate when its scratch fits: up to
// 32,768 queries one warp per query; above, the pruned scan over Z-ordered queries (the query
// ordering needs about 24 more bytes per query); otherwise, or when that does not fit, the split
// scan with as few splits as the area requires.
#include <mutex>

#include "aidw_internal.cuh"
#include "aidw_runtime.h"

namespace aidw {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;  // 16 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on `device` (which must be current); null on failure.
void *scratch_address(int device)
{
    if (device < 0 || device >= kMaxDevices)
        return nullptr;
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_scratch_ptr[device]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_scratch_ptr[device] = p;
    }
    return g_scratch_ptr[device];
}

}  // namespace

int noalloc_prepare(int device)
{
    return scratch_address(device) ? AIDW_OK : AIDW_ERR_CUDA;
}

}  // namespace aidw

using namespace aidw;

extern "C" int aidw_interpolate_noalloc(aidw_ctx *ctx, aidw_dataset ds, const float *qx,
                                        const float *qy, int64_t m, const aidw_params *p,
                                        float *out, void *stream)
{
    if (!ctx || !p)
        return AIDW_ERR_INVALID_ARG;
    DatasetDev dev;
    double r_exp;
    if (!dataset_lookup(ctx, ds, &dev, &r_exp))
        return AIDW_ERR_NOT_FOUND;
    int rc = validate_params(p, dev.n);
    if (rc)
        return rc;
    if (p->precision != AIDW_F32C || m < 0)
        return AIDW_ERR_INVALID_ARG;
    if (m == 0)
        return AIDW_OK;
    const int device = ctx_device(ctx);
    if (!qx || !qy || !out || pointer_kind(qx, device) != 1 || pointer_kind(qy, device) != 1 ||
        pointer_kind(out, device) != 1)
        return AIDW_ERR_INVALID_ARG;  // device arrays only: host arrays would need staging
    if (cudaSetDevice(device) != cudaSuccess)
        return AIDW_ERR_CUDA;
    void *base = scratch_address(device);  // resolved by aidw_init: a table read here
    if (!base)
        return AIDW_ERR_CUDA;
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const Plan planned = make_plan(ctx, AIDW_F32C, dev.n_pad, m, p->k, false, 0, 0);

    // Per-query phase 1 where aidw_interpolate would take it (one list per query, no ordering).
    if (use_warp_knn(AIDW_F32C, dev, m, 0)) {
        Plan pl = planned;
        pl.knn.splits = 1;
        pl.knn.split_len = dev.n_pad;
        while (scratch_bytes(AIDW_F32C, pl, p->k) > kNoAllocScratchBytes && pl.w.splits > 1) {
            pl = make_plan(ctx, AIDW_F32C, dev.n_pad, m, p->k, false, 0, pl.w.splits - 1);
            pl.knn.splits = 1;
            pl.knn.split_len = dev.n_pad;
        }
        if (scratch_bytes(AIDW_F32C, pl, p->k) <= kNoAllocScratchBytes) {
            Scratch sc;
            scratch_carve(base, AIDW_F32C, pl, p->k, &sc);
            return enqueue_warp(ctx, dev, r_exp, pl, *p, qx, qy, sc, out, nullptr, nullptr, st,
                                false);
        }
    }

    // Pruned phase 1 where aidw_interpolate would take it, with fewer phase-2 splits if the
    // area needs it (splits only regroup the FP32 partial sums).
    if (use_culled_knn(AIDW_F32C, dev, m, false, planned)) {
        Plan pl = planned;
        plan_culled_knn(&pl, dev.n_pad);
        const size_t extra = culled_extra_bytes(m, AIDW_F32C);
        while (scratch_bytes(AIDW_F32C, pl, p->k) + extra > kNoAllocScratchBytes &&
               pl.w.splits > 1) {
            pl = make_plan(ctx, AIDW_F32C, dev.n_pad, m, p->k, false, 0, pl.w.splits - 1);
            plan_culled_knn(&pl, dev.n_pad);
        }
        const size_t sb = scratch_bytes(AIDW_F32C, pl, p->k);
        if (sb + extra <= kNoAllocScratchBytes) {
            Scratch sc;
            scratch_carve(base, AIDW_F32C, pl, p->k, &sc);
            // Every scratch element (lists, parameters, partial sums, sort keys and counts,
            // ordered queries) is written before it is read, so nothing needs clearing.
            return enqueue_culled(ctx, dev, r_exp, pl, *p, qx, qy, sc,
                                  static_cast<char *>(base) + sb, out, nullptr, nullptr, st,
                                  false);
        }
    }

    // Split scan: plan as usual, then give up splits until the scratch fits the fixed area.
    Plan pl = planned;
    while (scratch_bytes(AIDW_F32C, pl, p->k) > kNoAllocScratchBytes &&
           (pl.knn.splits > 1 || pl.w.splits > 1)) {
        const int s1 = pl.knn.splits > 1 ? pl.knn.splits - 1 : 1;
        const int s2 = pl.w.splits > 1 ? pl.w.splits - 1 : 1;
        pl = make_plan(ctx, AIDW_F32C, dev.n_pad, m, p->k, false, s1, s2);
    }
    if (scratch_bytes(AIDW_F32C, pl, p->k) > kNoAllocScratchBytes)
        return AIDW_ERR_INVALID_ARG;  // m * (4k + 24) bytes exceed the 16 MiB area
    Scratch sc;
    scratch_carve(base, AIDW_F32C, pl, p->k, &sc);
    // Every scratch element is written before it is read, so nothing needs clearing.
    return enqueue_interpolation(ctx, dev, r_exp, pl, *p, qx, qy, sc, out, nullptr, nullptr, st,
                                 false);
}
