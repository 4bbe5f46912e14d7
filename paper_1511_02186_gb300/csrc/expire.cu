// Test hook for the failure path of the kernels' bounded waits. The kernel below waits with
// the same helpers the scans use (an mbarrier tile wait, a wait on another CTA's counter) on
// something that never completes: an mbarrier nobody arrives on, a counter nobody increments.
// With a short poll limit the wait runs out, the kernel raises the context's error word exactly
// as a scan does and returns; the host then reads AIDW_ERR_TIMEOUT through
// aidw_check_device_errors or the next synchronous call. Nothing faults, traps or hangs.
#include "aidw_runtime.h"

namespace aidw {
namespace {

__global__ void __launch_bounds__(kThreads)
expire_wait_kernel(int which, uint32_t polls, const uint32_t *never, int *err)
{
    __shared__ __align__(8) uint64_t bar;
    __shared__ int flag;
    bool ok;
    if (which == 0) {
        if (threadIdx.x == 0) {
            mbar_init(&bar, 1);
            fence_mbar_init();
        }
        __syncthreads();
        // Phase 0 would complete on one arrival; none comes.
        ok = __syncthreads_and(mbar_wait(&bar, 0, polls));
    } else {
        ok = cta_wait_count(never, 1u, &flag, polls);
    }
    if (!ok && threadIdx.x == 0)
        atomicOr(err, kErrTimeout);
}

}  // namespace
}  // namespace aidw

using namespace aidw;

extern "C" int aidw_debug_expire_wait(aidw_ctx *ctx, int32_t which, uint32_t polls)
{
    if (!ctx || (which != 0 && which != 1) || polls < 1 || polls > (1u << 20))
        return AIDW_ERR_INVALID_ARG;
    if (cudaSetDevice(ctx_device(ctx)) != cudaSuccess)
        return AIDW_ERR_CUDA;
    void *word = nullptr;
    int rc = ctx_alloc(ctx, 256, 0, &word);
    if (rc)
        return rc;
    bool ok = cudaMemsetAsync(word, 0, 256, 0) == cudaSuccess;
    if (ok) {
        expire_wait_kernel<<<1, kThreads, 0, 0>>>(which, polls,
                                                 static_cast<const uint32_t *>(word),
                                                 ctx_err_word(ctx));
        ok = cudaGetLastError() == cudaSuccess;
    }
    ok = cudaStreamSynchronize(0) == cudaSuccess && ok;
    ctx_free(ctx, word, 256, 0);
    return ok ? AIDW_OK : AIDW_ERR_CUDA;
}
