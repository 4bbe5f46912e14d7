// Microbenchmarks of the pipes that bound the AIDW scans: FP32 FFMA, MUFU ex2 and lg2, FMNMX,
// and FP64 DFMA. Each kernel runs many independent dependency chains per thread on every SM and
// records its own SM clock ticks and global-timer nanoseconds, so the result is in
// instructions per clock per SM and the observed clock is reported beside it.
#include <algorithm>
#include <vector>

#include "aidw_internal.cuh"

namespace aidw {
namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;
constexpr int kProbeThreads = 512;

struct ProbeTimes {
    unsigned long long clk0, clk1, ns0, ns1;
};

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <int OP>
__global__ void __launch_bounds__(kProbeThreads) probe_kernel(float seed, float *sink,
                                                              ProbeTimes *times)
{
    float v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        v[c] = seed + 0.001f * (threadIdx.x + c);
    const float a = seed * 0.5f, b = 1.0f - seed;
    __syncthreads();
    const unsigned long long c0 = clock64(), n0 = global_ns();
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            if (OP == 0)
                v[c] = __fmaf_rn(v[c], a, b);
            else if (OP == 1)
                v[c] = ex2_approx(v[c]);
            else if (OP == 2)
                v[c] = lg2_approx(v[c]);
            else
                v[c] = fminf(fmaxf(v[c], a), b);
        }
    }
    __syncthreads();
    const unsigned long long c1 = clock64(), n1 = global_ns();
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        s += v[c];
    if (s == 12345.678f)
        *sink = s;
    if (threadIdx.x == 0)
        times[blockIdx.x] = ProbeTimes{c0, c1, n0, n1};
}

// FP64 FMA chains (the pipe that bounds the FP64 path).
__global__ void __launch_bounds__(kProbeThreads) probe_dfma_kernel(double seed, double *sink,
                                                                   ProbeTimes *times)
{
    double v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        v[c] = seed + 0.001 * (threadIdx.x + c);
    const double a = seed * 0.5, b = 1.0 - seed;
    __syncthreads();
    const unsigned long long c0 = clock64(), n0 = global_ns();
    for (int i = 0; i < kIters / 8; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            v[c] = __fma_rn(v[c], a, b);
    }
    __syncthreads();
    const unsigned long long c1 = clock64(), n1 = global_ns();
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        s += v[c];
    if (s == 12345.678)
        *sink = s;
    if (threadIdx.x == 0)
        times[blockIdx.x] = ProbeTimes{c0, c1, n0, n1};
}

template <int OP>
cudaError_t run_one(int sm_count, int blocks_per_sm, float *sink, ProbeTimes *d_times,
                    double *per_clk_sm, double *mhz)
{
    const int blocks = sm_count * blocks_per_sm;
    if (OP == 4) {
        double *dsink = reinterpret_cast<double *>(sink);
        probe_dfma_kernel<<<blocks, kProbeThreads>>>(0.37, dsink, d_times);  // warm-up
        probe_dfma_kernel<<<blocks, kProbeThreads>>>(0.37, dsink, d_times);
    } else {
        probe_kernel<OP><<<blocks, kProbeThreads>>>(0.37f, sink, d_times);  // warm-up
        probe_kernel<OP><<<blocks, kProbeThreads>>>(0.37f, sink, d_times);
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess)
        return e;
    std::vector<ProbeTimes> h(blocks);
    e = cudaMemcpy(h.data(), d_times, sizeof(ProbeTimes) * blocks, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return e;
    // Every block is resident at once (blocks_per_sm fits). A pipe that serves the warps of an
    // SM unevenly lets some blocks finish early, so the span is the whole launch's, from the
    // first block's start to the last block's end on the global timer, in clocks at the median
    // clock rate the blocks observed.
    std::vector<double> mh(blocks);
    unsigned long long t0 = h[0].ns0, t1 = h[0].ns1;
    for (int i = 0; i < blocks; ++i) {
        const double ns = static_cast<double>(h[i].ns1 - h[i].ns0);
        mh[i] = ns > 0 ? static_cast<double>(h[i].clk1 - h[i].clk0) / ns * 1e3 : 0.0;
        t0 = std::min(t0, h[i].ns0);
        t1 = std::max(t1, h[i].ns1);
    }
    std::sort(mh.begin(), mh.end());
    const double span = static_cast<double>(t1 - t0) * mh[blocks / 2] * 1e-3;
    const double iters = OP == 4 ? kIters / 8 : kIters;
    const double ops_per_sm = static_cast<double>(blocks_per_sm) * kProbeThreads * iters * kChains;
    *per_clk_sm = ops_per_sm / span;
    *mhz = mh[blocks / 2];
    return cudaSuccess;
}

}  // namespace

cudaError_t run_pipe_probe(int sm_count, aidw_pipe_rates *out)
{
    float *sink = nullptr;
    ProbeTimes *d_times = nullptr;
    const int bps = 2;  // 2 x 512 threads: 32 warps per SM
    cudaError_t e = cudaMalloc(&sink, sizeof(double));
    if (e == cudaSuccess)
        e = cudaMalloc(&d_times, sizeof(ProbeTimes) * sm_count * bps);
    double mhz[4] = {};
    if (e == cudaSuccess)
        e = run_one<0>(sm_count, bps, sink, d_times, &out->ffma_per_clk_sm, &mhz[0]);
    if (e == cudaSuccess)
        e = run_one<1>(sm_count, bps, sink, d_times, &out->ex2_per_clk_sm, &mhz[1]);
    if (e == cudaSuccess)
        e = run_one<2>(sm_count, bps, sink, d_times, &out->lg2_per_clk_sm, &mhz[2]);
    if (e == cudaSuccess)
        e = run_one<3>(sm_count, bps, sink, d_times, &out->fmnmx_per_clk_sm, &mhz[3]);
    double mhz64 = 0.0;
    if (e == cudaSuccess)
        e = run_one<4>(sm_count, bps, sink, d_times, &out->dfma_per_clk_sm, &mhz64);
    out->sm_clock_mhz = (mhz[0] + mhz[1] + mhz[2] + mhz[3]) / 4.0;
    out->sm_count = sm_count;
    out->reserved = 0;
    // fmnmx probe runs two instructions (min and max) per chain step.
    out->fmnmx_per_clk_sm *= 2.0;
    if (sink)
        cudaFree(sink);
    if (d_times)
        cudaFree(d_times);
    return e;
}

}  // namespace aidw
