// rs_pipes.cu -- per-SM issue rates of the arithmetic pipes the deflection
// sum runs on (MUFU reciprocal, FP32 FMA, packed FP32x2 FMA, FP64 FMA).
//
// The deflection sum of Eq. 1 is bound by these pipes, not by HBM or tensor
// cores, so its roofline is SMs x clock x (operations per clock per SM).
// Each kernel runs independent dependency chains per thread and times itself
// with the SM cycle counter, so the rates are per clock and do not depend on
// the clock the GPU happens to run at.
#include <cuda_runtime.h>
#include <string.h>

#include "rs_internal.cuh"

namespace rs {
namespace {

constexpr int CH = 8;   // independent chains per thread

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// which: 0 MUFU rcp (each fed by one FP32 add, which the FP32 pipe absorbs),
// 1 FFMA, 2 FFMA2 (lanes), 3 DFMA
__global__ void pipes_kernel(int which, int iters, float seed, float* sink,
                             unsigned long long* cycles)
{
    const unsigned long long t0 = clock64();
    float v[CH];
    float2 w[CH];
    double d[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        v[c] = seed + 0.01f * c + 1e-3f * threadIdx.x;
        w[c] = make_float2(v[c], v[c] + 0.5f);
        d[c] = (double)v[c];
    }
    const float a = 0.999f, b = 1e-3f;
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    if (which == 0) {
        for (int k = 0; k < iters; ++k)
#pragma unroll
            for (int c = 0; c < CH; ++c) v[c] = rcp_approx(__fadd_rn(v[c], b));
    } else if (which == 1) {
        for (int k = 0; k < iters; ++k)
#pragma unroll
            for (int c = 0; c < CH; ++c) v[c] = __fmaf_rn(v[c], a, b);
    } else if (which == 2) {
        for (int k = 0; k < iters; ++k)
#pragma unroll
            for (int c = 0; c < CH; ++c) w[c] = __ffma2_rn(w[c], a2, b2);
    } else {
        for (int k = 0; k < iters; ++k)
#pragma unroll
            for (int c = 0; c < CH; ++c) d[c] = __fma_rn(d[c], 0.999, 1e-3);
    }
    float acc = 0.f;
#pragma unroll
    for (int c = 0; c < CH; ++c) acc += v[c] + w[c].x + w[c].y + (float)d[c];
    // the chains must finish before the second clock read: make the read
    // wait on their result
    asm volatile("" ::"f"(acc) : "memory");
    __syncthreads();
    const unsigned long long t1 = clock64();
    if (acc == 12345.678f) sink[0] = acc;   // keeps the chains alive
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace
}  // namespace rs

using namespace rs;

extern "C" RS_API int rs_pipe_rates(double* out, int n_out)
{
    clear_error();
    if (!out || n_out < 5) return fail(RS_EINVAL, "out must hold 5 doubles");
    const int sms = num_sms();
    const int blocks_per_sm = 4, threads = 256;
    const int grid = sms * blocks_per_sm;
    float* sink = nullptr;
    unsigned long long* cyc = nullptr;
    int rc = cuda_fail(cudaMalloc(&sink, sizeof(float)), "pipe bench alloc");
    if (!rc) rc = cuda_fail(cudaMalloc(&cyc, grid * sizeof(unsigned long long)), "pipe bench alloc");
    unsigned long long* h = new unsigned long long[grid];
    const int iters[4] = {4096, 16384, 16384, 1024};
    double clock_mhz = 0.0;
    for (int which = 0; which < 4 && !rc; ++which) {
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        pipes_kernel<<<grid, threads>>>(which, iters[which] / 8, 1.5f, sink, cyc);  // warm-up
        cudaEventRecord(e0);
        pipes_kernel<<<grid, threads>>>(which, iters[which], 1.5f, sink, cyc);
        cudaEventRecord(e1);
        rc = cuda_fail(cudaEventSynchronize(e1), "pipe bench");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (!rc) rc = cuda_fail(cudaMemcpy(h, cyc, grid * sizeof(unsigned long long),
                                           cudaMemcpyDeviceToHost), "pipe bench copy");
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rc) break;
        unsigned long long mx = 0;
        for (int k = 0; k < grid; ++k) mx = h[k] > mx ? h[k] : mx;
        // all blocks of an SM are co-resident (4 x 256 threads), so an SM's
        // operations complete within the longest block's cycle count
        const double ops_per_sm = (double)blocks_per_sm * threads * CH * iters[which] *
                                  (which == 2 ? 2.0 : 1.0);
        out[which] = ops_per_sm / (double)mx;
        if (which == 1 && ms > 0) clock_mhz = (double)mx / (ms * 1e3);
    }
    out[4] = clock_mhz;
    delete[] h;
    if (sink) cudaFree(sink);
    if (cyc) cudaFree(cyc);
    return rc;
}
