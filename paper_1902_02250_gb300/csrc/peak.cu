// Arithmetic-issue micro-benchmarks (include/kitc_peak.h): the denominators of
// the evaluator's and the weights pass's rooflines, measured on the device
// instead of derived from unit counts.
//
// Every thread runs CHAINS independent recurrences a <- a * b + c for `iters`
// rounds, so the only dependences are the chains' own and the issue rate of
// the pipe under test sets the time.  b and c are kernel arguments (no
// constant folding); the final values are written out so nothing is dead.
#include "common.cuh"
#include "kitc_peak.h"

namespace {

constexpr int CHAINS = 8;  // independent accumulators per thread

__global__ void __launch_bounds__(256) k_peak_ffma(float b, float c, int iters, float *sink)
{
    float a[CHAINS];
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) a[i] = (float)(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int i = 0; i < CHAINS; ++i) a[i] = fmaf(a[i], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) s += a[i];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_peak_ffma2(float b, float c, int iters, float *sink)
{
    float2 a[CHAINS];
    const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) a[i] = make_float2((float)(threadIdx.x + i), (float)i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int i = 0; i < CHAINS; ++i) a[i] = __ffma2_rn(a[i], b2, c2);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) s += a[i].x + a[i].y;
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_peak_dfma(double b, double c, int iters, float *sink)
{
    double a[CHAINS];
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) a[i] = (double)(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int i = 0; i < CHAINS; ++i) a[i] = fma(a[i], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) s += a[i];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

// One MUFU reciprocal square root per step of each chain, then an FMA to keep
// the value in range: counts rsqrt issues, the special-function unit's rate.
__global__ void __launch_bounds__(256) k_peak_rsqrt(float b, float c, int iters, float *sink)
{
    float a[CHAINS];
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) a[i] = 1.f + (float)(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int i = 0; i < CHAINS; ++i) {
                float y;
                asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[i]));
                a[i] = fmaf(y, b, c);
            }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) s += a[i];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" {

double kitc_peak_ops_per_launch(int kind, int blocks, int threads, int iters)
{
    const double per_thread_round = (double)iters * 16.0 * CHAINS;
    const double thr = (double)blocks * (double)threads;
    switch (kind) {
    case KITC_PEAK_FFMA: return thr * per_thread_round * 2.0;   // flops, FMA = 2
    case KITC_PEAK_FFMA2: return thr * per_thread_round * 4.0;  // two lanes of FMA
    case KITC_PEAK_DFMA: return thr * per_thread_round * 2.0;
    case KITC_PEAK_RSQRT: return thr * per_thread_round;        // rsqrt results
    default: return -1.0;
    }
}

kitc_status kitc_peak_launch(int kind, int blocks, int threads, int iters, float *sink,
                             void *stream)
{
    if (blocks < 1 || blocks > (1 << 20) || threads < 32 || threads > 256 || threads % 32 ||
        iters < 1 || !sink)
        return KITC_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // b slightly below 1 and c small keep every chain bounded and normal
    const float b = 0.999999f, c = 1e-3f;
    switch (kind) {
    case KITC_PEAK_FFMA: k_peak_ffma<<<blocks, threads, 0, s>>>(b, c, iters, sink); break;
    case KITC_PEAK_FFMA2: k_peak_ffma2<<<blocks, threads, 0, s>>>(b, c, iters, sink); break;
    case KITC_PEAK_DFMA: k_peak_dfma<<<blocks, threads, 0, s>>>((double)b, (double)c, iters, sink); break;
    case KITC_PEAK_RSQRT: k_peak_rsqrt<<<blocks, threads, 0, s>>>(0.5f, 1.f, iters, sink); break;
    default: return KITC_ERR_INVALID_ARG;
    }
    kitc_count_launch();
    return kitc_from_cuda(cudaGetLastError());
}

}  // extern "C"
