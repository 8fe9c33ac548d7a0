// peak.cu -- measured throughput of the arithmetic pipes that bound the
// compositing kernels (FP32 fused multiply-add, scalar and packed FP32x2, and
// the special-function unit's ex2), for the roofline fractions a benchmark
// reports against them.  No counterpart in the paper: measurement only.
//
// Each kernel runs independent dependency chains per thread (enough to cover
// the pipe's latency at full occupancy) on a grid of 8 blocks of 256 threads
// per SM and touches no memory; one write behind a condition that never holds
// keeps the chains alive.  The host times a launch of about a few milliseconds
// with CUDA events after a warm-up launch.
#include "gs_internal.cuh"

namespace gs {

__device__ float g_peak_sink;

constexpr int kPeakChains = 8;

__global__ void __launch_bounds__(256) peak_fma_kernel(int iters, float a, float b)
{
    float x[kPeakChains];
#pragma unroll
    for (int k = 0; k < kPeakChains; k++) x[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < 4; u++)
#pragma unroll
            for (int k = 0; k < kPeakChains; k++) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kPeakChains; k++) s += x[k];
    if (s == -1.2345f) g_peak_sink = s;
}

__global__ void __launch_bounds__(256) peak_fma2_kernel(int iters, float a, float b)
{
    float2 x[kPeakChains];
#pragma unroll
    for (int k = 0; k < kPeakChains; k++) x[k] = make_float2((float)(threadIdx.x + k) * 1e-3f, (float)k * 2e-3f);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < 4; u++)
#pragma unroll
            for (int k = 0; k < kPeakChains; k++) x[k] = __ffma2_rn(x[k], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kPeakChains; k++) s += x[k].x + x[k].y;
    if (s == -1.2345f) g_peak_sink = s;
}

__global__ void __launch_bounds__(256) peak_ex2_kernel(int iters)
{
    float x[kPeakChains];
#pragma unroll
    for (int k = 0; k < kPeakChains; k++) x[k] = -(float)(threadIdx.x + k) * 1e-3f;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < 4; u++)
#pragma unroll
            for (int k = 0; k < kPeakChains; k++) {
                float y;
                asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[k]));
                x[k] = -y; // stays in (-1, 0]: 2^x in (1/2, 1]
            }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kPeakChains; k++) s += x[k];
    if (s == -1.2345f) g_peak_sink = s;
}

template <typename F> static double time_kernel(F launch, cudaStream_t st, cudaError_t &err)
{
    cudaEvent_t e0, e1;
    if ((err = cudaEventCreate(&e0)) != cudaSuccess) return 0.0;
    if ((err = cudaEventCreate(&e1)) != cudaSuccess) { cudaEventDestroy(e0); return 0.0; }
    launch(); // warm-up
    cudaEventRecord(e0, st);
    launch();
    cudaEventRecord(e1, st);
    float ms = 0.f;
    if ((err = cudaEventSynchronize(e1)) == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess) err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return (double)ms * 1e-3;
}

} // namespace gs

extern "C" int gs_alu_peaks(gs_alu_peak *out, gs_stream stream)
{
    using namespace gs;
    if (!out) return report_error(GS_ERR_INVALID_ARG, "gs_alu_peaks: NULL out");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || sms <= 0) return report_error(GS_ERR_CUDA, "gs_alu_peaks: device query failed");
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned blocks = 8u * (unsigned)sms;
    const double threads = (double)blocks * 256.0;
    const int iters = 4096;
    const double per_thread = (double)iters * 4 * kPeakChains; // chain steps per thread
    const double t_fma = time_kernel([&] { peak_fma_kernel<<<blocks, 256, 0, st>>>(iters, 0.999f, 1e-4f); }, st, e);
    if (e != cudaSuccess) return report_error(GS_ERR_CUDA, "gs_alu_peaks: FMA kernel failed");
    const double t_fma2 = time_kernel([&] { peak_fma2_kernel<<<blocks, 256, 0, st>>>(iters, 0.999f, 1e-4f); }, st, e);
    if (e != cudaSuccess) return report_error(GS_ERR_CUDA, "gs_alu_peaks: FP32x2 kernel failed");
    const double t_ex2 = time_kernel([&] { peak_ex2_kernel<<<blocks, 256, 0, st>>>(iters / 4); }, st, e);
    if (e != cudaSuccess) return report_error(GS_ERR_CUDA, "gs_alu_peaks: ex2 kernel failed");
    for (int k = 0; k < 6; k++) note_launch(); // three kernels, each warmed up once
    out->sms = sms;
    out->fp32_fma_flops = threads * per_thread * 2.0 / t_fma;
    out->fp32x2_fma_flops = threads * per_thread * 4.0 / t_fma2;
    out->ex2_per_s = threads * (per_thread / 4.0) / t_ex2;
    return GS_OK;
}
