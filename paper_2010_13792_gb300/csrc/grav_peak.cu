// CUDA-core FMA throughput probe (FP32 or FP64), used to state the peak the
// force kernels are measured against.  Not part of the method.
#include <cmath>

#include "grav_common.cuh"

namespace grav {
namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kPeakThreads = 256;

// Sink that keeps the FMA chains live (written only if their sum hits a value
// it never reaches).
__device__ double g_peak_sink;

template <typename T>
__global__ void __launch_bounds__(kPeakThreads)
fma_peak_kernel(int iters, T a, T b)
{
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == (T)-1.2345) g_peak_sink = (double)s;
}

// Packed FP32x2 variant: each __ffma2_rn is two FMAs (four flops).
__global__ void __launch_bounds__(kPeakThreads)
fma2_peak_kernel(int iters, float2 a, float2 b)
{
    float2 x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = make_float2((threadIdx.x + c) * 1e-3f, (threadIdx.x - c) * 1e-3f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
    if (s == -1.2345f) g_peak_sink = (double)s;
}

template <typename T>
struct PeakKernel {
    static void launch(int blocks, int iters, cudaStream_t st)
    {
        fma_peak_kernel<T><<<blocks, kPeakThreads, 0, st>>>(iters, (T)0.999999, (T)1e-7);
    }
    static const void *fn() { return (const void *)fma_peak_kernel<T>; }
    static constexpr double flops_per_op = 2.0;
};

template <>
struct PeakKernel<float2> {
    static void launch(int blocks, int iters, cudaStream_t st)
    {
        fma2_peak_kernel<<<blocks, kPeakThreads, 0, st>>>(iters, make_float2(0.999999f, 0.999998f),
                                                          make_float2(1e-7f, 2e-7f));
    }
    static const void *fn() { return (const void *)fma2_peak_kernel; }
    static constexpr double flops_per_op = 4.0;
};

template <typename T>
int run(double seconds, double *flops, cudaStream_t st)
{
    int sms = 0;
    int rc = device_sm_count(&sms);
    if (rc) return rc;
    int per_sm = 0;
    rc = check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, PeakKernel<T>::fn(),
                                                                   kPeakThreads, 0),
                    "occupancy");
    if (rc) return rc;
    const int blocks = sms * (per_sm > 0 ? per_sm : 1);
    cudaEvent_t e0, e1;
    rc = check_cuda(cudaEventCreate(&e0), "cudaEventCreate");
    if (rc) return rc;
    rc = check_cuda(cudaEventCreate(&e1), "cudaEventCreate");
    if (rc) {
        cudaEventDestroy(e0);
        return rc;
    }
    int iters = 256;
    double best = 0.0, last = 0.0;
    for (int round = 0; round < 8 && rc == GRAV_OK; ++round) {
        cudaEventRecord(e0, st);
        PeakKernel<T>::launch(blocks, iters, st);
        cudaEventRecord(e1, st);
        rc = check_cuda(cudaEventSynchronize(e1), "fma peak kernel");
        if (rc) break;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double fl = PeakKernel<T>::flops_per_op * kChains * kUnroll * (double)iters * blocks *
                          kPeakThreads;
        const double rate = fl / (ms * 1e-3);
        last = rate;
        if (ms > 0.25 * seconds * 1e3) best = std::max(best, rate);
        if (ms < seconds * 1e3 && iters < (1 << 28)) {
            double scale = (seconds * 1e3) / std::max(ms, 1e-3f);
            iters = (int)std::min<double>((double)(1 << 28), iters * std::min(scale, 64.0));
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    *flops = best > 0.0 ? best : last;
    return GRAV_OK;
}

}  // namespace
}  // namespace grav

extern "C" int grav_measure_fma_peak(int32_t precision, double seconds_target, double *flops_per_s,
                                     void *stream)
{
    using namespace grav;
    if (!flops_per_s) return fail(GRAV_EINVAL, "grav_measure_fma_peak: null output");
    if (!(seconds_target > 0.0) || seconds_target > 30.0)
        return fail(GRAV_EINVAL, "grav_measure_fma_peak: seconds_target outside (0, 30]");
    if (precision == GRAV_MIXED) return run<float>(seconds_target, flops_per_s, as_stream(stream));
    if (precision == GRAV_F64) return run<double>(seconds_target, flops_per_s, as_stream(stream));
    if (precision == GRAV_PEAK_F32X2) return run<float2>(seconds_target, flops_per_s, as_stream(stream));
    return fail(GRAV_EINVAL, "grav_measure_fma_peak: bad precision");
}
