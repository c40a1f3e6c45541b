// Vector FMA throughput of the device (dtsph_fma_peak): the compute ceiling of
// the roofline for kernels bound by plain FP32 or FP64 arithmetic.
//
// Every thread runs kChains independent multiply-add chains x = x a + b, so the
// FMA pipe always has independent work; the grid fills every SM several times.
// The sum of the chains is stored only under a condition the inputs never meet,
// so the compiler keeps the arithmetic without the store adding traffic. Timed
// with CUDA events on a private stream, best of three launches, each sized to
// about 50 ms after a calibration launch.
#include <algorithm>

#include "dtsph_internal.cuh"

namespace dtsph {
namespace {

constexpr int kChains = 8;
constexpr int kPeakBlocksPerSm = 8;

template <typename T>
__device__ __forceinline__ T fma_op(T x, T a, T b);
template <>
__device__ __forceinline__ float fma_op<float>(float x, float a, float b) { return __fmaf_rn(x, a, b); }
template <>
__device__ __forceinline__ double fma_op<double>(double x, double a, double b) { return __fma_rn(x, a, b); }

template <typename T>
__global__ void __launch_bounds__(kBlock) k_fma_peak(T *out, long long iters, T a, T b)
{
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + 1) * (T)1e-3 + (T)c;
    for (long long k = 0; k < iters; ++k) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma_op<T>(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == (T)-1.25) out[blockIdx.x] = s;   // never true for these inputs
}

// Seconds of one launch of `iters` iterations.
template <typename T>
int time_launch(int grid, long long iters, T *out, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, double *sec)
{
    // a = 1 - 2^-20, b = 2^-30: the chains stay finite and normal for any length
    const T a = (T)(1.0 - 1.0 / 1048576.0), b = (T)(1.0 / 1073741824.0);
    if (cudaEventRecord(e0, st) != cudaSuccess) return DTSPH_E_CUDA;
    k_fma_peak<T><<<grid, kBlock, 0, st>>>(out, iters, a, b);
    if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return DTSPH_E_CUDA;
    float ms = 0;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return DTSPH_E_CUDA;
    *sec = 1e-3 * ms;
    return DTSPH_OK;
}

template <typename T>
int fma_peak(double *flops)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return DTSPH_E_CUDA;
    const int grid = sms * kPeakBlocksPerSm;
    T *out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int r = DTSPH_E_CUDA;
    if (cudaMalloc((void **)&out, sizeof(T) * grid) == cudaSuccess &&
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess && cudaEventCreate(&e0) == cudaSuccess &&
        cudaEventCreate(&e1) == cudaSuccess) {
        double sec = 0;
        long long iters = 1024;
        r = time_launch<T>(grid, iters, out, st, e0, e1, &sec);          // calibration (and module load)
        if (!r) r = time_launch<T>(grid, iters, out, st, e0, e1, &sec);
        if (!r) {
            iters = std::max(1024LL, (long long)(iters * 0.05 / std::max(sec, 1e-6)));
            double best = 1e30;
            for (int rep = 0; rep < 3 && !r; ++rep) {
                r = time_launch<T>(grid, iters, out, st, e0, e1, &sec);
                best = std::min(best, sec);
            }
            const double per_launch = 2.0 * kChains * (double)iters * (double)grid * kBlock;
            if (!r) *flops = per_launch / best;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (out) cudaFree(out);
    if (cudaGetLastError() != cudaSuccess) r = DTSPH_E_CUDA;
    return r;
}

}  // namespace
}  // namespace dtsph

extern "C" int dtsph_fma_peak(int32_t precision, double *flop_per_s)
{
    if (!flop_per_s || (precision != DTSPH_FP64 && precision != DTSPH_FP32C)) return DTSPH_E_ARG;
    return precision == DTSPH_FP64 ? dtsph::fma_peak<double>(flop_per_s) : dtsph::fma_peak<float>(flop_per_s);
}
