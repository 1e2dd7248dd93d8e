// Measured arithmetic peaks of the device for the roofline of the FP32 (condensing, ADMM) and
// FP64 (factorisation, KKT check) kernels: independent fused multiply-add chains in every lane,
// timed with CUDA events, and the L2 size from the device attributes.  Also the HBM rates of
// streams that only read, only write, or copy, for kernels whose traffic is mostly one way.
#include "ctx.h"

namespace gmi {
namespace {

constexpr int kChains = 8;      // independent FMA chains per thread (hides the pipe latency)
constexpr int kUnroll = 16;

template <class T>
__global__ void __launch_bounds__(256) fma_peak_kernel(T* out, int iters, T a, T b) {
    T x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = (T)(threadIdx.x + j) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int j = 0; j < kChains; ++j) x[j] = fma(x[j], a, b);
    }
    T s = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += x[j];
    if (s == (T)-12345.678) out[blockIdx.x] = s;   // never true for these inputs: keeps the work
}

template <class T>
gm_status time_fma(int sms, double* tflops, cudaStream_t st) {
    const int blocks = sms * 8, threads = 256, iters = sizeof(T) == 4 ? 4096 : 64;
    T* out = nullptr;   // never written (the guard above is false)
    cudaEvent_t e0, e1;
    GM_CUDA_TRY(cudaEventCreate(&e0));
    GM_CUDA_TRY(cudaEventCreate(&e1));
    fma_peak_kernel<T><<<blocks, threads, 0, st>>>(out, iters / 8, (T)0.999, (T)1e-4);   // warm-up
    GM_LAUNCH_CHECK();
    GM_CUDA_TRY(cudaEventRecord(e0, st));
    fma_peak_kernel<T><<<blocks, threads, 0, st>>>(out, iters, (T)0.999, (T)1e-4);
    GM_LAUNCH_CHECK();
    GM_CUDA_TRY(cudaEventRecord(e1, st));
    GM_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    GM_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double fmas = (double)blocks * threads * iters * kUnroll * kChains;
    *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
    return GM_OK;
}

// Streams over n float4 (grid-stride, 16-byte accesses).
__global__ void __launch_bounds__(512) hbm_read_kernel(const float4* __restrict__ a, long n, float* out) {
    float s = 0.f;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float4 v = __ldcs(a + i);
        s += v.x + v.y + v.z + v.w;
    }
    if (s == -12345.678f) out[0] = s;   // never true for the zero-filled buffer: keeps the loads
}
__global__ void __launch_bounds__(512) hbm_write_kernel(float4* __restrict__ b, long n) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        __stcs(b + i, make_float4(0.f, 0.f, 0.f, 0.f));
}
__global__ void __launch_bounds__(512) hbm_copy_kernel(const float4* __restrict__ a, float4* __restrict__ b, long n) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        __stcs(b + i, __ldcs(a + i));
}

}  // namespace
}  // namespace gmi

extern "C" gm_status gm_measure_hbm(void* buf, size_t bytes, int repeats, double* read_gbs, double* write_gbs,
                                    double* copy_gbs, void* stream) {
    using namespace gmi;
    clear_error();
    GM_CHECK_ARG(buf && read_gbs && write_gbs && copy_gbs, "NULL argument");
    GM_CHECK_ARG(((uintptr_t)buf & 15) == 0, "buffer must be 16-byte aligned");
    GM_CHECK_ARG(bytes >= ((size_t)64 << 20) && repeats >= 1, "buffer below 64 MB or repeats < 1");
    int dev = 0, sms = 0;
    GM_CUDA_TRY(cudaGetDevice(&dev));
    GM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long n = (long)(bytes / 2 / 16);           // float4 per half
    float4* a = static_cast<float4*>(buf);
    float4* b = a + n;
    const int grid = sms * 4, threads = 512;
    GM_CUDA_TRY(cudaMemsetAsync(buf, 0, (size_t)n * 32, st));
    cudaEvent_t e0, e1;
    GM_CUDA_TRY(cudaEventCreate(&e0));
    GM_CUDA_TRY(cudaEventCreate(&e1));
    double best[3] = {0.0, 0.0, 0.0};
    for (int r = 0; r <= repeats; ++r) {             // r = 0: warm-up
        for (int k = 0; k < 3; ++k) {
            GM_CUDA_TRY(cudaEventRecord(e0, st));
            if (k == 0) hbm_read_kernel<<<grid, threads, 0, st>>>(a, n, reinterpret_cast<float*>(b));
            else if (k == 1) hbm_write_kernel<<<grid, threads, 0, st>>>(b, n);
            else hbm_copy_kernel<<<grid, threads, 0, st>>>(a, b, n);
            GM_LAUNCH_CHECK();
            GM_CUDA_TRY(cudaEventRecord(e1, st));
            GM_CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0.f;
            GM_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            const double moved = (double)n * 16 * (k == 2 ? 2 : 1);
            if (r > 0) best[k] = std::max(best[k], moved / (ms * 1e-3) / 1e9);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *read_gbs = best[0];
    *write_gbs = best[1];
    *copy_gbs = best[2];
    return GM_OK;
}

extern "C" gm_status gm_measure_peaks(double* fp32_tflops, double* fp64_tflops, long long* l2_bytes, void* stream) {
    using namespace gmi;
    clear_error();
    GM_CHECK_ARG(fp32_tflops && fp64_tflops && l2_bytes, "NULL argument");
    int dev = 0, sms = 0, l2 = 0;
    GM_CUDA_TRY(cudaGetDevice(&dev));
    GM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    GM_CUDA_TRY(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    GM_TRY(time_fma<float>(sms, fp32_tflops, st));
    GM_TRY(time_fma<double>(sms, fp64_tflops, st));
    *l2_bytes = l2;
    return GM_OK;
}
