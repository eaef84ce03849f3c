// FP32 FMA throughput of the current device: the denominator of the residual kernels' ALU
// roofline (those kernels are bound by FP32 arithmetic, not by HBM). Every thread of a
// fully occupied grid (8 blocks of 256 threads per SM) runs eight independent FMA chains,
// either as scalar fma.rn.f32 or as four paired fma.rn.f32x2 chains; the rate is the
// executed FMA count x 2 flops over the CUDA-event time of the launch.
#include <cuda_runtime.h>

#include "sd_internal.h"

namespace {

constexpr int PEAK_THREADS = 256;
constexpr int PEAK_BLOCKS_PER_SM = 8;

template <int PACKED>
__global__ void __launch_bounds__(PEAK_THREADS) k_fma_rate(float* __restrict__ out, float b, float c, int iters) {
    float s = 0.0f;
    if constexpr (PACKED) {
        const unsigned long long bb = ((unsigned long long)__float_as_uint(b) << 32) | __float_as_uint(b);
        const unsigned long long cc = ((unsigned long long)__float_as_uint(c) << 32) | __float_as_uint(c);
        unsigned long long a[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float lo = 1.0f + 1e-3f * (threadIdx.x + k), hi = 2.0f + 1e-3f * (threadIdx.x + k);
            a[k] = ((unsigned long long)__float_as_uint(hi) << 32) | __float_as_uint(lo);
        }
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < 4; ++k) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[k]) : "l"(bb), "l"(cc));
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) s += __uint_as_float((unsigned)a[k]) + __uint_as_float((unsigned)(a[k] >> 32));
    } else {
        float a[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = 1.0f + 1e-3f * (threadIdx.x + k);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < 8; ++k) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a[k]) : "f"(b), "f"(c));
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) s += a[k];
    }
    // never true for these inputs; keeps the chains live
    if (s == -1.0f) out[threadIdx.x] = s;
}

}  // namespace

extern "C" sd_status sd_measure_fp32_peak(int packed, double* tflops) {
    if (!tflops || (packed != 0 && packed != 1)) { sdi_set_error("bad argument"); return SD_EINVAL; }
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
        sdi_set_error("no CUDA device");
        return SD_ECUDA;
    }
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float* out = nullptr;
    sd_status status = SD_OK;
    const int blocks = sms * PEAK_BLOCKS_PER_SM;
    const int iters = 1 << 16;
    float ms = 0.0f;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess || cudaMalloc(&out, PEAK_THREADS * sizeof(float)) != cudaSuccess) {
        status = SD_ECUDA;
    } else {
        for (int rep = 0; rep < 2 && status == SD_OK; ++rep) {   // first launch warms up
            cudaEventRecord(e0, st);
            if (packed) k_fma_rate<1><<<blocks, PEAK_THREADS, 0, st>>>(out, 0.9999999f, 1e-7f, iters);
            else k_fma_rate<0><<<blocks, PEAK_THREADS, 0, st>>>(out, 0.9999999f, 1e-7f, iters);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                status = SD_ECUDA;
        }
    }
    if (status != SD_OK) {
        cudaGetLastError();
        sdi_set_error("FP32 peak measurement failed");
    } else {
        const double fmas = (double)blocks * PEAK_THREADS * 8.0 * iters;
        *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
    }
    if (out) cudaFree(out);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    return status;
}
