// Measurement aid: the FP64 fused multiply-add rate of the device.
//
// The re-factorization is bound by the non-tensor FP64 pipe, so its
// roofline is that pipe's rate.  This kernel keeps it busy with eight
// independent multiply-add chains per thread, enough to cover the
// pipeline latency on every SM sub-partition, and the host side times it
// with CUDA events.  Not part of the paper's method.
#include <cuda_runtime.h>

#include <cstdint>

#include "gblu_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) dfma_rate_kernel(double *out, int iters, double a, double b)
{
    double v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) v[c] = threadIdx.x * 1e-3 + c;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < kChains; c++) v[c] = fma(v[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += v[c];
    // a store that the compiler cannot drop, almost never taken
    if (s == 1234.5) out[blockIdx.x * kThreads + threadIdx.x] = s;
}

}  // namespace

extern "C" int gblu_fp64_fma_rate(int device, double *tflops)
{
    using gblu::record_error;
    if (!tflops) return record_error(GBLU_ERR_INVALID_INPUT, "gblu_fp64_fma_rate: tflops is NULL");
    *tflops = 0.0;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return record_error(GBLU_ERR_CUDA, "gblu_fp64_fma_rate: cannot use the device");
    }
    int sms = 0, per = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, dfma_rate_kernel, kThreads, 0) != cudaSuccess) {
        cudaGetLastError();
        return record_error(GBLU_ERR_CUDA, "gblu_fp64_fma_rate: device query failed");
    }
    const int grid = sms * (per < 1 ? 1 : per);
    const int iters = 1 << 14;
    double *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = GBLU_OK;
    if (cudaMalloc(&out, sizeof(double) * (size_t)grid * kThreads) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = record_error(GBLU_ERR_CUDA, "gblu_fp64_fma_rate: allocation failed");
    } else {
        float best = 0.0f;
        for (int rep = 0; rep < 4 && rc == GBLU_OK; rep++) {   // the first run warms up
            cudaEventRecord(e0);
            dfma_rate_kernel<<<grid, kThreads>>>(out, iters, 0.999999, 1e-7);
            cudaEventRecord(e1);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = record_error(GBLU_ERR_CUDA, "gblu_fp64_fma_rate: launch failed");
                break;
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && (best == 0.0f || ms < best)) best = ms;
        }
        if (rc == GBLU_OK && best > 0.0f)
            *tflops = 2.0 * kChains * (double)iters * grid * kThreads / (best * 1e-3) / 1e12;
    }
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    return rc;
}
