// Measured float32 FMA throughput of the device: the peak the float32 direct assignment
// (one subtract and one FMA per attribute of every point-center distance) is graded
// against.  Not part of the method; a measurement service beside it.
//
// Each thread runs kChains independent FMA chains x <- x * a + b (a < 1, so the values stay
// bounded and finite), enough chains that the FMA latency is hidden at full occupancy.  The
// grid fills every SM; the kernel is timed with CUDA events after a warm-up launch, best of
// five, and the rate counts 2 flops per FMA.
#include <cuda_runtime.h>

#include <cstdio>

#include "pscl.h"
#include "pscl_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

__global__ void __launch_bounds__(kPeakThreads) k_fma_peak(float *out, int iters, float a, float b)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < 4; u++)
#pragma unroll
            for (int c = 0; c < kChains; c++) x[c] = __fmaf_rn(x[c], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += x[c];
    if (s == -1.0f) out[blockIdx.x] = s;      // never true; keeps the chains alive
}

int report(const char *what, cudaError_t e)
{
    char buf[256];
    snprintf(buf, sizeof buf, "%s failed: %s", what, cudaGetErrorString(e));
    cudaGetLastError();
    pscl::set_last_error(buf);
    return PSCL_ECUDA;
}

}  // namespace

extern "C" int pscl_measure_fp32_fma(int device, double *tflops)
{
    if (!tflops) {
        pscl::set_last_error("tflops is NULL");
        return PSCL_EINVAL;
    }
    cudaError_t e;
    if ((e = cudaSetDevice(device)) != cudaSuccess) return report("cudaSetDevice", e);
    int sms = 0, per_sm = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess)
        return report("cudaDeviceGetAttribute", e);
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_peak, kPeakThreads, 0)) != cudaSuccess)
        return report("cudaOccupancyMaxActiveBlocksPerMultiprocessor", e);
    const int grid = sms * (per_sm > 0 ? per_sm : 1);
    const int iters = 1 << 14;
    float *out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    int rc = PSCL_OK;
    float best = 0.0f;
    if ((e = cudaMalloc(&out, (size_t)grid * sizeof(float))) != cudaSuccess) return report("cudaMalloc", e);
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreate(&t0)) != cudaSuccess || (e = cudaEventCreate(&t1)) != cudaSuccess) {
        rc = report("stream/event creation", e);
    } else {
        k_fma_peak<<<grid, kPeakThreads, 0, st>>>(out, iters, 0.999f, 1e-3f);     // warm-up
        for (int r = 0; r < 5 && rc == PSCL_OK; r++) {
            cudaEventRecord(t0, st);
            k_fma_peak<<<grid, kPeakThreads, 0, st>>>(out, iters, 0.999f, 1e-3f);
            cudaEventRecord(t1, st);
            if ((e = cudaEventSynchronize(t1)) != cudaSuccess) {
                rc = report("k_fma_peak", e);
                break;
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, t0, t1);
            if (best == 0.0f || ms < best) best = ms;
        }
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (st) cudaStreamDestroy(st);
    cudaFree(out);
    if (rc != PSCL_OK) return rc;
    const double fmas = (double)grid * kPeakThreads * iters * 4.0 * kChains;
    *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
    return PSCL_OK;
}
