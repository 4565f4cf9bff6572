// md_peak.cu -- md_measure_fp32_peak: the FP32 FMA throughput of the current GPU, measured.
//
// The FP32 roofline of the step kernel (its pair arithmetic runs on the FP32 pipe) needs a peak
// that was measured on the device itself rather than taken from unit counts and a nominal clock.
// This kernel keeps every FP32 lane busy with independent fused multiply-add chains: each thread
// advances kChains accumulators, a <- a * b + c, for `iters` rounds, so each round issues kChains
// independent FMAs per thread (enough to cover the FMA latency with two warps per scheduler),
// and the grid fills every SM with its maximum resident threads.  Flops = 2 per FMA.  The
// accumulators are summed and written out so that no FMA can be removed.
#include "md.h"

#include <cuda_runtime.h>

#include <cstdio>

namespace {

constexpr int kChains = 8;
constexpr int kBlock = 256;

__global__ void __launch_bounds__(kBlock) k_fma_peak(float *out, int iters, float b, float c) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = __fmaf_rn(a[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int md_measure_fp32_peak(void *cuda_stream, int repeats, double *tflops, int *sms,
                                    double *ms) {
    if (!tflops || repeats < 1) return MD_EINVAL;
    int dev = 0, nsm = 0, thr = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&thr, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess) {
        cudaGetLastError();
        return MD_ECUDA;
    }
    const int grid = nsm * (thr / kBlock);
    const int iters = 1 << 16;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    float *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMalloc(&out, sizeof(float) * (size_t)grid * kBlock) != cudaSuccess) {
        cudaGetLastError();
        return MD_ENOMEM;
    }
    int rc = MD_OK;
    double best = 0.0, best_ms = 0.0;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = MD_ECUDA;
    } else {
        // one untimed launch (clocks up, code loaded), then the timed repeats
        k_fma_peak<<<grid, kBlock, 0, st>>>(out, iters, 0.999999f, 1e-6f);
        for (int r = 0; rc == MD_OK && r < repeats; ++r) {
            cudaEventRecord(e0, st);
            k_fma_peak<<<grid, kBlock, 0, st>>>(out, iters, 0.999999f, 1e-6f);
            cudaEventRecord(e1, st);
            float t = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&t, e0, e1) != cudaSuccess || !(t > 0.f)) {
                rc = MD_ECUDA;
                break;
            }
            const double flops = 2.0 * kChains * (double)iters * (double)grid * kBlock;
            const double tf = flops / (t * 1e-3) / 1e12;
            if (tf > best) {
                best = tf;
                best_ms = t;
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (rc != MD_OK) {
        cudaGetLastError();
        return rc;
    }
    *tflops = best;
    if (sms) *sms = nsm;
    if (ms) *ms = best_ms;
    return MD_OK;
}
