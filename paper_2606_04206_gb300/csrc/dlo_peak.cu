// dlo_peak.cu -- the FP32 roofline's denominator, measured on the device the library runs on:
// a kernel of independent register-only FMA chains that keeps every FP32 lane of every SM
// busy, timed with CUDA events.  Not part of the method; the rod kernels' achieved FLOP/s are
// reported against this figure.
#include <cuda_runtime.h>

#include "dlo.h"

namespace {

constexpr int kChains = 8;      // independent accumulators per thread (hides the FMA latency)
constexpr int kUnroll = 64;     // FMAs per chain per loop trip

__global__ void __launch_bounds__(256) fma_peak_kernel(float* sink, int trips, float m, float c) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (float)(threadIdx.x + k) * 1e-7f;
    for (int t = 0; t < trips; ++t) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], m, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == 1234.5f) sink[blockIdx.x] = s;   // keeps the chains live; never true for these inputs
}

}  // namespace

extern "C" dlo_status dlo_measure_fp32_peak(double seconds, void* cuda_stream, double* tflops) {
    if (!tflops || !(seconds > 0.0) || seconds > 60.0) return DLO_ERR_INVALID_ARG;
    *tflops = 0.0;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0, tpm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&tpm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    if (e != cudaSuccess) return DLO_ERR_CUDA;
    const int threads = 256, grid = sms * (tpm / threads);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float* sink = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(float) * grid);
    double result = 0.0;
    if (e == cudaSuccess) {
        // a short launch to warm up and estimate the rate, then one launch of about `seconds`
        int trips = 256;
        for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
            e = cudaEventRecord(e0, st);
            if (e == cudaSuccess) {
                fma_peak_kernel<<<grid, threads, 0, st>>>(sink, trips, 0.9999999f, 1e-7f);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess || !(ms > 0.f)) break;
            const double flops = 2.0 * kChains * kUnroll * (double)trips * (double)threads * (double)grid;
            result = flops / (ms * 1e-3) / 1e12;
            if (pass == 0) {
                const double want = seconds * 1e3 / ms * trips;
                trips = (int)(want < 256.0 ? 256.0 : (want > 2e9 ? 2e9 : want));
            }
        }
    }
    if (sink) cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return DLO_ERR_CUDA;
    *tflops = result;
    return DLO_OK;
}
