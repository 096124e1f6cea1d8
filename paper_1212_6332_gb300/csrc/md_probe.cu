// Fused multiply-add rate of the device, the denominator of the float64
// (pair pass, force pass) and float32 (mixed-precision passes) rooflines.
//
// Every resident thread runs kChains independent chains x <- x * a + b for
// a given number of steps; with kChains chains in flight per thread and the
// device full, the issue of the FMAs, not their latency, sets the time. The
// chains stay bounded (a < 1) and every one feeds the stored result, so the
// compiler keeps them all.
#include <cuda_runtime.h>

#include "md.h"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;
constexpr int kUnroll = 8;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(int64_t iters, T a, T b, T* __restrict__ out) {
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + 1 + c) * (T)1e-3;
    for (int64_t k = 0; k < iters; k += kUnroll) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int md_fma_probe(int precision, int64_t iters, double* flops, double* ms, int* n_sm, md_stream stream) {
    if (precision != 0 && precision != 1) return MD_ERR_ARG;  // 0: float64, 1: float32
    if (iters < 1 || !flops || !ms || !n_sm) return MD_ERR_ARG;
    iters = (iters + kUnroll - 1) / kUnroll * kUnroll;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess) {
        cudaGetLastError();
        return MD_ERR_CUDA;
    }
    const int blocks = sms * (per_sm / kProbeThreads);
    const size_t n_out = (size_t)blocks * kProbeThreads;
    void* out = nullptr;
    if (cudaMalloc(&out, n_out * 8) != cudaSuccess) {
        cudaGetLastError();
        return MD_ERR_NOMEM;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    if (precision == 0)
        k_fma_probe<double><<<blocks, kProbeThreads, 0, s>>>(iters, 0.999999, 1e-7, (double*)out);
    else
        k_fma_probe<float><<<blocks, kProbeThreads, 0, s>>>(iters, 0.999999f, 1e-7f, (float*)out);
    cudaEventRecord(e1, s);
    cudaError_t ce = cudaEventSynchronize(e1);
    float t = 0.0f;
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (ce != cudaSuccess || cudaGetLastError() != cudaSuccess) return MD_ERR_CUDA;
    *ms = t;
    *flops = 2.0 * kChains * (double)iters * (double)n_out / (t * 1e-3);
    *n_sm = sms;
    return MD_OK;
}
