// Fused multiply-add rate of the device, the denominator of the float64
// (pair pass, force pass) and float32 (mixed-precision passes) rooflines.
//
// Every resident thread runs CH independent chains x <- x * a + b for a
// given number of steps; with the device full and CH chains in flight per
// thread, the issue of the FMAs, not their latency, sets the time. The
// chains stay bounded (a < 1) and every one feeds the stored result, so the
// compiler keeps them all. The call runs 4, 8 and 16 chains per thread and
// keeps the fastest, so that no one operand pattern sets the figure.
#include <cuda_runtime.h>

#include "md.h"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kUnroll = 8;

template <typename T, int CH>
__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(int64_t iters, T a, T b, T* __restrict__ out) {
    T x[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = (T)(threadIdx.x + 1 + c) * (T)1e-3;
    for (int64_t k = 0; k < iters; k += kUnroll) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < CH; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < CH; ++c) s += x[c];
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// One timed launch of CH chains per thread for `iters` steps (8 x iters
// FMAs per thread at CH = 8, so every variant does the same work): ms.
template <typename T, int CH>
static cudaError_t probe_once(int blocks, int64_t iters, T a, T b, void* out, cudaStream_t s, float* ms) {
    const int64_t steps = (iters * 8 / CH + kUnroll - 1) / kUnroll * kUnroll;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    k_fma_probe<T, CH><<<blocks, kProbeThreads, 0, s>>>(steps, a, b, (T*)out);
    cudaEventRecord(e1, s);
    cudaError_t ce = cudaEventSynchronize(e1);
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ce;
}

template <typename T>
static cudaError_t probe_best(int blocks, int64_t iters, T a, T b, void* out, cudaStream_t s, float* ms) {
    float t[3] = {0.f, 0.f, 0.f};
    cudaError_t ce = probe_once<T, 4>(blocks, iters, a, b, out, s, &t[0]);
    if (ce == cudaSuccess) ce = probe_once<T, 8>(blocks, iters, a, b, out, s, &t[1]);
    if (ce == cudaSuccess) ce = probe_once<T, 16>(blocks, iters, a, b, out, s, &t[2]);
    *ms = t[0];
    for (int k = 1; k < 3; ++k)
        if (t[k] < *ms) *ms = t[k];
    return ce;
}

}  // namespace

extern "C" int md_fma_probe(int precision, int64_t iters, double* flops, double* ms, int* n_sm, md_stream stream) {
    if (precision != 0 && precision != 1) return MD_ERR_ARG;  // 0: float64, 1: float32
    if (iters < 1 || !flops || !ms || !n_sm) return MD_ERR_ARG;
    iters = (iters + 15) / 16 * 16;  // every variant then runs whole unrolled steps
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
    float t = 0.0f;
    cudaError_t ce = precision == 0 ? probe_best<double>(blocks, iters, 0.999999, 1e-7, out, s, &t)
                                    : probe_best<float>(blocks, iters, 0.999999f, 1e-7f, out, s, &t);
    cudaFree(out);
    if (ce != cudaSuccess || cudaGetLastError() != cudaSuccess || !(t > 0.0f)) return MD_ERR_CUDA;
    *ms = t;
    // every variant runs 8 x iters FMAs per thread
    *flops = 2.0 * 8.0 * (double)iters * (double)n_out / (t * 1e-3);
    *n_sm = sms;
    return MD_OK;
}
