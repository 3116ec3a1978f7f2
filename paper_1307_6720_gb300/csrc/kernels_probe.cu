// Arithmetic-rate probe: the sustained fused multiply-add throughput of the
// device in FP64 and in FP32.  The FP64 figure is the denominator of the
// roofline of the FP64 stencil kernels, which are bound by the FP64 pipe
// rather than by HBM on this part.
//
// Every thread runs eight independent multiply-add chains x <- x a + b (a
// just below 1, so the values stay bounded); the grid fills every SM with
// enough warps to cover the pipe latency.  One launch is timed with CUDA
// events after a warm-up launch of the same shape.
#include "mhs_internal.h"

namespace mhs {

namespace {

constexpr int PROBE_CHAINS = 8;

template <typename T>
__global__ void fma_probe_kernel(T* __restrict__ sink, int iters, T a, T b) {
    T x[PROBE_CHAINS];
#pragma unroll
    for (int q = 0; q < PROBE_CHAINS; ++q) x[q] = T(threadIdx.x) * T(1e-3) + T(q);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < PROBE_CHAINS; ++q) x[q] = fma(x[q], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int q = 0; q < PROBE_CHAINS; ++q) s += x[q];
    if (s == T(-1)) sink[0] = s;   // never true: keeps the chains live
}

template <typename T>
double probe(cudaStream_t st, int iters) {
    int dev = 0, sms = 0;
    MHS_CUDA(cudaGetDevice(&dev));
    MHS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8, threads = 256;
    cudaEvent_t e0, e1;
    MHS_CUDA(cudaEventCreate(&e0));
    MHS_CUDA(cudaEventCreate(&e1));
    float ms = 0.f;
    cudaError_t err = cudaSuccess;
    for (int rep = 0; rep < 2 && err == cudaSuccess; ++rep) {
        cudaEventRecord(e0, st);
        fma_probe_kernel<T><<<blocks, threads, 0, st>>>(nullptr, iters, T(0.999999), T(1e-6));
        count_launches(1);
        cudaEventRecord(e1, st);
        err = cudaEventSynchronize(e1);
        if (err == cudaSuccess) err = cudaGetLastError();
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    MHS_CUDA(err);
    const double flops = 2.0 * PROBE_CHAINS * double(iters) * double(blocks) * double(threads);
    return ms > 0.f ? flops / (double(ms) * 1e-3) : 0.0;
}

}  // namespace

double fma_rate(int precision, cudaStream_t st) {
    return precision == MHS_FP64 ? probe<double>(st, 2048) : probe<float>(st, 65536);
}

}  // namespace mhs
