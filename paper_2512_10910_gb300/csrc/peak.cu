// CUDA-core FMA throughput, the denominator of the ALU roofline of the FP64
// partition kernels and the FP32 cluster contractions.  Each thread runs
// eight independent FMA chains; the best of several event-timed runs counts.
#include <cuda_runtime.h>

#include "pne_internal.h"

namespace pne {

namespace {

template <typename T>
__global__ void __launch_bounds__(256) fma_chain_kernel(T *sink, int iters, T a, T b)
{
    T x0 = (T)threadIdx.x, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
    T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll 8
        for (int j = 0; j < 8; ++j) {
            x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
            x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
        }
    }
    const T s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
    if (s == (T)-12345.0) sink[0] = s;     // keeps the chains live
}

template <typename T>
pne_status time_fma(pne_ctx *ctx, cudaStream_t s, int iters, double *flops)
{
    DevBuf sink;
    pne_status st = dev_alloc(ctx, sink, 64, s);
    if (st) return st;
    const int blocks = ctx->n_sm * 8, threads = 256;
    cudaEvent_t a, b;
    cudaEventCreate(&a); cudaEventCreate(&b);
    double best = 0.0;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(a, s);
        fma_chain_kernel<T><<<blocks, threads, 0, s>>>((T *)sink.ptr, iters, (T)0.999999, (T)1e-7);
        cudaEventRecord(b, s);
        cudaError_t e = cudaEventSynchronize(b);
        if (e != cudaSuccess) { cudaEventDestroy(a); cudaEventDestroy(b); PNE_CUDA_TRY(ctx, e); }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        const double f = 2.0 * 64.0 * iters * (double)blocks * threads / (ms * 1e-3);
        if (rep > 0 && f > best) best = f;      // first run is a warm-up
    }
    cudaEventDestroy(a); cudaEventDestroy(b);
    dev_free(ctx, sink, s);
    *flops = best;
    return PNE_OK;
}

}  // namespace

pne_status launch_fma_peak(pne_ctx *ctx, int dtype, cudaStream_t s, double *flops)
{
    if (dtype == PNE_F64) return time_fma<double>(ctx, s, 2000, flops);
    return time_fma<float>(ctx, s, 40000, flops);
}

}  // namespace pne
