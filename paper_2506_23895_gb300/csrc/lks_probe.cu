// lks_fma_rate: the device's fused multiply-add throughput, measured.
//
// The plain FP64 path is bound by FP64 arithmetic rather than by memory, and the roofline it is
// reported against has to be a number measured on the device it runs on (vendor tables list
// FP64 rates that differ by an order of magnitude between parts of one family).  This kernel
// issues only FMAs: every thread runs kChains independent dependency chains of kIters FMAs each,
// enough independent work per warp to keep the FP64 (or FP32) pipes busy, and writes one sum so
// the chains are not removed.  The sink is a file-scope device array (no allocation).
#include <cstdio>

#include "lks.h"

namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;
constexpr int kThreads = 256;
constexpr int kMaxBlocks = 152 * 64;
static __device__ double g_probe_sink[kMaxBlocks];

template <class T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(T a, T b, int iters) {
    T x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    // one store per block keeps the chains alive; a and b make the value non-trivial
    if (s == (T)-1.2345e300 || threadIdx.x == 0) g_probe_sink[blockIdx.x] = (double)s;
}

template <class T>
cudaError_t time_fma(cudaStream_t st, int blocks, double* ms_out) {
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    // |a| < 1 keeps the chains bounded: x -> a x + b converges to b / (1 - a)
    const T a = (T)0.999, b = (T)1e-3;
    k_fma_chains<T><<<blocks, kThreads, 0, st>>>(a, b, kIters);   // warm-up
    e = cudaEventRecord(e0, st);
    for (int r = 0; r < 5 && e == cudaSuccess; ++r) {
        k_fma_chains<T><<<blocks, kThreads, 0, st>>>(a, b, kIters);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms_out = ms / 5.0;
    return e;
}

}  // namespace

extern "C" lks_status lks_fma_rate(int precision, void* stream, double* flops_per_s) {
    if (!flops_per_s || (precision != LKS_FP32 && precision != LKS_FP64)) return LKS_ERR_ARG;
    *flops_per_s = 0.0;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return LKS_ERR_CUDA;
    }
    // whole waves of 8 blocks of 256 threads per SM
    const int blocks = nsm * 8 > kMaxBlocks ? kMaxBlocks : nsm * 8;
    double ms = 0.0;
    const cudaError_t e = precision == LKS_FP64
                              ? time_fma<double>((cudaStream_t)stream, blocks, &ms)
                              : time_fma<float>((cudaStream_t)stream, blocks, &ms);
    if (e != cudaSuccess || ms <= 0.0) {
        cudaGetLastError();
        return LKS_ERR_CUDA;
    }
    const double fmas = (double)blocks * kThreads * kChains * kIters;
    *flops_per_s = 2.0 * fmas / (ms * 1e-3);
    return LKS_OK;
}
