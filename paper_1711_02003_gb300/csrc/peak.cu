// peak.cu -- FMA-throughput microbenchmark (lbcg_fma_peak).
//
// The FP64 step is bound by GB300's FP64 arithmetic rate, not by HBM; its roofline needs
// that rate as measured on the device the library runs on.  The same kernel in FP32
// gives the plain-ALU bound of the FP32 paths.  Not part of the method (the paper has
// no counterpart): a measurement utility of the library.
#include <string>

#include "lbcg_internal.h"

namespace lbcg {
namespace {

constexpr int kChains = 8;  // independent multiply-add chains per thread (latency hiding)

template <typename T>
__global__ void __launch_bounds__(256) k_fma(T* __restrict__ out, int iters, T a, T b)
{
    T acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = T(threadIdx.x + c) * T(1e-3);
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc[c] = fma(acc[c], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
cudaError_t run(cudaStream_t st, int iters, double* gflops)
{
    int sms = 0, dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int blocks = sms * 8, threads = 256;
    T* out = nullptr;
    e = cudaMalloc(&out, sizeof(T) * blocks * threads);
    if (e != cudaSuccess) return e;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const T a = T(0.999999), b = T(1e-6);
    k_fma<T><<<blocks, threads, 0, st>>>(out, iters / 8, a, b);  // warm-up
    cudaEventRecord(e0, st);
    k_fma<T><<<blocks, threads, 0, st>>>(out, iters, a, b);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) *gflops = 2.0 * kChains * (double)iters * blocks * threads / (ms * 1e-3) / 1e9;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    return e;
}

}  // namespace

int fma_peak(int precision, void* stream, double* gflops, std::string& err)
{
    if (!gflops) {
        err = "null output";
        return LBCG_ERR_ARG;
    }
    const cudaStream_t st = (cudaStream_t)stream;
    const cudaError_t e = precision == LBCG_FP64 ? run<double>(st, 1 << 12, gflops) : run<float>(st, 1 << 15, gflops);
    if (e != cudaSuccess) {
        err = std::string("fma peak: ") + cudaGetErrorString(e);
        return LBCG_ERR_CUDA;
    }
    return LBCG_OK;
}

}  // namespace lbcg
