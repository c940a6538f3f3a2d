// Throughput probes of the arithmetic pipes (diagnostics, not part of the method): the
// measured peaks against which the roofline fractions of the float32-pipe and float64-pipe
// kernels are stated.  Each thread runs eight independent chains of fused multiply-adds, so
// the pipe, not the dependency latency, bounds the rate; the grid holds eight blocks of 256
// threads per SM.
#include "efe_internal.h"

namespace efe {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(T* __restrict__ out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) x[u] = (T)(threadIdx.x + 1) * (T)1e-3 + (T)u;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = fma(x[u], a, b);
  }
  T s = 0;
#pragma unroll
  for (int u = 0; u < 8; ++u) s += x[u];
  out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the chains alive
}

template <typename T>
cudaError_t time_probe(int n_sm, int iters, T a, T b, double* tflops) {
  const int blocks = 8 * n_sm, threads = 256;
  T* out = nullptr;
  EFE_CUDA_TRY(cudaMalloc(&out, sizeof(T) * (size_t)blocks * threads));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fma_probe<T><<<blocks, threads>>>(out, iters / 16, a, b);   // warm-up (clocks, instruction cache)
  cudaEventRecord(e0);
  k_fma_probe<T><<<blocks, threads>>>(out, iters, a, b);
  cudaEventRecord(e1);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return e;
  *tflops = 2.0 * 8.0 * (double)iters * blocks * threads / (ms * 1e-3) / 1e12;
  return cudaSuccess;
}

}  // namespace
}  // namespace efe

extern "C" efe_status efe_pipe_peaks(double* fp32_tflops_host, double* fp64_tflops_host) {
  if (!fp32_tflops_host || !fp64_tflops_host) return EFE_ERR_ARG;
  int dev = 0, n_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return EFE_ERR_CUDA;
  if (efe::time_probe<float>(n_sm, 1 << 20, 1.0000001f, 1e-7f, fp32_tflops_host) != cudaSuccess) return EFE_ERR_CUDA;
  if (efe::time_probe<double>(n_sm, 1 << 14, 1.0000000001, 1e-12, fp64_tflops_host) != cudaSuccess) return EFE_ERR_CUDA;
  return EFE_OK;
}
