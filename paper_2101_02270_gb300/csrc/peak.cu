// FMA-throughput measurement used as the arithmetic roofline of the solver's
// kernels: every thread runs eight independent fused multiply-add chains.
#include <cuda_runtime.h>

#include "../../include/nrpf.h"

namespace {

template <typename T>
__global__ void k_fma_chains(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = (T)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int time_chains(int iters, double* tflops, cudaStream_t st) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return NRPF_ERR_CUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 8, threads = 256;
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * blocks * threads) != cudaSuccess) return NRPF_ERR_NOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fma_chains<T><<<blocks, threads, 0, st>>>(out, iters / 10, (T)0.999, (T)0.001);
  float best = 1e30f;
  for (int r = 0; r < 3; ++r) {
    cudaEventRecord(e0, st);
    k_fma_chains<T><<<blocks, threads, 0, st>>>(out, iters, (T)0.999, (T)0.001);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (cudaGetLastError() != cudaSuccess) return NRPF_ERR_CUDA;
  *tflops = 2.0 * 8.0 * (double)iters * blocks * threads / (best * 1e-3) / 1e12;
  return NRPF_OK;
}

}  // namespace

extern "C" int pf_fma_peak(double* fp64_tflops, double* fp32_tflops, void* stream) {
  if (!fp64_tflops || !fp32_tflops) return NRPF_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int rc = time_chains<double>(4000, fp64_tflops, st);
  if (rc) return rc;
  return time_chains<float>(100000, fp32_tflops, st);
}
