// Mismatch evaluation that allocates no device memory (pf_stage_mismatch_noalloc).
//
// Some callers cannot call cudaMalloc when they need the mismatch of a batch:
// code whose device memory is owned entirely by another allocator (a
// framework's caching pool that has reserved the GPU), or a real-time loop
// that must not take cudaMalloc's latency and implicit device-wide
// synchronisation.  This entry point keeps its only scratch - the per-instance
// running maxima of the cross-block max|F| reduction and an arrival counter -
// in a fixed, file-scope device array, so a call allocates nothing.  The plan
// (created earlier by pf_plan_create) supplies the read-only Ybus and index
// arrays; the caller passes inputs and outputs.
#include <cfloat>
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/nrpf.h"
#include "handle.h"

namespace {

constexpr int kThreads = 256;

// [0, NRPF_NOALLOC_MAX_BATCH): float64 bit patterns of max|F| per instance;
// [NRPF_NOALLOC_MAX_BATCH]: arrival counter of the blocks of one call.
// Zero-initialised at module load; every call clears the part it uses first.
static __device__ __align__(256) unsigned long long g_noalloc_scratch[NRPF_NOALLOC_MAX_BATCH + 32];

// One thread per (instance, bus) on the caller's [B, n] layout: nodal power
// (Eq. 1, rectangular form), mismatch rows written at their position in
// A = P J P^T, max |F| reduced per instance in shared memory, then across blocks
// with atomicMax on the scratch; the last block to arrive writes norm[].
__global__ void __launch_bounds__(kThreads) k_mismatch_noalloc(nrpf::DevPlan P, int B,
                                                               const double2* __restrict__ sbus,
                                                               const double2* __restrict__ v,
                                                               double* __restrict__ F,
                                                               double* __restrict__ norm,
                                                               unsigned long long* __restrict__ scratch) {
  __shared__ unsigned long long smax[kThreads + 2];
  __shared__ int last;
  const int64_t n = P.n;
  const int64_t t0 = (int64_t)blockIdx.x * kThreads;
  const int64_t t = t0 + threadIdx.x;
  const int64_t b0 = t0 / n;
  smax[threadIdx.x] = 0ull;
  if (threadIdx.x < 2) smax[kThreads + threadIdx.x] = 0ull;
  __syncthreads();
  if (t < (int64_t)B * n) {
    const int64_t b = t / n;
    const int i = (int)(t - b * n);
    const int bt = P.bus_type[i];
    if (bt != 3) {
      const double2* vb = v + b * n;
      const double2 vi = vb[i];
      double Ir = 0.0, Ii = 0.0;
      for (int d = P.rowptr[i]; d < P.rowptr[i + 1]; ++d) {
        const double2 vk = vb[P.colidx[d]];
        const double G = P.yre[d], Bv = P.yim[d];
        Ir += G * vk.x - Bv * vk.y;
        Ii += G * vk.y + Bv * vk.x;
      }
      const double2 s = sbus[b * n + i];
      const double dP = vi.x * Ir + vi.y * Ii - s.x;
      double a = fabs(dP);
      F[b * P.m + P.rhs_p[i]] = dP;
      if (bt == 1) {
        const double dQ = vi.y * Ir - vi.x * Ii - s.y;
        F[b * P.m + P.rhs_q[i]] = dQ;
        const double q = fabs(dQ);
        a = (q > a || q != q) ? q : a;
      }
      if (!(a <= DBL_MAX)) a = __longlong_as_double(0x7ff0000000000000ll);  // NaN -> +inf
      atomicMax(&smax[b - b0], (unsigned long long)__double_as_longlong(a));
    }
  }
  __syncthreads();
  // this block covers instances b0 .. b0 + span - 1
  const int64_t tl = t0 + kThreads < (int64_t)B * n ? t0 + kThreads : (int64_t)B * n;
  const int span = (int)((tl - 1) / n - b0 + 1);
  if (threadIdx.x < span) atomicMax(&scratch[b0 + threadIdx.x], smax[threadIdx.x]);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned long long ticket = atomicAdd(&scratch[NRPF_NOALLOC_MAX_BATCH], 1ull);
    last = ticket == (unsigned long long)(gridDim.x - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    const volatile unsigned long long* vs = scratch;  // written by other blocks' atomics
    for (int b = threadIdx.x; b < B; b += kThreads) norm[b] = __longlong_as_double((long long)vs[b]);
  }
}

std::mutex g_mu;
void* g_addr[256] = {};  // per-device address of g_noalloc_scratch

}  // namespace

extern "C" int pf_stage_mismatch_noalloc(const pf_plan* p, int B, const double* sbus, const double* v,
                                         double* F, double* norm, void* stream) {
  if (!p || p->host_only || B < 0) return NRPF_ERR_ARG;
  if (B > NRPF_NOALLOC_MAX_BATCH) return NRPF_ERR_CAPACITY;
  if (B == 0) return NRPF_OK;
  if (!sbus || !v || !F || !norm) return NRPF_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return NRPF_ERR_CUDA;
  void* scratch = nullptr;
  {
    // Set-up, once per device, with that device current: the host-side name of
    // the array is not a device address, so ask the runtime for it.
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      void* a = nullptr;
      if (cudaGetSymbolAddress(&a, g_noalloc_scratch) != cudaSuccess || !a) return NRPF_ERR_CUDA;
      g_addr[dev] = a;
    }
    scratch = g_addr[dev];
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  unsigned long long* s = reinterpret_cast<unsigned long long*>(scratch);
  // the running maxima of this call's instances and the arrival counter start at zero
  if (cudaMemsetAsync(s, 0, sizeof(unsigned long long) * (size_t)B, st) != cudaSuccess) return NRPF_ERR_CUDA;
  if (cudaMemsetAsync(s + NRPF_NOALLOC_MAX_BATCH, 0, sizeof(unsigned long long), st) != cudaSuccess)
    return NRPF_ERR_CUDA;
  const int64_t total = (int64_t)B * p->hp.n;
  const unsigned blocks = (unsigned)((total + kThreads - 1) / kThreads);
  k_mismatch_noalloc<<<blocks, kThreads, 0, st>>>(p->dp, B, reinterpret_cast<const double2*>(sbus),
                                                  reinterpret_cast<const double2*>(v), F, norm, s);
  return cudaGetLastError() == cudaSuccess ? NRPF_OK : NRPF_ERR_CUDA;
}
