// Branch power flows after a solve (pf_branch_flows): the power entering each
// branch at its two ends, from the solved bus voltages.
#include <cuda_runtime.h>

#include "../../include/nrpf.h"

namespace {

// One thread per (instance, branch), branches fastest, so the flow writes are
// coalesced; the two voltage reads per thread are gathers from the instance's
// row.  pi model: ys = 1/(r + jx), half the charging b at each end;
// I_f = ys (V_f - V_t) + j b/2 V_f, S_f = V_f conj(I_f), and symmetrically at t.
__global__ void k_branch_flows(int n, int nbr, const int32_t* __restrict__ f, const int32_t* __restrict__ t,
                               const double* __restrict__ r, const double* __restrict__ x,
                               const double* __restrict__ b, int B, const uint8_t* __restrict__ in_service,
                               const double2* __restrict__ v, double2* __restrict__ sf, double2* __restrict__ st) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)B * nbr) return;
  const int inst = (int)(q / nbr), e = (int)(q % nbr);
  if (in_service && !in_service[q]) {
    sf[q] = make_double2(0.0, 0.0);
    st[q] = make_double2(0.0, 0.0);
    return;
  }
  const double2 vf = v[(size_t)inst * n + f[e]], vt = v[(size_t)inst * n + t[e]];
  const double den = r[e] * r[e] + x[e] * x[e];
  const double gs = r[e] / den, bs = -x[e] / den, bh = 0.5 * b[e];
  const double dr = vf.x - vt.x, di = vf.y - vt.y;
  // I_f = ys (V_f - V_t) + j bh V_f
  const double ifr = gs * dr - bs * di - bh * vf.y;
  const double ifi = gs * di + bs * dr + bh * vf.x;
  // I_t = -ys (V_f - V_t) + j bh V_t
  const double itr = -(gs * dr - bs * di) - bh * vt.y;
  const double iti = -(gs * di + bs * dr) + bh * vt.x;
  // S = V conj(I)
  sf[q] = make_double2(vf.x * ifr + vf.y * ifi, vf.y * ifr - vf.x * ifi);
  st[q] = make_double2(vt.x * itr + vt.y * iti, vt.y * itr - vt.x * iti);
}

}  // namespace

extern "C" int pf_branch_flows(int n, int nbr, const int32_t* f, const int32_t* t, const double* r,
                               const double* x, const double* b, int B, const uint8_t* in_service,
                               const double* v, double* sf, double* st, void* stream) {
  if (n <= 0 || nbr < 0 || B < 0) return NRPF_ERR_ARG;
  if ((long long)B * nbr == 0) return NRPF_OK;
  if (!f || !t || !r || !x || !b || !v || !sf || !st) return NRPF_ERR_ARG;
  const long long total = (long long)B * nbr;
  const int threads = 256;
  const long long blocks = (total + threads - 1) / threads;
  if (blocks > 0x7fffffffLL) return NRPF_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  k_branch_flows<<<(unsigned)blocks, threads, 0, s>>>(n, nbr, f, t, r, x, b, B, in_service,
                                                      reinterpret_cast<const double2*>(v),
                                                      reinterpret_cast<double2*>(sf),
                                                      reinterpret_cast<double2*>(st));
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? NRPF_OK : NRPF_ERR_CUDA;
}
