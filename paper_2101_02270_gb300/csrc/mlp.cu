// Learned warm start: a small MLP that maps per-bus injections (P, Q) to an
// initial voltage guess (|V|, angle of the non-slack buses), trained on the
// solver's own solutions; Newton-Raphson always runs from its guess to the
// same tolerance.  All GEMMs (forward and backward) run on the tcgen05 tensor
// cores with BF16 operands and FP32 accumulation (gemm_tc.cuh); bias, GELU,
// loss, transposes and AdamW are plain CUDA kernels; master weights and
// optimiser state are FP32.
//   h1 = GELU(x W1^T + b1), h2 = GELU(h1 W2^T + b2), y = h2 W3^T + b3
// with W_l stored [out][in] (row-major), exact erf-GELU, loss = mean (y - t)^2
// on standardised inputs and targets.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <new>
#include <random>
#include <vector>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/nrpf.h"
#include "gemm_tc.cuh"
#include "handle.h"

namespace nrpf {
namespace {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.3989422804014327f * __expf(-0.5f * z * z);
}

// ---- GEMM epilogues ----
struct EpiF32 {  // C = acc
  float* C;
  int ldc;
  __device__ void operator()(int r, int c, float v) const { C[(int64_t)r * ldc + c] = v; }
};
struct EpiBiasGelu {  // Z = acc + b (FP32), H = GELU(Z) (BF16); padding columns -> 0
  const float* b;
  float* Z;
  bf16* H;
  int ld, nvalid;
  __device__ void operator()(int r, int c, float v) const {
    const float z = c < nvalid ? v + b[c] : 0.f;
    Z[(int64_t)r * ld + c] = z;
    H[(int64_t)r * ld + c] = __float2bfloat16(c < nvalid ? gelu_f(z) : 0.f);
  }
};
struct EpiBias {  // Y = acc + b
  const float* b;
  float* Y;
  int ld, nvalid;
  __device__ void operator()(int r, int c, float v) const {
    Y[(int64_t)r * ld + c] = c < nvalid ? v + b[c] : 0.f;
  }
};

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 2-D map of a row-major BF16 matrix [rows][K]: boxes of 64 (K) x 128 rows,
// 128-byte swizzle (the layout the UMMA descriptors expect)
bool make_tmap(CUtensorMap* m, const bf16* ptr, int rows, int K) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kGemmBK, (cuuint32_t)kGemmBM};
  const cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(ptr), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// variant: 0 = copy-then-MMA kernel, 1 = TMA pipeline (falls back to 0 when
// the tensor-map encoder is unavailable)
int g_gemm_variant = 1;

template <class Epi>
int gemm(const bf16* A, const bf16* B, int M, int N, int K, Epi epi, int* err, cudaStream_t st,
         int variant = -1) {
  if (M % kGemmBM || N % kGemmBN || K % kGemmBK || M <= 0 || N <= 0 || K <= 0) return NRPF_ERR_ARG;
  if (variant < 0) variant = g_gemm_variant;
  static bool configured[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !configured[dev]) {
    cudaFuncSetAttribute(k_gemm_tc<Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmSmem);
    cudaFuncSetAttribute(k_gemm_tma<Epi, CUtensorMap>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kGemmTmaSmem);
    if (dev >= 0 && dev < 64) configured[dev] = true;
  }
  CUtensorMap ta, tb;
  if (variant == 1 && make_tmap(&ta, A, M, K) && make_tmap(&tb, B, N, K)) {
    k_gemm_tma<Epi, CUtensorMap><<<dim3(N / kGemmBN, M / kGemmBM), kGemmThreads, kGemmTmaSmem, st>>>(ta, tb, M, N, K,
                                                                                                     epi, err);
  } else {
    k_gemm_tc<Epi><<<dim3(N / kGemmBN, M / kGemmBM), kGemmThreads, kGemmSmem, st>>>(A, B, M, N, K, epi, err);
  }
  return cudaGetLastError() == cudaSuccess ? NRPF_OK : NRPF_ERR_CUDA;
}

// ---- elementwise / layout kernels ----
// x (FP32 [B][nin]) -> standardised BF16 [Bp][nin_p], zero padding
__global__ void k_prep_x(const float* __restrict__ x, const float* __restrict__ mu, const float* __restrict__ sd,
                         bf16* __restrict__ xb, int B, int Bp, int nin, int nin_p) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)Bp * nin_p) return;
  const int r = (int)(i / nin_p), c = (int)(i % nin_p);
  float v = 0.f;
  if (r < B && c < nin) v = (x[(int64_t)r * nin + c] - mu[c]) / sd[c];
  xb[i] = __float2bfloat16(v);
}

// BF16 transpose [R][C] -> [C][R] through a 32 x 33 shared tile
__global__ void k_transpose_bf16(const bf16* __restrict__ in, bf16* __restrict__ out, int R, int C) {
  __shared__ bf16 t[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int r = r0 + j, c = c0 + threadIdx.x;
    t[j][threadIdx.x] = (r < R && c < C) ? in[(int64_t)r * C + c] : __float2bfloat16(0.f);
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int c = c0 + j, r = r0 + threadIdx.x;
    if (c < C && r < R) out[(int64_t)c * R + r] = t[threadIdx.x][j];
  }
}

// dY = 2 (Y - T_std) / (B * nout) in BF16 (padding rows/cols zero); loss partial sums
__global__ void k_loss_grad(const float* __restrict__ Y, const float* __restrict__ T, const float* __restrict__ mu,
                            const float* __restrict__ sd, bf16* __restrict__ dY, float* __restrict__ loss, int B,
                            int Bp, int nout, int nout_p) {
  __shared__ float red[256];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (i < (int64_t)Bp * nout_p) {
    const int r = (int)(i / nout_p), c = (int)(i % nout_p);
    float g = 0.f;
    if (r < B && c < nout) {
      const float t = (T[(int64_t)r * nout + c] - mu[c]) / sd[c];
      const float d = Y[i] - t;
      l = d * d;
      g = 2.f * d / ((float)B * (float)nout);
    }
    dY[i] = __float2bfloat16(g);
  }
  red[threadIdx.x] = l;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, red[0] / ((float)B * (float)nout));
}

// dZ = dH * GELU'(Z), BF16; rows >= B and columns >= nvalid -> 0
__global__ void k_gelu_back(const float* __restrict__ dH, const float* __restrict__ Z, bf16* __restrict__ dZ, int B,
                            int Bp, int ld, int nvalid) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)Bp * ld) return;
  const int r = (int)(i / ld), c = (int)(i % ld);
  dZ[i] = __float2bfloat16((r < B && c < nvalid) ? dH[i] * gelu_grad_f(Z[i]) : 0.f);
}

// column sums of a BF16 [Bp][ld] matrix into FP32 g[n] (bias gradients)
__global__ void k_colsum(const bf16* __restrict__ D, float* __restrict__ g, int Bp, int ld, int n) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  float s = 0.f;
  for (int r = 0; r < Bp; ++r) s += __bfloat162float(D[(int64_t)r * ld + c]);
  g[c] = s;
}

// AdamW on an FP32 tensor stored [rows][ld] (only the first cols columns are
// parameters); refreshes the padded BF16 copy
__global__ void k_adamw(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                        float* __restrict__ v, bf16* __restrict__ pb, int64_t n, int cols, int ld_b, float lr,
                        float b1, float b2, float eps, float wd, float c1, float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  float pi = p[i] * (1.f - lr * wd);
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  pi -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  p[i] = pi;
  if (pb) {
    const int64_t r = i / cols, c = i % cols;
    pb[r * ld_b + c] = __float2bfloat16(pi);
  }
}

// FP32 [rows][cols] -> BF16 [rows][ld] (padding untouched)
__global__ void k_to_bf16(const float* __restrict__ a, bf16* __restrict__ b, int64_t n, int cols, int ld) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  b[(i / cols) * ld + i % cols] = __float2bfloat16(a[i]);
}

// gradient of a weight from a padded FP32 GEMM result [rows][ldg] -> dense [rows][cols]
__global__ void k_compact(const float* __restrict__ gp, float* __restrict__ g, int64_t n, int cols, int ldg) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  g[i] = gp[(i / cols) * ldg + i % cols];
}

// y (standardised, FP32 [Bp][nout_p]) -> physical units FP32 [B][nout]
__global__ void k_unstd(const float* __restrict__ Y, const float* __restrict__ mu, const float* __restrict__ sd,
                        float* __restrict__ out, int B, int nout, int nout_p) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)B * nout) return;
  const int r = (int)(i / nout), c = (int)(i % nout);
  out[i] = Y[(int64_t)r * nout_p + c] * sd[c] + mu[c];
}

inline unsigned nb(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }
inline int rup(int x, int m) { return (x + m - 1) / m * m; }

}  // namespace
}  // namespace nrpf

using nrpf::bf16;

struct pf_mlp {
  int nin, nh1, nh2, nout, bmax;
  int nin_p, nout_p, bp;  // padded sizes
  int64_t step = 0;
  // parameters (FP32 master, dense [out][in]) and their BF16 padded copies
  float *W[3], *b[3], *mW[3], *vW[3], *mb[3], *vb[3], *gW[3], *gb[3];
  bf16 *Wb[3], *Wt[3];
  int fin[3], fout[3], fin_p[3], fout_p[3];
  // activations
  bf16 *xb, *xt, *h1, *h1t, *h2, *h2t, *dy, *dyt, *dz2, *dz2t, *dz1, *dz1t;
  float *z1, *z2, *y, *dh1, *dh2, *gtmp;
  float *mux, *sdx, *muy, *sdy;
  float* loss;
  int* err;
  std::vector<void*> allocs;
};

namespace {

int alloc_into(pf_mlp* p, size_t bytes, void** out) {
  void* d = nullptr;
  cudaError_t e = cudaMalloc(&d, std::max<size_t>(bytes, 256));
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? NRPF_ERR_NOMEM : NRPF_ERR_CUDA;
  p->allocs.push_back(d);
  cudaMemset(d, 0, std::max<size_t>(bytes, 256));
  *out = d;
  return NRPF_OK;
}

template <class T>
int al(pf_mlp* p, size_t count, T** out) {
  void* d = nullptr;
  int rc = alloc_into(p, count * sizeof(T), &d);
  *out = reinterpret_cast<T*>(d);
  return rc;
}

// refresh the BF16 copies (padded) and transposed copies of every weight
void refresh_bf16(pf_mlp* p, cudaStream_t st) {
  for (int l = 0; l < 3; ++l) {
    const int64_t n = (int64_t)p->fout[l] * p->fin[l];
    nrpf::k_to_bf16<<<nrpf::nb(n), 256, 0, st>>>(p->W[l], p->Wb[l], n, p->fin[l], p->fin_p[l]);
    nrpf::k_transpose_bf16<<<dim3(nrpf::nb(p->fin_p[l], 32), nrpf::nb(p->fout_p[l], 32)), dim3(32, 8), 0, st>>>(
        p->Wb[l], p->Wt[l], p->fout_p[l], p->fin_p[l]);
  }
}

int forward(pf_mlp* p, int B, const float* x, cudaStream_t st) {
  using namespace nrpf;
  const int Bp = rup(B, kGemmBM);
  k_prep_x<<<nb((int64_t)Bp * p->nin_p), 256, 0, st>>>(x, p->mux, p->sdx, p->xb, B, Bp, p->nin, p->nin_p);
  int rc;
  if ((rc = gemm(p->xb, p->Wb[0], Bp, p->fout_p[0], p->nin_p, EpiBiasGelu{p->b[0], p->z1, p->h1, p->fout_p[0], p->nh1},
                 p->err, st)))
    return rc;
  if ((rc = gemm(p->h1, p->Wb[1], Bp, p->fout_p[1], p->fin_p[1], EpiBiasGelu{p->b[1], p->z2, p->h2, p->fout_p[1], p->nh2},
                 p->err, st)))
    return rc;
  return gemm(p->h2, p->Wb[2], Bp, p->nout_p, p->fin_p[2], EpiBias{p->b[2], p->y, p->nout_p, p->nout}, p->err, st);
}

}  // namespace

extern "C" {

int pf_mlp_create(int nin, int nh1, int nh2, int nout, int bmax, uint64_t seed, pf_mlp** out) {
  if (!out || nin <= 0 || nh1 <= 0 || nh2 <= 0 || nout <= 0 || bmax <= 0) return NRPF_ERR_ARG;
  *out = nullptr;
  if (nh1 % nrpf::kGemmBN || nh2 % nrpf::kGemmBN) return NRPF_ERR_ARG;  // hidden widths: multiples of 128
  pf_mlp* p = new (std::nothrow) pf_mlp();
  if (!p) return NRPF_ERR_NOMEM;
  p->nin = nin; p->nh1 = nh1; p->nh2 = nh2; p->nout = nout; p->bmax = bmax;
  p->nin_p = nrpf::rup(nin, nrpf::kGemmBN);  // also the N of the first weight gradient
  p->nout_p = nrpf::rup(nout, nrpf::kGemmBN);
  p->bp = nrpf::rup(bmax, nrpf::kGemmBM);
  const int fin[3] = {nin, nh1, nh2}, fout[3] = {nh1, nh2, nout};
  const int fin_p[3] = {p->nin_p, nh1, nh2}, fout_p[3] = {nh1, nh2, p->nout_p};
  int rc = NRPF_OK;
  std::mt19937_64 rng(seed);
  for (int l = 0; l < 3 && !rc; ++l) {
    p->fin[l] = fin[l]; p->fout[l] = fout[l]; p->fin_p[l] = fin_p[l]; p->fout_p[l] = fout_p[l];
    const size_t nw = (size_t)fout[l] * fin[l];
    if ((rc = al(p, nw, &p->W[l])) || (rc = al(p, fout[l], &p->b[l])) || (rc = al(p, nw, &p->mW[l])) ||
        (rc = al(p, nw, &p->vW[l])) || (rc = al(p, fout[l], &p->mb[l])) || (rc = al(p, fout[l], &p->vb[l])) ||
        (rc = al(p, nw, &p->gW[l])) || (rc = al(p, fout[l], &p->gb[l])) ||
        (rc = al(p, (size_t)fout_p[l] * fin_p[l], &p->Wb[l])) || (rc = al(p, (size_t)fout_p[l] * fin_p[l], &p->Wt[l])))
      break;
    // uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases
    std::vector<float> w(nw);
    const double a = 1.0 / std::sqrt((double)fin[l]);
    std::uniform_real_distribution<double> U(-a, a);
    for (auto& x : w) x = (float)U(rng);
    cudaMemcpy(p->W[l], w.data(), nw * 4, cudaMemcpyHostToDevice);
  }
  const size_t bp = p->bp;
  if (!rc)
    if ((rc = al(p, bp * p->nin_p, &p->xb)) || (rc = al(p, bp * p->nin_p, &p->xt)) || (rc = al(p, bp * nh1, &p->h1)) ||
        (rc = al(p, bp * nh1, &p->h1t)) || (rc = al(p, bp * nh2, &p->h2)) || (rc = al(p, bp * nh2, &p->h2t)) ||
        (rc = al(p, bp * p->nout_p, &p->dy)) || (rc = al(p, bp * p->nout_p, &p->dyt)) ||
        (rc = al(p, bp * nh2, &p->dz2)) || (rc = al(p, bp * nh2, &p->dz2t)) || (rc = al(p, bp * nh1, &p->dz1)) ||
        (rc = al(p, bp * nh1, &p->dz1t)) || (rc = al(p, bp * nh1, &p->z1)) || (rc = al(p, bp * nh2, &p->z2)) ||
        (rc = al(p, bp * p->nout_p, &p->y)) || (rc = al(p, bp * nh1, &p->dh1)) || (rc = al(p, bp * nh2, &p->dh2)) ||
        (rc = al(p, (size_t)std::max({p->nout_p * nh2, nh2 * nh1, nh1 * p->nin_p}), &p->gtmp)) ||
        (rc = al(p, (size_t)nin, &p->mux)) || (rc = al(p, (size_t)nin, &p->sdx)) || (rc = al(p, (size_t)nout, &p->muy)) ||
        (rc = al(p, (size_t)nout, &p->sdy)) || (rc = al(p, 1, &p->loss)) || (rc = al(p, 1, &p->err))) {
    }
  if (rc) {
    pf_mlp_destroy(p);
    return rc;
  }
  // identity standardisation until pf_mlp_set_norm is called
  std::vector<float> zeros(std::max(nin, nout), 0.f), ones(std::max(nin, nout), 1.f);
  cudaMemcpy(p->mux, zeros.data(), nin * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(p->sdx, ones.data(), nin * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(p->muy, zeros.data(), nout * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(p->sdy, ones.data(), nout * 4, cudaMemcpyHostToDevice);
  refresh_bf16(p, nullptr);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    pf_mlp_destroy(p);
    return NRPF_ERR_CUDA;
  }
  *out = p;
  return NRPF_OK;
}

int pf_mlp_set_norm(pf_mlp* p, const float* mux, const float* sdx, const float* muy, const float* sdy) {
  if (!p || !mux || !sdx || !muy || !sdy) return NRPF_ERR_ARG;
  cudaMemcpy(p->mux, mux, p->nin * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(p->sdx, sdx, p->nin * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(p->muy, muy, p->nout * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(p->sdy, sdy, p->nout * 4, cudaMemcpyHostToDevice);
  return cudaGetLastError() == cudaSuccess ? NRPF_OK : NRPF_ERR_CUDA;
}

int pf_mlp_params(pf_mlp* p, int set, float* const* host) {
  if (!p || !host) return NRPF_ERR_ARG;
  cudaDeviceSynchronize();
  for (int l = 0; l < 3; ++l) {
    const size_t nw = (size_t)p->fout[l] * p->fin[l];
    if (!host[2 * l] || !host[2 * l + 1]) return NRPF_ERR_ARG;
    if (set) {
      cudaMemcpy(p->W[l], host[2 * l], nw * 4, cudaMemcpyHostToDevice);
      cudaMemcpy(p->b[l], host[2 * l + 1], p->fout[l] * 4, cudaMemcpyHostToDevice);
    } else {
      cudaMemcpy(host[2 * l], p->W[l], nw * 4, cudaMemcpyDeviceToHost);
      cudaMemcpy(host[2 * l + 1], p->b[l], p->fout[l] * 4, cudaMemcpyDeviceToHost);
    }
  }
  if (set) {
    refresh_bf16(p, nullptr);
    p->step = 0;
    for (int l = 0; l < 3; ++l) {
      cudaMemset(p->mW[l], 0, (size_t)p->fout[l] * p->fin[l] * 4);
      cudaMemset(p->vW[l], 0, (size_t)p->fout[l] * p->fin[l] * 4);
      cudaMemset(p->mb[l], 0, p->fout[l] * 4);
      cudaMemset(p->vb[l], 0, p->fout[l] * 4);
    }
  }
  return cudaDeviceSynchronize() == cudaSuccess ? NRPF_OK : NRPF_ERR_CUDA;
}

int pf_mlp_grads(pf_mlp* p, float* const* host) {
  if (!p || !host) return NRPF_ERR_ARG;
  cudaDeviceSynchronize();
  for (int l = 0; l < 3; ++l) {
    cudaMemcpy(host[2 * l], p->gW[l], (size_t)p->fout[l] * p->fin[l] * 4, cudaMemcpyDeviceToHost);
    cudaMemcpy(host[2 * l + 1], p->gb[l], p->fout[l] * 4, cudaMemcpyDeviceToHost);
  }
  return cudaGetLastError() == cudaSuccess ? NRPF_OK : NRPF_ERR_CUDA;
}

int pf_mlp_predict(pf_mlp* p, int B, const float* x, float* y, void* stream) {
  if (!p || B < 0 || B > p->bmax) return B > 0 && p && B > p->bmax ? NRPF_ERR_CAPACITY : NRPF_ERR_ARG;
  if (B == 0) return NRPF_OK;
  if (!x || !y) return NRPF_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int rc = forward(p, B, x, st);
  if (rc) return rc;
  nrpf::k_unstd<<<nrpf::nb((int64_t)B * p->nout), 256, 0, st>>>(p->y, p->muy, p->sdy, y, B, p->nout, p->nout_p);
  return cudaGetLastError() == cudaSuccess ? NRPF_OK : NRPF_ERR_CUDA;
}

int pf_mlp_train_step(pf_mlp* p, int B, const float* x, const float* t, float lr, float wd, int update,
                      float* loss_out, void* stream) {
  using namespace nrpf;
  if (!p || B <= 0 || B > p->bmax || !x || !t) return p && B > p->bmax ? NRPF_ERR_CAPACITY : NRPF_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int Bp = rup(B, kGemmBM);
  int rc = forward(p, B, x, st);
  if (rc) return rc;
  cudaMemsetAsync(p->loss, 0, 4, st);
  k_loss_grad<<<nb((int64_t)Bp * p->nout_p), 256, 0, st>>>(p->y, t, p->muy, p->sdy, p->dy, p->loss, B, Bp, p->nout,
                                                           p->nout_p);
  // transposes of the activations and output gradient ([Bp][w] -> [w][Bp])
  auto tr = [&](const bf16* a, bf16* at, int w) {
    k_transpose_bf16<<<dim3(nb(w, 32), nb(Bp, 32)), dim3(32, 8), 0, st>>>(a, at, Bp, w);
  };
  tr(p->dy, p->dyt, p->nout_p);
  tr(p->h2, p->h2t, p->nh2);
  tr(p->h1, p->h1t, p->nh1);
  tr(p->xb, p->xt, p->nin_p);
  // layer 3: dW3 = dY^T H2 ; dH2 = dY W3
  if ((rc = gemm(p->dyt, p->h2t, p->nout_p, p->nh2, Bp, EpiF32{p->gtmp, p->nh2}, p->err, st))) return rc;
  k_compact<<<nb((int64_t)p->nout * p->nh2), 256, 0, st>>>(p->gtmp, p->gW[2], (int64_t)p->nout * p->nh2, p->nh2, p->nh2);
  k_colsum<<<nb(p->nout), 256, 0, st>>>(p->dy, p->gb[2], Bp, p->nout_p, p->nout);
  if ((rc = gemm(p->dy, p->Wt[2], Bp, p->nh2, p->nout_p, EpiF32{p->dh2, p->nh2}, p->err, st))) return rc;
  k_gelu_back<<<nb((int64_t)Bp * p->nh2), 256, 0, st>>>(p->dh2, p->z2, p->dz2, B, Bp, p->nh2, p->nh2);
  tr(p->dz2, p->dz2t, p->nh2);
  // layer 2
  if ((rc = gemm(p->dz2t, p->h1t, p->nh2, p->nh1, Bp, EpiF32{p->gtmp, p->nh1}, p->err, st))) return rc;
  k_compact<<<nb((int64_t)p->nh2 * p->nh1), 256, 0, st>>>(p->gtmp, p->gW[1], (int64_t)p->nh2 * p->nh1, p->nh1, p->nh1);
  k_colsum<<<nb(p->nh2), 256, 0, st>>>(p->dz2, p->gb[1], Bp, p->nh2, p->nh2);
  if ((rc = gemm(p->dz2, p->Wt[1], Bp, p->nh1, p->nh2, EpiF32{p->dh1, p->nh1}, p->err, st))) return rc;
  k_gelu_back<<<nb((int64_t)Bp * p->nh1), 256, 0, st>>>(p->dh1, p->z1, p->dz1, B, Bp, p->nh1, p->nh1);
  tr(p->dz1, p->dz1t, p->nh1);
  // layer 1
  if ((rc = gemm(p->dz1t, p->xt, p->nh1, p->nin_p, Bp, EpiF32{p->gtmp, p->nin_p}, p->err, st))) return rc;
  k_compact<<<nb((int64_t)p->nh1 * p->nin), 256, 0, st>>>(p->gtmp, p->gW[0], (int64_t)p->nh1 * p->nin, p->nin, p->nin_p);
  k_colsum<<<nb(p->nh1), 256, 0, st>>>(p->dz1, p->gb[0], Bp, p->nh1, p->nh1);
  if (update) {
    p->step += 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - (float)std::pow(b1, (double)p->step), c2 = 1.f - (float)std::pow(b2, (double)p->step);
    for (int l = 0; l < 3; ++l) {
      const int64_t n = (int64_t)p->fout[l] * p->fin[l];
      k_adamw<<<nb(n), 256, 0, st>>>(p->W[l], p->gW[l], p->mW[l], p->vW[l], p->Wb[l], n, p->fin[l], p->fin_p[l], lr, b1,
                                     b2, eps, wd, c1, c2);
      k_adamw<<<nb(p->fout[l]), 256, 0, st>>>(p->b[l], p->gb[l], p->mb[l], p->vb[l], nullptr, p->fout[l], 1, 1, lr, b1,
                                              b2, eps, 0.f, c1, c2);
      k_transpose_bf16<<<dim3(nb(p->fin_p[l], 32), nb(p->fout_p[l], 32)), dim3(32, 8), 0, st>>>(
          p->Wb[l], p->Wt[l], p->fout_p[l], p->fin_p[l]);
    }
  }
  if (loss_out) cudaMemcpyAsync(loss_out, p->loss, 4, cudaMemcpyDeviceToDevice, st);
  return cudaGetLastError() == cudaSuccess ? NRPF_OK : NRPF_ERR_CUDA;
}

}  // extern "C"

namespace {
// per-column mean and standard deviation of a [B][n] FP32 matrix (FP64 sums)
__global__ void k_colstats(const float* __restrict__ X, int64_t B, int n, float* __restrict__ mu,
                           float* __restrict__ sd) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  double s = 0.0;
  for (int64_t r = 0; r < B; ++r) s += X[r * n + c];
  const double m = s / (double)B;
  double q = 0.0;
  for (int64_t r = 0; r < B; ++r) {
    const double d = X[r * n + c] - m;
    q += d * d;
  }
  const double v = q / (double)B;
  mu[c] = (float)m;
  sd[c] = v > 1e-24 ? (float)sqrt(v) : 1.0f;  // constant features keep unit scale
}
}  // namespace

extern "C" {

int pf_mlp_fit_norm(pf_mlp* p, int64_t B, const float* X, const float* T, void* stream) {
  if (!p || B <= 0 || !X || !T) return NRPF_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  k_colstats<<<nrpf::nb(p->nin), 256, 0, st>>>(X, B, p->nin, p->mux, p->sdx);
  k_colstats<<<nrpf::nb(p->nout), 256, 0, st>>>(T, B, p->nout, p->muy, p->sdy);
  return cudaGetLastError() == cudaSuccess ? NRPF_OK : NRPF_ERR_CUDA;
}

int pf_mlp_error(pf_mlp* p) {
  if (!p) return NRPF_ERR_ARG;
  int e = 0;
  cudaMemcpy(&e, p->err, 4, cudaMemcpyDeviceToHost);
  return e;
}

void pf_mlp_destroy(pf_mlp* p) {
  if (!p) return;
  cudaDeviceSynchronize();
  for (void* a : p->allocs) cudaFree(a);
  delete p;
}

// ---- warm-start glue between the solver's layouts and the network's ----
}  // extern "C"

namespace {
// features: X[b] = [P_0 .. P_{n-1}, Q_0 .. Q_{n-1}] from sbus [B, n] complex
__global__ void k_ws_features(int n, int B, const double2* __restrict__ sbus, float* __restrict__ X) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)B * n) return;
  const int64_t b = i / n;
  const int k = (int)(i % n);
  const double2 s = sbus[i];
  X[b * 2 * n + k] = (float)s.x;
  X[b * 2 * n + n + k] = (float)s.y;
}
// targets: T[b] = [|V| of non-slack buses, angles of non-slack buses] (ascending bus order)
__global__ void k_ws_targets(int n, int B, const int32_t* __restrict__ nsidx, const double2* __restrict__ V,
                             float* __restrict__ T, int nns) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)B * n) return;
  const int64_t b = i / n;
  const int k = (int)(i % n);
  const int q = nsidx[k];
  if (q < 0) return;
  const double2 v = V[i];
  T[b * 2 * nns + q] = (float)sqrt(v.x * v.x + v.y * v.y);
  T[b * 2 * nns + nns + q] = (float)atan2(v.y, v.x);
}
// V0 from a prediction: slack keeps v_flat, PV keeps |v_flat| with the
// predicted angle, PQ takes the predicted magnitude and angle
__global__ void k_ws_v0(int n, int B, const int32_t* __restrict__ nsidx, const int8_t* __restrict__ bt,
                        const float* __restrict__ Y, const double2* __restrict__ vflat, double2* __restrict__ v0,
                        int nns) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)B * n) return;
  const int64_t b = i / n;
  const int k = (int)(i % n);
  const double2 vf = vflat[i];
  const int q = nsidx[k];
  if (q < 0 || bt[k] == 3) {
    v0[i] = vf;
    return;
  }
  double mag = bt[k] == 2 ? sqrt(vf.x * vf.x + vf.y * vf.y) : (double)Y[b * 2 * nns + q];
  if (!(mag > 0.0) || !(mag < 10.0)) mag = sqrt(vf.x * vf.x + vf.y * vf.y);  // keep the guess sane
  double ang = (double)Y[b * 2 * nns + nns + q];
  if (!(fabs(ang) < 10.0)) ang = 0.0;
  double sn, cs;
  sincos(ang, &sn, &cs);
  v0[i] = make_double2(mag * cs, mag * sn);
}

// Screen of warm-started results: one warp per instance takes min |V|^2 over
// its buses; the instance is redone from flat start when it did not converge,
// or when some magnitude is below vmin (a low-voltage root of the power-flow
// equations, reached from a guess far from the operating point) or not finite.
__global__ void k_ws_screen(int n, int B, const double2* __restrict__ v, const uint8_t* __restrict__ status,
                            double vmin2, uint8_t* __restrict__ redo) {
  const int b = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (b >= B) return;
  const double2* vb = v + (size_t)b * n;
  double lo = INFINITY;
  bool finite = true;
  for (int k = lane; k < n; k += 32) {
    const double2 x = vb[k];
    const double m2 = x.x * x.x + x.y * x.y;
    finite = finite && isfinite(m2);
    lo = fmin(lo, m2);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
  finite = __all_sync(0xffffffffu, finite);
  if (lane == 0) redo[b] = (status[b] != 0 || !finite || lo < vmin2) ? 1 : 0;
}
}  // namespace

extern "C" {

int pf_warmstart_features(int n, int B, const double* sbus, float* X, void* stream) {
  if (n <= 0 || B < 0 || (B > 0 && (!sbus || !X))) return NRPF_ERR_ARG;
  if (B == 0) return NRPF_OK;
  k_ws_features<<<nrpf::nb((int64_t)B * n), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      n, B, reinterpret_cast<const double2*>(sbus), X);
  return cudaGetLastError() == cudaSuccess ? NRPF_OK : NRPF_ERR_CUDA;
}

int pf_warmstart_targets(int n, int B, const int32_t* nsidx, int nns, const double* v, float* T, void* stream) {
  if (n <= 0 || B < 0 || nns <= 0 || (B > 0 && (!nsidx || !v || !T))) return NRPF_ERR_ARG;
  if (B == 0) return NRPF_OK;
  k_ws_targets<<<nrpf::nb((int64_t)B * n), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      n, B, nsidx, reinterpret_cast<const double2*>(v), T, nns);
  return cudaGetLastError() == cudaSuccess ? NRPF_OK : NRPF_ERR_CUDA;
}

int pf_warmstart_v0(int n, int B, const int32_t* nsidx, const int8_t* bus_type, int nns, const float* Y,
                    const double* v_flat, double* v0, void* stream) {
  if (n <= 0 || B < 0 || nns <= 0 || (B > 0 && (!nsidx || !bus_type || !Y || !v_flat || !v0))) return NRPF_ERR_ARG;
  if (B == 0) return NRPF_OK;
  k_ws_v0<<<nrpf::nb((int64_t)B * n), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      n, B, nsidx, bus_type, Y, reinterpret_cast<const double2*>(v_flat), reinterpret_cast<double2*>(v0), nns);
  return cudaGetLastError() == cudaSuccess ? NRPF_OK : NRPF_ERR_CUDA;
}

int pf_warmstart_screen(int n, int B, const double* v, const uint8_t* status, double vmin, uint8_t* redo,
                        void* stream) {
  if (n <= 0 || B < 0 || !(vmin >= 0.0) || (B > 0 && (!v || !status || !redo))) return NRPF_ERR_ARG;
  if (B == 0) return NRPF_OK;
  k_ws_screen<<<(B + 7) / 8, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      n, B, reinterpret_cast<const double2*>(v), status, vmin * vmin, redo);
  return cudaGetLastError() == cudaSuccess ? NRPF_OK : NRPF_ERR_CUDA;
}

// Standalone tensor-core GEMM: C[M,N] (FP32) = A[M,K] B[N,K]^T (BF16, row-major).
int pf_gemm_bf16(const void* A, const void* B, float* C, int M, int N, int K, int variant, int* err,
                 void* stream) {
  if (!A || !B || !C || !err || variant < 0 || variant > 1) return NRPF_ERR_ARG;
  return nrpf::gemm(reinterpret_cast<const bf16*>(A), reinterpret_cast<const bf16*>(B), M, N, K, nrpf::EpiF32{C, N},
                    err, reinterpret_cast<cudaStream_t>(stream), variant);
}

int pf_gemm_set_variant(int variant) {
  if (variant < 0 || variant > 1) return NRPF_ERR_ARG;
  nrpf::g_gemm_variant = variant;
  return NRPF_OK;
}

}  // extern "C"
