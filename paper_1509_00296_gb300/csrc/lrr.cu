// Low-rank representation (Table 6, Type A) by the inexact ALM, on the GPU:
//
//     min ||L||_* + lam ||S||_{2,1}   s.t.   O = Z L + S   (dictionary Z = O, d x n)
//
// with the splitting J = L (the nuclear norm on J, one SVT per iteration).  Each iteration:
//     J  = FRSVT_{1/mu}(L + Y2 / mu)                         (Alg. 1 through an frsvt handle)
//     L  = C (Z^T (O - S + Y1 / mu) + J - Y2 / mu),  C = (I + Z^T Z)^{-1}
//     S  = colshrink_{lam/mu}(O - Z L + Y1 / mu)             (column i scaled by max(0, 1 - t / ||q_i||))
//     Y1 = Y1 + mu (O - Z L - S),  Y2 = Y2 + mu (L - J),  mu = min(rho mu, mu_max)
// C is formed once (frsvt_lrr_init) by Newton-Schulz iterations X <- X (2 I - A X) on
// A = I + Z^T Z from X0 = I / (1 + ||Z||_F^2) (every eigenvalue of A X0 lies in (0, 1]), in FP32
// GEMMs; each L solve then takes one step of iterative refinement, L = L0 + C (T - A L0), so
// that the FP32 inverse's error enters only squared.  All state lives on the device; mu is
// host bookkeeping (its sequence does not depend on the data).
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <new>
#include <string>

#include <cuda_runtime.h>

#include "../../include/frsvt.h"

namespace {

// ---------------------------------------------------------------- FP32 GEMM (CUDA cores)
// C = alpha op(A) op(B) + beta C0 (C0 may be C itself or null), row-major, op(X) = X or X^T.
// 64 x 64 output tiles, K in steps of 16 staged in shared memory, 4 x 4 outputs per thread.
constexpr int kGT = 64, kGK = 16, kGThr = 256;

template <bool TA, bool TB>
__global__ void __launch_bounds__(kGThr) k_lrr_gemm(int M, int N, int K, float alpha, const float* __restrict__ A,
                                                    int64_t lda, const float* __restrict__ B, int64_t ldb, float beta,
                                                    const float* C0, int64_t ldc0, float* C, int64_t ldc) {
  __shared__ float As[kGK][kGT + 4], Bs[kGK][kGT + 4];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int i0 = blockIdx.y * kGT, j0 = blockIdx.x * kGT;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += kGK) {
    for (int e = threadIdx.x; e < kGT * kGK; e += kGThr) {
      // A tile: element (i, k) of op(A); B tile: element (k, j) of op(B); consecutive threads take
      // consecutive addresses of the stored matrix
      int i, k;
      if (TA) { i = e % kGT; k = e / kGT; } else { k = e % kGK; i = e / kGK; }
      const int gi = i0 + i, gk = k0 + k;
      As[k][i] = (gi < M && gk < K) ? (TA ? A[static_cast<int64_t>(gk) * lda + gi] : A[static_cast<int64_t>(gi) * lda + gk])
                                    : 0.f;
      int j, kb;
      if (TB) { kb = e % kGK; j = e / kGK; } else { j = e % kGT; kb = e / kGT; }
      const int gj = j0 + j, gkb = k0 + kb;
      Bs[kb][j] = (gj < N && gkb < K) ? (TB ? B[static_cast<int64_t>(gj) * ldb + gkb] : B[static_cast<int64_t>(gkb) * ldb + gj])
                                      : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kGK; ++k) {
      const float4 a = *reinterpret_cast<const float4*>(&As[k][4 * ty]);
      const float4 b = *reinterpret_cast<const float4*>(&Bs[k][4 * tx]);
      const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int gi = i0 + 4 * ty + r;
    if (gi >= M) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int gj = j0 + 4 * tx + c;
      if (gj >= N) continue;
      float v = alpha * acc[r][c];
      if (C0 != nullptr) v = fmaf(beta, C0[static_cast<int64_t>(gi) * ldc0 + gj], v);
      C[static_cast<int64_t>(gi) * ldc + gj] = v;
    }
  }
}

cudaError_t gemm(bool ta, bool tb, int M, int N, int K, float alpha, const float* A, int64_t lda, const float* B,
                 int64_t ldb, float beta, const float* C0, int64_t ldc0, float* C, int64_t ldc, cudaStream_t st) {
  if (M == 0 || N == 0) return cudaSuccess;
  const dim3 grid((N + kGT - 1) / kGT, (M + kGT - 1) / kGT);
  if (!ta && !tb) k_lrr_gemm<false, false><<<grid, kGThr, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C0, ldc0, C, ldc);
  else if (ta && !tb) k_lrr_gemm<true, false><<<grid, kGThr, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C0, ldc0, C, ldc);
  else if (!ta && tb) k_lrr_gemm<false, true><<<grid, kGThr, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C0, ldc0, C, ldc);
  else k_lrr_gemm<true, true><<<grid, kGThr, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C0, ldc0, C, ldc);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- elementwise steps
// Z = a X + b Y over an m x n block (ld shared by the three).
__global__ void k_lrr_axpby(int64_t m, int64_t n, int64_t ld, float a, const float* __restrict__ X, float b,
                            const float* __restrict__ Y, float* __restrict__ Z) {
  const int64_t total = m * n;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = e / n, j = e % n;
    Z[i * ld + j] = a * X[i * ld + j] + b * Y[i * ld + j];
  }
}

// E = O - S + Y1 / mu (d x n).
__global__ void k_lrr_resid(int64_t d, int64_t n, const float* __restrict__ O, int64_t ldo, const float* __restrict__ S,
                            const float* __restrict__ Y1, int64_t ld, float inv_mu, float* __restrict__ E) {
  const int64_t total = d * n;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = e / n, j = e % n;
    E[i * ld + j] = O[i * ldo + j] - S[i * ld + j] + inv_mu * Y1[i * ld + j];
  }
}

__device__ __forceinline__ void atomic_max_nonneg(float* p, float v) {
  atomicMax(reinterpret_cast<unsigned int*>(p), __float_as_uint(v));   // order of non-negative floats = of their bits
}

// S step and Y1 step, one CTA per 32 columns: Q = O - ZL + Y1 / mu, S = colshrink_t(Q) with
// t = lam / mu, R1 = O - ZL - S, Y1 += mu R1; err[0] = max(err[0], max |R1|).
constexpr int kCSW = 32, kCSR = 8;
__global__ void __launch_bounds__(kCSW * kCSR) k_lrr_colshrink(int64_t d, int64_t n, const float* __restrict__ O,
                                                               int64_t ldo, const float* __restrict__ ZL,
                                                               float* __restrict__ S, float* __restrict__ Y1,
                                                               int64_t ld, float mu, float inv_mu, float t,
                                                               float* __restrict__ err) {
  __shared__ float part[kCSR][kCSW];
  __shared__ float wmax[kCSR];
  const int lane = threadIdx.x % kCSW, ry = threadIdx.x / kCSW;
  const int64_t j = static_cast<int64_t>(blockIdx.x) * kCSW + lane;
  float ss = 0.f;
  if (j < n)
    for (int64_t i = ry; i < d; i += kCSR) {
      const float q = O[i * ldo + j] - ZL[i * ld + j] + inv_mu * Y1[i * ld + j];
      ss = fmaf(q, q, ss);
    }
  part[ry][lane] = ss;
  __syncthreads();
  if (ry == 0) {
    float tot = 0.f;
    for (int r = 0; r < kCSR; ++r) tot += part[r][lane];
    part[0][lane] = tot;
  }
  __syncthreads();
  const float nrm = sqrtf(part[0][lane]);
  const float scale = nrm > t ? 1.f - t / nrm : 0.f;
  float mx = 0.f;
  if (j < n)
    for (int64_t i = ry; i < d; i += kCSR) {
      const float o = O[i * ldo + j], zl = ZL[i * ld + j], y = Y1[i * ld + j];
      const float s = scale * (o - zl + inv_mu * y);
      const float r1 = o - zl - s;
      S[i * ld + j] = s;
      Y1[i * ld + j] = fmaf(mu, r1, y);
      mx = fmaxf(mx, fabsf(r1));
    }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) wmax[ry] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m2 = 0.f;
    for (int r = 0; r < kCSR; ++r) m2 = fmaxf(m2, wmax[r]);
    atomic_max_nonneg(err, m2);
  }
}

// Y2 step: R2 = L - J, Y2 += mu R2; err[1] = max(err[1], max |R2|).
__global__ void k_lrr_dual2(int64_t n, int64_t ld, const float* __restrict__ L, const float* __restrict__ J,
                            float* __restrict__ Y2, float mu, float* __restrict__ err) {
  const int64_t total = n * n;
  float mx = 0.f;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = e / n, j = e % n;
    const float r2 = L[i * ld + j] - J[i * ld + j];
    Y2[i * ld + j] = fmaf(mu, r2, Y2[i * ld + j]);
    mx = fmaxf(mx, fabsf(r2));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(err + 1, mx);
}

// A = I + G (n x n; G = Z^T Z), and trace-free scale: s[0] = 1 + ||Z||_F^2 = 1 + trace(G) read off
// the diagonal (one CTA); X0 = I / s[0] is written by k_lrr_ns_init.
__global__ void k_lrr_shift(int64_t n, int64_t ld, float* __restrict__ A, float* __restrict__ s) {
  __shared__ float red[256];
  float tr = 0.f;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    tr += A[i * ld + i];
    A[i * ld + i] += 1.f;
  }
  red[threadIdx.x] = tr;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) s[0] = 1.f + red[0];
}

__global__ void k_lrr_ns_init(int64_t n, int64_t ld, const float* __restrict__ s, float* __restrict__ X) {
  const float v = 1.f / s[0];
  const int64_t total = n * n;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = e / n, j = e % n;
    X[i * ld + j] = (i == j) ? v : 0.f;
  }
}

int ew_grid(int64_t total) {
  int64_t g = (total + 255) / 256;
  if (g > 2048) g = 2048;
  return static_cast<int>(g < 1 ? 1 : g);
}

}  // namespace

struct frsvt_lrr {
  int64_t d_max = 0, n_max = 0, ldn = 0;
  int32_t l = 0;
  cudaStream_t stream = nullptr;
  frsvt_handle* svt = nullptr;
  // state and work: n x n (ldn) and d x n (ldn)
  float *L = nullptr, *J = nullptr, *Y2 = nullptr, *M = nullptr, *T = nullptr, *L0 = nullptr, *C = nullptr,
        *P = nullptr;
  float *S = nullptr, *Y1 = nullptr, *E = nullptr, *ZL = nullptr;
  float* err = nullptr;            // device: max |R1|, max |R2|, scale
  const float* O = nullptr;
  int64_t d = 0, n = 0, ldo = 0;
  double lam = 0.0, mu = 0.0, rho = 0.0, mu_max = 0.0;
  int iter = 0;
  int ns_iters = 0;
  std::string err_msg;
};

namespace {

frsvt_status lfail(frsvt_lrr* h, frsvt_status s, const std::string& msg) {
  if (h) h->err_msg = msg;
  return s;
}

#define LRR_CK(call)                                                                              \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) return lfail(h, FRSVT_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
  } while (0)

void lrr_free(frsvt_lrr* h) {
  float* bufs[] = {h->L, h->J, h->Y2, h->M, h->T, h->L0, h->C, h->P, h->S, h->Y1, h->E, h->ZL, h->err};
  for (float* b : bufs)
    if (b) cudaFree(b);
  if (h->svt) frsvt_destroy(h->svt);
}

}  // namespace

extern "C" {

frsvt_status frsvt_lrr_create(frsvt_lrr** out, int64_t d_max, int64_t n_max, int32_t l, int32_t q, uint64_t seed,
                              int32_t range_prop, void* stream) {
  if (out == nullptr) return FRSVT_ERR_INVALID_ARG;
  *out = nullptr;
  if (d_max < 1 || n_max < 2 || n_max > 16384 || d_max > (int64_t(1) << 24) || l < 1 || l > 128 || l > n_max ||
      q < 0 || q > 64)
    return FRSVT_ERR_INVALID_ARG;
  frsvt_lrr* h = new (std::nothrow) frsvt_lrr();
  if (h == nullptr) return FRSVT_ERR_ALLOC;
  h->d_max = d_max;
  h->n_max = n_max;
  h->ldn = (n_max + 3) / 4 * 4;
  h->l = l;
  h->stream = static_cast<cudaStream_t>(stream);
  frsvt_config cfg = {};
  cfg.m_max = n_max;
  cfg.n_max = n_max;
  cfg.l_max = l;
  cfg.q = q;
  cfg.range_prop = range_prop ? 1 : 0;
  cfg.precision = FRSVT_PREC_FP32;
  cfg.seed = seed;
  frsvt_status s = frsvt_create(&h->svt, &cfg, stream);
  if (s != FRSVT_OK) {
    h->svt = nullptr;
    delete h;
    return s;
  }
  const size_t nn = sizeof(float) * static_cast<size_t>(n_max) * h->ldn;
  const size_t dn = sizeof(float) * static_cast<size_t>(d_max) * h->ldn;
  bool ok = true;
  auto alloc = [&](float** p, size_t bytes) {
    if (ok && cudaMalloc(reinterpret_cast<void**>(p), bytes) != cudaSuccess) ok = false;
  };
  alloc(&h->L, nn);
  alloc(&h->J, nn);
  alloc(&h->Y2, nn);
  alloc(&h->M, nn);
  alloc(&h->T, nn);
  alloc(&h->L0, nn);
  alloc(&h->C, nn);
  alloc(&h->P, nn);
  alloc(&h->S, dn);
  alloc(&h->Y1, dn);
  alloc(&h->E, dn);
  alloc(&h->ZL, dn);
  alloc(&h->err, 4 * sizeof(float));
  if (!ok) {
    lrr_free(h);
    delete h;
    return FRSVT_ERR_ALLOC;
  }
  *out = h;
  return FRSVT_OK;
}

frsvt_status frsvt_lrr_destroy(frsvt_lrr* h) {
  if (h == nullptr) return FRSVT_ERR_INVALID_ARG;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  lrr_free(h);
  delete h;
  return FRSVT_OK;
}

frsvt_status frsvt_lrr_init(frsvt_lrr* h, const float* O, int64_t d, int64_t n, int64_t ldo, double lam, double mu0,
                            double rho, double mu_max) {
  if (h == nullptr || O == nullptr) return FRSVT_ERR_INVALID_ARG;
  if (d < 1 || n < 2 || d > h->d_max || n > h->n_max || ldo < n)
    return lfail(h, FRSVT_ERR_INVALID_ARG, "need 1 <= d <= d_max, 2 <= n <= n_max, ldo >= n");
  if (!(lam > 0.0) || !(mu0 > 0.0) || !(rho >= 1.0) || !(mu_max >= mu0) || !std::isfinite(mu_max))
    return lfail(h, FRSVT_ERR_INVALID_ARG, "need lam > 0, mu0 > 0, rho >= 1, mu0 <= mu_max < inf");
  h->O = O;
  h->d = d;
  h->n = n;
  h->ldo = ldo;
  h->lam = lam;
  h->mu = mu0;
  h->rho = rho;
  h->mu_max = mu_max;
  h->iter = 0;
  cudaStream_t st = h->stream;
  const int64_t ld = h->ldn;
  LRR_CK(cudaMemsetAsync(h->L, 0, sizeof(float) * n * ld, st));
  LRR_CK(cudaMemsetAsync(h->J, 0, sizeof(float) * n * ld, st));
  LRR_CK(cudaMemsetAsync(h->Y2, 0, sizeof(float) * n * ld, st));
  LRR_CK(cudaMemsetAsync(h->S, 0, sizeof(float) * d * ld, st));
  LRR_CK(cudaMemsetAsync(h->Y1, 0, sizeof(float) * d * ld, st));
  // A = I + Z^T Z into P, then Newton-Schulz for C = A^{-1}: X <- 2 X - X (A X)
  LRR_CK(gemm(true, false, static_cast<int>(n), static_cast<int>(n), static_cast<int>(d), 1.f, O, ldo, O, ldo, 0.f,
              nullptr, 0, h->P, ld, st));
  k_lrr_shift<<<1, 256, 0, st>>>(n, ld, h->P, h->err + 2);
  LRR_CK(cudaGetLastError());
  float scale = 0.f;
  LRR_CK(cudaMemcpyAsync(&scale, h->err + 2, sizeof(float), cudaMemcpyDeviceToHost, st));
  LRR_CK(cudaStreamSynchronize(st));
  if (!std::isfinite(scale)) return lfail(h, FRSVT_ERR_NONFINITE, "||O||_F is not finite");
  // every eigenvalue of A X0 lies in [1 / scale, 1]: the error I - A X squares each step, so
  // log2(scale) steps reach 1/2 and five more reach FP32 rounding
  h->ns_iters = static_cast<int>(std::ceil(std::log2(static_cast<double>(scale)))) + 6;
  k_lrr_ns_init<<<ew_grid(n * n), 256, 0, st>>>(n, ld, h->err + 2, h->C);
  LRR_CK(cudaGetLastError());
  for (int k = 0; k < h->ns_iters; ++k) {
    LRR_CK(gemm(false, false, static_cast<int>(n), static_cast<int>(n), static_cast<int>(n), 1.f, h->P, ld, h->C, ld,
                0.f, nullptr, 0, h->T, ld, st));                                               // T = A X
    LRR_CK(gemm(false, false, static_cast<int>(n), static_cast<int>(n), static_cast<int>(n), -1.f, h->C, ld, h->T, ld,
                2.f, h->C, ld, h->L0, ld, st));                                                // L0 = 2 X - X T
    float* t = h->C;
    h->C = h->L0;
    h->L0 = t;
  }
  return frsvt_reset(h->svt, 0) == FRSVT_OK ? FRSVT_OK : lfail(h, FRSVT_ERR_CUDA, "frsvt_reset failed");
}

frsvt_status frsvt_lrr_step(frsvt_lrr* h, double* err) {
  if (h == nullptr) return FRSVT_ERR_INVALID_ARG;
  if (h->O == nullptr) return lfail(h, FRSVT_ERR_INVALID_ARG, "frsvt_lrr_init first");
  cudaStream_t st = h->stream;
  const int64_t d = h->d, n = h->n, ld = h->ldn;
  const int ni = static_cast<int>(n), di = static_cast<int>(d);
  const float mu = static_cast<float>(h->mu), inv_mu = static_cast<float>(1.0 / h->mu);
  LRR_CK(cudaMemsetAsync(h->err, 0, 2 * sizeof(float), st));
  // J = FRSVT_{1/mu}(L + Y2 / mu)
  k_lrr_axpby<<<ew_grid(n * n), 256, 0, st>>>(n, n, ld, 1.f, h->L, inv_mu, h->Y2, h->M);
  LRR_CK(cudaGetLastError());
  frsvt_status s = frsvt_svt(h->svt, h->M, n, n, ld, inv_mu, h->l, h->J, ld);
  if (s != FRSVT_OK) return lfail(h, s, std::string("J step: ") + frsvt_last_error(h->svt));
  // T = Z^T (O - S + Y1 / mu) + J - Y2 / mu
  k_lrr_resid<<<ew_grid(d * n), 256, 0, st>>>(d, n, h->O, h->ldo, h->S, h->Y1, ld, inv_mu, h->E);
  k_lrr_axpby<<<ew_grid(n * n), 256, 0, st>>>(n, n, ld, 1.f, h->J, -inv_mu, h->Y2, h->T);
  LRR_CK(cudaGetLastError());
  LRR_CK(gemm(true, false, ni, ni, di, 1.f, h->O, h->ldo, h->E, ld, 1.f, h->T, ld, h->T, ld, st));
  // L0 = C T; refinement L = L0 + C (T - L0 - Z^T (Z L0))
  LRR_CK(gemm(false, false, ni, ni, ni, 1.f, h->C, ld, h->T, ld, 0.f, nullptr, 0, h->L0, ld, st));
  LRR_CK(gemm(false, false, di, ni, ni, 1.f, h->O, h->ldo, h->L0, ld, 0.f, nullptr, 0, h->ZL, ld, st));
  k_lrr_axpby<<<ew_grid(n * n), 256, 0, st>>>(n, n, ld, 1.f, h->T, -1.f, h->L0, h->P);
  LRR_CK(cudaGetLastError());
  LRR_CK(gemm(true, false, ni, ni, di, -1.f, h->O, h->ldo, h->ZL, ld, 1.f, h->P, ld, h->P, ld, st));
  LRR_CK(gemm(false, false, ni, ni, ni, 1.f, h->C, ld, h->P, ld, 1.f, h->L0, ld, h->L, ld, st));
  // S, Y1 (with Z L) and Y2
  LRR_CK(gemm(false, false, di, ni, ni, 1.f, h->O, h->ldo, h->L, ld, 0.f, nullptr, 0, h->ZL, ld, st));
  k_lrr_colshrink<<<static_cast<int>((n + kCSW - 1) / kCSW), kCSW * kCSR, 0, st>>>(
      d, n, h->O, h->ldo, h->ZL, h->S, h->Y1, ld, mu, inv_mu, static_cast<float>(h->lam / h->mu), h->err);
  k_lrr_dual2<<<ew_grid(n * n), 256, 0, st>>>(n, ld, h->L, h->J, h->Y2, mu, h->err);
  LRR_CK(cudaGetLastError());
  h->mu = std::fmin(h->rho * h->mu, h->mu_max);
  h->iter += 1;
  if (err != nullptr) {
    float e2[2];
    LRR_CK(cudaMemcpyAsync(e2, h->err, sizeof(e2), cudaMemcpyDeviceToHost, st));
    LRR_CK(cudaStreamSynchronize(st));
    *err = static_cast<double>(std::fmax(e2[0], e2[1]));
  }
  return FRSVT_OK;
}

frsvt_status frsvt_lrr_get(frsvt_lrr* h, float* L, int64_t ldl, float* S, int64_t lds, double* mu, int32_t* iters) {
  if (h == nullptr) return FRSVT_ERR_INVALID_ARG;
  cudaStream_t st = h->stream;
  if (L != nullptr) {
    if (ldl < h->n) return lfail(h, FRSVT_ERR_INVALID_ARG, "ldl < n");
    LRR_CK(cudaMemcpy2DAsync(L, sizeof(float) * ldl, h->L, sizeof(float) * h->ldn, sizeof(float) * h->n, h->n,
                             cudaMemcpyDeviceToDevice, st));
  }
  if (S != nullptr) {
    if (lds < h->n) return lfail(h, FRSVT_ERR_INVALID_ARG, "lds < n");
    LRR_CK(cudaMemcpy2DAsync(S, sizeof(float) * lds, h->S, sizeof(float) * h->ldn, sizeof(float) * h->n, h->d,
                             cudaMemcpyDeviceToDevice, st));
  }
  if (mu != nullptr) *mu = h->mu;
  if (iters != nullptr) *iters = h->iter;
  return FRSVT_OK;
}

const char* frsvt_lrr_last_error(const frsvt_lrr* h) { return h == nullptr ? "null handle" : h->err_msg.c_str(); }

}  // extern "C"
