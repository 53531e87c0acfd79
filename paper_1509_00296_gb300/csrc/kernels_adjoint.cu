// Adjoint (backward pass) of the FRSVT map with a fixed Omega, Alg. 1 differentiated step by
// step, and the forward that records what it needs.
//
// Tall orientation (A is m x n, m >= n, the basis Q on the column side, as in the forward path):
//   Y_0 = A^T Omega,  (Q_0, R_0) = CholeskyQR2(Y_0)
//   Z_i = A Q_{i-1},  Y_i = A^T Z_i,  (Q_i, R_i) = CholeskyQR2(Y_i)      i = 1..q
//   Z = A Q_q = B^T,  B = U diag(sigma) V_B^T (l x l SVD through the double-float Gram of Z),
//   X = V_B diag(f) (Q U)^T,  f_i = max(sigma_i - tau, 0).
// The forward keeps Q_i, R_i, U, sigma and V_B; the backward recomputes Omega and the Z_i.
// Given Xbar (m x n), with P = Xbar Q and Ubar = U^T P^T V_B:
//   Bbar^T = V_B (K - D Ubar)^T U^T + P U D U^T     (SVT adjoint on B, D = diag(f / sigma),
//            K_ij = Gs_ij sym(Ubar)_ij + Gk_ij skew(Ubar)_ij, K_ii = f'_i Ubar_ii,
//            Gs = divided differences of f, Gk_ij = (f_i + f_j) / (sigma_i + sigma_j))
//   taubar = -sum_{sigma_i > tau} Ubar_ii
//   Qbar_q = Xbar^T V_B diag(f) U^T + A^T Bbar^T,  Abar += Bbar^T Q^T
//   QR adjoint (Y = Q R, Rbar = 0): Ybar = (Qbar - Q copyltu(Qbar^T Q)) R^{-T}
//   power step i: Abar += Z_i Ybar_i^T + Zbar_i Q_{i-1}^T with Zbar_i = A Ybar_i,
//                 Qbar_{i-1} = A^T Zbar_i
//   sketch: Abar += Omega Ybar_0^T.
// The rank updates of Abar are collected as column blocks of L (m x K) and R (n x K) and
// written in one pass, Abar = L R^T.
// Kernels: tall-skinny products on CUDA cores (row pass C = M S, column pass C = M^T T with a
// fixed-order split-K reduction), the rank-K write, and single-CTA kernels for the small dense
// steps (CholeskyQR2, the l x l core, the SVT adjoint, the QR adjoint).
#include <cstdint>

#include "common.cuh"
#include "small_dense.cuh"
#include "state.cuh"

namespace frsvt {

namespace {

constexpr int kAdThr = 256;
constexpr int kAdGacc = 1024;

// ---------------------------------------------------------------- large passes
// C[i][coff + k] = beta C[i][coff + k] + sum_j M[i][j] S[j][k]   (C row stride ldc)
template <int LP>
__global__ void __launch_bounds__(kAdThr) k_ad_rows(const float* __restrict__ M, int64_t ldm, int64_t m, int n,
                                                   const float* __restrict__ S, float* __restrict__ C, int ldc,
                                                   int coff, float beta) {
  __shared__ float Ms[64][33];
  __shared__ __align__(16) float Ss[32][LP];
  constexpr int OPT = LP / 4;                        // outputs per thread
  const int t = threadIdx.x, r = t / 4, g = t % 4;
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * 64;
  float acc[OPT];
#pragma unroll
  for (int u = 0; u < OPT; ++u) acc[u] = 0.f;
  for (int j0 = 0; j0 < n; j0 += 32) {
    for (int e = t; e < 64 * 32; e += kAdThr) {
      const int rr = e / 32, jj = e % 32;
      Ms[rr][jj] = (r0 + rr < m && j0 + jj < n) ? M[(r0 + rr) * ldm + j0 + jj] : 0.f;
    }
    for (int e = t; e < 32 * LP; e += kAdThr) {
      const int jj = e / LP, k = e % LP;
      Ss[jj][k] = (j0 + jj < n) ? S[static_cast<int64_t>(j0 + jj) * LP + k] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int jj = 0; jj < 32; ++jj) {
      const float a = Ms[r][jj];
#pragma unroll
      for (int u = 0; u < OPT; ++u) acc[u] = fmaf(a, Ss[jj][g * OPT + u], acc[u]);
    }
    __syncthreads();
  }
  const int64_t row = r0 + r;
  if (row < m) {
    float* c = C + row * ldc + coff + g * OPT;
#pragma unroll
    for (int u = 0; u < OPT; ++u) c[u] = (beta == 0.f) ? acc[u] : fmaf(beta, c[u], acc[u]);
  }
}

// part[split][j][k] = sum_{i in split} M[i][j] T[i][k]   (64-column tiles x row splits), the
// products added exactly in double-float: the QR adjoint that consumes A^T T removes a large
// in-span part of it, and the FP32 rounding of long sums would dominate what is left.
template <int LP>
__global__ void __launch_bounds__(kAdThr) k_ad_cols(const float* __restrict__ M, int64_t ldm, int64_t m, int n,
                                                   const float* __restrict__ T, int ldt, int64_t rps,
                                                   double* __restrict__ part) {
  __shared__ float Ms[32][65];
  __shared__ __align__(16) float Ts[32][LP];
  constexpr int OPT = LP / 4;
  const int t = threadIdx.x, c = t % 64, g = t / 64;
  const int c0 = blockIdx.x * 64;
  const int64_t i0 = static_cast<int64_t>(blockIdx.y) * rps;
  const int64_t i1 = imin64(m, i0 + rps);
  df64 acc[OPT];
#pragma unroll
  for (int u = 0; u < OPT; ++u) acc[u] = df64{0.f, 0.f};
  for (int64_t ib = i0; ib < i1; ib += 32) {
    for (int e = t; e < 32 * 64; e += kAdThr) {
      const int ii = e / 64, cc = e % 64;
      Ms[ii][cc] = (ib + ii < i1 && c0 + cc < n) ? M[(ib + ii) * ldm + c0 + cc] : 0.f;
    }
    for (int e = t; e < 32 * LP; e += kAdThr) {
      const int ii = e / LP, k = e % LP;
      Ts[ii][k] = (ib + ii < i1) ? T[(ib + ii) * ldt + k] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int ii = 0; ii < 32; ++ii) {
      const float a = Ms[ii][c];
#pragma unroll
      for (int u = 0; u < OPT; ++u) df64_add_prod(acc[u], a, Ts[ii][g * OPT + u]);
    }
    __syncthreads();
  }
  if (c0 + c < n) {
    double* p = part + (static_cast<int64_t>(blockIdx.y) * n + c0 + c) * LP + g * OPT;
#pragma unroll
    for (int u = 0; u < OPT; ++u) p[u] = df64_value(acc[u]);
  }
}

// out[e] = beta out[e] + sum_s part[s][e], summed in split order (deterministic)
template <typename TO>
__global__ void k_ad_reduce(const double* __restrict__ part, int nsplit, int64_t count, TO* __restrict__ out,
                            int ldo, int LP, int coff, float beta) {
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= count) return;
  double s = 0.0;
  for (int sp = 0; sp < nsplit; ++sp) s += part[static_cast<int64_t>(sp) * count + e];
  const int64_t j = e / LP;
  const int k = static_cast<int>(e % LP);
  TO* o = out + j * ldo + coff + k;
  *o = (beta == 0.f) ? static_cast<TO>(s) : static_cast<TO>(static_cast<double>(beta) * static_cast<double>(*o) + s);
}

// A = beta A + L R^T   (L: m x K, R: n x K, row strides ldl / ldr), 64 x 64 tiles
__global__ void __launch_bounds__(kAdThr) k_ad_rank(float* __restrict__ A, int64_t lda, int64_t m, int n,
                                                    const float* __restrict__ L, int ldl,
                                                    const float* __restrict__ R, int ldr, int K, float beta) {
  __shared__ float Ls[32][65];
  __shared__ float Rs[32][65];
  const int t = threadIdx.x, ty = t / 16, tx = t % 16;
  const int64_t r0 = static_cast<int64_t>(blockIdx.y) * 64;
  const int c0 = blockIdx.x * 64;
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
  for (int k0 = 0; k0 < K; k0 += 32) {
    for (int e = t; e < 64 * 32; e += kAdThr) {
      const int rr = e / 32, kk = e % 32;
      Ls[kk][rr] = (r0 + rr < m && k0 + kk < K) ? L[(r0 + rr) * ldl + k0 + kk] : 0.f;
      Rs[kk][rr] = (c0 + rr < n && k0 + kk < K) ? R[static_cast<int64_t>(c0 + rr) * ldr + k0 + kk] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < 32; ++kk) {
      float lv[4], rv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) lv[a] = Ls[kk][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) rv[b] = Rs[kk][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(lv[a], rv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t row = r0 + ty + 16 * a;
    if (row >= m) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int col = c0 + tx + 16 * b;
      if (col >= n) continue;
      float* p = A + row * lda + col;
      *p = (beta == 0.f) ? acc[a][b] : fmaf(beta, *p, acc[a][b]);
    }
  }
}

// Omega[:m, :LP] of the (seed, stream) Philox stream, columns >= l zero (row stride ldo, offset coff)
template <int LP>
__global__ void k_ad_omega(float* __restrict__ out, int ldo, int coff, int64_t m, int l, uint64_t seed,
                           uint64_t stream) {
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= m * (LP / 4)) return;
  const int64_t i = e / (LP / 4);
  const int k4 = static_cast<int>(e % (LP / 4));
  const float4 g = gaussian4(seed, static_cast<uint64_t>(i), static_cast<uint64_t>(k4), stream, 0ull);
  const float v[4] = {g.x, g.y, g.z, g.w};
#pragma unroll
  for (int u = 0; u < 4; ++u) out[i * ldo + coff + 4 * k4 + u] = (4 * k4 + u < l) ? v[u] : 0.f;
}

// ---------------------------------------------------------------- small dense steps (one CTA)
// (Q, R) = CholeskyQR2(Y): Y n x LP (columns >= l zero), R LP x LP upper (R = R2 R1).  The second
// pass runs in double (exact double-float Gram of the FP32 Q_1, double-float Cholesky, double
// forward substitution), so Qd (double) is orthonormal to ~1e-14; Q is its FP32 rounding.  The
// QR adjoint needs that: it removes from Qbar an in-span part many orders larger than what
// remains, and an orthogonality error of Q of 1e-8 already shows in the gradient.
template <int LP>
__global__ void __launch_bounds__(kAdThr) k_ad_cholqr2(const float* __restrict__ Y, int n, int l,
                                                      double rank_tol, float* __restrict__ Q,
                                                      double* __restrict__ Qd, float* __restrict__ R,
                                                      DevState* dst) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ float R1[LP * LP];
  __shared__ double R2[LP * LP];
  SmallWs<LP> w = carve_small_ws<LP>(dsm, kAdGacc);
  const int tid = threadIdx.x;
  for (int e = tid; e < n * LP; e += kAdThr) w.W[e] = Y[e];
  __syncthreads();
  int dropped = 0;
  // pass 1: Q_1 = Y R_1^{-1} in FP32
  block_inner<LP>(w.W, n, 0, 0, l, l, true, w.G, w.gacc, w.gacc_n);
  block_cholesky<LP>(w, l, rank_tol);
  block_trsm_rows<LP>(w, w.W, n, 0, l);
  for (int c = 0; c < l; ++c) dropped |= w.iv[c];
  for (int e = tid; e < LP * LP; e += kAdThr) R1[e] = w.Rf32[e];
  __syncthreads();
  // pass 2 in double
  block_inner<LP>(w.W, n, 0, 0, l, l, true, w.G, w.gacc, w.gacc_n);
  block_cholesky<LP>(w, l, rank_tol);
  for (int c = 0; c < l; ++c) dropped |= w.iv[c];
  const df64* Rd = reinterpret_cast<const df64*>(w.R);
  for (int e = tid; e < LP * LP; e += kAdThr)
    R2[e] = static_cast<double>(Rd[e].hi) + static_cast<double>(Rd[e].lo);
  __syncthreads();
  for (int i = tid; i < n; i += kAdThr) {
    double x[LP];
#pragma unroll
    for (int b = 0; b < LP; ++b) {
      double v = 0.0;
      if (b < l && w.rinv[b] != 0.f) {
        v = static_cast<double>(w.W[i * LP + b]);
#pragma unroll
        for (int a = 0; a < b; ++a) v = fma(-x[a], R2[a * LP + b], v);
        v /= R2[b * LP + b];
      }
      x[b] = v;
    }
#pragma unroll
    for (int b = 0; b < LP; ++b) {
      Qd[static_cast<int64_t>(i) * LP + b] = x[b];
      Q[static_cast<int64_t>(i) * LP + b] = static_cast<float>(x[b]);
    }
  }
  for (int e = tid; e < LP * LP; e += kAdThr) {       // R = R2 R1 (both upper triangular)
    const int a = e / LP, b = e % LP;
    double acc = 0.0;
    for (int k = a; k <= b; ++k) acc = fma(R2[a * LP + k], static_cast<double>(R1[k * LP + b]), acc);
    R[e] = (a <= b) ? static_cast<float>(acc) : 0.f;
  }
  if (tid == 0 && dropped) dst->status |= kDevRankDeficient;
}

// l x l core from Z (m x LP): U (LP x LP, column b = left singular vector b of B), sigma,
// S1 = U diag(1 / sigma) (for V_B = Z S1) and S2 = U diag(f) (for the reconstruction factor).
template <int LP>
__global__ void __launch_bounds__(kAdThr) k_ad_core(const float* __restrict__ Z, int64_t m, int l, float tau,
                                                   double rank_tol, int max_sweeps, float* __restrict__ U,
                                                   float* __restrict__ sig, float* __restrict__ S1,
                                                   float* __restrict__ S2, DevState* dst) {
  extern __shared__ __align__(16) unsigned char dsm[];
  SmallWs<LP> w = carve_small_ws<LP>(dsm, kAdGacc);
  const int tid = threadIdx.x;
  for (int e = tid; e < LP * LP; e += kAdThr) w.G[e] = df64{0.f, 0.f};
  __syncthreads();
  block_inner<LP>(Z, m, 0, 0, l, l, true, w.G, w.gacc, w.gacc_n);
  const int sweeps = core_svd_block<LP>(w, l, rank_tol, max_sweeps);
  const float* s = w.vec;
  for (int e = tid; e < LP * LP; e += kAdThr) {
    const int a = e / LP, b = e % LP;
    const float u = w.U[e];
    U[e] = u;
    S1[e] = (s[b] > 0.f) ? u / s[b] : 0.f;
    S2[e] = u * fmaxf(s[b] - tau, 0.f);
  }
  if (tid < LP) sig[tid] = s[tid];
  if (tid == 0 && sweeps >= max_sweeps) dst->status |= kDevNotConverged;
}

// SVT adjoint on B from W1 = V_B^T P (LP x LP): C1 = (K - D Ubar)^T U^T, C2 = U D U^T,
// C3 = diag(f) U^T and taubar (see the file comment).
template <int LP>
__global__ void __launch_bounds__(kAdThr) k_ad_svt_adjoint(const float* __restrict__ W1, const float* __restrict__ U,
                                                          const float* __restrict__ sig, int l, float tau,
                                                          float* __restrict__ C1, float* __restrict__ C2,
                                                          float* __restrict__ C3, float* __restrict__ taubar) {
  __shared__ float Us[LP][LP], Ub[LP][LP], Km[LP][LP], s[LP], f[LP], fp[LP], d[LP];
  const int tid = threadIdx.x;
  for (int e = tid; e < LP * LP; e += kAdThr) Us[e / LP][e % LP] = U[e];
  if (tid < LP) {
    const float sv = (tid < l) ? sig[tid] : 0.f;
    s[tid] = sv;
    f[tid] = fmaxf(sv - tau, 0.f);
    fp[tid] = (sv > tau) ? 1.f : 0.f;
    d[tid] = (sv > 0.f) ? fmaxf(sv - tau, 0.f) / sv : 0.f;
  }
  __syncthreads();
  for (int e = tid; e < LP * LP; e += kAdThr) {       // Ubar = (W1 U)^T: Ubar[i][j] = sum_a W1[j][a] U[a][i]
    const int i = e / LP, j = e % LP;
    float acc = 0.f;
    for (int a = 0; a < LP; ++a) acc = fmaf(W1[j * LP + a], Us[a][i], acc);
    Ub[i][j] = (i < l && j < l) ? acc : 0.f;
  }
  __syncthreads();
  float smax = 0.f;
  for (int a = 0; a < LP; ++a) smax = fmaxf(smax, s[a]);
  for (int e = tid; e < LP * LP; e += kAdThr) {
    const int i = e / LP, j = e % LP;
    float k = 0.f;
    if (i < l && j < l) {
      if (i == j) {
        k = fp[i] * Ub[i][i];
      } else {
        const float ds = s[i] - s[j];
        const float gs = (fabsf(ds) > 1e-6f * smax) ? (f[i] - f[j]) / ds : 0.5f * (fp[i] + fp[j]);
        const float ss = s[i] + s[j];
        const float gk = (ss > 0.f) ? (f[i] + f[j]) / ss : 0.f;
        k = gs * 0.5f * (Ub[i][j] + Ub[j][i]) + gk * 0.5f * (Ub[i][j] - Ub[j][i]);
      }
      k -= d[i] * Ub[i][j];
    }
    Km[i][j] = k;                                      // K - D Ubar
  }
  __syncthreads();
  for (int e = tid; e < LP * LP; e += kAdThr) {
    const int a = e / LP, b = e % LP;
    float c1 = 0.f, c2 = 0.f;
    for (int k = 0; k < LP; ++k) {
      c1 = fmaf(Km[k][a], Us[b][k], c1);              // (K - D Ubar)^T U^T
      c2 = fmaf(Us[a][k] * d[k], Us[b][k], c2);       // U D U^T
    }
    C1[e] = c1;
    C2[e] = c2;
    C3[e] = f[a] * Us[b][a];                          // diag(f) U^T
  }
  if (tid == 0) {
    float tb = 0.f;
    for (int i = 0; i < l; ++i)
      if (s[i] > tau) tb -= Ub[i][i];
    *taubar = tb;
  }
}

// QR adjoint with Rbar = 0: Ybar = (Qbar - Q copyltu(Qbar^T Q)) R^{-T}  (n x LP, columns < l), in
// double (Qbar arrives in double; the bracket cancels most of it).
template <int LP>
__global__ void __launch_bounds__(kAdThr) k_ad_qr_adjoint(const double* __restrict__ Q, const float* __restrict__ R,
                                                         const double* __restrict__ Qbar, int n, int l,
                                                         float* __restrict__ Ybar) {
  __shared__ double Mm[LP][LP], Rs[LP][LP];
  const int tid = threadIdx.x;
  for (int e = tid; e < LP * LP; e += kAdThr) {       // M = Qbar^T Q
    const int a = e / LP, b = e % LP;
    double acc = 0.0;
    if (a < l && b < l)
      for (int i = 0; i < n; ++i)
        acc = fma(Qbar[static_cast<int64_t>(i) * LP + a], Q[static_cast<int64_t>(i) * LP + b], acc);
    Mm[a][b] = acc;
    Rs[a][b] = static_cast<double>(R[e]);
  }
  __syncthreads();
  for (int i = tid; i < n; i += kAdThr) {
    double bv[LP], y[LP];
#pragma unroll
    for (int a = 0; a < LP; ++a) {
      double acc = Qbar[static_cast<int64_t>(i) * LP + a];
#pragma unroll
      for (int c = 0; c < LP; ++c) {
        const double cm = (a >= c) ? Mm[a][c] : Mm[c][a];  // copyltu(M)[c][a]: lower triangle mirrored
        acc = fma(-Q[static_cast<int64_t>(i) * LP + c], cm, acc);
      }
      bv[a] = (a < l) ? acc : 0.0;
    }
#pragma unroll
    for (int j = LP - 1; j >= 0; --j) {                  // y R^T = b, R upper: back substitution
      double acc = bv[j];
#pragma unroll
      for (int k = j + 1; k < LP; ++k) acc = fma(-y[k], Rs[j][k], acc);
      y[j] = (j < l && Rs[j][j] != 0.0) ? acc / Rs[j][j] : 0.0;
    }
#pragma unroll
    for (int a = 0; a < LP; ++a) Ybar[static_cast<int64_t>(i) * LP + a] = static_cast<float>(y[a]);
  }
}

}  // namespace

// ---------------------------------------------------------------- host launchers
int ad_col_splits(int64_t m, int n) {
  const int tiles = (n + 63) / 64;
  int splits = static_cast<int>((m + 255) / 256);
  const int cap = (4 * 152 + tiles - 1) / tiles;
  if (splits > cap) splits = cap;
  if (splits > 64) splits = 64;
  return splits < 1 ? 1 : splits;
}

size_t ad_small_smem(int LP, int n) {
  return LP == 16 ? small_ws_bytes<16>(n, kAdGacc) : small_ws_bytes<32>(n, kAdGacc);
}

template <typename K>
cudaError_t ad_set_limit(K kernel, int smem_limit) {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              smem_limit - static_cast<int>(a.sharedSizeBytes));
}

cudaError_t prepare_adjoint_kernels(int smem_limit) {
  cudaError_t e = ad_set_limit(k_ad_cholqr2<16>, smem_limit);
  if (e == cudaSuccess) e = ad_set_limit(k_ad_cholqr2<32>, smem_limit);
  if (e == cudaSuccess) e = ad_set_limit(k_ad_core<16>, smem_limit);
  if (e == cudaSuccess) e = ad_set_limit(k_ad_core<32>, smem_limit);
  return e;
}

cudaError_t ad_rows(int LP, const float* M, int64_t ldm, int64_t m, int n, const float* S, float* C, int ldc, int coff,
                    float beta, cudaStream_t st) {
  const dim3 grid(static_cast<unsigned>((m + 63) / 64));
  if (LP == 16) k_ad_rows<16><<<grid, kAdThr, 0, st>>>(M, ldm, m, n, S, C, ldc, coff, beta);
  else k_ad_rows<32><<<grid, kAdThr, 0, st>>>(M, ldm, m, n, S, C, ldc, coff, beta);
  return cudaGetLastError();
}

// out (n x LP at row stride ldo, column offset coff) = beta out + M^T T   (T: m x LP, row stride ldt);
// exactly one of out / out_d (double) is non-null.
cudaError_t ad_cols(int LP, const float* M, int64_t ldm, int64_t m, int n, const float* T, int ldt, double* part,
                    float* out, double* out_d, int ldo, int coff, float beta, cudaStream_t st) {
  const int splits = ad_col_splits(m, n);
  const int64_t rps = (m + splits - 1) / splits;
  const dim3 grid(static_cast<unsigned>((n + 63) / 64), static_cast<unsigned>(splits));
  if (LP == 16) k_ad_cols<16><<<grid, kAdThr, 0, st>>>(M, ldm, m, n, T, ldt, rps, part);
  else k_ad_cols<32><<<grid, kAdThr, 0, st>>>(M, ldm, m, n, T, ldt, rps, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t count = static_cast<int64_t>(n) * LP;
  const unsigned blocks = static_cast<unsigned>((count + 255) / 256);
  if (out_d != nullptr) k_ad_reduce<double><<<blocks, 256, 0, st>>>(part, splits, count, out_d, ldo, LP, coff, beta);
  else k_ad_reduce<float><<<blocks, 256, 0, st>>>(part, splits, count, out, ldo, LP, coff, beta);
  return cudaGetLastError();
}

cudaError_t ad_rank(float* A, int64_t lda, int64_t m, int n, const float* L, int ldl, const float* R, int ldr, int K,
                    float beta, cudaStream_t st) {
  const dim3 grid(static_cast<unsigned>((n + 63) / 64), static_cast<unsigned>((m + 63) / 64));
  k_ad_rank<<<grid, kAdThr, 0, st>>>(A, lda, m, n, L, ldl, R, ldr, K, beta);
  return cudaGetLastError();
}

cudaError_t ad_omega(int LP, float* out, int ldo, int coff, int64_t m, int l, uint64_t seed, uint64_t stream,
                     cudaStream_t st) {
  const int64_t total = m * (LP / 4);
  const unsigned blocks = static_cast<unsigned>((total + 255) / 256);
  if (LP == 16) k_ad_omega<16><<<blocks, 256, 0, st>>>(out, ldo, coff, m, l, seed, stream);
  else k_ad_omega<32><<<blocks, 256, 0, st>>>(out, ldo, coff, m, l, seed, stream);
  return cudaGetLastError();
}

cudaError_t ad_cholqr2(int LP, const float* Y, int n, int l, double rank_tol, float* Q, double* Qd, float* R,
                       DevState* dst, cudaStream_t st) {
  const size_t smem = ad_small_smem(LP, n);
  if (LP == 16) k_ad_cholqr2<16><<<1, kAdThr, smem, st>>>(Y, n, l, rank_tol, Q, Qd, R, dst);
  else k_ad_cholqr2<32><<<1, kAdThr, smem, st>>>(Y, n, l, rank_tol, Q, Qd, R, dst);
  return cudaGetLastError();
}

cudaError_t ad_core(int LP, const float* Z, int64_t m, int l, float tau, double rank_tol, int max_sweeps, float* U,
                    float* sig, float* S1, float* S2, DevState* dst, cudaStream_t st) {
  const size_t smem = ad_small_smem(LP, 0);
  if (LP == 16) k_ad_core<16><<<1, kAdThr, smem, st>>>(Z, m, l, tau, rank_tol, max_sweeps, U, sig, S1, S2, dst);
  else k_ad_core<32><<<1, kAdThr, smem, st>>>(Z, m, l, tau, rank_tol, max_sweeps, U, sig, S1, S2, dst);
  return cudaGetLastError();
}

cudaError_t ad_svt_adjoint(int LP, const float* W1, const float* U, const float* sig, int l, float tau, float* C1,
                           float* C2, float* C3, float* taubar, cudaStream_t st) {
  if (LP == 16) k_ad_svt_adjoint<16><<<1, kAdThr, 0, st>>>(W1, U, sig, l, tau, C1, C2, C3, taubar);
  else k_ad_svt_adjoint<32><<<1, kAdThr, 0, st>>>(W1, U, sig, l, tau, C1, C2, C3, taubar);
  return cudaGetLastError();
}

cudaError_t ad_qr_adjoint(int LP, const double* Q, const float* R, const double* Qbar, int n, int l, float* Ybar,
                          cudaStream_t st) {
  if (LP == 16) k_ad_qr_adjoint<16><<<1, kAdThr, 0, st>>>(Q, R, Qbar, n, l, Ybar);
  else k_ad_qr_adjoint<32><<<1, kAdThr, 0, st>>>(Q, R, Qbar, n, l, Ybar);
  return cudaGetLastError();
}

}  // namespace frsvt
