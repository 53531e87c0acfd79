// Single-CTA kernels for the small l x l and short-side (n x l) work of Alg. 1.
//
// k_orth : orthonormal basis of the sketch (Alg. 1 steps 6, 10-11, 14).  The
//          paper uses QR with column pivoting; here the basis comes from a
//          Cholesky QR applied twice (CholeskyQR2) with the Gram matrix
//          accumulated in double-float, the Cholesky factor in FP64, and a
//          pivot cut that drops numerically dependent columns (s = min(l, rank)).
//          Under range propagation the new block is first projected out of the
//          propagated basis twice (block Gram-Schmidt with reorthogonalisation,
//          the "partial orthogonalization" of step 10).  Only span(Q) matters
//          for the result (Prop. 1), so the choice of QR does not change X.
// k_core : SVD of the projected matrix B = Q^T A through its Gram
//          B B^T = Z^T Z (Z = A Q): FP64 Cholesky Z^T Z = R^T R, then a
//          one-sided Jacobi SVD of R^T in FP32, which gives the singular
//          values D and left singular vectors U_B of B (the polar + eigen route
//          of Alg. 1 steps 16-18 computes the same factors).  Then the soft
//          shrinkage S_tau(D), the coefficient matrix M = U_B diag(S_tau(D)/D) U_B^T
//          of Eq. 6 (X = Z M Q^T), and the propagated basis Q~ = Q U_B (step 21).
#include "common.cuh"
#include "state.cuh"

namespace frsvt {

namespace {

constexpr int kBig = 1024;

// Cholesky G = R^T R (upper R) of the leading p x p block with column drops.
// A column j is dropped (row j of R set to zero) when its pivot is not above
// rank_tol * G_jj, when G_jj is below 1e-15 of the largest diagonal, or when
// the pivot is not a positive finite number.  A non-finite diagonal (NaN or Inf met in the Gram
// reduction) ORs FRSVT_DEV_NONFINITE into *status when given.  Run by one full warp.
template <int LP>
__device__ void chol_drop_warp(const double* G, double* R, int* dropped, int p, double rank_tol,
                               uint32_t* status = nullptr) {
  const int lane = threadIdx.x & 31;
  double maxdiag = 0.0;
  bool finite = true;
  for (int a = 0; a < p; ++a) {
    maxdiag = fmax(maxdiag, G[a * LP + a]);
    finite = finite && isfinite(G[a * LP + a]);
  }
  if (!finite && lane == 0 && status != nullptr) atomicOr(status, kDevNonfinite);
  for (int jj = 0; jj < p; ++jj) {
    double d = G[jj * LP + jj];
    for (int k = 0; k < jj; ++k) d -= R[k * LP + jj] * R[k * LP + jj];
    const double gjj = G[jj * LP + jj];
    const bool drop = !(d > rank_tol * gjj) || !(gjj > 1e-15 * maxdiag) || !(d < 1e300);
    const double rjj = drop ? 0.0 : sqrt(d);
    if (lane < LP) {
      double v = 0.0;
      if (lane == jj) {
        v = rjj;
      } else if (lane > jj && lane < p && !drop) {
        double t = G[jj * LP + lane];
        for (int k = 0; k < jj; ++k) t -= R[k * LP + jj] * R[k * LP + lane];
        v = t / rjj;
      }
      R[jj * LP + lane] = v;
    }
    if (lane == 0) dropped[jj] = drop ? 1 : 0;
    __syncwarp();
  }
}

// T = R^{-1} (upper triangular, zero rows / columns for dropped indices). One warp.
template <int LP>
__device__ void tri_inverse_warp(const double* R, const int* dropped, double* Td, float* T, int p) {
  const int lane = threadIdx.x & 31;
  for (int jj = 0; jj < p; ++jj) {
    if (lane < p) {
      double v = 0.0;
      if (!dropped[jj]) {
        const double tjj = 1.0 / R[jj * LP + jj];
        if (lane == jj) {
          v = tjj;
        } else if (lane < jj && !dropped[lane]) {
          double s = 0.0;
          for (int k = lane; k < jj; ++k) s += Td[lane * LP + k] * R[k * LP + jj];
          v = -s * tjj;
        }
      }
      Td[lane * LP + jj] = v;
      T[lane * LP + jj] = static_cast<float>(v);
    }
    __syncwarp();
  }
}

__device__ __forceinline__ void decode_pair(int pr, int p, int& a, int& b) {
  a = 0;
  while (pr >= p - a) { pr -= p - a; ++a; }
  b = a + pr;
}

template <int LP>
__global__ void __launch_bounds__(kBig)
k_orth(const float* __restrict__ Y, int64_t ns, int l, int use_rp, const float* __restrict__ Qt,
       float* __restrict__ Q, DevState* __restrict__ dst, double rank_tol) {
  extern __shared__ __align__(16) unsigned char smraw[];
  double* G = reinterpret_cast<double*>(smraw);
  double* R = G + LP * LP;
  double* Td = R + LP * LP;
  float* T = reinterpret_cast<float*>(Td + LP * LP);
  float* Cm = T + LP * LP;
  double* gacc = reinterpret_cast<double*>(Cm + LP * LP);    // kBig entries
  int* dropped = reinterpret_cast<int*>(gacc + kBig);          // LP
  float* W = reinterpret_cast<float*>(dropped + LP);          // ns x LP (offset is a multiple of 16 bytes)
  const int tid = threadIdx.x;
  const int nt = blockDim.x;

  int keep = use_rp ? dst->keep : 0;
  keep = max(0, min(keep, l));
  const int p = l - keep;
  for (int64_t e = tid; e < ns * LP; e += nt) {
    const int c = static_cast<int>(e % LP);
    const int64_t i = e / LP;
    float v = 0.f;
    if (c < keep) v = Qt[e];
    else if (c < l) v = Y[i * LP + (c - keep)];
    W[e] = v;
  }
  __syncthreads();

  // Partial orthogonalization of the new block against the propagated basis, twice.
  if (keep > 0 && p > 0) {
    for (int pass = 0; pass < 2; ++pass) {
      for (int pr = tid; pr < keep * p; pr += nt) {
        const int a = pr / p, b = pr % p;
        float acc = 0.f;
        for (int64_t i = 0; i < ns; ++i) acc = fmaf(W[i * LP + a], W[i * LP + keep + b], acc);
        Cm[a * LP + b] = acc;
      }
      __syncthreads();
      for (int64_t i = tid; i < ns; i += nt) {
        float w[LP];
#pragma unroll
        for (int c = 0; c < LP; ++c) w[c] = W[i * LP + c];
        for (int b = 0; b < p; ++b) {
          float acc = w[keep + b];
          for (int a = 0; a < keep; ++a) acc = fmaf(-w[a], Cm[a * LP + b], acc);
          W[i * LP + keep + b] = acc;
        }
      }
      __syncthreads();
    }
  }

  // Cholesky QR of the new block, twice.
  if (tid == 0 && use_rp && (keep == 0 || p == 0)) dst->rp_res = -1.f;
  int kept = 0;
  for (int pass = 0; pass < 2 && p > 0; ++pass) {
    const int np = p * (p + 1) / 2;
    const int groups = max(1, nt / np);
    if (tid < np * groups) {
      const int pr = tid % np, g = tid / np;
      int a, b;
      decode_pair(pr, p, a, b);
      df64 acc{0.f, 0.f};
      for (int64_t i = g; i < ns; i += groups) df64_add_prod(acc, W[i * LP + keep + a], W[i * LP + keep + b]);
      gacc[tid] = df64_value(acc);
    }
    __syncthreads();
    if (tid < np) {
      int a, b;
      decode_pair(tid, p, a, b);
      double s = 0.0;
      for (int g = 0; g < groups; ++g) s += gacc[g * np + tid];
      G[a * LP + b] = s;
      G[b * LP + a] = s;
    }
    __syncthreads();
    if (pass == 0 && tid == 0 && use_rp && keep > 0) dst->rp_res = sqrtf(static_cast<float>(G[0]));   // Prop. 4
    if (tid < 32) {
      chol_drop_warp<LP>(G, R, dropped, p, rank_tol, &dst->status);
      tri_inverse_warp<LP>(R, dropped, Td, T, p);
    }
    __syncthreads();
    for (int64_t i = tid; i < ns; i += nt) {
      float w[LP];
#pragma unroll
      for (int c = 0; c < LP; ++c) w[c] = (c < p) ? W[i * LP + keep + c] : 0.f;
      for (int b = 0; b < p; ++b) {
        float acc = 0.f;
        for (int a = 0; a <= b; ++a) acc = fmaf(w[a], T[a * LP + b], acc);
        W[i * LP + keep + b] = acc;
      }
    }
    __syncthreads();
    kept = 0;                                   // columns that survive the last pass
    for (int c = 0; c < p; ++c) kept += dropped[c] ? 0 : 1;
  }

  for (int64_t e = tid; e < ns * LP; e += nt) Q[e] = W[e];
  if (tid == 0) {
    dst->s = keep + kept;
    if (keep + kept < l) dst->status |= kDevRankDeficient;
  }
}

// Round-robin schedule: pair w of round rnd among N (even) indices.
__device__ __forceinline__ void rr_pair(int rnd, int w, int N, int& p, int& q) {
  if (w == 0) {
    p = N - 1;
    q = rnd;
  } else {
    p = (rnd + w) % (N - 1);
    q = (rnd - w + (N - 1)) % (N - 1);
  }
  if (p > q) { const int t = p; p = q; q = t; }
}

template <int LP>
__global__ void __launch_bounds__(kBig)
k_core(const float2* __restrict__ gpart, int gsplit, const float* __restrict__ Q, int64_t ns, int l,
       float tau_host, int tau_from_mu, int update_rp, int advance_counter, float* __restrict__ Rf,
       float* __restrict__ Qt, DevState* __restrict__ dst, double rank_tol, int max_sweeps) {
  __shared__ double G[LP * LP];
  __shared__ double R[LP * LP];
  __shared__ float Xt[LP * LP];     // Xt[b * LP + a] = R[b][a]: row b = column b of X = R^T
  __shared__ float U[LP * LP];      // U[a * LP + b]: left singular vector b of B
  __shared__ float M[LP * LP];
  __shared__ float sig[LP], coef[LP];
  __shared__ int perm[LP], dropped[LP];
  __shared__ int rotated, sweeps_done;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;

  // 1. Gram B B^T = Z^T Z from the df64 partials (FP64 sum in split order).
  for (int e = tid; e < LP * LP; e += nt) {
    const int a = e / LP, b = e % LP;
    double s = 0.0;
    if (a < l && b < l) {
      for (int g = 0; g < gsplit; ++g) {
        const float2 v = gpart[static_cast<int64_t>(g) * LP * LP + e];
        s += static_cast<double>(v.x) + static_cast<double>(v.y);
      }
    }
    G[e] = s;
  }
  __syncthreads();
  // 2. Cholesky with column drops.
  if (warp == 0) chol_drop_warp<LP>(G, R, dropped, l, rank_tol, &dst->status);
  __syncthreads();
  for (int e = tid; e < LP * LP; e += nt) {
    const int b = e / LP, a = e % LP;
    Xt[e] = (b < l && a < l) ? static_cast<float>(R[b * LP + a]) : 0.f;
  }
  if (tid == 0) { sweeps_done = 0; }
  __syncthreads();
  // 3. One-sided Jacobi on the columns of X = R^T (rows of Xt), FP32.
  const float tol = 1e-6f;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (tid == 0) rotated = 0;
    __syncthreads();
    for (int rnd = 0; rnd < LP - 1; ++rnd) {
      if (warp < LP / 2) {
        int p, q;
        rr_pair(rnd, warp, LP, p, q);
        const float xp = (lane < LP) ? Xt[p * LP + lane] : 0.f;
        const float xq = (lane < LP) ? Xt[q * LP + lane] : 0.f;
        const float alpha = warp_sum(xp * xp);
        const float beta = warp_sum(xq * xq);
        const float gamma = warp_sum(xp * xq);
        const float small = 1e-30f;
        if (fabsf(gamma) > tol * sqrtf(alpha * beta) && alpha > small && beta > small) {
          const float zeta = (beta - alpha) / (2.f * gamma);
          const float t = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
          const float c = rsqrtf(1.f + t * t);
          const float s = c * t;
          if (lane < LP) {
            Xt[p * LP + lane] = c * xp - s * xq;
            Xt[q * LP + lane] = s * xp + c * xq;
          }
          if (lane == 0) rotated = 1;
        }
      }
      __syncthreads();
    }
    if (tid == 0) sweeps_done = sweep + 1;
    const int any = rotated;
    __syncthreads();
    if (!any) break;
  }
  // 4. Singular values and vectors.
  if (tid < LP) {
    float s2 = 0.f;
    for (int a = 0; a < LP; ++a) s2 = fmaf(Xt[tid * LP + a], Xt[tid * LP + a], s2);
    sig[tid] = sqrtf(s2);
  }
  __syncthreads();
  for (int e = tid; e < LP * LP; e += nt) {
    const int a = e / LP, b = e % LP;
    U[e] = (sig[b] > 0.f) ? Xt[b * LP + a] / sig[b] : 0.f;
  }
  const float tau = tau_from_mu ? static_cast<float>(1.0 / dst->mu) : tau_host;
  if (tid < LP) {
    int rank = 0;
    rank = sigma_rank(sig, LP, tid);
    perm[rank] = tid;
    coef[tid] = (sig[tid] > tau) ? (sig[tid] - tau) / sig[tid] : 0.f;
  }
  __syncthreads();
  // 5. M = U diag(coef) U^T.
  for (int e = tid; e < LP * LP; e += nt) {
    const int a = e / LP, c = e % LP;
    float acc = 0.f;
    for (int b = 0; b < LP; ++b) acc = fmaf(U[a * LP + b] * coef[b], U[c * LP + b], acc);
    M[e] = acc;
  }
  int r = 0;
  for (int c = 0; c < LP; ++c) r += (sig[c] > tau) ? 1 : 0;
  const int keep = update_rp ? max(0, min(r, l - 2)) : 0;
  __syncthreads();
  // 6. Rf = Q M (so that X = Z Rf^T) and the propagated basis Qt = Q U[:, perm[:keep]].
  for (int64_t e = tid; e < ns * LP; e += nt) {
    const int64_t i = e / LP;
    const int k = static_cast<int>(e % LP);
    float acc = 0.f, accq = 0.f;
    const int pk = (k < keep) ? perm[k] : 0;
    for (int a = 0; a < LP; ++a) {
      const float qa = Q[i * LP + a];
      acc = fmaf(qa, M[a * LP + k], acc);
      accq = fmaf(qa, U[a * LP + pk], accq);
    }
    Rf[e] = acc;
    if (update_rp && k < keep) Qt[e] = accq;
  }
  if (tid == 0) {
    dst->r = r;
    if (update_rp) dst->keep = keep;
    if (advance_counter) dst->counter += 1;
    dst->sweeps = sweeps_done;
    if (sweeps_done >= max_sweeps) dst->status |= kDevNotConverged;
    bool finite = true;
    for (int c = 0; c < LP; ++c) {
      dst->sigma[c] = sig[perm[c]];
      finite = finite && isfinite(sig[c]);
    }
    for (int c = LP; c < kMaxL; ++c) dst->sigma[c] = 0.f;
    if (!finite) dst->status |= kDevNonfinite;
    dst->sigma1 = static_cast<double>(sig[perm[0]]);
  }
}

__global__ void k_alm_finish(const float2* __restrict__ rpart, int count, DevState* __restrict__ dst) {
  double s = 0.0;
  for (int i = threadIdx.x; i < count; i += 32) s += static_cast<double>(rpart[i].x) + static_cast<double>(rpart[i].y);
  s = warp_sum(s);
  if (threadIdx.x == 0) {
    const double ratio = (dst->normO_F > 0.0) ? sqrt(s) / dst->normO_F : 0.0;
    dst->resid_ratio = ratio;
    if (!isfinite(ratio)) dst->status |= kDevNonfinite;
    dst->mu = fmin(dst->rho * dst->mu, dst->mu_bar);
    dst->iter += 1;
  }
}

__global__ void k_init_scalars(const float* __restrict__ pmax, const float2* __restrict__ psum, int nblk,
                               double normO2_host, double lambda, double rho, double mu_bar_factor,
                               DevState* __restrict__ dst) {
  float mx = 0.f;
  double s = 0.0;
  for (int i = threadIdx.x; i < nblk; i += 32) {
    mx = fmaxf(mx, pmax[i]);
    s += static_cast<double>(psum[i].x) + static_cast<double>(psum[i].y);
  }
  s = warp_sum(s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (threadIdx.x == 0) {
    const double normO2 = (normO2_host > 0.0) ? normO2_host : dst->sigma1;
    const double J = fmax(normO2, static_cast<double>(mx) / lambda);
    const double mu0 = 1.25 / normO2;
    dst->normO_F = sqrt(s);
    dst->mu = mu0;
    dst->mu_bar = mu_bar_factor * mu0;
    dst->rho = rho;
    dst->lambda = lambda;
    dst->init_scale = 1.0 + 1.0 / (J * mu0);
    dst->sigma1 = normO2;
    dst->resid_ratio = 0.0;
    dst->iter = 0;
    dst->counter = 0;
    dst->keep = 0;
    if (!(normO2 > 0.0) || !isfinite(normO2)) dst->status |= kDevNonfinite;
  }
}

template <int LP>
size_t orth_smem(int64_t ns) {
  return static_cast<size_t>(3 * LP * LP) * sizeof(double) + static_cast<size_t>(2 * LP * LP) * sizeof(float) +
         kBig * sizeof(double) + LP * sizeof(int) + static_cast<size_t>(ns) * LP * sizeof(float);
}

}  // namespace

size_t orth_smem_bytes(int LP, int64_t ns) { return LP == 16 ? orth_smem<16>(ns) : orth_smem<32>(ns); }

cudaError_t launch_orth(int LP, const float* Y, int64_t ns, int l, int use_rp, const float* Qt, float* Q,
                        DevState* dst, double rank_tol, cudaStream_t st) {
  const size_t smem = orth_smem_bytes(LP, ns);
  if (LP == 16) k_orth<16><<<1, kBig, smem, st>>>(Y, ns, l, use_rp, Qt, Q, dst, rank_tol);
  else k_orth<32><<<1, kBig, smem, st>>>(Y, ns, l, use_rp, Qt, Q, dst, rank_tol);
  return cudaGetLastError();
}

cudaError_t prepare_small_kernels(int smem_limit) {
  cudaError_t e = cudaFuncSetAttribute(k_orth<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_limit);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_orth<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_limit);
}

cudaError_t launch_core(int LP, const float2* gpart, int gsplit, const float* Q, int64_t ns, int l, float tau_host,
                        int tau_from_mu, int update_rp, int advance_counter, float* Rf, float* Qt, DevState* dst,
                        double rank_tol, int max_sweeps, cudaStream_t st) {
  if (LP == 16)
    k_core<16><<<1, kBig, 0, st>>>(gpart, gsplit, Q, ns, l, tau_host, tau_from_mu, update_rp, advance_counter, Rf,
                                   Qt, dst, rank_tol, max_sweeps);
  else
    k_core<32><<<1, kBig, 0, st>>>(gpart, gsplit, Q, ns, l, tau_host, tau_from_mu, update_rp, advance_counter, Rf,
                                   Qt, dst, rank_tol, max_sweeps);
  return cudaGetLastError();
}

cudaError_t launch_alm_finish(const float2* rpart, int count, DevState* dst, cudaStream_t st) {
  k_alm_finish<<<1, 32, 0, st>>>(rpart, count, dst);
  return cudaGetLastError();
}

cudaError_t launch_init_scalars(const float* pmax, const float2* psum, int nblk, double normO2_host, double lambda,
                                double rho, double mu_bar_factor, DevState* dst, cudaStream_t st) {
  k_init_scalars<<<1, 32, 0, st>>>(pmax, psum, nblk, normO2_host, lambda, rho, mu_bar_factor, dst);
  return cudaGetLastError();
}

}  // namespace frsvt
