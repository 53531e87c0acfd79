// Batched weighted SVT of small matrices (the WNNM patch groups of the WSVT footnote, Sec. 1):
// X_b = U max(Sigma - w(Sigma), 0) V^T for every problem A_b (m x n_b, m <= 64), with the
// weights w_j = c sqrt(n_b) / (sigma_j + eps) evaluated on the problem's own singular values.
//
// One persistent launch serves the whole batch: each CTA takes the next problem from an atomic
// counter (the n_b differ, so static striding would leave CTAs idle), stages A_b in shared
// memory once and leaves X_b in global memory.
//
// Exact variant: Gram matrix on the short side (s = min(m, n_b) <= 64), two-sided cyclic Jacobi
// eigensolver on it (all N/2 disjoint rotations of a round-robin round applied at once: rows,
// then columns and the eigenvector matrix), sigma_j = sqrt(lambda_j), then
// X_h = V diag(phi) V^T A_h with phi_j = max(sigma_j - w_j, 0) / sigma_j.
// FRSVT variant: Alg. 1 on the problem in shared memory (Omega from the Philox stream with the
// problem index b, q power steps, CholeskyQR2 bases, double-float Gram and the Cholesky +
// one-sided Jacobi core of small_dense.cuh), the weights applied to D.
// The launch shape (threads per CTA, CTAs per SM) is a parameter chosen by the autotuner of
// the host API.
#include <cstdint>

#include "common.cuh"
#include "small_dense.cuh"
#include "state.cuh"

namespace frsvt {

namespace {

constexpr int kWMaxM = 64;
constexpr int kWGacc = 256;

struct WsvtArgs {
  const float* const* A;
  float* const* X;
  const int32_t* n;
  int batch, m, n_max;
  float c, eps;
  uint64_t seed, stream;
  int l, q;
  double rank_tol;
  int max_sweeps;
  unsigned* next;
  DevState* dst;
};

__host__ __device__ inline int wsvt_lda(int n_max) { return n_max | 1; }

// ---------------------------------------------------------------- shared-memory layouts
__host__ __device__ inline size_t wsvt_exact_smem(int m, int n_max) {
  const int s = m < n_max ? m : n_max;
  const int N = s + (s & 1);
  const size_t a = static_cast<size_t>(m) * wsvt_lda(n_max) * sizeof(float);
  const size_t g = static_cast<size_t>(N) * (N + 1) * sizeof(float);
  return a + 2 * g + 64 * sizeof(float) * 4 + 64 * sizeof(int) * 4;
}

template <int LP>
__host__ __device__ inline size_t wsvt_frsvt_smem(int m, int n_max) {
  const int L = m > n_max ? m : n_max;
  const size_t a = static_cast<size_t>(m) * wsvt_lda(n_max) * sizeof(float);
  const size_t z = static_cast<size_t>(L) * LP * sizeof(float);
  const size_t rf = static_cast<size_t>(kWMaxM) * LP * sizeof(float);
  return (a + 15) / 16 * 16 + z + rf + small_ws_bytes<LP>(kWMaxM, kWGacc);
}

// Problem index for the CTA (thread 0 draws it, everyone reads it).
__device__ __forceinline__ int next_problem(unsigned* next, int* slot) {
  __syncthreads();
  if (threadIdx.x == 0) *slot = static_cast<int>(atomicAdd(next, 1u));
  __syncthreads();
  return *slot;
}

// Stage A_b (m x n row-major, contiguous) at ld into shared memory.
__device__ __forceinline__ void stage_a(const float* __restrict__ A, int m, int n, int ld, float* As) {
  const int total = m * n;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int i = e / n, j = e - i * n;
    As[i * ld + j] = __ldg(A + e);
  }
}

// ---------------------------------------------------------------- exact variant
template <int NT>
__global__ void __launch_bounds__(NT) k_wsvt_exact(WsvtArgs p) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ int slot;
  const int ld = wsvt_lda(p.n_max);
  float* As = reinterpret_cast<float*>(dsm);
  const int sM = p.m < p.n_max ? p.m : p.n_max;
  const int NM = sM + (sM & 1);
  float* G = As + p.m * ld;                       // N x (N + 1)
  float* V = G + NM * (NM + 1);                   // N x (N + 1)
  float* csc = V + NM * (NM + 1);                 // 64 cos, 64 sin
  float* phi = csc + 128;                         // 64
  int* pq = reinterpret_cast<int*>(phi + 64);     // 64 pairs (p, q)
  int* act = pq + 128;                            // active components
  const int tid = threadIdx.x;
  for (int b = next_problem(p.next, &slot); b < p.batch; b = next_problem(p.next, &slot)) {
    const int m = p.m, n = p.n[b];
    if (n < 1 || n > p.n_max || m < 1 || m > kWMaxM) {
      if (tid == 0) atomicOr(&p.dst->status, kDevBadProblem);
      continue;
    }
    stage_a(p.A[b], m, n, ld, As);
    const bool rows = n >= m;                     // A_h = A (s = m) or A^T (s = n)
    const int s = rows ? m : n, L = rows ? n : m;
    const int N = s + (s & 1), gld = N + 1;
    __syncthreads();
    // Gram on the short side, 2 x 2 register blocks over the upper triangle
    const int nbk = N / 2, nblk = nbk * (nbk + 1) / 2;
    for (int e = tid; e < nblk; e += NT) {
      int bi, bj;
      decode_pair_sym(e, nbk, bi, bj);
      const int i0 = 2 * bi, j0 = 2 * bj;
      float g00 = 0.f, g01 = 0.f, g10 = 0.f, g11 = 0.f;
      for (int k = 0; k < L; ++k) {
        float a0, a1, c0, c1;
        if (rows) {
          a0 = As[i0 * ld + k];
          a1 = (i0 + 1 < s) ? As[(i0 + 1) * ld + k] : 0.f;
          c0 = As[j0 * ld + k];
          c1 = (j0 + 1 < s) ? As[(j0 + 1) * ld + k] : 0.f;
        } else {
          a0 = As[k * ld + i0];
          a1 = (i0 + 1 < s) ? As[k * ld + i0 + 1] : 0.f;
          c0 = As[k * ld + j0];
          c1 = (j0 + 1 < s) ? As[k * ld + j0 + 1] : 0.f;
        }
        g00 = fmaf(a0, c0, g00);
        g01 = fmaf(a0, c1, g01);
        g10 = fmaf(a1, c0, g10);
        g11 = fmaf(a1, c1, g11);
      }
      G[i0 * gld + j0] = g00;
      G[i0 * gld + j0 + 1] = g01;
      G[(i0 + 1) * gld + j0] = g10;
      G[(i0 + 1) * gld + j0 + 1] = g11;
      G[j0 * gld + i0] = g00;
      G[(j0 + 1) * gld + i0] = g01;
      G[j0 * gld + i0 + 1] = g10;
      G[(j0 + 1) * gld + i0 + 1] = g11;
    }
    for (int e = tid; e < N * N; e += NT) V[(e / N) * gld + e % N] = (e / N == e % N) ? 1.f : 0.f;
    __syncthreads();
    // cyclic Jacobi: round rnd pairs index N - 1 with rnd and (rnd + w) with (rnd - w) mod (N - 1)
    const float tol = 1e-6f;
    for (int sweep = 0; sweep < p.max_sweeps && N >= 2; ++sweep) {
      int any = 0;
      for (int rnd = 0; rnd < N - 1; ++rnd) {
        int rot = 0;
        if (tid < N / 2) {
          int a, c;
          if (tid == 0) {
            a = N - 1;
            c = rnd;
          } else {
            a = (rnd + tid) % (N - 1);
            c = (rnd - tid + (N - 1)) % (N - 1);
          }
          const int pp = a < c ? a : c, qq = a < c ? c : a;
          const float gpp = G[pp * gld + pp], gqq = G[qq * gld + qq], gpq = G[pp * gld + qq];
          float cs = 1.f, sn = 0.f;
          if (fabsf(gpq) > tol * sqrtf(fabsf(gpp * gqq)) && gpq != 0.f) {
            const float theta = (gqq - gpp) / (2.f * gpq);
            const float t = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(1.f + theta * theta));
            cs = rsqrtf(1.f + t * t);
            sn = t * cs;
            rot = 1;
          }
          pq[2 * tid] = pp;
          pq[2 * tid + 1] = qq;
          csc[tid] = cs;
          csc[64 + tid] = sn;
        }
        any |= __syncthreads_or(rot);
        for (int e = tid; e < (N / 2) * N; e += NT) {            // rows p, q of G
          const int t = e / N, j = e - t * N;
          const float cs = csc[t], sn = csc[64 + t];
          if (sn == 0.f) continue;
          const int pp = pq[2 * t], qq = pq[2 * t + 1];
          const float gp = G[pp * gld + j], gq = G[qq * gld + j];
          G[pp * gld + j] = cs * gp - sn * gq;
          G[qq * gld + j] = sn * gp + cs * gq;
        }
        __syncthreads();
        for (int e = tid; e < (N / 2) * N; e += NT) {            // columns p, q of G and V
          const int t = e / N, i = e - t * N;
          const float cs = csc[t], sn = csc[64 + t];
          if (sn == 0.f) continue;
          const int pp = pq[2 * t], qq = pq[2 * t + 1];
          const float gp = G[i * gld + pp], gq = G[i * gld + qq];
          G[i * gld + pp] = cs * gp - sn * gq;
          G[i * gld + qq] = sn * gp + cs * gq;
          const float vp = V[i * gld + pp], vq = V[i * gld + qq];
          V[i * gld + pp] = cs * vp - sn * vq;
          V[i * gld + qq] = sn * vp + cs * vq;
        }
        __syncthreads();
      }
      if (!any) break;
    }
    // weights on the eigenvalues' square roots; active components compacted
    if (tid < 64) phi[tid] = 0.f;
    __syncthreads();
    const float cw = p.c * sqrtf(static_cast<float>(n));
    if (tid < s) {
      const float sg = sqrtf(fmaxf(G[tid * gld + tid], 0.f));
      const float wj = cw / (sg + p.eps);
      phi[tid] = (sg > wj) ? (sg - wj) / sg : 0.f;
    }
    __syncthreads();
    if (tid == 0) {
      int ra = 0;
      for (int j = 0; j < s; ++j)
        if (phi[j] > 0.f) act[1 + ra++] = j;
      act[0] = ra;
    }
    __syncthreads();
    const int ra = act[0];
    // M = V_act diag(phi) V_act^T into G's storage
    for (int e = tid; e < s * s; e += NT) {
      const int i = e / s, j = e - i * s;
      float acc = 0.f;
      for (int a = 0; a < ra; ++a) {
        const int ja = act[1 + a];
        acc = fmaf(V[i * gld + ja] * phi[ja], V[j * gld + ja], acc);
      }
      G[i * gld + j] = acc;
    }
    __syncthreads();
    // X = M A_h in the orientation of A
    float* X = p.X[b];
    if (rows) {
      for (int e = tid; e < m * n; e += NT) {
        const int i = e / n, k = e - i * n;
        float acc = 0.f;
        for (int j = 0; j < s; ++j) acc = fmaf(G[i * gld + j], As[j * ld + k], acc);
        X[e] = acc;
      }
    } else {
      for (int e = tid; e < m * n; e += NT) {
        const int k = e / n, i = e - k * n;           // X[k][i] = (M A^T)[i][k]
        float acc = 0.f;
        for (int j = 0; j < s; ++j) acc = fmaf(G[i * gld + j], As[k * ld + j], acc);
        X[e] = acc;
      }
    }
  }
}

// ---------------------------------------------------------------- FRSVT variant
template <int NT, int LP>
__global__ void __launch_bounds__(NT) k_wsvt_frsvt(WsvtArgs p) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ int slot;
  const int ld = wsvt_lda(p.n_max);
  const int Lmax = p.m > p.n_max ? p.m : p.n_max;
  float* As = reinterpret_cast<float*>(dsm);
  float* Zb = reinterpret_cast<float*>(dsm + (static_cast<size_t>(p.m) * ld * sizeof(float) + 15) / 16 * 16);
  float* Rf = Zb + static_cast<size_t>(Lmax) * LP;
  unsigned char* wsb = reinterpret_cast<unsigned char*>(Rf + kWMaxM * LP);
  SmallWs<LP> w = carve_small_ws<LP>(wsb, kWGacc);
  float* W = w.W;                                   // s x LP: Y, then Q
  const int tid = threadIdx.x;
  for (int b = next_problem(p.next, &slot); b < p.batch; b = next_problem(p.next, &slot)) {
    const int m = p.m, n = p.n[b];
    if (n < 1 || n > p.n_max || m < 1 || m > kWMaxM || p.l < 1 || p.l > LP) {
      if (tid == 0) atomicOr(&p.dst->status, kDevBadProblem);
      continue;
    }
    stage_a(p.A[b], m, n, ld, As);
    const bool tr = m >= n;                      // A_h = A^T (short n x long m), ties transpose
    const int s = tr ? n : m, L = tr ? m : n;
    const int ls = p.l < s ? p.l : s;
    auto ah = [&](int i, int j) -> float { return tr ? As[j * ld + i] : As[i * ld + j]; };   // A_h[i][j]
    // Omega (L x LP, columns >= ls zero) in Zb
    for (int e = tid; e < L * (LP / 4); e += NT) {
      const int j = e / (LP / 4), k4 = e - j * (LP / 4);
      float4 g = gaussian4(p.seed, static_cast<uint64_t>(j), static_cast<uint64_t>(k4), p.stream,
                           static_cast<uint64_t>(b));
      float v[4] = {g.x, g.y, g.z, g.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) Zb[j * LP + 4 * k4 + u] = (4 * k4 + u < ls) ? v[u] : 0.f;
    }
    __syncthreads();
    // W = A_h Zb (s x LP)
    auto mul_ah = [&]() {
      for (int e = tid; e < s * LP; e += NT) {
        const int i = e / LP, k = e - i * LP;
        float acc = 0.f;
        for (int j = 0; j < L; ++j) acc = fmaf(ah(i, j), Zb[j * LP + k], acc);
        W[e] = acc;
      }
      __syncthreads();
    };
    // Zb = A_h^T W (L x LP)
    auto mul_aht = [&]() {
      for (int e = tid; e < L * LP; e += NT) {
        const int j = e / LP, k = e - j * LP;
        float acc = 0.f;
        for (int i = 0; i < s; ++i) acc = fmaf(ah(i, j), W[i * LP + k], acc);
        Zb[e] = acc;
      }
      __syncthreads();
    };
    mul_ah();
    orth_block<LP>(w, s, 0, ls, p.rank_tol, 2);
    for (int it = 0; it < p.q; ++it) {
      mul_aht();
      mul_ah();
      orth_block<LP>(w, s, 0, ls, p.rank_tol, 2);
    }
    mul_aht();                                     // Z = A_h^T Q = B^T
    for (int e = tid; e < LP * LP; e += NT) w.G[e] = df64{0.f, 0.f};
    __syncthreads();
    block_inner<LP>(Zb, L, 0, 0, ls, ls, true, w.G, w.gacc, w.gacc_n);
    core_svd_block<LP>(w, ls, p.rank_tol, p.max_sweeps);
    float* sig = w.vec;
    float* coef = w.vec + LP;
    const float cw = p.c * sqrtf(static_cast<float>(n));
    if (tid < LP) {
      const float sg = sig[tid];
      const float wj = cw / (sg + p.eps);
      coef[tid] = (tid < ls && sg > wj) ? (sg - wj) / sg : 0.f;
    }
    __syncthreads();
    for (int e = tid; e < LP * LP; e += NT) {      // M = U diag(coef) U^T
      const int a = e / LP, c = e - a * LP;
      float acc = 0.f;
      for (int k = 0; k < LP; ++k) acc = fmaf(w.U[a * LP + k] * coef[k], w.U[c * LP + k], acc);
      w.Cm[e] = acc;
    }
    __syncthreads();
    for (int e = tid; e < s * LP; e += NT) {       // Rf = Q M
      const int i = e / LP, k = e - i * LP;
      float acc = 0.f;
      for (int a = 0; a < LP; ++a) acc = fmaf(W[i * LP + a], w.Cm[a * LP + k], acc);
      Rf[e] = acc;
    }
    __syncthreads();
    float* X = p.X[b];                             // X_h = Rf Z^T (s x L) in the orientation of A
    if (!tr) {
      for (int e = tid; e < m * n; e += NT) {
        const int i = e / n, j = e - i * n;
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < LP; ++k) acc = fmaf(Rf[i * LP + k], Zb[j * LP + k], acc);
        X[e] = acc;
      }
    } else {
      for (int e = tid; e < m * n; e += NT) {
        const int j = e / n, i = e - j * n;        // X[j][i] = X_h[i][j]
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < LP; ++k) acc = fmaf(Rf[i * LP + k], Zb[j * LP + k], acc);
        X[e] = acc;
      }
    }
  }
}

template <typename K>
cudaError_t wsvt_prepare_one(K kernel, size_t smem) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
}

template <typename K>
int wsvt_occupancy(K kernel, int nt, size_t smem) {
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, nt, smem) != cudaSuccess) blocks = 0;
  (void)cudaGetLastError();
  return blocks;
}

}  // namespace

// Dynamic shared memory of a variant (0 exact, 1 FRSVT) for problems m x n (n <= n_max).
size_t wsvt_smem(int variant, int m, int n_max, int LP) {
  if (variant == 0) return wsvt_exact_smem(m, n_max);
  return LP == 16 ? wsvt_frsvt_smem<16>(m, n_max) : wsvt_frsvt_smem<32>(m, n_max);
}

// Resident CTAs per SM of a launch shape (0 if it does not fit).
int wsvt_ctas_per_sm(int variant, int nt, int m, int n_max, int LP) {
  const size_t smem = wsvt_smem(variant, m, n_max, LP);
  if (smem > 227 * 1024) return 0;
#define OCC(K)                                                              \
  do {                                                                      \
    if (wsvt_prepare_one(K, smem) != cudaSuccess) { (void)cudaGetLastError(); return 0; } \
    return wsvt_occupancy(K, nt, smem);                                     \
  } while (0)
  if (variant == 0) {
    if (nt == 128) OCC(k_wsvt_exact<128>);
    if (nt == 256) OCC(k_wsvt_exact<256>);
    if (nt == 512) OCC(k_wsvt_exact<512>);
  } else if (LP == 16) {
    if (nt == 128) OCC((k_wsvt_frsvt<128, 16>));
    if (nt == 256) OCC((k_wsvt_frsvt<256, 16>));
    if (nt == 512) OCC((k_wsvt_frsvt<512, 16>));
  } else {
    if (nt == 128) OCC((k_wsvt_frsvt<128, 32>));
    if (nt == 256) OCC((k_wsvt_frsvt<256, 32>));
    if (nt == 512) OCC((k_wsvt_frsvt<512, 32>));
  }
#undef OCC
  return 0;
}

cudaError_t launch_wsvt(int variant, int nt, int grid, int LP, const float* const* A, float* const* X,
                        const int32_t* n, int batch, int m, int n_max, float c, float eps, uint64_t seed,
                        uint64_t stream, int l, int q, double rank_tol, int max_sweeps, unsigned* next,
                        DevState* dst, cudaStream_t st) {
  WsvtArgs p{A, X, n, batch, m, n_max, c, eps, seed, stream, l, q, rank_tol, max_sweeps, next, dst};
  const size_t smem = wsvt_smem(variant, m, n_max, LP);
  cudaError_t e = cudaMemsetAsync(next, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
#define GO(K)                                  \
  do {                                         \
    e = wsvt_prepare_one(K, smem);             \
    if (e != cudaSuccess) return e;            \
    K<<<grid, nt, smem, st>>>(p);              \
    return cudaGetLastError();                 \
  } while (0)
  if (variant == 0) {
    if (nt == 128) GO(k_wsvt_exact<128>);
    if (nt == 256) GO(k_wsvt_exact<256>);
    if (nt == 512) GO(k_wsvt_exact<512>);
  } else if (LP == 16) {
    if (nt == 128) GO((k_wsvt_frsvt<128, 16>));
    if (nt == 256) GO((k_wsvt_frsvt<256, 16>));
    if (nt == 512) GO((k_wsvt_frsvt<512, 16>));
  } else {
    if (nt == 128) GO((k_wsvt_frsvt<128, 32>));
    if (nt == 256) GO((k_wsvt_frsvt<256, 32>));
    if (nt == 512) GO((k_wsvt_frsvt<512, 32>));
  }
#undef GO
  return cudaErrorInvalidValue;
}

}  // namespace frsvt
