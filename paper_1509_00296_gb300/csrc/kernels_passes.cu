// Streaming passes over the m x n iterate A (row-major, n <= m) on the CUDA cores.
//
// With the basis Q on the short side (n), Alg. 1 needs three kinds of pass
// over A (Table 2 lines 1, 3, 5, 8):
//   short_cols : Y = A^T B        (B = Omega for the sketch Y = A^T Omega, steps 4-5/8-9;
//                                  B = Z for the power step A^T (A Q), step 14)
//   long_rows  : Z = A Q          (power step and the projection B^T = A Q, step 16)
//   recon/alm  : X = Z Rf^T       (composition of Eq. 6), optionally fused with the
//                                  iALM sparse shrinkage and multiplier update
// Each pass reads A once with coalesced row accesses; the tall-skinny operands
// (Q, Z rows, Omega rows) are staged in shared memory.
#include "common.cuh"
#include "state.cuh"
#include "tma.cuh"

namespace frsvt {

namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 32;   // rows staged per shared-memory chunk

// ---------------------------------------------------------------- Y = A^T B (split over rows)
template <int LP, bool OMEGA>
__global__ void __launch_bounds__(kThreads)
k_short_cols(const float* __restrict__ A, int64_t m, int64_t n, int64_t lda,
             const float* __restrict__ Zl, uint64_t seed, uint64_t ctr_override,
             const DevState* __restrict__ dst, float* __restrict__ part, int64_t rps) {
  __shared__ __align__(16) float Bs[kChunk][LP];
  const int64_t j = static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x;
  const int64_t r0 = static_cast<int64_t>(blockIdx.y) * rps;
  const int64_t r1 = imin64(m, r0 + rps);
  uint64_t stream = 0;
  if (OMEGA) stream = (ctr_override == kCounterFromState) ? dst->counter : ctr_override;
  float acc[LP];
#pragma unroll
  for (int k = 0; k < LP; ++k) acc[k] = 0.f;

  for (int64_t i0 = r0; i0 < r1; i0 += kChunk) {
    const int nr = static_cast<int>(imin64(kChunk, r1 - i0));
    __syncthreads();
    if (OMEGA) {
      for (int t = threadIdx.x; t < kChunk * (LP / 4); t += kThreads) {
        const int rr = t / (LP / 4), blk = t % (LP / 4);
        float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
        if (rr < nr) g = gaussian4(seed, static_cast<uint64_t>(i0 + rr), static_cast<uint64_t>(blk), stream, 0ull);
        reinterpret_cast<float4*>(&Bs[rr][0])[blk] = g;
      }
    } else {
      for (int t = threadIdx.x; t < kChunk * LP; t += kThreads) {
        const int rr = t / LP, k = t % LP;
        Bs[rr][k] = (rr < nr) ? Zl[(i0 + rr) * LP + k] : 0.f;
      }
    }
    __syncthreads();
    if (j < n) {
      float a[kChunk];
#pragma unroll
      for (int rr = 0; rr < kChunk; ++rr) a[rr] = (rr < nr) ? __ldg(A + (i0 + rr) * lda + j) : 0.f;
#pragma unroll
      for (int rr = 0; rr < kChunk; ++rr) {
#pragma unroll
        for (int k4 = 0; k4 < LP / 4; ++k4) {
          const float4 b = reinterpret_cast<const float4*>(&Bs[rr][0])[k4];
          acc[4 * k4 + 0] = fmaf(a[rr], b.x, acc[4 * k4 + 0]);
          acc[4 * k4 + 1] = fmaf(a[rr], b.y, acc[4 * k4 + 1]);
          acc[4 * k4 + 2] = fmaf(a[rr], b.z, acc[4 * k4 + 2]);
          acc[4 * k4 + 3] = fmaf(a[rr], b.w, acc[4 * k4 + 3]);
        }
      }
    }
  }
  if (j < n) {
    float4* out = reinterpret_cast<float4*>(part + (static_cast<int64_t>(blockIdx.y) * n + j) * LP);
#pragma unroll
    for (int k4 = 0; k4 < LP / 4; ++k4)
      out[k4] = make_float4(acc[4 * k4], acc[4 * k4 + 1], acc[4 * k4 + 2], acc[4 * k4 + 3]);
  }
}

// ---------------------------------------------------------------- deterministic split-K reduction
__global__ void __launch_bounds__(kThreads)
k_reduce_parts(const float* __restrict__ part, int nsplit, int64_t count, float* __restrict__ Y) {
  const int64_t e = static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x;
  if (e >= count) return;
  float s = 0.f, c = 0.f;                      // Neumaier-compensated sum in split order
  for (int p = 0; p < nsplit; ++p) {
    const float v = part[static_cast<int64_t>(p) * count + e];
    const float t = s + v;
    c += (fabsf(s) >= fabsf(v)) ? ((s - t) + v) : ((v - t) + s);
    s = t;
  }
  Y[e] = s + c;
}

// ---------------------------------------------------------------- Z = A Q (warp per row group)
template <int LP, int R>
__global__ void __launch_bounds__(kThreads)
k_long_rows(const float* __restrict__ A, int64_t m, int64_t n, int64_t lda,
            const float* __restrict__ Q, float* __restrict__ Z) {
  extern __shared__ __align__(16) float Qs[];   // LP x n, k-major: Qs[k * n + j] = Q[j, k]
  for (int64_t t = threadIdx.x; t < n * LP; t += kThreads) {
    const int64_t jj = t / LP;
    const int k = static_cast<int>(t % LP);
    Qs[k * n + jj] = Q[t];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warp = (static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * kThreads) >> 5;
  for (int64_t i0 = warp * R; i0 < m; i0 += nwarps * R) {
    float acc[R][LP];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int k = 0; k < LP; ++k) acc[r][k] = 0.f;
    for (int64_t j = lane; j < n; j += 32) {
      float a[R];
#pragma unroll
      for (int r = 0; r < R; ++r) a[r] = (i0 + r < m) ? __ldg(A + (i0 + r) * lda + j) : 0.f;
#pragma unroll
      for (int k = 0; k < LP; ++k) {
        const float qk = Qs[k * n + j];
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r][k] = fmaf(a[r], qk, acc[r][k]);
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      float mine = 0.f;
#pragma unroll
      for (int k = 0; k < LP; ++k) {
        const float v = warp_sum(acc[r][k]);
        if (lane == k) mine = v;
      }
      if (lane < LP && i0 + r < m) Z[(i0 + r) * LP + lane] = mine;
    }
  }
}

// ---------------------------------------------------------------- Gram of Z (df64 partials)
template <int LP>
__global__ void __launch_bounds__(kThreads)
k_gram_long(const float* __restrict__ Z, int64_t m, float2* __restrict__ gpart, int64_t rps) {
  constexpr int NP = LP * (LP + 1) / 2;
  constexpr int PPT = (NP + kThreads - 1) / kThreads;
  __shared__ __align__(16) float Zs[kChunk][LP];
  __shared__ unsigned char pa[NP], pb[NP];
  if (threadIdx.x == 0) {
    int t = 0;
    for (int a = 0; a < LP; ++a)
      for (int b = a; b < LP; ++b) { pa[t] = static_cast<unsigned char>(a); pb[t] = static_cast<unsigned char>(b); ++t; }
  }
  __syncthreads();
  df64 acc[PPT];
#pragma unroll
  for (int u = 0; u < PPT; ++u) acc[u] = df64{0.f, 0.f};
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * rps;
  const int64_t r1 = imin64(m, r0 + rps);
  for (int64_t i0 = r0; i0 < r1; i0 += kChunk) {
    const int nr = static_cast<int>(imin64(kChunk, r1 - i0));
    __syncthreads();
    for (int t = threadIdx.x; t < kChunk * LP; t += kThreads) {
      const int rr = t / LP, k = t % LP;
      Zs[rr][k] = (rr < nr) ? Z[(i0 + rr) * LP + k] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < PPT; ++u) {
      const int pr = threadIdx.x + u * kThreads;
      if (pr < NP) {
        const int a = pa[pr], b = pb[pr];
        for (int rr = 0; rr < nr; ++rr) df64_add_prod(acc[u], Zs[rr][a], Zs[rr][b]);
      }
    }
  }
#pragma unroll
  for (int u = 0; u < PPT; ++u) {
    const int pr = threadIdx.x + u * kThreads;
    if (pr < NP) {
      const int a = pa[pr], b = pb[pr];
      float2* g = gpart + static_cast<int64_t>(blockIdx.x) * LP * LP;
      g[a * LP + b] = make_float2(acc[u].hi, acc[u].lo);
      g[b * LP + a] = make_float2(acc[u].hi, acc[u].lo);
    }
  }
}

// ---------------------------------------------------------------- X = Z Rf^T
template <int LP>
__global__ void __launch_bounds__(kThreads)
k_recon(const float* __restrict__ Z, const float* __restrict__ Rf, int64_t m, int64_t n,
        float* __restrict__ X, int64_t ldx, int64_t rps) {
  __shared__ __align__(16) float Zs[kChunk][LP];
  const int64_t j = static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x;
  const int64_t r0 = static_cast<int64_t>(blockIdx.y) * rps;
  const int64_t r1 = imin64(m, r0 + rps);
  float rf[LP];
#pragma unroll
  for (int k = 0; k < LP; ++k) rf[k] = (j < n) ? Rf[j * LP + k] : 0.f;
  for (int64_t i0 = r0; i0 < r1; i0 += kChunk) {
    const int nr = static_cast<int>(imin64(kChunk, r1 - i0));
    __syncthreads();
    for (int t = threadIdx.x; t < kChunk * LP; t += kThreads) {
      const int rr = t / LP, k = t % LP;
      Zs[rr][k] = (rr < nr) ? Z[(i0 + rr) * LP + k] : 0.f;
    }
    __syncthreads();
    if (j < n) {
      for (int rr = 0; rr < nr; ++rr) {
        float x = 0.f;
#pragma unroll
        for (int k4 = 0; k4 < LP / 4; ++k4) {
          const float4 z = reinterpret_cast<const float4*>(&Zs[rr][0])[k4];
          x = fmaf(z.x, rf[4 * k4], x);
          x = fmaf(z.y, rf[4 * k4 + 1], x);
          x = fmaf(z.z, rf[4 * k4 + 2], x);
          x = fmaf(z.w, rf[4 * k4 + 3], x);
        }
        X[(i0 + rr) * ldx + j] = x;
      }
    }
  }
}

// ---------------------------------------------------------------- fused reconstruction + iALM update
template <int LP>
__global__ void __launch_bounds__(kThreads)
k_alm(const float* __restrict__ Z, const float* __restrict__ Rf, const float* __restrict__ O,
      float* __restrict__ S, float* __restrict__ A, int64_t m, int64_t n, int64_t ld,
      float* __restrict__ L, int64_t ldl, const DevState* __restrict__ dst,
      float2* __restrict__ rpart, int64_t rps) {
  __shared__ __align__(16) float Zs[kChunk][LP];
  __shared__ double red[kThreads / 32];
  const int64_t j = static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x;
  const int64_t r0 = static_cast<int64_t>(blockIdx.y) * rps;
  const int64_t r1 = imin64(m, r0 + rps);
  const double mu = dst->mu;
  const double mu_next = fmin(dst->rho * mu, dst->mu_bar);
  const float thr = static_cast<float>(dst->lambda / mu);
  const float ratio = static_cast<float>(mu / mu_next);
  float rf[LP];
#pragma unroll
  for (int k = 0; k < LP; ++k) rf[k] = (j < n) ? Rf[j * LP + k] : 0.f;
  float res2 = 0.f;
  for (int64_t i0 = r0; i0 < r1; i0 += kChunk) {
    const int nr = static_cast<int>(imin64(kChunk, r1 - i0));
    __syncthreads();
    for (int t = threadIdx.x; t < kChunk * LP; t += kThreads) {
      const int rr = t / LP, k = t % LP;
      Zs[rr][k] = (rr < nr) ? Z[(i0 + rr) * LP + k] : 0.f;
    }
    __syncthreads();
    if (j < n) {
      for (int rr = 0; rr < nr; ++rr) {
        float x = 0.f;
#pragma unroll
        for (int k4 = 0; k4 < LP / 4; ++k4) {
          const float4 z = reinterpret_cast<const float4*>(&Zs[rr][0])[k4];
          x = fmaf(z.x, rf[4 * k4], x);
          x = fmaf(z.y, rf[4 * k4 + 1], x);
          x = fmaf(z.z, rf[4 * k4 + 2], x);
          x = fmaf(z.w, rf[4 * k4 + 3], x);
        }
        const int64_t idx = (i0 + rr) * ld + j;
        const float o = __ldg(O + idx);
        const float s = S[idx];
        const float a = A[idx];
        const float t = a + s - x;                                   // O - L + Y/mu
        const float sn = (t > thr) ? (t - thr) : ((t < -thr) ? (t + thr) : 0.f);
        const float an = o - sn + ratio * (t - sn);                  // O - S' + Y'/mu'
        const float rz = o - x - sn;                                 // Z = O - L - S'
        res2 = fmaf(rz, rz, res2);
        S[idx] = sn;
        A[idx] = an;
        if (L != nullptr) L[(i0 + rr) * ldl + j] = x;
      }
    }
  }
  double v = warp_sum(static_cast<double>(res2));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    const float hi = static_cast<float>(t);
    rpart[static_cast<int64_t>(blockIdx.y) * gridDim.x + blockIdx.x] =
        make_float2(hi, static_cast<float>(t - static_cast<double>(hi)));
  }
}

// ---------------------------------------------------------------- rpca_init helpers
__global__ void __launch_bounds__(kThreads)
k_absmax_sumsq(const float* __restrict__ O, int64_t m, int64_t n, int64_t ld,
               float* __restrict__ pmax, float2* __restrict__ psum) {
  __shared__ float smax[kThreads / 32];
  __shared__ double ssum[kThreads / 32];
  float mx = 0.f, sq = 0.f;
  const int64_t total = m * n;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * kThreads) {
    const int64_t i = e / n, jj = e % n;
    const float v = O[i * ld + jj];
    mx = fmaxf(mx, fabsf(v));
    sq = fmaf(v, v, sq);
  }
  double d = warp_sum(static_cast<double>(sq));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) { smax[threadIdx.x >> 5] = mx; ssum[threadIdx.x >> 5] = d; }
  __syncthreads();
  if (threadIdx.x == 0) {
    float M = 0.f;
    double T = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) { M = fmaxf(M, smax[w]); T += ssum[w]; }
    pmax[blockIdx.x] = M;
    const float hi = static_cast<float>(T);
    psum[blockIdx.x] = make_float2(hi, static_cast<float>(T - static_cast<double>(hi)));
  }
}

__global__ void __launch_bounds__(kThreads)
k_init_state(const float* __restrict__ O, float* __restrict__ S, float* __restrict__ A,
             int64_t m, int64_t n, int64_t ld, const DevState* __restrict__ dst) {
  const float c = static_cast<float>(dst->init_scale);
  const int64_t total = m * n;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * kThreads) {
    const int64_t i = e / n, jj = e % n;
    const float v = O[i * ld + jj];
    S[i * ld + jj] = 0.f;
    A[i * ld + jj] = c * v;
  }
}

// ---------------------------------------------------------------- debug: Omega / raw Philox
__global__ void k_debug_omega(float* out, int64_t rows, int cols, uint64_t seed, uint64_t stream,
                              uint64_t problem) {
  const int nblk = (cols + 3) / 4;
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= rows * nblk) return;
  const int64_t i = t / nblk;
  const int blk = static_cast<int>(t % nblk);
  const float4 g = gaussian4(seed, static_cast<uint64_t>(i), static_cast<uint64_t>(blk), stream, problem);
  const float v[4] = {g.x, g.y, g.z, g.w};
  for (int k = 0; k < 4; ++k)
    if (4 * blk + k < cols) out[i * cols + 4 * blk + k] = v[k];
}

__global__ void k_debug_philox(uint64_t* out, int64_t rows, int blocks, uint64_t seed, uint64_t stream,
                               uint64_t problem) {
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= rows * blocks) return;
  const u64x4 w = philox4x64_10(u64x4{static_cast<uint64_t>(t / blocks), static_cast<uint64_t>(t % blocks),
                                      stream, problem}, seed, 0ull);
  out[4 * t + 0] = w.x;
  out[4 * t + 1] = w.y;
  out[4 * t + 2] = w.z;
  out[4 * t + 3] = w.w;
}

inline unsigned grid_1d(int64_t work, int per_block, int cap) {
  int64_t g = (work + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return static_cast<unsigned>(g);
}

}  // namespace

// ---------------------------------------------------------------- launchers
cudaError_t launch_short_cols(int LP, const float* A, int64_t m, int64_t n, int64_t lda, const float* Zl,
                              uint64_t seed, uint64_t ctr, const DevState* dst, float* part, int nsplit,
                              int64_t rps, cudaStream_t st) {
  dim3 grid(static_cast<unsigned>((n + kThreads - 1) / kThreads), static_cast<unsigned>(nsplit));
  if (LP == 16) {
    if (Zl) k_short_cols<16, false><<<grid, kThreads, 0, st>>>(A, m, n, lda, Zl, seed, ctr, dst, part, rps);
    else k_short_cols<16, true><<<grid, kThreads, 0, st>>>(A, m, n, lda, Zl, seed, ctr, dst, part, rps);
  } else {
    if (Zl) k_short_cols<32, false><<<grid, kThreads, 0, st>>>(A, m, n, lda, Zl, seed, ctr, dst, part, rps);
    else k_short_cols<32, true><<<grid, kThreads, 0, st>>>(A, m, n, lda, Zl, seed, ctr, dst, part, rps);
  }
  return cudaGetLastError();
}

cudaError_t launch_reduce_parts(const float* part, int nsplit, int64_t count, float* Y, cudaStream_t st) {
  k_reduce_parts<<<grid_1d(count, kThreads, 1 << 20), kThreads, 0, st>>>(part, nsplit, count, Y);
  return cudaGetLastError();
}

cudaError_t launch_long_rows(int LP, const float* A, int64_t m, int64_t n, int64_t lda, const float* Q,
                             float* Z, int grid_cap, cudaStream_t st) {
  constexpr int R = 4;
  const size_t smem = static_cast<size_t>(n) * LP * sizeof(float);
  const unsigned grid = grid_1d(m, (kThreads / 32) * R, grid_cap);
  if (LP == 16) k_long_rows<16, R><<<grid, kThreads, smem, st>>>(A, m, n, lda, Q, Z);
  else k_long_rows<32, R><<<grid, kThreads, smem, st>>>(A, m, n, lda, Q, Z);
  return cudaGetLastError();
}

cudaError_t prepare_pass_kernels(int smem_limit) {
  cudaError_t e = cudaFuncSetAttribute(k_long_rows<16, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_limit);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_long_rows<32, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_limit);
}

cudaError_t launch_gram_long(int LP, const float* Z, int64_t m, float2* gpart, int gsplit, cudaStream_t st) {
  int64_t rps = (m + gsplit - 1) / gsplit;
  if (rps < 1) rps = 1;
  if (LP == 16) k_gram_long<16><<<gsplit, kThreads, 0, st>>>(Z, m, gpart, rps);
  else k_gram_long<32><<<gsplit, kThreads, 0, st>>>(Z, m, gpart, rps);
  return cudaGetLastError();
}

cudaError_t launch_recon(int LP, const float* Z, const float* Rf, int64_t m, int64_t n, float* X, int64_t ldx,
                         int nsplit, int64_t rps, cudaStream_t st) {
  dim3 grid(static_cast<unsigned>((n + kThreads - 1) / kThreads), static_cast<unsigned>(nsplit));
  if (LP == 16) k_recon<16><<<grid, kThreads, 0, st>>>(Z, Rf, m, n, X, ldx, rps);
  else k_recon<32><<<grid, kThreads, 0, st>>>(Z, Rf, m, n, X, ldx, rps);
  return cudaGetLastError();
}

cudaError_t launch_alm(int LP, const float* Z, const float* Rf, const float* O, float* S, float* A, int64_t m,
                       int64_t n, int64_t ld, float* L, int64_t ldl, const DevState* dst, float2* rpart,
                       int nsplit, int64_t rps, cudaStream_t st) {
  dim3 grid(static_cast<unsigned>((n + kThreads - 1) / kThreads), static_cast<unsigned>(nsplit));
  if (LP == 16) k_alm<16><<<grid, kThreads, 0, st>>>(Z, Rf, O, S, A, m, n, ld, L, ldl, dst, rpart, rps);
  else k_alm<32><<<grid, kThreads, 0, st>>>(Z, Rf, O, S, A, m, n, ld, L, ldl, dst, rpart, rps);
  return cudaGetLastError();
}

cudaError_t launch_absmax_sumsq(const float* O, int64_t m, int64_t n, int64_t ld, float* pmax, float2* psum,
                                int nblk, cudaStream_t st) {
  k_absmax_sumsq<<<nblk, kThreads, 0, st>>>(O, m, n, ld, pmax, psum);
  return cudaGetLastError();
}

cudaError_t launch_init_state(const float* O, float* S, float* A, int64_t m, int64_t n, int64_t ld,
                              const DevState* dst, cudaStream_t st) {
  k_init_state<<<grid_1d(m * n, kThreads, 4096), kThreads, 0, st>>>(O, S, A, m, n, ld, dst);
  return cudaGetLastError();
}

cudaError_t launch_debug_omega(float* out, int64_t rows, int cols, uint64_t seed, uint64_t stream,
                               uint64_t problem, cudaStream_t st) {
  const int64_t work = rows * ((cols + 3) / 4);
  k_debug_omega<<<grid_1d(work, 256, 1 << 30), 256, 0, st>>>(out, rows, cols, seed, stream, problem);
  return cudaGetLastError();
}

cudaError_t launch_debug_philox(uint64_t* out, int64_t rows, int blocks, uint64_t seed, uint64_t stream,
                                uint64_t problem, cudaStream_t st) {
  k_debug_philox<<<grid_1d(rows * blocks, 256, 1 << 30), 256, 0, st>>>(out, rows, blocks, seed, stream, problem);
  return cudaGetLastError();
}

// One thread initialises an mbarrier that expects one arrival, which nothing ever makes, and
// waits on it with the bounded poll every pipeline wait of the library uses (here with a caller-
// chosen limit).  When the wait gives up the kernel records kDevTimeout and returns: no copy is
// in flight and no tensor memory is held, so the context stays usable.
__global__ void k_debug_wait_timeout(uint32_t spin_limit, DevState* __restrict__ dst) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  fence_mbar_init();
  if (!mbar_wait_n(&bar, 0u, spin_limit)) atomicOr(&dst->status, kDevTimeout);
}

cudaError_t launch_debug_wait_timeout(uint32_t spin_limit, DevState* dst, cudaStream_t st) {
  k_debug_wait_timeout<<<1, 32, 0, st>>>(spin_limit, dst);
  return cudaGetLastError();
}

}  // namespace frsvt
