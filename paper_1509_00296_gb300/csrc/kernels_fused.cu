// Fused streaming passes for a short side that fits one CTA's shared memory.
//
// Each pass over A ends with a split-K reduction of a small result (Y = A^T B,
// the Gram Z^T Z, or the iALM residual).  The CTAs of a pass form thread-block
// clusters of kCL; a cluster sums its members' partials through distributed
// shared memory, the cluster that finishes last (an atomic ticket, no
// spin-wait) sums the cluster partials in a fixed order, and the CTA of rank 0
// of that last cluster then runs the small dense step that depends on the sum:
//   sketch / power pass -> orthonormal basis        (Alg. 1 steps 6, 10-11, 14)
//   projection pass     -> SVD of B, shrinkage, M    (steps 16-21, Eq. 6)
//   iALM epilogue       -> residual and mu update    (Sec. 4.1)
// so one iALM iteration needs 3 + 2q launches and no separate small kernels.
#include <cooperative_groups.h>

#include "cluster.cuh"
#include "common.cuh"
#include "small_dense.cuh"
#include "state.cuh"

namespace cg = cooperative_groups;

namespace frsvt {

namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 32;
constexpr int kGacc = 1024;         // double-float partial slots of the small routines

// ---------------------------------------------------------------- Y = A^T B, cluster reduce, orth tail
template <int LP, bool OMEGA>
__global__ void __cluster_dims__(1, kCL, 1) __launch_bounds__(kThreads)
k_sc_orth(const float* __restrict__ A, int64_t m, int64_t n, int64_t lda, const float* __restrict__ Zl,
          uint64_t seed, uint64_t ctr_override, DevState* __restrict__ dst, int64_t rps,
          float* __restrict__ cpart, float* __restrict__ Y, unsigned* __restrict__ tickets, int l, int use_rp,
          const float* __restrict__ Qt, float* __restrict__ Qout, double rank_tol) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ __align__(16) float Bs[kChunk][LP];
  __shared__ int flag;
  float* part_sm = reinterpret_cast<float*>(dsm);           // kThreads x LP, then reused by the tail
  const int tile = blockIdx.x;
  const int64_t j = static_cast<int64_t>(tile) * kThreads + threadIdx.x;
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
#pragma unroll
  for (int k = 0; k < LP; ++k) part_sm[threadIdx.x * LP + k] = acc[k];
  // columns of this tile that exist
  const int tile_cols = static_cast<int>(imin64(kThreads, n - static_cast<int64_t>(tile) * kThreads));
  const int count = tile_cols * LP;
  const int nclusters = gridDim.y / kCL;
  const int cl_idx = blockIdx.y / kCL;
  float* cp = cpart + static_cast<int64_t>(tile) * nclusters * kThreads * LP;
  float* Yt = Y + static_cast<int64_t>(tile) * kThreads * LP;
  if (!cluster_split_reduce<float>(part_sm, count, cp, Yt, tickets + tile, cl_idx, nclusters, &flag)) return;
  if (cg::this_cluster().block_rank() != 0) return;
  if (!last_of(tickets + gridDim.x, gridDim.x, &flag)) return;
  // tail: orthonormal basis of Y (this CTA alone)
  SmallWs<LP> w = carve_small_ws<LP>(dsm, kGacc);
  int keep = use_rp ? dst->keep : 0;
  keep = max(0, min(keep, l));
  load_basis_block<LP>(w.W, static_cast<int>(n), keep, l, Qt, Y);
  __syncthreads();
  float rp_res = -1.f;
  const int s = orth_block<LP>(w, n, keep, l, rank_tol, 2, &rp_res, &dst->status);
  for (int64_t e = threadIdx.x; e < n * LP; e += kThreads) Qout[e] = w.W[e];
  if (threadIdx.x == 0) {
    if (use_rp) dst->rp_res = rp_res;
    dst->s = s;
    if (s < l) dst->status |= kDevRankDeficient;
  }
}

// ---------------------------------------------------------------- Z = A Q (+ Gram, cluster reduce, core tail)
template <int LP, int R, bool GRAM>
__global__ void __cluster_dims__(kCL, 1, 1) __launch_bounds__(kThreads)
k_lr(const float* __restrict__ A, int64_t m, int64_t n, int64_t lda, const float* __restrict__ Q,
     float* __restrict__ Z, double* __restrict__ cpart, double* __restrict__ Gout, unsigned* __restrict__ tickets,
     int l, float tau_host, int tau_from_mu, int update_rp, int advance_counter, float* __restrict__ Rf,
     float* __restrict__ Qt, DevState* __restrict__ dst, double rank_tol, int max_sweeps) {
  constexpr int NP = LP * (LP + 1) / 2;
  constexpr int PPL = (NP + 31) / 32;
  extern __shared__ __align__(16) unsigned char dsm[];
  float* Qs = reinterpret_cast<float*>(dsm);                   // LP x n, k-major
  __shared__ float zrow[kThreads / 32][R][LP];
  __shared__ double gsm[NP];
  __shared__ unsigned char pa[NP], pb[NP];
  __shared__ int flag;
  for (int64_t t = threadIdx.x; t < n * LP; t += kThreads) {
    const int64_t jj = t / LP;
    const int k = static_cast<int>(t % LP);
    Qs[k * n + jj] = Q[t];
  }
  if (GRAM)
    for (int t = threadIdx.x; t < NP; t += kThreads) {
      int a, b;
      decode_pair_sym(t, LP, a, b);
      pa[t] = static_cast<unsigned char>(a);
      pb[t] = static_cast<unsigned char>(b);
    }
  __syncthreads();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t warp = (static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * kThreads) >> 5;
  df64 g[PPL];
#pragma unroll
  for (int u = 0; u < PPL; ++u) g[u] = df64{0.f, 0.f};
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
      if (lane < LP) {
        if (i0 + r < m) Z[(i0 + r) * LP + lane] = mine;
        if (GRAM) zrow[wib][r][lane] = (i0 + r < m) ? mine : 0.f;
      }
    }
    if (GRAM) {
      __syncwarp();
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int u = 0; u < PPL; ++u) {
          const int pr = lane + 32 * u;
          if (pr < NP) df64_add_prod(g[u], zrow[wib][r][pa[pr]], zrow[wib][r][pb[pr]]);
        }
      __syncwarp();
    }
  }
  if (!GRAM) return;
  // deterministic combination of the 8 warps' partials (warp order), in the dynamic buffer
  __syncthreads();
  double* gw = reinterpret_cast<double*>(dsm);                 // (kThreads / 32) x NP
#pragma unroll
  for (int u = 0; u < PPL; ++u) {
    const int pr = lane + 32 * u;
    if (pr < NP) gw[wib * NP + pr] = df64_value(g[u]);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < NP; t += kThreads) {
    double sum = 0.0;
    for (int w2 = 0; w2 < kThreads / 32; ++w2) sum += gw[w2 * NP + t];
    gsm[t] = sum;
  }
  const int nclusters = gridDim.x / kCL;
  const int cl_idx = blockIdx.x / kCL;
  if (!cluster_split_reduce<double>(gsm, NP, cpart, Gout, tickets, cl_idx, nclusters, &flag)) return;
  if (cg::this_cluster().block_rank() != 0) return;
  // tail: core SVD of B (this CTA alone)
  SmallWs<LP> w = carve_small_ws<LP>(dsm, kGacc);
  for (int e = threadIdx.x; e < LP * LP; e += kThreads) {
    const int a = e / LP, b = e % LP;
    double v = 0.0;
    if (a < l && b < l) {
      const int lo = a < b ? a : b, hi = a < b ? b : a;
      v = __ldcg(Gout + (lo * LP - lo * (lo - 1) / 2 + (hi - lo)));
    }
    w.G[e] = df_from_double(v);
  }
  __syncthreads();
  const float tau = tau_from_mu ? static_cast<float>(1.0 / dst->mu) : tau_host;
  core_block<LP>(w, Q, n, l, tau, update_rp, advance_counter, Rf, Qt, dst, rank_tol, max_sweeps);
}

// ---------------------------------------------------------------- fused reconstruction + iALM update
// Tile of up to 256 columns per blockIdx.x; threads = column quads x row groups.
template <int LP>
__global__ void __cluster_dims__(1, kCL, 1) __launch_bounds__(kThreads)
k_alm2(const float* __restrict__ Z, const float* __restrict__ Rf, const float* __restrict__ O,
       float* __restrict__ S, float* __restrict__ A, int64_t m, int64_t n, int64_t ld, float* __restrict__ L,
       int64_t ldl, DevState* __restrict__ dst, int64_t rps, double* __restrict__ cpart,
       double* __restrict__ rsum, unsigned* __restrict__ tickets) {
  __shared__ double red[kThreads / 32];
  __shared__ int flag;
  const int tile = blockIdx.x;
  const int64_t c0 = static_cast<int64_t>(tile) * 256;
  const int tcols = static_cast<int>(imin64(256, n - c0));
  const int nq = (tcols + 3) / 4;
  const int rgc = kThreads / nq;
  const int qd = threadIdx.x % nq;
  const int rg = threadIdx.x / nq;
  const bool active = rg < rgc;
  const int64_t col = c0 + 4 * qd;
  const double mu = dst->mu;
  const double mu_next = fmin(dst->rho * mu, dst->mu_bar);
  const float thr = static_cast<float>(dst->lambda / mu);
  const float ratio = static_cast<float>(mu / mu_next);
  float rf[4][LP];
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int k = 0; k < LP; ++k) rf[c][k] = (active && col + c < n) ? Rf[(col + c) * LP + k] : 0.f;
  const int64_t r0 = static_cast<int64_t>(blockIdx.y) * rps;
  const int64_t r1 = imin64(m, r0 + rps);
  float res2 = 0.f;
  const bool full = active && (col + 3 < n);
  if (active) {
    for (int64_t i = r0 + rg; i < r1; i += rgc) {
      float z[LP];
#pragma unroll
      for (int k4 = 0; k4 < LP / 4; ++k4) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(Z + i * LP) + k4);
        z[4 * k4] = v.x;
        z[4 * k4 + 1] = v.y;
        z[4 * k4 + 2] = v.z;
        z[4 * k4 + 3] = v.w;
      }
      float x[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float t = 0.f;
#pragma unroll
        for (int k = 0; k < LP; ++k) t = fmaf(z[k], rf[c][k], t);
        x[c] = t;
      }
      const int64_t idx = i * ld + col;
      float ov[4] = {0.f, 0.f, 0.f, 0.f}, sv[4] = {0.f, 0.f, 0.f, 0.f}, av[4] = {0.f, 0.f, 0.f, 0.f};
      if (full) {
        const float4 o4 = __ldg(reinterpret_cast<const float4*>(O + idx));
        const float4 s4 = *reinterpret_cast<const float4*>(S + idx);
        const float4 a4 = *reinterpret_cast<const float4*>(A + idx);
        ov[0] = o4.x; ov[1] = o4.y; ov[2] = o4.z; ov[3] = o4.w;
        sv[0] = s4.x; sv[1] = s4.y; sv[2] = s4.z; sv[3] = s4.w;
        av[0] = a4.x; av[1] = a4.y; av[2] = a4.z; av[3] = a4.w;
      } else {
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (col + c < n) {       // the ragged last quad: never read past column n - 1
            ov[c] = __ldg(O + idx + c);
            sv[c] = S[idx + c];
            av[c] = A[idx + c];
          }
      }
      float sn[4], an[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float t = av[c] + sv[c] - x[c];                        // O - L + Y/mu
        sn[c] = (t > thr) ? (t - thr) : ((t < -thr) ? (t + thr) : 0.f);
        an[c] = ov[c] - sn[c] + ratio * (t - sn[c]);                  // O - S' + Y'/mu'
        const float rz = ov[c] - x[c] - sn[c];                        // O - L - S'
        if (col + c < n) res2 = fmaf(rz, rz, res2);
      }
      if (full) {
        *reinterpret_cast<float4*>(S + idx) = make_float4(sn[0], sn[1], sn[2], sn[3]);
        *reinterpret_cast<float4*>(A + idx) = make_float4(an[0], an[1], an[2], an[3]);
        if (L != nullptr) *reinterpret_cast<float4*>(L + i * ldl + col) = make_float4(x[0], x[1], x[2], x[3]);
      } else {
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (col + c < n) {
            S[idx + c] = sn[c];
            A[idx + c] = an[c];
            if (L != nullptr) L[i * ldl + col + c] = x[c];
          }
      }
    }
  }
  const double v = warp_sum(static_cast<double>(res2));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  __shared__ double mine;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    mine = t;
  }
  const int nclusters = gridDim.y / kCL;
  const int cl_idx = blockIdx.y / kCL;
  double* cp = cpart + static_cast<int64_t>(tile) * nclusters;
  if (!cluster_split_reduce<double>(&mine, 1, cp, rsum + tile, tickets + tile, cl_idx, nclusters, &flag)) return;
  if (cg::this_cluster().block_rank() != 0) return;
  if (!last_of(tickets + gridDim.x, gridDim.x, &flag)) return;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (unsigned t = 0; t < gridDim.x; ++t) s += __ldcg(rsum + t);
    const double rr = (dst->normO_F > 0.0) ? sqrt(s) / dst->normO_F : 0.0;
    dst->resid_ratio = rr;
    if (!isfinite(rr)) dst->status |= kDevNonfinite;
    dst->mu = mu_next;
    dst->iter += 1;
  }
}

}  // namespace

size_t fused_orth_smem(int LP, int64_t ns) {
  const size_t part = static_cast<size_t>(kThreads) * LP * sizeof(float);
  const size_t ws = LP == 16 ? small_ws_bytes<16>(ns, kGacc) : small_ws_bytes<32>(ns, kGacc);
  return part > ws ? part : ws;
}

size_t fused_core_smem(int LP, int64_t ns) {
  const size_t q = static_cast<size_t>(ns) * LP * sizeof(float);
  const size_t ws = LP == 16 ? small_ws_bytes<16>(0, kGacc) : small_ws_bytes<32>(0, kGacc);
  const size_t gw = static_cast<size_t>(kThreads / 32) * (LP * (LP + 1) / 2) * sizeof(double);
  size_t b = q > ws ? q : ws;
  return b > gw ? b : gw;
}

// The dynamic limit of a kernel is the per-block maximum minus its static shared memory.
template <typename K>
cudaError_t set_dynamic_limit(K kernel, int smem_limit) {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              smem_limit - static_cast<int>(a.sharedSizeBytes));
}

cudaError_t prepare_fused_kernels(int smem_limit) {
  cudaError_t e = cudaSuccess;
#define PREP(k) \
  if (e == cudaSuccess) e = set_dynamic_limit(k, smem_limit);
  PREP((k_sc_orth<16, true>));
  PREP((k_sc_orth<16, false>));
  PREP((k_sc_orth<32, true>));
  PREP((k_sc_orth<32, false>));
  PREP((k_lr<16, 4, true>));
  PREP((k_lr<16, 4, false>));
  PREP((k_lr<32, 2, true>));
  PREP((k_lr<32, 2, false>));
#undef PREP
  return e;
}

cudaError_t launch_sc_orth(int LP, const float* A, int64_t m, int64_t n, int64_t lda, const float* Zl, uint64_t seed,
                           uint64_t ctr, DevState* dst, int nsplit, int64_t rps, float* cpart, float* Y,
                           unsigned* tickets, int l, int use_rp, const float* Qt, float* Q, double rank_tol,
                           cudaStream_t st) {
  dim3 grid(static_cast<unsigned>((n + kThreads - 1) / kThreads), static_cast<unsigned>(nsplit));
  const size_t smem = fused_orth_smem(LP, n);
  if (LP == 16) {
    if (Zl) k_sc_orth<16, false><<<grid, kThreads, smem, st>>>(A, m, n, lda, Zl, seed, ctr, dst, rps, cpart, Y,
                                                              tickets, l, use_rp, Qt, Q, rank_tol);
    else k_sc_orth<16, true><<<grid, kThreads, smem, st>>>(A, m, n, lda, Zl, seed, ctr, dst, rps, cpart, Y, tickets,
                                                          l, use_rp, Qt, Q, rank_tol);
  } else {
    if (Zl) k_sc_orth<32, false><<<grid, kThreads, smem, st>>>(A, m, n, lda, Zl, seed, ctr, dst, rps, cpart, Y,
                                                              tickets, l, use_rp, Qt, Q, rank_tol);
    else k_sc_orth<32, true><<<grid, kThreads, smem, st>>>(A, m, n, lda, Zl, seed, ctr, dst, rps, cpart, Y, tickets,
                                                          l, use_rp, Qt, Q, rank_tol);
  }
  return cudaGetLastError();
}

cudaError_t launch_lr(int LP, bool gram, const float* A, int64_t m, int64_t n, int64_t lda, const float* Q, float* Z,
                      int nblocks, double* cpart, double* G, unsigned* tickets, int l, float tau_host,
                      int tau_from_mu, int update_rp, int advance_counter, float* Rf, float* Qt, DevState* dst,
                      double rank_tol, int max_sweeps, cudaStream_t st) {
  const size_t smem = fused_core_smem(LP, n);
#define ARGS A, m, n, lda, Q, Z, cpart, G, tickets, l, tau_host, tau_from_mu, update_rp, advance_counter, Rf, Qt, \
             dst, rank_tol, max_sweeps
  if (LP == 16) {
    if (gram) k_lr<16, 4, true><<<nblocks, kThreads, smem, st>>>(ARGS);
    else k_lr<16, 4, false><<<nblocks, kThreads, smem, st>>>(ARGS);
  } else {
    if (gram) k_lr<32, 2, true><<<nblocks, kThreads, smem, st>>>(ARGS);
    else k_lr<32, 2, false><<<nblocks, kThreads, smem, st>>>(ARGS);
  }
#undef ARGS
  return cudaGetLastError();
}

cudaError_t launch_alm2(int LP, const float* Z, const float* Rf, const float* O, float* S, float* A, int64_t m,
                        int64_t n, int64_t ld, float* L, int64_t ldl, DevState* dst, int nsplit, int64_t rps,
                        double* cpart, double* rsum, unsigned* tickets, cudaStream_t st) {
  dim3 grid(static_cast<unsigned>((n + 255) / 256), static_cast<unsigned>(nsplit));
  if (LP == 16) k_alm2<16><<<grid, kThreads, 0, st>>>(Z, Rf, O, S, A, m, n, ld, L, ldl, dst, rps, cpart, rsum, tickets);
  else k_alm2<32><<<grid, kThreads, 0, st>>>(Z, Rf, O, S, A, m, n, ld, L, ldl, dst, rps, cpart, rsum, tickets);
  return cudaGetLastError();
}

}  // namespace frsvt
