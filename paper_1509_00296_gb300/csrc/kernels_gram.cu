// Gram matrix of the projection and the l x l core of Alg. 1 (steps 16-19) from Z = A Q.
//
// After the tensor-core row pass has written Z = A Q = B^T (m x LP, L2-resident), this kernel
// forms B B^T = Z^T Z in double-float arithmetic: each thread owns Gram entries (a, b) of the
// packed upper triangle and a residue class of rows, and adds the exact products
// Z[r][a] Z[r][b] (df64_add_prod) over the rows of its CTA, staged tile by tile in shared
// memory.  The per-CTA partials go through the cluster split-K reduction (cluster.cuh); the
// CTA that finishes it last runs the core (small_dense.cuh: Cholesky-preconditioned one-sided
// Jacobi SVD of B, soft thresholding, factors for the reconstruction and range propagation).
#include "cluster.cuh"
#include "common.cuh"
#include "small_dense.cuh"
#include "state.cuh"

namespace frsvt {

namespace {

constexpr int kGThr = 512;
constexpr int kGRows = 1024;      // rows of Z staged per tile (dynamic shared memory)
constexpr int kGaccG = 1024;

template <int LP>
__global__ void __cluster_dims__(kCL, 1, 1) __launch_bounds__(kGThr, 1)
k_gram_core(const float* __restrict__ Z, int64_t m, int n, int64_t rpc, const float* __restrict__ Q,
            double* __restrict__ cpart, double* __restrict__ Gout, unsigned* __restrict__ tickets, int l,
            float tau_host, int tau_from_mu, int update_rp, int advance_counter, float* __restrict__ Rf,
            float* __restrict__ Qt, DevState* __restrict__ dst, double rank_tol, int max_sweeps) {
  if (l <= 0) l = min(max(dst->l_cur, 1), LP);            // adaptive rank prediction: l lives on the device
  constexpr int NP = LP * (LP + 1) / 2;
  constexpr int PPT = (NP + kGThr - 1) / kGThr;                   // pairs per thread
  constexpr int RG = (kGThr / NP) > 0 ? (kGThr / NP) : 1;         // row classes
  extern __shared__ __align__(16) unsigned char dsm[];
  float (*zt)[LP] = reinterpret_cast<float (*)[LP]>(dsm);        // kGRows x LP, reused by the core
  __shared__ double gpart[RG][NP];
  __shared__ int flag;
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * rpc;
  const int64_t r1 = imin64(m, r0 + rpc);
  // thread t: pairs t % NP (+ kGThr ...), row class t / NP
  const int rg = (PPT == 1) ? static_cast<int>(threadIdx.x) / NP : 0;
  int pa[PPT], pb[PPT];
#pragma unroll
  for (int u = 0; u < PPT; ++u) {
    const int pr = (PPT == 1) ? static_cast<int>(threadIdx.x) % NP : static_cast<int>(threadIdx.x) + kGThr * u;
    pa[u] = pb[u] = -1;
    if (pr < NP && rg < RG) decode_pair_sym(pr, LP, pa[u], pb[u]);
  }
  // four independent accumulators per pair (rows rr, rr + RG, rr + 2 RG, rr + 3 RG) break the
  // dependence chain of the double-float additions; the staged tile is zero-padded.
  df64 g[PPT][4];
#pragma unroll
  for (int u = 0; u < PPT; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) g[u][v] = df64{0.f, 0.f};
  for (int64_t t0 = r0; t0 < r1; t0 += kGRows) {
    const int nr = static_cast<int>(imin64(kGRows, r1 - t0));
    const int nr4 = (nr + 4 * RG - 1) / (4 * RG) * (4 * RG);     // zero-padded to whole unrolled steps
#pragma unroll 4
    for (int e = threadIdx.x; e < nr4 * (LP / 4); e += kGThr) {
      const int rr = e / (LP / 4), c4 = e % (LP / 4);
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (rr < nr) v = __ldcg(reinterpret_cast<const float4*>(Z + (t0 + rr) * LP) + c4);
      reinterpret_cast<float4*>(&zt[rr][0])[c4] = v;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < PPT; ++u)
      if (pa[u] >= 0)
        for (int rr = rg; rr < nr; rr += 4 * RG) {
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const int r = rr + v * RG;
            df64_add_prod(g[u][v], zt[r][pa[u]], zt[r][pb[u]]);
          }
        }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < PPT; ++u)
    if (pa[u] >= 0) {
      const int pr = (PPT == 1) ? static_cast<int>(threadIdx.x) % NP : static_cast<int>(threadIdx.x) + kGThr * u;
      gpart[rg][pr] = df64_value(df_add(df_add(g[u][0], g[u][1]), df_add(g[u][2], g[u][3])));
    }
  __syncthreads();
  double* gsm = reinterpret_cast<double*>(dsm);                   // NP (the workspace is idle)
  for (int pr = threadIdx.x; pr < NP; pr += kGThr) {
    double s = 0.0;
    for (int r = 0; r < RG; ++r) s += gpart[r][pr];
    gsm[pr] = s;
  }
  const int nclusters = gridDim.x / kCL;
  if (!cluster_split_reduce<double>(gsm, NP, cpart, Gout, tickets, blockIdx.x / kCL, nclusters, &flag)) return;
  if (cooperative_groups::this_cluster().block_rank() != 0) return;
  SmallWs<LP> w = carve_small_ws<LP>(dsm, kGaccG);
  for (int e = threadIdx.x; e < LP * LP; e += kGThr) {
    const int a = e / LP, b = e % LP;
    double v = 0.0;
    if (a < l && b < l) {
      const int lo = a < b ? a : b, hi = a < b ? b : a;
      v = __ldcg(Gout + (lo * LP - lo * (lo - 1) / 2 + (hi - lo)));
    }
    w.G[e] = df_from_double(v);
  }
  block_copy(w.W, Q, n * LP);
  __syncthreads();
  const float tau = tau_from_mu ? static_cast<float>(1.0 / dst->mu) : tau_host;
  core_block<LP>(w, w.W, n, l, tau, update_rp, advance_counter, Rf, Qt, dst, rank_tol, max_sweeps);
}

template <typename K>
cudaError_t set_limit_g(K kernel, int smem_limit) {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              smem_limit - static_cast<int>(a.sharedSizeBytes));
}

}  // namespace

size_t gram_core_smem(int LP, int64_t n) {
  const size_t ws = LP == 16 ? small_ws_bytes<16>(n, kGaccG) : small_ws_bytes<32>(n, kGaccG);
  const size_t np = static_cast<size_t>(LP) * (LP + 1) / 2 * sizeof(double);
  const size_t zt = static_cast<size_t>(kGRows + 64) * LP * sizeof(float);
  size_t r = ws > np ? ws : np;
  return r > zt ? r : zt;
}

cudaError_t prepare_gram_kernels(int smem_limit) {
  cudaError_t e = set_limit_g(k_gram_core<16>, smem_limit);
  if (e == cudaSuccess) e = set_limit_g(k_gram_core<32>, smem_limit);
  return e;
}

// Largest grid of whole clusters that is resident at once (one wave).
int gram_resident_grid(int LP, int64_t n) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kCL, 1, 1);
  cfg.blockDim = dim3(kGThr, 1, 1);
  cfg.dynamicSmemBytes = gram_core_smem(LP, n);
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = kCL;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  int nc = 0;
  const void* fn = LP == 16 ? reinterpret_cast<const void*>(k_gram_core<16>) : reinterpret_cast<const void*>(k_gram_core<32>);
  if (cudaOccupancyMaxActiveClusters(&nc, fn, &cfg) != cudaSuccess) nc = 0;
  (void)cudaGetLastError();
  return nc * kCL;
}

// Z: m x LP (ld = LP); grid: a multiple of the cluster size.
cudaError_t launch_gram_core(int LP, const float* Z, int64_t m, int64_t n, int grid, const float* Q, double* cpart,
                             double* G, unsigned* tickets, int l, float tau_host, int tau_from_mu, int update_rp,
                             int advance_counter, float* Rf, float* Qt, DevState* dst, double rank_tol,
                             int max_sweeps, cudaStream_t st) {
  const int64_t rpc = (m + grid - 1) / grid;
  const size_t smem = gram_core_smem(LP, n);
  const int nn = static_cast<int>(n);
#define ARGS Z, m, nn, rpc, Q, cpart, G, tickets, l, tau_host, tau_from_mu, update_rp, advance_counter, Rf, Qt, dst, \
             rank_tol, max_sweeps
  if (LP == 16) k_gram_core<16><<<grid, kGThr, smem, st>>>(ARGS);
  else k_gram_core<32><<<grid, kGThr, smem, st>>>(ARGS);
#undef ARGS
  return cudaGetLastError();
}

}  // namespace frsvt
