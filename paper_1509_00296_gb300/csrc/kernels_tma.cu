// Persistent, TMA-pipelined passes over A for a short side of at most 256 columns.
//
// One CTA per SM (clusters of kCL along x, as many as can be resident at once).
// A producer warp streams row tiles of A (and, for A^T Z, the matching rows of Z)
// as 2-D tensor-map boxes into a shared-memory ring guarded by mbarriers; rows and
// columns outside the matrix are zero-filled by the TMA unit.  NC consumer threads
// (512 for l <= 16, 256 for l <= 32) compute on the tiles; the ring keeps ~100 KB of
// loads in flight per SM without register cost.  Each pass ends with a cluster
// split-K reduction (cluster.cuh) whose last cluster runs the small dense step of
// Alg. 1 that depends on the reduced result (k_tp_alm, which reduces a single value,
// runs without clusters on every SM and with 256 consumer threads):
//   k_tp_sc  : Y = A^T Omega (sketch, steps 4-5 / 8-9) or Y = A^T Z (power step 14),
//              then the orthonormal basis (steps 6, 10-11, 14)
//   k_tp_lr  : Z = A Q (power step 14 / projection step 16); with GRAM also B B^T = Z^T Z
//              in double-float and the core SVD + shrinkage (steps 16-21, Eq. 6)
//   k_tp_alm : X = Z (Q M)^T fused with the iALM sparse shrinkage, multiplier update and
//              residual (Sec. 4.1), then the mu update
// Waits on mbarriers are bounded (tma.cuh): on a timeout the kernel records
// FRSVT_DEV_TIMEOUT, stops computing, and still walks every barrier so that no
// thread is left waiting.
#include <cuda.h>
#include <cuda_bf16.h>

#include "cluster.cuh"
#include "common.cuh"
#include "small_dense.cuh"
#include "state.cuh"
#include "tma.cuh"

namespace frsvt {

namespace {

constexpr int kRB = 32;               // rows per tile of the column pass
constexpr int kStages = 4;
constexpr int kRBL = 64;              // rows per tile of the row pass
constexpr int kRBE = 16;              // rows per tile of the epilogue
constexpr int kStagesE = 5;              // deepest epilogue ring (fewer stages where n is wide)
constexpr size_t kAlmSmemCap = 219 * 1024; // dynamic shared memory the epilogue may take
constexpr int kGacc = 1024;

template <int LP>
struct Cfg {
  static constexpr int NC = (LP <= 16) ? 512 : 256;   // consumer threads
  static constexpr int NT = NC + 32;                    // + one producer warp
};

__host__ __device__ inline uint32_t align1k(uint32_t b) { return (b + 1023u) / 1024u * 1024u; }

struct Rows {
  int64_t r0, r1;
  int nchunks;
};

__device__ __forceinline__ Rows cta_rows(int64_t m, int64_t rpc, int rb) {
  Rows r;
  r.r0 = static_cast<int64_t>(blockIdx.x) * rpc;
  r.r1 = imin64(m, r.r0 + rpc);
  r.nchunks = (r.r1 > r.r0) ? static_cast<int>((r.r1 - r.r0 + rb - 1) / rb) : 0;
  return r;
}

// One box source of a stage: tensor map, bytes of its box and offset inside the stage.
struct Box {
  const CUtensorMap* map;
  uint32_t bytes;
  uint32_t offset;
};

// Producer (one thread): stream nchunks tiles of every box source into the ring.
template <int NB>
__device__ void produce(const Box (&boxes)[NB], int nst, unsigned char* ring, uint32_t sbytes, uint64_t* full,
                        uint64_t* empty, const Rows& rw, int rb, int ncw, DevState* dst) {
  uint32_t total = 0;
#pragma unroll
  for (int t = 0; t < NB; ++t) total += boxes[t].bytes;
  (void)ncw;
  for (int c = 0; c < rw.nchunks; ++c) {
    const int s = c % nst;
    const uint32_t ph = static_cast<uint32_t>(c / nst) & 1u;
    if (c >= nst && !mbar_wait(&empty[s], ph ^ 1u)) {
      atomicOr(&dst->status, kDevTimeout);
      return;                 // consumers time out on the missing tiles and skip them
    }
    mbar_arrive_expect_tx(&full[s], total);
    const int y = static_cast<int>(rw.r0 + static_cast<int64_t>(c) * rb);
#pragma unroll
    for (int t = 0; t < NB; ++t) tma_load_2d(ring + s * sbytes + boxes[t].offset, boxes[t].map, 0, y, &full[s]);
  }
}

__device__ __forceinline__ void init_ring(uint64_t* full, uint64_t* empty, int nst, int ncw) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], ncw);
    }
    fence_mbar_init();
  }
  __syncthreads();
}

// Bounded wait for tile c; a timeout is recorded once and turns `ok` off for the rest.
__device__ __forceinline__ void wait_tile(uint64_t* full, int c, int nst, bool& ok, DevState* dst) {
  if (!ok) return;
  if (!mbar_wait(&full[c % nst], static_cast<uint32_t>(c / nst) & 1u)) {
    ok = false;
    atomicOr(&dst->status, kDevTimeout);
  }
}

// ---------------------------------------------------------------- Y = A^T B (+ orth tail)
// Consumer thread t owns the column quad qd = t % nq (one 16-byte shared load per row) for
// rows rr = rg, rg + rgc, ... of each tile (rg = t / nq); the row groups are added in order.
// B = Omega is generated per tile by the consumers; B = Z arrives with the tile through TMA.
template <int LP, bool OMEGA>
__global__ void __cluster_dims__(kCL, 1, 1) __launch_bounds__(Cfg<LP>::NT, 1)
k_tp_sc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmZ, int64_t m, int n,
        int np4, int64_t rpc, uint64_t seed, uint64_t ctr, DevState* __restrict__ dst, float* __restrict__ cpart,
        float* __restrict__ Y, unsigned* __restrict__ tickets, int l, int use_rp, int passes,
        const float* __restrict__ Qt, float* __restrict__ Qout, double rank_tol) {
  constexpr int NC = Cfg<LP>::NC, NT = Cfg<LP>::NT;
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages];
  __shared__ __align__(16) float Bs[OMEGA ? kRB : 1][LP];
  __shared__ int flag;
  const uint32_t abytes = static_cast<uint32_t>(kRB * np4 * 4);
  const uint32_t zbytes = OMEGA ? 0u : static_cast<uint32_t>(kRB * LP * 4);
  const uint32_t sb = align1k(abytes + zbytes);
  unsigned char* ring = dsm;
  float* part_sm = reinterpret_cast<float*>(dsm + kStages * sb);      // n x LP
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const Rows rw = cta_rows(m, rpc, kRB);
  const int nq = np4 / 4;
  int rgc = NC / nq;
  if (rgc > kRB) rgc = kRB;
  init_ring(full, empty, kStages, NC / 32);
  if (warp == NC / 32) {
    if (lane == 0) {
      prefetch_tensormap(&tmA);
      if (OMEGA) {
        const Box boxes[1] = {{&tmA, abytes, 0u}};
        produce<1>(boxes, kStages, ring, sb, full, empty, rw, kRB, NC / 32, dst);
      } else {
        prefetch_tensormap(&tmZ);
        const Box boxes[2] = {{&tmA, abytes, 0u}, {&tmZ, zbytes, abytes}};
        produce<2>(boxes, kStages, ring, sb, full, empty, rw, kRB, NC / 32, dst);
      }
    }
  } else {
    const int qd = threadIdx.x % nq;
    const int rg = threadIdx.x / nq;
    const bool active = rg < rgc;
    const uint64_t stream = OMEGA ? ((ctr == kCounterFromState) ? dst->counter : ctr) : 0ull;
    float acc[4][LP];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int k = 0; k < LP; ++k) acc[c][k] = 0.f;
    bool ok = true;
    for (int c = 0; c < rw.nchunks; ++c) {
      const int64_t i0 = rw.r0 + static_cast<int64_t>(c) * kRB;
      const int nr = static_cast<int>(imin64(kRB, rw.r1 - i0));
      if (OMEGA) {
        named_bar(1, NC);
        for (int t = threadIdx.x; t < kRB * (LP / 4); t += NC) {
          const int rr = t / (LP / 4), blk = t % (LP / 4);
          float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
          if (rr < nr) g = gaussian4(seed, static_cast<uint64_t>(i0 + rr), static_cast<uint64_t>(blk), stream, 0ull);
          reinterpret_cast<float4*>(&Bs[rr][0])[blk] = g;
        }
        named_bar(1, NC);
      }
      wait_tile(full, c, kStages, ok, dst);
      const int s = c % kStages;
      if (ok && active) {
        const float* tile = reinterpret_cast<const float*>(ring + s * sb);
        const float* brow = OMEGA ? &Bs[0][0] : reinterpret_cast<const float*>(ring + s * sb + abytes);
        for (int rr = rg; rr < kRB; rr += rgc) {
          const float4 a4 = reinterpret_cast<const float4*>(tile + rr * np4)[qd];
          const float a[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
          for (int k4 = 0; k4 < LP / 4; ++k4) {
            const float4 b = reinterpret_cast<const float4*>(brow + rr * LP)[k4];
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
              acc[cc][4 * k4 + 0] = fmaf(a[cc], b.x, acc[cc][4 * k4 + 0]);
              acc[cc][4 * k4 + 1] = fmaf(a[cc], b.y, acc[cc][4 * k4 + 1]);
              acc[cc][4 * k4 + 2] = fmaf(a[cc], b.z, acc[cc][4 * k4 + 2]);
              acc[cc][4 * k4 + 3] = fmaf(a[cc], b.w, acc[cc][4 * k4 + 3]);
            }
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
    }
    // add the row groups into part_sm (n x LP) one group after the other (deterministic order)
    for (int g2 = 0; g2 < rgc; ++g2) {               // rgc is uniform across the consumers
      if (rg == g2) {
#pragma unroll
        for (int cc = 0; cc < 4; ++cc)
          if (4 * qd + cc < n)
#pragma unroll
            for (int k = 0; k < LP; ++k) {
              float* p = part_sm + (4 * qd + cc) * LP + k;
              *p = (g2 == 0) ? acc[cc][k] : (*p + acc[cc][k]);
            }
      }
      named_bar(1, NC);
    }
  }
  __syncthreads();
  const int nclusters = gridDim.x / kCL;
  if (!cluster_split_reduce<float>(part_sm, n * LP, cpart, Y, tickets, blockIdx.x / kCL, nclusters, &flag)) return;
  if (cooperative_groups::this_cluster().block_rank() != 0) return;
  // tail: orthonormal basis of Y (this CTA alone), workspace in the ring
  SmallWs<LP> w = carve_small_ws<LP>(dsm, kGacc);
  int keep = use_rp ? dst->keep : 0;
  keep = max(0, min(keep, l));
  load_basis_block<LP>(w.W, n, keep, l, Qt, Y);
  __syncthreads();
  float rp_res = -1.f;
  const int s = orth_block<LP>(w, n, keep, l, rank_tol, passes, &rp_res, &dst->status);
  for (int e = threadIdx.x; e < n * LP; e += NT) Qout[e] = w.W[e];
  if (threadIdx.x == 0) {
    if (use_rp) dst->rp_res = rp_res;
    dst->s = s;
    if (s < l) dst->status |= kDevRankDeficient;
  }
}

// ---------------------------------------------------------------- Z = A Q (+ Gram + core tail)
// Tiles of kRBL rows; G = NC / kRBL consumer threads share a row: thread t owns row t / G and
// the column quads t % G, t % G + G, ...; Q sits in shared memory k-major, so the threads of a
// row read consecutive 16-byte words.  The G partial rows are summed with log2(G) shuffles.
template <int LP, bool GRAM>
__global__ void __cluster_dims__(kCL, 1, 1) __launch_bounds__(Cfg<LP>::NT, 1)
k_tp_lr(const __grid_constant__ CUtensorMap tmA, int64_t m, int n, int np4, int64_t rpc, int nst,
        const float* __restrict__ Q, float* __restrict__ Z, double* __restrict__ cpart, double* __restrict__ Gout,
        unsigned* __restrict__ tickets, int l, float tau_host, int tau_from_mu, int update_rp, int advance_counter,
        float* __restrict__ Rf, float* __restrict__ Qt, DevState* __restrict__ dst, double rank_tol,
        int max_sweeps) {
  constexpr int NC = Cfg<LP>::NC, NT = Cfg<LP>::NT;
  constexpr int G = NC / kRBL;                         // threads per row (8 or 4)
  constexpr int NP = LP * (LP + 1) / 2;
  constexpr int PPT = (NP + NC - 1) / NC;              // Gram pairs per consumer thread
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ __align__(8) uint64_t full[4], empty[4];
  __shared__ __align__(16) float zt[GRAM ? kRBL : 1][LP];
  __shared__ double gsm[NP];
  __shared__ unsigned char pa[NP], pb[NP];
  __shared__ int flag;
  const uint32_t sb = align1k(static_cast<uint32_t>(kRBL * np4 * 4));
  unsigned char* ring = dsm;
  float* Qs = reinterpret_cast<float*>(dsm + nst * sb);              // LP x np4, k-major
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const Rows rw = cta_rows(m, rpc, kRBL);
  const int nq = np4 / 4;
  for (int t = threadIdx.x; t < LP * np4; t += NT) {
    const int k = t / np4, jj = t % np4;
    Qs[t] = (jj < n) ? Q[jj * LP + k] : 0.f;
  }
  if (GRAM)
    for (int t = threadIdx.x; t < NP; t += NT) {
      int a, b;
      decode_pair_sym(t, LP, a, b);
      pa[t] = static_cast<unsigned char>(a);
      pb[t] = static_cast<unsigned char>(b);
    }
  init_ring(full, empty, nst, NC / 32);
  df64 g[PPT];
#pragma unroll
  for (int u = 0; u < PPT; ++u) g[u] = df64{0.f, 0.f};
  if (warp == NC / 32) {
    if (lane == 0) {
      prefetch_tensormap(&tmA);
      const Box boxes[1] = {{&tmA, static_cast<uint32_t>(kRBL * np4 * 4), 0u}};
      produce<1>(boxes, nst, ring, sb, full, empty, rw, kRBL, NC / 32, dst);
    }
  } else {
    const int r = threadIdx.x / G, gq = threadIdx.x % G;
    bool ok = true;
    for (int c = 0; c < rw.nchunks; ++c) {
      const int64_t i0 = rw.r0 + static_cast<int64_t>(c) * kRBL;
      wait_tile(full, c, nst, ok, dst);
      const int s = c % nst;
      float z[LP];
#pragma unroll
      for (int k = 0; k < LP; ++k) z[k] = 0.f;
      if (ok) {
        const float4* arow = reinterpret_cast<const float4*>(ring + s * sb) + r * nq;
        for (int qd = gq; qd < nq; qd += G) {
          const float4 a = arow[qd];
#pragma unroll
          for (int k = 0; k < LP; ++k) {
            const float4 q = reinterpret_cast<const float4*>(Qs + k * np4)[qd];
            z[k] = fmaf(a.x, q.x, fmaf(a.y, q.y, fmaf(a.z, q.z, fmaf(a.w, q.w, z[k]))));
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
#pragma unroll
      for (int k = 0; k < LP; ++k)
#pragma unroll
        for (int o = 1; o < G; o <<= 1) z[k] += __shfl_xor_sync(0xffffffffu, z[k], o);
      const int64_t row = i0 + r;
      const bool valid = row < rw.r1;
      if (gq == 0 && valid) {
        float4* zo = reinterpret_cast<float4*>(Z + row * LP);
#pragma unroll
        for (int k4 = 0; k4 < LP / 4; ++k4) zo[k4] = make_float4(z[4 * k4], z[4 * k4 + 1], z[4 * k4 + 2], z[4 * k4 + 3]);
      }
      if (GRAM) {
        if (gq == 0)
#pragma unroll
          for (int k = 0; k < LP; ++k) zt[r][k] = valid ? z[k] : 0.f;
        named_bar(1, NC);
#pragma unroll
        for (int u = 0; u < PPT; ++u) {
          const int pr = threadIdx.x + NC * u;
          if (pr < NP) {
            const int a = pa[pr], b = pb[pr];
            for (int rr = 0; rr < kRBL; ++rr) df64_add_prod(g[u], zt[rr][a], zt[rr][b]);
          }
        }
        named_bar(1, NC);
      }
    }
  }
  if (!GRAM) return;
  __syncthreads();
  if (warp < NC / 32)
#pragma unroll
    for (int u = 0; u < PPT; ++u) {
      const int pr = threadIdx.x + NC * u;
      if (pr < NP) gsm[pr] = df64_value(g[u]);
    }
  const int nclusters = gridDim.x / kCL;
  if (!cluster_split_reduce<double>(gsm, NP, cpart, Gout, tickets, blockIdx.x / kCL, nclusters, &flag)) return;
  if (cooperative_groups::this_cluster().block_rank() != 0) return;
  SmallWs<LP> w = carve_small_ws<LP>(dsm, kGacc);
  for (int e = threadIdx.x; e < LP * LP; e += NT) {
    const int a = e / LP, b = e % LP;
    double v = 0.0;
    if (a < l && b < l) {
      const int lo = a < b ? a : b, hi = a < b ? b : a;
      v = __ldcg(Gout + (lo * LP - lo * (lo - 1) / 2 + (hi - lo)));
    }
    w.G[e] = df_from_double(v);
  }
  block_copy(w.W, Q, n * LP);                                         // the basis, staged
  __syncthreads();
  const float tau = tau_from_mu ? static_cast<float>(1.0 / dst->mu) : tau_host;
  core_block<LP>(w, w.W, n, l, tau, update_rp, advance_counter, Rf, Qt, dst, rank_tol, max_sweeps);
}

// ---------------------------------------------------------------- fused reconstruction + iALM update
// One CTA per SM and no cluster: the kernel only reduces one value (the residual) across CTAs,
// by per-CTA partials and a ticket, so every SM streams.
// 256 consumer threads for either basis width: each holds four rows of Rf (4 LP registers), which
// 512 threads (at most 96 registers each) would spill.
constexpr int kAlmNC = 256;
constexpr int kAlmNT = kAlmNC + 32;

template <int LP>
__global__ void __launch_bounds__(kAlmNT, 1)
k_tp_alm(const __grid_constant__ CUtensorMap tmO, const __grid_constant__ CUtensorMap tmS,
         const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmZ, int64_t m, int n, int np4,
         int64_t rpc, const float* __restrict__ Rf, float* __restrict__ S, float* __restrict__ A, int64_t ld,
         float* __restrict__ L, int64_t ldl, DevState* __restrict__ dst, double* __restrict__ cpart,
         unsigned* __restrict__ tickets, __nv_bfloat16* __restrict__ Ab, int64_t ldb, int nse) {
  constexpr int NC = kAlmNC, NT = kAlmNT;
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ __align__(8) uint64_t full[kStagesE], empty[kStagesE];
  __shared__ double red[NT / 32];
  __shared__ double mine;
  __shared__ int flag;
  const uint32_t box = static_cast<uint32_t>(kRBE * np4 * 4);
  const uint32_t zbox = static_cast<uint32_t>(kRBE * LP * 4);
  const uint32_t sb = align1k(3 * box + zbox);
  unsigned char* ring = dsm;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const Rows rw = cta_rows(m, rpc, kRBE);
  const double mu = dst->mu;
  const double mu_next = fmin(dst->rho * mu, dst->mu_bar);
  const float thr = static_cast<float>(dst->lambda / mu);
  const float ratio = static_cast<float>(mu / mu_next);
  init_ring(full, empty, nse, NC / 32);
  float res2 = 0.f;
  if (warp == NC / 32) {
    if (lane == 0) {
      prefetch_tensormap(&tmO);
      prefetch_tensormap(&tmS);
      prefetch_tensormap(&tmA);
      prefetch_tensormap(&tmZ);
      // Tiles of O, S, A, Z in; once the consumers have overwritten the S and A slots of a tile
      // with S' and A', TMA stores them before the stage is refilled.
      const uint32_t total = 3 * box + zbox;
      bool pok = true;
      for (int c = 0; c < rw.nchunks && pok; ++c) {
        const int s = c % nse;
        if (c >= nse) {
          if (!mbar_wait(&empty[s], static_cast<uint32_t>(c / nse - 1) & 1u)) {
            atomicOr(&dst->status, kDevTimeout);
            pok = false;
            break;
          }
          const int yp = static_cast<int>(rw.r0 + static_cast<int64_t>(c - nse) * kRBE);
          tma_store_2d(&tmS, 0, yp, ring + s * sb + box);
          tma_store_2d(&tmA, 0, yp, ring + s * sb + 2 * box);
          bulk_commit();
          bulk_wait_read_all();
        }
        mbar_arrive_expect_tx(&full[s], total);
        const int y = static_cast<int>(rw.r0 + static_cast<int64_t>(c) * kRBE);
        tma_load_2d(ring + s * sb, &tmO, 0, y, &full[s]);
        tma_load_2d(ring + s * sb + box, &tmS, 0, y, &full[s]);
        tma_load_2d(ring + s * sb + 2 * box, &tmA, 0, y, &full[s]);
        tma_load_2d(ring + s * sb + 3 * box, &tmZ, 0, y, &full[s]);
      }
      const int c0 = rw.nchunks > nse ? rw.nchunks - nse : 0;
      for (int c = c0; c < rw.nchunks && pok; ++c) {
        const int s = c % nse;
        if (!mbar_wait(&empty[s], static_cast<uint32_t>(c / nse) & 1u)) {
          atomicOr(&dst->status, kDevTimeout);
          break;
        }
        const int yp = static_cast<int>(rw.r0 + static_cast<int64_t>(c) * kRBE);
        tma_store_2d(&tmS, 0, yp, ring + s * sb + box);
        tma_store_2d(&tmA, 0, yp, ring + s * sb + 2 * box);
        bulk_commit();
      }
      bulk_wait_all();
    }
  } else {
    const int nq = np4 / 4;
    int rgc = NC / nq;
    if (rgc > kRBE) rgc = kRBE;
    const int qd = threadIdx.x % nq;
    const int rg = threadIdx.x / nq;
    const bool active = rg < rgc;
    const int col = 4 * qd;
    float rf[4][LP];                                  // rows col .. col + 3 of Rf, 16-byte loads
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      const bool in = active && col + cc < n;
      const float4* r4 = reinterpret_cast<const float4*>(Rf + (col + cc) * LP);
#pragma unroll
      for (int k4 = 0; k4 < LP / 4; ++k4) {
        const float4 v = in ? __ldg(r4 + k4) : make_float4(0.f, 0.f, 0.f, 0.f);
        rf[cc][4 * k4] = v.x;
        rf[cc][4 * k4 + 1] = v.y;
        rf[cc][4 * k4 + 2] = v.z;
        rf[cc][4 * k4 + 3] = v.w;
      }
    }
    const bool fullq = col + 3 < n;
    bool ok = true;
    for (int c = 0; c < rw.nchunks; ++c) {
      const int64_t i0 = rw.r0 + static_cast<int64_t>(c) * kRBE;
      const int nr = static_cast<int>(imin64(kRBE, rw.r1 - i0));
      wait_tile(full, c, nse, ok, dst);
      const int s = c % nse;
      if (ok && active) {
        const float* tO = reinterpret_cast<const float*>(ring + s * sb);
        float* tS = reinterpret_cast<float*>(ring + s * sb) + kRBE * np4;
        float* tA = tS + kRBE * np4;
        const float* tZ = tA + kRBE * np4;
        for (int rr = rg; rr < nr; rr += rgc) {
          float x[4];
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) {
            float t = 0.f;
#pragma unroll
            for (int k4 = 0; k4 < LP / 4; ++k4) {
              const float4 z = reinterpret_cast<const float4*>(tZ + rr * LP)[k4];
              t = fmaf(z.x, rf[cc][4 * k4], t);
              t = fmaf(z.y, rf[cc][4 * k4 + 1], t);
              t = fmaf(z.z, rf[cc][4 * k4 + 2], t);
              t = fmaf(z.w, rf[cc][4 * k4 + 3], t);
            }
            x[cc] = t;
          }
          const float4 o4 = reinterpret_cast<const float4*>(tO + rr * np4)[qd];
          const float4 s4 = reinterpret_cast<const float4*>(tS + rr * np4)[qd];
          const float4 a4 = reinterpret_cast<const float4*>(tA + rr * np4)[qd];
          const float ov[4] = {o4.x, o4.y, o4.z, o4.w};
          const float sv[4] = {s4.x, s4.y, s4.z, s4.w};
          const float av[4] = {a4.x, a4.y, a4.z, a4.w};
          float sn[4], an[4];
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) {
            const float t = av[cc] + sv[cc] - x[cc];                      // O - L + Y/mu
            sn[cc] = (t > thr) ? (t - thr) : ((t < -thr) ? (t + thr) : 0.f);
            an[cc] = ov[cc] - sn[cc] + ratio * (t - sn[cc]);               // O - S' + Y'/mu'
            const float rz = ov[cc] - x[cc] - sn[cc];                      // O - L - S'
            if (col + cc < n) res2 = fmaf(rz, rz, res2);
          }
          const int64_t row = i0 + rr;
          // S' and A' replace S and A in the tile; the producer stores the tile by TMA
          reinterpret_cast<float4*>(tS + rr * np4)[qd] = make_float4(sn[0], sn[1], sn[2], sn[3]);
          reinterpret_cast<float4*>(tA + rr * np4)[qd] = make_float4(an[0], an[1], an[2], an[3]);
          if (fullq) {
            if (L != nullptr) *reinterpret_cast<float4*>(L + row * ldl + col) = make_float4(x[0], x[1], x[2], x[3]);
            if (Ab != nullptr) {                                             // BF16 shadow of A'
              __nv_bfloat162* ab = reinterpret_cast<__nv_bfloat162*>(Ab + row * ldb + col);
              ab[0] = __floats2bfloat162_rn(an[0], an[1]);
              ab[1] = __floats2bfloat162_rn(an[2], an[3]);
            }
          } else {
#pragma unroll
            for (int cc = 0; cc < 4; ++cc)
              if (col + cc < n) {
                if (L != nullptr) L[row * ldl + col + cc] = x[cc];
                if (Ab != nullptr) Ab[row * ldb + col + cc] = __float2bfloat16_rn(an[cc]);
              }
          }
        }
      }
      fence_proxy_async();                          // S', A' in the tile -> visible to the TMA store
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
    }
  }
  const double v = warp_sum(static_cast<double>(res2));
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w2 = 0; w2 < NT / 32; ++w2) t += red[w2];
    cpart[blockIdx.x] = t;                       // this CTA's share of ||O - L - S'||^2
  }
  if (!last_of(tickets, gridDim.x, &flag)) return;
  // the CTA that finishes last adds the per-CTA partials in a fixed order (lane-strided, then the
  // warp tree): the result does not depend on which CTA that is
  if (threadIdx.x < 32) {
    double t = 0.0;
    for (int b = lane; b < static_cast<int>(gridDim.x); b += 32) t += __ldcg(cpart + b);
    t = warp_sum(t);
    if (lane == 0) mine = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double s2 = mine;
    const double rr = (dst->normO_F > 0.0) ? sqrt(s2) / dst->normO_F : 0.0;
    dst->resid_ratio = rr;
    if (!isfinite(rr)) dst->status |= kDevNonfinite;
    dst->mu = mu_next;
    dst->iter += 1;
  }
}

template <typename K>
cudaError_t set_dyn_limit(K kernel, int smem_limit) {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              smem_limit - static_cast<int>(a.sharedSizeBytes));
}

int threads_of(int LP) { return LP <= 16 ? Cfg<16>::NT : Cfg<32>::NT; }

}  // namespace

// ---------------------------------------------------------------- host side
int tma_np4(int64_t n) { return static_cast<int>((n + 3) / 4 * 4); }

size_t tma_sc_smem(int LP, int64_t n) {
  const int np4 = tma_np4(n);
  const size_t ring = static_cast<size_t>(kStages) * align1k(static_cast<uint32_t>(kRB * np4 * 4 + kRB * LP * 4));
  const size_t part = static_cast<size_t>(n) * LP * sizeof(float);
  const size_t ws = LP == 16 ? small_ws_bytes<16>(n, kGacc) : small_ws_bytes<32>(n, kGacc);
  const size_t a = ring + part;
  return a > ws ? a : ws;
}

// Stages of the row pass that fit next to the staged Q (at most 4).
int tma_lr_stages(int LP, int64_t n, size_t limit) {
  const int np4 = tma_np4(n);
  const size_t sbb = align1k(static_cast<uint32_t>(kRBL * np4 * 4));
  const size_t qs = static_cast<size_t>(LP) * np4 * sizeof(float);
  int s = static_cast<int>((limit - qs) / sbb);
  return s > 4 ? 4 : s;
}

size_t tma_lr_smem(int LP, int64_t n, int nst) {
  const int np4 = tma_np4(n);
  const size_t ring = static_cast<size_t>(nst) * align1k(static_cast<uint32_t>(kRBL * np4 * 4));
  const size_t qs = static_cast<size_t>(LP) * np4 * sizeof(float);
  const size_t ws = LP == 16 ? small_ws_bytes<16>(n, kGacc) : small_ws_bytes<32>(n, kGacc);
  const size_t a = ring + qs;
  return ws > a ? ws : a;
}

// Ring depth of the epilogue: as many stages (<= kStagesE) as fit in kAlmSmemCap; 0 if fewer than 2 fit.
int tma_alm_stages(int LP, int64_t n) {
  const size_t sb = align1k(static_cast<uint32_t>(3 * kRBE * tma_np4(n) * 4 + kRBE * LP * 4));
  int ns = static_cast<int>(kAlmSmemCap / sb);
  if (ns > kStagesE) ns = kStagesE;
  return ns >= 2 ? ns : 0;
}

size_t tma_alm_smem(int LP, int64_t n) {
  const int ns = tma_alm_stages(LP, n);
  const size_t sb = align1k(static_cast<uint32_t>(3 * kRBE * tma_np4(n) * 4 + kRBE * LP * 4));
  return static_cast<size_t>(ns > 0 ? ns : kStagesE) * sb;
}

int tma_rows_per_tile() { return kRB; }
int tma_rows_per_tile_lr() { return kRBL; }
int tma_rows_per_tile_epilogue() { return kRBE; }

// Largest grid of the persistent passes whose clusters of kCL are all resident at once: a GPC
// only holds whole clusters, so the answer can be below the SM count.  The smallest of the
// three kernels' counts is used for every pass.
int tma_resident_grid(int LP, int64_t n) {
  int best = 1 << 30;
  auto probe = [&](const void* fn, size_t smem) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kCL, 1, 1);
    cfg.blockDim = dim3(threads_of(LP), 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = kCL;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, fn, &cfg) != cudaSuccess) nc = 0;
    if (nc < best) best = nc;
  };
  const int nst = tma_lr_stages(LP, n, 227 * 1024 - 16384);
  if (LP == 16) {
    probe(reinterpret_cast<const void*>(k_tp_sc<16, false>), tma_sc_smem(16, n));
    probe(reinterpret_cast<const void*>(k_tp_lr<16, true>), tma_lr_smem(16, n, nst));
  } else {
    probe(reinterpret_cast<const void*>(k_tp_sc<32, false>), tma_sc_smem(32, n));
    probe(reinterpret_cast<const void*>(k_tp_lr<32, true>), tma_lr_smem(32, n, nst));
  }
  (void)cudaGetLastError();
  return best * kCL;
}

// Resident grid of the epilogue kernel (blocks per SM times SMs).
int tma_alm_resident_grid(int LP, int64_t n) {
  int per = 0, dev = 0, sms = 0;
  const void* fn = LP == 16 ? reinterpret_cast<const void*>(k_tp_alm<16>) : reinterpret_cast<const void*>(k_tp_alm<32>);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kAlmNT, tma_alm_smem(LP, n)) != cudaSuccess ||
      cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    per = 0;
    sms = 0;
  }
  (void)cudaGetLastError();
  return per * sms;
}

cudaError_t prepare_tma_kernels(int smem_limit) {
  cudaError_t e = cudaSuccess;
#define PREP(k) \
  if (e == cudaSuccess) e = set_dyn_limit(k, smem_limit);
  PREP((k_tp_sc<16, true>));
  PREP((k_tp_sc<16, false>));
  PREP((k_tp_sc<32, true>));
  PREP((k_tp_sc<32, false>));
  PREP((k_tp_lr<16, true>));
  PREP((k_tp_lr<16, false>));
  PREP((k_tp_lr<32, true>));
  PREP((k_tp_lr<32, false>));
  PREP((k_tp_alm<16>));
  PREP((k_tp_alm<32>));
#undef PREP
  return e;
}

cudaError_t launch_tp_sc(int LP, const CUtensorMap& tmA, const CUtensorMap* tmZ, int64_t m, int64_t n, int64_t rpc,
                         int grid, uint64_t seed, uint64_t ctr, DevState* dst, float* cpart, float* Y, unsigned* tickets,
                         int l, int use_rp, int passes, const float* Qt, float* Q, double rank_tol, cudaStream_t st) {
  const int np4 = tma_np4(n);
  const size_t smem = tma_sc_smem(LP, n);
  const int nn = static_cast<int>(n);
  const CUtensorMap& z = tmZ ? *tmZ : tmA;
#define ARGS tmA, z, m, nn, np4, rpc, seed, ctr, dst, cpart, Y, tickets, l, use_rp, passes, Qt, Q, rank_tol
  if (LP == 16) {
    if (tmZ) k_tp_sc<16, false><<<grid, Cfg<16>::NT, smem, st>>>(ARGS);
    else k_tp_sc<16, true><<<grid, Cfg<16>::NT, smem, st>>>(ARGS);
  } else {
    if (tmZ) k_tp_sc<32, false><<<grid, Cfg<32>::NT, smem, st>>>(ARGS);
    else k_tp_sc<32, true><<<grid, Cfg<32>::NT, smem, st>>>(ARGS);
  }
#undef ARGS
  return cudaGetLastError();
}

cudaError_t launch_tp_lr(int LP, bool gram, const CUtensorMap& tmA, int64_t m, int64_t n, int64_t rpc, int grid,
                         int nst, const float* Q, float* Z, double* cpart, double* G, unsigned* tickets, int l,
                         float tau_host, int tau_from_mu, int update_rp, int advance_counter, float* Rf, float* Qt,
                         DevState* dst, double rank_tol, int max_sweeps, cudaStream_t st) {
  const int np4 = tma_np4(n);
  const size_t smem = tma_lr_smem(LP, n, nst);
  const int nn = static_cast<int>(n);
#define ARGS tmA, m, nn, np4, rpc, nst, Q, Z, cpart, G, tickets, l, tau_host, tau_from_mu, update_rp, advance_counter, \
             Rf, Qt, dst, rank_tol, max_sweeps
  if (LP == 16) {
    if (gram) k_tp_lr<16, true><<<grid, Cfg<16>::NT, smem, st>>>(ARGS);
    else k_tp_lr<16, false><<<grid, Cfg<16>::NT, smem, st>>>(ARGS);
  } else {
    if (gram) k_tp_lr<32, true><<<grid, Cfg<32>::NT, smem, st>>>(ARGS);
    else k_tp_lr<32, false><<<grid, Cfg<32>::NT, smem, st>>>(ARGS);
  }
#undef ARGS
  return cudaGetLastError();
}

cudaError_t launch_tp_alm(int LP, const CUtensorMap& tmO, const CUtensorMap& tmS, const CUtensorMap& tmA,
                          const CUtensorMap& tmZ, int64_t m, int64_t n, int64_t rpc, int grid, const float* Rf,
                          float* S, float* A, int64_t ld, float* L, int64_t ldl, DevState* dst, double* cpart,
                          unsigned* tickets, void* Ab, int64_t ldb, cudaStream_t st) {
  const int np4 = tma_np4(n);
  const size_t smem = tma_alm_smem(LP, n);
  const int nse = tma_alm_stages(LP, n);
  if (nse < 2) return cudaErrorInvalidValue;
  const int nn = static_cast<int>(n);
  __nv_bfloat16* ab = static_cast<__nv_bfloat16*>(Ab);
  if (LP == 16)
    k_tp_alm<16><<<grid, kAlmNT, smem, st>>>(tmO, tmS, tmA, tmZ, m, nn, np4, rpc, Rf, S, A, ld, L, ldl, dst,
                                                   cpart, tickets, ab, ldb, nse);
  else
    k_tp_alm<32><<<grid, kAlmNT, smem, st>>>(tmO, tmS, tmA, tmZ, m, nn, np4, rpc, Rf, S, A, ld, L, ldl, dst,
                                                   cpart, tickets, ab, ldb, nse);
  return cudaGetLastError();
}

}  // namespace frsvt
