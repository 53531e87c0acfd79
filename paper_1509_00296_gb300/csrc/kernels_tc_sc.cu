// Y = A^T B on the fifth-generation tensor cores (tcgen05), FP32-accurate, with the
// orthonormal basis of Y computed by the CTA that finishes the reduction last.
//
// This is the column pass of Alg. 1: the sketch Y = A^T Omega (steps 4-5 / 8-9, Omega drawn
// in-kernel from the Philox stream) and the second half of a power step, Y = A^T Z (step 14).
// As an MMA, D (n x LP) += A_blk^T (n x 32 rows) B_blk (32 rows x LP): the A tile is the
// MN-major operand (each loaded 128-byte row holds 32 consecutive columns of A, the MN
// index), B_blk^T is written by the split warps as a K-major operand.  M = 128 columns of A
// per MMA (one or two M tiles cover n <= 256), N = LP, K = 8; the accumulators stay in tensor
// memory across all row blocks of the CTA (split-K over rows), then go to shared memory, to
// the cluster reduction (cluster.cuh) and to the orthonormalisation (small_dense.cuh).
// 3xTF32: the split warps rewrite each tile as A_hi in place and write A_lo to a small ring.
// Warp roles: 0 TMA producer, 1 tensor-memory owner + MMA issuer, 2-5 split / drain.
#include <cuda.h>

#include "cluster.cuh"
#include "common.cuh"
#include "small_dense.cuh"
#include "state.cuh"
#include "tc.cuh"
#include "tma.cuh"

namespace frsvt {

namespace {

constexpr int kRows = 32;                 // rows of A per block (the MMA K of one block)
constexpr int kChunk = kRows * 128;       // one 32-column chunk of a block: 4 KB
constexpr int kThr = 192;
constexpr int kGaccT = 1024;

struct ScLayout {
  int mt, nch, ns;
  uint32_t a_bytes, z_bytes, stage, lo, b;
  uint32_t off_lo, off_b, total;
};

__host__ __device__ inline ScLayout sc_layout(int LP, int n, bool omega, int ns) {
  ScLayout L;
  L.mt = (n + 127) / 128;
  L.nch = 4 * L.mt;
  L.ns = ns;
  L.a_bytes = static_cast<uint32_t>(L.nch) * kChunk;
  L.z_bytes = omega ? 0u : static_cast<uint32_t>(kRows * LP * 4);
  L.stage = (L.a_bytes + L.z_bytes + 1023u) / 1024u * 1024u;
  L.lo = L.a_bytes;
  L.b = static_cast<uint32_t>(LP) * 128u * 2u;      // B_hi | B_lo of one block
  L.off_lo = static_cast<uint32_t>(ns) * L.stage;
  L.off_b = L.off_lo + 2u * L.lo;
  L.total = L.off_b + 2u * L.b;
  return L;
}

template <int LP, bool OMEGA, bool TAIL>
__global__ void __cluster_dims__(kCL, 1, 1) __launch_bounds__(kThr, 1)
k_tc_sc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmZ, int64_t m, int n,
        int64_t rpc, int ns, uint64_t seed, uint64_t ctr, DevState* __restrict__ dst, float* __restrict__ cpart,
        float* __restrict__ Y, unsigned* __restrict__ tickets, int l, int use_rp, int passes,
        const float* __restrict__ Qt, float* __restrict__ Qout, double rank_tol) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ __align__(8) uint64_t full[4], ready[4], empty[4], lofree[2], acc_full;
  __shared__ uint32_t tmem_base;
  __shared__ int flag;
  const ScLayout Lt = sc_layout(LP, n, OMEGA, ns);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * rpc;
  const int64_t r1 = imin64(m, r0 + rpc);
  const int nb = (r1 > r0) ? static_cast<int>((r1 - r0 + kRows - 1) / kRows) : 0;
  const uint32_t ncols = (Lt.mt * LP >= 32) ? static_cast<uint32_t>(Lt.mt * LP) : 32u;
  const uint64_t stream = OMEGA ? ((ctr == kCounterFromState) ? dst->counter : ctr) : 0ull;
  if (threadIdx.x == 0) {
    for (int s = 0; s < ns; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&ready[s], 4);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&lofree[0], 1);
    mbar_init(&lofree[1], 1);
    mbar_init(&acc_full, 1);
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc(&tmem_base, ncols <= 32 ? 32u : 64u);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base;
  bool ok = true;

  if (warp == 0) {
    if (lane == 0) {
      prefetch_tensormap(&tmA);
      if (!OMEGA) prefetch_tensormap(&tmZ);
      for (int b = 0; b < nb && ok; ++b) {
        const int s = b % ns, u = b / ns;
        if (u > 0 && !mbar_wait(&empty[s], static_cast<uint32_t>(u - 1) & 1u)) {
          ok = false;
          atomicOr(&dst->status, kDevTimeout);
          break;
        }
        unsigned char* st = dsm + s * Lt.stage;
        const int y = static_cast<int>(r0 + static_cast<int64_t>(b) * kRows);
        mbar_arrive_expect_tx(&full[s], Lt.a_bytes + Lt.z_bytes);
        for (int c = 0; c < Lt.nch; ++c) tma_load_2d(st + c * kChunk, &tmA, 32 * c, y, &full[s]);
        if (!OMEGA) tma_load_2d(st + Lt.a_bytes, &tmZ, 0, y, &full[s]);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_tf32(128, LP, true, false);
      for (int b = 0; b < nb; ++b) {
        const int s = b % ns, u = b / ns;
        if (ok && !mbar_wait(&ready[s], static_cast<uint32_t>(u) & 1u)) {
          ok = false;
          atomicOr(&dst->status, kDevTimeout);
        }
        tc_fence_after();
        const unsigned char* ahi = dsm + s * Lt.stage;
        const unsigned char* alo = dsm + Lt.off_lo + (b & 1) * Lt.lo;
        const unsigned char* bh = dsm + Lt.off_b + (b & 1) * Lt.b;
        const unsigned char* bl = bh + LP * 128;
        for (int mt = 0; mt < Lt.mt; ++mt) {
          const uint32_t d = tbase + static_cast<uint32_t>(mt * LP);
#pragma unroll
          for (int ks = 0; ks < kRows / 8; ++ks) {
            const uint64_t dah = smem_desc_sw128a32_mn(ahi + (4 * mt) * kChunk + ks * 1024, kChunk);
            const uint64_t dal = smem_desc_sw128a32_mn(alo + (4 * mt) * kChunk + ks * 1024, kChunk);
            const uint64_t dbh = smem_desc_sw128(bh + 32 * ks, 16, 1024);
            const uint64_t dbl = smem_desc_sw128(bl + 32 * ks, 16, 1024);
            tc_mma_tf32(d, dah, dbh, idesc, b > 0 || ks > 0);
            tc_mma_tf32(d, dah, dbl, idesc, true);
            tc_mma_tf32(d, dal, dbh, idesc, true);
          }
        }
        tc_commit(&empty[s]);
        tc_commit(&lofree[b & 1]);
      }
      tc_commit(&acc_full);
    }
  } else {
    const int t = threadIdx.x - 64;                                  // 0..127
    for (int b = 0; b < nb; ++b) {
      const int s = b % ns, u = b / ns;
      if (ok && !mbar_wait(&full[s], static_cast<uint32_t>(u) & 1u)) {
        ok = false;
        atomicOr(&dst->status, kDevTimeout);
      }
      if (b >= 2 && ok && !mbar_wait(&lofree[b & 1], static_cast<uint32_t>(b / 2 - 1) & 1u)) {
        ok = false;
        atomicOr(&dst->status, kDevTimeout);
      }
      float4* hi = reinterpret_cast<float4*>(dsm + s * Lt.stage);
      float4* lo = reinterpret_cast<float4*>(dsm + Lt.off_lo + (b & 1) * Lt.lo);
      const int nv = static_cast<int>(Lt.a_bytes / 16);
      for (int e = t; e < nv; e += 128) {
        const float4 v = hi[e];
        const float4 h = make_float4(tf32_hi(v.x), tf32_hi(v.y), tf32_hi(v.z), tf32_hi(v.w));
        hi[e] = h;
        lo[e] = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
      }
      // B^T of the block: row k (0..LP) of 32 K-elements = B[row r of the block][k]
      unsigned char* bh = dsm + Lt.off_b + (b & 1) * Lt.b;
      unsigned char* bl = bh + LP * 128;
      const int64_t i0 = r0 + static_cast<int64_t>(b) * kRows;
      if (OMEGA) {
        for (int q = t; q < kRows * (LP / 4); q += 128) {
          const int r = q / (LP / 4), blk = q % (LP / 4);
          float4 gv = make_float4(0.f, 0.f, 0.f, 0.f);
          if (i0 + r < r1) gv = gaussian4(seed, static_cast<uint64_t>(i0 + r), static_cast<uint64_t>(blk), stream, 0ull);
          const float vals[4] = {gv.x, gv.y, gv.z, gv.w};
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int k = 4 * blk + c;
            const float hv = tf32_hi(vals[c]);
            *reinterpret_cast<float*>(bh + sw128_offset(k, r)) = hv;
            *reinterpret_cast<float*>(bl + sw128_offset(k, r)) = vals[c] - hv;
          }
        }
      } else {
        const float* zt = reinterpret_cast<const float*>(dsm + s * Lt.stage + Lt.a_bytes);   // kRows x LP
        for (int q = t; q < kRows * LP; q += 128) {
          const int r = q / LP, k = q % LP;
          const float v = (i0 + r < r1) ? zt[r * LP + k] : 0.f;
          const float hv = tf32_hi(v);
          *reinterpret_cast<float*>(bh + sw128_offset(k, r)) = hv;
          *reinterpret_cast<float*>(bl + sw128_offset(k, r)) = v - hv;
        }
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(&ready[s]);
    }
    // drain the accumulators: warp quarter q reads tensor-memory lanes 32q..32q+31 = columns of A
    if (ok && !mbar_wait(&acc_full, 0u)) {
      ok = false;
      atomicOr(&dst->status, kDevTimeout);
    }
    tc_fence_after();
  }
  __syncthreads();
  float* part_sm = reinterpret_cast<float*>(dsm);                   // n x LP (the pipeline is idle)
  if (warp >= 2) {
    const int sub = warp & 3;
    for (int mt = 0; mt < Lt.mt; ++mt) {
      const int j = 128 * mt + 32 * sub + lane;
#pragma unroll
      for (int h16 = 0; h16 < LP / 16; ++h16) {
        float v[16];
        tmem_ld16(tbase + (static_cast<uint32_t>(32 * sub) << 16) + static_cast<uint32_t>(mt * LP + 16 * h16), v);
        if (j < n)
#pragma unroll
          for (int k = 0; k < 16; ++k) part_sm[j * LP + 16 * h16 + k] = (nb > 0) ? v[k] : 0.f;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tbase, ncols <= 32 ? 32u : 64u);
  const int nclusters = gridDim.x / kCL;
  if (!cluster_split_reduce<float>(part_sm, n * LP, cpart, Y, tickets, blockIdx.x / kCL, nclusters, &flag)) return;
  if (!TAIL) return;
  if (cooperative_groups::this_cluster().block_rank() != 0) return;
  SmallWs<LP> w = carve_small_ws<LP>(dsm, kGaccT);
  int keep = use_rp ? dst->keep : 0;
  keep = max(0, min(keep, l));
  for (int e = threadIdx.x; e < n * LP; e += kThr) {
    const int col = e % LP;
    const int i = e / LP;
    float v = 0.f;
    if (col < keep) v = Qt[e];
    else if (col < l) v = __ldcg(Y + i * LP + (col - keep));
    w.W[e] = v;
  }
  __syncthreads();
  const int s = orth_block<LP>(w, n, keep, l, rank_tol, passes);
  for (int e = threadIdx.x; e < n * LP; e += kThr) Qout[e] = w.W[e];
  if (threadIdx.x == 0) {
    dst->s = s;
    if (s < l) dst->status |= kDevRankDeficient;
  }
}

template <typename K>
cudaError_t set_limit(K kernel, int smem_limit) {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              smem_limit - static_cast<int>(a.sharedSizeBytes));
}

}  // namespace

// Stages of the tensor-core column pass that fit in `limit` bytes (0 if none fits).
int tc_sc_stages(int LP, int64_t n, bool omega, size_t limit) {
  for (int ns = 4; ns >= 2; --ns)
    if (sc_layout(LP, static_cast<int>(n), omega, ns).total <= limit) return ns;
  return 0;
}

size_t tc_sc_smem(int LP, int64_t n, bool omega, int ns) {
  const size_t a = sc_layout(LP, static_cast<int>(n), omega, ns).total;
  const size_t ws = LP == 16 ? small_ws_bytes<16>(n, kGaccT) : small_ws_bytes<32>(n, kGaccT);
  const size_t part = static_cast<size_t>(n) * LP * sizeof(float);
  size_t r = a > ws ? a : ws;
  return r > part ? r : part;
}

cudaError_t prepare_tc_sc_kernels(int smem_limit) {
  cudaError_t e = cudaSuccess;
#define PREP(...) \
  if (e == cudaSuccess) e = set_limit(__VA_ARGS__, smem_limit);
  PREP(k_tc_sc<16, true, true>);
  PREP(k_tc_sc<16, false, true>);
  PREP(k_tc_sc<32, true, true>);
  PREP(k_tc_sc<32, false, true>);
  PREP(k_tc_sc<16, true, false>);
  PREP(k_tc_sc<16, false, false>);
  PREP(k_tc_sc<32, true, false>);
  PREP(k_tc_sc<32, false, false>);
#undef PREP
  return e;
}

// Largest resident grid of this kernel in whole clusters.
int tc_sc_resident_grid(int LP, int64_t n, int ns) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kCL, 1, 1);
  cfg.blockDim = dim3(kThr, 1, 1);
  cfg.dynamicSmemBytes = tc_sc_smem(LP, n, false, ns);
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = kCL;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  int nc = 0;
  const void* fn = LP == 16 ? reinterpret_cast<const void*>(k_tc_sc<16, false, true>)
                            : reinterpret_cast<const void*>(k_tc_sc<32, false, true>);
  if (cudaOccupancyMaxActiveClusters(&nc, fn, &cfg) != cudaSuccess) nc = 0;
  (void)cudaGetLastError();
  return nc * kCL;
}

// tmA: 32-column x 32-row boxes in the 128-byte swizzle with 32-byte atoms; tmZ (when B = Z): LP x 32-row boxes of Z.
cudaError_t launch_tc_sc(int LP, const CUtensorMap& tmA, const CUtensorMap* tmZ, int64_t m, int64_t n, int grid,
                         int ns, uint64_t seed, uint64_t ctr, DevState* dst, float* cpart, float* Y,
                         unsigned* tickets, bool tail, int l, int use_rp, int passes, const float* Qt, float* Q,
                         double rank_tol, cudaStream_t st) {
  int64_t rpc = (m + grid - 1) / grid;
  rpc = (rpc + kRows - 1) / kRows * kRows;
  const bool omega = tmZ == nullptr;
  const size_t smem = tc_sc_smem(LP, n, omega, ns);
  const int nn = static_cast<int>(n);
  const CUtensorMap& z = tmZ ? *tmZ : tmA;
#define ARGS tmA, z, m, nn, rpc, ns, seed, ctr, dst, cpart, Y, tickets, l, use_rp, passes, Qt, Q, rank_tol
#define GO(LPV, OM, TL) k_tc_sc<LPV, OM, TL><<<grid, kThr, smem, st>>>(ARGS)
  if (LP == 16) {
    if (omega) { if (tail) GO(16, true, true); else GO(16, true, false); }
    else { if (tail) GO(16, false, true); else GO(16, false, false); }
  } else {
    if (omega) { if (tail) GO(32, true, true); else GO(32, true, false); }
    else { if (tail) GO(32, false, true); else GO(32, false, false); }
  }
#undef GO
#undef ARGS
  return cudaGetLastError();
}

int tc_sc_rows() { return kRows; }

}  // namespace frsvt
