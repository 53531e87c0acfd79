// Y = A^T B on the fifth-generation tensor cores (tcgen05), FP32-accurate, with the
// orthonormal basis of Y computed by the CTA that finishes the reduction last.
//
// This is the column pass of Alg. 1: the sketch Y = A^T Omega (steps 4-5 / 8-9, Omega drawn
// in-kernel from the Philox stream) and the second half of a power step, Y = A^T Z (step 14).
//
// A kind::tf32 MMA instruction (K = 8) occupies the tensor core for about the same time
// whatever its N (up to 256), so every instruction covers all n <= 256 columns of A:
//     D (128 x N) += Bs (128 x 8 rows of A) . A_blk (8 rows x N),  N = n rounded up to 16,
// i.e. D holds Y^T.  Bs is B_blk^T split into TF32 parts and stacked (row 32 (k / 16) +
// 16 part + k % 16 holds part hi / lo of column k of B), written K-major by the B warps; the
// rest of its 128-row window is whatever follows in shared memory and only feeds accumulator
// rows that are never read.  The A tile is the MN-major operand (each loaded 128-byte row
// holds 32 consecutive columns of A), which kind::tf32 reads only in the 128-byte swizzle with
// 32-byte atoms.  3xTF32: Bs . A_hi + Bs . A_lo with the raw tile as A_hi (the MMA reads only
// the 19 leading bits of each word); once the A_hi MMAs of a block have completed, split warps
// overwrite the tile in place with A_lo = A - A_hi.  The accumulator stays in tensor memory
// across all row blocks of the CTA (split-K over rows), then goes to shared memory, to the
// cluster reduction (cluster.cuh) and to the orthonormalisation (small_dense.cuh).
// Warp roles: 0 TMA producer, 1 tensor-memory owner + MMA issuer (A_hi MMAs of block b, then
// the A_lo MMAs of block b - 1), 2-5 B warps, 6-13 split warps; lane-quarter 0 / 1 warps drain.
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
constexpr int kChunk = kRows * 128;       // one 32-column group of a block: 4 KB
constexpr int kBWarps = 4;
constexpr int kSplitWarps = 8;
constexpr int kThr = 64 + 32 * (kBWarps + kSplitWarps);
constexpr int kScCL = 4;                  // CTAs per cluster of the split-K reduction
constexpr int kMaxNS = 6;                 // most pipeline stages
constexpr int kGaccT = 1024;

struct ScLayout {
  int nch, ns, N;
  uint32_t a_bytes, z_bytes, stage, bslot;
  uint32_t off_b, total;
};

__host__ __device__ inline ScLayout sc_layout(int LP, int n, bool omega, int ns) {
  ScLayout L;
  L.nch = (n + 31) / 32;
  L.ns = ns;
  L.N = (n + 15) / 16 * 16;
  L.a_bytes = static_cast<uint32_t>(L.nch) * kChunk;
  L.z_bytes = omega ? 0u : static_cast<uint32_t>(kRows * LP * 4);
  L.stage = (L.a_bytes + L.z_bytes + 1023u) / 1024u * 1024u;
  L.bslot = static_cast<uint32_t>(2 * LP) * 128u;
  L.off_b = static_cast<uint32_t>(ns) * L.stage;
  L.total = L.off_b + static_cast<uint32_t>(ns) * L.bslot + static_cast<uint32_t>(128 - 2 * LP) * 128u;
  return L;
}

// Stacked row of part (0 hi, 1 lo) of column k in the M operand.
__host__ __device__ constexpr int stack_row(int k, int part) { return 32 * (k / 16) + 16 * part + (k % 16); }

// Tensor-memory columns for `need` accumulator columns (a power of two, at least 32).
__host__ __device__ constexpr uint32_t tmem_cols(int need) {
  return need <= 32 ? 32u : need <= 64 ? 64u : need <= 128 ? 128u : 256u;
}

template <int LP, bool OMEGA, bool TAIL>
__global__ void __cluster_dims__(kScCL, 1, 1) __launch_bounds__(kThr, 1)
k_tc_sc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmZ, int64_t m, int n,
        int64_t rpc, int ns, uint64_t seed, uint64_t ctr, DevState* __restrict__ dst, float* __restrict__ cpart,
        float* __restrict__ Y, unsigned* __restrict__ tickets, int l, int use_rp, int passes,
        const float* __restrict__ Qt, float* __restrict__ Qout, double rank_tol) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ __align__(8) uint64_t full[kMaxNS], bready[kMaxNS], hidone[kMaxNS], lo_ready[kMaxNS], empty[kMaxNS],
      acc_full;
  __shared__ uint32_t tmem_base;
  __shared__ int flag;
  const ScLayout Lt = sc_layout(LP, n, OMEGA, ns);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * rpc;
  const int64_t r1 = imin64(m, r0 + rpc);
  const int nb = (r1 > r0) ? static_cast<int>((r1 - r0 + kRows - 1) / kRows) : 0;
  const uint32_t ncols = tmem_cols(Lt.N);
  constexpr int kDrainQ = LP / 16;
  const uint64_t stream = OMEGA ? ((ctr == kCounterFromState) ? dst->counter : ctr) : 0ull;
  unsigned char* bring = dsm + Lt.off_b;
  for (uint32_t e = threadIdx.x; e < (Lt.total - Lt.off_b) / 4; e += kThr) reinterpret_cast<float*>(bring)[e] = 0.f;
  fence_proxy_async();
  if (threadIdx.x == 0) {
    for (int s = 0; s < ns; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&bready[s], kBWarps);
      mbar_init(&hidone[s], 1);
      mbar_init(&lo_ready[s], kSplitWarps);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&acc_full, 1);
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc(&tmem_base, ncols);
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
      const uint32_t idesc = idesc_tf32(128, Lt.N, false, true);
      auto issue = [&](int b, bool lo_part) {
        const int s = b % ns;
        const unsigned char* bs = bring + s * Lt.bslot;
        const unsigned char* at = dsm + s * Lt.stage;
#pragma unroll
        for (int ks = 0; ks < kRows / 8; ++ks)
          tc_mma_tf32(tbase, smem_desc_sw128(bs + 32 * ks, 16, 1024), smem_desc_sw128a32_mn(at + ks * 1024, kChunk),
                      idesc, lo_part || b > 0 || ks > 0);
      };
      auto issue_lo = [&](int b) {
        const int s = b % ns, u = b / ns;
        if (ok && !mbar_wait(&lo_ready[s], static_cast<uint32_t>(u) & 1u)) {
          ok = false;
          atomicOr(&dst->status, kDevTimeout);
        }
        tc_fence_after();
        issue(b, true);
        tc_commit(&empty[s]);
      };
      for (int b = 0; b < nb; ++b) {
        const int s = b % ns, u = b / ns;
        if (ok && (!mbar_wait(&full[s], static_cast<uint32_t>(u) & 1u) ||
                   !mbar_wait(&bready[s], static_cast<uint32_t>(u) & 1u))) {
          ok = false;
          atomicOr(&dst->status, kDevTimeout);
        }
        tc_fence_after();
        issue(b, false);
        tc_commit(&hidone[s]);
        if (b > 0) issue_lo(b - 1);
      }
      if (nb > 0) issue_lo(nb - 1);
      tc_commit(&acc_full);
    }
  } else if (warp < 2 + kBWarps) {
    // B warps: [B_hi; B_lo]^T of each block into its slot (K-major, 128-byte swizzle).
    const int t = threadIdx.x - 64;
    for (int b = 0; b < nb; ++b) {
      const int s = b % ns, u = b / ns;
      if (ok && !mbar_wait(&full[s], static_cast<uint32_t>(u) & 1u)) {
        ok = false;
        atomicOr(&dst->status, kDevTimeout);
      }
      unsigned char* bs = bring + s * Lt.bslot;
      const int64_t i0 = r0 + static_cast<int64_t>(b) * kRows;
      if (OMEGA) {
        for (int q = t; q < kRows * (LP / 4); q += 32 * kBWarps) {
          const int r = q / (LP / 4), blk = q % (LP / 4);
          float4 gv = make_float4(0.f, 0.f, 0.f, 0.f);
          if (i0 + r < r1) gv = gaussian4(seed, static_cast<uint64_t>(i0 + r), static_cast<uint64_t>(blk), stream, 0ull);
          const float vals[4] = {gv.x, gv.y, gv.z, gv.w};
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int k = 4 * blk + c;
            const float hv = tf32_hi(vals[c]);
            *reinterpret_cast<float*>(bs + sw128_offset(stack_row(k, 0), r)) = hv;
            *reinterpret_cast<float*>(bs + sw128_offset(stack_row(k, 1), r)) = vals[c] - hv;
          }
        }
      } else {
        const float* zt = reinterpret_cast<const float*>(dsm + s * Lt.stage + Lt.a_bytes);   // kRows x LP
        for (int q = t; q < kRows * LP; q += 32 * kBWarps) {
          const int r = q / LP, k = q % LP;
          const float v = (i0 + r < r1) ? zt[r * LP + k] : 0.f;
          const float hv = tf32_hi(v);
          *reinterpret_cast<float*>(bs + sw128_offset(stack_row(k, 0), r)) = hv;
          *reinterpret_cast<float*>(bs + sw128_offset(stack_row(k, 1), r)) = v - hv;
        }
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bready[s]);
    }
    if (ok && !mbar_wait(&acc_full, 0u)) {
      ok = false;
      atomicOr(&dst->status, kDevTimeout);
    }
  } else {
    // split warps: once the A_hi MMAs of a block are done, its tile becomes A_lo in place
    const int t = threadIdx.x - 32 * (2 + kBWarps);
    const int nv = static_cast<int>(Lt.a_bytes / 16);
    for (int b = 0; b < nb; ++b) {
      const int s = b % ns, u = b / ns;
      if (ok && !mbar_wait(&hidone[s], static_cast<uint32_t>(u) & 1u)) {
        ok = false;
        atomicOr(&dst->status, kDevTimeout);
      }
      float4* a = reinterpret_cast<float4*>(dsm + s * Lt.stage);
#pragma unroll 4
      for (int e = t; e < nv; e += 32 * kSplitWarps) {
        const float4 v = a[e];
        a[e] = make_float4(v.x - tf32_hi(v.x), v.y - tf32_hi(v.y), v.z - tf32_hi(v.z), v.w - tf32_hi(v.w));
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(&lo_ready[s]);
    }
    if (ok && !mbar_wait(&acc_full, 0u)) {
      ok = false;
      atomicOr(&dst->status, kDevTimeout);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // drain: accumulator row 32 q + L (lane quarter q) is part (L / 16) of column 16 q + L % 16
  // of Y; TMEM column j is column j of A.  The three warps of a quarter take every third group
  // of 16 columns.
  float* part_sm = reinterpret_cast<float*>(dsm);                   // n x LP (the pipeline is idle)
  if (warp >= 4 && (warp & 3) < kDrainQ) {
    const int q = warp & 3, idx = (warp >> 2) - 1;
    const int nwq = (kThr / 32 - 1 - q) / 4;                        // warps >= 4 in quarter q
    for (int grp = idx; grp < Lt.N / 16; grp += nwq) {
      float v[16];
      tmem_ld16(tbase + (static_cast<uint32_t>(32 * q) << 16) + static_cast<uint32_t>(16 * grp), v);
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] += __shfl_down_sync(0xffffffffu, v[i], 16);
      if (lane < 16) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int j = 16 * grp + i;
          if (j < n) part_sm[j * LP + 16 * q + lane] = (nb > 0) ? v[i] : 0.f;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tbase, ncols);
  const int nclusters = gridDim.x / kScCL;
  if (!cluster_split_reduce<float, kScCL>(part_sm, n * LP, cpart, Y, tickets, blockIdx.x / kScCL, nclusters, &flag))
    return;
  if (!TAIL) return;
  if (cooperative_groups::this_cluster().block_rank() != 0) return;
  SmallWs<LP> w = carve_small_ws<LP>(dsm, kGaccT);
  if (l <= 0) l = min(max(dst->l_cur, 1), LP);            // adaptive rank prediction: l lives on the device
  int keep = use_rp ? dst->keep : 0;
  keep = max(0, min(keep, l));
  load_basis_block<LP>(w.W, n, keep, l, Qt, Y);
  __syncthreads();
  float rp_res = -1.f;
  const int s = orth_block<LP>(w, n, keep, l, rank_tol, passes, &rp_res, &dst->status);
  for (int e = threadIdx.x; e < n * LP; e += kThr) Qout[e] = w.W[e];
  if (threadIdx.x == 0) {
    if (use_rp) dst->rp_res = rp_res;
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
  for (int ns = kMaxNS; ns >= 2; --ns)
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
  cfg.gridDim = dim3(kScCL, 1, 1);
  cfg.blockDim = dim3(kThr, 1, 1);
  cfg.dynamicSmemBytes = tc_sc_smem(LP, n, false, ns);
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = kScCL;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  int nc = 0;
  const void* fn = LP == 16 ? reinterpret_cast<const void*>(k_tc_sc<16, false, true>)
                            : reinterpret_cast<const void*>(k_tc_sc<32, false, true>);
  if (cudaOccupancyMaxActiveClusters(&nc, fn, &cfg) != cudaSuccess) nc = 0;
  (void)cudaGetLastError();
  return nc * kScCL;
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
