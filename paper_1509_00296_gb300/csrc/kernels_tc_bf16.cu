// Row and column passes of Alg. 1 on a BF16 shadow of A (the reduced-precision sketch and early
// power steps; the last power step and the projection stay FP32-accurate).
//
// Same layouts as the FP32-accurate passes (kernels_tc.cu, kernels_tc_sc.cu) with kind::f16
// MMAs (BF16 operands, FP32 accumulation, K = 16 per instruction): the long side of A is the MMA
// N, the narrow factor (Q, Omega or Z) is split into BF16 hi / lo parts stacked in the M = 128
// operand, so its rounding does not count and only A's BF16 rounding remains.  A 128-byte row
// holds 64 BF16 elements; the column pass reads A MN-major in the plain 128-byte swizzle.  No
// split warps: one MMA per K step reads half the bytes of the FP32 passes.
#include <cuda.h>
#include <cuda_bf16.h>

#include "cluster.cuh"
#include "common.cuh"
#include "small_dense.cuh"
#include "state.cuh"
#include "tc.cuh"
#include "tma.cuh"

namespace frsvt {

namespace {

constexpr int kMaxNSb = 6;

// Stacked row of part (0 hi, 1 lo) of column k in the M operand.
__host__ __device__ constexpr int stack_row_b(int k, int part) { return 32 * (k / 16) + 16 * part + (k % 16); }

// Byte offset of element (row, k) (k < 64) in a K-major 128-byte-swizzled BF16 tile.
__device__ __forceinline__ uint32_t sw128_bf16(int row, int k) {
  return static_cast<uint32_t>(row) * 128u + (static_cast<uint32_t>((k >> 3) ^ (row & 7)) * 16u) +
         static_cast<uint32_t>(k & 7) * 2u;
}

// kind::f16 instruction descriptor, BF16 A and B, FP32 accumulation, shape M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, bool b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((b_mn ? 1u : 0u) << 16) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, bool acc) {
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "setp.ne.u32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc ? 1u : 0u)
      : "memory");
}

__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(v);
  lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// ---------------------------------------------------------------- row pass Z = A_b Q
constexpr int kBNb = 256;                      // rows of A per block (MMA N)
constexpr int kBKb = 64;                       // BF16 per K-chunk (128 bytes)
constexpr uint32_t kChunkB = kBNb * 128u;      // 32 KB
constexpr int kLrThr = 64 + 128;               // producer, MMA, 4 drain warps

__host__ __device__ inline uint32_t lrb_q_bytes(int LP, int n) {
  const int nkc = (n + kBKb - 1) / kBKb;
  return static_cast<uint32_t>(nkc) * 2u * LP * 128u + static_cast<uint32_t>(128 - 2 * LP) * 128u;
}

template <int LP>
__global__ void __launch_bounds__(kLrThr, 1)
k_tb_lr(const __grid_constant__ CUtensorMap tmA, int64_t m, int n, int64_t rpc, int ns, const float* __restrict__ Q,
        float* __restrict__ Z, DevState* __restrict__ dst) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ __align__(8) uint64_t full[kMaxNSb], empty[kMaxNSb], acc_full[2], acc_empty[2], fin;
  __shared__ uint32_t tmem_base;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkc = (n + kBKb - 1) / kBKb;
  const uint32_t qchunk = 2u * LP * 128u;
  const uint32_t qbytes = lrb_q_bytes(LP, n);
  unsigned char* Qs = dsm;
  unsigned char* ring = dsm + qbytes;
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * rpc;
  const int64_t r1 = imin64(m, r0 + rpc);
  const int nb = (r1 > r0) ? static_cast<int>((r1 - r0 + kBNb - 1) / kBNb) : 0;
  const int total = nb * nkc;
  constexpr int kDrainQ = LP / 16;
  for (int e = threadIdx.x; e < static_cast<int>(qbytes / 4); e += kLrThr) reinterpret_cast<float*>(Qs)[e] = 0.f;
  __syncthreads();
  for (int e = threadIdx.x; e < nkc * kBKb * LP; e += kLrThr) {
    const int k = e % LP, j = e / LP;
    const float q = (j < n) ? Q[static_cast<int64_t>(j) * LP + k] : 0.f;
    __nv_bfloat16 hi, lo;
    split_bf16(q, hi, lo);
    unsigned char* qc = Qs + static_cast<uint32_t>(j / kBKb) * qchunk;
    *reinterpret_cast<__nv_bfloat16*>(qc + sw128_bf16(stack_row_b(k, 0), j % kBKb)) = hi;
    *reinterpret_cast<__nv_bfloat16*>(qc + sw128_bf16(stack_row_b(k, 1), j % kBKb)) = lo;
  }
  fence_proxy_async();
  if (threadIdx.x == 0) {
    for (int s = 0; s < ns; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], kDrainQ);
    }
    mbar_init(&fin, 1);
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc(&tmem_base, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base;
  bool ok = true;
  if (warp == 0) {
    if (lane == 0) {
      prefetch_tensormap(&tmA);
      for (int g = 0; g < total && ok; ++g) {
        const int s = g % ns, u = g / ns;
        if (u > 0 && !mbar_wait(&empty[s], static_cast<uint32_t>(u - 1) & 1u)) {
          ok = false;
          atomicOr(&dst->status, kDevTimeout);
          break;
        }
        mbar_arrive_expect_tx(&full[s], kChunkB);
        tma_load_2d(ring + s * kChunkB, &tmA, (g % nkc) * kBKb,
                    static_cast<int>(r0 + static_cast<int64_t>(g / nkc) * kBNb), &full[s]);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16(128, kBNb, false);
      for (int g = 0; g < total; ++g) {
        const int s = g % ns, u = g / ns, c = g % nkc, b = g / nkc;
        if (c == 0 && b >= 2 && ok && !mbar_wait(&acc_empty[b & 1], static_cast<uint32_t>(b / 2 - 1) & 1u)) {
          ok = false;
          atomicOr(&dst->status, kDevTimeout);
        }
        if (ok && !mbar_wait(&full[s], static_cast<uint32_t>(u) & 1u)) {
          ok = false;
          atomicOr(&dst->status, kDevTimeout);
        }
        tc_fence_after();
        const uint32_t d = tbase + static_cast<uint32_t>((b & 1) * kBNb);
#pragma unroll
        for (int ks = 0; ks < kBKb / 16; ++ks)
          tc_mma_bf16(d, smem_desc_sw128(Qs + c * qchunk + 32 * ks, 16, 1024),
                      smem_desc_sw128(ring + s * kChunkB + 32 * ks, 16, 1024), idesc, c > 0 || ks > 0);
        tc_commit(&empty[s]);
        if (c == nkc - 1) tc_commit(&acc_full[b & 1]);
      }
      tc_commit(&fin);
      if (!mbar_wait(&fin, 0u)) atomicOr(&dst->status, kDevTimeout);
    }
  } else {
    const int sub = warp & 3;                  // warps 2..5: lane quarters 2, 3, 0, 1
    if (sub < kDrainQ) {
      for (int b = 0; b < nb; ++b) {
        const int buf = b & 1;
        if (ok && !mbar_wait(&acc_full[buf], static_cast<uint32_t>(b / 2) & 1u)) {
          ok = false;
          atomicOr(&dst->status, kDevTimeout);
        }
        tc_fence_after();
        const int k = 16 * sub + (lane & 15);
        const int64_t rb = r0 + static_cast<int64_t>(b) * kBNb;
        for (int cg = 0; cg < kBNb / 16; ++cg) {
          float v[16];
          tmem_ld16(tbase + (static_cast<uint32_t>(32 * sub) << 16) + static_cast<uint32_t>(buf * kBNb + 16 * cg), v);
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] += __shfl_down_sync(0xffffffffu, v[i], 16);
          if (lane < 16) {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const int64_t row = rb + 16 * cg + i;
              if (row < r1) Z[row * LP + k] = v[i];
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[buf]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tbase, 512);
}

// ---------------------------------------------------------------- column pass Y = A_b^T B
constexpr int kRowsB = 64;                     // rows of A per block (the MMA K of a block)
constexpr uint32_t kBoxB = kRowsB * 128u;      // one 64-column box: 8 KB
constexpr int kScThr = 64 + 128;               // producer, MMA, 4 B warps (drain: quarter warps)
constexpr int kScCLb = 4;
constexpr int kGaccB = 1024;

struct ScbLayout {
  int nch, ns, N;
  uint32_t a_bytes, z_bytes, stage, bslot, off_b, total;
};

__host__ __device__ inline ScbLayout scb_layout(int LP, int n, bool omega, int ns) {
  ScbLayout L;
  L.nch = (n + 63) / 64;
  L.ns = ns;
  L.N = (n + 15) / 16 * 16;
  L.a_bytes = static_cast<uint32_t>(L.nch) * kBoxB;
  L.z_bytes = omega ? 0u : static_cast<uint32_t>(kRowsB * LP * 4);
  L.stage = (L.a_bytes + L.z_bytes + 1023u) / 1024u * 1024u;
  L.bslot = static_cast<uint32_t>(2 * LP) * 128u;
  L.off_b = static_cast<uint32_t>(ns) * L.stage;
  L.total = L.off_b + static_cast<uint32_t>(ns) * L.bslot + static_cast<uint32_t>(128 - 2 * LP) * 128u;
  return L;
}

__host__ __device__ constexpr uint32_t tmem_cols_b(int need) {
  return need <= 32 ? 32u : need <= 64 ? 64u : need <= 128 ? 128u : 256u;
}

template <int LP, bool OMEGA, bool TAIL>
__global__ void __cluster_dims__(kScCLb, 1, 1) __launch_bounds__(kScThr, 1)
k_tb_sc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmZ, int64_t m, int n,
        int64_t rpc, int ns, uint64_t seed, uint64_t ctr, DevState* __restrict__ dst, float* __restrict__ cpart,
        float* __restrict__ Y, unsigned* __restrict__ tickets, int l, int use_rp, int passes,
        const float* __restrict__ Qt, float* __restrict__ Qout, double rank_tol) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ __align__(8) uint64_t full[kMaxNSb], bready[kMaxNSb], empty[kMaxNSb], acc_full;
  __shared__ uint32_t tmem_base;
  __shared__ int flag;
  const ScbLayout Lt = scb_layout(LP, n, OMEGA, ns);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * rpc;
  const int64_t r1 = imin64(m, r0 + rpc);
  const int nb = (r1 > r0) ? static_cast<int>((r1 - r0 + kRowsB - 1) / kRowsB) : 0;
  const uint32_t ncols = tmem_cols_b(Lt.N);
  constexpr int kDrainQ = LP / 16;
  const uint64_t stream = OMEGA ? ((ctr == kCounterFromState) ? dst->counter : ctr) : 0ull;
  unsigned char* bring = dsm + Lt.off_b;
  for (uint32_t e = threadIdx.x; e < (Lt.total - Lt.off_b) / 4; e += kScThr) reinterpret_cast<float*>(bring)[e] = 0.f;
  fence_proxy_async();
  if (threadIdx.x == 0) {
    for (int s = 0; s < ns; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&bready[s], 4);
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
        const int y = static_cast<int>(r0 + static_cast<int64_t>(b) * kRowsB);
        mbar_arrive_expect_tx(&full[s], Lt.a_bytes + Lt.z_bytes);
        for (int c = 0; c < Lt.nch; ++c) tma_load_2d(st + c * kBoxB, &tmA, 64 * c, y, &full[s]);
        if (!OMEGA) tma_load_2d(st + Lt.a_bytes, &tmZ, 0, y, &full[s]);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(128, Lt.N, true);
      for (int b = 0; b < nb; ++b) {
        const int s = b % ns, u = b / ns;
        if (ok && (!mbar_wait(&full[s], static_cast<uint32_t>(u) & 1u) ||
                   !mbar_wait(&bready[s], static_cast<uint32_t>(u) & 1u))) {
          ok = false;
          atomicOr(&dst->status, kDevTimeout);
        }
        tc_fence_after();
        const unsigned char* bs = bring + s * Lt.bslot;
        const unsigned char* at = dsm + s * Lt.stage;
#pragma unroll
        for (int ks = 0; ks < kRowsB / 16; ++ks)
          tc_mma_bf16(tbase, smem_desc_sw128(bs + 32 * ks, 16, 1024), smem_desc_sw128(at + ks * 2048, kBoxB, 1024),
                      idesc, b > 0 || ks > 0);
        tc_commit(&empty[s]);
      }
      tc_commit(&acc_full);
    }
  } else {
    // B warps: [B_hi; B_lo]^T of each block (K-major BF16 rows of 64 K-elements)
    const int t = threadIdx.x - 64;
    for (int b = 0; b < nb; ++b) {
      const int s = b % ns, u = b / ns;
      if (ok && !mbar_wait(&full[s], static_cast<uint32_t>(u) & 1u)) {
        ok = false;
        atomicOr(&dst->status, kDevTimeout);
      }
      unsigned char* bs = bring + s * Lt.bslot;
      const int64_t i0 = r0 + static_cast<int64_t>(b) * kRowsB;
      if (OMEGA) {
        for (int q = t; q < kRowsB * (LP / 4); q += 128) {
          const int r = q / (LP / 4), blk = q % (LP / 4);
          float4 gv = make_float4(0.f, 0.f, 0.f, 0.f);
          if (i0 + r < r1) gv = gaussian4(seed, static_cast<uint64_t>(i0 + r), static_cast<uint64_t>(blk), stream, 0ull);
          const float vals[4] = {gv.x, gv.y, gv.z, gv.w};
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int k = 4 * blk + c;
            __nv_bfloat16 hi, lo;
            split_bf16(vals[c], hi, lo);
            *reinterpret_cast<__nv_bfloat16*>(bs + sw128_bf16(stack_row_b(k, 0), r)) = hi;
            *reinterpret_cast<__nv_bfloat16*>(bs + sw128_bf16(stack_row_b(k, 1), r)) = lo;
          }
        }
      } else {
        const float* zt = reinterpret_cast<const float*>(dsm + s * Lt.stage + Lt.a_bytes);   // kRowsB x LP
        for (int q = t; q < kRowsB * LP; q += 128) {
          const int r = q / LP, k = q % LP;
          const float v = (i0 + r < r1) ? zt[r * LP + k] : 0.f;
          __nv_bfloat16 hi, lo;
          split_bf16(v, hi, lo);
          *reinterpret_cast<__nv_bfloat16*>(bs + sw128_bf16(stack_row_b(k, 0), r)) = hi;
          *reinterpret_cast<__nv_bfloat16*>(bs + sw128_bf16(stack_row_b(k, 1), r)) = lo;
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
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  float* part_sm = reinterpret_cast<float*>(dsm);   // n x LP
  // drain: lane quarter q holds the stacked rows 32 q .. 32 q + 31 (hi in lanes < 16, lo above);
  // warps 4 and 5 are the warps >= 2 of quarters 0 and 1
  if (warp >= 4 && (warp & 3) < kDrainQ) {
    const int q = warp & 3;
    for (int grp = 0; grp < Lt.N / 16; ++grp) {
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
  const int nclusters = gridDim.x / kScCLb;
  if (!cluster_split_reduce<float, kScCLb>(part_sm, n * LP, cpart, Y, tickets, blockIdx.x / kScCLb, nclusters, &flag))
    return;
  if (!TAIL) return;
  if (cooperative_groups::this_cluster().block_rank() != 0) return;
  SmallWs<LP> w = carve_small_ws<LP>(dsm, kGaccB);
  int keep = use_rp ? dst->keep : 0;
  keep = max(0, min(keep, l));
  load_basis_block<LP>(w.W, n, keep, l, Qt, Y);
  __syncthreads();
  float rp_res = -1.f;
  const int s = orth_block<LP>(w, n, keep, l, rank_tol, passes, &rp_res, &dst->status);
  for (int e = threadIdx.x; e < n * LP; e += kScThr) Qout[e] = w.W[e];
  if (threadIdx.x == 0) {
    if (use_rp) dst->rp_res = rp_res;
    dst->s = s;
    if (s < l) dst->status |= kDevRankDeficient;
  }
}

// A_b = bf16(A), row-major at ldb (the shadow written once for a stand-alone call)
__global__ void k_to_bf16(const float* __restrict__ A, int64_t lda, int64_t m, int n, __nv_bfloat16* __restrict__ Ab,
                          int64_t ldb) {
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= m * n) return;
  const int64_t i = e / n;
  const int j = static_cast<int>(e - i * n);
  Ab[i * ldb + j] = __float2bfloat16_rn(A[i * lda + j]);
}

template <typename K>
cudaError_t set_limit_b(K kernel, int smem_limit) {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              smem_limit - static_cast<int>(a.sharedSizeBytes));
}

}  // namespace

int tb_lr_stages(int LP, int64_t n, size_t limit) {
  const size_t q = lrb_q_bytes(LP, static_cast<int>(n));
  if (limit <= q) return 0;
  const size_t ns = (limit - q) / kChunkB;
  return ns > static_cast<size_t>(kMaxNSb) ? kMaxNSb : static_cast<int>(ns);
}

size_t tb_lr_smem(int LP, int64_t n, int ns) { return lrb_q_bytes(LP, static_cast<int>(n)) + static_cast<size_t>(ns) * kChunkB; }

int tb_sc_stages(int LP, int64_t n, bool omega, size_t limit) {
  for (int ns = kMaxNSb; ns >= 2; --ns)
    if (scb_layout(LP, static_cast<int>(n), omega, ns).total <= limit) return ns;
  return 0;
}

size_t tb_sc_smem(int LP, int64_t n, bool omega, int ns) {
  const size_t a = scb_layout(LP, static_cast<int>(n), omega, ns).total;
  const size_t ws = LP == 16 ? small_ws_bytes<16>(n, kGaccB) : small_ws_bytes<32>(n, kGaccB);
  const size_t part = static_cast<size_t>(n) * LP * sizeof(float);
  size_t r = a > ws ? a : ws;
  return r > part ? r : part;
}

cudaError_t prepare_tb_kernels(int smem_limit) {
  cudaError_t e = cudaSuccess;
#define PREP(...) \
  if (e == cudaSuccess) e = set_limit_b(__VA_ARGS__, smem_limit);
  PREP(k_tb_lr<16>);
  PREP(k_tb_lr<32>);
  PREP(k_tb_sc<16, true, true>);
  PREP(k_tb_sc<16, false, true>);
  PREP(k_tb_sc<32, true, true>);
  PREP(k_tb_sc<32, false, true>);
#undef PREP
  return e;
}

int tb_sc_resident_grid(int LP, int64_t n, int ns) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kScCLb, 1, 1);
  cfg.blockDim = dim3(kScThr, 1, 1);
  cfg.dynamicSmemBytes = tb_sc_smem(LP, n, false, ns);
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = kScCLb;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  int nc = 0;
  const void* fn = LP == 16 ? reinterpret_cast<const void*>(k_tb_sc<16, false, true>)
                            : reinterpret_cast<const void*>(k_tb_sc<32, false, true>);
  if (cudaOccupancyMaxActiveClusters(&nc, fn, &cfg) != cudaSuccess) nc = 0;
  (void)cudaGetLastError();
  return nc * kScCLb;
}

cudaError_t launch_tb_lr(int LP, const CUtensorMap& tmA, int64_t m, int64_t n, int grid, int ns, const float* Q,
                         float* Z, DevState* dst, cudaStream_t st) {
  int64_t rpc = (m + grid - 1) / grid;
  rpc = (rpc + kBNb - 1) / kBNb * kBNb;
  const size_t smem = tb_lr_smem(LP, n, ns);
  const int nn = static_cast<int>(n);
  if (LP == 16) k_tb_lr<16><<<grid, kLrThr, smem, st>>>(tmA, m, nn, rpc, ns, Q, Z, dst);
  else k_tb_lr<32><<<grid, kLrThr, smem, st>>>(tmA, m, nn, rpc, ns, Q, Z, dst);
  return cudaGetLastError();
}

cudaError_t launch_tb_sc(int LP, const CUtensorMap& tmA, const CUtensorMap* tmZ, int64_t m, int64_t n, int grid,
                         int ns, uint64_t seed, uint64_t ctr, DevState* dst, float* cpart, float* Y,
                         unsigned* tickets, int l, int use_rp, int passes, const float* Qt, float* Q,
                         double rank_tol, cudaStream_t st) {
  int64_t rpc = (m + grid - 1) / grid;
  rpc = (rpc + kRowsB - 1) / kRowsB * kRowsB;
  const bool omega = tmZ == nullptr;
  const size_t smem = tb_sc_smem(LP, n, omega, ns);
  const int nn = static_cast<int>(n);
  const CUtensorMap& z = tmZ ? *tmZ : tmA;
#define ARGS tmA, z, m, nn, rpc, ns, seed, ctr, dst, cpart, Y, tickets, l, use_rp, passes, Qt, Q, rank_tol
  if (LP == 16) {
    if (omega) k_tb_sc<16, true, true><<<grid, kScThr, smem, st>>>(ARGS);
    else k_tb_sc<16, false, true><<<grid, kScThr, smem, st>>>(ARGS);
  } else {
    if (omega) k_tb_sc<32, true, true><<<grid, kScThr, smem, st>>>(ARGS);
    else k_tb_sc<32, false, true><<<grid, kScThr, smem, st>>>(ARGS);
  }
#undef ARGS
  return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float* A, int64_t lda, int64_t m, int64_t n, void* Ab, int64_t ldb, cudaStream_t st) {
  const int64_t total = m * n;
  if (total == 0) return cudaSuccess;
  k_to_bf16<<<static_cast<unsigned>((total + 255) / 256), 256, 0, st>>>(A, lda, m, static_cast<int>(n),
                                                                         static_cast<__nv_bfloat16*>(Ab), ldb);
  return cudaGetLastError();
}

int tb_box_rows_lr() { return kBNb; }
int tb_box_rows_sc() { return kRowsB; }

}  // namespace frsvt
