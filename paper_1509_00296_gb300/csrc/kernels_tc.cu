// Z = A Q on the fifth-generation tensor cores (tcgen05), FP32-accurate.
//
// The row pass of Alg. 1 (Z = A Q for the power step 14 and the projection B^T = A Q of
// step 16) is a contraction over the short side n with a narrow result (LP columns).  On
// CUDA cores every four FMAs need a 16-byte shared-memory read of Q, which makes the pass
// bound by shared-memory bandwidth; the tensor core reads its operands from shared memory
// through its own datapath instead.
//
// Layout: persistent CTAs (one per SM), each owning a contiguous range of rows.  A row block
// of 128 rows is cut into K-chunks of 32 columns (128 bytes), loaded by TMA with the 128-byte
// swizzle that tcgen05 reads as a K-major operand.  FP32 accuracy comes from 3xTF32:
// A Q = A_hi Q_hi + A_hi Q_lo + A_lo Q_hi with X_hi = X truncated to TF32 and X_lo = X - X_hi;
// four "split" warps rewrite each loaded chunk as A_hi in place and A_lo next to it.
// Warp roles: warp 0 issues TMA loads, warp 1 allocates tensor memory and one of its threads
// issues the MMAs (M = 128, N = LP, K = 8 per instruction), warps 2-5 split the chunks and
// drain the accumulators (tcgen05.ld) into Z.  The accumulator is double-buffered in tensor
// memory so the drain of one row block overlaps the MMAs of the next.  Every wait is
// bounded; a timeout sets FRSVT_DEV_TIMEOUT and the kernel still releases its tensor memory.
#include <cuda.h>

#include "common.cuh"
#include "state.cuh"
#include "tc.cuh"
#include "tma.cuh"

namespace frsvt {

namespace {

constexpr int kBM = 128;          // rows per block (MMA M)
constexpr int kBK = 32;           // floats per K-chunk (128 bytes)
constexpr int kNS = 4;            // pipeline stages
constexpr int kTcThreads = 192;   // 6 warps
constexpr uint32_t kChunkBytes = kBM * kBK * 4;   // 16 KB

template <int LP>
__global__ void __launch_bounds__(kTcThreads, 1)
k_tc_lr(const __grid_constant__ CUtensorMap tmA, int64_t m, int n, int64_t rpc, const float* __restrict__ Q,
        float* __restrict__ Z, DevState* __restrict__ dst) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ __align__(8) uint64_t full[kNS], lo_ready[kNS], empty[kNS], acc_full[2], acc_empty[2], fin;
  __shared__ uint32_t tmem_base;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkc = (n + kBK - 1) / kBK;
  const uint32_t bchunk = LP * 128u;                               // one K-chunk of Q^T
  unsigned char* stages = dsm;                                     // kNS x (hi 16 KB | lo 16 KB)
  unsigned char* Bhi = dsm + kNS * 2 * kChunkBytes;
  unsigned char* Blo = Bhi + nkc * bchunk;
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * rpc;
  const int64_t r1 = imin64(m, r0 + rpc);
  const int nb = (r1 > r0) ? static_cast<int>((r1 - r0 + kBM - 1) / kBM) : 0;
  const int total = nb * nkc;

  // Q^T split into TF32 hi / lo, K-major with the 128-byte swizzle: row = output column k.
  for (int e = threadIdx.x; e < nkc * kBK * LP; e += kTcThreads) {
    const int k = e % LP, j = e / LP;                  // j: column of A (K index)
    const float q = (j < n) ? Q[static_cast<int64_t>(j) * LP + k] : 0.f;
    const float h = tf32_hi(q);
    const uint32_t off = static_cast<uint32_t>(j / kBK) * bchunk + sw128_offset(k, j % kBK);
    *reinterpret_cast<float*>(Bhi + off) = h;
    *reinterpret_cast<float*>(Blo + off) = q - h;
  }
  fence_proxy_async();
  if (threadIdx.x == 0) {
    for (int s = 0; s < kNS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&lo_ready[s], 4);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);
    }
    mbar_init(&fin, 1);
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc(&tmem_base, 2 * LP >= 32 ? 2 * LP : 32);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base;
  bool ok = true;

  if (warp == 0) {
    if (lane == 0) {
      prefetch_tensormap(&tmA);
      for (int g = 0; g < total && ok; ++g) {
        const int s = g % kNS, u = g / kNS;
        if (u > 0 && !mbar_wait(&empty[s], static_cast<uint32_t>(u - 1) & 1u)) {
          ok = false;
          atomicOr(&dst->status, kDevTimeout);
          break;
        }
        mbar_arrive_expect_tx(&full[s], kChunkBytes);
        tma_load_2d(stages + s * 2 * kChunkBytes, &tmA, (g % nkc) * kBK,
                    static_cast<int>(r0 + static_cast<int64_t>(g / nkc) * kBM), &full[s]);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_tf32(kBM, LP);
      for (int b = 0; b < nb; ++b) {
        const int buf = b & 1;
        if (b >= 2 && ok && !mbar_wait(&acc_empty[buf], static_cast<uint32_t>(b / 2 - 1) & 1u)) {
          ok = false;
          atomicOr(&dst->status, kDevTimeout);
        }
        tc_fence_after();
        const uint32_t d = tbase + static_cast<uint32_t>(buf * LP);
        for (int c = 0; c < nkc; ++c) {
          const int g = b * nkc + c, s = g % kNS, u = g / kNS;
          if (ok && !mbar_wait(&lo_ready[s], static_cast<uint32_t>(u) & 1u)) {
            ok = false;
            atomicOr(&dst->status, kDevTimeout);
          }
          tc_fence_after();
          const unsigned char* ahi = stages + s * 2 * kChunkBytes;
          const unsigned char* alo = ahi + kChunkBytes;
          const unsigned char* bh = Bhi + c * bchunk;
          const unsigned char* bl = Blo + c * bchunk;
#pragma unroll
          for (int ks = 0; ks < kBK / 8; ++ks) {
            const uint64_t dah = smem_desc_sw128(ahi + 32 * ks, 16, 1024);
            const uint64_t dal = smem_desc_sw128(alo + 32 * ks, 16, 1024);
            const uint64_t dbh = smem_desc_sw128(bh + 32 * ks, 16, 1024);
            const uint64_t dbl = smem_desc_sw128(bl + 32 * ks, 16, 1024);
            tc_mma_tf32(d, dah, dbh, idesc, c > 0 || ks > 0);
            tc_mma_tf32(d, dah, dbl, idesc, true);
            tc_mma_tf32(d, dal, dbh, idesc, true);
          }
          tc_commit(&empty[s]);                 // the stage is free once these MMAs have read it
        }
        tc_commit(&acc_full[buf]);
      }
      tc_commit(&fin);
      if (!mbar_wait(&fin, 0u)) atomicOr(&dst->status, kDevTimeout);
    }
  } else {
    const int t = threadIdx.x - 64;                                // 0..127
    const int sub = warp & 3;                                      // tensor-memory lane quarter
    for (int b = 0; b < nb; ++b) {
      for (int c = 0; c < nkc; ++c) {
        const int g = b * nkc + c, s = g % kNS, u = g / kNS;
        if (ok && !mbar_wait(&full[s], static_cast<uint32_t>(u) & 1u)) {
          ok = false;
          atomicOr(&dst->status, kDevTimeout);
        }
        float4* hi = reinterpret_cast<float4*>(stages + s * 2 * kChunkBytes);
        float4* lo = reinterpret_cast<float4*>(stages + s * 2 * kChunkBytes + kChunkBytes);
#pragma unroll
        for (int i = 0; i < static_cast<int>(kChunkBytes / 16 / 128); ++i) {
          const int e = t + 128 * i;
          const float4 v = hi[e];
          const float4 h = make_float4(tf32_hi(v.x), tf32_hi(v.y), tf32_hi(v.z), tf32_hi(v.w));
          hi[e] = h;
          lo[e] = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
        }
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(&lo_ready[s]);
      }
      const int buf = b & 1;
      if (ok && !mbar_wait(&acc_full[buf], static_cast<uint32_t>(b / 2) & 1u)) {
        ok = false;
        atomicOr(&dst->status, kDevTimeout);
      }
      tc_fence_after();
      const int64_t row = r0 + static_cast<int64_t>(b) * kBM + 32 * sub + lane;
#pragma unroll
      for (int h16 = 0; h16 < LP / 16; ++h16) {
        float v[16];
        tmem_ld16(tbase + (static_cast<uint32_t>(32 * sub) << 16) + static_cast<uint32_t>(buf * LP + 16 * h16), v);
        if (row < r1) {
          float4* zo = reinterpret_cast<float4*>(Z + row * LP + 16 * h16);
#pragma unroll
          for (int k4 = 0; k4 < 4; ++k4) zo[k4] = make_float4(v[4 * k4], v[4 * k4 + 1], v[4 * k4 + 2], v[4 * k4 + 3]);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);
    }
    (void)t;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tbase, 2 * LP >= 32 ? 2 * LP : 32);
}

}  // namespace

size_t tc_lr_smem(int LP, int64_t n) {
  const int nkc = static_cast<int>((n + kBK - 1) / kBK);
  return static_cast<size_t>(kNS) * 2 * kChunkBytes + 2u * nkc * LP * 128u;
}

cudaError_t prepare_tc_kernels(int smem_limit) {
  cudaError_t e = cudaFuncSetAttribute(k_tc_lr<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_limit - 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tc_lr<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_limit - 1024);
  return e;
}

// Z = A Q (A: m x n through tmA with 32-column x 128-row boxes and the 128-byte swizzle).
cudaError_t launch_tc_lr(int LP, const CUtensorMap& tmA, int64_t m, int64_t n, int grid, const float* Q, float* Z,
                         DevState* dst, cudaStream_t st) {
  int64_t rpc = (m + grid - 1) / grid;
  rpc = (rpc + kBM - 1) / kBM * kBM;
  const size_t smem = tc_lr_smem(LP, n);
  const int nn = static_cast<int>(n);
  if (LP == 16) k_tc_lr<16><<<grid, kTcThreads, smem, st>>>(tmA, m, nn, rpc, Q, Z, dst);
  else k_tc_lr<32><<<grid, kTcThreads, smem, st>>>(tmA, m, nn, rpc, Q, Z, dst);
  return cudaGetLastError();
}

int tc_box_cols() { return kBK; }
int tc_box_rows() { return kBM; }

}  // namespace frsvt
