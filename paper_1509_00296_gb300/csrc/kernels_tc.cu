// Z = A Q on the fifth-generation tensor cores (tcgen05), FP32-accurate.
//
// The row pass of Alg. 1 (Z = A Q for the power step 14 and the projection B^T = A Q of
// step 16) is a contraction over the short side n with a narrow result (LP columns).
//
// A kind::tf32 MMA instruction (K = 8) occupies the tensor core for about the same time
// whatever its N (up to 256) and M, so the pass is laid out to make every instruction as wide
// as possible: the MMA computes Z^T for 256 rows at a time,
//     D (128 x 256) += Qs (128 x 8) . A_blk^T (8 x 256 rows),
// with the long side of A in N.  The rows of the M = 128 operand Qs are Q^T split into TF32
// parts and stacked, row 32 (k / 16) + 16 part + k % 16 holding part (hi / lo) of column k of
// Q; the remaining rows of the 128-row window are whatever follows in shared memory (they
// only feed accumulator rows that are never read).  FP32 accuracy by 3xTF32:
// A Q = A_hi [Q_hi Q_lo] + A_lo [Q_hi Q_lo] with X_hi = X truncated to TF32, X_lo = X - X_hi;
// kind::tf32 reads only the 19 leading bits of a 32-bit word, so the raw tile is A_hi and,
// once the A_hi MMAs of a chunk have completed, split warps overwrite it in place with A_lo.
//
// Layout: persistent CTAs (one per SM), each owning a contiguous range of rows.  A block of
// 256 rows is cut into K-chunks of 32 columns (128 bytes), loaded by TMA with the 128-byte
// swizzle (the K-major B operand).  Warp roles: 0 TMA producer; 1 tensor-memory owner and MMA
// issuer (A_hi MMAs of chunk g, then the A_lo MMAs of chunk g - 1); 2-5 drain the
// double-buffered accumulator into Z (the warps of lane quarters 0 / 1 hold the stacked
// rows); 6-13 split.  Warps 2-13 first stage Q^T while the producer already streams A.
// Every wait is bounded; a timeout sets FRSVT_DEV_TIMEOUT and the kernel still releases its
// tensor memory.
#include <cuda.h>

#include "common.cuh"
#include "state.cuh"
#include "tc.cuh"
#include "tma.cuh"

namespace frsvt {

namespace {

constexpr int kBN = 256;          // rows of A per block (MMA N)
constexpr int kBK = 32;           // floats per K-chunk (128 bytes)
constexpr int kMaxNS = 6;
constexpr int kDrainWarps = 4;
constexpr int kSplitWarps = 8;
constexpr int kTcThreads = 64 + 32 * (kDrainWarps + kSplitWarps);
constexpr uint32_t kChunkBytes = kBN * kBK * 4;   // 32 KB

// Stacked row of part (0 hi, 1 lo) of column k in the M operand.
__host__ __device__ constexpr int stack_row(int k, int part) { return 32 * (k / 16) + 16 * part + (k % 16); }

__host__ __device__ inline uint32_t lr_q_bytes(int LP, int n) {
  const int nkc = (n + kBK - 1) / kBK;
  return static_cast<uint32_t>(nkc) * 2u * LP * 128u + static_cast<uint32_t>(128 - 2 * LP) * 128u;
}

template <int LP>
__global__ void __launch_bounds__(kTcThreads, 1)
k_tc_lr(const __grid_constant__ CUtensorMap tmA, int64_t m, int n, int64_t rpc, int ns, const float* __restrict__ Q,
        float* __restrict__ Z, DevState* __restrict__ dst, int normalize) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ __align__(8) uint64_t full[kMaxNS], hidone[kMaxNS], lo_ready[kMaxNS], empty[kMaxNS], acc_full[2],
      acc_empty[2], fin, qready;
  __shared__ uint32_t tmem_base;
  __shared__ float qmax[kDrainWarps + kSplitWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkc = (n + kBK - 1) / kBK;
  const uint32_t qchunk = 2u * LP * 128u;                          // stacked rows of one K-chunk
  const uint32_t qbytes = lr_q_bytes(LP, n);
  unsigned char* Qs = dsm;                                         // qbytes (multiple of 1 KB)
  unsigned char* ring = dsm + qbytes;                              // ns x 32 KB
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * rpc;
  const int64_t r1 = imin64(m, r0 + rpc);
  const int nb = (r1 > r0) ? static_cast<int>((r1 - r0 + kBN - 1) / kBN) : 0;
  const int total = nb * nkc;
  constexpr int kDrainQ = LP / 16;                                 // lane quarters holding stacked rows

  if (threadIdx.x == 0) {
    for (int s = 0; s < ns; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&hidone[s], 1);
      mbar_init(&lo_ready[s], kSplitWarps);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], kDrainQ);
    }
    mbar_init(&fin, 1);
    mbar_init(&qready, kDrainWarps + kSplitWarps);
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc(&tmem_base, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // The producer starts streaming A at once; meanwhile the drain and split warps stage Q^T
  // (hi / lo, stacked) and zero the rest of the M window, then release the MMA issuer.
  if (warp >= 2) {
    const int t = threadIdx.x - 64, nst = kTcThreads - 64;
    const int tail0 = nkc * static_cast<int>(qchunk) / 4;
    for (int e = tail0 + t; e < static_cast<int>(qbytes / 4); e += nst) reinterpret_cast<float*>(Qs)[e] = 0.f;
    constexpr int U = 8;
    const int count = nkc * kBK * LP;
    // normalize: Q is an unnormalised power-step block (A^T A Q, Sec. 2.5); it is staged times the
    // power of two 2^-e that brings its largest entry into [1/2, 1) (the same in every CTA: the max
    // is exact), so repeated steps cannot leave the float range.  Z = A Q 2^-e has the same span.
    float scale = 1.f;
    if (normalize) {
      float mx = 0.f;
      for (int e = t; e < n * LP; e += nst) mx = fmaxf(mx, fabsf(Q[e]));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (lane == 0) qmax[warp - 2] = mx;
      named_bar(1, 32 * (kDrainWarps + kSplitWarps));
      mx = 0.f;
#pragma unroll
      for (int w = 0; w < kDrainWarps + kSplitWarps; ++w) mx = fmaxf(mx, qmax[w]);
      if (mx > 0.f && mx < INFINITY) {
        int ex;
        (void)frexpf(mx, &ex);
        scale = ldexpf(1.f, -ex);
      }
    }
    for (int e0 = t; e0 < count; e0 += U * nst) {
      float q[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * nst;
        const int k = e % LP, j = e / LP;              // j: column of A (K index)
        q[u] = (e < count && j < n) ? Q[static_cast<int64_t>(j) * LP + k] * scale : 0.f;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * nst;
        if (e < count) {
          const int k = e % LP, j = e / LP;
          const float h = tf32_hi(q[u]);
          unsigned char* qc = Qs + static_cast<uint32_t>(j / kBK) * qchunk;
          *reinterpret_cast<float*>(qc + sw128_offset(stack_row(k, 0), j % kBK)) = h;
          *reinterpret_cast<float*>(qc + sw128_offset(stack_row(k, 1), j % kBK)) = q[u] - h;
        }
      }
    }
    fence_proxy_async();
    __syncwarp();
    if (lane == 0) mbar_arrive(&qready);
  }
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
        mbar_arrive_expect_tx(&full[s], kChunkBytes);
        tma_load_2d(ring + s * kChunkBytes, &tmA, (g % nkc) * kBK,
                    static_cast<int>(r0 + static_cast<int64_t>(g / nkc) * kBN), &full[s]);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_tf32(128, kBN);
      if (!mbar_wait(&qready, 0u)) {
        ok = false;
        atomicOr(&dst->status, kDevTimeout);
      }
      // K-steps (8 columns each) that hold columns of A: the last chunk may be partly padding
      auto ksteps = [&](int c) { const int rem = n - c * kBK; return rem >= kBK ? kBK / 8 : (rem + 7) / 8; };
      // A_lo MMAs of chunk g (after the split warps rewrote its stage); closes the block.
      auto issue_lo = [&](int g) {
        const int s = g % ns, u = g / ns, c = g % nkc, b = g / nkc;
        if (ok && !mbar_wait(&lo_ready[s], static_cast<uint32_t>(u) & 1u)) {
          ok = false;
          atomicOr(&dst->status, kDevTimeout);
        }
        tc_fence_after();
        const uint32_t d = tbase + static_cast<uint32_t>((b & 1) * kBN);
        const int nks = ksteps(c);
#pragma unroll
        for (int ks = 0; ks < kBK / 8; ++ks)
          if (ks < nks)
            tc_mma_tf32(d, smem_desc_sw128(Qs + c * qchunk + 32 * ks, 16, 1024),
                        smem_desc_sw128(ring + s * kChunkBytes + 32 * ks, 16, 1024), idesc, true);
        tc_commit(&empty[s]);
        if (c == nkc - 1) tc_commit(&acc_full[b & 1]);
      };
      for (int g = 0; g < total; ++g) {
        const int s = g % ns, u = g / ns, c = g % nkc, b = g / nkc;
        if (c == 0 && b >= 2 && ok &&
            !mbar_wait(&acc_empty[b & 1], static_cast<uint32_t>(b / 2 - 1) & 1u)) {
          ok = false;
          atomicOr(&dst->status, kDevTimeout);
        }
        if (ok && !mbar_wait(&full[s], static_cast<uint32_t>(u) & 1u)) {
          ok = false;
          atomicOr(&dst->status, kDevTimeout);
        }
        tc_fence_after();
        const uint32_t d = tbase + static_cast<uint32_t>((b & 1) * kBN);
        const int nks = ksteps(c);
#pragma unroll
        for (int ks = 0; ks < kBK / 8; ++ks)
          if (ks < nks)
            tc_mma_tf32(d, smem_desc_sw128(Qs + c * qchunk + 32 * ks, 16, 1024),
                        smem_desc_sw128(ring + s * kChunkBytes + 32 * ks, 16, 1024), idesc, c > 0 || ks > 0);
        tc_commit(&hidone[s]);
        if (g > 0) issue_lo(g - 1);
      }
      if (total > 0) issue_lo(total - 1);
      tc_commit(&fin);
      if (!mbar_wait(&fin, 0u)) atomicOr(&dst->status, kDevTimeout);
    }
  } else if (warp < 2 + kDrainWarps) {
    const int sub = warp & 3;                                      // tensor-memory lane quarter
    if (sub < kDrainQ) {
      for (int b = 0; b < nb; ++b) {
        const int buf = b & 1;
        if (ok && !mbar_wait(&acc_full[buf], static_cast<uint32_t>(b / 2) & 1u)) {
          ok = false;
          atomicOr(&dst->status, kDevTimeout);
        }
        tc_fence_after();
        // lane L < 16 holds hi, lane 16 + L lo, of column k = 16 sub + L; TMEM column = row.
        const int k = 16 * sub + (lane & 15);
        const int64_t rb = r0 + static_cast<int64_t>(b) * kBN;
        for (int cg = 0; cg < kBN / 16; ++cg) {
          float v[16];
          tmem_ld16(tbase + (static_cast<uint32_t>(32 * sub) << 16) + static_cast<uint32_t>(buf * kBN + 16 * cg), v);
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
  } else {
    const int t = threadIdx.x - 32 * (2 + kDrainWarps);            // 0 .. 32 kSplitWarps - 1
    for (int g = 0; g < total; ++g) {
      const int s = g % ns, u = g / ns;
      if (ok && !mbar_wait(&hidone[s], static_cast<uint32_t>(u) & 1u)) {
        ok = false;
        atomicOr(&dst->status, kDevTimeout);
      }
      float4* a = reinterpret_cast<float4*>(ring + s * kChunkBytes);
      // 16-byte unit e: row e / 8 of the tile, logical column group (e % 8) ^ (row % 8) (128-byte swizzle)
      const int cvalid = n - (g % nkc) * kBK;
#pragma unroll
      for (int i = 0; i < static_cast<int>(kChunkBytes / 16 / (32 * kSplitWarps)); ++i) {
        const int e = t + 32 * kSplitWarps * i;
        if (4 * ((e & 7) ^ ((e >> 3) & 7)) < cvalid) {
          const float4 v = a[e];
          a[e] = make_float4(v.x - tf32_hi(v.x), v.y - tf32_hi(v.y), v.z - tf32_hi(v.z), v.w - tf32_hi(v.w));
        }
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(&lo_ready[s]);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tbase, 512);
}

}  // namespace

// Stages of the row pass that fit in `limit` bytes of dynamic shared memory.
int tc_lr_stages(int LP, int64_t n, size_t limit) {
  const size_t q = lr_q_bytes(LP, static_cast<int>(n));
  if (limit <= q) return 0;
  const size_t ns = (limit - q) / kChunkBytes;
  return ns > static_cast<size_t>(kMaxNS) ? kMaxNS : static_cast<int>(ns);
}

size_t tc_lr_smem(int LP, int64_t n, int ns) {
  return lr_q_bytes(LP, static_cast<int>(n)) + static_cast<size_t>(ns) * kChunkBytes;
}

cudaError_t prepare_tc_kernels(int smem_limit) {
  cudaError_t e = cudaFuncSetAttribute(k_tc_lr<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_limit - 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tc_lr<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_limit - 1024);
  return e;
}

// Z = A Q (A: m x n through tmA with 32-column x 256-row boxes and the 128-byte swizzle).
cudaError_t launch_tc_lr(int LP, const CUtensorMap& tmA, int64_t m, int64_t n, int grid, int ns, const float* Q,
                         float* Z, DevState* dst, cudaStream_t st, int normalize) {
  int64_t rpc = (m + grid - 1) / grid;
  rpc = (rpc + kBN - 1) / kBN * kBN;
  const size_t smem = tc_lr_smem(LP, n, ns);
  const int nn = static_cast<int>(n);
  if (LP == 16) k_tc_lr<16><<<grid, kTcThreads, smem, st>>>(tmA, m, nn, rpc, ns, Q, Z, dst, normalize);
  else k_tc_lr<32><<<grid, kTcThreads, smem, st>>>(tmA, m, nn, rpc, ns, Q, Z, dst, normalize);
  return cudaGetLastError();
}

int tc_box_cols() { return kBK; }
int tc_box_rows() { return kBN; }

}  // namespace frsvt
