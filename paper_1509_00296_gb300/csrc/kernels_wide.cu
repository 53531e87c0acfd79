// FRSVT (Alg. 1) for a wide oversampled basis (32 < l <= 128) and any short side n: the
// large low-rank recovery shape (8192 x 8192, l = 120).
//
// At this size the basis (n x 128 floats) no longer fits in one CTA, so every step that the
// l <= 32 path runs as a single-CTA tail becomes a grid-wide kernel, and the narrow factor of
// each pass streams from L2 next to the tiles of A:
//
//   k_wd_omega  Omega^T (128 x m) from the Philox stream (steps 4 / 8), split into TF32 hi / lo.
//   k_wd_pass   the passes over A on tcgen05, FP32-accurate (3xTF32), or on a BF16 / FP8 shadow:
//                 row pass    Z^T = Q^T A^T   (steps 14 and 16: Z = A Q = B^T)
//                 column pass Y^T = M^T A     (steps 5 / 9 with M = Omega, step 14 with M = Z)
//               D (128 x 256) accumulates in tensor memory, the M = 128 operand being the
//               basis side (k = 0..127) and N = 256 the long side of the tile; the (tile,
//               K-chunk) units are cut into one contiguous range per SM, each range writing a
//               partial per tile it touches.
//   k_wd_psum   the partials of each tile summed in a fixed order into the pass outputs.
//   k_wd_gram   X^T X (128 x 128) of a basis-side matrix in double-float arithmetic, one partial
//               per SM; k_wd_gsum adds the partials in a fixed order.
//   k_wd_orth   one CTA: Cholesky of the Gram with the rank cut (Cholesky QR, steps 6 / 11 / 14);
//   k_wd_trsm   Q^T = R^{-T} Y^T by forward substitution.
//   k_wd_core   the core (steps 16-19, Eq. 6): Cholesky of B B^T, one-sided Jacobi SVD on an
//               8-CTA cluster, shrinkage, M and the propagated basis factor.
//   k_wd_apply  Out = T^T In for a 128 x 128 T: Rf = Q M, Q~ = Q U.
//   k_wd_alm    X = Z Rf^T on tcgen05 (3xTF32) fused with the iALM sparse shrinkage, dual update
//               and residual (or X written out for a plain SVT).
//
// Layouts: basis-side matrices are kept transposed (128 x len, row stride ld*) so that they are
// K-major MMA operands and coalesced along the long side; Z and Rf are also kept row-major
// (len x 128) for the reconstruction.  Every wait is bounded (FRSVT_DEV_TIMEOUT on expiry).
#include <cooperative_groups.h>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "cluster.cuh"
#include "common.cuh"
#include "state.cuh"
#include "tc.cuh"
#include "tma.cuh"

namespace frsvt {

namespace {

constexpr int kWL = 128;                       // basis width of this path
constexpr int kWN = 256;                       // long-side extent of a pass tile (MMA N)
constexpr int kWK = 32;                        // floats per K-chunk (128 bytes)
constexpr int kWStages = 3;
constexpr int kWSplit = 8;                     // split warps of the pass
constexpr int kWParts = 8;                     // partial planes of the pass workspace
constexpr int kWThr = 64 + 32 * (4 + kWSplit); // 448
constexpr uint32_t kWABytes = kWN * kWK * 4;   // 32 KB
constexpr uint32_t kWMBytes = kWL * kWK * 4;   // 16 KB
constexpr uint32_t kWStage = kWABytes + 2 * kWMBytes;

__device__ __forceinline__ void flag_timeout(bool& ok, DevState* dst) {
  ok = false;
  atomicOr(&dst->status, kDevTimeout);
}

__device__ __forceinline__ float4 f4_lo(float4 v) {
  return make_float4(v.x - tf32_hi(v.x), v.y - tf32_hi(v.y), v.z - tf32_hi(v.z), v.w - tf32_hi(v.w));
}

// kind::f16 MMA with BF16 A and B (FP32 accumulation); instruction descriptor for M x N with
// A K-major and B K-major (b_mn = false) or MN-major (b_mn = true).
__host__ __device__ constexpr uint32_t idesc_bf16w(int M, int N, bool b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((b_mn ? 1u : 0u) << 16) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma_bf16w(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, bool acc) {
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "setp.ne.u32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc ? 1u : 0u)
      : "memory");
}

// BF16 hi / lo parts of a float (hi = bf16(v), lo = bf16(v - hi)).
__device__ __forceinline__ void bf16_split(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(v);
  lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

__device__ __forceinline__ float4 f4_add(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

// ---------------------------------------------------------------- Omega^T
// OT[k][i] = Omega[i][k] for k < p (p = l, or l - keep under range propagation), 0 for k >= p;
// OTl = OT - tf32(OT).  One Philox call gives Omega[i][4 blk .. 4 blk + 3].
__global__ void k_wd_omega(float* __restrict__ OT, float* __restrict__ OTl, __nv_bfloat16* __restrict__ OTb,
                           __nv_bfloat16* __restrict__ OTbl, int64_t ldo, int64_t m, int l, int use_rp, uint64_t seed,
                           uint64_t ctr, const DevState* __restrict__ dst) {
  const uint64_t stream = (ctr == kCounterFromState) ? dst->counter : ctr;
  int p = l;
  if (use_rp) {
    const int keep = max(0, min(dst->keep, l));
    if (keep > 0) p = l - keep;
  }
  const int64_t total = m * (kWL / 4);
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = e % m;
    const int blk = static_cast<int>(e / m);
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
    if (4 * blk < p) g = gaussian4(seed, static_cast<uint64_t>(i), static_cast<uint64_t>(blk), stream, 0ull);
    const float v[4] = {g.x, g.y, g.z, g.w};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int k = 4 * blk + c;
      const float x = (k < p) ? v[c] : 0.f;
      OT[k * ldo + i] = x;
      OTl[k * ldo + i] = x - tf32_hi(x);
      if (OTb != nullptr) bf16_split(x, OTb[k * ldo + i], OTbl[k * ldo + i]);
    }
  }
}

// ---------------------------------------------------------------- range propagation
// Alg. 1 steps 8-11 on the wide basis: the sketch Y^T = Omega_p^T A filled rows 0 .. p - 1
// (p = l - keep, Omega_p the first p columns of the stream's Omega); rows p .. l - 1 take the
// propagated basis Q~^T (rows 0 .. keep - 1 of QtT, keep from the device state).  The span of
// [Y_p, Q~] is that of the paper's [Q~, Y_p orthogonalised against Q~], which the Cholesky QR
// that follows makes orthonormal.
__global__ void k_wd_rp_insert(float* __restrict__ YT, const float* __restrict__ QtT, int64_t ld, int64_t ns, int l,
                               const DevState* __restrict__ dst) {
  const int keep = max(0, min(dst->keep, l));
  if (keep == 0) return;
  const int p = l - keep;
  const int64_t total = static_cast<int64_t>(keep) * ns;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t j = e / ns, x = e % ns;
    YT[(p + j) * ld + x] = QtT[j * ld + x];
  }
}

// Diagonal of T (otherwise the identity) for an unnormalised power step: T_aa = 2^-e with
// ||row a of Y^T|| = f 2^e, f in [1/2, 1) (1 for a zero row), so that k_wd_trsm with T writes
// Q = Y diag(T) exactly (a power-of-two scaling: same span, and no overflow however many
// unnormalised steps follow).  One CTA per row.
__global__ void k_wd_colscale(const float* __restrict__ YT, int64_t ld, int64_t ns, float* __restrict__ T) {
  __shared__ float red[256];
  const int a = blockIdx.x;
  float ss = 0.f;
  for (int64_t x = threadIdx.x; x < ns; x += blockDim.x) {
    const float v = YT[a * ld + x];
    ss = fmaf(v, v, ss);
  }
  red[threadIdx.x] = ss;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const float nrm = sqrtf(red[0]);
    int e = 0;
    if (nrm > 0.f && isfinite(nrm)) frexpf(nrm, &e);
    T[a * kWL + a] = ldexpf(1.f, -e);
  }
}

// T = the identity (the triangular operand of k_wd_trsm for Q = Y, the unnormalised power steps).
__global__ void k_wd_identity(float* __restrict__ T) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kWL * kWL; e += gridDim.x * blockDim.x)
    T[e] = (e / kWL == e % kWL) ? 1.f : 0.f;
}

// ---------------------------------------------------------------- FP8 shadow of A
// One CTA per 128 x 128 tile of A: s = the smallest power of two with max|A_tile| / s <= 448 (the
// E4M3 range), A8 = e4m3(A / s) (round to nearest, saturating), scales[tile] = s.  The tile is
// read once (coalesced float4) and held in registers.
constexpr int kQT = 128;                       // tile side
constexpr int kQThr = 256;

__global__ void __launch_bounds__(kQThr)
k_wd_quant8(const float* __restrict__ A, int64_t lda, int64_t m, int64_t n, uint8_t* __restrict__ A8, int64_t ld8,
            float* __restrict__ scales, int ntc) {
  __shared__ float red[kQThr / 32];
  const int tr = blockIdx.x / ntc, tc = blockIdx.x % ntc;
  const int64_t r0 = static_cast<int64_t>(tr) * kQT;
  const int64_t c0 = static_cast<int64_t>(tc) * kQT;
  const int t = threadIdx.x, c4 = t & 31;
  float4 v[16];
  float amax = 0.f;
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int64_t row = r0 + 8 * i + (t >> 5);
    const int64_t col = c0 + 4 * c4;
    float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
    if (row < m) {
      if (col + 3 < n) {
        x = __ldcs(reinterpret_cast<const float4*>(A + row * lda + col));
      } else {
        if (col < n) x.x = A[row * lda + col];
        if (col + 1 < n) x.y = A[row * lda + col + 1];
        if (col + 2 < n) x.z = A[row * lda + col + 2];
      }
    }
    v[i] = x;
    amax = fmaxf(amax, fmaxf(fmaxf(fabsf(x.x), fabsf(x.y)), fmaxf(fabsf(x.z), fabsf(x.w))));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  if ((t & 31) == 0) red[t >> 5] = amax;
  __syncthreads();
  amax = 0.f;
#pragma unroll
  for (int w = 0; w < kQThr / 32; ++w) amax = fmaxf(amax, red[w]);
  float sc = 1.f;
  if (amax > 0.f && isfinite(amax)) {
    int ex;
    const float f = frexpf(amax / 448.f, &ex);                 // amax / 448 = f 2^ex, f in [0.5, 1)
    sc = ldexpf(1.f, f == 0.5f ? ex - 1 : ex);
  }
  if (t == 0) scales[blockIdx.x] = sc;
  const float inv = 1.f / sc;                                   // exact: sc is a power of two
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int64_t row = r0 + 8 * i + (t >> 5);
    const int64_t col = c0 + 4 * c4;
    if (row >= m || col >= n) continue;
    const float xs[4] = {v[i].x * inv, v[i].y * inv, v[i].z * inv, v[i].w * inv};
    uint8_t b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) b[u] = static_cast<uint8_t>(__nv_cvt_float_to_fp8(xs[u], __NV_SATFINITE, __NV_E4M3));
    if (col + 3 < n) {
      *reinterpret_cast<uint32_t*>(A8 + row * ld8 + col) =
          static_cast<uint32_t>(b[0]) | (static_cast<uint32_t>(b[1]) << 8) | (static_cast<uint32_t>(b[2]) << 16) |
          (static_cast<uint32_t>(b[3]) << 24);
    } else {
      for (int u = 0; u < 4; ++u)
        if (col + u < n) A8[row * ld8 + col + u] = b[u];
    }
  }
}

// Sixteen E4M3 values times a power-of-two scale, as eight packed BF16 pairs (exact: an E4M3
// value times a power of two has at most four significant bits).
__device__ __forceinline__ void fp8x16_to_bf16(const uint4 q, float sc, uint4& lo8, uint4& hi8) {
  const uint32_t w[4] = {q.x, q.y, q.z, q.w};
  uint32_t o[8];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const __nv_fp8x2_storage_t pr = static_cast<__nv_fp8x2_storage_t>((w[i] >> (16 * h)) & 0xFFFFu);
      const __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2(pr, __NV_E4M3);
      const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&hr));
      const __nv_bfloat162 bb = __floats2bfloat162_rn(f.x * sc, f.y * sc);
      o[2 * i + h] = *reinterpret_cast<const uint32_t*>(&bb);
    }
  }
  lo8 = make_uint4(o[0], o[1], o[2], o[3]);
  hi8 = make_uint4(o[4], o[5], o[6], o[7]);
}

// The CTA whose range holds unit x when U units are cut into G contiguous ranges
// [b U / G, (b + 1) U / G): the largest b with floor(b U / G) <= x.
__device__ __forceinline__ int pass_cta_of(int64_t x, int64_t U, int G) {
  return static_cast<int>(((x + 1) * G + U - 1) / U) - 1;
}

// Stores of one float4 of a reduced pass tile (row k, long-side columns x0 + 4 x4 .. + 3): the
// TF32 hi / lo and BF16 hi / lo layouts, and the shared-memory staging of the row-major outputs.
__device__ __forceinline__ void pass_store_out(const float4 v, int k, int x4, int x0, float* __restrict__ outT,
                                               float* __restrict__ outTl, __nv_bfloat16* __restrict__ outTb,
                                               __nv_bfloat16* __restrict__ outTbl, int64_t ldo, float* sm) {
  constexpr int kSt = kWL + 1;
  if (outT != nullptr) reinterpret_cast<float4*>(outT + k * ldo + x0)[x4] = v;
  if (outTl != nullptr) reinterpret_cast<float4*>(outTl + k * ldo + x0)[x4] = f4_lo(v);
  if (outTb != nullptr) {
    __nv_bfloat16 h[4], l[4];
    bf16_split(v.x, h[0], l[0]);
    bf16_split(v.y, h[1], l[1]);
    bf16_split(v.z, h[2], l[2]);
    bf16_split(v.w, h[3], l[3]);
    __nv_bfloat162* hb = reinterpret_cast<__nv_bfloat162*>(outTb + k * ldo + x0 + 4 * x4);
    __nv_bfloat162* lb = reinterpret_cast<__nv_bfloat162*>(outTbl + k * ldo + x0 + 4 * x4);
    hb[0] = __halves2bfloat162(h[0], h[1]);
    hb[1] = __halves2bfloat162(h[2], h[3]);
    lb[0] = __halves2bfloat162(l[0], l[1]);
    lb[1] = __halves2bfloat162(l[2], l[3]);
  }
  if (sm != nullptr) {
    sm[(4 * x4 + 0) * kSt + k] = v.x;
    sm[(4 * x4 + 1) * kSt + k] = v.y;
    sm[(4 * x4 + 2) * kSt + k] = v.z;
    sm[(4 * x4 + 3) * kSt + k] = v.w;
  }
}

// ---------------------------------------------------------------- passes over A
// COL = false (row pass): D[k][i] = sum_j M[k][j] A[i][j] for the 256 rows i of the tile, K = n,
//   A tiles 256 rows x one K-chunk (K-major, 128-byte swizzle).
// COL = true (column pass): D[k][j] = sum_i M[k][i] A[i][j] for the 256 columns j of the tile,
//   K = m, A tiles one K-chunk of rows x 256 columns read MN-major.
// PR = 0 (FP32-accurate): K-chunks of 32 floats; M and M_lo (128 x K, TF32 hi / lo parts of the
//   narrow factor) arrive by TMA with each chunk of A; the MMAs are M_hi A_hi + M_lo A_hi, then
//   (after the split warps rewrote the A tile as A_lo in place) M_hi A_lo: 3xTF32.  The column
//   pass reads A in the 32-byte-atom swizzle (8 boxes of 32 x 32) that kind::tf32 takes MN-major.
// PR = 1 (BF16 shadow of A): K-chunks of 64 BF16; M arrives as BF16 hi / lo parts, so only A's
//   BF16 rounding remains: kind::f16 MMAs M_hi A + M_lo A (the column pass reads A MN-major in
//   the plain 128-byte swizzle, 4 boxes of 64 x 64); no split.
// Work split: the ntiles x nkc (tile, K-chunk) units, tile-major, are cut into G contiguous
// ranges, one per CTA (G CTAs cover the SMs once, G >= ntiles), so a CTA ends one tile and starts
// at most one more: a segment per tile, each with its own TMEM accumulator (columns 0-255 and
// 256-511) and its own partial, slot = its index among the tile's segments.  The last CTA to
// finish a tile sums that tile's partials in slot order (a fixed order) and writes the outputs:
// outT / outTl (128 x ldo, TF32 hi / lo parts), outTb / outTbl (the same as BF16 hi / lo parts),
// outR / outRl (row-major).
// Warps: 0 TMA, 1 tensor memory + MMA, 2-5 drain, 6-13 split (PR = 0).
template <bool COL, int PR>
__global__ void __launch_bounds__(kWThr, 1)
k_wd_pass(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmM,
          const __grid_constant__ CUtensorMap tmMl, int64_t nlong, int64_t nk, int G, float* __restrict__ part,
          int64_t ldp, DevState* __restrict__ dst, const float* __restrict__ scales, int ntr8, int ntc8) {
  constexpr int KC = PR ? 64 : kWK;                         // elements of K per chunk (128-byte rows)
  constexpr int NS = (PR == 2) ? 2 : kWStages;              // pipeline stages
  constexpr uint32_t SB = (PR == 2) ? kWStage + 16384u : kWStage;   // stage bytes (+ the FP8 tile)
  constexpr uint32_t TX = (PR == 2) ? 16384u + 2 * kWMBytes : kWStage;   // bytes the TMA brings per stage
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ __align__(8) uint64_t full[kWStages], hidone[kWStages], lo_ready[kWStages], empty[kWStages], acc_full[2];
  __shared__ uint32_t tmem_base;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nkc = (nk + KC - 1) / KC;
  const int64_t U = ((nlong + kWN - 1) / kWN) * nkc;
  const int64_t u0 = static_cast<int64_t>(blockIdx.x) * U / G;
  const int nc = static_cast<int>(static_cast<int64_t>(blockIdx.x + 1) * U / G - u0);   // units of this CTA
  const int t0 = static_cast<int>(u0 / nkc);                                                // its first tile
  const int nseg = (nc > 0 && (u0 + nc - 1) / nkc > t0) ? 2 : 1;
  const int gsplit = nseg == 2 ? static_cast<int>((t0 + 1) * nkc - u0) : nc;              // first unit of tile t0 + 1
  const uint32_t tcols = nseg == 2 ? 512u : 256u;
  // every block-scope declaration of dsm in this file asks for 1024-byte alignment (one entity);
  // the swizzled TMA destinations need it, so a misplaced base is reported and nothing is issued
  if ((smem_addr(dsm) & 1023u) != 0u) {
    if (threadIdx.x == 0) atomicOr(&dst->status, kDevBadProblem);
    return;
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&hidone[s], 1);
      mbar_init(&lo_ready[s], kWSplit);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&acc_full[0], 1);
    mbar_init(&acc_full[1], 1);
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc(&tmem_base, tcols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base;
  bool ok = true;

  if (warp == 0) {
    if (lane == 0) {
      prefetch_tensormap(&tmA);
      prefetch_tensormap(&tmM);
      prefetch_tensormap(&tmMl);
      for (int g = 0; g < nc && ok; ++g) {
        const int s = g % NS, u = g / NS;
        if (u > 0 && !mbar_wait(&empty[s], static_cast<uint32_t>(u - 1) & 1u)) {
          flag_timeout(ok, dst);
          break;
        }
        unsigned char* st = dsm + s * SB;
        const int tg = t0 + (g >= gsplit ? 1 : 0);
        const int c = static_cast<int>(u0 + g - static_cast<int64_t>(tg) * nkc);
        const int x0 = tg * kWN;
        mbar_arrive_expect_tx(&full[s], TX);
        if (PR == 2) {
          if (COL) tma_load_2d(st + kWABytes + 2 * kWMBytes, &tmA, x0, KC * c, &full[s]);
          else tma_load_2d(st + kWABytes + 2 * kWMBytes, &tmA, KC * c, x0, &full[s]);
        } else if (COL) {
          if (PR) {
#pragma unroll
            for (int v = 0; v < kWN / 64; ++v) tma_load_2d(st + v * 8192, &tmA, x0 + 64 * v, KC * c, &full[s]);
          } else {
#pragma unroll
            for (int v = 0; v < kWN / 32; ++v) tma_load_2d(st + v * 4096, &tmA, x0 + 32 * v, KC * c, &full[s]);
          }
        } else {
          tma_load_2d(st, &tmA, KC * c, x0, &full[s]);
        }
        tma_load_2d(st + kWABytes, &tmM, KC * c, 0, &full[s]);
        tma_load_2d(st + kWABytes + kWMBytes, &tmMl, KC * c, 0, &full[s]);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      if (PR) {
        constexpr uint32_t idesc = idesc_bf16w(128, kWN, COL);
        for (int g = 0; g < nc; ++g) {
          const int s = g % NS, u = g / NS;
          if (ok && !mbar_wait(PR == 2 ? &lo_ready[s] : &full[s], static_cast<uint32_t>(u) & 1u)) flag_timeout(ok, dst);
          tc_fence_after();
          const unsigned char* st = dsm + s * SB;
          const uint32_t dacc = tbase + (g >= gsplit ? 256u : 0u);
          const bool first = g == 0 || g == gsplit;
#pragma unroll
          for (int ks = 0; ks < KC / 16; ++ks) {
            const uint64_t bd = COL ? smem_desc_sw128(st + ks * 2048, 8192, 1024) : smem_desc_sw128(st + 32 * ks, 16, 1024);
            tc_mma_bf16w(dacc, smem_desc_sw128(st + kWABytes + 32 * ks, 16, 1024), bd, idesc, !first || ks > 0);
            tc_mma_bf16w(dacc, smem_desc_sw128(st + kWABytes + kWMBytes + 32 * ks, 16, 1024), bd, idesc, true);
          }
          tc_commit(&empty[s]);
          if (g == gsplit - 1 && nseg == 2) tc_commit(&acc_full[0]);
        }
        tc_commit(&acc_full[nseg - 1]);
      } else {
        constexpr uint32_t idesc = idesc_tf32(128, kWN, false, COL);
        auto bdesc = [&](const unsigned char* a, int ks) -> uint64_t {
          return COL ? smem_desc_sw128a32_mn(a + ks * 1024, 4096) : smem_desc_sw128(a + 32 * ks, 16, 1024);
        };
        auto issue_lo = [&](int g) {
          const int s = g % NS, u = g / NS;
          if (ok && !mbar_wait(&lo_ready[s], static_cast<uint32_t>(u) & 1u)) flag_timeout(ok, dst);
          tc_fence_after();
          const unsigned char* st = dsm + s * SB;
          const uint32_t dacc = tbase + (g >= gsplit ? 256u : 0u);
#pragma unroll
          for (int ks = 0; ks < kWK / 8; ++ks)
            tc_mma_tf32(dacc, smem_desc_sw128(st + kWABytes + 32 * ks, 16, 1024), bdesc(st, ks), idesc, true);
          tc_commit(&empty[s]);
          if (g == gsplit - 1 && nseg == 2) tc_commit(&acc_full[0]);
        };
        for (int g = 0; g < nc; ++g) {
          const int s = g % NS, u = g / NS;
          if (ok && !mbar_wait(&full[s], static_cast<uint32_t>(u) & 1u)) flag_timeout(ok, dst);
          tc_fence_after();
          const unsigned char* st = dsm + s * SB;
          const uint32_t dacc = tbase + (g >= gsplit ? 256u : 0u);
          const bool first = g == 0 || g == gsplit;
#pragma unroll
          for (int ks = 0; ks < kWK / 8; ++ks) {
            tc_mma_tf32(dacc, smem_desc_sw128(st + kWABytes + 32 * ks, 16, 1024), bdesc(st, ks), idesc,
                        !first || ks > 0);
            tc_mma_tf32(dacc, smem_desc_sw128(st + kWABytes + kWMBytes + 32 * ks, 16, 1024), bdesc(st, ks), idesc,
                        true);
          }
          tc_commit(&hidone[s]);
          if (g > 0) issue_lo(g - 1);
        }
        if (nc > 0) issue_lo(nc - 1);
        tc_commit(&acc_full[nseg - 1]);
      }
    }
  } else if (warp < 6) {
    // drain only (below)
  } else if (PR == 2) {
    // FP8 tile (plain rows) -> BF16 tile in the layout the MMA reads, times the tile scales
    const int t = threadIdx.x - 32 * 6;
    for (int g = 0; g < nc; ++g) {
      const int s = g % NS, u = g / NS;
      const int tg = t0 + (g >= gsplit ? 1 : 0);
      const int c = static_cast<int>(u0 + g - static_cast<int64_t>(tg) * nkc);
      const int x0 = tg * kWN;
      if (ok && !mbar_wait(&full[s], static_cast<uint32_t>(u) & 1u)) flag_timeout(ok, dst);
      unsigned char* ab = dsm + s * SB;
      const uint4* a8 = reinterpret_cast<const uint4*>(ab + kWABytes + 2 * kWMBytes);
#pragma unroll 2
      for (int e = t; e < 1024; e += 32 * kWSplit) {
        int rt, ct;
        uint32_t off0, off1;
        if (COL) {                                     // 64 rows x 256 columns; MN-major boxes of 64 columns
          const int r = e >> 4, j0 = (e & 15) * 16, gb = j0 >> 6, jj = j0 & 63;
          rt = (KC * c + r) / kQT;
          ct = (x0 + j0) / kQT;
          off0 = gb * 8192u + r * 128u + ((((jj >> 3)) ^ (r & 7)) << 4);
          off1 = gb * 8192u + r * 128u + ((((jj >> 3) + 1) ^ (r & 7)) << 4);
        } else {                                       // 256 rows x 64 columns, K-major
          const int r = e >> 2, k0 = (e & 3) * 16;
          rt = (x0 + r) / kQT;
          ct = (KC * c) / kQT;
          off0 = r * 128u + ((((k0 >> 3)) ^ (r & 7)) << 4);
          off1 = r * 128u + ((((k0 >> 3) + 1) ^ (r & 7)) << 4);
        }
        const float sc = (rt < ntr8 && ct < ntc8) ? __ldg(scales + rt * ntc8 + ct) : 1.f;
        uint4 lo8, hi8;
        fp8x16_to_bf16(a8[e], sc, lo8, hi8);
        *reinterpret_cast<uint4*>(ab + off0) = lo8;
        *reinterpret_cast<uint4*>(ab + off1) = hi8;
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(&lo_ready[s]);
    }
  } else if (!PR) {
    const int t = threadIdx.x - 32 * 6;
    for (int g = 0; g < nc; ++g) {
      const int s = g % NS, u = g / NS;
      if (ok && !mbar_wait(&hidone[s], static_cast<uint32_t>(u) & 1u)) flag_timeout(ok, dst);
      float4* a = reinterpret_cast<float4*>(dsm + s * SB);
#pragma unroll 4
      for (int e = t; e < static_cast<int>(kWABytes / 16); e += 32 * kWSplit) a[e] = f4_lo(a[e]);
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(&lo_ready[s]);
    }
  }
  if (warp >= 2) {
    // drain by warps 2-13: warp w reads the TMEM lanes of its quarter q = w mod 4 (lane 32 q + L is
    // row k of D, column x its long-side index), column groups i, i + 3, ... with i = (w - 2) / 4;
    // the segment in slot j of tile t goes to part[j][k][t kWN + x].
    const int q = warp & 3, i0 = (warp - 2) >> 2;
    const int k = 32 * q + lane;
    for (int sg = 0; sg < nseg; ++sg) {
      if (!mbar_wait(&acc_full[sg], 0u)) flag_timeout(ok, dst);
      tc_fence_after();
      const int t = t0 + sg;
      const int j = static_cast<int>(blockIdx.x) - pass_cta_of(static_cast<int64_t>(t) * nkc, U, G);
      float* dstp = part + (static_cast<int64_t>(j) * kWL + k) * ldp + static_cast<int64_t>(t) * kWN;
      for (int grp = i0; grp < kWN / 16; grp += 3) {
        float v[16];
        tmem_ld16(tbase + (static_cast<uint32_t>(32 * q) << 16) + static_cast<uint32_t>(256 * sg + 16 * grp), v);
        float4* d4 = reinterpret_cast<float4*>(dstp + 16 * grp);
#pragma unroll
        for (int u = 0; u < 4; ++u)
          d4[u] = (nc > 0 && ok) ? make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3])
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tbase, tcols);
}

// The pass outputs: the partials of each tile summed in slot order (a fixed order).  CTA (t, kb)
// takes rows k = kPsRows kb .. + kPsRows - 1 of tile t, thread (r, c) row r and the float4 columns
// c, c + 16, c + 32, c + 48; the row-major outputs go through a shared-memory transpose.
constexpr int kPsRows = 16;
constexpr int kPsThr = kPsRows * 16;
__global__ void __launch_bounds__(kPsThr)
k_wd_psum(const float* __restrict__ part, int64_t ldp, int64_t nlong, int64_t nkc, int G, float* __restrict__ outT,
          float* __restrict__ outTl, __nv_bfloat16* __restrict__ outTb, __nv_bfloat16* __restrict__ outTbl, int64_t ldo,
          float* __restrict__ outR, float* __restrict__ outRl) {
  __shared__ float sm[kWN * (kPsRows + 1)];
  const int t = blockIdx.x / (kWL / kPsRows), kb = blockIdx.x % (kWL / kPsRows);
  const int64_t U = ((nlong + kWN - 1) / kWN) * nkc;
  const int jf = pass_cta_of(static_cast<int64_t>(t) * nkc, U, G);
  const int nparts = pass_cta_of(static_cast<int64_t>(t + 1) * nkc - 1, U, G) - jf + 1;
  const int x0 = t * kWN;
  const int r = threadIdx.x >> 4, c = threadIdx.x & 15;
  const int k = kb * kPsRows + r;
  float4 v[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) v[j] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 2
  for (int s = 0; s < nparts; ++s) {
    const float4* ps = reinterpret_cast<const float4*>(part + (static_cast<int64_t>(s) * kWL + k) * ldp + x0);
    float4 w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) w[j] = __ldcg(ps + c + 16 * j);
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = f4_add(v[j], w[j]);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int x4 = c + 16 * j;
    pass_store_out(v[j], k, x4, x0, outT, outTl, outTb, outTbl, ldo, nullptr);
    if (outR != nullptr) {
      sm[(4 * x4 + 0) * (kPsRows + 1) + r] = v[j].x;
      sm[(4 * x4 + 1) * (kPsRows + 1) + r] = v[j].y;
      sm[(4 * x4 + 2) * (kPsRows + 1) + r] = v[j].z;
      sm[(4 * x4 + 3) * (kPsRows + 1) + r] = v[j].w;
    }
  }
  if (outR == nullptr) return;
  __syncthreads();
  const int nx = static_cast<int>(imin64(kWN, nlong - x0));
  for (int e = threadIdx.x; e < nx * (kPsRows / 4); e += kPsThr) {
    const int x = e / (kPsRows / 4), k4 = e % (kPsRows / 4);
    const float* rr = sm + x * (kPsRows + 1) + 4 * k4;
    const float4 o = make_float4(rr[0], rr[1], rr[2], rr[3]);
    float4* d = reinterpret_cast<float4*>(outR + (x0 + x) * static_cast<int64_t>(kWL) + kb * kPsRows) + k4;
    *d = o;
    if (outRl != nullptr)
      reinterpret_cast<float4*>(outRl + (x0 + x) * static_cast<int64_t>(kWL) + kb * kPsRows)[k4] = f4_lo(o);
  }
}

// ---------------------------------------------------------------- Gram + small dense tails
// Gram kernel: warps 0-15 own the 496 strictly-upper 4 x 4 blocks (threads 496-511 idle), warp 16
// the 32 diagonal blocks (10 products each), so that every scheduler carries four full warps and
// the first one also the lighter diagonal warp.
constexpr int kGW = 544;
constexpr int kGOff = 496;               // strictly-upper 4 x 4 blocks
constexpr int kGB = 528;                 // 4 x 4 blocks (bi <= bj) of a 128 x 128 symmetric matrix
constexpr int kGCount = kGB * 16;        // packed partial (df64 entries)
constexpr int kGCols = 64;               // long-side columns staged per step
constexpr int kGSt = kWL + 4;            // staging row stride (floats)
constexpr int kGSumE = 64;               // entries per CTA of the partial sum
constexpr int kGSumQ = 8;                // groups of threads per entry, each summing every 8th partial
constexpr int kGSumB = 20;               // partials a thread has in flight
constexpr int kGSumT = kGSumQ * kGSumE;  // threads of a partial-sum CTA
// threads of the one-CTA orthonormalisation tail after a Gram matrix
constexpr int kTW = 512;


// Shared-memory regions of the tails (the Gram staging and partial are dead by then).
constexpr size_t kTG = 0;                                      // df64 G, 128 x 128 (128 KB)
constexpr size_t kTR = kTG + sizeof(df64) * kWL * kWL;         // float 128 x 128 (64 KB)
constexpr size_t kTV = kTR + sizeof(float) * kWL * kWL;        // small vectors
constexpr size_t kTP = kTV + 8 * 1024;                         // Cholesky panels of R (df64)
constexpr size_t kTEnd = kTP + 8 * 1024;                       // two panels of R, 128 x 4 df64 each
constexpr size_t kGSmem = sizeof(float) * kGCols * kGSt + sizeof(df64) * kGCount;     // Gram kernel
constexpr size_t kTSmem = kTEnd;                                                          // tail kernel

__device__ __forceinline__ void block_of(int t, int& bi, int& bj) {
  // row bi of the 32 x 32 block triangle starts at S(bi) = bi (65 - bi) / 2: bi is the largest
  // root bound (65 - sqrt(4225 - 8 t)) / 2, made exact by one integer check each way
  int b = static_cast<int>((65.f - sqrtf(static_cast<float>(4225 - 8 * t))) * 0.5f);
  if (b < 31 && (b + 1) * (64 - b) / 2 <= t) ++b;
  if (b * (65 - b) / 2 > t) --b;
  bi = b;
  bj = b + t - b * (65 - b) / 2;
}

struct TailVec {
  df64* rdiag;     // 128: R_jj
  int* drop;       // 128
  float* thr;      // 128: drop thresholds on the pivots
  float* g0;       // 128: original diagonal
  float* sig;      // 128
  float* coef;     // 128
  int* perm;       // 128
  int* misc;       // 16
};

__device__ TailVec carve_vec(unsigned char* base) {
  TailVec v;
  unsigned char* p = base + kTV;
  v.rdiag = reinterpret_cast<df64*>(p);
  p += sizeof(df64) * kWL;
  v.drop = reinterpret_cast<int*>(p);
  p += sizeof(int) * kWL;
  v.thr = reinterpret_cast<float*>(p);
  p += sizeof(float) * kWL;
  v.g0 = reinterpret_cast<float*>(p);
  p += sizeof(float) * kWL;
  v.sig = reinterpret_cast<float*>(p);
  p += sizeof(float) * kWL;
  v.coef = reinterpret_cast<float*>(p);
  p += sizeof(float) * kWL;
  v.perm = reinterpret_cast<int*>(p);
  p += sizeof(int) * kWL;
  v.misc = reinterpret_cast<int*>(p);
  return v;
}

// Right-looking Cholesky G = R^T R of the leading p x p block of G (double-float, upper triangle,
// in shared memory), with the column drops of the l <= 32 path: column j is dropped (row j of R
// zero, the trailing block untouched) when its pivot is not above rank_tol * G_jj (original), when
// G_jj is below 1e-15 of the largest diagonal, or when it is not a finite positive number.
//
// Blocked by kCB columns, with one panel of look-ahead and the warps split by role:
//   - the factor warp factors the panel's kCB x kCB diagonal block (every lane alike, in
//     registers) and publishes R11 and 1 / R_ii (double-buffered in shared memory);
//   - 384 update threads then form the panel's rows of R right of the block, R12 = R11^{-T} G12
//     (forward substitution, one column per thread), into a double-buffered panel Rp, meet on a
//     barrier of their own, and apply the panel's rank-kCB update to the elements of the upper
//     triangle they own (thread (pair c, group g): columns c and 127 - c, rows g, g + 6,
//     g + 12, ...).  Each first updates its element in the next panel's rows (at most one per
//     column, as the row stride 6 exceeds kCB) and arrives on a named barrier, which lets the
//     factor warp start on the next block while the rest of the trailing update runs.
// The update threads are warps 0-11 and the factor warp is warp 15 (warps 12-14 idle): measured
// on GB300, this layout lets the serial chain of the diagonal blocks wait least for issue behind
// the update warps, which always have independent work (75 us against 81 us for a 120 x 120
// Gram with the factor warp at warp 3 and the update warps on the other three schedulers).
// Rp[(panel & 1)][b][k] holds row k of the panel's rows of R at column b.  Every wait is a
// hardware barrier whose arrival counts are fixed by p alone: per panel one "block ready" phase
// (factor warp arrives, update threads wait), one "panel ready" phase (update threads only) and,
// except after the last panel, one "next rows ready" phase (update threads arrive, factor warp
// waits).
// R (FP32, row-major, upper, dropped rows zero) goes to Rout; v.rdiag / v.drop get the diagonal
// and the flags.  A non-finite diagonal of G (NaN or Inf met in the Gram reduction) ORs
// FRSVT_DEV_NONFINITE into *status.  Needs blockDim.x = 512.
constexpr int kCB = 4;                   // panel width of the Cholesky
constexpr int kChG = 6;                  // row groups of the update threads (row stride > kCB)
constexpr int kChU = 64 * kChG;          // update threads: 64 column pairs x 6 row groups (12 warps)
constexpr int kChFactorWarp = 15;
constexpr int kChBar = kChU + 32;        // threads on the barriers between the factor warp and the update threads
constexpr int kBarRowsReady = 1;         // named barrier ids (0 is __syncthreads)
constexpr int kBarBlockReady = 2;
constexpr int kBarPanelReady = 3;
static_assert(kChG > kCB, "one element per column and thread in the look-ahead rows");

__device__ __forceinline__ void named_bar_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void named_bar_arrive(int id, int n) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// g - sum_k x_k y_k in double-float: each product split exactly with FMAs (the cross terms of the
// low parts folded into its error), its high part taken off g by two-sum, every low-order term
// gathered in one float and the pair renormalised at the end.
__device__ __forceinline__ df64 df_sub_dot(df64 g, const df64* x, const df64* y) {
  float hi = g.hi, lo = g.lo;
#pragma unroll
  for (int k = 0; k < kCB; ++k) {
    const float pr = __fmul_rn(x[k].hi, y[k].hi);
    float e = __fmaf_rn(x[k].hi, y[k].hi, -pr);
    e = __fmaf_rn(x[k].hi, y[k].lo, e);
    e = __fmaf_rn(x[k].lo, y[k].hi, e);
    const float s = __fsub_rn(hi, pr);
    const float bb = __fsub_rn(s, hi);
    const float err = __fsub_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fadd_rn(pr, bb));
    hi = s;
    lo = __fadd_rn(lo, __fsub_rn(err, e));
  }
  return df_quick(hi, lo);
}

__device__ __forceinline__ void load_panel_col(const df64* Rpb, int b, df64* x) {
  const float4 u0 = *reinterpret_cast<const float4*>(Rpb + b * kCB);
  const float4 u1 = *reinterpret_cast<const float4*>(Rpb + b * kCB + 2);
  x[0] = df64{u0.x, u0.y};
  x[1] = df64{u0.z, u0.w};
  x[2] = df64{u1.x, u1.y};
  x[3] = df64{u1.z, u1.w};
}

// The update of column `col` (rows a0, a0 + kChG, ... <= col), two elements per step.
__device__ __forceinline__ void chol_update_col(df64* G, const df64* Rpb, int col, int a0, const df64* y) {
  int a = a0;
  for (; a + kChG <= col; a += 2 * kChG) {
    df64 x0[kCB], x1[kCB];
    load_panel_col(Rpb, a, x0);
    load_panel_col(Rpb, a + kChG, x1);
    const df64 g0 = G[a * kWL + col], g1 = G[(a + kChG) * kWL + col];
    G[a * kWL + col] = df_sub_dot(g0, x0, y);
    G[(a + kChG) * kWL + col] = df_sub_dot(g1, x1, y);
  }
  if (a <= col) {
    df64 x0[kCB];
    load_panel_col(Rpb, a, x0);
    G[a * kWL + col] = df_sub_dot(G[a * kWL + col], x0, y);
  }
}

__device__ void wide_cholesky(df64* G, const TailVec& v, float* Rout, int p, double rank_tol, uint32_t* status,
                              df64* Rp) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < kWL * kWL; e += blockDim.x) Rout[e] = 0.f;
  if (tid < kWL) {
    const float g0 = tid < p ? G[tid * kWL + tid].hi : 0.f;
    v.g0[tid] = g0;
    v.thr[tid] = static_cast<float>(rank_tol * static_cast<double>(g0));
    v.drop[tid] = 1;
    v.rdiag[tid] = df64{0.f, 0.f};
    if (tid < p && !isfinite(g0)) atomicOr(status, kDevNonfinite);
  }
  __shared__ df64 sBlk[2][kCB * kCB + kCB];         // the panel's diagonal block of R and 1 / R_ii
  __shared__ int sDrop[2][kCB];
  __syncthreads();
  if (warp == kChFactorWarp) {                       // ---- the factor warp
    float maxdiag = 0.f;
    for (int a = lane; a < p; a += 32) maxdiag = fmaxf(maxdiag, v.g0[a]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) maxdiag = fmaxf(maxdiag, __shfl_xor_sync(0xffffffffu, maxdiag, o));
    for (int j0 = 0, jp = 0; j0 < p; j0 += kCB, ++jp) {
      if (jp > 0) named_bar_sync(kBarRowsReady, kChBar);   // rows j0 .. j0 + kCB - 1 are final
      const int j1 = min(p, j0 + kCB);
      const int nk = j1 - j0;
      df64 g[kCB * kCB], r[kCB * kCB], inv[kCB];
      int dr[kCB];
      // few shared-memory instructions (the update warps keep the shared-memory pipe busy): the
      // block's rows as 32-byte vectors, the thresholds as one float4 each
#pragma unroll
      for (int i = 0; i < kCB; ++i) {
        const float4* row = reinterpret_cast<const float4*>(G + (j0 + min(i, nk - 1)) * kWL + j0);
        const float4 u0 = row[0], u1 = row[1];
        const df64 e[4] = {df64{u0.x, u0.y}, df64{u0.z, u0.w}, df64{u1.x, u1.y}, df64{u1.z, u1.w}};
#pragma unroll
        for (int c = 0; c < kCB; ++c) {
          g[i * kCB + c] = (i <= c && c < nk) ? e[c] : df64{0.f, 0.f};
          r[i * kCB + c] = df64{0.f, 0.f};
        }
      }
      const float4 thr4 = *reinterpret_cast<const float4*>(v.thr + j0);
      const float4 gd4 = *reinterpret_cast<const float4*>(v.g0 + j0);
      const float thr[kCB] = {thr4.x, thr4.y, thr4.z, thr4.w};
      const float gd[kCB] = {gd4.x, gd4.y, gd4.z, gd4.w};
#pragma unroll
      for (int i = 0; i < kCB; ++i) {
        const df64 d = g[i * kCB + i];
        const bool drop = i >= nk || !(d.hi > thr[i]) || !(gd[i] > 1e-15f * maxdiag) || !(d.hi > 1e-30f) ||
                          !(d.hi < 1e30f);
        dr[i] = drop ? 1 : 0;
        inv[i] = drop ? df64{0.f, 0.f} : df_rsqrt_fma(d);
        if (!drop) {
#pragma unroll
          for (int c = i + 1; c < kCB; ++c) r[i * kCB + c] = df_mul(g[i * kCB + c], inv[i]);
#pragma unroll
          for (int a = i + 1; a < kCB; ++a)              // the next pivot's entry first
#pragma unroll
            for (int c = a; c < kCB; ++c) g[a * kCB + c] = df_fms(g[a * kCB + c], r[i * kCB + a], r[i * kCB + c]);
          r[i * kCB + i] = df_mul(d, inv[i]);
        }
      }
      {                                              // one store instruction per output, lane u storing entry u
        df64 ru = r[0];
        int du = dr[0];
#pragma unroll
        for (int u = 1; u < kCB * kCB; ++u)
          if (lane == u) ru = r[u];
#pragma unroll
        for (int i = 0; i < kCB; ++i)
          if (lane == kCB * kCB + i) ru = inv[i];
#pragma unroll
        for (int i = 1; i < kCB; ++i)
          if (lane == i) du = dr[i];
        if (lane < kCB * kCB + kCB) sBlk[jp & 1][lane] = ru;     // R11 (row-major), then 1 / R_ii
        const int i = lane / kCB, c = lane % kCB;
        if (lane < kCB * kCB && i <= c && c < nk) Rout[(j0 + i) * kWL + j0 + c] = ru.hi;
        if (lane < kCB) {
          sDrop[jp & 1][lane] = du;
          if (lane < nk) v.drop[j0 + lane] = du;
        }
        df64 dg = r[0];
#pragma unroll
        for (int k = 1; k < kCB; ++k)
          if (lane == k) dg = r[k * kCB + k];
        if (lane < nk) v.rdiag[j0 + lane] = dg;
      }
      __syncwarp();
      named_bar_arrive(kBarBlockReady, kChBar);
    }
  } else if (warp < kChU / 32) {                     // ---- the update threads
    const int ut = tid;
    const int pc = ut & 63, grp = ut >> 6;
    const int colA = pc, colB = kWL - 1 - pc;
    for (int j0 = 0, jp = 0; j0 < p; j0 += kCB, ++jp) {
      named_bar_sync(kBarBlockReady, kChBar);
      const int j1 = j0 + kCB;                       // rows >= j1 take this panel's update
      df64* Rpb = Rp + (jp & 1) * (kWL * kCB);
      {                                              // rows j0 .. j0 + 3 of R at column b = j1 + ut
        const int b = j1 + ut;
        if (b < p) {
          const df64* blk = sBlk[jp & 1];
          const int nk = min(kCB, p - j0);
          df64 x[kCB];
#pragma unroll
          for (int i = 0; i < kCB; ++i) x[i] = i < nk ? G[(j0 + i) * kWL + b] : df64{0.f, 0.f};
#pragma unroll
          for (int i = 0; i < kCB; ++i) {
#pragma unroll
            for (int k = 0; k < i; ++k) x[i] = df_fms(x[i], blk[k * kCB + i], x[k]);
            x[i] = sDrop[jp & 1][i] ? df64{0.f, 0.f} : df_mul(x[i], blk[kCB * kCB + i]);   // dropped: 0, NaN or not
          }
          *reinterpret_cast<float4*>(Rpb + b * kCB) = make_float4(x[0].hi, x[0].lo, x[1].hi, x[1].lo);
          *reinterpret_cast<float4*>(Rpb + b * kCB + 2) = make_float4(x[2].hi, x[2].lo, x[3].hi, x[3].lo);
#pragma unroll
          for (int i = 0; i < kCB; ++i)
            if (i < nk) Rout[(j0 + i) * kWL + b] = x[i].hi;
        }
      }
      named_bar_sync(kBarPanelReady, kChU);          // the panel's rows of R are in Rp
      const int a0 = j1 <= grp ? grp : grp + (j1 - grp + kChG - 1) / kChG * kChG;   // first row >= j1
      const bool onA = colA < p && a0 <= colA, onB = colB < p && a0 <= colB;
      df64 yA[kCB], yB[kCB];
      if (onA) load_panel_col(Rpb, colA, yA);
      if (onB) load_panel_col(Rpb, colB, yB);
      const bool look = a0 < j1 + kCB;               // a0 lies in the next panel's rows
      if (look && (onA || onB)) {                    // (a0 <= a column < p: inside the panel)
        df64 x[kCB];
        load_panel_col(Rpb, a0, x);
        if (onA) G[a0 * kWL + colA] = df_sub_dot(G[a0 * kWL + colA], x, yA);
        if (onB) G[a0 * kWL + colB] = df_sub_dot(G[a0 * kWL + colB], x, yB);
      }
      if (j1 < p) {
        __syncwarp();
        named_bar_arrive(kBarRowsReady, kChBar);
      }
      const int a1 = look ? a0 + kChG : a0;
      if (onA) chol_update_col(G, Rpb, colA, a1, yA);
      if (onB) chol_update_col(G, Rpb, colB, a1, yB);
    }
  }
  __syncthreads();
}

// The packed Gram (4 x 4 blocks, bi <= bj) unpacked into G (128 x 128 df64, upper blocks): two
// entries of a block row per 16-byte load, all of a thread's loads issued before any store.
template <int NT>
__device__ __forceinline__ void unpack_gram(const double* __restrict__ Gpk, df64* G) {
  constexpr int kPairs = kGCount / 2;
  constexpr int kPer = (kPairs + NT - 1) / NT;
  float4 w[kPer];
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int e2 = static_cast<int>(threadIdx.x) + j * NT;
    w[j] = e2 < kPairs ? __ldcg(reinterpret_cast<const float4*>(Gpk) + e2) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int e2 = static_cast<int>(threadIdx.x) + j * NT;
    if (e2 < kPairs) {
      const int t = e2 >> 3, u = (2 * e2) & 15;
      int bi, bj;
      block_of(t, bi, bj);
      *reinterpret_cast<float4*>(G + (4 * bi + (u >> 2)) * kWL + 4 * bj + (u & 3)) = w[j];
    }
  }
}

struct CoreArgs {
  int l;
  float tau_host;
  int tau_from_mu;
  int update_rp;
  int advance_counter;
  int max_sweeps;
};

// Packed index of the 4 x 4 block (bi, bj), bi <= bj, in row-major order of the upper triangle.
__device__ __forceinline__ int block_slot(int bi, int bj) { return 32 * bi - bi * (bi - 1) / 2 + (bj - bi); }

// X^T X (128 x 128, packed 4 x 4 blocks of the upper triangle) of a basis-side matrix in
// double-float arithmetic over this CTA's range of long-side columns, written as the CTA's
// partial: cpart[blockIdx.x][kGCount] (df64 pairs, float hi then float lo, where a double is
// declared).  k_wd_gsum adds the partials.
__global__ void __launch_bounds__(kGW, 1)
k_wd_gram(const float* __restrict__ XT, int64_t ldx, int64_t len, int64_t per_cta, double* __restrict__ cpart,
          int p) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  float* stg = reinterpret_cast<float*>(dsm);                                          // kGCols x kGSt
  df64* part_sm = reinterpret_cast<df64*>(dsm + sizeof(float) * kGCols * kGSt);       // kGCount
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool diag = warp == kGOff / 32 + 1;          // warp 16
  int bi = 0, bj = 0;
  if (diag) {
    bi = bj = lane;
  } else if (tid < kGOff) {                          // strictly-upper block number tid
    int rem = tid;
    while (rem >= 31 - bi) {
      rem -= 31 - bi;
      ++bi;
    }
    bj = bi + 1 + rem;
  }
  const bool on = diag || tid < kGOff;
  df64 acc[16];
#pragma unroll
  for (int u = 0; u < 16; ++u) acc[u] = df64{0.f, 0.f};
  const int64_t x0 = static_cast<int64_t>(blockIdx.x) * per_cta;
  const int64_t x1 = imin64(len, x0 + per_cta);
  for (int64_t xs = x0; xs < x1; xs += kGCols) {
    const int nxc = static_cast<int>(imin64(kGCols, x1 - xs));
#pragma unroll 4                                     // four loads in flight per thread
    for (int e = tid; e < kWL * kGCols; e += kGW) {
      const int a = e / kGCols, x = e % kGCols;
      stg[x * kGSt + a] = (x < nxc && a < p) ? __ldcg(XT + a * ldx + xs + x) : 0.f;
    }
    __syncthreads();
    if (diag) {                                      // the upper triangle of a diagonal block
      for (int x = 0; x < nxc; ++x) {
        const float4 ua = *reinterpret_cast<const float4*>(stg + x * kGSt + 4 * bi);
        const float va[4] = {ua.x, ua.y, ua.z, ua.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = i; j < 4; ++j) df64_add_prod(acc[4 * i + j], va[i], va[j]);
      }
    } else if (on) {
      for (int x = 0; x < nxc; ++x) {
        const float4 ua = *reinterpret_cast<const float4*>(stg + x * kGSt + 4 * bi);
        const float4 ub = *reinterpret_cast<const float4*>(stg + x * kGSt + 4 * bj);
        const float va[4] = {ua.x, ua.y, ua.z, ua.w};
        const float vb[4] = {ub.x, ub.y, ub.z, ub.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) df64_add_prod(acc[4 * i + j], va[i], vb[j]);
      }
    }
    __syncthreads();
  }
  if (on) {
    const int slot = block_slot(bi, bj);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const df64 a = (diag && i > j) ? acc[4 * j + i] : acc[4 * i + j];   // the lower half mirrored
        part_sm[slot * 16 + 4 * i + j] = df_quick(a.hi, a.lo);
      }
  }
  __syncthreads();
  float4* dst = reinterpret_cast<float4*>(cpart + static_cast<int64_t>(blockIdx.x) * kGCount);
  const float4* src = reinterpret_cast<const float4*>(part_sm);
  for (int e = tid; e < kGCount / 2; e += kGW) __stcg(dst + e, src[e]);
}

// Gpk = the sum of the nparts partials, entry by entry in a fixed order: each CTA takes kGSumE
// entries; group q of its threads sums partials q, q + kGSumQ, q + 2 kGSumQ, ... (kGSumB loads in
// flight, one batch for 152 partials; pairwise within a batch), then the group sums are added in
// group order.
__global__ void __launch_bounds__(kGSumT)
k_wd_gsum(const double* __restrict__ cpart, int nparts, double* __restrict__ Gpk) {
  __shared__ df64 red[kGSumQ][kGSumE];
  const int t = threadIdx.x, el = t % kGSumE, q = t / kGSumE;
  const int e = blockIdx.x * kGSumE + el;
  const float2* cp = reinterpret_cast<const float2*>(cpart);
  df64 sum{0.f, 0.f};
  if (e < kGCount) {
    for (int k0 = q; k0 < nparts; k0 += kGSumQ * kGSumB) {
      df64 v[kGSumB];
#pragma unroll
      for (int u = 0; u < kGSumB; ++u) {
        const int k = k0 + kGSumQ * u;
        const float2 w = k < nparts ? __ldcg(cp + static_cast<int64_t>(k) * kGCount + e) : make_float2(0.f, 0.f);
        v[u] = df64{w.x, w.y};
      }
#pragma unroll
      for (int h = 1; h < kGSumB; h *= 2)
#pragma unroll
        for (int u = 0; u + h < kGSumB; u += 2 * h) v[u] = df_add(v[u], v[u + h]);
      sum = df_add(sum, v[0]);
    }
  }
  red[q][el] = sum;
  __syncthreads();
  if (q == 0 && e < kGCount) {
    df64 g = red[0][el];
#pragma unroll
    for (int r = 1; r < kGSumQ; ++r) g = df_add(g, red[r][el]);
    reinterpret_cast<float2*>(Gpk)[e] = make_float2(g.hi, g.lo);
  }
}

// The orthonormalisation tail after the Gram of Y (one CTA of kTW threads; Alg. 1 steps 6 / 11 /
// 14): Cholesky of Gpk with the rank cut, T1 = R with 1 / R_cc on the diagonal (0 for dropped
// columns: the operand of the forward substitution Q^T = R^{-T} Y^T in k_wd_trsm), the basis size s.
__global__ void __launch_bounds__(kTW, 1)
k_wd_orth(const double* __restrict__ Gpk, int p, double rank_tol, float* __restrict__ T1, DevState* __restrict__ dst) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  const int tid = threadIdx.x, nt = blockDim.x;
  df64* G = reinterpret_cast<df64*>(dsm + kTG);                 // 128 x 128 (upper triangle used)
  float* R = reinterpret_cast<float*>(dsm + kTR);               // R (FP32, upper)
  const TailVec v = carve_vec(dsm);
  unpack_gram<kTW>(Gpk, G);
  __syncthreads();
  wide_cholesky(G, v, R, p, rank_tol, &dst->status, reinterpret_cast<df64*>(dsm + kTP));
  for (int e = tid; e < kWL * kWL; e += nt) {
    const int a = e / kWL, c = e % kWL;
    float x = R[e];
    if (a == c) x = (c < p && !v.drop[c] && x != 0.f) ? 1.f / x : 0.f;
    T1[e] = x;
  }
  if (tid == 0) {
    int s = 0;
    for (int j = 0; j < p; ++j) s += v.drop[j] ? 0 : 1;
    dst->s = s;
    if (s < p) dst->status |= kDevRankDeficient;
  }
}

// ---------------------------------------------------------------- core on a cluster
// The l x l core (Alg. 1 steps 16-19) with its one-sided Jacobi spread over a cluster of kJC CTAs.
// The 128 columns of R^T are 16 blocks of 8; CTA c holds two blocks (its top and bot slot) in
// shared memory.  A sweep is 15 outer rounds of the block round-robin: in every outer round each
// CTA rotates all 64 pairs between its two blocks (8 inner rounds of 8 disjoint pairs, a_i with
// b_{(i + r) mod 8}), in the first one also the 28 pairs inside each block (7 inner rounds of the
// round-robin of 8); then the blocks move one place round the ring of the 15 slots other than
// CTA 0's top (bot_0 -> top_1 -> ... -> top_7 -> bot_7 -> ... -> bot_1 -> bot_0), written straight
// into the receiving CTA's other buffer through distributed shared memory, one cluster barrier per
// outer round.  Every pair meets once per sweep and the blocks are back in place after it.  Only
// the inner rounds touch the columns often, and they stay inside one SM's shared memory.
constexpr int kJC = 8;                   // CTAs of the core cluster
constexpr int kJB = 8;                   // columns per block
constexpr int kJP = 16;                  // threads per pair in an inner round
constexpr int kJW = kJB * kJP;           // worker threads of a CTA (8 pairs per inner round)
constexpr int kCW = 512;                 // threads of a core CTA
constexpr size_t kTJ = kTG;              // two working buffers of 16 columns (over the dead G)

// Pair (p, q) of the 8 columns of a block in round r of the round-robin of 8 (slot w < 4).
__device__ __forceinline__ void rr8(int r, int w, int& p, int& q) {
  if (w == 0) {
    p = kJB - 1;
    q = r;
  } else {
    p = r + w;
    if (p >= kJB - 1) p -= kJB - 1;
    q = r - w;
    if (q < 0) q += kJB - 1;
  }
}

// Rotate local columns p and q of X (16 columns of kWL floats) if they are not orthogonal to
// tol; kJP threads (sub 0 .. kJP - 1) share the pair.  Returns whether it rotated.
__device__ __forceinline__ int jacobi_pair(float* X, int p, int q, int sub, float tol) {
  constexpr int E = kWL / kJP;
  float4* xp = reinterpret_cast<float4*>(X + p * kWL);
  float4* xq = reinterpret_cast<float4*>(X + q * kWL);
  float4 a[E / 4], b[E / 4];
#pragma unroll
  for (int jj = 0; jj < E / 4; ++jj) {
    a[jj] = xp[sub + kJP * jj];
    b[jj] = xq[sub + kJP * jj];
  }
  float al = 0.f, be = 0.f, ga = 0.f, al2 = 0.f, be2 = 0.f, ga2 = 0.f;
#pragma unroll
  for (int jj = 0; jj < E / 4; ++jj) {
    al = fmaf(a[jj].x, a[jj].x, al); al2 = fmaf(a[jj].y, a[jj].y, al2);
    al = fmaf(a[jj].z, a[jj].z, al); al2 = fmaf(a[jj].w, a[jj].w, al2);
    be = fmaf(b[jj].x, b[jj].x, be); be2 = fmaf(b[jj].y, b[jj].y, be2);
    be = fmaf(b[jj].z, b[jj].z, be); be2 = fmaf(b[jj].w, b[jj].w, be2);
    ga = fmaf(a[jj].x, b[jj].x, ga); ga2 = fmaf(a[jj].y, b[jj].y, ga2);
    ga = fmaf(a[jj].z, b[jj].z, ga); ga2 = fmaf(a[jj].w, b[jj].w, ga2);
  }
  al += al2;
  be += be2;
  ga += ga2;
#pragma unroll
  for (int o = 1; o < kJP; o <<= 1) {
    al += __shfl_xor_sync(0xffffffffu, al, o);
    be += __shfl_xor_sync(0xffffffffu, be, o);
    ga += __shfl_xor_sync(0xffffffffu, ga, o);
  }
  if (!(al > 1e-30f && be > 1e-30f && fabsf(ga) * rsqrtf(al) * rsqrtf(be) > tol)) return 0;
  const float zeta = __fdividef(be - al, 2.f * ga);
  const float az = fabsf(zeta);
  const float w2 = fmaf(zeta, zeta, 1.f);
  const float t = az < 1e15f ? copysignf(__fdividef(1.f, az + w2 * rsqrtf(w2)), zeta) : __fdividef(0.5f, zeta);
  const float c = rsqrtf(fmaf(t, t, 1.f));
  const float sn = c * t;
#pragma unroll
  for (int jj = 0; jj < E / 4; ++jj) {
    const float4 x = a[jj], y = b[jj];
    xp[sub + kJP * jj] = make_float4(c * x.x - sn * y.x, c * x.y - sn * y.y, c * x.z - sn * y.z, c * x.w - sn * y.w);
    xq[sub + kJP * jj] = make_float4(sn * x.x + c * y.x, sn * x.y + c * y.y, sn * x.z + c * y.z, sn * x.w + c * y.w);
  }
  return 1;
}

// Cluster Jacobi on the rows of R (rank 0's R, 128 x kWL; rows >= the live count are zero):
// scattered to the CTAs, rotated, gathered back into rank 0's R.  All threads of every CTA call
// it, rank 0 once its R is complete (the first cluster barrier waits for that).  Every CTA passes
// the same sequence of cluster barriers: the sweep loop ends on a decision all CTAs take from the
// same eight flags.  Returns the sweeps taken (the same in every CTA).
__device__ int cluster_jacobi(float* R0, int max_sweeps, float tol, float* buf, int* rotflag) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = static_cast<int>(cl.block_rank());
  const int tid = threadIdx.x;
  constexpr int COLS = 2 * kJB;                     // local columns: top block 0..7, bot block 8..15
  constexpr int BUF = COLS * kWL;                   // floats per working buffer
  cl.sync();                                        // rank 0's R is complete
  // scatter: this CTA's blocks 2 rank (top) and 2 rank + 1 (bot) = rows 16 rank .. 16 rank + 15
  {
    const float4* src = reinterpret_cast<const float4*>(cl.map_shared_rank(R0, 0) + rank * COLS * kWL);
    for (int e = tid; e < BUF / 4; e += blockDim.x) reinterpret_cast<float4*>(buf)[e] = src[e];
  }
  if (tid < 2 * kJC) rotflag[tid] = 0;
  cl.sync();                                        // R0 read by everyone; flags cleared everywhere
  int wb = 0, sweeps = 0;
  const int pair = tid / kJP, sub = tid % kJP;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    int rotated = 0;
    for (int R = 0; R < 2 * kJC - 1; ++R) {
      float* X = buf + wb * BUF;
      if (tid < kJW) {
        if (R == 0)
          for (int r = 0; r < kJB - 1; ++r) {       // pairs inside each block
            int p, q;
            rr8(r, pair & 3, p, q);
            const int off = (pair >> 2) * kJB;
            rotated |= jacobi_pair(X, off + p, off + q, sub, tol);
            named_bar(1, kJW);
          }
        for (int r = 0; r < kJB; ++r) {             // pairs across the two blocks
          rotated |= jacobi_pair(X, pair, kJB + ((pair + r) & (kJB - 1)), sub, tol);
          named_bar(1, kJW);
        }
      }
      __syncthreads();
      // move the blocks round the ring into the receivers' other buffer
      {
        const int c = tid / (kWL / 4), f = tid % (kWL / 4);      // local column, float4 index
        if (c < COLS) {
          const bool top = c < kJB;
          int dst_rank, dst_slot;
          if (top) {
            dst_rank = rank == 0 ? 0 : (rank == kJC - 1 ? rank : rank + 1);
            dst_slot = rank == kJC - 1 ? 1 : 0;
          } else {
            dst_rank = rank == 0 ? 1 : rank - 1;
            dst_slot = rank == 0 ? 0 : 1;
          }
          float* dst = cl.map_shared_rank(buf + (1 - wb) * BUF, dst_rank);
          reinterpret_cast<float4*>(dst + (dst_slot * kJB + (c & (kJB - 1))) * kWL)[f] =
              reinterpret_cast<const float4*>(X + c * kWL)[f];
        }
      }
      cl.sync();
      wb = 1 - wb;
    }
    // convergence: every CTA tells every CTA whether it rotated in this sweep
    const int any_local = __syncthreads_or(rotated);
    int* flags = rotflag + (sweep & 1) * kJC;
    if (tid < kJC) *cl.map_shared_rank(flags + rank, tid) = any_local;
    cl.sync();
    int any = 0;
    for (int c = 0; c < kJC; ++c) any |= flags[c];
    __syncthreads();
    if (tid < kJC) flags[tid] = 0;                  // reused two sweeps later, after two cluster barriers
    sweeps = sweep + 1;
    if (!any) break;
  }
  // gather the rotated rows back into rank 0's R (the blocks are in their starting slots)
  {
    float4* dst = reinterpret_cast<float4*>(cl.map_shared_rank(R0, 0) + rank * COLS * kWL);
    const float4* src = reinterpret_cast<const float4*>(buf + wb * BUF);
    for (int e = tid; e < BUF / 4; e += blockDim.x) dst[e] = src[e];
  }
  cl.sync();
  return sweeps;
}

// Alg. 1 steps 18-19 after the Jacobi, by one CTA: row c of R now holds sigma_c u_c^T (u_c a
// right singular vector of Z = B^T), so sigma_c = ||row c||, and M = U diag(coef) U^T = X^T diag(w) X
// with w_c = coef_c / sigma_c^2 (X: the rotated rows, coef the shrinkage of Eq. 6 or the partial
// threshold); T2 = the propagated basis factor U[:, perm[:keep]]; r, sweeps, sigma and the status
// bits go to the device state.
__device__ void core_post(const float* R, const TailVec& v, int p, int sweeps, const CoreArgs& ca,
                          float* __restrict__ T1, float* __restrict__ T2, DevState* __restrict__ dst) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int N = (p + 1) / 2 * 2;
  const int warp = tid >> 5, lane = tid & 31;
  for (int c = warp; c < kWL; c += nt / 32) {
    float s2 = 0.f;
    for (int a = lane; a < kWL; a += 32) s2 = fmaf(R[c * kWL + a], R[c * kWL + a], s2);
    s2 = warp_sum(s2);
    if (lane == 0) v.sig[c] = (c < N) ? sqrtf(s2) : 0.f;
  }
  __syncthreads();
  const float tau = ca.tau_from_mu ? static_cast<float>(1.0 / dst->mu) : ca.tau_host;
  float* wv = v.thr;                                            // w_c (the thresholds are no longer needed)
  if (tid < kWL) {
    const float sc = v.sig[tid];
    const int rank = sigma_rank(v.sig, kWL, tid);
    v.perm[rank] = tid;
    const float cf = (rank < dst->partial_k && sc > 0.f) ? 1.f : ((sc > tau) ? (sc - tau) / sc : 0.f);
    v.coef[tid] = cf;
    wv[tid] = (cf > 0.f) ? cf / (sc * sc) : 0.f;
  }
  __syncthreads();
  int r = 0;
  for (int c = 0; c < kWL; ++c) r += (v.coef[c] > 0.f) ? 1 : 0;
  const int keep = ca.update_rp ? max(0, min(r, ca.l - 2)) : 0;
  for (int t = tid; t < kGB; t += nt) {          // one 4 x 4 block of M per thread and pass
    int bi2, bj2;
    block_of(t, bi2, bj2);
    float m4[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) m4[u] = 0.f;
    for (int c = 0; c < N; ++c) {
      const float w = wv[c];
      if (w == 0.f) continue;
      const float4 xa = *reinterpret_cast<const float4*>(R + c * kWL + 4 * bi2);
      const float4 xb = *reinterpret_cast<const float4*>(R + c * kWL + 4 * bj2);
      const float va[4] = {xa.x * w, xa.y * w, xa.z * w, xa.w * w};
      const float vb[4] = {xb.x, xb.y, xb.z, xb.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) m4[4 * i + j] = fmaf(va[i], vb[j], m4[4 * i + j]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        T1[(4 * bi2 + i) * kWL + 4 * bj2 + j] = m4[4 * i + j];
        T1[(4 * bj2 + j) * kWL + 4 * bi2 + i] = m4[4 * i + j];
      }
  }
  if (ca.update_rp)
    for (int e = tid; e < kWL * kWL; e += nt) {
      const int j = e / kWL, a = e % kWL;
      const int c = v.perm[j];
      T2[a * kWL + j] = (j < keep && v.sig[c] > 0.f) ? R[c * kWL + a] / v.sig[c] : 0.f;
    }
  if (tid == 0) {
    dst->r = r;
    dst->sweeps = sweeps;
    if (ca.update_rp) dst->keep = keep;
    if (ca.advance_counter) dst->counter += 1;
    if (sweeps >= ca.max_sweeps) dst->status |= kDevNotConverged;
    bool finite = true;
    for (int c = 0; c < kWL; ++c) {
      dst->sigma[c] = v.sig[v.perm[c]];
      finite = finite && isfinite(v.sig[c]);
    }
    for (int c = kWL; c < kMaxL; ++c) dst->sigma[c] = 0.f;
    if (!finite) dst->status |= kDevNonfinite;
    dst->sigma1 = static_cast<double>(v.sig[v.perm[0]]);
  }
}

// The core of Alg. 1 steps 16-19 after the Gram of Z (rank 0 factors and post-processes; the
// cluster runs the Jacobi): Cholesky of Gpk with the rank cut, one-sided Jacobi SVD of R^T,
// shrinkage, M = U diag(coef) U^T into T1 and the propagated basis factor into T2.
__global__ void __cluster_dims__(kJC, 1, 1) __launch_bounds__(kCW, 1)
k_wd_core(const double* __restrict__ Gpk, int p, double rank_tol, CoreArgs ca, float* __restrict__ T1,
          float* __restrict__ T2, DevState* __restrict__ dst) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ int rotflag[2 * kJC];
  const int rank = static_cast<int>(cooperative_groups::this_cluster().block_rank());
  df64* G = reinterpret_cast<df64*>(dsm + kTG);
  float* R = reinterpret_cast<float*>(dsm + kTR);
  const TailVec v = carve_vec(dsm);
  if (rank == 0) {
    unpack_gram<kCW>(Gpk, G);
    __syncthreads();
    wide_cholesky(G, v, R, p, rank_tol, &dst->status, reinterpret_cast<df64*>(dsm + kTP));
  }
  const int sweeps = cluster_jacobi(R, ca.max_sweeps, 8e-6f, reinterpret_cast<float*>(dsm + kTJ), rotflag);
  if (rank != 0) return;
  core_post(R, v, p, sweeps, ca, T1, T2, dst);
}

// ---------------------------------------------------------------- Q^T = R^{-T} Y^T
// One thread per long-side column x: q_c = (y_c - sum_{a<c} R[a][c] q_a) / R_cc (forward
// substitution, T = R with 1 / R_cc on the diagonal).  R^T (row c = column c of R, stride kTS)
// and the CTA's 128 input columns are staged in shared memory with coalesced loads; the column
// is solved in four blocks of 32: the block first takes the contributions of the solved blocks
// (read back from shared memory), then its own 32 x 32 triangle in registers.  The results go
// back through shared memory to coalesced stores; the output may alias the input.
constexpr int kTThr = 128;
constexpr int kTS = kWL + 4;
constexpr int kTX = kTThr + 4;                     // staged column block stride (floats)
constexpr int kTB = 32;                            // rows per block of the substitution

__global__ void __launch_bounds__(kTThr, 1)
k_wd_trsm(const float* in, int64_t ldi, int64_t len, const float* __restrict__ T, float* outT, float* outTl,
          __nv_bfloat16* __restrict__ outTb, __nv_bfloat16* __restrict__ outTbl, int64_t ldo) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  float* RT = reinterpret_cast<float*>(dsm);                 // kWL x kTS
  float* Ys = RT + kWL * kTS;                                 // kWL x kTX: Ys[c][x]
  const int64_t x0 = static_cast<int64_t>(blockIdx.x) * kTThr;
  const int nx = static_cast<int>(imin64(kTThr, len - x0));
  // staging: float4 loads, eight in flight per thread (T transposed into RT on the way)
#pragma unroll 8
  for (int e = threadIdx.x; e < kWL * kWL / 4; e += kTThr) {
    const int a = e % kWL, c4 = e / kWL;                  // consecutive threads: consecutive rows of RT
    const float4 t = __ldcg(reinterpret_cast<const float4*>(T + a * kWL) + c4);
    RT[(4 * c4) * kTS + a] = t.x;
    RT[(4 * c4 + 1) * kTS + a] = t.y;
    RT[(4 * c4 + 2) * kTS + a] = t.z;
    RT[(4 * c4 + 3) * kTS + a] = t.w;
  }
#pragma unroll 8
  for (int e = threadIdx.x; e < kWL * (kTThr / 4); e += kTThr) {
    const int c = e / (kTThr / 4), x4 = e % (kTThr / 4);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (4 * x4 < nx) v = __ldcg(reinterpret_cast<const float4*>(in + c * ldi + x0) + x4);
    *reinterpret_cast<float4*>(Ys + c * kTX + 4 * x4) = v;
  }
  __syncthreads();
  const int x = threadIdx.x;
  for (int cb = 0; cb < kWL; cb += kTB) {
    float q[kTB];
#pragma unroll
    for (int i = 0; i < kTB; ++i) q[i] = Ys[(cb + i) * kTX + x];
    // contributions of the solved rows a < cb: q_i -= sum_a R[a][cb + i] q_a
    for (int a = 0; a < cb; a += 4) {
      const float y0 = Ys[a * kTX + x], y1 = Ys[(a + 1) * kTX + x];
      const float y2 = Ys[(a + 2) * kTX + x], y3 = Ys[(a + 3) * kTX + x];
#pragma unroll
      for (int i = 0; i < kTB; ++i) {
        const float4 rv = *reinterpret_cast<const float4*>(RT + (cb + i) * kTS + a);
        q[i] = fmaf(-rv.x, y0, q[i]);
        q[i] = fmaf(-rv.y, y1, q[i]);
        q[i] = fmaf(-rv.z, y2, q[i]);
        q[i] = fmaf(-rv.w, y3, q[i]);
      }
    }
    // the block's own triangle
#pragma unroll
    for (int i = 0; i < kTB; ++i) {
      const float* rt = RT + (cb + i) * kTS + cb;
      float acc = q[i];
#pragma unroll
      for (int k = 0; k < i; ++k) acc = fmaf(-rt[k], q[k], acc);
      q[i] = acc * rt[i];
    }
#pragma unroll
    for (int i = 0; i < kTB; ++i) Ys[(cb + i) * kTX + x] = q[i];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kWL * (kTThr / 4); e += kTThr) {
    const int c = e / (kTThr / 4), x4 = e % (kTThr / 4);
    if (4 * x4 >= nx) continue;
    const float4 v = *reinterpret_cast<const float4*>(Ys + c * kTX + 4 * x4);
    reinterpret_cast<float4*>(outT + c * ldo + x0)[x4] = v;
    reinterpret_cast<float4*>(outTl + c * ldo + x0)[x4] = f4_lo(v);
    if (outTb != nullptr) {
      __nv_bfloat16 h[4], l[4];
      bf16_split(v.x, h[0], l[0]);
      bf16_split(v.y, h[1], l[1]);
      bf16_split(v.z, h[2], l[2]);
      bf16_split(v.w, h[3], l[3]);
      __nv_bfloat162* hb = reinterpret_cast<__nv_bfloat162*>(outTb + c * ldo + x0 + 4 * x4);
      __nv_bfloat162* lb = reinterpret_cast<__nv_bfloat162*>(outTbl + c * ldo + x0 + 4 * x4);
      hb[0] = __halves2bfloat162(h[0], h[1]);
      hb[1] = __halves2bfloat162(h[2], h[3]);
      lb[0] = __halves2bfloat162(l[0], l[1]);
      lb[1] = __halves2bfloat162(l[2], l[3]);
    }
  }
}

// ---------------------------------------------------------------- Out = T^T In
// out[b][x] = sum_a T[a][b] in[a][x] for the 64 long-side columns x of the CTA (staged first, so
// the output may alias the input).  Thread: x4 = t % 16 (4 columns), b4 = t / 16 (4 rows).
constexpr int kAThr = 512;
constexpr int kACols = 64;

__global__ void __launch_bounds__(kAThr, 1)
k_wd_apply(const float* in, int64_t ldi, int64_t len, const float* __restrict__ T, float* outT, float* outTl,
           int64_t ldo, float* __restrict__ outR, float* __restrict__ outRl) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  float* Ts = reinterpret_cast<float*>(dsm);              // 128 x 128
  float* Is = Ts + kWL * kWL;                             // 128 x 64
  const int64_t xs = static_cast<int64_t>(blockIdx.x) * kACols;
  const int nx = static_cast<int>(imin64(kACols, len - xs));
#pragma unroll 8                                           // eight loads in flight per thread
  for (int e = threadIdx.x; e < kWL * kWL / 4; e += kAThr)
    reinterpret_cast<float4*>(Ts)[e] = __ldcg(reinterpret_cast<const float4*>(T) + e);
#pragma unroll 8
  for (int e = threadIdx.x; e < kWL * kACols; e += kAThr) {
    const int a = e / kACols, x = e % kACols;
    Is[e] = (x < nx) ? __ldcg(in + a * ldi + xs + x) : 0.f;
  }
  __syncthreads();
  const int x4 = threadIdx.x % 16, b4 = threadIdx.x / 16;
  float acc[4][4] = {};
  for (int a = 0; a < kWL; ++a) {
    const float4 t = reinterpret_cast<const float4*>(Ts + a * kWL)[b4];
    const float4 u = reinterpret_cast<const float4*>(Is + a * kACols)[x4];
    const float tb[4] = {t.x, t.y, t.z, t.w};
    const float ux[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(tb[i], ux[j], acc[i][j]);
  }
  __syncthreads();                                         // all reads of `in` done (in-place outputs)
  for (int i = 0; i < 4; ++i) {
    const int b = 4 * b4 + i;
    const float4 v = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
    if (4 * x4 < nx) {
      if (outT != nullptr) reinterpret_cast<float4*>(outT + b * ldo + xs)[x4] = v;
      if (outTl != nullptr) reinterpret_cast<float4*>(outTl + b * ldo + xs)[x4] = f4_lo(v);
    }
  }
  if (outR != nullptr) {
    for (int j = 0; j < 4; ++j) {
      const int x = 4 * x4 + j;
      if (x >= nx) continue;
      const float4 v = make_float4(acc[0][j], acc[1][j], acc[2][j], acc[3][j]);
      reinterpret_cast<float4*>(outR + (xs + x) * kWL)[b4] = v;
      if (outRl != nullptr) reinterpret_cast<float4*>(outRl + (xs + x) * kWL)[b4] = f4_lo(v);
    }
  }
}

// ---------------------------------------------------------------- reconstruction (+ iALM)
// X tile (128 rows x 256 columns) = Z_blk Rf_blk^T on tcgen05: M = 128 rows of Z, N = 256 rows
// of Rf (columns of X), K = 128 in 4 chunks of 32; 3xTF32 as Z_hi Rf_hi + Z_lo Rf_hi + Z_hi Rf_lo
// (Z_lo, Rf_lo precomputed).  Persistent CTAs walk the tiles; the accumulator is double
// buffered in tensor memory so the epilogue of one tile overlaps the MMAs of the next.
// Epilogue: 8 warps, two per lane quarter (columns 0-127 / 128-255 of the tile).  A warp reads
// its 32 rows x 32 columns of X from tensor memory (one row per lane), stages them through shared
// memory and reads them back transposed, so that every global load of O, S, A and every store of
// S', A' (and L) covers four rows x 128 contiguous bytes per warp instruction.
constexpr int kEStages = 2;
constexpr int kEW = 8;                                   // epilogue warps
constexpr int kEThr = 64 + 32 * kEW;
constexpr uint32_t kEZ = 128 * kWK * 4;                  // 16 KB
constexpr uint32_t kER = kWN * kWK * 4;                  // 32 KB
constexpr uint32_t kEStage = 2 * kEZ + 2 * kER;          // 96 KB
constexpr int kEXs = 33;                                  // staged X chunk row stride (floats)
constexpr int kEBatch = 4;                                // row groups whose O, S, A loads are in flight together

// O, S, A at rows rbase + 4 (i0 + ii) + rr (ii < kEBatch), columns colg .. colg + 3, for the
// transposed epilogue read; full[ii]: the whole float4 is inside the matrix.
__device__ __forceinline__ void epi_load(const float* O, const float* S, const float* A, int64_t ld, int64_t m,
                                         int64_t n, int64_t rbase, int64_t colg, int i0, int rr,
                                         float (&ov)[kEBatch][4], float (&sv)[kEBatch][4], float (&av)[kEBatch][4],
                                         bool (&full)[kEBatch]) {
#pragma unroll
  for (int ii = 0; ii < kEBatch; ++ii) {
    const int64_t rowg = rbase + 4 * (i0 + ii) + rr;
    full[ii] = rowg < m && colg + 4 <= n;
    if (full[ii]) {
      const float4 o = __ldcs(reinterpret_cast<const float4*>(O + rowg * ld + colg));
      const float4 s4 = __ldcs(reinterpret_cast<const float4*>(S + rowg * ld + colg));
      const float4 a = __ldcs(reinterpret_cast<const float4*>(A + rowg * ld + colg));
      ov[ii][0] = o.x; ov[ii][1] = o.y; ov[ii][2] = o.z; ov[ii][3] = o.w;
      sv[ii][0] = s4.x; sv[ii][1] = s4.y; sv[ii][2] = s4.z; sv[ii][3] = s4.w;
      av[ii][0] = a.x; av[ii][1] = a.y; av[ii][2] = a.z; av[ii][3] = a.w;
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const bool in = rowg < m && colg + e < n;
        ov[ii][e] = in ? O[rowg * ld + colg + e] : 0.f;
        sv[ii][e] = in ? S[rowg * ld + colg + e] : 0.f;
        av[ii][e] = in ? A[rowg * ld + colg + e] : 0.f;
      }
    }
  }
}
constexpr uint32_t kESmem = kEStages * kEStage + kEW * 32 * kEXs * 4;   // + 8 x 4.2 KB for the transpose
// The iALM form keeps one operand stage (a tile's four K-chunks are loaded and multiplied well
// within the time its epilogue takes) and gives the other 96 KB to a per-warp ring of O, S, A:
// two slots of 16 rows x 32 columns of each, filled by cp.async two half-chunks ahead.
constexpr int kESlot = 3 * 16 * 32;                                      // floats per ring slot
constexpr uint32_t kESmemAlm = kEStage + kEW * 32 * kEXs * 4 + kEW * 2 * kESlot * 4;

template <bool ALM>
__global__ void __launch_bounds__(kEThr, 1)
k_wd_alm(const __grid_constant__ CUtensorMap tmZ, const __grid_constant__ CUtensorMap tmZl,
         const __grid_constant__ CUtensorMap tmR, const __grid_constant__ CUtensorMap tmRl, int64_t m, int64_t n,
         const float* __restrict__ O, float* __restrict__ S, float* __restrict__ A, int64_t ld, float* __restrict__ L,
         int64_t ldl, DevState* __restrict__ dst, double* __restrict__ cpart, unsigned* __restrict__ ticket,
         __nv_bfloat16* __restrict__ Ab, int64_t ldb) {
  constexpr int NS = ALM ? 1 : kEStages;              // operand stages
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ __align__(8) uint64_t full[kEStages], empty[kEStages], acc_full[2], acc_empty[2];
  __shared__ uint32_t tmem_base;
  __shared__ double red[kEThr / 32];
  __shared__ int flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntr = static_cast<int>((m + 127) / 128), ntc = static_cast<int>((n + kWN - 1) / kWN);
  const int ntiles = ntr * ntc;
  const int mine = (blockIdx.x < ntiles) ? (ntiles - 1 - static_cast<int>(blockIdx.x)) / gridDim.x + 1 : 0;
  if ((smem_addr(dsm) & 1023u) != 0u) {               // swizzled TMA destinations need 1024-byte alignment
    if (threadIdx.x == 0) atomicOr(&dst->status, kDevBadProblem);
    return;
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], kEW);
    }
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc(&tmem_base, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base;
  bool ok = true;
  float res2 = 0.f;
  if (warp == 0) {
    if (lane == 0) {
      prefetch_tensormap(&tmZ);
      prefetch_tensormap(&tmZl);
      prefetch_tensormap(&tmR);
      prefetch_tensormap(&tmRl);
      for (int g = 0; g < 4 * mine && ok; ++g) {
        const int s = g % NS, u = g / NS;
        const int tl = static_cast<int>(blockIdx.x) + (g / 4) * static_cast<int>(gridDim.x);
        const int tr = tl / ntc, tc = tl % ntc, c = g % 4;
        if (u > 0 && !mbar_wait(&empty[s], static_cast<uint32_t>(u - 1) & 1u)) {
          flag_timeout(ok, dst);
          break;
        }
        unsigned char* st = dsm + s * kEStage;
        mbar_arrive_expect_tx(&full[s], kEStage);
        tma_load_2d(st, &tmZ, kWK * c, 128 * tr, &full[s]);
        tma_load_2d(st + kEZ, &tmZl, kWK * c, 128 * tr, &full[s]);
        tma_load_2d(st + 2 * kEZ, &tmR, kWK * c, kWN * tc, &full[s]);
        tma_load_2d(st + 2 * kEZ + kER, &tmRl, kWK * c, kWN * tc, &full[s]);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_tf32(128, kWN);
      for (int k = 0; k < mine; ++k) {
        const int buf = k & 1;
        if (k >= 2 && ok && !mbar_wait(&acc_empty[buf], static_cast<uint32_t>(k / 2 - 1) & 1u)) flag_timeout(ok, dst);
        tc_fence_after();
        const uint32_t d = tbase + static_cast<uint32_t>(buf * kWN);
        for (int c = 0; c < 4; ++c) {
          const int g = 4 * k + c;
          const int s = g % NS, u = g / NS;
          if (ok && !mbar_wait(&full[s], static_cast<uint32_t>(u) & 1u)) flag_timeout(ok, dst);
          tc_fence_after();
          const unsigned char* st = dsm + s * kEStage;
#pragma unroll
          for (int ks = 0; ks < kWK / 8; ++ks) {
            const uint64_t zh = smem_desc_sw128(st + 32 * ks, 16, 1024);
            const uint64_t zl = smem_desc_sw128(st + kEZ + 32 * ks, 16, 1024);
            const uint64_t rh = smem_desc_sw128(st + 2 * kEZ + 32 * ks, 16, 1024);
            const uint64_t rl = smem_desc_sw128(st + 2 * kEZ + kER + 32 * ks, 16, 1024);
            tc_mma_tf32(d, zh, rh, idesc, c > 0 || ks > 0);
            tc_mma_tf32(d, zl, rh, idesc, true);
            tc_mma_tf32(d, zh, rl, idesc, true);
          }
          tc_commit(&empty[s]);
        }
        tc_commit(&acc_full[buf]);
      }
    }
  } else if (ALM) {
    // epilogue warps, iALM form: lane (rr, c4) takes rows 4 i + rr and columns c4 .. c4 + 3 of
    // each 16-row half of the warp's 32 x 32 chunk of X; its O, S, A come from the ring slot that
    // cp.async filled two half-chunks earlier.  Step s = 8 k + 2 cg + hh: tile k of this CTA,
    // column group cg, row half hh.
    const int q = warp & 3, half = (warp - 2) >> 2;
    const double mu = dst->mu;
    const double mu_next = fmin(dst->rho * mu, dst->mu_bar);
    const float thr = static_cast<float>(dst->lambda / mu);
    const float ratio = static_cast<float>(mu / mu_next);
    float* sX = reinterpret_cast<float*>(dsm + NS * kEStage) + (warp - 2) * (32 * kEXs);
    float* ring = reinterpret_cast<float*>(dsm + NS * kEStage + kEW * 32 * kEXs * 4) + (warp - 2) * (2 * kESlot);
    const int rr = lane >> 3, c4 = 4 * (lane & 7);
    auto fill = [&](int s) {                           // one cp.async group per step, empty past the end
      if (s < 8 * mine) {
        const int k = s >> 3, cg = (s >> 1) & 3, hh = s & 1;
        const int tl = static_cast<int>(blockIdx.x) + k * static_cast<int>(gridDim.x);
        const int64_t rbase = 128 * static_cast<int64_t>(tl / ntc) + 32 * q + 16 * hh;
        const int64_t colg = static_cast<int64_t>(kWN) * (tl % ntc) + 128 * half + 32 * cg + c4;
        float* slot = ring + (s & 1) * kESlot;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int64_t rowg = rbase + 4 * i + rr;
          const bool in = rowg < m && colg < n;
          const int bytes = in ? 4 * static_cast<int>(imin64(4, n - colg)) : 0;
          const int64_t off = in ? rowg * ld + colg : 0;
          float* d = slot + (4 * i + rr) * 32 + c4;
          cp_async16(d, O + off, bytes);
          cp_async16(d + 512, S + off, bytes);
          cp_async16(d + 1024, A + off, bytes);
        }
      }
      cp_async_commit();
    };
    fill(0);
    fill(1);
    for (int k = 0; k < mine; ++k) {
      const int buf = k & 1;
      const int tl = static_cast<int>(blockIdx.x) + k * static_cast<int>(gridDim.x);
      const int tr = tl / ntc, tc = tl % ntc;
      if (ok && !mbar_wait(&acc_full[buf], static_cast<uint32_t>(k / 2) & 1u)) flag_timeout(ok, dst);
      tc_fence_after();
      const int64_t rbase = 128 * static_cast<int64_t>(tr) + 32 * q;   // the warp's 32 rows
      for (int cg = 0; cg < 4; ++cg) {
        const int colt = 128 * half + 32 * cg;
        const int64_t colg = static_cast<int64_t>(kWN) * tc + colt + c4;
        {                                              // the 32 x 32 chunk of X, staged row-major
          float x[16];
          const uint32_t ta = tbase + (static_cast<uint32_t>(32 * q) << 16) + static_cast<uint32_t>(buf * kWN + colt);
          tmem_ld16(ta, x);
#pragma unroll
          for (int j = 0; j < 16; ++j) sX[lane * kEXs + j] = x[j];
          tmem_ld16(ta + 16, x);
#pragma unroll
          for (int j = 0; j < 16; ++j) sX[lane * kEXs + 16 + j] = x[j];
        }
        for (int hh = 0; hh < 2; ++hh) {
          const int s = 8 * k + 2 * cg + hh;
          cp_async_wait<1>();                          // step s's group has landed (s + 1 may be in flight)
          __syncwarp();                                // ... for every lane, and sX is complete
          const float* slot = ring + (s & 1) * kESlot;
          float4 ov[4], sv[4], av[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float* src = slot + (4 * i + rr) * 32 + c4;
            ov[i] = *reinterpret_cast<const float4*>(src);
            sv[i] = *reinterpret_cast<const float4*>(src + 512);
            av[i] = *reinterpret_cast<const float4*>(src + 1024);
          }
          __syncwarp();                                // the slot is free again
          fill(s + 2);
          if (!ok) continue;
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int r = 16 * hh + 4 * i + rr;
            const int64_t rowg = rbase + r;
            const float o4[4] = {ov[i].x, ov[i].y, ov[i].z, ov[i].w};
            const float s4[4] = {sv[i].x, sv[i].y, sv[i].z, sv[i].w};
            const float a4[4] = {av[i].x, av[i].y, av[i].z, av[i].w};
            float sn[4], an[4], xv[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              xv[e] = sX[r * kEXs + c4 + e];
              const float t = a4[e] + s4[e] - xv[e];                            // O - L + Y / mu
              sn[e] = (t > thr) ? (t - thr) : ((t < -thr) ? (t + thr) : 0.f);
              an[e] = o4[e] - sn[e] + ratio * (t - sn[e]);                      // O - S' + Y' / mu'
              const float rz = o4[e] - xv[e] - sn[e];                           // O - L - S'
              if (rowg < m && colg + e < n) res2 = fmaf(rz, rz, res2);
            }
            if (rowg < m && colg + 4 <= n) {
              __stcs(reinterpret_cast<float4*>(S + rowg * ld + colg), make_float4(sn[0], sn[1], sn[2], sn[3]));
              __stcs(reinterpret_cast<float4*>(A + rowg * ld + colg), make_float4(an[0], an[1], an[2], an[3]));
              if (L != nullptr)
                *reinterpret_cast<float4*>(L + rowg * ldl + colg) = make_float4(xv[0], xv[1], xv[2], xv[3]);
              if (Ab != nullptr) {                                              // BF16 shadow of A'
                const __nv_bfloat162 b0 = __floats2bfloat162_rn(an[0], an[1]);
                const __nv_bfloat162 b1 = __floats2bfloat162_rn(an[2], an[3]);
                __stcs(reinterpret_cast<uint2*>(Ab + rowg * ldb + colg),
                       make_uint2(*reinterpret_cast<const uint32_t*>(&b0), *reinterpret_cast<const uint32_t*>(&b1)));
              }
            } else {
              for (int e = 0; e < 4; ++e)
                if (rowg < m && colg + e < n) {
                  S[rowg * ld + colg + e] = sn[e];
                  A[rowg * ld + colg + e] = an[e];
                  if (L != nullptr) L[rowg * ldl + colg + e] = xv[e];
                  if (Ab != nullptr) Ab[rowg * ldb + colg + e] = __float2bfloat16_rn(an[e]);
                }
            }
          }
        }
        __syncwarp();                                  // sX is rewritten by the next chunk
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);
    }
    cp_async_wait<0>();
  } else {
    const int q = warp & 3, half = (warp - 2) >> 2;
    double mu = 0.0, mu_next = 0.0;
    float thr = 0.f, ratio = 0.f;
    if (ALM) {
      mu = dst->mu;
      mu_next = fmin(dst->rho * mu, dst->mu_bar);
      thr = static_cast<float>(dst->lambda / mu);
      ratio = static_cast<float>(mu / mu_next);
    }
    float* sX = reinterpret_cast<float*>(dsm + kEStages * kEStage) + (warp - 2) * (32 * kEXs);
    const int rr = lane >> 3, c4 = 4 * (lane & 7);      // transposed read: row group, column quad
    for (int k = 0; k < mine; ++k) {
      const int buf = k & 1;
      const int tl = static_cast<int>(blockIdx.x) + k * static_cast<int>(gridDim.x);
      const int tr = tl / ntc, tc = tl % ntc;
      if (ok && !mbar_wait(&acc_full[buf], static_cast<uint32_t>(k / 2) & 1u)) flag_timeout(ok, dst);
      tc_fence_after();
      const int64_t rbase = 128 * static_cast<int64_t>(tr) + 32 * q;   // the warp's 32 rows
      for (int cg = 0; cg < 4; ++cg) {
        const int colt = 128 * half + 32 * cg;
        const int64_t col0 = static_cast<int64_t>(kWN) * tc + colt;
        const bool act = ok && rbase < m && col0 < n;  // warp-uniform
        const int64_t colg = col0 + c4;
        float ov[kEBatch][4], sv[kEBatch][4], av[kEBatch][4];
        bool full[kEBatch];
        // the first row groups' O, S, A loads go out before the tensor-memory read (they do not
        // depend on X), so that their latency overlaps it
        if (ALM && act) epi_load(O, S, A, ld, m, n, rbase, colg, 0, rr, ov, sv, av, full);
        {                                              // the 32 x 32 chunk of X, staged row-major
          float x[16];
          const uint32_t ta = tbase + (static_cast<uint32_t>(32 * q) << 16) + static_cast<uint32_t>(buf * kWN + colt);
          tmem_ld16(ta, x);
#pragma unroll
          for (int j = 0; j < 16; ++j) sX[lane * kEXs + j] = x[j];
          tmem_ld16(ta + 16, x);
#pragma unroll
          for (int j = 0; j < 16; ++j) sX[lane * kEXs + 16 + j] = x[j];
        }
        __syncwarp();
        if (act) {
          // lane (rr, c4) takes rows 4 i + rr, columns c4 .. c4 + 3: every load and store below
          // covers four rows x 128 contiguous bytes per warp
#pragma unroll
          for (int i0 = 0; i0 < 8; i0 += kEBatch) {
            if (i0 > 0) {
              if (ALM) {
                epi_load(O, S, A, ld, m, n, rbase, colg, i0, rr, ov, sv, av, full);
              } else {
#pragma unroll
                for (int ii = 0; ii < kEBatch; ++ii) full[ii] = rbase + 4 * (i0 + ii) + rr < m && colg + 4 <= n;
              }
            } else if (!ALM) {
#pragma unroll
              for (int ii = 0; ii < kEBatch; ++ii) full[ii] = rbase + 4 * ii + rr < m && colg + 4 <= n;
            }
#pragma unroll
            for (int ii = 0; ii < kEBatch; ++ii) {
              const int r = 4 * (i0 + ii) + rr;
              const int64_t rowg = rbase + r;
              float xv[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) xv[e] = sX[r * kEXs + c4 + e];
              if (!ALM) {
                if (full[ii]) {
                  *reinterpret_cast<float4*>(L + rowg * ldl + colg) = make_float4(xv[0], xv[1], xv[2], xv[3]);
                } else {
                  for (int e = 0; e < 4; ++e)
                    if (rowg < m && colg + e < n) L[rowg * ldl + colg + e] = xv[e];
                }
                continue;
              }
              float sn[4], an[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const float t = av[ii][e] + sv[ii][e] - xv[e];                  // O - L + Y / mu
                sn[e] = (t > thr) ? (t - thr) : ((t < -thr) ? (t + thr) : 0.f);
                an[e] = ov[ii][e] - sn[e] + ratio * (t - sn[e]);                // O - S' + Y' / mu'
                const float rz = ov[ii][e] - xv[e] - sn[e];                     // O - L - S'
                if (rowg < m && colg + e < n) res2 = fmaf(rz, rz, res2);
              }
              if (full[ii]) {
                __stcs(reinterpret_cast<float4*>(S + rowg * ld + colg), make_float4(sn[0], sn[1], sn[2], sn[3]));
                __stcs(reinterpret_cast<float4*>(A + rowg * ld + colg), make_float4(an[0], an[1], an[2], an[3]));
                if (L != nullptr)
                  *reinterpret_cast<float4*>(L + rowg * ldl + colg) = make_float4(xv[0], xv[1], xv[2], xv[3]);
                if (Ab != nullptr) {                                            // BF16 shadow of A'
                  const __nv_bfloat162 b0 = __floats2bfloat162_rn(an[0], an[1]);
                  const __nv_bfloat162 b1 = __floats2bfloat162_rn(an[2], an[3]);
                  __stcs(reinterpret_cast<uint2*>(Ab + rowg * ldb + colg),
                         make_uint2(*reinterpret_cast<const uint32_t*>(&b0), *reinterpret_cast<const uint32_t*>(&b1)));
                }
              } else {
                for (int e = 0; e < 4; ++e)
                  if (rowg < m && colg + e < n) {
                    S[rowg * ld + colg + e] = sn[e];
                    A[rowg * ld + colg + e] = an[e];
                    if (L != nullptr) L[rowg * ldl + colg + e] = xv[e];
                    if (Ab != nullptr) Ab[rowg * ldb + colg + e] = __float2bfloat16_rn(an[e]);
                  }
              }
            }
          }
        }
        __syncwarp();                                  // sX is rewritten by the next chunk
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tbase, 512);
  if (!ALM) return;
  const double v = warp_sum(static_cast<double>(res2));
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kEThr / 32; ++w) t += red[w];
    cpart[blockIdx.x] = t;
  }
  if (!last_of(ticket, gridDim.x, &flag)) return;
  if (threadIdx.x == 0) {
    double s2 = 0.0;
    for (int b = 0; b < static_cast<int>(gridDim.x); ++b) s2 += __ldcg(cpart + b);
    const double rr = (dst->normO_F > 0.0) ? sqrt(s2) / dst->normO_F : 0.0;
    const double mu = dst->mu;
    dst->resid_ratio = rr;
    if (!isfinite(rr)) dst->status |= kDevNonfinite;
    dst->mu = fmin(dst->rho * mu, dst->mu_bar);
    dst->iter += 1;
  }
}

template <typename K>
cudaError_t set_dyn(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
}

}  // namespace

// ---------------------------------------------------------------- host side
int wide_lp() { return kWL; }
int wide_tile() { return kWN; }

cudaError_t prepare_wide_kernels() {
  cudaError_t e = set_dyn(k_wd_pass<false, 0>, kWStages * kWStage);
  if (e == cudaSuccess) e = set_dyn(k_wd_pass<true, 0>, kWStages * kWStage);
  if (e == cudaSuccess) e = set_dyn(k_wd_pass<false, 1>, kWStages * kWStage);
  if (e == cudaSuccess) e = set_dyn(k_wd_pass<true, 1>, kWStages * kWStage);
  if (e == cudaSuccess) e = set_dyn(k_wd_pass<false, 2>, 2 * (kWStage + 16384));
  if (e == cudaSuccess) e = set_dyn(k_wd_pass<true, 2>, 2 * (kWStage + 16384));
  if (e == cudaSuccess) e = set_dyn(k_wd_gram, kGSmem);
  if (e == cudaSuccess) e = set_dyn(k_wd_orth, kTSmem);
  if (e == cudaSuccess) e = set_dyn(k_wd_core, kTSmem);
  if (e == cudaSuccess) e = set_dyn(k_wd_apply, sizeof(float) * kWL * (kWL + kACols));
  if (e == cudaSuccess) e = set_dyn(k_wd_trsm, sizeof(float) * kWL * (kTS + kTX));
  if (e == cudaSuccess) e = set_dyn(k_wd_alm<true>, kESmemAlm);
  if (e == cudaSuccess) e = set_dyn(k_wd_alm<false>, kESmem);
  return e;
}

// CTAs of the Gram kernel: one per SM (each holds one partial).
int wide_gram_grid() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms = 0;
  (void)cudaGetLastError();
  return sms;
}

int wide_gram_count() { return kGCount; }

cudaError_t launch_wd_omega(float* OT, float* OTl, void* OTb, void* OTbl, int64_t ldo, int64_t m, int l, int use_rp,
                            uint64_t seed, uint64_t ctr, const DevState* dst, cudaStream_t st) {
  const int64_t total = m * (kWL / 4);
  int64_t grid = (total + 255) / 256;
  if (grid > 4096) grid = 4096;
  k_wd_omega<<<static_cast<int>(grid), 256, 0, st>>>(OT, OTl, static_cast<__nv_bfloat16*>(OTb),
                                                     static_cast<__nv_bfloat16*>(OTbl), ldo, m, l, use_rp, seed, ctr,
                                                     dst);
  return cudaGetLastError();
}

// CTAs of a pass: the ntiles x nkc units cut into G ranges, G = the SM count (at least two units
// per CTA, at least one CTA per tile), lowered until no tile is cut into more than kWParts
// segments (the partial planes of the workspace).  Host copy of pass_cta_of.
static int64_t pass_cta_of_host(int64_t x, int64_t U, int64_t G) { return ((x + 1) * G + U - 1) / U - 1; }

int wide_pass_grid(int64_t nlong, int64_t nk, int prec, int sms) {
  const int64_t ntiles = (nlong + kWN - 1) / kWN;
  const int64_t nkc = (nk + (prec ? 64 : kWK) - 1) / (prec ? 64 : kWK);
  const int64_t U = ntiles * nkc;
  if (ntiles < 1 || nkc < 1) return 0;
  int64_t G = sms < U / 2 ? sms : U / 2;
  if (G < ntiles) G = ntiles;
  for (; G > ntiles; --G) {
    int64_t worst = 0;
    for (int64_t t = 0; t < ntiles; ++t) {
      const int64_t n = pass_cta_of_host((t + 1) * nkc - 1, U, G) - pass_cta_of_host(t * nkc, U, G) + 1;
      worst = n > worst ? n : worst;
    }
    if (worst <= kWParts) break;
  }
  return static_cast<int>(G);
}

// The plan wide_pass_grid gives a pass: its CTA count, the most segments (partials) of one tile
// and the most tiles one CTA's range touches.
void wide_pass_plan(int64_t nlong, int64_t nk, int prec, int sms, int* grid, int* max_parts, int* max_tiles) {
  const int64_t ntiles = (nlong + kWN - 1) / kWN;
  const int64_t nkc = (nk + (prec ? 64 : kWK) - 1) / (prec ? 64 : kWK);
  const int64_t U = ntiles * nkc;
  const int G = wide_pass_grid(nlong, nk, prec, sms);
  int mp = 0, mt = 0;
  if (G > 0) {
    for (int64_t t = 0; t < ntiles; ++t) {
      const int64_t n = pass_cta_of_host((t + 1) * nkc - 1, U, G) - pass_cta_of_host(t * nkc, U, G) + 1;
      mp = n > mp ? static_cast<int>(n) : mp;
    }
    for (int64_t b = 0; b < G; ++b) {
      const int64_t u0 = b * U / G, u1 = (b + 1) * U / G;
      const int64_t n = u1 > u0 ? (u1 - 1) / nkc - u0 / nkc + 1 : 0;
      mt = n > mt ? static_cast<int>(n) : mt;
    }
  }
  *grid = G;
  *max_parts = mp;
  *max_tiles = mt;
}

cudaError_t launch_wd_pass(bool col, int prec, const CUtensorMap& tmA, const CUtensorMap& tmM, const CUtensorMap& tmMl,
                           int64_t nlong, int64_t nk, int sms, float* part, int64_t ldp, float* outT, float* outTl,
                           void* outTb, void* outTbl, int64_t ldo, float* outR, float* outRl, DevState* dst,
                           cudaStream_t st, const float* scales, int ntr8, int ntc8) {
  const int G = wide_pass_grid(nlong, nk, prec, sms);
  if (G < 1) return cudaErrorInvalidValue;
  const size_t smem = prec == 2 ? 2 * (kWStage + 16384) : kWStages * kWStage;
  __nv_bfloat16* tb = static_cast<__nv_bfloat16*>(outTb);
  __nv_bfloat16* tbl = static_cast<__nv_bfloat16*>(outTbl);
#define ARGS tmA, tmM, tmMl, nlong, nk, G, part, ldp, dst, scales, ntr8, ntc8
  if (prec == 0) {
    if (col) k_wd_pass<true, 0><<<G, kWThr, smem, st>>>(ARGS);
    else k_wd_pass<false, 0><<<G, kWThr, smem, st>>>(ARGS);
  } else if (prec == 1) {
    if (col) k_wd_pass<true, 1><<<G, kWThr, smem, st>>>(ARGS);
    else k_wd_pass<false, 1><<<G, kWThr, smem, st>>>(ARGS);
  } else {
    if (col) k_wd_pass<true, 2><<<G, kWThr, smem, st>>>(ARGS);
    else k_wd_pass<false, 2><<<G, kWThr, smem, st>>>(ARGS);
  }
#undef ARGS
  const int64_t ntiles = (nlong + kWN - 1) / kWN;
  const int64_t nkc = (nk + (prec ? 64 : kWK) - 1) / (prec ? 64 : kWK);
  k_wd_psum<<<static_cast<int>(ntiles * (kWL / kPsRows)), kPsThr, 0, st>>>(part, ldp, nlong, nkc, G, outT, outTl, tb,
                                                                           tbl, ldo, outR, outRl);
  return cudaGetLastError();
}

cudaError_t launch_wd_gram(bool core, const float* XT, int64_t ldx, int64_t len, int grid, double* cpart, double* Gpk,
                           int p, double rank_tol, int l, float tau_host, int tau_from_mu, int update_rp,
                           int advance_counter, int max_sweeps, float* T1, float* T2, DevState* dst,
                           cudaStream_t st) {
  const int64_t per = (len + grid - 1) / grid;
  CoreArgs ca{l, tau_host, tau_from_mu, update_rp, advance_counter, max_sweeps};
  k_wd_gram<<<grid, kGW, kGSmem, st>>>(XT, ldx, len, per, cpart, p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_wd_gsum<<<(kGCount + kGSumE - 1) / kGSumE, kGSumT, 0, st>>>(cpart, grid, Gpk);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (core)
    k_wd_core<<<kJC, kCW, kTSmem, st>>>(Gpk, p, rank_tol, ca, T1, T2, dst);
  else
    k_wd_orth<<<1, kTW, kTSmem, st>>>(Gpk, p, rank_tol, T1, dst);
  return cudaGetLastError();
}

cudaError_t launch_wd_apply(const float* in, int64_t ldi, int64_t len, const float* T, float* outT, float* outTl,
                            int64_t ldo, float* outR, float* outRl, cudaStream_t st) {
  const int grid = static_cast<int>((len + kACols - 1) / kACols);
  if (grid == 0) return cudaSuccess;
  k_wd_apply<<<grid, kAThr, sizeof(float) * kWL * (kWL + kACols), st>>>(in, ldi, len, T, outT, outTl, ldo, outR, outRl);
  return cudaGetLastError();
}

cudaError_t launch_wd_quant8(const float* A, int64_t lda, int64_t m, int64_t n, void* A8, int64_t ld8, float* scales,
                             cudaStream_t st) {
  const int ntr = static_cast<int>((m + kQT - 1) / kQT), ntc = static_cast<int>((n + kQT - 1) / kQT);
  if (ntr == 0 || ntc == 0) return cudaSuccess;
  k_wd_quant8<<<ntr * ntc, kQThr, 0, st>>>(A, lda, m, n, static_cast<uint8_t*>(A8), ld8, scales, ntc);
  return cudaGetLastError();
}

cudaError_t launch_wd_rp_insert(float* YT, const float* QtT, int64_t ld, int64_t ns, int l, const DevState* dst,
                               cudaStream_t st) {
  const int64_t total = static_cast<int64_t>(l) * ns;
  int64_t grid = (total + 255) / 256;
  if (grid > 1024) grid = 1024;
  if (grid == 0) return cudaSuccess;
  k_wd_rp_insert<<<static_cast<int>(grid), 256, 0, st>>>(YT, QtT, ld, ns, l, dst);
  return cudaGetLastError();
}

cudaError_t launch_wd_colscale(const float* YT, int64_t ld, int64_t ns, float* T, cudaStream_t st) {
  k_wd_colscale<<<kWL, 256, 0, st>>>(YT, ld, ns, T);
  return cudaGetLastError();
}

cudaError_t launch_wd_identity(float* T, cudaStream_t st) {
  k_wd_identity<<<16, 256, 0, st>>>(T);
  return cudaGetLastError();
}

cudaError_t launch_wd_trsm(const float* in, int64_t ldi, int64_t len, const float* T, float* outT, float* outTl,
                           void* outTb, void* outTbl, int64_t ldo, cudaStream_t st) {
  const int grid = static_cast<int>((len + kTThr - 1) / kTThr);
  if (grid == 0) return cudaSuccess;
  k_wd_trsm<<<grid, kTThr, sizeof(float) * kWL * (kTS + kTX), st>>>(in, ldi, len, T, outT, outTl,
                                                                       static_cast<__nv_bfloat16*>(outTb),
                                                                       static_cast<__nv_bfloat16*>(outTbl), ldo);
  return cudaGetLastError();
}

cudaError_t launch_wd_alm(bool alm, const CUtensorMap& tmZ, const CUtensorMap& tmZl, const CUtensorMap& tmR,
                          const CUtensorMap& tmRl, int64_t m, int64_t n, const float* O, float* S, float* A, int64_t ld,
                          float* L, int64_t ldl, DevState* dst, double* cpart, unsigned* ticket, int grid,
                          void* Ab, int64_t ldb, cudaStream_t st) {
  const size_t smem = alm ? kESmemAlm : kESmem;
  __nv_bfloat16* ab = static_cast<__nv_bfloat16*>(Ab);
  if (alm)
    k_wd_alm<true><<<grid, kEThr, smem, st>>>(tmZ, tmZl, tmR, tmRl, m, n, O, S, A, ld, L, ldl, dst, cpart, ticket, ab,
                                              ldb);
  else
    k_wd_alm<false><<<grid, kEThr, smem, st>>>(tmZ, tmZl, tmR, tmRl, m, n, O, S, A, ld, L, ldl, dst, cpart, ticket,
                                               nullptr, 0);
  return cudaGetLastError();
}

}  // namespace frsvt
