// Device-side helpers shared by the FRSVT kernels (sm_103a).
//
// - Philox4x64-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11)
//   and the Box-Muller map that draw the Gaussian test matrix Omega of Alg. 1
//   (steps 4 and 8; Sec. 2.4 uses dense N(0,1) entries).  The stream contract:
//     key = (seed, 0); counter = (row i, column block j, stream t, problem b);
//     u(x) = ((x >> 41) + 0.5) * 2^-23;
//     (z0, z1) = sqrt(-2 ln u(x0)) (cos 2pi u(x1), sin 2pi u(x1)), same for (x2, x3);
//     Omega[i, 4j + k] = z_k.
// - Double-float ("df64") accumulation: the exact product of two floats as an
//   unevaluated sum hi + lo (FMA-based two-product) added into a (hi, lo) pair
//   with Knuth's two-sum.  GB300 runs FP64 at a small fraction of its FP32
//   rate, so Gram matrices that must be accumulated beyond FP32 precision are
//   accumulated this way on the FP32 pipes (about 44 significant bits).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace frsvt {

constexpr uint64_t kPhiloxM0 = 0xD2E7470EE14C6C93ull;
constexpr uint64_t kPhiloxM1 = 0xCA5A826395121157ull;
constexpr uint64_t kPhiloxW0 = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kPhiloxW1 = 0xBB67AE8584CAA73Bull;

struct u64x4 { uint64_t x, y, z, w; };

__device__ __forceinline__ u64x4 philox4x64_10(u64x4 c, uint64_t k0, uint64_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += kPhiloxW0; k1 += kPhiloxW1; }
    const uint64_t lo0 = kPhiloxM0 * c.x, hi0 = __umul64hi(kPhiloxM0, c.x);
    const uint64_t lo1 = kPhiloxM1 * c.z, hi1 = __umul64hi(kPhiloxM1, c.z);
    c = u64x4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
  }
  return c;
}

__device__ __forceinline__ float uniform23(uint64_t x) {
  return (static_cast<float>(static_cast<uint32_t>(x >> 41)) + 0.5f) * 1.1920928955078125e-07f;  // 2^-23
}

// Four N(0,1) values Omega[row, 4*blk .. 4*blk+3] of the (seed, stream, problem) stream.
__device__ __forceinline__ float4 gaussian4(uint64_t seed, uint64_t row, uint64_t blk,
                                            uint64_t stream, uint64_t problem) {
  const u64x4 w = philox4x64_10(u64x4{row, blk, stream, problem}, seed, 0ull);
  float s0, c0, s1, c1;
  const float r0 = sqrtf(-2.0f * logf(uniform23(w.x)));
  sincospif(2.0f * uniform23(w.y), &s0, &c0);
  const float r1 = sqrtf(-2.0f * logf(uniform23(w.z)));
  sincospif(2.0f * uniform23(w.w), &s1, &c1);
  return make_float4(r0 * c0, r0 * s0, r1 * c1, r1 * s1);
}

// ---------------------------------------------------------------- df64 accumulation
struct df64 { float hi, lo; };

__device__ __forceinline__ void df64_add_prod(df64& acc, float a, float b) {
  const float p = a * b;
  const float e = __fmaf_rn(a, b, -p);          // exact: a*b = p + e
  const float s = __fadd_rn(acc.hi, p);         // two-sum(acc.hi, p)
  const float bb = __fsub_rn(s, acc.hi);
  const float err = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  acc.hi = s;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(err, e));
}

__device__ __forceinline__ double df64_value(df64 a) {
  return static_cast<double>(a.hi) + static_cast<double>(a.lo);
}

// Double-float arithmetic (Dekker / Knuth error-free transformations) with round-to-nearest
// intrinsics, which the compiler never contracts or reassociates.  ~48 significant bits.
__device__ __forceinline__ df64 df_quick(float hi, float lo) {
  const float s = __fadd_rn(hi, lo);
  return df64{s, __fsub_rn(lo, __fsub_rn(s, hi))};
}

__device__ __forceinline__ df64 df_add(df64 a, df64 b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  return df_quick(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df64 df_neg(df64 a) { return df64{-a.hi, -a.lo}; }

__device__ __forceinline__ df64 df_mul(df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_quick(p, e);
}

__device__ __forceinline__ df64 df_from_double(double x) {
  const float hi = static_cast<float>(x);
  return df64{hi, static_cast<float>(x - static_cast<double>(hi))};
}

// 1 / sqrt(a) for a > 0 in the float range: float seed and one Newton step in double-float,
// y1 = y0 + y0 (1 - a y0^2) / 2 (the error squares: ~2^-46 relative).
__device__ __forceinline__ df64 df_rsqrt(df64 a) {
  const df64 y{rsqrtf(a.hi), 0.f};
  const df64 r = df_add(df64{1.f, 0.f}, df_neg(df_mul(a, df_mul(y, y))));
  df64 c = df_mul(y, r);
  c.hi = __fmul_rn(c.hi, 0.5f);
  c.lo = __fmul_rn(c.lo, 0.5f);
  return df_add(y, c);
}

// The same Newton step with a shorter dependency chain: the residual h = 1 - a y0^2 is formed by
// FMAs from the exact square y0^2 = t + te (te = fma(y0, y0, -t)), h = 1 - a.hi t - a.hi te -
// a.lo t, and y1 = y0 + y0 h / 2 is returned as the pair (y0, y0 h / 2) renormalised.
__device__ __forceinline__ df64 df_rsqrt_fma(df64 a) {
  const float y = rsqrtf(a.hi);
  const float t = __fmul_rn(y, y);
  const float te = __fmaf_rn(y, y, -t);
  float h = __fmaf_rn(-a.hi, t, 1.f);
  h = __fmaf_rn(-a.hi, te, h);
  h = __fmaf_rn(-a.lo, t, h);
  return df_quick(y, __fmul_rn(__fmul_rn(0.5f, y), h));
}

// g - x y in double-float: the product split exactly with FMAs (the cross terms with the low
// parts folded into its error), its high part taken off g.hi by two-sum, the low-order terms
// gathered in one float, the pair renormalised.
__device__ __forceinline__ df64 df_fms(df64 g, df64 x, df64 y) {
  const float pr = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -pr);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  const float s = __fsub_rn(g.hi, pr);
  const float bb = __fsub_rn(s, g.hi);
  const float err = __fsub_rn(__fsub_rn(g.hi, __fsub_rn(s, bb)), __fadd_rn(pr, bb));
  return df_quick(s, __fadd_rn(g.lo, __fsub_rn(err, e)));
}

// ---------------------------------------------------------------- small utilities
// Sort key of a singular value for the descending order of D: NaN ranks below every number, so
// that ranking by (key, index) is a permutation whatever the values are.
__device__ __forceinline__ float sigma_rank_key(float x) { return x == x ? x : -3.0e38f; }

// Position of entry `self` in the descending order of v[0..count) (ties: lower index first).
__device__ __forceinline__ int sigma_rank(const float* v, int count, int self) {
  const float k = sigma_rank_key(v[self]);
  int r = 0;
  for (int c = 0; c < count; ++c) {
    const float kc = sigma_rank_key(v[c]);
    r += (kc > k || (kc == k && c < self)) ? 1 : 0;
  }
  return r;
}
__host__ __device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace frsvt
