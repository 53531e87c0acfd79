// Elementwise steps of the unrolled inexact-ALM RPCA (the differentiable workload) and their
// adjoints.  Step k of the unrolled iteration (the iALM of Sec. 4.1 with a learnable threshold
// tau_k and penalty mu_k per step):
//
//   A_k = O - S_{k-1} + Y_{k-1} / mu_k
//   L_k = FRSVT_{tau_k}(A_k)                                  (Alg. 1; frsvt_svt_save)
//   T_k = O - L_k + Y_{k-1} / mu_k
//   S_k = shrink_{lam / mu_k}(T_k)
//   Y_k = Y_{k-1} + mu_k (O - L_k - S_k)
//
// k_ur_post forms S_k, Y_k and A_{k+1} from L_k in one pass.  The reverse pass of a step, with the
// cotangents Sb = dS_k and Yb = dY_k flowing back from step k + 1 and Lin = dL_k from the loss:
//
//   St   = Sb - mu_k Yb                          (S_k feeds Y_k as well)
//   Tb   = St [|T_k| > lam / mu_k]               (shrinkage)
//   Lb   = Lin - mu_k Yb - Tb                    (-> the FRSVT adjoint, which returns Ab = dA_k)
//   dY_{k-1} = Yb + (Tb + Ab) / mu_k,   dS_{k-1} = -Ab
//   dmu_k = sum Yb (O - L_k - S_k) + sum St sgn(T_k) [|T_k| > lam / mu_k] lam / mu_k^2
//           - sum (Tb + Ab) Y_{k-1} / mu_k^2
//
// k_ur_bwd_post does everything up to Lb (and the first two sums of dmu_k), k_ur_bwd_pre the rest
// after the FRSVT adjoint.  Sums are double per CTA, added in CTA order by k_ur_sum (deterministic).
// Matrices are m x n row-major with leading dimension ld; float4 accesses need ld % 4 == 0 and
// 16-byte aligned bases, which the host checks.
#include <cstdint>

#include "common.cuh"
#include "state.cuh"

namespace frsvt {

namespace {

constexpr int kUThr = 256;

__device__ __forceinline__ float shrinkf(float t, float th) {
  const float a = fabsf(t) - th;
  return a > 0.f ? copysignf(a, t) : 0.f;
}

__device__ __forceinline__ void block_sum_store(double v, double* out) {
  __shared__ double red[kUThr / 32];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kUThr / 32; ++w) s += red[w];
    *out = s;
  }
}

// A = O - S + Y / mu (S == nullptr: S = 0); Y == nullptr: Y = ys O (the initial multiplier).
__global__ void __launch_bounds__(kUThr) k_ur_pre(const float* __restrict__ O, const float* __restrict__ S,
                                                  const float* __restrict__ Y, float ys, float* __restrict__ A,
                                                  int64_t m, int64_t n4, int64_t ld, float mu) {
  const float rmu = 1.f / mu;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < m * n4;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t off = (e / n4) * ld + 4 * (e % n4);
    const float4 o = *reinterpret_cast<const float4*>(O + off);
    const float4 s = S ? *reinterpret_cast<const float4*>(S + off) : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 y = Y ? *reinterpret_cast<const float4*>(Y + off) : make_float4(ys * o.x, ys * o.y, ys * o.z, ys * o.w);
    *reinterpret_cast<float4*>(A + off) =
        make_float4(o.x - s.x + y.x * rmu, o.y - s.y + y.y * rmu, o.z - s.z + y.z * rmu, o.w - s.w + y.w * rmu);
  }
}

// From L_k: S_k, Y_k (Yout may alias nothing that is read) and, when An != nullptr, A_{k+1} with mu_next.
__global__ void __launch_bounds__(kUThr) k_ur_post(const float* __restrict__ O, const float* __restrict__ L,
                                                   const float* __restrict__ Y, float ys, float* __restrict__ Sout,
                                                   float* __restrict__ Yout, float* __restrict__ An, int64_t m,
                                                   int64_t n4, int64_t ld, float mu, float mu_next, float lam) {
  const float rmu = 1.f / mu, th = lam / mu, rmn = 1.f / mu_next;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < m * n4;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t off = (e / n4) * ld + 4 * (e % n4);
    const float4 o4 = *reinterpret_cast<const float4*>(O + off);
    const float4 l4 = *reinterpret_cast<const float4*>(L + off);
    const float4 y4 = Y ? *reinterpret_cast<const float4*>(Y + off)
                        : make_float4(ys * o4.x, ys * o4.y, ys * o4.z, ys * o4.w);
    const float o[4] = {o4.x, o4.y, o4.z, o4.w}, l[4] = {l4.x, l4.y, l4.z, l4.w}, y[4] = {y4.x, y4.y, y4.z, y4.w};
    float so[4], yo[4], an[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float t = o[u] - l[u] + y[u] * rmu;
      so[u] = shrinkf(t, th);
      yo[u] = y[u] + mu * (o[u] - l[u] - so[u]);
      an[u] = o[u] - so[u] + yo[u] * rmn;
    }
    *reinterpret_cast<float4*>(Sout + off) = make_float4(so[0], so[1], so[2], so[3]);
    *reinterpret_cast<float4*>(Yout + off) = make_float4(yo[0], yo[1], yo[2], yo[3]);
    if (An) *reinterpret_cast<float4*>(An + off) = make_float4(an[0], an[1], an[2], an[3]);
  }
}

// Reverse of the shrinkage and the multiplier update (see the file header).  In: O, L_k, Y_{k-1}
// (Y == nullptr: ys O), Sb (nullable: 0), Yb (nullable: 0), Lin (nullable: 0).  Out: Lb, Yb2 =
// Yb + Tb / mu (in place over Yb allowed), Tb saved into Tbo for k_ur_bwd_pre; part[cta] = the
// first two sums of dmu_k.
__global__ void __launch_bounds__(kUThr) k_ur_bwd_post(const float* __restrict__ O, const float* __restrict__ L,
                                                       const float* __restrict__ Y, float ys, const float* Sb,
                                                       const float* Yb, const float* __restrict__ Lin,
                                                       float* __restrict__ Lb, float* Yb2, float* __restrict__ Tbo,
                                                       int64_t m, int64_t n4, int64_t ld, float mu, float lam,
                                                       double* __restrict__ part) {
  const float rmu = 1.f / mu, th = lam / mu, c2 = lam / (mu * mu);
  double acc = 0.0;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < m * n4;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t off = (e / n4) * ld + 4 * (e % n4);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 o4 = *reinterpret_cast<const float4*>(O + off);
    const float4 l4 = *reinterpret_cast<const float4*>(L + off);
    const float4 y4 = Y ? *reinterpret_cast<const float4*>(Y + off)
                        : make_float4(ys * o4.x, ys * o4.y, ys * o4.z, ys * o4.w);
    const float4 sb4 = Sb ? *reinterpret_cast<const float4*>(Sb + off) : z4;
    const float4 yb4 = Yb ? *reinterpret_cast<const float4*>(Yb + off) : z4;
    const float4 li4 = Lin ? *reinterpret_cast<const float4*>(Lin + off) : z4;
    const float o[4] = {o4.x, o4.y, o4.z, o4.w}, l[4] = {l4.x, l4.y, l4.z, l4.w}, y[4] = {y4.x, y4.y, y4.z, y4.w};
    const float sb[4] = {sb4.x, sb4.y, sb4.z, sb4.w}, yb[4] = {yb4.x, yb4.y, yb4.z, yb4.w};
    const float li[4] = {li4.x, li4.y, li4.z, li4.w};
    float lb[4], y2[4], tb[4];
    float a = 0.f;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float t = o[u] - l[u] + y[u] * rmu;
      const bool on = fabsf(t) > th;
      const float s = on ? copysignf(fabsf(t) - th, t) : 0.f;
      const float st = sb[u] - mu * yb[u];
      tb[u] = on ? st : 0.f;
      lb[u] = li[u] - mu * yb[u] - tb[u];
      y2[u] = yb[u] + tb[u] * rmu;
      a = fmaf(yb[u], o[u] - l[u] - s, a);
      if (on) a = fmaf(st, copysignf(c2, t), a);
    }
    acc += static_cast<double>(a);
    *reinterpret_cast<float4*>(Lb + off) = make_float4(lb[0], lb[1], lb[2], lb[3]);
    *reinterpret_cast<float4*>(Yb2 + off) = make_float4(y2[0], y2[1], y2[2], y2[3]);
    *reinterpret_cast<float4*>(Tbo + off) = make_float4(tb[0], tb[1], tb[2], tb[3]);
  }
  block_sum_store(acc, part + blockIdx.x);
}

// After the FRSVT adjoint returned Ab = dA_k: dS_{k-1} = -Ab, dY_{k-1} = Yb2 + Ab / mu (in place),
// part[cta] = -sum (Tb + Ab) Y_{k-1} / mu^2.
__global__ void __launch_bounds__(kUThr) k_ur_bwd_pre(const float* __restrict__ O, const float* __restrict__ Y,
                                                      float ys, const float* __restrict__ Ab,
                                                      const float* __restrict__ Tb, float* __restrict__ Sbo,
                                                      float* __restrict__ Yb2, int64_t m, int64_t n4, int64_t ld,
                                                      float mu, double* __restrict__ part) {
  const float rmu = 1.f / mu, c = -1.f / (mu * mu);
  double acc = 0.0;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < m * n4;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t off = (e / n4) * ld + 4 * (e % n4);
    const float4 o4 = *reinterpret_cast<const float4*>(O + off);
    const float4 y4 = Y ? *reinterpret_cast<const float4*>(Y + off)
                        : make_float4(ys * o4.x, ys * o4.y, ys * o4.z, ys * o4.w);
    const float4 a4 = *reinterpret_cast<const float4*>(Ab + off);
    const float4 t4 = *reinterpret_cast<const float4*>(Tb + off);
    const float4 b4 = *reinterpret_cast<const float4*>(Yb2 + off);
    acc += static_cast<double>(c * ((t4.x + a4.x) * y4.x + (t4.y + a4.y) * y4.y + (t4.z + a4.z) * y4.z +
                                    (t4.w + a4.w) * y4.w));
    *reinterpret_cast<float4*>(Sbo + off) = make_float4(-a4.x, -a4.y, -a4.z, -a4.w);
    *reinterpret_cast<float4*>(Yb2 + off) =
        make_float4(b4.x + a4.x * rmu, b4.y + a4.y * rmu, b4.z + a4.z * rmu, b4.w + a4.w * rmu);
  }
  block_sum_store(acc, part + blockIdx.x);
}

// out[0] (+)= sum of part[0 .. count) in index order (one thread: count is a few hundred).
__global__ void k_ur_sum(const double* __restrict__ part, int count, float* __restrict__ out, int accumulate) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int i = 0; i < count; ++i) s += part[i];
  *out = accumulate ? static_cast<float>(static_cast<double>(*out) + s) : static_cast<float>(s);
}

// *out += *in (one float, stream-ordered; sums the FRSVT adjoints' dtau over the batch).
__global__ void k_ur_addf(const float* __restrict__ in, float* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *out += *in;
}

__global__ void k_ur_addv(const float* __restrict__ in, float* __restrict__ out, int count) {
  for (int i = threadIdx.x; i < count; i += blockDim.x) out[i] += in[i];
}

int ur_grid(int64_t m, int64_t n4, int sms) {
  const int64_t want = (m * n4 + kUThr - 1) / kUThr;
  const int64_t cap = 4LL * sms;
  return static_cast<int>(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace

int unrolled_grid(int64_t m, int64_t n, int sms) { return ur_grid(m, (n + 3) / 4, sms); }

cudaError_t launch_ur_pre(const float* O, const float* S, const float* Y, float ys, float* A, int64_t m, int64_t n,
                          int64_t ld, float mu, int grid, cudaStream_t st) {
  k_ur_pre<<<grid, kUThr, 0, st>>>(O, S, Y, ys, A, m, n / 4, ld, mu);
  return cudaGetLastError();
}

cudaError_t launch_ur_post(const float* O, const float* L, const float* Y, float ys, float* S, float* Yout, float* An,
                           int64_t m, int64_t n, int64_t ld, float mu, float mu_next, float lam, int grid,
                           cudaStream_t st) {
  k_ur_post<<<grid, kUThr, 0, st>>>(O, L, Y, ys, S, Yout, An, m, n / 4, ld, mu, mu_next, lam);
  return cudaGetLastError();
}

cudaError_t launch_ur_bwd_post(const float* O, const float* L, const float* Y, float ys, const float* Sb,
                               const float* Yb, const float* Lin, float* Lb, float* Yb2, float* Tb, int64_t m,
                               int64_t n, int64_t ld, float mu, float lam, double* part, int grid, cudaStream_t st) {
  k_ur_bwd_post<<<grid, kUThr, 0, st>>>(O, L, Y, ys, Sb, Yb, Lin, Lb, Yb2, Tb, m, n / 4, ld, mu, lam, part);
  return cudaGetLastError();
}

cudaError_t launch_ur_bwd_pre(const float* O, const float* Y, float ys, const float* Ab, const float* Tb, float* Sb,
                              float* Yb2, int64_t m, int64_t n, int64_t ld, float mu, double* part, int grid,
                              cudaStream_t st) {
  k_ur_bwd_pre<<<grid, kUThr, 0, st>>>(O, Y, ys, Ab, Tb, Sb, Yb2, m, n / 4, ld, mu, part);
  return cudaGetLastError();
}

cudaError_t launch_ur_addf(const float* in, float* out, cudaStream_t st) {
  k_ur_addf<<<1, 32, 0, st>>>(in, out);
  return cudaGetLastError();
}

cudaError_t launch_ur_addv(const float* in, float* out, int count, cudaStream_t st) {
  k_ur_addv<<<1, 256, 0, st>>>(in, out, count);
  return cudaGetLastError();
}

cudaError_t launch_ur_sum(const double* part, int count, float* out, int accumulate, cudaStream_t st) {
  k_ur_sum<<<1, 32, 0, st>>>(part, count, out, accumulate);
  return cudaGetLastError();
}

}  // namespace frsvt
