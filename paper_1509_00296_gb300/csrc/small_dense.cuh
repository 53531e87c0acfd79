// Block-level small dense linear algebra for Alg. 1 (device functions).
//
// These routines run inside one CTA (any blockDim that is a multiple of 32 and
// at least 64) and are used both by stand-alone single-CTA kernels and as the
// "tail" of a streaming pass, executed by the CTA that finishes its split-K
// reduction last.
//
// orth_block : orthonormal basis of the sketch, Alg. 1 steps 6, 10-11, 14.
//              Cholesky QR applied twice (CholeskyQR2): Gram matrix and Cholesky
//              with a pivot drop (s = min(l, rank)) in double-float arithmetic,
//              FP32 triangular solves.  Under range propagation the new block is
//              projected out of the propagated basis twice first (the partial
//              orthogonalization of step 10).  Only span(Q) matters (Prop. 1).
// core_block : singular values / vectors of B = Q^T A from B B^T = Z^T Z
//              (Z = A Q): double-float Cholesky R^T R = Z^T Z, FP32 one-sided Jacobi SVD
//              of R^T (the D and V of Alg. 1 steps 16-18), soft shrinkage,
//              M = U diag(S_tau(D) / D) U^T (Eq. 6: X = Z M Q^T), Rf = Q M and
//              the propagated basis Q~ = Q U[:, :keep] (step 21).
#pragma once
#include "common.cuh"
#include "state.cuh"

namespace frsvt {

// Shared-memory workspace of orth_block / core_block, carved from one buffer.
template <int LP>
struct SmallWs {
  df64* G;          // LP x LP (double-float)
  df64* R;          // LP x LP (double-float)
  double* gdiag;    // LP (spare)
  df64* gacc;       // gacc_n partial sums (double-float)
  float* Rf32;      // LP x LP  (FP32 copy of R / Jacobi columns)
  float* rinv;      // LP       (FP32 1 / R_jj, 0 for dropped)
  float* Cm;        // LP x LP  (projection coefficients / M)
  float* U;         // LP x LP
  float* vec;       // 4 * LP   (sigma, coef, ...)
  int* iv;          // 4 * LP   (dropped, perm, flags)
  float* W;         // ns x LP  (orth_block only)
  int gacc_n;
};

template <int LP>
__host__ __device__ constexpr size_t small_ws_fixed_bytes(int gacc_n) {
  return sizeof(double) * (2 * LP * LP + LP + gacc_n) + sizeof(float) * (3 * LP * LP + LP + 4 * LP) +
         sizeof(int) * 4 * LP;
}

template <int LP>
__host__ __device__ constexpr size_t small_ws_bytes(int64_t ns, int gacc_n) {
  return (small_ws_fixed_bytes<LP>(gacc_n) + 15) / 16 * 16 + static_cast<size_t>(ns) * LP * sizeof(float);
}

template <int LP>
__device__ SmallWs<LP> carve_small_ws(unsigned char* base, int gacc_n) {
  SmallWs<LP> w;
  w.gacc_n = gacc_n;
  df64* d = reinterpret_cast<df64*>(base);                  // 8-byte entries, same layout as double
  w.G = d;
  w.R = w.G + LP * LP;
  w.gdiag = reinterpret_cast<double*>(w.R + LP * LP);
  w.gacc = reinterpret_cast<df64*>(w.gdiag + LP);
  float* f = reinterpret_cast<float*>(w.gacc + gacc_n);
  w.Rf32 = f;
  w.rinv = w.Rf32 + LP * LP;
  w.Cm = w.rinv + LP;
  w.U = w.Cm + LP * LP;
  w.vec = w.U + LP * LP;
  w.iv = reinterpret_cast<int*>(w.vec + 4 * LP);
  w.W = reinterpret_cast<float*>(base + (small_ws_fixed_bytes<LP>(gacc_n) + 15) / 16 * 16);
  return w;
}

__device__ __forceinline__ void decode_pair_sym(int pr, int p, int& a, int& b) {
  a = 0;
  while (pr >= p - a) { pr -= p - a; ++a; }
  b = a + pr;
}

// G[a][b] = sum_i X[i][ca + a] * X[i][cb + b] for the (a, b) pairs requested, accumulated
// in double-float over the rows i < ns of X (row stride LP).  sym: a <= b < na (symmetric, both
// triangles written); otherwise a < na, b < nb.  Up to eight row groups split the rows (four
// independent chains each); their partial sums are added in double-float too: no FP64
// instruction runs here (GB300's FP64 pipe issues a warp instruction in many cycles).
// Block-wide; ends with __syncthreads.
template <int LP>
__device__ void block_inner(const float* X, int64_t ns, int ca, int cb, int na, int nb, bool sym, df64* G,
                            df64* gacc, int gacc_n) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int np = sym ? na * (na + 1) / 2 : na * nb;
  if (np == 0) { __syncthreads(); return; }
  int groups = gacc_n / np;
  if (groups > nt / np) groups = nt / np;
  if (groups > 8) groups = 8;
  if (groups < 1) groups = 1;
  for (int t = tid; t < np * groups; t += nt) {
    const int pr = t % np, g = t / np;
    int a, b;
    if (sym) decode_pair_sym(pr, na, a, b);
    else { a = pr / nb; b = pr % nb; }
    const float* xa = X + ca + a;
    const float* xb = X + cb + b;
    df64 acc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};   // 4 independent chains
    int64_t i = g;
    for (; i + 3 * groups < ns; i += 4 * groups) {
      float va[4], vb[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        va[u] = xa[(i + u * groups) * LP];
        vb[u] = xb[(i + u * groups) * LP];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) df64_add_prod(acc[u], va[u], vb[u]);
    }
    for (; i < ns; i += groups) df64_add_prod(acc[0], xa[i * LP], xb[i * LP]);
    gacc[t] = df_add(df_add(acc[0], acc[1]), df_add(acc[2], acc[3]));
  }
  __syncthreads();
  for (int pr = tid; pr < np; pr += nt) {
    int a, b;
    if (sym) decode_pair_sym(pr, na, a, b);
    else { a = pr / nb; b = pr % nb; }
    df64 v = gacc[pr];
    for (int g = 1; g < groups; ++g) v = df_add(v, gacc[g * np + pr]);
    G[a * LP + b] = v;
    if (sym) G[b * LP + a] = v;
  }
  __syncthreads();
}

// W (ns x LP, shared) <- [Qt[:, :keep] | Y[:, :l - keep] | 0] (global; Y is read through L2).
// Each thread issues U independent loads before its shared stores, so the copy costs one memory
// latency per U elements instead of one per element.
template <int LP, int U = 8>
__device__ void load_basis_block(float* W, int ns, int keep, int l, const float* Qt, const float* Y) {
  const int count = ns * LP, nt = blockDim.x;
  for (int e0 = threadIdx.x; e0 < count; e0 += U * nt) {
    float v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * nt;
      const int col = e % LP, i = e / LP;
      v[u] = 0.f;
      if (e < count) {
        if (col < keep) v[u] = Qt[e];
        else if (col < l) v[u] = __ldcg(Y + i * LP + (col - keep));
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * nt;
      if (e < count) W[e] = v[u];
    }
  }
}

// dst[e] = src[e], e < count (U loads in flight per thread).
template <int U = 8>
__device__ void block_copy(float* dst, const float* src, int count) {
  const int nt = blockDim.x;
  for (int e0 = threadIdx.x; e0 < count; e0 += U * nt) {
    float v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * nt;
      v[u] = (e < count) ? src[e] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * nt;
      if (e < count) dst[e] = v[u];
    }
  }
}

// Right-looking Cholesky G = R^T R (upper R) of the leading p x p block of the double-float
// G, by warp 0, with column drops: column j is dropped (row j of R zero, rinv[j] = 0) when its
// pivot is not above rank_tol * (original G_jj), when G_jj is below 1e-15 of the largest
// diagonal, or when it is not a finite positive number.  G is overwritten.  Returns via
// iv[0..p) the drop flags.  A non-finite diagonal of G (NaN or Inf met in the Gram reduction) is
// reported by OR-ing FRSVT_DEV_NONFINITE into *status (when given).  Block-wide (contains
// __syncthreads).
//
// The factorization runs in double-float arithmetic on the FP32 pipes (~48 significant bits):
// on GB300 every FP64 operation of this serial chain costs far more latency than the dozen
// FP32 operations of its double-float counterpart.  Lane b owns column b of the trailing
// block: at step j it forms R[j][b] and subtracts R[j][a] R[j][b] from G[a][b] for j < a <= b.
template <int LP>
__device__ void block_cholesky(SmallWs<LP>& w, int p, double rank_tol, uint32_t* status = nullptr) {
  static_assert(LP <= 32, "one lane per column");
  const int tid = threadIdx.x;
  df64* Gd = w.G;
  df64* Rd = w.R;
  int* dropped = w.iv;
  if (tid < 32) {
    const int lane = tid;
    const float tolf = static_cast<float>(rank_tol);
    const float g0 = (lane < p) ? Gd[lane * LP + lane].hi : 0.f;   // original diagonal
    float maxdiag = g0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) maxdiag = fmaxf(maxdiag, __shfl_xor_sync(0xffffffffu, maxdiag, o));
    if (__any_sync(0xffffffffu, lane < p && !isfinite(g0)) && lane == 0 && status != nullptr)
      atomicOr(status, kDevNonfinite);
    for (int j = 0; j < p; ++j) {
      const df64 d = Gd[j * LP + j];
      const float g0j = __shfl_sync(0xffffffffu, g0, j);
      const df64 gjb = (lane > j && lane < p) ? Gd[j * LP + lane] : df64{0.f, 0.f};
      const bool drop = !(d.hi > tolf * g0j) || !(g0j > 1e-15f * maxdiag) || !(d.hi > 1e-30f) || !(d.hi < 1e30f);
      df64 inv{0.f, 0.f}, rjj{0.f, 0.f};
      if (!drop) {
        inv = df_rsqrt_fma(d);
        rjj = df_mul(d, inv);
      }
      df64 rjb{0.f, 0.f};
      if (lane > j && lane < p && !drop) rjb = df_mul(gjb, inv);
      if (lane < LP) Rd[j * LP + lane] = (lane == j) ? rjj : rjb;
      if (lane == j) {
        dropped[j] = drop ? 1 : 0;
        w.rinv[j] = inv.hi;
      }
      __syncwarp();
      if (!drop && lane > j && lane < p) {
        // four independent updates at a time: every load first, then the fused multiply-subtracts,
        // then the stores (the dependent chain per column is what sets the pace of this warp)
        int a = j + 1;
        for (; a + 3 <= lane; a += 4) {
          df64 r4[4], g4[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            r4[u] = Rd[j * LP + a + u];
            g4[u] = Gd[(a + u) * LP + lane];
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) Gd[(a + u) * LP + lane] = df_fms(g4[u], r4[u], rjb);
        }
        for (; a <= lane; ++a) Gd[a * LP + lane] = df_fms(Gd[a * LP + lane], Rd[j * LP + a], rjb);
      }
      __syncwarp();
    }
    if (lane < LP) {
      for (int a = p; a < LP; ++a) Rd[a * LP + lane] = df64{0.f, 0.f};
      for (int a = 0; a < LP; ++a) w.Rf32[a * LP + lane] = (a < p) ? Rd[a * LP + lane].hi : 0.f;
      if (lane >= p) w.rinv[lane] = 0.f;
    }
  }
  __syncthreads();
}

// W[i][c0 + b] <- (W[i][c0 .. c0+p) R^{-1})_b for every row (forward substitution in FP32).
template <int LP>
__device__ void block_trsm_rows(SmallWs<LP>& w, float* W, int64_t ns, int c0, int p) {
  for (int64_t i = threadIdx.x; i < ns; i += blockDim.x) {
    float* row = W + i * LP + c0;
    float x[LP];                           // fully unrolled: the solution stays in registers
#pragma unroll
    for (int b = 0; b < LP; ++b) {
      if (b < p) {
        float acc = row[b];
#pragma unroll
        for (int a = 0; a < b; ++a) acc = fmaf(-x[a], w.Rf32[a * LP + b], acc);
        x[b] = acc * w.rinv[b];
      } else {
        x[b] = 0.f;
      }
    }
#pragma unroll
    for (int b = 0; b < LP; ++b)
      if (b < p) row[b] = x[b];
  }
  __syncthreads();
}

// Orthonormal basis (Alg. 1 steps 6 / 10-11 / 14).  W (ns x LP, shared) holds
// [Qt[:, :keep] | Y[:, :l - keep] | 0]; on return W holds Q.  Returns s (surviving columns).
// rp_res (optional, written by thread 0): the norm of the first new column once it has been
// projected out of the propagated basis, ||(I - Qt Qt^T) y_0|| (Prop. 4); -1 when keep = 0.
// passes = 2 is Cholesky QR2 (orthonormal to FP32 rounding); passes = 1 gives a basis of the
// same span whose orthogonality error is ~u kappa(Y), enough for a basis that only feeds the
// next power step (only its span matters there).
template <int LP>
__device__ int orth_block(SmallWs<LP>& w, int64_t ns, int keep, int l, double rank_tol, int passes,
                          float* rp_res = nullptr, uint32_t* status = nullptr) {
  float* W = w.W;
  const int p = l - keep;
  if (keep > 0 && p > 0) {
    for (int pass = 0; pass < 2; ++pass) {
      block_inner<LP>(W, ns, 0, keep, keep, p, false, w.G, w.gacc, w.gacc_n);
      for (int e = threadIdx.x; e < keep * p; e += blockDim.x) {
        const int a = e / p, b = e % p;
        w.Cm[a * LP + b] = w.G[a * LP + b].hi;
      }
      __syncthreads();
      for (int64_t i = threadIdx.x; i < ns; i += blockDim.x) {
        float qa[LP];
#pragma unroll
        for (int a = 0; a < LP; ++a) qa[a] = (a < keep) ? W[i * LP + a] : 0.f;
        for (int b = 0; b < p; ++b) {
          float acc = W[i * LP + keep + b];
#pragma unroll
          for (int a = 0; a < LP; ++a)
            if (a < keep) acc = fmaf(-qa[a], w.Cm[a * LP + b], acc);
          W[i * LP + keep + b] = acc;
        }
      }
      __syncthreads();
    }
  }
  int kept = 0;
  if (rp_res != nullptr && threadIdx.x == 0 && (keep == 0 || p == 0)) *rp_res = -1.f;
  for (int pass = 0; pass < passes && p > 0; ++pass) {
    block_inner<LP>(W, ns, keep, keep, p, p, true, w.G, w.gacc, w.gacc_n);
    if (pass == 0 && keep > 0 && rp_res != nullptr && threadIdx.x == 0) *rp_res = sqrtf(w.G[0].hi);
    block_cholesky<LP>(w, p, rank_tol, status);
    block_trsm_rows<LP>(w, W, ns, keep, p);
    kept = 0;
    for (int c = 0; c < p; ++c) kept += w.iv[c] ? 0 : 1;
    __syncthreads();
  }
  return keep + kept;
}

// Round-robin schedule: pair w of round rnd among N (even) indices.
__device__ __forceinline__ void rr_pair(int rnd, int w, int N, int& p, int& q) {
  if (w == 0) {
    p = N - 1;
    q = rnd;
  } else {
    p = (rnd + w) % (N - 1);
    q = (rnd - w + (N - 1)) % (N - 1);
  }
  if (p > q) { const int t = p; p = q; q = t; }
}

// SVD of B (B B^T = w.G = Z^T Z, LP x LP, leading l x l live), Alg. 1 steps 16-18: Cholesky
// R^T R = G, one-sided Jacobi on the columns of R^T.  On return w.vec[0..LP) holds sigma_b,
// w.U the left singular vectors (column b), w.iv[LP..2LP) the order by descending sigma (perm[k]
// = index of the k-th largest).  Returns the number of Jacobi sweeps.  Block-wide.
template <int LP>
__device__ int core_svd_block(SmallWs<LP>& w, int l, double rank_tol, int max_sweeps,
                              uint32_t* status = nullptr) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;
  float* Xt = w.Rf32;          // after the Cholesky: Xt[b * LP + a] = R[b][a] (columns of R^T)
  float* sig = w.vec;
  int* perm = w.iv + LP;
  int* flag = w.iv + 2 * LP;
  block_cholesky<LP>(w, l, rank_tol, status);
  const int N = (l + 1) / 2 * 2;   // even number of Jacobi columns covering the live ones
  const float tol = 1e-6f;
  int sweeps = 0;
  // One-sided Jacobi on the columns of R^T by one warp: lane c holds column c in registers and,
  // in round rnd of the round-robin schedule, meets partner (2 rnd - c) mod (N - 1) (lane rnd
  // meets N - 1).  Both lanes of a pair form alpha, beta, gamma with the same operations in
  // the same order, so they agree bit for bit on the rotation.
  if (warp == 0) {
    float x[LP];
#pragma unroll
    for (int a = 0; a < LP; ++a) x[a] = (lane < N) ? Xt[lane * LP + a] : 0.f;
    for (int sweep = 0; sweep < max_sweeps && N >= 2; ++sweep) {
      bool rotated = false;
      const int N1 = N - 1;
      for (int rnd = 0; rnd < N1; ++rnd) {
        int partner;
        if (lane == N1) partner = rnd;
        else if (lane == rnd) partner = N1;
        else {                                   // (2 rnd - lane) mod (N - 1), argument in [-(N - 2), 2N - 4]
          int v = 2 * rnd - lane;
          v += (v < 0) ? N1 : 0;
          v -= (v >= N1) ? N1 : 0;
          partner = v;
        }
        if (lane >= N) partner = lane;
        float y[LP];
#pragma unroll
        for (int a = 0; a < LP; ++a) y[a] = __shfl_sync(0xffffffffu, x[a], partner);
        const bool is_p = lane < partner;
        // own / partner squared norms and the inner product, two partial chains each
        float so0 = 0.f, so1 = 0.f, sp0 = 0.f, sp1 = 0.f, g0 = 0.f, g1 = 0.f;
#pragma unroll
        for (int a = 0; a < LP; a += 2) {
          so0 = fmaf(x[a], x[a], so0);
          so1 = fmaf(x[a + 1], x[a + 1], so1);
          sp0 = fmaf(y[a], y[a], sp0);
          sp1 = fmaf(y[a + 1], y[a + 1], sp1);
          g0 = fmaf(x[a], y[a], g0);
          g1 = fmaf(x[a + 1], y[a + 1], g1);
        }
        const float so = so0 + so1, sp = sp0 + sp1, gamma = g0 + g1;
        const float alpha = is_p ? so : sp, beta = is_p ? sp : so;  // column p, column q
        // rotation test |gamma| > tol sqrt(alpha beta) with hardware reciprocal square roots, and
        // the angle (Rutishauser's tan formula) with fast reciprocals: both lanes of a pair evaluate
        // the same expressions on the same operands, so they still agree bit for bit; the rotation
        // stays orthogonal to rounding through c = 1 / sqrt(1 + t^2), s = c t
        if (lane < N && partner != lane && alpha > 1e-30f && beta > 1e-30f && alpha < 1e30f && beta < 1e30f &&
            fabsf(gamma) * rsqrtf(alpha) * rsqrtf(beta) > tol) {
          const float zeta = __fdividef(beta - alpha, 2.f * gamma);
          const float az = fabsf(zeta);
          const float t = az < 1e18f ? copysignf(__fdividef(1.f, az + sqrtf(fmaf(zeta, zeta, 1.f))), zeta)
                                     : __fdividef(0.5f, zeta);
          const float c = rsqrtf(fmaf(t, t, 1.f));
          const float sy = is_p ? -(c * t) : (c * t);           // x_p' = c x_p - s x_q, x_q' = s x_p + c x_q
#pragma unroll
          for (int a = 0; a < LP; ++a) x[a] = fmaf(sy, y[a], c * x[a]);
          rotated = true;
        }
      }
      sweeps = sweep + 1;
      if (!__any_sync(0xffffffffu, rotated)) break;
    }
    if (lane < N)
#pragma unroll
      for (int a = 0; a < LP; ++a) Xt[lane * LP + a] = x[a];
    if (lane == 0) flag[1] = sweeps;
  }
  __syncthreads();
  sweeps = flag[1];
  if (tid < LP) {
    float s2 = 0.f;
    for (int a = 0; a < LP; ++a) s2 = fmaf(Xt[tid * LP + a], Xt[tid * LP + a], s2);
    sig[tid] = sqrtf(s2);
  }
  __syncthreads();
  for (int e = tid; e < LP * LP; e += nt) {
    const int a = e / LP, b = e % LP;
    w.U[e] = (sig[b] > 0.f) ? Xt[b * LP + a] / sig[b] : 0.f;
  }
  if (tid < LP) {
    int rank = 0;
    rank = sigma_rank(sig, LP, tid);
    perm[rank] = tid;
  }
  __syncthreads();
  return sweeps;
}

// Core of Alg. 1 steps 16-21 from the Gram w.G = Z^T Z (LP x LP, leading l x l live).
// Q: ns x LP (global).  Writes Rf = Q M (ns x LP), the first keep columns of Qt = Q U[:, perm],
// and the DevState fields r, keep, sigma, status, counter.  Block-wide.
template <int LP>
__device__ void core_block(SmallWs<LP>& w, const float* Q, int64_t ns, int l, float tau, int update_rp,
                           int advance_counter, float* Rf, float* Qt, DevState* dst, double rank_tol,
                           int max_sweeps) {
  const int tid = threadIdx.x, nt = blockDim.x;
  float* sig = w.vec;
  float* coef = w.vec + LP;
  int* perm = w.iv + LP;
  const int sweeps = core_svd_block<LP>(w, l, rank_tol, max_sweeps, &dst->status);
  const int pk = dst->partial_k;                   // partial SVT: the pk leading values stay
  if (tid < LP) {
    int rk = 0;
    for (int c = 0; c < LP; ++c) rk += (sig[c] > sig[tid] || (sig[c] == sig[tid] && c < tid)) ? 1 : 0;
    coef[tid] = (rk < pk && sig[tid] > 0.f) ? 1.f : ((sig[tid] > tau) ? (sig[tid] - tau) / sig[tid] : 0.f);
  }
  __syncthreads();
  float* M = w.Cm;
  for (int e = tid; e < LP * LP; e += nt) {
    const int a = e / LP, c = e % LP;
    float acc = 0.f;
    for (int b = 0; b < LP; ++b) acc = fmaf(w.U[a * LP + b] * coef[b], w.U[c * LP + b], acc);
    M[e] = acc;
  }
  int r = 0;
  for (int c = 0; c < LP; ++c) r += (coef[c] > 0.f) ? 1 : 0;
  // propagated columns: min(r, l - 2) for a fixed l; under the adaptive rank prediction of Eq. 7
  // the next sampling rate l' = min(r + (r < l ? a : ceil(rho n)), b) and min(r, l' - a) columns
  const int ap_a = dst->ap_a;
  const int l_next = ap_a > 0 ? min(r + (r < l ? ap_a : dst->ap_pn), dst->ap_b) : l;
  const int keep = update_rp ? max(0, min(r, l_next - (ap_a > 0 ? ap_a : 2))) : 0;
  __syncthreads();
  // Q~ columns in order: Up[a][k] = U[a][perm[k]] for k < keep (the Jacobi columns in Rf32 are dead)
  float* Up = w.Rf32;
  for (int e = tid; e < LP * LP; e += nt) {
    const int a = e / LP, k = e % LP;
    Up[e] = (k < keep) ? w.U[a * LP + perm[k]] : 0.f;
  }
  __syncthreads();
  // one row of Q per thread: Rf[i] = Q[i] M, then Q~[i] = Q[i] Up; the rows of M / Up are read as
  // float4 broadcasts and the result row stays in registers (the loop over a is only partly
  // unrolled so that the loads hoisted ahead of it do not exhaust the register file)
  for (int pass = 0; pass < (update_rp && keep > 0 ? 2 : 1); ++pass) {
    const float* F = pass == 0 ? M : Up;
    float* out = pass == 0 ? Rf : Qt;
    for (int64_t i = tid; i < ns; i += nt) {
      const float* qrow = Q + i * LP;
      float acc[LP];
#pragma unroll
      for (int k = 0; k < LP; ++k) acc[k] = 0.f;
#pragma unroll 4
      for (int a = 0; a < LP; ++a) {
        const float qa = qrow[a];
#pragma unroll
        for (int k4 = 0; k4 < LP / 4; ++k4) {
          const float4 f4 = reinterpret_cast<const float4*>(F + a * LP)[k4];
          acc[4 * k4] = fmaf(qa, f4.x, acc[4 * k4]);
          acc[4 * k4 + 1] = fmaf(qa, f4.y, acc[4 * k4 + 1]);
          acc[4 * k4 + 2] = fmaf(qa, f4.z, acc[4 * k4 + 2]);
          acc[4 * k4 + 3] = fmaf(qa, f4.w, acc[4 * k4 + 3]);
        }
      }
      if (pass == 0) {
#pragma unroll
        for (int k4 = 0; k4 < LP / 4; ++k4)
          reinterpret_cast<float4*>(out + i * LP)[k4] =
              make_float4(acc[4 * k4], acc[4 * k4 + 1], acc[4 * k4 + 2], acc[4 * k4 + 3]);
      } else {
#pragma unroll
        for (int k = 0; k < LP; ++k)
          if (k < keep) out[i * LP + k] = acc[k];
      }
    }
  }
  if (tid == 0) {
    dst->r = r;
    dst->sweeps = sweeps;
    if (update_rp) dst->keep = keep;
    if (update_rp && ap_a > 0) dst->l_cur = max(1, l_next);
    if (advance_counter) dst->counter += 1;
    if (sweeps >= max_sweeps) dst->status |= kDevNotConverged;
    bool finite = true;
    for (int c = 0; c < LP; ++c) {
      dst->sigma[c] = sig[perm[c]];
      finite = finite && isfinite(sig[c]);
    }
    for (int c = LP; c < kMaxL; ++c) dst->sigma[c] = 0.f;
    if (!finite) dst->status |= kDevNonfinite;
    dst->sigma1 = static_cast<double>(sig[perm[0]]);
  }
  __syncthreads();
}

}  // namespace frsvt
