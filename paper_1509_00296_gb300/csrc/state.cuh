// Device-resident state of one FRSVT handle and the kernel entry points of the
// FRSVT / iALM path.  Everything a kernel needs between launches lives in
// DevState so that a sequence of launches can be captured in a CUDA graph and
// replayed without host round trips.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace frsvt {

constexpr int kMaxL = 128;               // largest padded basis width (l_max <= 128)
constexpr uint64_t kCounterFromState = ~0ull;

struct DevState {
  double mu;            // iALM penalty of the current iteration
  double mu_bar;        // upper bound of mu
  double rho;           // growth factor of mu
  double lambda;        // weight of the l1 term
  double normO_F;       // ||O||_F
  double resid_ratio;   // ||O - L - S||_F / ||O||_F of the last step
  double init_scale;    // A0 = init_scale * O
  double sigma1;        // last spectral-norm estimate
  uint64_t counter;     // Omega stream index of the next SVT
  int32_t r;            // #{sigma > tau} of the last SVT
  int32_t s;            // basis columns kept by the last orthonormalisation
  int32_t keep;         // propagated basis columns for the next SVT
  int32_t iter;         // iALM iterations since rpca_init
  uint32_t status;      // sticky FRSVT_DEV_* bits
  int32_t sweeps;       // Jacobi sweeps of the last core SVD
  int32_t l_cur;        // sampling rate of the next SVT under adaptive rank prediction (Eq. 7)
  int32_t ap_a;         // Eq. 7: over-sampling a when r < l (0: prediction off)
  int32_t ap_pn;        // Eq. 7: ceil(rho n), the over-sampling when r >= l
  int32_t ap_b;         // Eq. 7: the bound b = ceil(gamma n) (<= the panel width)
  int32_t partial_k;    // leading singular values kept unshrunk (partial SVT, Table 6 Type B)
  float rp_res;         // Prop. 4: ||(I - Q~ Q~^T) y|| of the first new sample column of the last
                        // range-propagated sketch (-1: the last sketch had no propagated basis)
  float sigma[kMaxL];   // singular values of B of the last SVT, descending
};

// Device status bits (mirror of the FRSVT_DEV_* macros of frsvt.h).
constexpr uint32_t kDevRankDeficient = 1u << 0;
constexpr uint32_t kDevNotConverged = 1u << 1;
constexpr uint32_t kDevNonfinite = 1u << 2;
constexpr uint32_t kDevTimeout = 1u << 3;
constexpr uint32_t kDevBadProblem = 1u << 4;

// ------------------------------------------------------------------ launchers
// All launchers enqueue on `st` (cudaStream_t) and return the launch error.
// Sizes: A is m x n row-major (lda), n <= m; LP in {16, 32} is the padded
// basis width; l <= LP is the live width.

// part[split][j][k] = sum_{i in split} A[i, j] * B[i, k]  (B = Zl, or Omega when Zl == nullptr)
cudaError_t launch_short_cols(int LP, const float* A, int64_t m, int64_t n, int64_t lda,
                              const float* Zl, uint64_t seed, uint64_t counter_override,
                              const DevState* dst, float* part, int nsplit, int64_t rows_per_split,
                              cudaStream_t st);
// Y[e] = sum_s part[s][e] (compensated, fixed order), e < count
cudaError_t launch_reduce_parts(const float* part, int nsplit, int64_t count, float* Y, cudaStream_t st);
// Z[i, k] = sum_j A[i, j] Q[j, k]
cudaError_t launch_long_rows(int LP, const float* A, int64_t m, int64_t n, int64_t lda,
                             const float* Q, float* Z, int grid_cap, cudaStream_t st);
// one-time kernel attributes (dynamic shared memory limits); not a stream operation
cudaError_t prepare_pass_kernels(int smem_limit);
cudaError_t prepare_small_kernels(int smem_limit);
// Q = orth([Qt[:, :keep], Y[:, :l-keep]]) by block Gram-Schmidt + Cholesky QR (twice)
cudaError_t launch_orth(int LP, const float* Y, int64_t ns, int l, int use_rp, const float* Qt,
                        float* Q, DevState* dst, double rank_tol, cudaStream_t st);
// gpart[split] = (df64) Z[rows of split]^T Z[rows of split]
cudaError_t launch_gram_long(int LP, const float* Z, int64_t m, float2* gpart, int gsplit,
                             cudaStream_t st);
// l x l core: Cholesky of sum(gpart), one-sided Jacobi SVD, shrinkage, Rf = Q M, Qt = Q U[:, :keep]
cudaError_t launch_core(int LP, const float2* gpart, int gsplit, const float* Q, int64_t ns, int l,
                        float tau_host, int tau_from_mu, int update_rp, int advance_counter,
                        float* Rf, float* Qt, DevState* dst, double rank_tol, int max_sweeps,
                        cudaStream_t st);
// X[i, j] = sum_k Z[i, k] Rf[j, k]
cudaError_t launch_recon(int LP, const float* Z, const float* Rf, int64_t m, int64_t n, float* X,
                         int64_t ldx, int nsplit, int64_t rows_per_split, cudaStream_t st);
// fused iALM update with the reconstruction; rpart[cta] = df64 partial of ||O - L - S'||^2
cudaError_t launch_alm(int LP, const float* Z, const float* Rf, const float* O, float* S, float* A,
                       int64_t m, int64_t n, int64_t ld, float* L, int64_t ldl, const DevState* dst,
                       float2* rpart, int nsplit, int64_t rows_per_split, cudaStream_t st);
cudaError_t launch_alm_finish(const float2* rpart, int count, DevState* dst, cudaStream_t st);
// rpca_init helpers
cudaError_t launch_absmax_sumsq(const float* O, int64_t m, int64_t n, int64_t ld, float* pmax,
                                float2* psum, int nblk, cudaStream_t st);
cudaError_t launch_init_scalars(const float* pmax, const float2* psum, int nblk, double normO2_host,
                                double lambda, double rho, double mu_bar_factor, DevState* dst,
                                cudaStream_t st);
cudaError_t launch_init_state(const float* O, float* S, float* A, int64_t m, int64_t n, int64_t ld,
                              const DevState* dst, cudaStream_t st);
// debug
cudaError_t launch_debug_omega(float* out, int64_t rows, int cols, uint64_t seed, uint64_t stream,
                               uint64_t problem, cudaStream_t st);
// one CTA waits, with at most spin_limit polls, on an mbarrier that nothing arrives at, and ORs
// kDevTimeout into dst->status when the wait gives up (the path every bounded wait takes)
cudaError_t launch_debug_wait_timeout(uint32_t spin_limit, DevState* dst, cudaStream_t st);
cudaError_t launch_debug_philox(uint64_t* out, int64_t rows, int blocks, uint64_t seed,
                                uint64_t stream, uint64_t problem, cudaStream_t st);

}  // namespace frsvt
