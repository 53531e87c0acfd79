/*
 * frsvt.h -- C ABI of libfrsvt.so: fast randomized singular value thresholding
 * (FRSVT) and robust PCA by the inexact augmented Lagrange multiplier method,
 * on one NVIDIA GB300 (sm_103a).
 *
 * Method: T.-H. Oh, Y. Matsushita, Y.-W. Tai, I. S. Kweon, "Fast Randomized
 * Singular Value Thresholding for Low-rank Optimization", arXiv:1509.00296.
 *   - SVT operator S_tau(A) = U S_tau(Sigma) V^T          (Def. 1, Eq. 3)
 *   - reduction S_tau(QB) = Q S_tau(B), Q orthonormal      (Prop. 1, Eq. 4)
 *   - FRSVT with range propagation and power iterations    (Alg. 1, Sec. 2.1-2.2, Eq. 6)
 *   - RPCA host loop (inexact ALM)                         (Sec. 4.1, Robust PCA test)
 *
 * Conventions for every entry point:
 *   - Matrices are row-major float32 in DEVICE memory owned by the caller, with
 *     a leading dimension (row stride, in elements) ld >= number of columns.
 *     Base pointers must be 16-byte aligned and ld a multiple of 4, otherwise
 *     the call returns FRSVT_ERR_INVALID_ARG (no silent copy is made).
 *   - Work is enqueued asynchronously on the handle's CUDA stream; no call
 *     synchronizes unless its description says so.  Errors found on the host
 *     are returned at once; errors found by kernels are OR-ed into a sticky
 *     device status word read (and cleared) by frsvt_get_info().
 *   - The handle owns all scratch memory; it is allocated once by
 *     frsvt_create() for the largest sizes given in frsvt_config.  No other
 *     call allocates.
 *   - Orientation: the orthonormal basis Q of Alg. 1 is kept on the shorter
 *     side of A (Sec. 2.5 asks for the transposed problem when needed).  The
 *     Gaussian test matrix Omega therefore has max(m, n) rows.  The wide-basis
 *     handle (cfg.l_max > 32) serves both orientations: for m < n its two
 *     passes over A swap roles (no copy of A is made).  The narrow-basis handle
 *     (cfg.l_max <= 32) serves m >= n; m < n returns FRSVT_ERR_UNSUPPORTED.
 */
#ifndef FRSVT_H_
#define FRSVT_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum frsvt_status {
  FRSVT_OK = 0,
  FRSVT_ERR_INVALID_ARG = 1,     /* bad pointer, size, alignment or parameter */
  FRSVT_ERR_UNSUPPORTED = 2,     /* valid request this build does not serve */
  FRSVT_ERR_ALLOC = 3,           /* device allocation failed in frsvt_create */
  FRSVT_ERR_CUDA = 4,            /* a CUDA runtime call or kernel launch failed */
  FRSVT_ERR_RANK_DEFICIENT = 5,  /* device bit, informational: basis size s < l */
  FRSVT_ERR_NOT_CONVERGED = 6,   /* device bit: a Jacobi solve hit max sweeps */
  FRSVT_ERR_NONFINITE = 7        /* device bit: NaN or Inf met in a reduction */
} frsvt_status;

/* Device status word bits (frsvt_info.device_status). */
#define FRSVT_DEV_RANK_DEFICIENT (1u << 0)
#define FRSVT_DEV_NOT_CONVERGED  (1u << 1)
#define FRSVT_DEV_NONFINITE      (1u << 2)
#define FRSVT_DEV_TIMEOUT        (1u << 3)   /* a bounded wait on an asynchronous copy gave up */
#define FRSVT_DEV_BAD_PROBLEM    (1u << 4)   /* a batched problem had an unsupported size and was skipped */

/* Precision of the passes over A (Alg. 1 steps 5, 9, 14, 16).  FRSVT_PREC_BF16: the handle keeps
 * a BF16 shadow of A (written by rpca_init and by every rpca_ialm_step epilogue, converted by
 * frsvt_svt); the sketch and the first q - 1 power steps read the shadow (BF16 operands, FP32
 * accumulation), the last power step and the projection stay FP32-accurate (the "residual"
 * step that wins the accuracy back).  With cfg.l_max <= 32 BF16 is served for n <= 256.
 * FRSVT_PREC_FP8 (cfg.l_max > 32 only): an E4M3 shadow with one power-of-two scale per 128 x 128
 * tile of A (the smallest with max|A_tile| / scale <= 448), quantized at the start of every SVT,
 * for the same passes.  frsvt_create returns FRSVT_ERR_UNSUPPORTED for a precision it does not
 * build. */
typedef enum frsvt_precision {
  FRSVT_PREC_FP32 = 0,           /* float32 data, FP32-accurate passes */
  FRSVT_PREC_BF16 = 1,           /* BF16 shadow for the sketch and the early power steps */
  FRSVT_PREC_FP8 = 2             /* E4M3 shadow, one power-of-two scale per 128 x 128 tile of A, for the
                                    sketch and the early power steps (cfg.l_max > 32 only) */
} frsvt_precision;

#define FRSVT_CFG_ADJOINT 1      /* allocate the workspace of frsvt_svt_save / frsvt_backward */
#define FRSVT_CFG_ORTH_LAST 2    /* orthonormalise only after the last power step (Sec. 2.5): the
                                    intermediate steps of Alg. 1 step 14 pass A A^T Q on unnormalised.
                                    X is the same in exact arithmetic (only span(Q) enters it); honoured
                                    by frsvt_svt and rpca_ialm_step on the wide basis and on the FP32
                                    tensor-core path of the narrow basis (both scale the unnormalised
                                    step by powers of two, exactly), the other paths orthonormalise
                                    every step; frsvt_spectral_norm always orthonormalises. */

typedef struct frsvt_config {
  int64_t m_max;                 /* largest row count served by the handle */
  int64_t n_max;                 /* largest column count served by the handle */
  int32_t l_max;                 /* largest oversampled rank l = k + p, 1..128 (see frsvt_create) */
  int32_t q;                     /* power iterations eta (Alg. 1 steps 13-15), >= 0 */
  int32_t range_prop;            /* 1: range propagation between calls (Sec. 2.1) */
  int32_t precision;             /* frsvt_precision */
  uint64_t seed;                 /* Philox4x64-10 key of Omega */
  int32_t max_jacobi_sweeps;     /* cap of the l x l Jacobi SVD (<= 0: 30) */
  int32_t flags;                 /* FRSVT_CFG_* bits (other bits: FRSVT_ERR_INVALID_ARG) */
  double rank_tol;               /* relative pivot cut of the Cholesky QR (<= 0: 1e-12) */
  int32_t problem_streams;       /* 0 or 1: one stream; 2..16 (with FRSVT_CFG_ADJOINT): frsvt_create
                                    also makes that many child handles, each with its own stream and
                                    workspace, and rpca_unrolled_forward / rpca_unrolled_backward run
                                    the batch's problems on them concurrently (problem b on child
                                    b mod problem_streams), joined back into the handle's stream */
} frsvt_config;

typedef struct frsvt_info {
  int32_t r;                     /* #{sigma_i > tau} of the last SVT */
  int32_t s;                     /* basis size used by the last SVT (<= l) */
  int32_t keep;                  /* propagated basis columns for the next call */
  uint32_t device_status;        /* sticky FRSVT_DEV_* bits, cleared by the read */
  uint64_t counter;              /* Omega stream index the next SVT will use */
  int32_t alm_iter;              /* iALM iterations done since rpca_init */
  int32_t sweeps;                /* Jacobi sweeps of the last l x l core SVD (Alg. 1 step 18) */
  double mu;                     /* iALM penalty mu for the next iteration */
  double residual;               /* ||O - L - S||_F / ||O||_F of the last iALM step */
  float rp_residual;             /* Prop. 4 / Eq. 14: ||(I - Q~ Q~^T) y|| for the first new sample
                                    column y = A^T omega of the last range-propagated sketch, a
                                    by-product of its Gram-Schmidt step; alpha sqrt(2/pi) times it
                                    bounds ||(I - Q~ Q~^T) A||_2 >= sigma_{k+1}(A) with probability
                                    >= 1 - 1/alpha.  -1 when that sketch had no propagated basis
                                    (and before any sketch with range propagation). */
  int32_t reserved;
} frsvt_info;

typedef struct frsvt_handle frsvt_handle;

/*
 * Create a handle.  cfg sizes the workspace; stream is a cudaStream_t (NULL:
 * the legacy default stream).  Allocates all device scratch memory.
 * cfg.l_max <= 32 builds the narrow-basis handle (16- or 32-column panels);
 * 32 < cfg.l_max <= 128 the wide-basis handle (128-column panels, any short
 * side, grid-wide Cholesky QR and core), which serves frsvt_svt,
 * frsvt_svt_factors, frsvt_spectral_norm, rpca_init and rpca_ialm_step, with
 * range propagation and FRSVT_CFG_ORTH_LAST; for it FRSVT_CFG_ADJOINT and
 * m_max >= 2^31 return FRSVT_ERR_UNSUPPORTED, and the batched WSVT and debug
 * entry points return FRSVT_ERR_UNSUPPORTED.  The wide handle computes no
 * Prop. 4 residual (frsvt_info.rp_residual stays -1).
 * Returns FRSVT_ERR_INVALID_ARG for out-of-range sizes, FRSVT_ERR_ALLOC if
 * the device allocation fails.
 */
frsvt_status frsvt_create(frsvt_handle** h, const frsvt_config* cfg, void* stream);

/* Destroy a handle and free its workspace (synchronizes its stream). */
frsvt_status frsvt_destroy(frsvt_handle* h);

/* Change the stream later calls are enqueued on. */
frsvt_status frsvt_set_stream(frsvt_handle* h, void* stream);

/*
 * Forget the propagated basis (Alg. 1 then takes its non-propagating branch)
 * and set the Omega stream index of the next SVT.  Enqueued on the stream.
 */
frsvt_status frsvt_reset(frsvt_handle* h, uint64_t counter);

/*
 * X = FRSVT_tau(A) (Alg. 1): Gaussian sketch of l columns (or, with range
 * propagation, the propagated basis plus l - keep new columns), q power
 * iterations with re-orthonormalisation, projection B = Q^T A, SVD of B and
 * soft shrinkage of its singular values (Eq. 6).  A is m x n (lda), X is
 * m x n (ldx); X may not alias A.  l is clamped to min(m, n).  The Omega
 * stream index advances by one per call.  1 <= l <= cfg.l_max.
 */
frsvt_status frsvt_svt(frsvt_handle* h, const float* A, int64_t m, int64_t n, int64_t lda,
                       float tau, int32_t l, float* X, int64_t ldx);

/*
 * The same FRSVT as frsvt_svt, returned in factored form instead of forming X (Eq. 6 with the
 * small factors folded in):  X = U V^T  with U (m x l, ldu) and V (n x l, ldv).  For m >= n,
 * U = A Q and V = Q M; for m < n (wide-basis handles), U = Q M and V = A^T Q; Q is the orthonormal
 * basis of Alg. 1 on the short side and M = V_B diag(f(sigma) / sigma) V_B^T the l x l core
 * (f the soft threshold, or the partial threshold after frsvt_set_partial).  Columns of U and V
 * past the basis size are zero.  r (nullable, device memory) receives #{sigma_i > tau}.  Under
 * adaptive rank prediction U and V get the panel width (16 or 32) of columns, so ldu and ldv must
 * be at least that.  Same arguments, limits, side effects (Omega counter, propagated basis) and
 * errors as frsvt_svt; U, V and r are caller-owned device memory; asynchronous.
 */
frsvt_status frsvt_svt_factors(frsvt_handle* h, const float* A, int64_t m, int64_t n, int64_t lda,
                               float tau, int32_t l, float* U, int64_t ldu, float* V, int64_t ldv,
                               int32_t* r);

/*
 * Largest singular value of A by block power iteration (the range finder of
 * Sec. 2.1 with `iters` power steps and l = cfg.l_max columns).  Synchronizes
 * and writes the value to *sigma1.  Does not touch the propagated basis or
 * the Omega counter.
 */
frsvt_status frsvt_spectral_norm(frsvt_handle* h, const float* A, int64_t m, int64_t n,
                                 int64_t lda, int32_t iters, double* sigma1);

/*
 * Robust PCA by inexact ALM (Sec. 4.1), state kept as (S, A) with
 * A = O - S + Y/mu (the dual Y is mu (A - O + S)).
 *
 * rpca_init: S := 0, A := O + Y0/mu0 with Y0 = O / max(||O||_2, ||O||_inf/lambda),
 * mu0 = 1.25/||O||_2 (||O||_2 by frsvt_spectral_norm with power_iters steps
 * when normO2 <= 0, else the given value), mu_bar = mu_bar_factor * mu0.
 * Resets the propagated basis and sets the Omega counter to 0.  Synchronizes.
 */
frsvt_status rpca_init(frsvt_handle* h, const float* O, float* S, float* A,
                       int64_t m, int64_t n, int64_t ld, double lambda, double rho,
                       double mu_bar_factor, double normO2, int32_t power_iters);

/*
 * One inexact-ALM iteration with an FRSVT of l columns:
 *   L  = FRSVT_{1/mu}(A)
 *   S' = shrink_{lambda/mu}(A + S - L)
 *   A' = O - S' + (mu/mu') (A + S - L - S'),  mu' = min(rho mu, mu_bar)
 * and ||O - L - S'||_F / ||O||_F is recorded on the device.  L (nullable,
 * ldl) receives the low-rank iterate when given; otherwise L is never
 * materialised.  O, S, A share the leading dimension ld.  When residual is not
 * NULL the call synchronizes and writes ||O - L - S'||_F / ||O||_F there.
 * The first call with a given (O, S, A, m, n, ld, l, L, ldl) captures the
 * iteration's kernels into a CUDA graph on a stream private to the handle;
 * later calls with the same arguments replay it on the handle's stream (the
 * iteration's state lives on the device); the graphs of the four most
 * recently used argument tuples are kept.  rpca_init, frsvt_reset,
 * frsvt_set_stream, frsvt_set_rank_prediction and frsvt_set_partial retire
 * the graphs.  While the handle's stream is being captured by the caller, or
 * with phase timing on, the kernels are launched directly.
 */
frsvt_status rpca_ialm_step(frsvt_handle* h, const float* O, float* S, float* A,
                            int64_t m, int64_t n, int64_t ld, int32_t l,
                            float* L, int64_t ldl, double* residual);

/* Synchronize the handle's stream, then report (and clear) the device state. */
frsvt_status frsvt_get_info(frsvt_handle* h, frsvt_info* info);

/* Copy the singular values D of the last SVT (descending, s of them) to host memory. */
frsvt_status frsvt_get_sigma(frsvt_handle* h, float* sigma_host, int32_t capacity, int32_t* count);

/*
 * Adaptive rank prediction (Sec. 2.3, Eq. 7).  From the next frsvt_svt / rpca_init on, the
 * sampling rate of each SVT is chosen on the device from the previous one: with r the number of
 * singular values above the threshold and l the last sampling rate,
 *     l' = min(r + p, b),  p = a if r < l, else ceil(rho n),  b = ceil(gamma n),
 * n the short side of the problem; the first SVT uses l_0 = ceil(0.1 b), and the propagated basis
 * keeps min(r, l' - a) columns (so that at least a new Gaussian columns are drawn).  The `l`
 * argument of later frsvt_svt / rpca_ialm_step calls is then ignored.  Requires range
 * propagation, FP32 precision, cfg.l_max <= 32 and the tensor-core path (short side <= 256):
 * b is clamped to the handle's panel width (16 or 32).  a >= 1, 0 < rho <= 1, 0 < gamma <= 1;
 * a = 0 switches the prediction off.  Returns FRSVT_ERR_UNSUPPORTED for other handles.
 * Synchronizes the handle's stream.
 */
frsvt_status frsvt_set_rank_prediction(frsvt_handle* h, int32_t a, double rho, double gamma);

/* The sampling rate the next SVT will use under adaptive rank prediction (synchronizes). */
frsvt_status frsvt_get_rank_prediction(frsvt_handle* h, int32_t* l_next);

/*
 * Partial thresholding (Table 6, Type B: the proximal step of the truncated nuclear norm
 * sum_{i>k} sigma_i): from the next SVT on, the k leading singular values of B are kept and the
 * others soft-thresholded, in frsvt_svt and in the L-step of rpca_ialm_step (the Type B RPCA
 * of the weather-removal application).  r then counts the non-zero values.  0 <= k <= cfg.l_max;
 * k = 0 restores the plain SVT.  Synchronizes the handle's stream.
 */
frsvt_status frsvt_set_partial(frsvt_handle* h, int32_t k);

/*
 * Tracing.  Phases of the path, in launch order within one SVT / iALM step.
 * When timing is enabled every kernel launch is bracketed by CUDA events on
 * the handle's stream (recording events does not synchronize; it adds a few
 * microseconds per launch).  frsvt_get_timings synchronizes, then returns per
 * phase the summed device time in milliseconds and the number of timed
 * launch groups since the previous call, and clears them.  A group is one
 * launcher call and may hold more than one kernel (the wide-basis Gram and
 * the small dense factorisation that consumes it are one group).  ms and
 * launches have FRSVT_NPHASE entries.  Disabling collects pending events
 * first.
 */
#define FRSVT_NPHASE 11
#define FRSVT_PHASE_SKETCH    0   /* Y = A^T Omega            (Alg. 1 steps 4-5, 8-9) */
#define FRSVT_PHASE_POWER_AQ  1   /* Z = A Q in a power step  (step 14) */
#define FRSVT_PHASE_POWER_ATZ 2   /* Y = A^T Z in a power step (step 14) */
#define FRSVT_PHASE_REDUCE    3   /* split-K reduction of Y */
#define FRSVT_PHASE_ORTH      4   /* orthonormalisation       (steps 6, 10-11, 14) */
#define FRSVT_PHASE_PROJECT   5   /* Z = A Q = B^T            (step 16) */
#define FRSVT_PHASE_GRAM      6   /* B B^T = Z^T Z in double-float */
#define FRSVT_PHASE_CORE      7   /* l x l SVD and shrinkage  (steps 16-19) */
#define FRSVT_PHASE_EPILOGUE  8   /* X = Z M Q^T, fused with the iALM update (Eq. 6) */
#define FRSVT_PHASE_FINISH    9   /* residual reduction and mu update */
#define FRSVT_PHASE_APPLY    10   /* products with the small factors on the wide basis:
                                     Q = Y R^{-1} (steps 6 / 14), Rf = Q M and Q~ = Q U (step 19) */
frsvt_status frsvt_enable_timing(frsvt_handle* h, int32_t enable);
frsvt_status frsvt_get_timings(frsvt_handle* h, double* ms, int32_t* launches);
const char* frsvt_phase_name(int32_t phase);

/*
 * Kernels per iALM step.  *kernels = the number of kernel launches in the CUDA
 * graph that the most recent rpca_ialm_step call replayed (counted from the
 * graph's kernel nodes when it was captured), or 0 when that call launched its
 * kernels directly (phase timing on, or the caller's stream being captured).
 * Host-only; does not synchronize.
 */
frsvt_status frsvt_step_kernels(frsvt_handle* h, int32_t* kernels);

/*
 * Work split of one pass over A on the wide basis (Alg. 1 steps 5, 9, 14, 16: Y^T = M^T A or
 * Z^T = Q^T A^T with a 128-row basis side).  The long side (nlong) is cut into tiles of 256, the
 * contracted side (nk) into K-chunks of 32 columns for an FP32-accurate pass
 * (precision = FRSVT_PREC_FP32) or of 64 for a BF16 / FP8 shadow pass; the tile-major
 * (tile, K-chunk) units are cut into *grid contiguous ranges, one CTA each, for a GPU of `sms`
 * SMs.  *max_parts = the most CTA ranges that touch one tile (the partials its fixed-order sum
 * adds; the workspace holds 8), *max_tiles = the most tiles one range touches (its TMEM
 * accumulators; at most 2).  Host-only arithmetic, no device work; FRSVT_ERR_INVALID_ARG for
 * null outputs, nlong, nk or sms below 1, or an unknown precision.
 */
frsvt_status frsvt_wide_pass_plan(int64_t nlong, int64_t nk, int32_t precision, int32_t sms, int32_t* grid,
                                  int32_t* max_parts, int32_t* max_tiles);

/*
 * Allocation-free FRSVT (the paper has no counterpart: this is a deployment
 * entry point, not part of the method).
 *
 * Some callers cannot allocate device memory: plug-ins whose host framework
 * owns every device allocation through its own pool, real-time paths that must
 * not enter the allocator (cudaMalloc / cudaFree may synchronize the device and
 * take unbounded time), services that fix their device-memory budget at
 * start-up.
 * frsvt_svt_noalloc computes the same X = FRSVT_tau(A) as frsvt_svt (no range
 * propagation; Omega stream index `counter`, key `seed`) without a handle and
 * without allocating: no cudaMalloc, no cudaFree, no allocating library call.
 * Its scratch is one static device array of FRSVT_NOALLOC_SCRATCH_BYTES (8 MiB)
 * that every GPU which loads this library keeps until the process exits.
 *
 * Limits (checked; larger sizes return FRSVT_ERR_INVALID_ARG):
 *   m <= FRSVT_NOALLOC_MAX_M, n <= FRSVT_NOALLOC_MAX_N, m >= n (m < n:
 *   FRSVT_ERR_UNSUPPORTED), 1 <= l <= 16, 0 <= q <= 64, tau finite and >= 0,
 *   counter != UINT64_MAX (a reserved value).  A and X are caller-owned device
 *   buffers with the alignment rules above.  The kernels' device status bits
 *   (non-finite values, an unconverged core, a rank-deficient sketch) are not
 *   reported by this entry point.
 * The first call on a device performs a one-time set-up on that device (the
 * device address of the scratch array, kernel attributes); make that first call
 * before any stream capture.  Every call shares the one array and keeps the
 * previous call's contents; the call clears what must start at zero.  Calls
 * that overlap on the GPU (different streams or host threads) race: serialize
 * them.  Work is enqueued on `stream` (a cudaStream_t, NULL = legacy default).
 */
#define FRSVT_NOALLOC_SCRATCH_BYTES (8u << 20)
#define FRSVT_NOALLOC_MAX_M 65536
#define FRSVT_NOALLOC_MAX_N 256
frsvt_status frsvt_svt_noalloc(const float* A, int64_t m, int64_t n, int64_t lda, float tau,
                               int32_t l, int32_t q, uint64_t seed, uint64_t counter,
                               float* X, int64_t ldx, void* stream);

/*
 * Low-rank representation (Table 6, Type A; the robust-LRR application of Sec. 4): min ||L||_* + lam ||S||_{2,1}
 * s.t. O = Z L + S with the dictionary Z = O (d x n), by the inexact ALM with the splitting J = L:
 * per iteration J = FRSVT_{1/mu}(L + Y2 / mu) (Alg. 1, Omega stream = iteration index, range
 * propagation across iterations when asked), L = (I + Z^T Z)^{-1} (Z^T (O - S + Y1 / mu) + J -
 * Y2 / mu), S = the column shrinkage of O - Z L + Y1 / mu by lam / mu (column i scaled by
 * max(0, 1 - (lam / mu) / ||q_i||)), Y1 += mu (O - Z L - S), Y2 += mu (L - J),
 * mu = min(rho mu, mu_max).
 *
 * frsvt_lrr_create: workspace for d <= d_max, 2 <= n <= n_max (<= 16384), FRSVT rank l
 *   (1 <= l <= min(128, n_max)) and q power steps; owns an frsvt handle for the n x n J step
 *   (l > 32: the wide basis).  Allocates all device memory.  stream: a cudaStream_t.
 * frsvt_lrr_init: O is a caller-owned device matrix (d x n, row-major, ldo >= n) that must stay
 *   valid while the handle iterates; zeroes L, S, J, Y1, Y2, sets mu = mu0, and forms
 *   (I + O^T O)^{-1} on the device by Newton-Schulz iterations (synchronizes the stream once).
 *   Needs lam > 0, mu0 > 0, rho >= 1, mu0 <= mu_max < inf (FRSVT_ERR_INVALID_ARG otherwise).
 * frsvt_lrr_step: one iteration, enqueued on the stream; with err != NULL it synchronizes and
 *   writes max(||O - Z L - S||_inf, ||L - J||_inf) (the stopping quantity) to *err (host).
 * frsvt_lrr_get: copies L (n x n) and S (d x n) into caller-owned device buffers (either may be
 *   NULL), and the next mu and the iteration count to host pointers (either may be NULL).
 * Errors of the J step are returned as the frsvt status; frsvt_lrr_last_error explains.
 */
typedef struct frsvt_lrr frsvt_lrr;
frsvt_status frsvt_lrr_create(frsvt_lrr** h, int64_t d_max, int64_t n_max, int32_t l, int32_t q, uint64_t seed,
                              int32_t range_prop, void* stream);
frsvt_status frsvt_lrr_destroy(frsvt_lrr* h);
frsvt_status frsvt_lrr_init(frsvt_lrr* h, const float* O, int64_t d, int64_t n, int64_t ldo, double lam, double mu0,
                            double rho, double mu_max);
frsvt_status frsvt_lrr_step(frsvt_lrr* h, double* err);
frsvt_status frsvt_lrr_get(frsvt_lrr* h, float* L, int64_t ldl, float* S, int64_t lds, double* mu, int32_t* iters);
const char* frsvt_lrr_last_error(const frsvt_lrr* h);

const char* frsvt_status_string(frsvt_status s);
const char* frsvt_last_error(const frsvt_handle* h);

/* ------------------------------------------------------------------ adjoint (backward pass)
 * Differentiation of the FRSVT map with a fixed Omega, X = FRSVT_tau(A) of Alg. 1 (steps 3-19:
 * Gaussian sketch, q power steps with re-orthonormalisation, projection, l x l SVD, shrinkage,
 * reconstruction), for the tall orientation m >= n; the basis Q lives on the column side.
 * The handle must be created with FRSVT_CFG_ADJOINT in cfg.flags (this allocates the backward
 * workspace); n <= 2048 (l <= 16) or n <= 1024 (l <= 32).
 *
 * frsvt_adjoint_saved_bytes: size of the device buffer `saved` for an m x n problem (it holds
 *   Q_i and R_i of the q + 1 CholeskyQR2 factorisations, U_B, sigma and V_B).
 * frsvt_svt_save: X = FRSVT_tau(A) with Omega from the Philox stream (cfg.seed, omega_stream),
 *   every orthonormalisation by CholeskyQR2, and the factors written to `saved` (caller-owned
 *   device memory of frsvt_adjoint_saved_bytes).  Range propagation is not used here.
 * frsvt_backward: given dX (m x n, the cotangent of X), writes dA (m x n, overwritten) and *dtau
 *   (one float in device memory): the vector-Jacobian product of the same map, with the
 *   divided-difference adjoint of the shrinkage on B (Gs_ij = (f_i - f_j) / (sigma_i - sigma_j),
 *   replaced by the mean of f' where sigma_i and sigma_j coincide: the gap regularisation of the
 *   1 / (sigma_j^2 - sigma_i^2) term), the QR adjoint Ybar = (Qbar - Q copyltu(Qbar^T Q)) R^{-T}
 *   through each CholeskyQR2, and the recomputed power-step products.  A, tau, l and
 *   omega_stream must be those of the frsvt_svt_save call that wrote `saved`.
 * All pointers are device pointers; row-major; lda, ldx >= n.  Asynchronous on the handle's
 * stream, no allocation.  Errors: FRSVT_ERR_INVALID_ARG, FRSVT_ERR_UNSUPPORTED (no adjoint
 * workspace, m < n, size limits), FRSVT_ERR_CUDA.  Rank deficiency of a sketch sets
 * FRSVT_DEV_RANK_DEFICIENT (the QR adjoint then is not defined for the dropped columns). */
size_t frsvt_adjoint_saved_bytes(const frsvt_handle* h, int64_t m, int64_t n);
frsvt_status frsvt_svt_save(frsvt_handle* h, const float* A, int64_t m, int64_t n, int64_t lda, float tau,
                            int32_t l, uint64_t omega_stream, float* X, int64_t ldx, void* saved);
frsvt_status frsvt_backward(frsvt_handle* h, const void* saved, const float* A, int64_t m, int64_t n, int64_t lda,
                            float tau, int32_t l, uint64_t omega_stream, const float* dX, int64_t lddx, float* dA,
                            int64_t ldda, float* dtau);

/* ------------------------------------------------------------------ unrolled iALM RPCA
 * The differentiable workload: K inexact-ALM steps of robust PCA (the host algorithm of Sec. 4.1)
 * unrolled, with a threshold tau_k and a penalty mu_k per step as learnable parameters, over a
 * batch of B matrices (each m x n, m >= n, n % 4 == 0, row-major with leading dimension ld; the
 * batch is contiguous, problem b at O + b m ld):
 *     A_k = O - S_{k-1} + Y_{k-1} / mu_k,   L_k = FRSVT_{tau_k}(A_k)  (Alg. 1, Omega stream k),
 *     S_k = shrink_{lambda / mu_k}(O - L_k + Y_{k-1} / mu_k),   Y_k = Y_{k-1} + mu_k (O - L_k - S_k),
 * from S_0 = 0 and Y_0 = y0_scale_b O (y0_scale_b = 1 / max(||O_b||_2, ||O_b||_inf / lambda), the
 * iALM initialisation).  The output is L_K.  The library runs the whole batch and every step in
 * one call: the FRSVT and its adjoint (frsvt_svt_save / frsvt_backward) and fused elementwise
 * kernels for the shrinkage, the multiplier update and their adjoints.  The handle must be
 * created with FRSVT_CFG_ADJOINT (the adjoint's size limits apply).
 *
 * rpca_unrolled_saved_bytes: size of the caller-owned device buffer `saved` (per problem and step:
 *   A_k, L_k, Y_{k-1} and the FRSVT factors; plus the backward scratch).
 * rpca_unrolled_init: y0_scale (HOST array of B floats) from ||O_b||_2 (frsvt_spectral_norm with
 *   power_iters steps) and the largest |O_b| entry.  Synchronizes.
 * rpca_unrolled_forward: tau, mu: HOST arrays of K floats (tau_k >= 0, mu_k > 0); L: B x m x ld
 *   device output (L_K of every problem); saved: written for the backward pass.  Asynchronous.
 * rpca_unrolled_backward: dL (B x m x ld, the cotangent of L_K) -> dtau, dmu (DEVICE arrays of K
 *   floats, overwritten): the gradient of <dL, L_K> summed over the batch.  Same O, y0_scale,
 *   tau, mu, lambda, l as the forward call that wrote `saved`.  Asynchronous.
 * Errors: FRSVT_ERR_INVALID_ARG (sizes, pointers, alignment, parameters), FRSVT_ERR_UNSUPPORTED
 * (no adjoint workspace, adjoint size limits), FRSVT_ERR_CUDA. */
size_t rpca_unrolled_saved_bytes(const frsvt_handle* h, int32_t batch, int32_t steps, int64_t m, int64_t n,
                                 int64_t ld);
frsvt_status rpca_unrolled_init(frsvt_handle* h, int32_t batch, const float* O, int64_t m, int64_t n, int64_t ld,
                                double lambda, int32_t power_iters, float* y0_scale);
frsvt_status rpca_unrolled_forward(frsvt_handle* h, int32_t batch, int32_t steps, const float* O, int64_t m,
                                   int64_t n, int64_t ld, const float* y0_scale, const float* tau, const float* mu,
                                   float lambda, int32_t l, float* L, void* saved);
frsvt_status rpca_unrolled_backward(frsvt_handle* h, int32_t batch, int32_t steps, const float* O, int64_t m,
                                    int64_t n, int64_t ld, const float* y0_scale, const float* tau, const float* mu,
                                    float lambda, int32_t l, const void* saved, const float* dL, float* dtau,
                                    float* dmu);

/* ------------------------------------------------------------------ batched weighted SVT
 * Weighted SVT (the WSVT footnote of Sec. 1) of a batch of small independent matrices, the
 * patch groups of weighted nuclear norm minimisation:
 *     X_b = U_b max(Sigma_b - w_b, 0) V_b^T,   w_{b,j} = c sqrt(n_b) / (sigma_{b,j} + eps),
 * with the weights evaluated on the problem's own singular values (non-descending in j, so the
 * closed form is the exact minimiser of sum_j w_j sigma_j(X) + 1/2 ||X - A_b||_F^2).
 *   A, X : device arrays of `batch` device pointers; problem b is m x n_b, row-major and
 *          contiguous (ld = n_b), FP32.  X_b may not alias A_b.  Caller-owned.
 *   n_i  : device array of the `batch` column counts, 1 <= n_b <= cfg.n_max of the handle.
 *   m    : rows of every problem, 1 <= m <= 64.
 *   variant FRSVT_WSVT_EXACT: Gram matrix on the short side and a two-sided Jacobi eigensolver
 *          (FP32).  FRSVT_WSVT_FRSVT: Alg. 1 per problem with l sketch columns (l <= 32),
 *          cfg.q power steps, Omega from the Philox stream (cfg.seed, stream 0, problem b),
 *          double-float Gram / Cholesky and the l x l SVD, the weights applied to D.
 * One persistent launch on the handle's stream: no allocation, no host synchronisation, so a
 * call can be captured in a CUDA graph.  A problem with an unsupported size is skipped and sets
 * FRSVT_DEV_BAD_PROBLEM in the device status.  The launch shape (threads per CTA, CTAs per
 * SM) is the one frsvt_wsvt_tune chose for the variant, else 256 threads and as many CTAs as fit.
 * Errors: FRSVT_ERR_INVALID_ARG (null arrays, m, l, c < 0, eps <= 0), FRSVT_ERR_UNSUPPORTED
 * (m > 64 or n_max too large for shared memory), FRSVT_ERR_CUDA. */
#define FRSVT_WSVT_EXACT 0
#define FRSVT_WSVT_FRSVT 1
frsvt_status frsvt_wsvt(frsvt_handle* h, int32_t batch, const float* const* A, const int32_t* n_i, int32_t m,
                        float c, float eps, float* const* X, int32_t variant, int32_t l);
/* Autotuner of frsvt_wsvt: runs the batch with every candidate launch shape (128 / 256 / 512
 * threads per CTA x 1 .. resident CTAs per SM), timed with CUDA events on the handle's stream
 * (synchronises; not capturable), and keeps the fastest for `variant` in the handle.  X holds
 * the result of the last run.  Same arguments and errors as frsvt_wsvt. */
frsvt_status frsvt_wsvt_tune(frsvt_handle* h, int32_t batch, const float* const* A, const int32_t* n_i, int32_t m,
                             float c, float eps, float* const* X, int32_t variant, int32_t l);
/* The launch shape frsvt_wsvt uses for `variant` (ctas_per_sm 0: as many as fit). */
frsvt_status frsvt_wsvt_get_tuning(const frsvt_handle* h, int32_t variant, int32_t* threads, int32_t* ctas_per_sm);

/* Debug access to stages of the path, for parity tests of single kernels. */
/* Omega[:rows, :cols] of (seed, stream, problem) into a device buffer (ld = cols). */
frsvt_status frsvt_debug_omega(float* out, int64_t rows, int32_t cols, uint64_t seed,
                               uint64_t stream, uint64_t problem, void* cuda_stream);
/* Z = A Q on the tensor cores (tcgen05, 3xTF32): the row pass of Alg. 1 steps 14 / 16 alone.
 * A: m x n (lda, n <= 256), Q: n x LP row-major (LP = 16 when cfg.l_max <= 16, else 32), Z: m x LP.
 * Enqueued on the handle's stream; device errors go to the handle's status word. */
frsvt_status frsvt_debug_rows_tc(frsvt_handle* h, const float* A, int64_t m, int64_t n, int64_t lda,
                                 const float* Q, float* Z);
/* Y = A^T B on the tensor cores (tcgen05, 3xTF32): the column pass of Alg. 1 steps 5 / 9 / 14 alone.
 * B: m x LP row-major, or NULL for B = Omega of the (seed, stream) Philox stream (Alg. 1 step 4).
 * Y: n x LP row-major (n <= 256).  Enqueued on the handle's stream. */
frsvt_status frsvt_debug_cols_tc(frsvt_handle* h, const float* A, int64_t m, int64_t n, int64_t lda,
                                 const float* B, uint64_t seed, uint64_t stream, float* Y);
/* Failure detection of the bounded waits: one CTA waits, polling at most spin_limit times
 * (1 <= spin_limit <= 2^20), on an mbarrier that nothing arrives at, with the same bounded poll
 * that every pipeline wait of the library uses (where the limit is fixed at 2^26 polls).  The
 * wait gives up, the kernel ORs FRSVT_DEV_TIMEOUT into the handle's device status and returns
 * (it holds no tensor memory and has no copy in flight, so the handle and the context stay
 * usable).  Enqueued on the handle's stream; read the bit with frsvt_get_info. */
frsvt_status frsvt_debug_wait_timeout(frsvt_handle* h, uint32_t spin_limit);
/* Raw Philox4x64-10 words for counters (i, j, stream, problem), i < rows, j < blocks: rows x blocks x 4 uint64. */
frsvt_status frsvt_debug_philox(uint64_t* out, int64_t rows, int32_t blocks, uint64_t seed,
                                uint64_t stream, uint64_t problem, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* FRSVT_H_ */
