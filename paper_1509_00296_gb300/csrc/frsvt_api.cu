// Host side of the C ABI declared in include/frsvt.h: handle and workspace
// management, argument validation, and the launch sequence of FRSVT (Alg. 1)
// and of one inexact-ALM iteration.  No entry point allocates except
// frsvt_create; no entry point synchronizes unless its contract says so.
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "../../include/frsvt.h"
#include "state.cuh"

namespace frsvt {
size_t orth_smem_bytes(int LP, int64_t ns);
size_t fused_orth_smem(int LP, int64_t ns);
size_t fused_core_smem(int LP, int64_t ns);
cudaError_t prepare_fused_kernels(int smem_limit);
cudaError_t launch_sc_orth(int LP, const float* A, int64_t m, int64_t n, int64_t lda, const float* Zl, uint64_t seed,
                           uint64_t ctr, DevState* dst, int nsplit, int64_t rps, float* cpart, float* Y,
                           unsigned* tickets, int l, int use_rp, const float* Qt, float* Q, double rank_tol,
                           cudaStream_t st);
cudaError_t launch_lr(int LP, bool gram, const float* A, int64_t m, int64_t n, int64_t lda, const float* Q, float* Z,
                      int nblocks, double* cpart, double* G, unsigned* tickets, int l, float tau_host,
                      int tau_from_mu, int update_rp, int advance_counter, float* Rf, float* Qt, DevState* dst,
                      double rank_tol, int max_sweeps, cudaStream_t st);
cudaError_t launch_alm2(int LP, const float* Z, const float* Rf, const float* O, float* S, float* A, int64_t m,
                        int64_t n, int64_t ld, float* L, int64_t ldl, DevState* dst, int nsplit, int64_t rps,
                        double* cpart, double* rsum, unsigned* tickets, cudaStream_t st);
int tma_np4(int64_t n);
size_t tma_sc_smem(int LP, int64_t n);
size_t tma_lr_smem(int LP, int64_t n, int nst);
int tma_lr_stages(int LP, int64_t n, size_t limit);
int tma_rows_per_tile_lr();
int tma_resident_grid(int LP, int64_t n);
int tma_alm_resident_grid(int LP, int64_t n);
size_t tma_alm_smem(int LP, int64_t n);
int tma_rows_per_tile();
int tma_rows_per_tile_epilogue();
cudaError_t prepare_tma_kernels(int smem_limit);
cudaError_t launch_tp_sc(int LP, const CUtensorMap& tmA, const CUtensorMap* tmZ, int64_t m, int64_t n, int64_t rpc,
                         int grid, uint64_t seed, uint64_t ctr, DevState* dst, float* cpart, float* Y, unsigned* tickets,
                         int l, int use_rp, int passes, const float* Qt, float* Q, double rank_tol, cudaStream_t st);
cudaError_t launch_tp_lr(int LP, bool gram, const CUtensorMap& tmA, int64_t m, int64_t n, int64_t rpc, int grid,
                         int nst, const float* Q, float* Z, double* cpart, double* G, unsigned* tickets, int l, float tau_host,
                         int tau_from_mu, int update_rp, int advance_counter, float* Rf, float* Qt, DevState* dst,
                         double rank_tol, int max_sweeps, cudaStream_t st);
cudaError_t launch_tp_alm(int LP, const CUtensorMap& tmO, const CUtensorMap& tmS, const CUtensorMap& tmA,
                          const CUtensorMap& tmZ, int64_t m, int64_t n, int64_t rpc, int grid, const float* Rf,
                          float* S, float* A, int64_t ld, float* L, int64_t ldl, DevState* dst, double* cpart,
                          unsigned* tickets, void* Ab, int64_t ldb, cudaStream_t st);
int tb_lr_stages(int LP, int64_t n, size_t limit);
int tb_sc_stages(int LP, int64_t n, bool omega, size_t limit);
size_t tb_sc_smem(int LP, int64_t n, bool omega, int ns);
cudaError_t prepare_tb_kernels(int smem_limit);
int tb_sc_resident_grid(int LP, int64_t n, int ns);
cudaError_t launch_tb_lr(int LP, const CUtensorMap& tmA, int64_t m, int64_t n, int grid, int ns, const float* Q,
                         float* Z, DevState* dst, cudaStream_t st);
cudaError_t launch_tb_sc(int LP, const CUtensorMap& tmA, const CUtensorMap* tmZ, int64_t m, int64_t n, int grid,
                         int ns, uint64_t seed, uint64_t ctr, DevState* dst, float* cpart, float* Y,
                         unsigned* tickets, int l, int use_rp, int passes, const float* Qt, float* Q,
                         double rank_tol, cudaStream_t st);
cudaError_t launch_to_bf16(const float* A, int64_t lda, int64_t m, int64_t n, void* Ab, int64_t ldb, cudaStream_t st);
int tb_box_rows_lr();
int tb_box_rows_sc();
size_t tc_lr_smem(int LP, int64_t n, int ns);
int tc_lr_stages(int LP, int64_t n, size_t limit);
size_t gram_core_smem(int LP, int64_t n);
int gram_resident_grid(int LP, int64_t n);
size_t wsvt_smem(int variant, int m, int n_max, int LP);
int ad_col_splits(int64_t m, int n);
cudaError_t prepare_adjoint_kernels(int smem_limit);
cudaError_t ad_rows(int LP, const float* M, int64_t ldm, int64_t m, int n, const float* S, float* C, int ldc, int coff,
                    float beta, cudaStream_t st);
cudaError_t ad_cols(int LP, const float* M, int64_t ldm, int64_t m, int n, const float* T, int ldt, double* part,
                    float* out, double* out_d, int ldo, int coff, float beta, cudaStream_t st);
cudaError_t ad_rank(float* A, int64_t lda, int64_t m, int n, const float* L, int ldl, const float* R, int ldr, int K,
                    float beta, cudaStream_t st);
cudaError_t ad_omega(int LP, float* out, int ldo, int coff, int64_t m, int l, uint64_t seed, uint64_t stream,
                     cudaStream_t st);
cudaError_t ad_cholqr2(int LP, const float* Y, int n, int l, double rank_tol, float* Q, double* Qd, float* R,
                       DevState* dst, cudaStream_t st);
cudaError_t ad_core(int LP, const float* Z, int64_t m, int l, float tau, double rank_tol, int max_sweeps, float* U,
                    float* sig, float* S1, float* S2, DevState* dst, cudaStream_t st);
cudaError_t ad_svt_adjoint(int LP, const float* W1, const float* U, const float* sig, int l, float tau, float* C1,
                           float* C2, float* C3, float* taubar, cudaStream_t st);
cudaError_t ad_qr_adjoint(int LP, const double* Q, const float* R, const double* Qbar, int n, int l, float* Ybar,
                          cudaStream_t st);
int wsvt_ctas_per_sm(int variant, int nt, int m, int n_max, int LP);
cudaError_t launch_wsvt(int variant, int nt, int grid, int LP, const float* const* A, float* const* X,
                        const int32_t* n, int batch, int m, int n_max, float c, float eps, uint64_t seed,
                        uint64_t stream, int l, int q, double rank_tol, int max_sweeps, unsigned* next,
                        DevState* dst, cudaStream_t st);
cudaError_t prepare_gram_kernels(int smem_limit);
cudaError_t launch_gram_core(int LP, const float* Z, int64_t m, int64_t n, int grid, const float* Q, double* cpart,
                             double* G, unsigned* tickets, int l, float tau_host, int tau_from_mu, int update_rp,
                             int advance_counter, float* Rf, float* Qt, DevState* dst, double rank_tol,
                             int max_sweeps, cudaStream_t st);
cudaError_t prepare_tc_kernels(int smem_limit);
cudaError_t launch_tc_lr(int LP, const CUtensorMap& tmA, int64_t m, int64_t n, int grid, int ns, const float* Q, float* Z,
                         DevState* dst, cudaStream_t st, int normalize = 0);
int tc_box_cols();
int tc_box_rows();
int tc_sc_stages(int LP, int64_t n, bool omega, size_t limit);
size_t tc_sc_smem(int LP, int64_t n, bool omega, int ns);
cudaError_t prepare_tc_sc_kernels(int smem_limit);
int tc_sc_resident_grid(int LP, int64_t n, int ns);
cudaError_t launch_tc_sc(int LP, const CUtensorMap& tmA, const CUtensorMap* tmZ, int64_t m, int64_t n, int grid,
                         int ns, uint64_t seed, uint64_t ctr, DevState* dst, float* cpart, float* Y,
                         unsigned* tickets, bool tail, int l, int use_rp, int passes, const float* Qt, float* Q,
                         double rank_tol, cudaStream_t st);
int tc_sc_rows();
int wide_lp();
int wide_tile();
cudaError_t prepare_wide_kernels();
int wide_gram_grid();
int wide_gram_count();
cudaError_t launch_wd_rp_insert(float* YT, const float* QtT, int64_t ld, int64_t ns, int l, const DevState* dst,
                               cudaStream_t st);
cudaError_t launch_wd_identity(float* T, cudaStream_t st);
cudaError_t launch_wd_colscale(const float* YT, int64_t ld, int64_t ns, float* T, cudaStream_t st);
cudaError_t launch_wd_omega(float* OT, float* OTl, void* OTb, void* OTbl, int64_t ldo, int64_t m, int l, int use_rp,
                            uint64_t seed, uint64_t ctr, const DevState* dst, cudaStream_t st);
void wide_pass_plan(int64_t nlong, int64_t nk, int prec, int sms, int* grid, int* max_parts, int* max_tiles);
cudaError_t launch_wd_pass(bool col, int prec, const CUtensorMap& tmA, const CUtensorMap& tmM, const CUtensorMap& tmMl,
                           int64_t nlong, int64_t nk, int sms, float* part, int64_t ldp, float* outT, float* outTl,
                           void* outTb, void* outTbl, int64_t ldo, float* outR, float* outRl, DevState* dst,
                           cudaStream_t st, const float* scales = nullptr, int ntr8 = 0, int ntc8 = 0);
cudaError_t launch_wd_quant8(const float* A, int64_t lda, int64_t m, int64_t n, void* A8, int64_t ld8, float* scales,
                             cudaStream_t st);
cudaError_t launch_wd_gram(bool core, const float* XT, int64_t ldx, int64_t len, int grid, double* cpart, double* Gpk,
                           int p, double rank_tol, int l, float tau_host, int tau_from_mu, int update_rp,
                           int advance_counter, int max_sweeps, float* T1, float* T2, DevState* dst,
                           cudaStream_t st);
cudaError_t launch_wd_apply(const float* in, int64_t ldi, int64_t len, const float* T, float* outT, float* outTl,
                            int64_t ldo, float* outR, float* outRl, cudaStream_t st);
cudaError_t launch_wd_trsm(const float* in, int64_t ldi, int64_t len, const float* T, float* outT, float* outTl,
                           void* outTb, void* outTbl, int64_t ldo, cudaStream_t st);
int unrolled_grid(int64_t m, int64_t n, int sms);
cudaError_t launch_ur_pre(const float* O, const float* S, const float* Y, float ys, float* A, int64_t m, int64_t n,
                          int64_t ld, float mu, int grid, cudaStream_t st);
cudaError_t launch_ur_post(const float* O, const float* L, const float* Y, float ys, float* S, float* Yout, float* An,
                           int64_t m, int64_t n, int64_t ld, float mu, float mu_next, float lam, int grid,
                           cudaStream_t st);
cudaError_t launch_ur_bwd_post(const float* O, const float* L, const float* Y, float ys, const float* Sb,
                               const float* Yb, const float* Lin, float* Lb, float* Yb2, float* Tb, int64_t m,
                               int64_t n, int64_t ld, float mu, float lam, double* part, int grid, cudaStream_t st);
cudaError_t launch_ur_bwd_pre(const float* O, const float* Y, float ys, const float* Ab, const float* Tb, float* Sb,
                              float* Yb2, int64_t m, int64_t n, int64_t ld, float mu, double* part, int grid,
                              cudaStream_t st);
cudaError_t launch_ur_sum(const double* part, int count, float* out, int accumulate, cudaStream_t st);
cudaError_t launch_ur_addf(const float* in, float* out, cudaStream_t st);
cudaError_t launch_ur_addv(const float* in, float* out, int count, cudaStream_t st);
cudaError_t launch_absmax_sumsq(const float* O, int64_t m, int64_t n, int64_t ld, float* pmax, float2* psum, int nblk,
                                cudaStream_t st);
cudaError_t launch_wd_alm(bool alm, const CUtensorMap& tmZ, const CUtensorMap& tmZl, const CUtensorMap& tmR,
                          const CUtensorMap& tmRl, int64_t m, int64_t n, const float* O, float* S, float* A, int64_t ld,
                          float* L, int64_t ldl, DevState* dst, double* cpart, unsigned* ticket, int grid,
                          void* Ab, int64_t ldb, cudaStream_t st);
}

using namespace frsvt;

struct frsvt_handle {
  frsvt_config cfg{};
  cudaStream_t stream = nullptr;
  int LP = 16;
  int sms = 1;
  int target_ctas = 4;
  int64_t part_elems = 0;
  int rpart_max = 0;
  int gsplit_max = 0;
  int absmax_blocks = 0;
  DevState* dst = nullptr;
  float* Ys = nullptr;
  float* Qs = nullptr;
  float* Qt = nullptr;
  float* Zl = nullptr;
  float* Rf = nullptr;
  float* part = nullptr;
  float2* gpart = nullptr;
  float2* rpart = nullptr;
  float* pmax = nullptr;
  float2* psum = nullptr;
  // fused path (short side small enough for one CTA): cluster partials, final sums, tickets
  bool fused = false;
  bool tma = false;          // persistent TMA-pipelined passes (short side <= 256 columns)
  int tma_grid = 8;
  int tc_sc_ns = 0;          // stages of the tensor-core column pass (0: not available)
  int tc_lr_ns = 0;          // stages of the tensor-core row pass
  int gram_grid = 8;         // CTAs of the Gram / core kernel (whole clusters)
  int alm_grid = 4;          // CTAs of the fused iALM epilogue (whole clusters)
  unsigned* wsvt_next = nullptr;   // work counter of the batched WSVT launch
  float* ad_ws = nullptr;          // adjoint workspace (FRSVT_CFG_ADJOINT)
  void* Ab = nullptr;              // BF16 shadow of A (FRSVT_PREC_BF16)
  int64_t ldb = 0;                 // its row stride in elements
  int tb_lr_ns = 0, tb_sc_ns = 0, tb_sc_grid = 0;
  int ad_K = 0;                    // columns of the stacked rank-update factors
  int wsvt_nt[2] = {256, 256};     // threads per CTA per variant (autotuner)
  int wsvt_cps[2] = {0, 0};        // CTAs per SM per variant (0: as many as fit)
  int tc_sc_grid = 0;
  float* cpart_sc = nullptr;
  double* cpart_lr = nullptr;
  double* cpart_alm = nullptr;
  double* Gfin = nullptr;
  double* rsum = nullptr;
  unsigned* tickets = nullptr;
  int64_t cpart_sc_elems = 0, cpart_alm_elems = 0;
  int lr_blocks = 8;
  int64_t last_m = -1, last_n = -1;
  int last_l = -1;
  // rpca_ialm_step replays its launches from a CUDA graph captured on the first call with a given
  // argument tuple (capture_stream is private to the handle; the graph runs on the user's stream).
  // epoch changes whenever a setter changes what a step launches, which retires the graph.
  struct StepKey {
    const float* O;
    float* S;
    float* A;
    int64_t m, n, ld;
    int32_t l;
    float* L;
    int64_t ldl;
    uint64_t epoch;
    bool operator==(const StepKey& o) const {
      return O == o.O && S == o.S && A == o.A && m == o.m && n == o.n && ld == o.ld && l == o.l && L == o.L &&
             ldl == o.ldl && epoch == o.epoch;
    }
  };
  uint64_t epoch = 1;
  cudaStream_t capture_stream = nullptr;
  // child handles (cfg.problem_streams): independent problems of an unrolled batch run on them,
  // each on its own stream, forked from and joined back into `stream`
  std::vector<frsvt_handle*> kids;
  std::vector<cudaStream_t> kid_streams;
  std::vector<cudaEvent_t> kid_events;
  cudaEvent_t fork_event = nullptr;
  static constexpr int kGraphSlots = 4;          // graphs kept for the most recent argument tuples
  cudaGraphExec_t step_exec[kGraphSlots] = {};
  StepKey step_key[kGraphSlots] = {};
  uint64_t step_used[kGraphSlots] = {};           // last use (LRU eviction)
  int32_t step_kernels[kGraphSlots] = {};         // kernel nodes of each captured graph
  int32_t last_step_kernels = 0;                  // ... of the graph the last step replayed
  uint64_t step_clock = 0;
  // wide basis (cfg.l_max > 32, LP = 128, any short side): basis-side matrices transposed
  // (128 x ld_m / ld_n), Z and Rf row-major (len x 128), K-split partials, Gram partials
  bool wide = false;
  int64_t w_ldl = 0, w_lds = 0, w_ldp = 0;      // long-side / short-side / partial row strides
  float *wOT = nullptr, *wOTl = nullptr, *wZT = nullptr, *wZTl = nullptr, *wZ = nullptr, *wZl = nullptr;
  float *wYT = nullptr, *wQT = nullptr, *wQTl = nullptr, *wQp = nullptr, *wRf = nullptr, *wRfl = nullptr;
  float *wT1 = nullptr, *wT2 = nullptr, *wpart = nullptr;
  float* wI = nullptr;             // diagonal T of the unnormalised power steps (identity off the diagonal)
  void *wOTb = nullptr, *wOTbl = nullptr, *wZTb = nullptr, *wZTbl = nullptr, *wQTb = nullptr, *wQTbl = nullptr;
  void* A8 = nullptr;              // E4M3 shadow of A (FRSVT_PREC_FP8), row stride ld8 bytes
  float* w8s = nullptr;            // its per-128 x 128-tile scales
  int64_t ld8 = 0;
  double *wgc = nullptr, *wGpk = nullptr, *wac = nullptr;
  unsigned* wtick = nullptr;       // the epilogue ticket
  int w_gram_grid = 8;
  // adaptive rank prediction (Eq. 7): parameters; the state lives in DevState
  int ap_a = 0;
  double ap_rho = 0.0, ap_gamma = 0.0;
  int64_t ap_n = -1;               // short side the device state was set up for
  std::string err;
  // tracing: CUDA events around every launch when enabled
  int timing = 0;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<int> ev_phase;      // phase of the pair (2k, 2k+1)
  size_t ev_used = 0;             // events recorded since the last collection
  double phase_ms[FRSVT_NPHASE] = {0};
  int32_t phase_launches[FRSVT_NPHASE] = {0};
};

namespace {

constexpr size_t kSmemLimit = 227 * 1024;
const float kNoResidual = -1.f;    // DevState::rp_res before any range-propagated sketch (static storage: async copy)

frsvt_status fail(frsvt_handle* h, frsvt_status s, const std::string& msg) {
  if (h) h->err = msg;
  return s;
}

#define FRSVT_CK(call)                                                              \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) return fail(h, FRSVT_ERR_CUDA, std::string(#call ": ") + \
                                       cudaGetErrorString(e_));                     \
  } while (0)

constexpr size_t kEventPairs = 2048;

frsvt_status collect_timings(frsvt_handle* h) {
  if (h->ev_used == 0) return FRSVT_OK;
  FRSVT_CK(cudaStreamSynchronize(h->stream));
  for (size_t k = 0; k + 1 < h->ev_used; k += 2) {
    float ms = 0.f;
    FRSVT_CK(cudaEventElapsedTime(&ms, h->ev_pool[k], h->ev_pool[k + 1]));
    const int ph = h->ev_phase[k / 2];
    h->phase_ms[ph] += ms;
    h->phase_launches[ph] += 1;
  }
  h->ev_used = 0;
  return FRSVT_OK;
}

// Launch `call` as phase `ph`, bracketed by events when tracing is on.
#define FRSVT_LAUNCH(ph, call)                                                       \
  do {                                                                               \
    if (h->timing) {                                                                 \
      if (h->ev_used + 2 > h->ev_pool.size()) {                                      \
        frsvt_status cs_ = collect_timings(h);                                       \
        if (cs_ != FRSVT_OK) return cs_;                                             \
      }                                                                              \
      h->ev_phase[h->ev_used / 2] = (ph);                                            \
      FRSVT_CK(cudaEventRecord(h->ev_pool[h->ev_used], h->stream));                  \
    }                                                                                \
    FRSVT_CK(call);                                                                  \
    if (h->timing) {                                                                 \
      FRSVT_CK(cudaEventRecord(h->ev_pool[h->ev_used + 1], h->stream));              \
      h->ev_used += 2;                                                               \
    }                                                                                \
  } while (0)

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link against libcuda).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (fn == nullptr) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 2-D float32 tensor map of a row-major rows x cols matrix (leading dimension ld) with
// box_rows x box_cols boxes, no swizzle, zero fill outside the matrix.
bool make_row_map(CUtensorMap* map, const float* base, int64_t rows, int64_t cols, int64_t ld, int box_cols,
                  int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (enc == nullptr) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * sizeof(float)};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(box_cols), static_cast<cuuint32_t>(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Same with 32-column (128-byte) boxes in a 128-byte swizzle: 16-byte chunks (read by tcgen05 as a
// K-major operand) or, with sw = CU_TENSOR_MAP_SWIZZLE_128B_ATOM_32B, 32-byte chunks (the layout a
// kind::tf32 MMA takes for an MN-major operand).
bool make_row_map_sw128(CUtensorMap* map, const float* base, int64_t rows, int64_t cols, int64_t ld, int box_rows,
                        CUtensorMapSwizzle sw = CU_TENSOR_MAP_SWIZZLE_128B) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (enc == nullptr) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * sizeof(float)};
  cuuint32_t box[2] = {32u, static_cast<cuuint32_t>(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// BF16 row-major matrix, boxes of 64 columns (128 bytes) x box_rows in the 128-byte swizzle.
bool make_row_map_bf16(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (enc == nullptr) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * 2u};
  cuuint32_t box[2] = {64u, static_cast<cuuint32_t>(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 8-bit row-major matrix (the E4M3 shadow), box_cols x box_rows boxes, no swizzle.
bool make_row_map_u8(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_cols,
                     int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (enc == nullptr) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld)};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(box_cols), static_cast<cuuint32_t>(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int g_tc_prepared = 0;

int64_t ns_limit(int LP) {
  // short-side rows that fit the single-CTA orthonormalisation and the staged Q of the row pass
  const int64_t by_orth = (static_cast<int64_t>(kSmemLimit) - static_cast<int64_t>(orth_smem_bytes(LP, 0))) /
                          (LP * static_cast<int64_t>(sizeof(float)));
  const int64_t by_rows = static_cast<int64_t>(kSmemLimit) / (LP * static_cast<int64_t>(sizeof(float)));
  return by_orth < by_rows ? by_orth : by_rows;
}

struct Splits {
  int nsplit;
  int64_t rps;
  int ntiles;
};

Splits row_splits(const frsvt_handle* h, int64_t m, int64_t n) {
  Splits s;
  s.ntiles = static_cast<int>(cdiv(n, 256));
  int64_t ns = cdiv(h->target_ctas, s.ntiles);
  const int64_t by_rows = cdiv(m, 32);
  if (ns > by_rows) ns = by_rows;
  if (ns < 1) ns = 1;
  int64_t rps = cdiv(m, ns);
  rps = cdiv(rps, 32) * 32;
  s.rps = rps;
  s.nsplit = static_cast<int>(cdiv(m, rps));
  if (s.nsplit < 1) s.nsplit = 1;
  return s;
}

int gram_splits(const frsvt_handle* h, int64_t m) {
  int64_t g = cdiv(m, 32);
  if (g > h->gsplit_max) g = h->gsplit_max;
  if (g < 1) g = 1;
  return static_cast<int>(g);
}

// Row splits of the fused passes: a multiple of the cluster size (8).
Splits fused_splits(const frsvt_handle* h, int64_t m, int64_t n) {
  Splits s;
  s.ntiles = static_cast<int>(cdiv(n, 256));
  int64_t ns = cdiv(cdiv(h->target_ctas, s.ntiles), 8) * 8;
  const int64_t by_rows = cdiv(cdiv(m, 32), 8) * 8;
  if (ns > by_rows) ns = by_rows;
  if (ns < 8) ns = 8;
  s.rps = cdiv(cdiv(m, ns), 32) * 32;
  s.nsplit = static_cast<int>(ns);
  return s;
}

frsvt_status check_matrix(frsvt_handle* h, const void* p, int64_t m, int64_t n, int64_t ld, const char* name) {
  if (m == 0 || n == 0) return FRSVT_OK;
  if (p == nullptr) return fail(h, FRSVT_ERR_INVALID_ARG, std::string(name) + " is NULL");
  if (!aligned16(p)) return fail(h, FRSVT_ERR_INVALID_ARG, std::string(name) + " is not 16-byte aligned");
  if (ld < n || (ld % 4) != 0)
    return fail(h, FRSVT_ERR_INVALID_ARG, std::string(name) + ": leading dimension must be >= n and a multiple of 4");
  return FRSVT_OK;
}

frsvt_status check_shape(frsvt_handle* h, int64_t m, int64_t n) {
  if (m < 0 || n < 0) return fail(h, FRSVT_ERR_INVALID_ARG, "negative size");
  if (m < n && !h->wide)
    return fail(h, FRSVT_ERR_UNSUPPORTED, "m < n is served by the wide-basis handle (l_max > 32) only");
  if (m > h->cfg.m_max || n > h->cfg.n_max)
    return fail(h, FRSVT_ERR_INVALID_ARG, "problem larger than the handle's m_max / n_max");
  return FRSVT_OK;
}

// Alg. 1 up to the core SVD: sketch (steps 3-12), q power steps (13-15),
// projection and the l x l core (16-19).  Leaves Z in h->Zl and Rf in h->Rf
// so that X = Z Rf^T.
frsvt_status range_and_core(frsvt_handle* h, const float* A, int64_t m, int64_t n, int64_t lda, int l, int q,
                            int use_rp, uint64_t ctr, float tau_host, int tau_from_mu, int update_rp,
                            int advance_counter, const void* Ab = nullptr) {
  const int LP = h->LP;
  cudaStream_t st = h->stream;
  const double tol = h->cfg.rank_tol;
  if (h->tma && n <= 256 && m < (int64_t(1) << 31)) {
    CUtensorMap tmA, tmAl, tmZ;
    if (!make_row_map(&tmA, A, m, n, lda, tma_np4(n), tma_rows_per_tile()) ||
        !make_row_map(&tmAl, A, m, n, lda, tma_np4(n), tma_rows_per_tile_lr()) ||
        !make_row_map(&tmZ, h->Zl, m, LP, LP, LP, tma_rows_per_tile()))
      return fail(h, FRSVT_ERR_CUDA, "cuTensorMapEncodeTiled failed for A / Z");
    const int G = h->tma_grid;
    const int64_t rpc = cdiv(cdiv(m, G), tma_rows_per_tile()) * tma_rows_per_tile();
    const int64_t rpl = cdiv(cdiv(m, G), tma_rows_per_tile_lr()) * tma_rows_per_tile_lr();
    const int nst = tma_lr_stages(LP, n, kSmemLimit - 16384);
    // Column passes (A^T Omega, A^T Z): on the tensor cores when the handle prepared them, with A
    // read MN-major (32-byte-atom swizzle) and Omega / Z as the K-major operand.
    const bool tcc = h->tc_sc_ns > 0;
    CUtensorMap tmAc, tmZc;
    if (tcc && (!make_row_map_sw128(&tmAc, A, m, n, lda, tc_sc_rows(), CU_TENSOR_MAP_SWIZZLE_128B_ATOM_32B) ||
                !make_row_map(&tmZc, h->Zl, m, LP, LP, LP, tc_sc_rows())))
      return fail(h, FRSVT_ERR_CUDA, "cuTensorMapEncodeTiled failed for A / Z (column pass)");
    // Reduced precision (a BF16 shadow Ab of A is current): the sketch and the first q - 1 power
    // steps read Ab; the last power step and the projection stay FP32-accurate.
    const bool bf = Ab != nullptr && h->tb_sc_ns > 0;
    CUtensorMap tmBr, tmBc, tmZb;
    if (bf && (!make_row_map_bf16(&tmBr, Ab, m, n, h->ldb, tb_box_rows_lr()) ||
               !make_row_map_bf16(&tmBc, Ab, m, n, h->ldb, tb_box_rows_sc()) ||
               !make_row_map(&tmZb, h->Zl, m, LP, LP, LP, tb_box_rows_sc())))
      return fail(h, FRSVT_ERR_CUDA, "cuTensorMapEncodeTiled failed for the BF16 shadow");
    if (bf)
      FRSVT_LAUNCH(FRSVT_PHASE_SKETCH, launch_tb_sc(LP, tmBc, nullptr, m, n, h->tb_sc_grid, h->tb_sc_ns, h->cfg.seed,
                                                    ctr, h->dst, h->cpart_sc, h->Ys, h->tickets, l, use_rp,
                                                    q == 0 ? 2 : 1, h->Qt, h->Qs, tol, st));
    else if (tcc)
      FRSVT_LAUNCH(FRSVT_PHASE_SKETCH, launch_tc_sc(LP, tmAc, nullptr, m, n, h->tc_sc_grid, h->tc_sc_ns, h->cfg.seed,
                                                    ctr, h->dst, h->cpart_sc, h->Ys, h->tickets, true, l, use_rp,
                                                    q == 0 ? 2 : 1, h->Qt, h->Qs, tol, st));
    else
      FRSVT_LAUNCH(FRSVT_PHASE_SKETCH, launch_tp_sc(LP, tmA, nullptr, m, n, rpc, G, h->cfg.seed, ctr, h->dst,
                                                    h->cpart_sc, h->Ys, h->tickets, l, use_rp, q == 0 ? 2 : 1, h->Qt,
                                                    h->Qs, tol, st));
    CUtensorMap tmAs;                       // 128-byte swizzled boxes for the tensor-core row pass
    if (!make_row_map_sw128(&tmAs, A, m, n, lda, tc_box_rows()))
      return fail(h, FRSVT_ERR_CUDA, "cuTensorMapEncodeTiled failed for A (swizzled)");
    const float* qin = h->Qs;                 // basis read by the next A Q pass
    for (int it = 0; it < q; ++it) {
      const int passes = it == q - 1 ? 2 : 1;
      if (bf && it < q - 1) {
        FRSVT_LAUNCH(FRSVT_PHASE_POWER_AQ, launch_tb_lr(LP, tmBr, m, n, h->sms, h->tb_lr_ns, h->Qs, h->Zl, h->dst, st));
        FRSVT_LAUNCH(FRSVT_PHASE_POWER_ATZ, launch_tb_sc(LP, tmBc, &tmZb, m, n, h->tb_sc_grid, h->tb_sc_ns,
                                                         h->cfg.seed, ctr, h->dst, h->cpart_sc, h->Ys, h->tickets, l,
                                                         0, passes, h->Qt, h->Qs, tol, st));
        continue;
      }
      FRSVT_LAUNCH(FRSVT_PHASE_POWER_AQ, launch_tc_lr(LP, tmAs, m, n, h->sms, h->tc_lr_ns, qin, h->Zl, h->dst, st,
                                                      qin == h->Ys ? 1 : 0));
      // Sec. 2.5: with FRSVT_CFG_ORTH_LAST the intermediate power steps skip the orthonormalisation
      // and the next A Q pass reads Y = A^T Z itself (same span)
      const bool skip = tcc && (h->cfg.flags & FRSVT_CFG_ORTH_LAST) && it < q - 1;
      qin = skip ? h->Ys : h->Qs;
      if (tcc)
        FRSVT_LAUNCH(FRSVT_PHASE_POWER_ATZ, launch_tc_sc(LP, tmAc, &tmZc, m, n, h->tc_sc_grid, h->tc_sc_ns,
                                                         h->cfg.seed, ctr, h->dst, h->cpart_sc, h->Ys, h->tickets,
                                                         !skip, l, 0, passes, h->Qt, h->Qs, tol, st));
      else
        FRSVT_LAUNCH(FRSVT_PHASE_POWER_ATZ, launch_tp_sc(LP, tmA, &tmZ, m, n, rpc, G, h->cfg.seed, ctr, h->dst,
                                                         h->cpart_sc, h->Ys, h->tickets, l, 0, passes, h->Qt, h->Qs,
                                                         tol, st));
    }
    // Projection B^T = Z = A Q on the tensor cores, then B B^T = Z^T Z and the core (steps 16-19).
    FRSVT_LAUNCH(FRSVT_PHASE_PROJECT, launch_tc_lr(LP, tmAs, m, n, h->sms, h->tc_lr_ns, h->Qs, h->Zl, h->dst, st));
    FRSVT_LAUNCH(FRSVT_PHASE_CORE, launch_gram_core(LP, h->Zl, m, n, h->gram_grid, h->Qs, h->cpart_lr, h->Gfin,
                                                    h->tickets, l, tau_host, tau_from_mu, update_rp, advance_counter,
                                                    h->Rf, h->Qt, h->dst, tol, h->cfg.max_jacobi_sweeps, st));
    (void)rpl;
    (void)nst;
    (void)tmAl;
    return FRSVT_OK;
  }
  if (h->fused) {
    const Splits fs = fused_splits(h, m, n);
    FRSVT_LAUNCH(FRSVT_PHASE_SKETCH, launch_sc_orth(LP, A, m, n, lda, nullptr, h->cfg.seed, ctr, h->dst, fs.nsplit,
                                                    fs.rps, h->cpart_sc, h->Ys, h->tickets, l, use_rp, h->Qt, h->Qs,
                                                    tol, st));
    for (int it = 0; it < q; ++it) {
      FRSVT_LAUNCH(FRSVT_PHASE_POWER_AQ, launch_lr(LP, false, A, m, n, lda, h->Qs, h->Zl, h->lr_blocks, h->cpart_lr,
                                                   h->Gfin, h->tickets, l, 0.f, 0, 0, 0, h->Rf, h->Qt, h->dst, tol,
                                                   h->cfg.max_jacobi_sweeps, st));
      FRSVT_LAUNCH(FRSVT_PHASE_POWER_ATZ, launch_sc_orth(LP, A, m, n, lda, h->Zl, h->cfg.seed, ctr, h->dst,
                                                         fs.nsplit, fs.rps, h->cpart_sc, h->Ys, h->tickets, l, 0,
                                                         h->Qt, h->Qs, tol, st));
    }
    FRSVT_LAUNCH(FRSVT_PHASE_PROJECT, launch_lr(LP, true, A, m, n, lda, h->Qs, h->Zl, h->lr_blocks, h->cpart_lr,
                                                h->Gfin, h->tickets, l, tau_host, tau_from_mu, update_rp,
                                                advance_counter, h->Rf, h->Qt, h->dst, tol,
                                                h->cfg.max_jacobi_sweeps, st));
    return FRSVT_OK;
  }
  const Splits sp = row_splits(h, m, n);
  FRSVT_LAUNCH(FRSVT_PHASE_SKETCH, launch_short_cols(LP, A, m, n, lda, nullptr, h->cfg.seed, ctr, h->dst, h->part,
                                                     sp.nsplit, sp.rps, st));
  FRSVT_LAUNCH(FRSVT_PHASE_REDUCE, launch_reduce_parts(h->part, sp.nsplit, n * LP, h->Ys, st));
  FRSVT_LAUNCH(FRSVT_PHASE_ORTH, launch_orth(LP, h->Ys, n, l, use_rp, h->Qt, h->Qs, h->dst, tol, st));
  for (int it = 0; it < q; ++it) {
    FRSVT_LAUNCH(FRSVT_PHASE_POWER_AQ, launch_long_rows(LP, A, m, n, lda, h->Qs, h->Zl, 8 * h->sms, st));
    FRSVT_LAUNCH(FRSVT_PHASE_POWER_ATZ, launch_short_cols(LP, A, m, n, lda, h->Zl, h->cfg.seed, ctr, h->dst, h->part,
                                                          sp.nsplit, sp.rps, st));
    FRSVT_LAUNCH(FRSVT_PHASE_REDUCE, launch_reduce_parts(h->part, sp.nsplit, n * LP, h->Ys, st));
    FRSVT_LAUNCH(FRSVT_PHASE_ORTH, launch_orth(LP, h->Ys, n, l, 0, h->Qt, h->Qs, h->dst, tol, st));
  }
  FRSVT_LAUNCH(FRSVT_PHASE_PROJECT, launch_long_rows(LP, A, m, n, lda, h->Qs, h->Zl, 8 * h->sms, st));
  const int gs = gram_splits(h, m);
  FRSVT_LAUNCH(FRSVT_PHASE_GRAM, launch_gram_long(LP, h->Zl, m, h->gpart, gs, st));
  FRSVT_LAUNCH(FRSVT_PHASE_CORE, launch_core(LP, h->gpart, gs, h->Qs, n, l, tau_host, tau_from_mu, update_rp,
                                             advance_counter, h->Rf, h->Qt, h->dst, tol, h->cfg.max_jacobi_sweeps, st));
  return FRSVT_OK;
}

frsvt_status sync_rp_shape(frsvt_handle* h, int64_t m, int64_t n, int l) {
  if (h->last_m != m || h->last_n != n || h->last_l != l) {
    FRSVT_CK(cudaMemsetAsync(&h->dst->keep, 0, sizeof(int32_t), h->stream));
    h->last_m = m;
    h->last_n = n;
    h->last_l = l;
  }
  return FRSVT_OK;
}

void free_all(frsvt_handle* h) {
  for (frsvt_handle* k : h->kids) frsvt_destroy(k);
  h->kids.clear();
  for (cudaStream_t s : h->kid_streams) cudaStreamDestroy(s);
  h->kid_streams.clear();
  for (cudaEvent_t e : h->kid_events) cudaEventDestroy(e);
  h->kid_events.clear();
  if (h->fork_event) cudaEventDestroy(h->fork_event);
  h->fork_event = nullptr;
  for (auto& g : h->step_exec) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
  }
  if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
  h->capture_stream = nullptr;
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  h->ev_pool.clear();
  void* ptrs[] = {h->dst, h->Ys,       h->Qs,       h->Qt,        h->Zl,   h->Rf,   h->part,    h->gpart,
                  h->rpart, h->pmax,   h->psum,     h->cpart_sc,  h->cpart_lr, h->cpart_alm, h->Gfin, h->rsum,
                  h->tickets, h->wsvt_next, h->ad_ws, h->Ab,
                  h->wOT, h->wOTl, h->wZT, h->wZTl, h->wZ, h->wZl, h->wYT, h->wQT, h->wQTl, h->wQp, h->wRf,
                  h->wRfl, h->wT1, h->wT2, h->wI, h->wpart, h->wgc, h->wGpk, h->wac, h->wtick,
                  h->wOTb, h->wOTbl, h->wZTb, h->wZTbl, h->wQTb, h->wQTbl, h->A8, h->w8s};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

// ---------------------------------------------------------------- wide basis (32 < l <= 128)
// Orientation (reading R1): the basis lives on the short side of A.  For m >= n (tall) the short
// side is the columns, and the passes over A are the column pass (reduce over the rows, output on
// the column side) and the row pass (reduce over the columns, output on the row side); for m < n
// (wide) the same two kernels swap roles, with no copy of A.  Basis-side matrices (Y^T, Q^T) have
// ns = min(m, n) columns (stride w_lds), long-side ones (Omega^T, Z^T, Z) nl = max(m, n) (w_ldl).

// Orthonormal basis of the columns of Y (given transposed, 128 x ns at h->wYT) into QT / QTl:
// Cholesky QR, `passes` times (Alg. 1 steps 6 / 14; only span(Q) matters, Prop. 1).
// With bf_next the basis is also written as BF16 hi / lo parts (the next pass reads the shadow).
frsvt_status wide_orth(frsvt_handle* h, int64_t ns, int l, int passes, bool bf_next) {
  cudaStream_t st = h->stream;
  const int64_t ld = h->w_lds;
  for (int pass = 0; pass < passes; ++pass) {
    const float* src = pass == 0 ? h->wYT : h->wQT;
    const bool last = pass == passes - 1;
    FRSVT_LAUNCH(FRSVT_PHASE_ORTH, launch_wd_gram(false, src, ld, ns, h->w_gram_grid, h->wgc, h->wGpk, l,
                                                  h->cfg.rank_tol, l, 0.f, 0, 0, 0, h->cfg.max_jacobi_sweeps, h->wT1,
                                                  h->wT2, h->dst, st));
    FRSVT_LAUNCH(FRSVT_PHASE_APPLY, launch_wd_trsm(src, ld, ns, h->wT1, h->wQT, h->wQTl,
                                                  (bf_next && last) ? h->wQTb : nullptr,
                                                  (bf_next && last) ? h->wQTbl : nullptr, ld, st));
  }
  return FRSVT_OK;
}

// Alg. 1 up to the core on the wide basis: leaves Z / Z_lo (nl x 128) and Rf / Rf_lo (ns x 128)
// so that X = Z Rf^T (tall) or X = Rf Z^T (wide), and sets r, s, sigma (and the counter) in the
// device state.  Shadow the reduced-precision passes read: 0 none, 1 the BF16 shadow (kept current
// by rpca_init, frsvt_svt and the epilogue), 2 the E4M3 shadow (quantized at the start of each SVT).
int wide_lowp(const frsvt_handle* h) { return h->A8 != nullptr ? 2 : (h->Ab != nullptr ? 1 : 0); }

// Reduced precision (lowp, see wide_lowp): the sketch and the first q - 1 power steps
// read the shadow with BF16 copies of the narrow factors; the last power step and the projection
// stay FP32-accurate.
// use_rp: range propagation (Alg. 1 steps 8-11): the sketch takes l - keep new columns and the
// propagated basis Q~ of the previous call (wQp, Q~^T), and the core leaves the next Q~.
// orth_last_ok: the SVT calls honour FRSVT_CFG_ORTH_LAST; the spectral-norm estimate (up to 64
// power steps, whose unnormalised growth sigma_1^(2 q) would overflow FP32) always
// orthonormalises.
frsvt_status wide_range_and_core(frsvt_handle* h, const float* A, int64_t m, int64_t n, int64_t lda, int l, int q,
                                 uint64_t ctr, float tau_host, int tau_from_mu, int advance_counter, int lowp = 0,
                                 int use_rp = 0, bool orth_last_ok = false) {
  cudaStream_t st = h->stream;
  const int64_t LW = wide_lp();
  const bool tall = m >= n;
  const int64_t nl = tall ? m : n, ns = tall ? n : m;
  const int64_t ldl = h->w_ldl, lds = h->w_lds;
  CUtensorMap tmAr, tmAc, tmOT, tmOTl, tmZT, tmZTl, tmQT, tmQTl;
  if (!make_row_map_sw128(&tmAr, A, m, n, lda, wide_tile()) ||
      !make_row_map_sw128(&tmAc, A, m, n, lda, 32, CU_TENSOR_MAP_SWIZZLE_128B_ATOM_32B) ||
      !make_row_map_sw128(&tmOT, h->wOT, LW, nl, ldl, 128) ||
      !make_row_map_sw128(&tmOTl, h->wOTl, LW, nl, ldl, 128) ||
      !make_row_map_sw128(&tmZT, h->wZT, LW, nl, ldl, 128) ||
      !make_row_map_sw128(&tmZTl, h->wZTl, LW, nl, ldl, 128) ||
      !make_row_map_sw128(&tmQT, h->wQT, LW, ns, lds, 128) ||
      !make_row_map_sw128(&tmQTl, h->wQTl, LW, ns, lds, 128))
    return fail(h, FRSVT_ERR_CUDA, "cuTensorMapEncodeTiled failed (wide basis)");
  const bool bf = lowp != 0;
  CUtensorMap tmBr, tmBc, tmOTb, tmOTbl, tmZTb, tmZTbl, tmQTb, tmQTbl;
  if (lowp == 2) {
    if (!make_row_map_u8(&tmBr, h->A8, m, n, h->ld8, 64, wide_tile()) ||
        !make_row_map_u8(&tmBc, h->A8, m, n, h->ld8, wide_tile(), 64))
      return fail(h, FRSVT_ERR_CUDA, "cuTensorMapEncodeTiled failed (wide basis, FP8 shadow)");
    FRSVT_LAUNCH(FRSVT_PHASE_SKETCH, launch_wd_quant8(A, lda, m, n, h->A8, h->ld8, h->w8s, st));
  } else if (lowp == 1 && (!make_row_map_bf16(&tmBr, h->Ab, m, n, h->ldb, wide_tile()) ||
                           !make_row_map_bf16(&tmBc, h->Ab, m, n, h->ldb, 64)))
    return fail(h, FRSVT_ERR_CUDA, "cuTensorMapEncodeTiled failed (wide basis, BF16 shadow)");
  const float* sc8 = lowp == 2 ? h->w8s : nullptr;
  const int ntr8 = static_cast<int>(cdiv(m, 128)), ntc8 = static_cast<int>(cdiv(n, 128));
  if (bf && (!make_row_map_bf16(&tmOTb, h->wOTb, LW, nl, ldl, 128) ||
             !make_row_map_bf16(&tmOTbl, h->wOTbl, LW, nl, ldl, 128) ||
             !make_row_map_bf16(&tmZTb, h->wZTb, LW, nl, ldl, 128) ||
             !make_row_map_bf16(&tmZTbl, h->wZTbl, LW, nl, ldl, 128) ||
             !make_row_map_bf16(&tmQTb, h->wQTb, LW, ns, lds, 128) ||
             !make_row_map_bf16(&tmQTbl, h->wQTbl, LW, ns, lds, 128)))
    return fail(h, FRSVT_ERR_CUDA, "cuTensorMapEncodeTiled failed (wide basis, BF16 factors)");
  // P_short reduces over the long side of A (output on the basis side: Y^T = M^T A or M^T A^T),
  // P_long reduces over the short side (output on the long side: Z^T = Q^T A^T or Q^T A)
  const bool short_col = tall;                   // P_short is the column pass for a tall A
  const CUtensorMap& tmS = short_col ? tmAc : tmAr;
  const CUtensorMap& tmL = short_col ? tmAr : tmAc;
  const CUtensorMap& tmSb = short_col ? tmBc : tmBr;
  const CUtensorMap& tmLb = short_col ? tmBr : tmBc;
  FRSVT_LAUNCH(FRSVT_PHASE_SKETCH, launch_wd_omega(h->wOT, h->wOTl, bf ? h->wOTb : nullptr, bf ? h->wOTbl : nullptr,
                                                   ldl, nl, l, use_rp, h->cfg.seed, ctr, h->dst, st));
  if (bf)
    FRSVT_LAUNCH(FRSVT_PHASE_SKETCH, launch_wd_pass(short_col, lowp, tmSb, tmOTb, tmOTbl, ns, nl, h->sms, h->wpart,
                                                    h->w_ldp, h->wYT, nullptr, nullptr, nullptr, lds, nullptr,
                                                    nullptr, h->dst, st, sc8, ntr8, ntc8));
  else
    FRSVT_LAUNCH(FRSVT_PHASE_SKETCH, launch_wd_pass(short_col, 0, tmS, tmOT, tmOTl, ns, nl, h->sms, h->wpart, h->w_ldp,
                                                    h->wYT, nullptr, nullptr, nullptr, lds, nullptr,
                                                    nullptr, h->dst, st));
  if (use_rp) FRSVT_LAUNCH(FRSVT_PHASE_SKETCH, launch_wd_rp_insert(h->wYT, h->wQp, lds, ns, l, h->dst, st));
  frsvt_status s = wide_orth(h, ns, l, q == 0 ? 2 : 1, bf && q > 1);
  if (s != FRSVT_OK) return s;
  const bool orth_last = orth_last_ok && (h->cfg.flags & FRSVT_CFG_ORTH_LAST) != 0;
  for (int it = 0; it < q; ++it) {
    if (bf && it < q - 1) {
      FRSVT_LAUNCH(FRSVT_PHASE_POWER_AQ, launch_wd_pass(!short_col, lowp, tmLb, tmQTb, tmQTbl, nl, ns, h->sms, h->wpart,
                                                        h->w_ldp, nullptr, nullptr, h->wZTb, h->wZTbl, ldl,
                                                        nullptr, nullptr, h->dst, st, sc8, ntr8, ntc8));
      FRSVT_LAUNCH(FRSVT_PHASE_POWER_ATZ, launch_wd_pass(short_col, lowp, tmSb, tmZTb, tmZTbl, ns, nl, h->sms, h->wpart,
                                                         h->w_ldp, h->wYT, nullptr, nullptr, nullptr, lds,
                                                         nullptr, nullptr, h->dst, st, sc8, ntr8, ntc8));
    } else {
      FRSVT_LAUNCH(FRSVT_PHASE_POWER_AQ, launch_wd_pass(!short_col, 0, tmL, tmQT, tmQTl, nl, ns, h->sms, h->wpart,
                                                        h->w_ldp, h->wZT, h->wZTl, nullptr, nullptr, ldl,
                                                        nullptr, nullptr, h->dst, st));
      FRSVT_LAUNCH(FRSVT_PHASE_POWER_ATZ, launch_wd_pass(short_col, 0, tmS, tmZT, tmZTl, ns, nl, h->sms, h->wpart,
                                                         h->w_ldp, h->wYT, nullptr, nullptr, nullptr, lds,
                                                         nullptr, nullptr, h->dst, st));
    }
    if (orth_last && it < q - 1) {
      // Sec. 2.5: the intermediate power step passes Y = A A^T Q on without orthonormalising it (same
      // span): Q = Y with each column scaled by a power of two (exact; keeps FP32 in range), split
      // into its TF32 parts (and BF16 copies) by the substitution kernel with that diagonal T
      const bool bfn = bf && it + 1 < q - 1;
      FRSVT_LAUNCH(FRSVT_PHASE_APPLY, launch_wd_colscale(h->wYT, lds, ns, h->wI, st));
      FRSVT_LAUNCH(FRSVT_PHASE_APPLY, launch_wd_trsm(h->wYT, lds, ns, h->wI, h->wQT, h->wQTl, bfn ? h->wQTb : nullptr,
                                                    bfn ? h->wQTbl : nullptr, lds, st));
      continue;
    }
    if ((s = wide_orth(h, ns, l, it == q - 1 ? 2 : 1, bf && it + 1 < q - 1)) != FRSVT_OK) return s;
  }
  // projection B^T = Z (step 16), then B B^T = Z^T Z and the core (steps 16-19)
  FRSVT_LAUNCH(FRSVT_PHASE_PROJECT, launch_wd_pass(!short_col, 0, tmL, tmQT, tmQTl, nl, ns, h->sms, h->wpart, h->w_ldp,
                                                   h->wZT, nullptr, nullptr, nullptr, ldl, h->wZ, h->wZl,
                                                   h->dst, st));
  FRSVT_LAUNCH(FRSVT_PHASE_CORE, launch_wd_gram(true, h->wZT, ldl, nl, h->w_gram_grid, h->wgc, h->wGpk,
                                                l, h->cfg.rank_tol, l, tau_host, tau_from_mu, use_rp,
                                                advance_counter, h->cfg.max_jacobi_sweeps, h->wT1, h->wT2, h->dst,
                                                st));
  FRSVT_LAUNCH(FRSVT_PHASE_APPLY, launch_wd_apply(h->wQT, lds, ns, h->wT1, nullptr, nullptr, 0, h->wRf, h->wRfl,
                                                 st));
  if (use_rp)                                    // step 21: Q~ = Q U_B[:, :keep], kept as Q~^T
    FRSVT_LAUNCH(FRSVT_PHASE_APPLY, launch_wd_apply(h->wQT, lds, ns, h->wT2, h->wQp, nullptr, lds, nullptr, nullptr,
                                                   st));
  return FRSVT_OK;
}

// X = Z Rf^T (tall) or Rf Z^T (wide): written to L (alm = false) or fused with the iALM update
// (alm = true).  The epilogue kernel forms X[i][j] = sum_k P[i][k] Q[j][k] for its row factor P
// (m x 128) and column factor Q (n x 128): (Z, Rf) for a tall A, (Rf, Z) for a wide one.
frsvt_status wide_epilogue(frsvt_handle* h, bool alm, int64_t m, int64_t n, const float* O, float* S, float* A,
                           int64_t ld, float* L, int64_t ldl) {
  const bool tall = m >= n;
  const float* P = tall ? h->wZ : h->wRf;
  const float* Pl = tall ? h->wZl : h->wRfl;
  const float* Qf = tall ? h->wRf : h->wZ;
  const float* Ql = tall ? h->wRfl : h->wZl;
  CUtensorMap tmZ, tmZl, tmR, tmRl;
  if (!make_row_map_sw128(&tmZ, P, m, wide_lp(), wide_lp(), 128) ||
      !make_row_map_sw128(&tmZl, Pl, m, wide_lp(), wide_lp(), 128) ||
      !make_row_map_sw128(&tmR, Qf, n, wide_lp(), wide_lp(), wide_tile()) ||
      !make_row_map_sw128(&tmRl, Ql, n, wide_lp(), wide_lp(), wide_tile()))
    return fail(h, FRSVT_ERR_CUDA, "cuTensorMapEncodeTiled failed (wide epilogue)");
  const int64_t ntiles = cdiv(m, 128) * cdiv(n, wide_tile());
  const int grid = static_cast<int>(ntiles < h->sms ? ntiles : h->sms);
  FRSVT_LAUNCH(FRSVT_PHASE_EPILOGUE, launch_wd_alm(alm, tmZ, tmZl, tmR, tmRl, m, n, O, S, A, ld, L, ldl, h->dst,
                                                   h->wac, h->wtick, grid, alm ? h->Ab : nullptr,
                                                   h->ldb, h->stream));
  return FRSVT_OK;
}

// Workspace of a wide handle (sizes from the configuration); false on an allocation failure.
bool wide_alloc(frsvt_handle* h) {
  const frsvt_config* cfg = &h->cfg;
  const int64_t T = wide_tile(), LW = wide_lp();
  const int64_t lmax = cfg->m_max > cfg->n_max ? cfg->m_max : cfg->n_max;   // long side of any served problem
  const int64_t smax = cfg->m_max < cfg->n_max ? cfg->m_max : cfg->n_max;   // short side
  h->w_ldl = cdiv(lmax, T) * T;
  h->w_lds = cdiv(smax, T) * T;
  h->w_ldp = h->w_ldl;
  h->w_gram_grid = wide_gram_grid();
  if (h->w_gram_grid < 1) h->w_gram_grid = 1;
  bool ok = true;
  auto alloc = [&](void** p, size_t bytes) {
    if (ok && cudaMalloc(p, bytes < 16 ? 16 : bytes) != cudaSuccess) ok = false;
  };
  const size_t fm = sizeof(float) * LW * h->w_ldl, fn = sizeof(float) * LW * h->w_lds;
  alloc(reinterpret_cast<void**>(&h->wOT), fm);
  alloc(reinterpret_cast<void**>(&h->wOTl), fm);
  alloc(reinterpret_cast<void**>(&h->wZT), fm);
  alloc(reinterpret_cast<void**>(&h->wZTl), fm);
  alloc(reinterpret_cast<void**>(&h->wZ), fm);
  alloc(reinterpret_cast<void**>(&h->wZl), fm);
  alloc(reinterpret_cast<void**>(&h->wYT), fn);
  alloc(reinterpret_cast<void**>(&h->wQT), fn);
  alloc(reinterpret_cast<void**>(&h->wQTl), fn);
  alloc(reinterpret_cast<void**>(&h->wQp), fn);
  alloc(reinterpret_cast<void**>(&h->wRf), fn);
  alloc(reinterpret_cast<void**>(&h->wRfl), fn);
  alloc(reinterpret_cast<void**>(&h->wT1), sizeof(float) * LW * LW);
  alloc(reinterpret_cast<void**>(&h->wT2), sizeof(float) * LW * LW);
  alloc(reinterpret_cast<void**>(&h->wI), sizeof(float) * LW * LW);
  alloc(reinterpret_cast<void**>(&h->wpart), sizeof(float) * 8 * LW * h->w_ldp);   // 8 partial planes per pass tile
  alloc(reinterpret_cast<void**>(&h->wgc), sizeof(double) * h->w_gram_grid * wide_gram_count());
  alloc(reinterpret_cast<void**>(&h->wGpk), sizeof(double) * wide_gram_count());
  alloc(reinterpret_cast<void**>(&h->wac), sizeof(double) * (h->sms > 0 ? h->sms : 1));
  alloc(reinterpret_cast<void**>(&h->wtick), sizeof(unsigned));
  alloc(reinterpret_cast<void**>(&h->dst), sizeof(DevState));
  alloc(reinterpret_cast<void**>(&h->pmax), sizeof(float) * h->absmax_blocks);
  alloc(reinterpret_cast<void**>(&h->psum), sizeof(float2) * h->absmax_blocks);
  alloc(reinterpret_cast<void**>(&h->wsvt_next), sizeof(unsigned));
  if (cfg->precision == FRSVT_PREC_BF16 || cfg->precision == FRSVT_PREC_FP8) {
    const size_t bm = sizeof(uint16_t) * LW * h->w_ldl, bn = sizeof(uint16_t) * LW * h->w_lds;
    if (cfg->precision == FRSVT_PREC_BF16) {
      h->ldb = (cfg->n_max + 7) / 8 * 8;
      alloc(&h->Ab, sizeof(uint16_t) * static_cast<size_t>(cfg->m_max) * h->ldb);
    } else {
      h->ld8 = (cfg->n_max + 15) / 16 * 16;
      alloc(&h->A8, static_cast<size_t>(cfg->m_max) * h->ld8);
      alloc(reinterpret_cast<void**>(&h->w8s), sizeof(float) * cdiv(cfg->m_max, 128) * cdiv(cfg->n_max, 128));
    }
    alloc(&h->wOTb, bm);
    alloc(&h->wOTbl, bm);
    alloc(&h->wZTb, bm);
    alloc(&h->wZTbl, bm);
    alloc(&h->wQTb, bn);
    alloc(&h->wQTbl, bn);
  }
  if (!ok) return false;
  return cudaMemsetAsync(h->wtick, 0, sizeof(unsigned), h->stream) == cudaSuccess &&
         cudaMemsetAsync(h->wT2, 0, sizeof(float) * LW * LW, h->stream) == cudaSuccess &&
         launch_wd_identity(h->wI, h->stream) == cudaSuccess;
}

// Adjoint workspace (floats): L (m x K), R (n x K), P, T, Z (m x LP each), Yb, Y, RQ (n x LP
// each), small (16 x LP x LP), then doubles: Qbar (n x LP) and column-pass partials (64 x n x LP).
struct AdWs {
  float *L, *R, *P, *T, *Z, *Y, *Yb, *RQ, *W1, *C1, *C2, *C3, *S1, *S2;
  double *Qb, *part;
};

int64_t ad_ws_floats(const frsvt_handle* h, int64_t m, int64_t n) {
  const int64_t LP = h->LP, K = h->ad_K;
  const int64_t f = m * K + n * K + 4 * m * LP + 4 * n * LP + 16 * LP * LP;
  return (f + 1) / 2 * 2 + 2 * (n * LP + 64 * (n > LP ? n : LP) * LP);
}

AdWs ad_carve(const frsvt_handle* h, int64_t m, int64_t n) {
  const int64_t LP = h->LP, K = h->ad_K;
  float* p = h->ad_ws;
  AdWs w;
  w.L = p; p += m * K;
  w.R = p; p += n * K;
  w.P = p; p += m * LP;
  w.T = p; p += m * LP;
  w.Z = p; p += m * LP;
  p += m * LP;                        // spare m x LP block
  w.Y = p; p += n * LP;
  p += n * LP;                        // spare n x LP block
  w.Yb = p; p += n * LP;
  w.RQ = p; p += n * LP;
  w.W1 = p; p += LP * LP;
  w.C1 = p; p += LP * LP;
  w.C2 = p; p += LP * LP;
  w.C3 = p; p += LP * LP;
  w.S1 = p; p += LP * LP;
  w.S2 = p; p += LP * LP;
  const int64_t used = p - h->ad_ws;
  double* d = reinterpret_cast<double*>(h->ad_ws + (used + 1) / 2 * 2);
  w.Qb = d;
  w.part = d + n * LP;
  return w;
}

// Saved buffer: Qd_0..Qd_q (double, n x LP each), then floats Q_0..Q_q, R_0..R_q, U, sigma, V_B.
struct AdSaved {
  double* Qd;
  float *Q, *R, *U, *sig, *VB;
};

size_t ad_saved_floats(const frsvt_handle* h, int64_t m, int64_t n) {
  const int64_t LP = h->LP, q1 = h->cfg.q + 1;
  return static_cast<size_t>(2 * q1 * n * LP + q1 * n * LP + q1 * LP * LP + LP * LP + LP + m * LP);
}

AdSaved ad_saved(const frsvt_handle* h, float* base, int64_t n) {
  const int64_t LP = h->LP, q1 = h->cfg.q + 1;
  AdSaved s;
  s.Qd = reinterpret_cast<double*>(base);
  s.Q = base + 2 * q1 * n * LP;
  s.R = s.Q + q1 * n * LP;
  s.U = s.R + q1 * LP * LP;
  s.sig = s.U + LP * LP;
  s.VB = s.sig + LP;
  return s;
}

frsvt_status ad_check(frsvt_handle* h, const float* A, int64_t m, int64_t n, int64_t lda, int32_t l) {
  if (h->ad_ws == nullptr) return fail(h, FRSVT_ERR_UNSUPPORTED, "handle created without FRSVT_CFG_ADJOINT");
  frsvt_status s = check_shape(h, m, n);
  if (s != FRSVT_OK) return s;
  if ((s = check_matrix(h, A, m, n, lda, "A")) != FRSVT_OK) return s;
  if (l < 1 || l > h->cfg.l_max) return fail(h, FRSVT_ERR_INVALID_ARG, "l must be in [1, l_max]");
  if (n > (h->LP == 16 ? 2048 : 1024)) return fail(h, FRSVT_ERR_UNSUPPORTED, "the adjoint path serves n <= 2048 / 1024");
  return FRSVT_OK;
}

}  // namespace

extern "C" {

const char* frsvt_status_string(frsvt_status s) {
  switch (s) {
    case FRSVT_OK: return "ok";
    case FRSVT_ERR_INVALID_ARG: return "invalid argument";
    case FRSVT_ERR_UNSUPPORTED: return "unsupported";
    case FRSVT_ERR_ALLOC: return "device allocation failed";
    case FRSVT_ERR_CUDA: return "CUDA error";
    case FRSVT_ERR_RANK_DEFICIENT: return "rank deficient basis (informational)";
    case FRSVT_ERR_NOT_CONVERGED: return "Jacobi SVD did not converge";
    case FRSVT_ERR_NONFINITE: return "non-finite value";
  }
  return "unknown status";
}

const char* frsvt_last_error(const frsvt_handle* h) { return h ? h->err.c_str() : "null handle"; }

frsvt_status ap_setup(frsvt_handle* h, int64_t n);

frsvt_status frsvt_create(frsvt_handle** out, const frsvt_config* cfg, void* stream) {
  frsvt_handle* h = nullptr;
  if (out == nullptr || cfg == nullptr) return FRSVT_ERR_INVALID_ARG;
  *out = nullptr;
  if (cfg->m_max < 1 || cfg->n_max < 1 || cfg->l_max < 1 || cfg->l_max > kMaxL || cfg->q < 0 || cfg->q > 64)
    return FRSVT_ERR_INVALID_ARG;
  if ((cfg->flags & ~(FRSVT_CFG_ADJOINT | FRSVT_CFG_ORTH_LAST)) != 0) return FRSVT_ERR_INVALID_ARG;
  if (cfg->problem_streams < 0 || cfg->problem_streams > 16 ||
      (cfg->problem_streams > 1 && !(cfg->flags & FRSVT_CFG_ADJOINT)))
    return FRSVT_ERR_INVALID_ARG;
  if (cfg->precision != FRSVT_PREC_FP32 && cfg->precision != FRSVT_PREC_BF16 &&
      !(cfg->precision == FRSVT_PREC_FP8 && cfg->l_max > 32))
    return FRSVT_ERR_UNSUPPORTED;
  h = new (std::nothrow) frsvt_handle();
  if (h == nullptr) return FRSVT_ERR_ALLOC;
  h->cfg = *cfg;
  if (h->cfg.max_jacobi_sweeps <= 0) h->cfg.max_jacobi_sweeps = 30;
  if (!(h->cfg.rank_tol > 0.0)) h->cfg.rank_tol = 1e-12;
  h->stream = static_cast<cudaStream_t>(stream);
  h->wide = cfg->l_max > 32;
  h->LP = cfg->l_max <= 16 ? 16 : (cfg->l_max <= 32 ? 32 : wide_lp());
  const int64_t nsmax = cfg->n_max < cfg->m_max ? cfg->n_max : cfg->m_max;
  if (h->wide ? ((cfg->flags & FRSVT_CFG_ADJOINT) || cfg->m_max >= (int64_t(1) << 31))
              : nsmax > ns_limit(h->LP)) {
    delete h;
    return FRSVT_ERR_UNSUPPORTED;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    delete h;
    return FRSVT_ERR_CUDA;
  }
  if (h->wide) {
    h->absmax_blocks = 2 * h->sms;
    if (tensor_map_encoder() == nullptr || prepare_wide_kernels() != cudaSuccess ||
        prepare_pass_kernels(static_cast<int>(kSmemLimit)) != cudaSuccess ||
        prepare_small_kernels(static_cast<int>(kSmemLimit)) != cudaSuccess) {
      delete h;
      return FRSVT_ERR_CUDA;
    }
    if (!wide_alloc(h)) {
      free_all(h);
      delete h;
      return FRSVT_ERR_ALLOC;
    }
    if (cudaMemsetAsync(h->dst, 0, sizeof(DevState), h->stream) != cudaSuccess ||
        cudaMemcpyAsync(&h->dst->rp_res, &kNoResidual, sizeof(float), cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess) {
      free_all(h);
      delete h;
      return FRSVT_ERR_CUDA;
    }
    *out = h;
    return FRSVT_OK;
  }
  if (prepare_pass_kernels(static_cast<int>(kSmemLimit)) != cudaSuccess ||
      prepare_small_kernels(static_cast<int>(kSmemLimit)) != cudaSuccess ||
      prepare_fused_kernels(static_cast<int>(kSmemLimit)) != cudaSuccess ||
      prepare_tma_kernels(static_cast<int>(kSmemLimit)) != cudaSuccess ||
      prepare_tc_kernels(static_cast<int>(kSmemLimit)) != cudaSuccess ||
      prepare_tc_sc_kernels(static_cast<int>(kSmemLimit)) != cudaSuccess ||
      prepare_gram_kernels(static_cast<int>(kSmemLimit)) != cudaSuccess ||
      prepare_adjoint_kernels(static_cast<int>(kSmemLimit)) != cudaSuccess ||
      prepare_tb_kernels(static_cast<int>(kSmemLimit)) != cudaSuccess) {
    delete h;
    return FRSVT_ERR_CUDA;
  }
  h->target_ctas = 4 * h->sms;
  h->gsplit_max = h->sms;
  h->absmax_blocks = 2 * h->sms;
  const int64_t LP = h->LP;
  const int64_t ntiles_max = cdiv(cfg->n_max, 256);
  h->part_elems = (static_cast<int64_t>(h->target_ctas) * 256 + cfg->n_max) * LP;
  h->rpart_max = static_cast<int>(h->target_ctas + ntiles_max + 1);
  bool ok = true;
  auto alloc = [&](void** p, size_t bytes) {
    if (ok && cudaMalloc(p, bytes < 16 ? 16 : bytes) != cudaSuccess) ok = false;
  };
  alloc(reinterpret_cast<void**>(&h->dst), sizeof(DevState));
  alloc(reinterpret_cast<void**>(&h->Ys), sizeof(float) * cfg->n_max * LP);
  alloc(reinterpret_cast<void**>(&h->Qs), sizeof(float) * cfg->n_max * LP);
  alloc(reinterpret_cast<void**>(&h->Qt), sizeof(float) * cfg->n_max * LP);
  alloc(reinterpret_cast<void**>(&h->Rf), sizeof(float) * cfg->n_max * LP);
  alloc(reinterpret_cast<void**>(&h->Zl), sizeof(float) * cfg->m_max * LP);
  alloc(reinterpret_cast<void**>(&h->part), sizeof(float) * h->part_elems);
  alloc(reinterpret_cast<void**>(&h->gpart), sizeof(float2) * h->gsplit_max * LP * LP);
  alloc(reinterpret_cast<void**>(&h->rpart), sizeof(float2) * h->rpart_max);
  alloc(reinterpret_cast<void**>(&h->pmax), sizeof(float) * h->absmax_blocks);
  // fused path: short side whose small dense work fits comfortably in one CTA
  h->fused = fused_orth_smem(h->LP, cfg->n_max) <= 96 * 1024 && fused_core_smem(h->LP, cfg->n_max) <= 96 * 1024;
  h->lr_blocks = 8 * h->sms;
  {
    const int64_t nt = cfg->n_max < 256 ? cfg->n_max : 256;
    const int nst = tma_lr_stages(h->LP, nt, kSmemLimit - 16384);
    h->tc_lr_ns = tc_lr_stages(h->LP, nt, kSmemLimit - 2048);
    h->gram_grid = gram_resident_grid(h->LP, nt);
    h->alm_grid = tma_alm_resident_grid(h->LP, nt);
    if (h->gram_grid < 8) h->gram_grid = 8;
    h->tma = tensor_map_encoder() != nullptr && nst >= 2 && h->tc_lr_ns >= 2 && h->alm_grid >= 4 &&
             tma_sc_smem(h->LP, nt) <= kSmemLimit - 8192 &&
             tma_lr_smem(h->LP, nt, nst) <= kSmemLimit - 8192 && tma_alm_smem(h->LP, nt) <= kSmemLimit - 8192;
    // clusters of 8 that can be resident at once (GPCs hold a whole number of clusters)
    h->tma_grid = h->tma ? tma_resident_grid(h->LP, nt) : 0;
    if (h->tma_grid < 8) h->tma = false;
    if (h->tma) {
      const int ns_o = tc_sc_stages(h->LP, nt, true, kSmemLimit - 8192);
      const int ns_z = tc_sc_stages(h->LP, nt, false, kSmemLimit - 8192);
      h->tc_sc_ns = ns_o < ns_z ? ns_o : ns_z;
      if (h->tc_sc_ns >= 2 && tc_sc_smem(h->LP, nt, false, h->tc_sc_ns) <= kSmemLimit - 8192) {
        h->tc_sc_grid = tc_sc_resident_grid(h->LP, nt, h->tc_sc_ns);
        if (h->tc_sc_grid < 8) h->tc_sc_ns = 0;
      } else {
        h->tc_sc_ns = 0;
      }
    }
  }
  {
    const int64_t ntl = ntiles_max;
    const int64_t ncl_sc = cdiv(cdiv(h->target_ctas, 1), 8) + 1;          // clusters per tile, upper bound
    h->cpart_sc_elems = ntl * ncl_sc * 256 * LP;
    h->cpart_alm_elems = ntl * ncl_sc + 2 * static_cast<int64_t>(h->sms);   // >= one partial per epilogue CTA
    const int64_t np = LP * (LP + 1) / 2;
    alloc(reinterpret_cast<void**>(&h->cpart_sc), sizeof(float) * h->cpart_sc_elems);
    alloc(reinterpret_cast<void**>(&h->cpart_lr), sizeof(double) * (h->lr_blocks / 8) * np);
    alloc(reinterpret_cast<void**>(&h->cpart_alm), sizeof(double) * h->cpart_alm_elems);
    alloc(reinterpret_cast<void**>(&h->Gfin), sizeof(double) * np);
    alloc(reinterpret_cast<void**>(&h->rsum), sizeof(double) * ntl);
    alloc(reinterpret_cast<void**>(&h->tickets), sizeof(unsigned) * (ntl + 1));
  }
  alloc(reinterpret_cast<void**>(&h->psum), sizeof(float2) * h->absmax_blocks);
  alloc(reinterpret_cast<void**>(&h->wsvt_next), sizeof(unsigned));
  if (cfg->precision == FRSVT_PREC_BF16 && h->tma) {
    const int64_t nt = cfg->n_max < 256 ? cfg->n_max : 256;
    h->ldb = (cfg->n_max + 7) / 8 * 8;
    h->tb_lr_ns = tb_lr_stages(h->LP, nt, kSmemLimit - 2048);
    const int ns_o = tb_sc_stages(h->LP, nt, true, kSmemLimit - 8192);
    const int ns_z = tb_sc_stages(h->LP, nt, false, kSmemLimit - 8192);
    h->tb_sc_ns = ns_o < ns_z ? ns_o : ns_z;
    h->tb_sc_grid = (h->tb_sc_ns >= 2 && h->tb_lr_ns >= 2) ? tb_sc_resident_grid(h->LP, nt, h->tb_sc_ns) : 0;
    if (h->tb_sc_grid < 4) h->tb_sc_ns = 0;
    if (h->tb_sc_ns > 0) alloc(&h->Ab, 2 * static_cast<size_t>(cfg->m_max) * h->ldb);
  }
  if (cfg->flags & FRSVT_CFG_ADJOINT) {
    h->ad_K = static_cast<int>(LP) * (2 + 2 * h->cfg.q);
    alloc(reinterpret_cast<void**>(&h->ad_ws), sizeof(float) * ad_ws_floats(h, cfg->m_max, cfg->n_max));
  }
  if (!ok) {
    free_all(h);
    delete h;
    return FRSVT_ERR_ALLOC;
  }
  if (cudaMemsetAsync(h->dst, 0, sizeof(DevState), h->stream) != cudaSuccess ||
      cudaMemcpyAsync(&h->dst->rp_res, &kNoResidual, sizeof(float), cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->Qt, 0, sizeof(float) * cfg->n_max * LP, h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->tickets, 0, sizeof(unsigned) * (ntiles_max + 1), h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess) {
    free_all(h);
    delete h;
    return FRSVT_ERR_CUDA;
  }
  if (cfg->problem_streams > 1) {                   // child handles for concurrent problems
    frsvt_config kc = *cfg;
    kc.problem_streams = 0;
    bool ok = cudaEventCreateWithFlags(&h->fork_event, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; ok && i < cfg->problem_streams; ++i) {
      cudaStream_t ks = nullptr;
      cudaEvent_t ke = nullptr;
      ok = cudaStreamCreateWithFlags(&ks, cudaStreamNonBlocking) == cudaSuccess;
      if (ok) h->kid_streams.push_back(ks);
      ok = ok && cudaEventCreateWithFlags(&ke, cudaEventDisableTiming) == cudaSuccess;
      if (ok) h->kid_events.push_back(ke);
      frsvt_handle* kid = nullptr;
      const frsvt_status ks2 = ok ? frsvt_create(&kid, &kc, ks) : FRSVT_ERR_CUDA;
      if (ks2 == FRSVT_OK) h->kids.push_back(kid);
      ok = ok && ks2 == FRSVT_OK;
    }
    if (!ok) {
      free_all(h);
      delete h;
      return FRSVT_ERR_ALLOC;
    }
  }
  *out = h;
  return FRSVT_OK;
}

frsvt_status frsvt_destroy(frsvt_handle* h) {
  if (h == nullptr) return FRSVT_ERR_INVALID_ARG;
  cudaStreamSynchronize(h->stream);
  free_all(h);
  delete h;
  return FRSVT_OK;
}

frsvt_status frsvt_set_stream(frsvt_handle* h, void* stream) {
  if (h == nullptr) return FRSVT_ERR_INVALID_ARG;
  h->stream = static_cast<cudaStream_t>(stream);
  h->epoch += 1;
  return FRSVT_OK;
}

frsvt_status frsvt_reset(frsvt_handle* h, uint64_t counter) {
  if (h == nullptr) return FRSVT_ERR_INVALID_ARG;
  h->epoch += 1;
  FRSVT_CK(cudaMemsetAsync(&h->dst->keep, 0, sizeof(int32_t), h->stream));
  FRSVT_CK(cudaMemcpyAsync(&h->dst->counter, &counter, sizeof(uint64_t), cudaMemcpyHostToDevice, h->stream));
  FRSVT_CK(cudaStreamSynchronize(h->stream));   // the host value lives on this stack frame
  return FRSVT_OK;
}

// Alg. 1 up to the core for frsvt_svt / frsvt_svt_factors: leaves X = Z Rf^T in the handle
// (Z = A Q, Rf = Q M; narrow: Zl / Rf, m x LP / n x LP; wide: wZ / wRf, long side x 128 / short
// side x 128, with X = Rf Z^T when m < n).
static frsvt_status svt_range_and_core(frsvt_handle* h, const float* A, int64_t m, int64_t n, int64_t lda,
                                       float tau, int32_t l) {
  frsvt_status s = FRSVT_OK;
  if (h->ap_a > 0) {                                   // adaptive rank prediction: l on the device
    if (!(h->tma && n <= 256)) return fail(h, FRSVT_ERR_UNSUPPORTED, "rank prediction needs n <= 256");
    if (h->ap_n != n && (s = ap_setup(h, n)) != FRSVT_OK) return s;
    h->last_m = m;
    h->last_n = n;
    h->last_l = -1;
    return range_and_core(h, A, m, n, lda, -1, h->cfg.q, 1, kCounterFromState, tau, 0, 1, 1);
  }
  if ((s = sync_rp_shape(h, m, n, l)) != FRSVT_OK) return s;
  if (h->wide) {
    if (h->Ab != nullptr) FRSVT_CK(launch_to_bf16(A, lda, m, n, h->Ab, h->ldb, h->stream));
    return wide_range_and_core(h, A, m, n, lda, l, h->cfg.q, kCounterFromState, tau, 0, 1, wide_lowp(h),
                               h->cfg.range_prop ? 1 : 0, true);
  }
  const int rp = h->cfg.range_prop ? 1 : 0;
  const bool bf = h->Ab != nullptr && h->tma && n <= 256;
  if (bf) FRSVT_CK(launch_to_bf16(A, lda, m, n, h->Ab, h->ldb, h->stream));
  return range_and_core(h, A, m, n, lda, l, h->cfg.q, rp, kCounterFromState, tau, 0, rp, 1, bf ? h->Ab : nullptr);
}

static frsvt_status svt_check(frsvt_handle* h, const float* A, int64_t m, int64_t n, int64_t lda, float tau,
                              int32_t l) {
  frsvt_status s = check_shape(h, m, n);
  if (s != FRSVT_OK) return s;
  if ((s = check_matrix(h, A, m, n, lda, "A")) != FRSVT_OK) return s;
  if (l < 1 || l > h->cfg.l_max) return fail(h, FRSVT_ERR_INVALID_ARG, "l must be in [1, l_max]");
  if (!(tau >= 0.f) || !std::isfinite(tau)) return fail(h, FRSVT_ERR_INVALID_ARG, "tau must be finite and >= 0");
  return FRSVT_OK;
}

frsvt_status frsvt_svt(frsvt_handle* h, const float* A, int64_t m, int64_t n, int64_t lda, float tau, int32_t l,
                       float* X, int64_t ldx) {
  if (h == nullptr) return FRSVT_ERR_INVALID_ARG;
  frsvt_status s = svt_check(h, A, m, n, lda, tau, l);
  if (s != FRSVT_OK) return s;
  if ((s = check_matrix(h, X, m, n, ldx, "X")) != FRSVT_OK) return s;
  if (m == 0 || n == 0) return FRSVT_OK;
  if (static_cast<const void*>(A) == static_cast<const void*>(X)) return fail(h, FRSVT_ERR_INVALID_ARG, "X aliases A");
  if (l > n) l = static_cast<int32_t>(n);
  if ((s = svt_range_and_core(h, A, m, n, lda, tau, l)) != FRSVT_OK) return s;
  if (h->wide) return wide_epilogue(h, false, m, n, nullptr, nullptr, nullptr, 0, X, ldx);
  const Splits sp = row_splits(h, m, n);
  FRSVT_LAUNCH(FRSVT_PHASE_EPILOGUE, launch_recon(h->LP, h->Zl, h->Rf, m, n, X, ldx, sp.nsplit, sp.rps, h->stream));
  return FRSVT_OK;
}

frsvt_status frsvt_svt_factors(frsvt_handle* h, const float* A, int64_t m, int64_t n, int64_t lda, float tau,
                               int32_t l, float* U, int64_t ldu, float* V, int64_t ldv, int32_t* r) {
  if (h == nullptr) return FRSVT_ERR_INVALID_ARG;
  frsvt_status s = svt_check(h, A, m, n, lda, tau, l);
  if (s != FRSVT_OK) return s;
  if (m == 0 || n == 0) return FRSVT_OK;
  if (l > n) l = static_cast<int32_t>(n);
  const int32_t lw = h->ap_a > 0 ? h->LP : l;          // under rank prediction l is chosen on the device
  if (U == nullptr || V == nullptr || ldu < lw || ldv < lw)
    return fail(h, FRSVT_ERR_INVALID_ARG, "U and V are required, with ldu, ldv >= l");
  if ((s = svt_range_and_core(h, A, m, n, lda, tau, l)) != FRSVT_OK) return s;
  const bool tall = m >= n;                           // wide handles serve m < n with X = Rf Z^T
  const float* Zs = h->wide ? (tall ? h->wZ : h->wRf) : h->Zl;
  const float* Rs = h->wide ? (tall ? h->wRf : h->wZ) : h->Rf;
  const int64_t lds = h->wide ? wide_lp() : h->LP;
  FRSVT_CK(cudaMemcpy2DAsync(U, sizeof(float) * ldu, Zs, sizeof(float) * lds, sizeof(float) * lw, m,
                             cudaMemcpyDeviceToDevice, h->stream));
  FRSVT_CK(cudaMemcpy2DAsync(V, sizeof(float) * ldv, Rs, sizeof(float) * lds, sizeof(float) * lw, n,
                             cudaMemcpyDeviceToDevice, h->stream));
  if (r != nullptr)
    FRSVT_CK(cudaMemcpyAsync(r, &h->dst->r, sizeof(int32_t), cudaMemcpyDeviceToDevice, h->stream));
  return FRSVT_OK;
}

frsvt_status frsvt_spectral_norm(frsvt_handle* h, const float* A, int64_t m, int64_t n, int64_t lda, int32_t iters,
                                 double* sigma1) {
  if (h == nullptr || sigma1 == nullptr) return FRSVT_ERR_INVALID_ARG;
  frsvt_status s = check_shape(h, m, n);
  if (s != FRSVT_OK) return s;
  if ((s = check_matrix(h, A, m, n, lda, "A")) != FRSVT_OK) return s;
  if (iters < 0 || iters > 64) return fail(h, FRSVT_ERR_INVALID_ARG, "iters must be in [0, 64]");
  *sigma1 = 0.0;
  if (m == 0 || n == 0) return FRSVT_OK;
  const int l = static_cast<int>(n < h->cfg.l_max ? n : h->cfg.l_max);
  const uint64_t ctr = 0x5350454354524131ull;   // a fixed stream index reserved for this estimate
  if ((s = h->wide ? wide_range_and_core(h, A, m, n, lda, l, iters, ctr, FLT_MAX, 0, 0)
                   : range_and_core(h, A, m, n, lda, l, iters, 0, ctr, FLT_MAX, 0, 0, 0)) != FRSVT_OK)
    return s;
  double v = 0.0;
  FRSVT_CK(cudaMemcpyAsync(&v, &h->dst->sigma1, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  FRSVT_CK(cudaStreamSynchronize(h->stream));
  *sigma1 = v;
  return FRSVT_OK;
}

frsvt_status rpca_init(frsvt_handle* h, const float* O, float* S, float* A, int64_t m, int64_t n, int64_t ld,
                       double lambda, double rho, double mu_bar_factor, double normO2, int32_t power_iters) {
  if (h == nullptr) return FRSVT_ERR_INVALID_ARG;
  h->epoch += 1;                                     // what a step launches may change
  frsvt_status s = check_shape(h, m, n);
  if (s != FRSVT_OK) return s;
  if ((s = check_matrix(h, O, m, n, ld, "O")) != FRSVT_OK) return s;
  if ((s = check_matrix(h, S, m, n, ld, "S")) != FRSVT_OK) return s;
  if ((s = check_matrix(h, A, m, n, ld, "A")) != FRSVT_OK) return s;
  if (!(lambda > 0.0) || !(rho >= 1.0) || !(mu_bar_factor >= 1.0) || power_iters < 0 || power_iters > 64)
    return fail(h, FRSVT_ERR_INVALID_ARG, "need lambda > 0, rho >= 1, mu_bar_factor >= 1, 0 <= power_iters <= 64");
  if (m == 0 || n == 0) return FRSVT_OK;
  if (!(normO2 > 0.0)) {
    const int l = static_cast<int>(n < h->cfg.l_max ? n : h->cfg.l_max);
    if ((s = h->wide ? wide_range_and_core(h, O, m, n, ld, l, power_iters, 0x5350454354524131ull, FLT_MAX, 0, 0)
                     : range_and_core(h, O, m, n, ld, l, power_iters, 0, 0x5350454354524131ull, FLT_MAX, 0, 0, 0)) !=
        FRSVT_OK)
      return s;
  }
  FRSVT_CK(launch_absmax_sumsq(O, m, n, ld, h->pmax, h->psum, h->absmax_blocks, h->stream));
  FRSVT_CK(launch_init_scalars(h->pmax, h->psum, h->absmax_blocks, normO2, lambda, rho, mu_bar_factor, h->dst,
                               h->stream));
  FRSVT_CK(launch_init_state(O, S, A, m, n, ld, h->dst, h->stream));
  if (h->Ab != nullptr) FRSVT_CK(launch_to_bf16(A, ld, m, n, h->Ab, h->ldb, h->stream));
  h->last_m = m;
  h->last_n = n;
  h->last_l = -1;
  if (h->ap_a > 0) {
    frsvt_status sa = ap_setup(h, n);                   // l_0, empty propagated basis
    if (sa != FRSVT_OK) return sa;
  }
  FRSVT_CK(cudaStreamSynchronize(h->stream));
  return FRSVT_OK;
}

// The kernels of one iALM iteration (range finder, core, fused epilogue) on h->stream.
static frsvt_status ialm_launches(frsvt_handle* h, const frsvt_handle::StepKey& k) {
  const float* O = k.O;
  float* S = k.S;
  float* A = k.A;
  const int64_t m = k.m, n = k.n, ld = k.ld;
  const int l = k.l;
  float* L = k.L;
  const int64_t ldl = k.ldl;
  frsvt_status s = FRSVT_OK;
  const int rp = h->cfg.range_prop ? 1 : 0;
  const bool bf = h->Ab != nullptr && h->tma && n <= 256;   // the shadow is kept current by rpca_init / the epilogue
  if (h->wide) {
    if ((s = wide_range_and_core(h, A, m, n, ld, l, h->cfg.q, kCounterFromState, 0.f, 1, 1, wide_lowp(h), rp,
                                 true)) != FRSVT_OK)
      return s;
    if ((s = wide_epilogue(h, true, m, n, O, S, A, ld, L, ldl)) != FRSVT_OK) return s;
  } else {
  if ((s = range_and_core(h, A, m, n, ld, l, h->cfg.q, rp, kCounterFromState, 0.f, 1, rp, 1,
                          bf ? h->Ab : nullptr)) != FRSVT_OK)
    return s;
  if (h->tma && n <= 256 && m < (int64_t(1) << 31)) {
    CUtensorMap tO, tS, tA, tZ;
    const int re = tma_rows_per_tile_epilogue();
    if (!make_row_map(&tO, O, m, n, ld, tma_np4(n), re) || !make_row_map(&tS, S, m, n, ld, tma_np4(n), re) ||
        !make_row_map(&tA, A, m, n, ld, tma_np4(n), re) || !make_row_map(&tZ, h->Zl, m, h->LP, h->LP, h->LP, re))
      return fail(h, FRSVT_ERR_CUDA, "cuTensorMapEncodeTiled failed for O/S/A/Z");
    const int G = h->alm_grid;
    const int64_t rpc = cdiv(cdiv(m, G), re) * re;
    FRSVT_LAUNCH(FRSVT_PHASE_EPILOGUE, launch_tp_alm(h->LP, tO, tS, tA, tZ, m, n, rpc, G, h->Rf, S, A, ld, L, ldl,
                                                     h->dst, h->cpart_alm, h->tickets, bf ? h->Ab : nullptr,
                                                     h->ldb, h->stream));
  } else if (h->fused) {
    const Splits fs = fused_splits(h, m, n);
    FRSVT_LAUNCH(FRSVT_PHASE_EPILOGUE, launch_alm2(h->LP, h->Zl, h->Rf, O, S, A, m, n, ld, L, ldl, h->dst, fs.nsplit,
                                                   fs.rps, h->cpart_alm, h->rsum, h->tickets, h->stream));
  } else {
  const Splits sp = row_splits(h, m, n);
  FRSVT_LAUNCH(FRSVT_PHASE_EPILOGUE, launch_alm(h->LP, h->Zl, h->Rf, O, S, A, m, n, ld, L, ldl, h->dst, h->rpart,
                                                 sp.nsplit, sp.rps, h->stream));
  FRSVT_LAUNCH(FRSVT_PHASE_FINISH, launch_alm_finish(h->rpart, sp.nsplit * sp.ntiles, h->dst, h->stream));
  }
  }
  return FRSVT_OK;
}

// Runs ialm_launches through a CUDA graph: captured on the handle's private stream the first time
// a StepKey is seen, then replayed on the user's stream (one launch instead of eight or more, and
// no tensor-map encoding on the host).  The graphs of the four most recent keys are kept (a caller
// that alternates, e.g. with and without L, does not recapture).  When the user's stream is itself
// being captured, or phase timing is on, the kernels are launched directly; a capture that fails
// falls back the same way.
static frsvt_status ialm_step_launch(frsvt_handle* h, const frsvt_handle::StepKey& key) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (h->timing || cudaStreamIsCapturing(h->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    (void)cudaGetLastError();
    return ialm_launches(h, key);
  }
  int slot = -1;
  for (int i = 0; i < frsvt_handle::kGraphSlots; ++i)
    if (h->step_exec[i] != nullptr && h->step_key[i] == key) slot = i;
  if (slot < 0) {
    slot = 0;                                  // an empty slot, else the least recently used one
    for (int i = 0; i < frsvt_handle::kGraphSlots; ++i) {
      if (h->step_exec[i] == nullptr) {
        slot = i;
        break;
      }
      if (h->step_used[i] < h->step_used[slot]) slot = i;
    }
    if (h->step_exec[slot]) {                  // a replay of the old graph may still be queued
      FRSVT_CK(cudaStreamSynchronize(h->stream));
      cudaGraphExecDestroy(h->step_exec[slot]);
      h->step_exec[slot] = nullptr;
    }
    if (h->capture_stream == nullptr &&
        cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
      h->capture_stream = nullptr;
      (void)cudaGetLastError();
      return ialm_launches(h, key);
    }
    cudaStream_t user = h->stream;
    h->stream = h->capture_stream;
    frsvt_status s = FRSVT_OK;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      s = ialm_launches(h, key);
      e = cudaStreamEndCapture(h->capture_stream, &g);
    }
    h->stream = user;
    int32_t kernels = 0;
    if (e == cudaSuccess && s == FRSVT_OK && g != nullptr) {
      size_t nn = 0;
      if (cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn > 0) {
        std::vector<cudaGraphNode_t> nodes(nn);
        if (cudaGraphGetNodes(g, nodes.data(), &nn) == cudaSuccess)
          for (size_t i = 0; i < nn; ++i) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
          }
      }
      (void)cudaGetLastError();
      e = cudaGraphInstantiate(&h->step_exec[slot], g, 0);
    }
    if (g) cudaGraphDestroy(g);
    if (s != FRSVT_OK) return s;
    if (e != cudaSuccess || h->step_exec[slot] == nullptr) {
      h->step_exec[slot] = nullptr;
      (void)cudaGetLastError();
      return ialm_launches(h, key);
    }
    h->step_key[slot] = key;
    h->step_kernels[slot] = kernels;
  }
  h->step_used[slot] = ++h->step_clock;
  h->last_step_kernels = h->step_kernels[slot];
  FRSVT_CK(cudaGraphLaunch(h->step_exec[slot], h->stream));
  return FRSVT_OK;
}

frsvt_status rpca_ialm_step(frsvt_handle* h, const float* O, float* S, float* A, int64_t m, int64_t n, int64_t ld,
                            int32_t l, float* L, int64_t ldl, double* residual) {
  if (h == nullptr) return FRSVT_ERR_INVALID_ARG;
  frsvt_status s = check_shape(h, m, n);
  if (s != FRSVT_OK) return s;
  if ((s = check_matrix(h, O, m, n, ld, "O")) != FRSVT_OK) return s;
  if ((s = check_matrix(h, S, m, n, ld, "S")) != FRSVT_OK) return s;
  if ((s = check_matrix(h, A, m, n, ld, "A")) != FRSVT_OK) return s;
  if (L != nullptr && (s = check_matrix(h, L, m, n, ldl, "L")) != FRSVT_OK) return s;
  if (l < 1 || l > h->cfg.l_max) return fail(h, FRSVT_ERR_INVALID_ARG, "l must be in [1, l_max]");
  if (m == 0 || n == 0) return FRSVT_OK;
  if (l > n) l = static_cast<int32_t>(n);
  if (h->ap_a > 0) {                                   // adaptive rank prediction: l on the device
    if (!(h->tma && n <= 256)) return fail(h, FRSVT_ERR_UNSUPPORTED, "rank prediction needs n <= 256");
    if (h->ap_n != n && (s = ap_setup(h, n)) != FRSVT_OK) return s;
    h->last_m = m;
    h->last_n = n;
    l = -1;
  } else if ((s = sync_rp_shape(h, m, n, l)) != FRSVT_OK) {
    return s;
  }
  const frsvt_handle::StepKey key{O, S, A, m, n, ld, l, L, ldl, h->epoch};
  if ((s = ialm_step_launch(h, key)) != FRSVT_OK) return s;
  if (residual != nullptr) {
    double v = 0.0;
    FRSVT_CK(cudaMemcpyAsync(&v, &h->dst->resid_ratio, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    FRSVT_CK(cudaStreamSynchronize(h->stream));
    *residual = v;
  }
  return FRSVT_OK;
}

static frsvt_status wsvt_check(frsvt_handle* h, int32_t batch, const float* const* A, const int32_t* n_i, int32_t m,
                        float c, float eps, float* const* X, int32_t variant, int32_t l) {
  if (h == nullptr) return FRSVT_ERR_INVALID_ARG;
  if (h->wide) return fail(h, FRSVT_ERR_UNSUPPORTED, "batched WSVT needs a handle with l_max <= 32");
  if (batch < 0) return fail(h, FRSVT_ERR_INVALID_ARG, "negative batch");
  if (variant != FRSVT_WSVT_EXACT && variant != FRSVT_WSVT_FRSVT) return fail(h, FRSVT_ERR_INVALID_ARG, "unknown variant");
  if (m < 1 || m > 64) return fail(h, FRSVT_ERR_UNSUPPORTED, "batched WSVT serves m in [1, 64]");
  if (variant == FRSVT_WSVT_FRSVT && (l < 1 || l > 32)) return fail(h, FRSVT_ERR_INVALID_ARG, "l must be in [1, 32]");
  if (!(c >= 0.f) || !(eps > 0.f)) return fail(h, FRSVT_ERR_INVALID_ARG, "c must be >= 0 and eps > 0");
  if (batch > 0 && (A == nullptr || X == nullptr || n_i == nullptr))
    return fail(h, FRSVT_ERR_INVALID_ARG, "A, X and n_i are required");
  return FRSVT_OK;
}

static int wsvt_grid(frsvt_handle* h, int variant, int nt, int cps_req, int m, int LP, int batch) {
  const int occ = wsvt_ctas_per_sm(variant, nt, m, static_cast<int>(h->cfg.n_max), LP);
  if (occ <= 0) return 0;
  const int cps = (cps_req > 0 && cps_req < occ) ? cps_req : occ;
  const int grid = h->sms * cps;
  return grid < batch ? grid : batch;
}

frsvt_status frsvt_wsvt(frsvt_handle* h, int32_t batch, const float* const* A, const int32_t* n_i, int32_t m,
                        float c, float eps, float* const* X, int32_t variant, int32_t l) {
  frsvt_status s = wsvt_check(h, batch, A, n_i, m, c, eps, X, variant, l);
  if (s != FRSVT_OK || batch == 0) return s;
  const int LP = (variant == FRSVT_WSVT_FRSVT && l > 16) ? 32 : 16;
  const int nt = h->wsvt_nt[variant];
  const int grid = wsvt_grid(h, variant, nt, h->wsvt_cps[variant], m, LP, batch);
  if (grid <= 0) return fail(h, FRSVT_ERR_UNSUPPORTED, "batched WSVT problem does not fit in shared memory");
  FRSVT_CK(launch_wsvt(variant, nt, grid, LP, A, X, n_i, batch, m, static_cast<int>(h->cfg.n_max), c, eps,
                       h->cfg.seed, 0ull, l, h->cfg.q, h->cfg.rank_tol, h->cfg.max_jacobi_sweeps, h->wsvt_next,
                       h->dst, h->stream));
  return FRSVT_OK;
}

frsvt_status frsvt_wsvt_tune(frsvt_handle* h, int32_t batch, const float* const* A, const int32_t* n_i, int32_t m,
                             float c, float eps, float* const* X, int32_t variant, int32_t l) {
  frsvt_status s = wsvt_check(h, batch, A, n_i, m, c, eps, X, variant, l);
  if (s != FRSVT_OK || batch == 0) return s;
  const int LP = (variant == FRSVT_WSVT_FRSVT && l > 16) ? 32 : 16;
  cudaEvent_t e0, e1;
  FRSVT_CK(cudaEventCreate(&e0));
  FRSVT_CK(cudaEventCreate(&e1));
  float best = -1.f;
  int best_nt = h->wsvt_nt[variant], best_cps = h->wsvt_cps[variant];
  const int nts[3] = {128, 256, 512};
  for (int nt : nts) {
    const int occ = wsvt_ctas_per_sm(variant, nt, m, static_cast<int>(h->cfg.n_max), LP);
    for (int cps = 1; cps <= occ; ++cps) {
      const int grid = wsvt_grid(h, variant, nt, cps, m, LP, batch);
      if (grid <= 0) continue;
      float tot = 0.f;
      for (int rep = 0; rep < 3; ++rep) {
        cudaError_t e = launch_wsvt(variant, nt, grid, LP, A, X, n_i, batch, m, static_cast<int>(h->cfg.n_max), c,
                                    eps, h->cfg.seed, 0ull, l, h->cfg.q, h->cfg.rank_tol, h->cfg.max_jacobi_sweeps,
                                    h->wsvt_next, h->dst, h->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
        if (e == cudaSuccess)
          e = launch_wsvt(variant, nt, grid, LP, A, X, n_i, batch, m, static_cast<int>(h->cfg.n_max), c, eps,
                          h->cfg.seed, 0ull, l, h->cfg.q, h->cfg.rank_tol, h->cfg.max_jacobi_sweeps, h->wsvt_next,
                          h->dst, h->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
          return fail(h, FRSVT_ERR_CUDA, cudaGetErrorString(e));
        }
        tot += ms;
      }
      if (best < 0.f || tot < best) {
        best = tot;
        best_nt = nt;
        best_cps = cps;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best < 0.f) return fail(h, FRSVT_ERR_UNSUPPORTED, "no WSVT launch shape fits");
  h->wsvt_nt[variant] = best_nt;
  h->wsvt_cps[variant] = best_cps;
  return FRSVT_OK;
}

frsvt_status frsvt_wsvt_get_tuning(const frsvt_handle* h, int32_t variant, int32_t* threads, int32_t* ctas_per_sm) {
  if (h == nullptr || threads == nullptr || ctas_per_sm == nullptr) return FRSVT_ERR_INVALID_ARG;
  if (variant != FRSVT_WSVT_EXACT && variant != FRSVT_WSVT_FRSVT) return FRSVT_ERR_INVALID_ARG;
  *threads = h->wsvt_nt[variant];
  *ctas_per_sm = h->wsvt_cps[variant];
  return FRSVT_OK;
}

size_t frsvt_adjoint_saved_bytes(const frsvt_handle* h, int64_t m, int64_t n) {
  if (h == nullptr || m < 0 || n < 0) return 0;
  return ad_saved_floats(h, m, n) * sizeof(float);
}

frsvt_status frsvt_svt_save(frsvt_handle* h, const float* A, int64_t m, int64_t n, int64_t lda, float tau,
                            int32_t l, uint64_t omega_stream, float* X, int64_t ldx, void* saved) {
  if (h == nullptr) return FRSVT_ERR_INVALID_ARG;
  frsvt_status s = ad_check(h, A, m, n, lda, l);
  if (s != FRSVT_OK) return s;
  if ((s = check_matrix(h, X, m, n, ldx, "X")) != FRSVT_OK) return s;
  if (saved == nullptr) return fail(h, FRSVT_ERR_INVALID_ARG, "saved is required");
  if (!(tau >= 0.f)) return fail(h, FRSVT_ERR_INVALID_ARG, "tau must be >= 0");
  if (m == 0 || n == 0) return FRSVT_OK;
  const int LP = h->LP, q = h->cfg.q, nn = static_cast<int>(n);
  cudaStream_t st = h->stream;
  AdWs w = ad_carve(h, m, n);
  AdSaved sv = ad_saved(h, static_cast<float*>(saved), n);
  const double tol = h->cfg.rank_tol;
  FRSVT_CK(ad_omega(LP, w.Z, LP, 0, m, l, h->cfg.seed, omega_stream, st));                  // Omega (m x LP)
  FRSVT_CK(ad_cols(LP, A, lda, m, nn, w.Z, LP, w.part, w.Y, nullptr, LP, 0, 0.f, st));       // Y_0 = A^T Omega
  FRSVT_CK(ad_cholqr2(LP, w.Y, nn, l, tol, sv.Q, sv.Qd, sv.R, h->dst, st));
  for (int i = 1; i <= q; ++i) {
    const float* Qp = sv.Q + static_cast<int64_t>(i - 1) * n * LP;
    FRSVT_CK(ad_rows(LP, A, lda, m, nn, Qp, w.Z, LP, 0, 0.f, st));                          // Z_i = A Q_{i-1}
    FRSVT_CK(ad_cols(LP, A, lda, m, nn, w.Z, LP, w.part, w.Y, nullptr, LP, 0, 0.f, st));     // Y_i = A^T Z_i
    FRSVT_CK(ad_cholqr2(LP, w.Y, nn, l, tol, sv.Q + static_cast<int64_t>(i) * n * LP,
                        sv.Qd + static_cast<int64_t>(i) * n * LP, sv.R + static_cast<int64_t>(i) * LP * LP, h->dst,
                        st));
  }
  const float* Qf = sv.Q + static_cast<int64_t>(q) * n * LP;
  FRSVT_CK(ad_rows(LP, A, lda, m, nn, Qf, w.Z, LP, 0, 0.f, st));                              // Z = A Q = B^T
  FRSVT_CK(ad_core(LP, w.Z, m, l, tau, tol, h->cfg.max_jacobi_sweeps, sv.U, sv.sig, w.S1, w.S2, h->dst, st));
  FRSVT_CK(ad_rows(LP, w.Z, LP, m, LP, w.S1, sv.VB, LP, 0, 0.f, st));                         // V_B = Z U / sigma
  FRSVT_CK(ad_rows(LP, Qf, LP, n, LP, w.S2, w.RQ, LP, 0, 0.f, st));                           // Q U diag(f)
  FRSVT_CK(ad_rank(X, ldx, m, nn, sv.VB, LP, w.RQ, LP, LP, 0.f, st));                          // X = V_B (Q U f)^T
  return FRSVT_OK;
}

frsvt_status frsvt_backward(frsvt_handle* h, const void* saved, const float* A, int64_t m, int64_t n, int64_t lda,
                            float tau, int32_t l, uint64_t omega_stream, const float* dX, int64_t lddx, float* dA,
                            int64_t ldda, float* dtau) {
  if (h == nullptr) return FRSVT_ERR_INVALID_ARG;
  frsvt_status s = ad_check(h, A, m, n, lda, l);
  if (s != FRSVT_OK) return s;
  if ((s = check_matrix(h, dX, m, n, lddx, "dX")) != FRSVT_OK) return s;
  if ((s = check_matrix(h, dA, m, n, ldda, "dA")) != FRSVT_OK) return s;
  if (saved == nullptr || dtau == nullptr) return fail(h, FRSVT_ERR_INVALID_ARG, "saved and dtau are required");
  if (m == 0 || n == 0) return FRSVT_OK;
  const int LP = h->LP, q = h->cfg.q, nn = static_cast<int>(n), K = h->ad_K;
  cudaStream_t st = h->stream;
  AdWs w = ad_carve(h, m, n);
  AdSaved sv = ad_saved(h, static_cast<float*>(const_cast<void*>(saved)), n);
  const float* Qf = sv.Q + static_cast<int64_t>(q) * n * LP;
  auto copy_cols = [&](float* dst, int ldd, int coff, const float* src, int64_t rows) {
    return cudaMemcpy2DAsync(dst + coff, sizeof(float) * ldd, src, sizeof(float) * LP, sizeof(float) * LP, rows,
                             cudaMemcpyDeviceToDevice, st);
  };
  // SVT adjoint on B
  FRSVT_CK(ad_rows(LP, dX, lddx, m, nn, Qf, w.P, LP, 0, 0.f, st));                            // P = dX Q
  FRSVT_CK(ad_cols(LP, sv.VB, LP, m, LP, w.P, LP, w.part, w.W1, nullptr, LP, 0, 0.f, st));    // W1 = V_B^T P
  FRSVT_CK(ad_svt_adjoint(LP, w.W1, sv.U, sv.sig, l, tau, w.C1, w.C2, w.C3, dtau, st));
  FRSVT_CK(ad_rows(LP, sv.VB, LP, m, LP, w.C1, w.L, K, 0, 0.f, st));                          // Bbar^T ...
  FRSVT_CK(ad_rows(LP, w.P, LP, m, LP, w.C2, w.L, K, 0, 1.f, st));                            // ... + P C2
  FRSVT_CK(copy_cols(w.R, K, 0, Qf, n));                                                      // dA += Bbar^T Q^T
  FRSVT_CK(ad_rows(LP, sv.VB, LP, m, LP, w.C3, w.T, LP, 0, 0.f, st));                         // V_B diag(f) U^T
  FRSVT_CK(ad_cols(LP, dX, lddx, m, nn, w.T, LP, w.part, nullptr, w.Qb, LP, 0, 0.f, st));      // Qbar = dX^T ...
  FRSVT_CK(ad_cols(LP, A, lda, m, nn, w.L, K, w.part, nullptr, w.Qb, LP, 0, 1.f, st));         // ... + A^T Bbar^T
  // power steps, last to first
  for (int i = q; i >= 1; --i) {
    const float* Ri = sv.R + static_cast<int64_t>(i) * LP * LP;
    const float* Qp = sv.Q + static_cast<int64_t>(i - 1) * n * LP;
    const int b1 = 1 + 2 * (q - i), b2 = b1 + 1;
    FRSVT_CK(ad_qr_adjoint(LP, sv.Qd + static_cast<int64_t>(i) * n * LP, Ri, w.Qb, nn, l, w.Yb, st));  // Ybar_i
    FRSVT_CK(ad_rows(LP, A, lda, m, nn, Qp, w.L, K, b1 * LP, 0.f, st));                          // Z_i (recomputed)
    FRSVT_CK(copy_cols(w.R, K, b1 * LP, w.Yb, n));                                              // dA += Z_i Ybar_i^T
    FRSVT_CK(ad_rows(LP, A, lda, m, nn, w.Yb, w.L, K, b2 * LP, 0.f, st));                        // Zbar_i = A Ybar_i
    FRSVT_CK(copy_cols(w.R, K, b2 * LP, Qp, n));                                                // dA += Zbar_i Q_{i-1}^T
    FRSVT_CK(ad_cols(LP, A, lda, m, nn, w.L + b2 * LP, K, w.part, nullptr, w.Qb, LP, 0, 0.f, st));  // Qbar_{i-1}
  }
  // sketch
  const int bl = 1 + 2 * q;
  FRSVT_CK(ad_qr_adjoint(LP, sv.Qd, sv.R, w.Qb, nn, l, w.Yb, st));                              // Ybar_0
  FRSVT_CK(ad_omega(LP, w.L, K, bl * LP, m, l, h->cfg.seed, omega_stream, st));                // Omega
  FRSVT_CK(copy_cols(w.R, K, bl * LP, w.Yb, n));                                                // dA += Omega Ybar_0^T
  FRSVT_CK(ad_rank(dA, ldda, m, nn, w.L, K, w.R, K, K, 0.f, st));
  return FRSVT_OK;
}

// Device state of the adaptive rank prediction for a problem with short side n: the parameters
// of Eq. 7, l_0 = ceil(0.1 b) and an empty propagated basis.  Enqueued on the stream.
frsvt_status ap_setup(frsvt_handle* h, int64_t n) {
  int32_t v[4] = {0, 0, 0, 0};                          // l_cur, a, ceil(rho n), b
  if (h->ap_a > 0) {
    int64_t b = static_cast<int64_t>(std::ceil(h->ap_gamma * static_cast<double>(n)));
    if (b > h->LP) b = h->LP;
    if (b > n) b = n;
    if (b < 1) b = 1;
    int64_t l0 = static_cast<int64_t>(std::ceil(0.1 * static_cast<double>(b)));
    v[0] = static_cast<int32_t>(l0 < 1 ? 1 : l0);
    v[1] = h->ap_a;
    v[2] = static_cast<int32_t>(std::ceil(h->ap_rho * static_cast<double>(n)));
    v[3] = static_cast<int32_t>(b);
  }
  FRSVT_CK(cudaMemcpyAsync(&h->dst->l_cur, v, sizeof(v), cudaMemcpyHostToDevice, h->stream));
  FRSVT_CK(cudaMemsetAsync(&h->dst->keep, 0, sizeof(int32_t), h->stream));
  FRSVT_CK(cudaStreamSynchronize(h->stream));          // v lives on this stack frame
  h->ap_n = n;
  return FRSVT_OK;
}

frsvt_status frsvt_set_rank_prediction(frsvt_handle* h, int32_t a, double rho, double gamma) {
  if (h == nullptr) return FRSVT_ERR_INVALID_ARG;
  h->epoch += 1;                                     // what a step launches may change
  if (a < 0 || (a > 0 && (!(rho > 0.0) || rho > 1.0 || !(gamma > 0.0) || gamma > 1.0)))
    return fail(h, FRSVT_ERR_INVALID_ARG, "need a >= 0, 0 < rho <= 1, 0 < gamma <= 1");
  if (a > 0 && (h->wide || !h->cfg.range_prop || h->cfg.precision != FRSVT_PREC_FP32 || !h->tma ||
                h->tc_sc_ns == 0))
    return fail(h, FRSVT_ERR_UNSUPPORTED,
                "adaptive rank prediction needs range propagation, FP32 and the tensor-core path (l_max <= 32)");
  h->ap_a = a;
  h->ap_rho = rho;
  h->ap_gamma = gamma;
  h->ap_n = -1;
  if (a == 0) return ap_setup(h, 0);
  return FRSVT_OK;
}

frsvt_status frsvt_set_partial(frsvt_handle* h, int32_t k) {
  if (h == nullptr) return FRSVT_ERR_INVALID_ARG;
  h->epoch += 1;                                     // what a step launches may change
  if (k < 0 || k > h->cfg.l_max) return fail(h, FRSVT_ERR_INVALID_ARG, "k must be in [0, l_max]");
  FRSVT_CK(cudaMemcpyAsync(&h->dst->partial_k, &k, sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
  FRSVT_CK(cudaStreamSynchronize(h->stream));          // k lives on this stack frame
  return FRSVT_OK;
}

frsvt_status frsvt_get_rank_prediction(frsvt_handle* h, int32_t* l_next) {
  if (h == nullptr || l_next == nullptr) return FRSVT_ERR_INVALID_ARG;
  int32_t v = 0;
  FRSVT_CK(cudaMemcpyAsync(&v, &h->dst->l_cur, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
  FRSVT_CK(cudaStreamSynchronize(h->stream));
  *l_next = v;
  return FRSVT_OK;
}

frsvt_status frsvt_get_info(frsvt_handle* h, frsvt_info* info) {
  if (h == nullptr || info == nullptr) return FRSVT_ERR_INVALID_ARG;
  DevState d;
  FRSVT_CK(cudaStreamSynchronize(h->stream));
  FRSVT_CK(cudaMemcpy(&d, h->dst, sizeof(DevState), cudaMemcpyDeviceToHost));
  FRSVT_CK(cudaMemsetAsync(&h->dst->status, 0, sizeof(uint32_t), h->stream));
  FRSVT_CK(cudaStreamSynchronize(h->stream));
  std::memset(info, 0, sizeof(*info));
  info->r = d.r;
  info->s = d.s;
  info->keep = d.keep;
  info->device_status = d.status;
  info->counter = d.counter;
  info->alm_iter = d.iter;
  info->sweeps = d.sweeps;
  info->mu = d.mu;
  info->residual = d.resid_ratio;
  info->rp_residual = d.rp_res;
  return FRSVT_OK;
}

frsvt_status frsvt_get_sigma(frsvt_handle* h, float* sigma_host, int32_t capacity, int32_t* count) {
  if (h == nullptr || sigma_host == nullptr || count == nullptr || capacity < 0) return FRSVT_ERR_INVALID_ARG;
  DevState d;
  FRSVT_CK(cudaStreamSynchronize(h->stream));
  FRSVT_CK(cudaMemcpy(&d, h->dst, sizeof(DevState), cudaMemcpyDeviceToHost));
  int c = d.s < kMaxL ? d.s : kMaxL;
  if (c > capacity) c = capacity;
  for (int i = 0; i < c; ++i) sigma_host[i] = d.sigma[i];
  *count = c;
  return FRSVT_OK;
}

frsvt_status frsvt_enable_timing(frsvt_handle* h, int32_t enable) {
  if (h == nullptr) return FRSVT_ERR_INVALID_ARG;
  if (enable && h->ev_pool.empty()) {
    h->ev_pool.resize(2 * kEventPairs);
    h->ev_phase.resize(kEventPairs);
    for (auto& e : h->ev_pool) FRSVT_CK(cudaEventCreate(&e));
  }
  if (!enable) {
    frsvt_status s = collect_timings(h);
    if (s != FRSVT_OK) return s;
  }
  h->timing = enable ? 1 : 0;
  return FRSVT_OK;
}

frsvt_status frsvt_step_kernels(frsvt_handle* h, int32_t* kernels) {
  if (h == nullptr || kernels == nullptr) return FRSVT_ERR_INVALID_ARG;
  *kernels = h->last_step_kernels;
  return FRSVT_OK;
}

frsvt_status frsvt_wide_pass_plan(int64_t nlong, int64_t nk, int32_t precision, int32_t sms, int32_t* grid,
                                  int32_t* max_parts, int32_t* max_tiles) {
  if (grid == nullptr || max_parts == nullptr || max_tiles == nullptr) return FRSVT_ERR_INVALID_ARG;
  if (nlong < 1 || nk < 1 || sms < 1 || precision < FRSVT_PREC_FP32 || precision > FRSVT_PREC_FP8)
    return FRSVT_ERR_INVALID_ARG;
  int g = 0, mp = 0, mt = 0;
  wide_pass_plan(nlong, nk, precision == FRSVT_PREC_FP32 ? 0 : (precision == FRSVT_PREC_BF16 ? 1 : 2), sms, &g, &mp,
                 &mt);
  *grid = g;
  *max_parts = mp;
  *max_tiles = mt;
  return FRSVT_OK;
}

frsvt_status frsvt_get_timings(frsvt_handle* h, double* ms, int32_t* launches) {
  if (h == nullptr || ms == nullptr || launches == nullptr) return FRSVT_ERR_INVALID_ARG;
  frsvt_status s = collect_timings(h);
  if (s != FRSVT_OK) return s;
  for (int p = 0; p < FRSVT_NPHASE; ++p) {
    ms[p] = h->phase_ms[p];
    launches[p] = h->phase_launches[p];
    h->phase_ms[p] = 0.0;
    h->phase_launches[p] = 0;
  }
  return FRSVT_OK;
}

const char* frsvt_phase_name(int32_t phase) {
  static const char* names[FRSVT_NPHASE] = {"sketch", "power_AQ", "power_AtZ", "reduce", "orth",
                                            "project", "gram", "core", "epilogue", "finish", "apply"};
  return (phase >= 0 && phase < FRSVT_NPHASE) ? names[phase] : "unknown";
}

frsvt_status frsvt_debug_omega(float* out, int64_t rows, int32_t cols, uint64_t seed, uint64_t stream,
                               uint64_t problem, void* cuda_stream) {
  frsvt_handle* h = nullptr;
  if (rows < 0 || cols < 0) return FRSVT_ERR_INVALID_ARG;
  if (rows == 0 || cols == 0) return FRSVT_OK;
  if (out == nullptr) return FRSVT_ERR_INVALID_ARG;
  FRSVT_CK(launch_debug_omega(out, rows, cols, seed, stream, problem, static_cast<cudaStream_t>(cuda_stream)));
  return FRSVT_OK;
}

frsvt_status frsvt_debug_philox(uint64_t* out, int64_t rows, int32_t blocks, uint64_t seed, uint64_t stream,
                                uint64_t problem, void* cuda_stream) {
  frsvt_handle* h = nullptr;
  if (rows < 0 || blocks < 0) return FRSVT_ERR_INVALID_ARG;
  if (rows == 0 || blocks == 0) return FRSVT_OK;
  if (out == nullptr) return FRSVT_ERR_INVALID_ARG;
  FRSVT_CK(launch_debug_philox(out, rows, blocks, seed, stream, problem, static_cast<cudaStream_t>(cuda_stream)));
  return FRSVT_OK;
}

frsvt_status frsvt_debug_wait_timeout(frsvt_handle* h, uint32_t spin_limit) {
  if (h == nullptr) return FRSVT_ERR_INVALID_ARG;
  if (spin_limit < 1 || spin_limit > (1u << 20))
    return fail(h, FRSVT_ERR_INVALID_ARG, "spin_limit must be in [1, 2^20]");
  FRSVT_CK(launch_debug_wait_timeout(spin_limit, h->dst, h->stream));
  return FRSVT_OK;
}

frsvt_status frsvt_debug_rows_tc(frsvt_handle* h, const float* A, int64_t m, int64_t n, int64_t lda, const float* Q,
                                 float* Z) {
  if (h != nullptr && h->wide) return fail(h, FRSVT_ERR_UNSUPPORTED, "needs a handle with l_max <= 32");
  if (h == nullptr) return FRSVT_ERR_INVALID_ARG;
  frsvt_status s = check_shape(h, m, n);
  if (s != FRSVT_OK) return s;
  if ((s = check_matrix(h, A, m, n, lda, "A")) != FRSVT_OK) return s;
  if (Q == nullptr || Z == nullptr) return fail(h, FRSVT_ERR_INVALID_ARG, "Q and Z are required");
  if (n > 256) return fail(h, FRSVT_ERR_UNSUPPORTED, "the tensor-core row pass serves n <= 256");
  if (m == 0 || n == 0) return FRSVT_OK;
  if (!g_tc_prepared) {
    FRSVT_CK(prepare_tc_kernels(static_cast<int>(kSmemLimit)));
    g_tc_prepared = 1;
  }
  CUtensorMap tm;
  if (!make_row_map_sw128(&tm, A, m, n, lda, tc_box_rows()))
    return fail(h, FRSVT_ERR_CUDA, "cuTensorMapEncodeTiled failed for A");
  const int ns = tc_lr_stages(h->LP, n, kSmemLimit - 2048);
  if (ns < 2) return fail(h, FRSVT_ERR_UNSUPPORTED, "tensor-core row pass does not fit");
  FRSVT_CK(launch_tc_lr(h->LP, tm, m, n, h->sms, ns, Q, Z, h->dst, h->stream));
  return FRSVT_OK;
}

frsvt_status frsvt_debug_cols_tc(frsvt_handle* h, const float* A, int64_t m, int64_t n, int64_t lda, const float* B,
                                 uint64_t seed, uint64_t stream, float* Y) {
  if (h != nullptr && h->wide) return fail(h, FRSVT_ERR_UNSUPPORTED, "needs a handle with l_max <= 32");
  if (h == nullptr) return FRSVT_ERR_INVALID_ARG;
  frsvt_status s = check_shape(h, m, n);
  if (s != FRSVT_OK) return s;
  if ((s = check_matrix(h, A, m, n, lda, "A")) != FRSVT_OK) return s;
  if (Y == nullptr) return fail(h, FRSVT_ERR_INVALID_ARG, "Y is required");
  if (n > 256) return fail(h, FRSVT_ERR_UNSUPPORTED, "the tensor-core column pass serves n <= 256");
  if (m == 0 || n == 0) return FRSVT_OK;
  if (!h->tc_sc_ns) return fail(h, FRSVT_ERR_UNSUPPORTED, "tensor-core column pass unavailable for this handle");
  CUtensorMap tmA, tmZ;
  if (!make_row_map_sw128(&tmA, A, m, n, lda, tc_sc_rows(), CU_TENSOR_MAP_SWIZZLE_128B_ATOM_32B) ||
      (B != nullptr && !make_row_map(&tmZ, B, m, h->LP, h->LP, h->LP, tc_sc_rows())))
    return fail(h, FRSVT_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  FRSVT_CK(launch_tc_sc(h->LP, tmA, B ? &tmZ : nullptr, m, n, h->tc_sc_grid, h->tc_sc_ns, seed, stream, h->dst,
                        h->cpart_sc, Y, h->tickets, false, 0, 0, 1, h->Qt, h->Qs, h->cfg.rank_tol, h->stream));
  return FRSVT_OK;
}

// ------------------------------------------------------------------ unrolled iALM RPCA
// Saved-buffer layout of rpca_unrolled_forward, per batch element b and step k (1 <= k <= K):
// A_k, L_k, Y_{k-1} (m x ld floats each; Y_0 = y0_scale_b O is not stored) and the FRSVT factors
// of step k (frsvt_adjoint_saved_bytes), then the backward scratch: Sb, Yb, Lb, Tb, Ab (m x ld
// each) and two arrays of per-CTA partial sums.
struct UrLayout {
  size_t mat, blob, per_step, scratch_off, part_off, acc_off, kid_block, total;
  int grid, kids;
};

static size_t ur_align(size_t x) { return (x + 255) / 256 * 256; }

static UrLayout ur_layout(const frsvt_handle* h, int32_t batch, int32_t steps, int64_t m, int64_t n, int64_t ld) {
  UrLayout u{};
  u.mat = ur_align(sizeof(float) * static_cast<size_t>(m) * static_cast<size_t>(ld));
  u.blob = ur_align(frsvt_adjoint_saved_bytes(h, m, n));
  u.per_step = 3 * u.mat + u.blob;
  u.scratch_off = static_cast<size_t>(batch) * static_cast<size_t>(steps) * u.per_step;
  u.grid = unrolled_grid(m, n, h->sms);
  u.kids = h->kids.empty() ? 1 : static_cast<int>(h->kids.size());
  // per child (or the handle alone): five scratch matrices, two partial arrays and the tt slot,
  // then the child's dtau / dmu accumulators (2 x steps floats)
  u.part_off = 5 * u.mat;
  u.acc_off = u.part_off + ur_align(sizeof(double) * 2 * static_cast<size_t>(u.grid) + 64);
  u.kid_block = u.acc_off + ur_align(sizeof(float) * 2 * static_cast<size_t>(steps));
  u.total = u.scratch_off + static_cast<size_t>(u.kids) * u.kid_block;
  return u;
}

static frsvt_status ur_check(frsvt_handle* h, int32_t batch, int32_t steps, const float* O, int64_t m, int64_t n,
                             int64_t ld, float lambda, int32_t l) {
  if (h == nullptr) return FRSVT_ERR_INVALID_ARG;
  if (h->ad_ws == nullptr) return fail(h, FRSVT_ERR_UNSUPPORTED, "handle created without FRSVT_CFG_ADJOINT");
  if (batch < 0 || steps < 1 || steps > 1024) return fail(h, FRSVT_ERR_INVALID_ARG, "need batch >= 0, 1 <= steps <= 1024");
  frsvt_status s = ad_check(h, O, m, n, ld, l);
  if (s != FRSVT_OK) return s;
  if ((n % 4) != 0) return fail(h, FRSVT_ERR_INVALID_ARG, "the unrolled steps need n % 4 == 0");
  if (!(lambda > 0.f) || !std::isfinite(lambda)) return fail(h, FRSVT_ERR_INVALID_ARG, "lambda must be finite and > 0");
  return FRSVT_OK;
}

// The handle (or child j of it) that runs problem b, and fork / join of the children's streams
// around a batch (the children start after everything enqueued so far on the handle's stream,
// and the handle's stream resumes after all of them).
static frsvt_handle* ur_worker(frsvt_handle* h, int32_t b) {
  return h->kids.empty() ? h : h->kids[static_cast<size_t>(b) % h->kids.size()];
}

static frsvt_status ur_fork(frsvt_handle* h) {
  if (h->kids.empty()) return FRSVT_OK;
  FRSVT_CK(cudaEventRecord(h->fork_event, h->stream));
  for (cudaStream_t ks : h->kid_streams) FRSVT_CK(cudaStreamWaitEvent(ks, h->fork_event, 0));
  return FRSVT_OK;
}

static frsvt_status ur_join(frsvt_handle* h) {
  for (size_t i = 0; i < h->kids.size(); ++i) {
    FRSVT_CK(cudaEventRecord(h->kid_events[i], h->kid_streams[i]));
    FRSVT_CK(cudaStreamWaitEvent(h->stream, h->kid_events[i], 0));
  }
  return FRSVT_OK;
}

size_t rpca_unrolled_saved_bytes(const frsvt_handle* h, int32_t batch, int32_t steps, int64_t m, int64_t n,
                                 int64_t ld) {
  if (h == nullptr || batch < 0 || steps < 1 || m < 0 || n < 0 || ld < n) return 0;
  return ur_layout(h, batch, steps, m, n, ld).total;
}

frsvt_status rpca_unrolled_init(frsvt_handle* h, int32_t batch, const float* O, int64_t m, int64_t n, int64_t ld,
                                double lambda, int32_t power_iters, float* y0_scale) {
  if (h == nullptr || y0_scale == nullptr) return FRSVT_ERR_INVALID_ARG;
  if (batch < 0 || !(lambda > 0.0) || power_iters < 0 || power_iters > 64)
    return fail(h, FRSVT_ERR_INVALID_ARG, "need batch >= 0, lambda > 0, 0 <= power_iters <= 64");
  const size_t step = static_cast<size_t>(m) * static_cast<size_t>(ld);
  for (int32_t b = 0; b < batch; ++b) {
    const float* Ob = O + step * b;
    double nrm = 0.0;
    frsvt_status s = frsvt_spectral_norm(h, Ob, m, n, ld, power_iters, &nrm);
    if (s != FRSVT_OK) return s;
    FRSVT_CK(launch_absmax_sumsq(Ob, m, n, ld, h->pmax, h->psum, h->absmax_blocks, h->stream));
    std::vector<float> pm(h->absmax_blocks);
    FRSVT_CK(cudaMemcpyAsync(pm.data(), h->pmax, sizeof(float) * h->absmax_blocks, cudaMemcpyDeviceToHost, h->stream));
    FRSVT_CK(cudaStreamSynchronize(h->stream));
    double amax = 0.0;
    for (float v : pm) amax = amax > v ? amax : v;
    const double den = nrm > amax / lambda ? nrm : amax / lambda;
    y0_scale[b] = den > 0.0 ? static_cast<float>(1.0 / den) : 0.f;
  }
  return FRSVT_OK;
}

frsvt_status rpca_unrolled_forward(frsvt_handle* h, int32_t batch, int32_t steps, const float* O, int64_t m,
                                   int64_t n, int64_t ld, const float* y0_scale, const float* tau, const float* mu,
                                   float lambda, int32_t l, float* L, void* saved) {
  frsvt_status s = ur_check(h, batch, steps, O, m, n, ld, lambda, l);
  if (s != FRSVT_OK) return s;
  if ((s = check_matrix(h, L, m, n, ld, "L")) != FRSVT_OK) return s;
  if (y0_scale == nullptr || tau == nullptr || mu == nullptr || saved == nullptr)
    return fail(h, FRSVT_ERR_INVALID_ARG, "y0_scale, tau, mu and saved are required");
  for (int32_t k = 0; k < steps; ++k)
    if (!(mu[k] > 0.f) || !std::isfinite(mu[k]) || !(tau[k] >= 0.f) || !std::isfinite(tau[k]))
      return fail(h, FRSVT_ERR_INVALID_ARG, "every mu_k must be finite and > 0, every tau_k finite and >= 0");
  if (batch == 0 || m == 0 || n == 0) return FRSVT_OK;
  const UrLayout u = ur_layout(h, batch, steps, m, n, ld);
  unsigned char* base = static_cast<unsigned char*>(saved);
  const size_t step = static_cast<size_t>(m) * static_cast<size_t>(ld);
  if ((s = ur_fork(h)) != FRSVT_OK) return s;
  for (int32_t b = 0; b < batch; ++b) {
    frsvt_handle* hw = ur_worker(h, b);
    cudaStream_t st = hw->stream;
    float* Sw = reinterpret_cast<float*>(base + u.scratch_off + (b % u.kids) * u.kid_block);   // S_k of the running step
    const float* Ob = O + step * b;
    for (int32_t k = 0; k < steps; ++k) {
      unsigned char* slot = base + (static_cast<size_t>(b) * steps + k) * u.per_step;
      float* Ak = reinterpret_cast<float*>(slot);
      float* Lk = reinterpret_cast<float*>(slot + u.mat);
      float* Yp = reinterpret_cast<float*>(slot + 2 * u.mat);          // Y_{k-1} (k >= 1)
      void* blob = slot + 3 * u.mat;
      if (k == 0) FRSVT_CK(launch_ur_pre(Ob, nullptr, nullptr, y0_scale[b], Ak, m, n, ld, mu[0], u.grid, st));
      float* Lout = (k == steps - 1) ? L + step * b : Lk;
      if ((s = frsvt_svt_save(hw, Ak, m, n, ld, tau[k], l, static_cast<uint64_t>(k), Lout, ld, blob)) != FRSVT_OK)
        return fail(h, s, frsvt_last_error(hw));
      if (k == steps - 1) {
        FRSVT_CK(cudaMemcpy2DAsync(Lk, sizeof(float) * ld, Lout, sizeof(float) * ld, sizeof(float) * n, m,
                                   cudaMemcpyDeviceToDevice, st));
        break;
      }
      unsigned char* next = slot + u.per_step;
      FRSVT_CK(launch_ur_post(Ob, Lk, k == 0 ? nullptr : Yp, y0_scale[b], Sw,
                              reinterpret_cast<float*>(next + 2 * u.mat), reinterpret_cast<float*>(next), m, n, ld,
                              mu[k], mu[k + 1], lambda, u.grid, st));
    }
  }
  return ur_join(h);
}

frsvt_status rpca_unrolled_backward(frsvt_handle* h, int32_t batch, int32_t steps, const float* O, int64_t m,
                                    int64_t n, int64_t ld, const float* y0_scale, const float* tau, const float* mu,
                                    float lambda, int32_t l, const void* saved, const float* dL, float* dtau,
                                    float* dmu) {
  frsvt_status s = ur_check(h, batch, steps, O, m, n, ld, lambda, l);
  if (s != FRSVT_OK) return s;
  if ((s = check_matrix(h, dL, m, n, ld, "dL")) != FRSVT_OK) return s;
  if (y0_scale == nullptr || tau == nullptr || mu == nullptr || saved == nullptr || dtau == nullptr || dmu == nullptr)
    return fail(h, FRSVT_ERR_INVALID_ARG, "y0_scale, tau, mu, saved, dtau and dmu are required");
  FRSVT_CK(cudaMemsetAsync(dtau, 0, sizeof(float) * steps, h->stream));
  FRSVT_CK(cudaMemsetAsync(dmu, 0, sizeof(float) * steps, h->stream));
  if (batch == 0 || m == 0 || n == 0) return FRSVT_OK;
  const UrLayout u = ur_layout(h, batch, steps, m, n, ld);
  unsigned char* base = static_cast<unsigned char*>(const_cast<void*>(saved));
  for (int j = 0; j < u.kids; ++j)                 // the per-worker dtau / dmu accumulators
    FRSVT_CK(cudaMemsetAsync(base + u.scratch_off + j * u.kid_block + u.acc_off, 0, sizeof(float) * 2 * steps,
                             h->stream));
  const size_t step = static_cast<size_t>(m) * static_cast<size_t>(ld);
  if ((s = ur_fork(h)) != FRSVT_OK) return s;
  for (int32_t b = 0; b < batch; ++b) {
    frsvt_handle* hw = ur_worker(h, b);
    cudaStream_t st = hw->stream;
    unsigned char* sc = base + u.scratch_off + (b % u.kids) * u.kid_block;
    float* Sb = reinterpret_cast<float*>(sc);
    float* Yb = reinterpret_cast<float*>(sc + u.mat);
    float* Lb = reinterpret_cast<float*>(sc + 2 * u.mat);
    float* Tb = reinterpret_cast<float*>(sc + 3 * u.mat);
    float* Ab = reinterpret_cast<float*>(sc + 4 * u.mat);
    double* part = reinterpret_cast<double*>(sc + u.part_off);
    double* part2 = part + u.grid;
    float* tt = reinterpret_cast<float*>(part2 + u.grid);              // dtau of one FRSVT adjoint
    float* kdtau = reinterpret_cast<float*>(sc + u.acc_off);
    float* kdmu = kdtau + steps;
    const float* Ob = O + step * b;
    for (int32_t k = steps - 1; k >= 0; --k) {
      unsigned char* slot = base + (static_cast<size_t>(b) * steps + k) * u.per_step;
      const float* Ak = reinterpret_cast<const float*>(slot);
      const float* Lk = reinterpret_cast<const float*>(slot + u.mat);
      const float* Yp = k == 0 ? nullptr : reinterpret_cast<const float*>(slot + 2 * u.mat);
      const void* blob = slot + 3 * u.mat;
      const bool last = k == steps - 1;
      // the last step's L is the output: only the loss's cotangent flows into it
      FRSVT_CK(launch_ur_bwd_post(Ob, Lk, Yp, y0_scale[b], last ? nullptr : Sb, last ? nullptr : Yb,
                                  last ? dL + step * b : nullptr, Lb, Yb, Tb, m, n, ld, mu[k], lambda, part, u.grid,
                                  st));
      if ((s = frsvt_backward(hw, blob, Ak, m, n, ld, tau[k], l, static_cast<uint64_t>(k), Lb, ld, Ab, ld, tt)) !=
          FRSVT_OK)
        return fail(h, s, frsvt_last_error(hw));
      FRSVT_CK(launch_ur_bwd_pre(Ob, Yp, y0_scale[b], Ab, Tb, Sb, Yb, m, n, ld, mu[k], part2, u.grid, st));
      FRSVT_CK(launch_ur_sum(part, u.grid, kdmu + k, 1, st));
      FRSVT_CK(launch_ur_sum(part2, u.grid, kdmu + k, 1, st));
      FRSVT_CK(launch_ur_addf(tt, kdtau + k, st));
    }
  }
  if ((s = ur_join(h)) != FRSVT_OK) return s;
  for (int j = 0; j < u.kids; ++j) {               // the workers' sums, in worker order
    const float* acc = reinterpret_cast<const float*>(base + u.scratch_off + j * u.kid_block + u.acc_off);
    FRSVT_CK(launch_ur_addv(acc, dtau, steps, h->stream));
    FRSVT_CK(launch_ur_addv(acc + steps, dmu, steps, h->stream));
  }
  return FRSVT_OK;
}

}  // extern "C"
