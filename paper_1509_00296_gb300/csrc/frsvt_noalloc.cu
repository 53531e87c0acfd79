// frsvt_svt_noalloc: the FRSVT of frsvt_svt for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc at all: plug-ins hosted by a framework
// that owns every device allocation through its own pool (a second allocator
// would fragment or overcommit that pool), real-time paths that must not enter
// the allocator (cudaMalloc and cudaFree may synchronize the device and take
// unbounded time), and services that fix their device-memory budget at
// start-up.  This entry point needs no handle and allocates nothing: its
// scratch (split-K partials, the basis, the long-side projection, the Gram
// partials and the small device state) lives in one file-scope __device__
// array of FRSVT_NOALLOC_SCRATCH_BYTES that every GPU loading this library
// holds until the process exits.
//
// The address of that array is looked up once per device (with the device
// current) by cudaGetSymbolAddress; host code never passes the array's own
// name to a kernel, because on the host that name is only a stand-in, not a
// device address.  All calls share the array: calls that overlap on the GPU
// (two streams, two host threads) race and corrupt each other's results.
// The device status bits of the kernels (non-finite values, an unconverged
// Jacobi core, a rank-deficient sketch) land in the scratch state and are not
// reported: the call returns FRSVT_OK for every input that passes the host
// checks.
#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/frsvt.h"
#include "state.cuh"

namespace frsvt {

namespace {

constexpr int kNaLP = 16;                       // padded basis width (l <= 16)
constexpr int64_t kNaMaxM = FRSVT_NOALLOC_MAX_M;
constexpr int64_t kNaMaxN = FRSVT_NOALLOC_MAX_N;
constexpr int kNaMaxSplit = 128;                // split-K partials of the row passes
constexpr int kNaMaxGram = 160;                 // Gram partials
constexpr int kNaMaxDevices = 64;

constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t kOffState = 0;
constexpr size_t kOffYs = align256(sizeof(DevState));
constexpr size_t kOffQs = kOffYs + align256(sizeof(float) * kNaMaxN * kNaLP);
constexpr size_t kOffQt = kOffQs + align256(sizeof(float) * kNaMaxN * kNaLP);
constexpr size_t kOffRf = kOffQt + align256(sizeof(float) * kNaMaxN * kNaLP);
constexpr size_t kOffZl = kOffRf + align256(sizeof(float) * kNaMaxN * kNaLP);
constexpr size_t kOffPart = kOffZl + align256(sizeof(float) * kNaMaxM * kNaLP);
constexpr size_t kOffGram = kOffPart + align256(sizeof(float) * kNaMaxSplit * kNaMaxN * kNaLP);
constexpr size_t kNaEnd = kOffGram + align256(sizeof(float2) * kNaMaxGram * kNaLP * kNaLP);
static_assert(kNaEnd <= FRSVT_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds FRSVT_NOALLOC_SCRATCH_BYTES");

struct NaDevice {
  bool ready = false;
  unsigned char* base = nullptr;   // device address of g_noalloc_scratch on this device
  int sms = 1;
};
NaDevice g_na_dev[kNaMaxDevices];
std::mutex g_na_mu;

int64_t cdiv64(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace

// The scratch array.  Device code may name it directly; host code uses the
// address obtained by cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[FRSVT_NOALLOC_SCRATCH_BYTES];

namespace {

frsvt_status na_setup(NaDevice** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) return FRSVT_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_na_mu);
  NaDevice& d = g_na_dev[dev];
  if (!d.ready) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return FRSVT_ERR_CUDA;
    if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return FRSVT_ERR_CUDA;
    if (prepare_pass_kernels(227 * 1024) != cudaSuccess || prepare_small_kernels(227 * 1024) != cudaSuccess)
      return FRSVT_ERR_CUDA;
    d.base = static_cast<unsigned char*>(p);
    d.ready = true;
  }
  *out = &d;
  return FRSVT_OK;
}

}  // namespace
}  // namespace frsvt

using namespace frsvt;

extern "C" frsvt_status frsvt_svt_noalloc(const float* A, int64_t m, int64_t n, int64_t lda, float tau, int32_t l,
                                          int32_t q, uint64_t seed, uint64_t counter, float* X, int64_t ldx,
                                          void* stream) {
  if (m < 0 || n < 0) return FRSVT_ERR_INVALID_ARG;
  if (m < n) return FRSVT_ERR_UNSUPPORTED;
  if (m > kNaMaxM || n > kNaMaxN) return FRSVT_ERR_INVALID_ARG;      // beyond the scratch array
  if (l < 1 || l > kNaLP || q < 0 || q > 64) return FRSVT_ERR_INVALID_ARG;
  if (!(tau >= 0.f) || !std::isfinite(tau)) return FRSVT_ERR_INVALID_ARG;
  if (counter == kCounterFromState) return FRSVT_ERR_INVALID_ARG;   // reserved stream index
  if (m == 0 || n == 0) return FRSVT_OK;
  if (A == nullptr || X == nullptr || static_cast<const void*>(A) == static_cast<const void*>(X))
    return FRSVT_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(A) & 15u) || (reinterpret_cast<uintptr_t>(X) & 15u)) return FRSVT_ERR_INVALID_ARG;
  if (lda < n || ldx < n || (lda % 4) || (ldx % 4)) return FRSVT_ERR_INVALID_ARG;
  if (l > n) l = static_cast<int32_t>(n);

  NaDevice* d = nullptr;
  frsvt_status s = na_setup(&d);
  if (s != FRSVT_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  DevState* dst = reinterpret_cast<DevState*>(d->base + kOffState);
  float* Ys = reinterpret_cast<float*>(d->base + kOffYs);
  float* Qs = reinterpret_cast<float*>(d->base + kOffQs);
  float* Qt = reinterpret_cast<float*>(d->base + kOffQt);
  float* Rf = reinterpret_cast<float*>(d->base + kOffRf);
  float* Zl = reinterpret_cast<float*>(d->base + kOffZl);
  float* part = reinterpret_cast<float*>(d->base + kOffPart);
  float2* gpart = reinterpret_cast<float2*>(d->base + kOffGram);

  // Split-K layout of the row passes, bounded by the scratch reserved for partials.
  const int64_t ntiles = cdiv64(n, 256);
  int64_t nsplit = cdiv64(4 * d->sms, ntiles);
  if (nsplit > kNaMaxSplit / ntiles) nsplit = kNaMaxSplit / ntiles;
  if (nsplit > cdiv64(m, 32)) nsplit = cdiv64(m, 32);
  if (nsplit < 1) nsplit = 1;
  const int64_t rps = cdiv64(cdiv64(m, nsplit), 32) * 32;
  nsplit = cdiv64(m, rps);
  int gsplit = static_cast<int>(cdiv64(m, 32));
  if (gsplit > d->sms) gsplit = d->sms;
  if (gsplit > kNaMaxGram) gsplit = kNaMaxGram;
  const double tol = 1e-12;

#define NA_CK(call)                                  \
  do {                                               \
    if ((call) != cudaSuccess) return FRSVT_ERR_CUDA; \
  } while (0)
  // Every region a kernel reads before writing it in this call starts at zero.
  NA_CK(cudaMemsetAsync(dst, 0, sizeof(DevState), st));
  NA_CK(launch_short_cols(kNaLP, A, m, n, lda, nullptr, seed, counter, dst, part, static_cast<int>(nsplit), rps, st));
  NA_CK(launch_reduce_parts(part, static_cast<int>(nsplit), n * kNaLP, Ys, st));
  NA_CK(launch_orth(kNaLP, Ys, n, l, 0, Qt, Qs, dst, tol, st));
  for (int it = 0; it < q; ++it) {
    NA_CK(launch_long_rows(kNaLP, A, m, n, lda, Qs, Zl, 8 * d->sms, st));
    NA_CK(launch_short_cols(kNaLP, A, m, n, lda, Zl, seed, counter, dst, part, static_cast<int>(nsplit), rps, st));
    NA_CK(launch_reduce_parts(part, static_cast<int>(nsplit), n * kNaLP, Ys, st));
    NA_CK(launch_orth(kNaLP, Ys, n, l, 0, Qt, Qs, dst, tol, st));
  }
  NA_CK(launch_long_rows(kNaLP, A, m, n, lda, Qs, Zl, 8 * d->sms, st));
  NA_CK(launch_gram_long(kNaLP, Zl, m, gpart, gsplit, st));
  NA_CK(launch_core(kNaLP, gpart, gsplit, Qs, n, l, tau, 0, 0, 0, Rf, Qt, dst, tol, 30, st));
  NA_CK(launch_recon(kNaLP, Zl, Rf, m, n, X, ldx, static_cast<int>(nsplit), rps, st));
#undef NA_CK
  return FRSVT_OK;
}
