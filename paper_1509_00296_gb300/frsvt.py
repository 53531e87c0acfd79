"""Thin ctypes binding of libfrsvt.so (argument marshalling only).

Every computation runs in the library's CUDA kernels; this module only turns
torch tensors into device pointers and the caller's CUDA stream into the
handle's stream.  If the library has not been built the first call raises:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfrsvt.so")

FRSVT_OK = 0
STATUS_NAMES = {0: "FRSVT_OK", 1: "FRSVT_ERR_INVALID_ARG", 2: "FRSVT_ERR_UNSUPPORTED", 3: "FRSVT_ERR_ALLOC",
                4: "FRSVT_ERR_CUDA", 5: "FRSVT_ERR_RANK_DEFICIENT", 6: "FRSVT_ERR_NOT_CONVERGED",
                7: "FRSVT_ERR_NONFINITE"}
DEV_RANK_DEFICIENT, DEV_NOT_CONVERGED, DEV_NONFINITE, DEV_TIMEOUT, DEV_BAD_PROBLEM = 1, 2, 4, 8, 16
WSVT_EXACT, WSVT_FRSVT = 0, 1
CFG_ADJOINT = 1
CFG_ORTH_LAST = 2
PREC_FP32, PREC_BF16, PREC_FP8 = 0, 1, 2
NPHASE = 11


class FrsvtError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [("m_max", ctypes.c_int64), ("n_max", ctypes.c_int64), ("l_max", ctypes.c_int32),
                ("q", ctypes.c_int32), ("range_prop", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("max_jacobi_sweeps", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("rank_tol", ctypes.c_double), ("problem_streams", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("r", ctypes.c_int32), ("s", ctypes.c_int32), ("keep", ctypes.c_int32),
                ("device_status", ctypes.c_uint32), ("counter", ctypes.c_uint64), ("alm_iter", ctypes.c_int32),
                ("sweeps", ctypes.c_int32), ("mu", ctypes.c_double), ("residual", ctypes.c_double),
                ("rp_residual", ctypes.c_float), ("reserved", ctypes.c_int32)]


_lib = None
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_SIGS = {
    "frsvt_create": [ctypes.POINTER(_P), ctypes.POINTER(Config), _P],
    "frsvt_destroy": [_P],
    "frsvt_set_stream": [_P, _P],
    "frsvt_reset": [_P, ctypes.c_uint64],
    "frsvt_svt": [_P, _P, _I64, _I64, _I64, ctypes.c_float, ctypes.c_int32, _P, _I64],
    "frsvt_spectral_norm": [_P, _P, _I64, _I64, _I64, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)],
    "frsvt_svt_factors": [_P, _P, _I64, _I64, _I64, ctypes.c_float, ctypes.c_int32, _P, _I64, _P, _I64, _P],
    "rpca_init": [_P, _P, _P, _P, _I64, _I64, _I64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                  ctypes.c_double, ctypes.c_int32],
    "rpca_ialm_step": [_P, _P, _P, _P, _I64, _I64, _I64, ctypes.c_int32, _P, _I64, ctypes.POINTER(ctypes.c_double)],
    "frsvt_get_info": [_P, ctypes.POINTER(Info)],
    "frsvt_get_sigma": [_P, ctypes.POINTER(ctypes.c_float), ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)],
    "frsvt_set_rank_prediction": [_P, ctypes.c_int32, ctypes.c_double, ctypes.c_double],
    "frsvt_get_rank_prediction": [_P, ctypes.POINTER(ctypes.c_int32)],
    "frsvt_set_partial": [_P, ctypes.c_int32],
    "frsvt_status_string": [ctypes.c_int],
    "frsvt_last_error": [_P],
    "frsvt_enable_timing": [_P, ctypes.c_int32],
    "frsvt_get_timings": [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)],
    "frsvt_step_kernels": [_P, ctypes.POINTER(ctypes.c_int32)],
    "frsvt_wide_pass_plan": [_I64, _I64, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                             ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)],
    "frsvt_lrr_create": [ctypes.POINTER(_P), _I64, _I64, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                         ctypes.c_int32, _P],
    "frsvt_lrr_destroy": [_P],
    "frsvt_lrr_init": [_P, _P, _I64, _I64, _I64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                       ctypes.c_double],
    "frsvt_lrr_step": [_P, ctypes.POINTER(ctypes.c_double)],
    "frsvt_lrr_get": [_P, _P, _I64, _P, _I64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)],
    "frsvt_lrr_last_error": [_P],
    "frsvt_phase_name": [ctypes.c_int32],
    "frsvt_svt_save": [_P, _P, _I64, _I64, _I64, ctypes.c_float, ctypes.c_int32, ctypes.c_uint64, _P, _I64, _P],
    "frsvt_backward": [_P, _P, _P, _I64, _I64, _I64, ctypes.c_float, ctypes.c_int32, ctypes.c_uint64, _P, _I64, _P,
                       _I64, _P],
    "frsvt_wsvt": [_P, ctypes.c_int32, _P, _P, ctypes.c_int32, ctypes.c_float, ctypes.c_float, _P, ctypes.c_int32,
                   ctypes.c_int32],
    "frsvt_wsvt_tune": [_P, ctypes.c_int32, _P, _P, ctypes.c_int32, ctypes.c_float, ctypes.c_float, _P,
                        ctypes.c_int32, ctypes.c_int32],
    "frsvt_wsvt_get_tuning": [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)],
    "frsvt_debug_rows_tc": [_P, _P, _I64, _I64, _I64, _P, _P],
    "frsvt_debug_cols_tc": [_P, _P, _I64, _I64, _I64, _P, ctypes.c_uint64, ctypes.c_uint64, _P],
    "frsvt_debug_omega": [_P, _I64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, _P],
    "frsvt_debug_philox": [_P, _I64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, _P],
    "frsvt_debug_wait_timeout": [_P, ctypes.c_uint32],
    "rpca_unrolled_init": [_P, ctypes.c_int32, _P, _I64, _I64, _I64, ctypes.c_double, ctypes.c_int32, _P],
    "rpca_unrolled_forward": [_P, ctypes.c_int32, ctypes.c_int32, _P, _I64, _I64, _I64, _P, _P, _P, ctypes.c_float,
                              ctypes.c_int32, _P, _P],
    "rpca_unrolled_backward": [_P, ctypes.c_int32, ctypes.c_int32, _P, _I64, _I64, _I64, _P, _P, _P, ctypes.c_float,
                               ctypes.c_int32, _P, _P, _P, _P],
}


def lib():
    """Load libfrsvt.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1509_00296_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = (ctypes.c_char_p if name in ("frsvt_status_string", "frsvt_last_error", "frsvt_phase_name",
                                                      "frsvt_lrr_last_error")
                          else ctypes.c_int)
        L.frsvt_adjoint_saved_bytes.argtypes = [_P, _I64, _I64]
        L.frsvt_adjoint_saved_bytes.restype = ctypes.c_size_t
        L.rpca_unrolled_saved_bytes.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, _I64, _I64, _I64]
        L.rpca_unrolled_saved_bytes.restype = ctypes.c_size_t
        _lib = L
    return _lib


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _check_f32_cuda(t, name):
    import torch
    if t.dtype != torch.float32 or not t.is_cuda:
        raise TypeError(f"{name} must be a float32 CUDA tensor")
    if t.dim() != 2 or t.stride(1) != 1:
        raise TypeError(f"{name} must be a 2-D tensor with unit column stride")


@dataclass
class SVTInfo:
    r: int
    s: int
    keep: int
    device_status: int
    counter: int
    alm_iter: int
    mu: float
    residual: float
    sweeps: int = 0
    rp_residual: float = -1.0

    def residual_estimate(self, alpha: float = 20.0) -> float:
        """Prop. 4 / Eq. 14: alpha sqrt(2/pi) ||(I - Q~ Q~^T) A^T omega||, an upper bound on
        sigma_{k+1} with probability >= 1 - 1/alpha (-1 when unavailable)."""
        if self.rp_residual < 0:
            return -1.0
        return alpha * math.sqrt(2.0 / math.pi) * self.rp_residual


class Handle:
    """An FRSVT handle: workspace, propagated basis and Omega counter (include/frsvt.h)."""

    def __init__(self, m_max: int, n_max: int, l_max: int, q: int = 2, range_prop: bool = True,
                 seed: int = 0, max_jacobi_sweeps: int = 30, rank_tol: float = 1e-12, stream=None,
                 adjoint: bool = False, precision: int = 0, orth_last: bool = False, problem_streams: int = 0):
        flags = (CFG_ADJOINT if adjoint else 0) | (CFG_ORTH_LAST if orth_last else 0)
        cfg = Config(m_max, n_max, l_max, q, 1 if range_prop else 0, precision, seed, max_jacobi_sweeps,
                     flags, rank_tol, problem_streams)
        h = _P()
        self._stream = stream
        st = lib().frsvt_create(ctypes.byref(h), ctypes.byref(cfg), _stream_ptr(stream))
        if st != FRSVT_OK:
            raise FrsvtError(st, "frsvt_create failed")
        self._h = h
        self.cfg = cfg

    def close(self):
        if getattr(self, "_h", None):
            lib().frsvt_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, st):
        if st != FRSVT_OK:
            raise FrsvtError(st, lib().frsvt_last_error(self._h).decode())

    def set_stream(self, stream=None):
        self._stream = stream
        self._chk(lib().frsvt_set_stream(self._h, _stream_ptr(stream)))

    def reset(self, counter: int = 0):
        self._chk(lib().frsvt_reset(self._h, counter))

    def svt(self, A, tau: float, l: int, X=None):
        """X = FRSVT_tau(A) with l sketch columns (Alg. 1)."""
        import torch
        _check_f32_cuda(A, "A")
        if X is None:
            X = torch.empty_like(A)
        _check_f32_cuda(X, "X")
        m, n = A.shape
        self._chk(lib().frsvt_svt(self._h, _ptr(A), m, n, A.stride(0), float(tau), int(l), _ptr(X), X.stride(0)))
        return X

    def svt_factors(self, A, tau: float, l: int, width: int | None = None):
        """FRSVT_tau(A) in factored form: returns (U, V, r) with X = U V^T, U = A Q (m x width),
        V = Q M (n x width), r a 1-element int32 CUDA tensor (#{sigma > tau}); width defaults to l."""
        import torch
        _check_f32_cuda(A, "A")
        m, n = A.shape
        w = int(l if width is None else width)
        U = torch.empty((m, w), dtype=torch.float32, device=A.device)
        V = torch.empty((n, w), dtype=torch.float32, device=A.device)
        r = torch.empty(1, dtype=torch.int32, device=A.device)
        self._chk(lib().frsvt_svt_factors(self._h, _ptr(A), m, n, A.stride(0), float(tau), int(l), _ptr(U), w,
                                          _ptr(V), w, _ptr(r)))
        return U, V, r

    def spectral_norm(self, A, iters: int = 20) -> float:
        _check_f32_cuda(A, "A")
        out = ctypes.c_double()
        m, n = A.shape
        self._chk(lib().frsvt_spectral_norm(self._h, _ptr(A), m, n, A.stride(0), int(iters), ctypes.byref(out)))
        return out.value

    def rpca_init(self, O, S, A, lam: float, rho: float = 1.5, mu_bar_factor: float = 1e7,
                  normO2: float = 0.0, power_iters: int = 30):
        for t, nm in ((O, "O"), (S, "S"), (A, "A")):
            _check_f32_cuda(t, nm)
        m, n = O.shape
        self._chk(lib().rpca_init(self._h, _ptr(O), _ptr(S), _ptr(A), m, n, O.stride(0), float(lam), float(rho),
                                  float(mu_bar_factor), float(normO2), int(power_iters)))

    def ialm_step(self, O, S, A, l: int, L=None, sync_residual: bool = False):
        m, n = O.shape
        res = ctypes.c_double()
        self._chk(lib().rpca_ialm_step(self._h, _ptr(O), _ptr(S), _ptr(A), m, n, O.stride(0), int(l),
                                       _ptr(L), L.stride(0) if L is not None else 0,
                                       ctypes.byref(res) if sync_residual else None))
        return res.value if sync_residual else None

    def set_rank_prediction(self, a: int = 2, rho: float = 0.05, gamma: float = 0.1):
        """Adaptive rank prediction of Eq. 7 (a = 0 switches it off)."""
        self._chk(lib().frsvt_set_rank_prediction(self._h, int(a), float(rho), float(gamma)))

    def set_partial(self, k: int):
        """Partial thresholding (Table 6, Type B): keep the k leading singular values (0: plain SVT)."""
        self._chk(lib().frsvt_set_partial(self._h, int(k)))

    def rank_prediction(self) -> int:
        """Sampling rate the next SVT will use under adaptive rank prediction."""
        v = ctypes.c_int32()
        self._chk(lib().frsvt_get_rank_prediction(self._h, ctypes.byref(v)))
        return v.value

    def info(self) -> SVTInfo:
        inf = Info()
        self._chk(lib().frsvt_get_info(self._h, ctypes.byref(inf)))
        return SVTInfo(inf.r, inf.s, inf.keep, inf.device_status, inf.counter, inf.alm_iter, inf.mu, inf.residual,
                       inf.sweeps, inf.rp_residual)

    def enable_timing(self, on: bool = True):
        self._chk(lib().frsvt_enable_timing(self._h, 1 if on else 0))

    def step_kernels(self) -> int:
        """Kernel launches of the graph the last ialm_step replayed (0 if it launched directly)."""
        n = ctypes.c_int32(0)
        self._chk(lib().frsvt_step_kernels(self._h, ctypes.byref(n)))
        return n.value

    def timings(self):
        """{phase name: (device ms, launches)} since the last call (synchronizes)."""
        ms = (ctypes.c_double * NPHASE)()
        cnt = (ctypes.c_int32 * NPHASE)()
        self._chk(lib().frsvt_get_timings(self._h, ms, cnt))
        return {lib().frsvt_phase_name(p).decode(): (ms[p], cnt[p]) for p in range(NPHASE)}

    def debug_rows_tc(self, A, Q):
        """Z = A Q by the tensor-core row pass (Q: n x LP float32 CUDA tensor)."""
        import torch
        _check_f32_cuda(A, "A")
        m, n = A.shape
        Z = torch.empty((m, Q.shape[1]), dtype=torch.float32, device=A.device)
        self._chk(lib().frsvt_debug_rows_tc(self._h, _ptr(A), m, n, A.stride(0), _ptr(Q), _ptr(Z)))
        return Z

    def debug_cols_tc(self, A, LP: int, B=None, seed: int = 0, stream: int = 0):
        """Y = A^T B by the tensor-core column pass (B: m x LP tensor, or None for the Omega stream)."""
        import torch
        _check_f32_cuda(A, "A")
        m, n = A.shape
        Y = torch.empty((n, LP), dtype=torch.float32, device=A.device)
        self._chk(lib().frsvt_debug_cols_tc(self._h, _ptr(A), m, n, A.stride(0), _ptr(B), seed, stream, _ptr(Y)))
        return Y

    def debug_wait_timeout(self, spin_limit: int = 1000):
        """Run one bounded mbarrier wait that nothing satisfies (sets DEV_TIMEOUT in the status)."""
        self._chk(lib().frsvt_debug_wait_timeout(self._h, int(spin_limit)))

    def svt_save(self, A, tau: float, l: int, omega_stream: int = 0, X=None, saved=None):
        """X = FRSVT_tau(A) recording the factors of the backward pass; returns (X, saved)."""
        import torch
        _check_f32_cuda(A, "A")
        m, n = A.shape
        if X is None:
            X = torch.empty_like(A)
        if saved is None:
            nb = lib().frsvt_adjoint_saved_bytes(self._h, m, n)
            saved = torch.empty(nb, dtype=torch.uint8, device=A.device)
        self._chk(lib().frsvt_svt_save(self._h, _ptr(A), m, n, A.stride(0), tau, l, omega_stream, _ptr(X),
                                       X.stride(0), _ptr(saved)))
        return X, saved

    def backward(self, saved, A, tau: float, l: int, omega_stream: int, dX, dA=None, dtau=None):
        """Vector-Jacobian product of the FRSVT map: returns (dA, dtau) for the cotangent dX."""
        import torch
        _check_f32_cuda(A, "A")
        _check_f32_cuda(dX, "dX")
        m, n = A.shape
        if dA is None:
            dA = torch.empty_like(A)
        if dtau is None:
            dtau = torch.empty(1, dtype=torch.float32, device=A.device)
        self._chk(lib().frsvt_backward(self._h, _ptr(saved), _ptr(A), m, n, A.stride(0), tau, l, omega_stream,
                                       _ptr(dX), dX.stride(0), _ptr(dA), dA.stride(0), _ptr(dtau)))
        return dA, dtau

    def unrolled_init(self, Ob, lam: float, power_iters: int = 30):
        """y0 scales of a batch (B, m, n contiguous float32 CUDA tensor): a list of B floats."""
        B, m, n = Ob.shape
        out = (ctypes.c_float * B)()
        self._chk(lib().rpca_unrolled_init(self._h, B, _ptr(Ob), m, n, n, float(lam), int(power_iters), out))
        return [out[i] for i in range(B)]

    def unrolled_forward(self, Ob, y0_scale, tau, mu, lam: float, l: int, saved=None):
        """L_K of the unrolled iALM for a batch (B, m, n); tau, mu: sequences of K floats.
        Returns (L, saved)."""
        import torch
        B, m, n = Ob.shape
        K = len(tau)
        if saved is None:
            nb = lib().rpca_unrolled_saved_bytes(self._h, B, K, m, n, n)
            saved = torch.empty(nb, dtype=torch.uint8, device=Ob.device)
        L = torch.empty_like(Ob)
        f = ctypes.c_float
        self._chk(lib().rpca_unrolled_forward(self._h, B, K, _ptr(Ob), m, n, n, (f * B)(*y0_scale), (f * K)(*tau),
                                              (f * K)(*mu), float(lam), int(l), _ptr(L), _ptr(saved)))
        return L, saved

    def unrolled_backward(self, Ob, y0_scale, tau, mu, lam: float, l: int, saved, dL):
        """(dtau, dmu) as float32 CUDA tensors of K entries for the cotangent dL of L_K."""
        import torch
        B, m, n = Ob.shape
        K = len(tau)
        dtau = torch.empty(K, dtype=torch.float32, device=Ob.device)
        dmu = torch.empty(K, dtype=torch.float32, device=Ob.device)
        f = ctypes.c_float
        self._chk(lib().rpca_unrolled_backward(self._h, B, K, _ptr(Ob), m, n, n, (f * B)(*y0_scale), (f * K)(*tau),
                                               (f * K)(*mu), float(lam), int(l), _ptr(saved), _ptr(dL.contiguous()),
                                               _ptr(dtau), _ptr(dmu)))
        return dtau, dmu

    def wsvt_raw(self, A_ptrs, n_i, m: int, c: float, eps: float, X_ptrs, variant: int = WSVT_EXACT,
                 l: int = 12, tune: bool = False):
        """Batched weighted SVT on device arrays: A_ptrs / X_ptrs int64 CUDA tensors of device
        pointers (problem b: m x n_b row-major contiguous float32), n_i an int32 CUDA tensor."""
        import torch
        if A_ptrs.dtype != torch.int64 or X_ptrs.dtype != torch.int64 or n_i.dtype != torch.int32:
            raise TypeError("A_ptrs / X_ptrs must be int64 and n_i int32 CUDA tensors")
        batch = int(n_i.numel())
        fn = lib().frsvt_wsvt_tune if tune else lib().frsvt_wsvt
        self._chk(fn(self._h, batch, _ptr(A_ptrs), _ptr(n_i), m, c, eps, _ptr(X_ptrs), variant, l))

    def wsvt(self, mats, c: float, eps: float, variant: int = WSVT_EXACT, l: int = 12, out=None,
             tune: bool = False):
        """Batched weighted SVT of a list of m x n_b float32 CUDA tensors; returns the list of X_b."""
        import torch
        if not mats:
            return []
        m = mats[0].shape[0]
        for t in mats:
            _check_f32_cuda(t, "A_b")
            if t.shape[0] != m or not t.is_contiguous():
                raise TypeError("every A_b must be a contiguous m x n_b tensor with the same m")
        if out is None:
            out = [torch.empty_like(t) for t in mats]
        dev = mats[0].device
        a = torch.tensor([t.data_ptr() for t in mats], dtype=torch.int64, device=dev)
        x = torch.tensor([t.data_ptr() for t in out], dtype=torch.int64, device=dev)
        n = torch.tensor([t.shape[1] for t in mats], dtype=torch.int32, device=dev)
        self._keep = (a, x, n)                 # alive until the asynchronous launch has read them
        self.wsvt_raw(a, n, m, c, eps, x, variant, l, tune)
        return out

    def wsvt_tuning(self, variant: int = WSVT_EXACT):
        nt, cps = ctypes.c_int32(), ctypes.c_int32()
        self._chk(lib().frsvt_wsvt_get_tuning(self._h, variant, ctypes.byref(nt), ctypes.byref(cps)))
        return nt.value, cps.value

    def sigma(self):
        buf = (ctypes.c_float * 128)()
        cnt = ctypes.c_int32()
        self._chk(lib().frsvt_get_sigma(self._h, buf, 128, ctypes.byref(cnt)))
        return [buf[i] for i in range(cnt.value)]


def wide_pass_plan(nlong: int, nk: int, precision: int = 0, sms: int = 152):
    """(grid, max_parts, max_tiles) of one wide-basis pass over A (frsvt_wide_pass_plan): the CTA
    count, the most partials of one tile, the most tiles of one CTA's range.  Host arithmetic."""
    g, mp, mt = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
    st = lib().frsvt_wide_pass_plan(int(nlong), int(nk), int(precision), int(sms), ctypes.byref(g), ctypes.byref(mp),
                                    ctypes.byref(mt))
    if st != 0:
        raise FrsvtError(st, "frsvt_wide_pass_plan")
    return g.value, mp.value, mt.value


def debug_omega(rows: int, cols: int, seed: int, stream: int, problem: int = 0):
    """Omega[:rows, :cols] of the (seed, stream, problem) Philox stream, computed by the CUDA kernel."""
    import torch
    out = torch.empty((rows, cols), dtype=torch.float32, device="cuda")
    st = lib().frsvt_debug_omega(_ptr(out), rows, cols, seed, stream, problem, _stream_ptr())
    if st != FRSVT_OK:
        raise FrsvtError(st, "frsvt_debug_omega")
    return out


def debug_philox(rows: int, blocks: int, seed: int, stream: int, problem: int = 0):
    """Raw Philox4x64-10 words (rows x blocks x 4, as int64 bit patterns) from the CUDA kernel."""
    import torch
    out = torch.empty((rows, blocks, 4), dtype=torch.int64, device="cuda")
    st = lib().frsvt_debug_philox(_ptr(out), rows, blocks, seed, stream, problem, _stream_ptr())
    if st != FRSVT_OK:
        raise FrsvtError(st, "frsvt_debug_philox")
    return out


def rpca(O, lam=None, l: int = 10, q: int = 2, iters: int = 30, rho: float = 1.5, mu_bar_factor: float = 1e7,
         seed: int = 0, range_prop: bool = True, tol: float = 0.0, return_L: bool = True):
    """Robust PCA of O (float32 CUDA tensor) by inexact ALM with FRSVT; returns (L, S, info).

    Runs `iters` iterations, or stops early once ||O - L - S||_F / ||O||_F < tol
    (checked on the host each iteration when tol > 0).
    """
    import torch
    m, n = O.shape
    lam = 1.0 / max(m, n) ** 0.5 if lam is None else lam
    h = Handle(m, n, l, q=q, range_prop=range_prop, seed=seed)
    S = torch.empty_like(O)
    A = torch.empty_like(O)
    L = torch.empty_like(O) if return_L else None
    h.rpca_init(O, S, A, lam, rho, mu_bar_factor)
    for k in range(iters):
        last = k == iters - 1
        res = h.ialm_step(O, S, A, l, L=L if (last or tol > 0) else None, sync_residual=tol > 0)
        if tol > 0 and res < tol:
            break
    info = h.info()
    h.close()
    return L, S, info


def _autograd_function():
    import torch

    class FRSVTFunction(torch.autograd.Function):
        """X = FRSVT_tau(A) (fixed Omega stream) with the library's adjoint as its backward.

        Inputs: A (m x n float32 CUDA, m >= n), tau (0-d float32 tensor), and non-tensor
        arguments handle (created with adjoint=True), l, omega_stream.
        """

        @staticmethod
        def forward(ctx, A, tau, handle, l, omega_stream):
            A = A.contiguous()
            t = float(tau)
            X, saved = handle.svt_save(A, t, l, omega_stream)
            ctx.save_for_backward(A, saved)
            ctx.meta = (handle, t, l, omega_stream)
            return X

        @staticmethod
        def backward(ctx, dX):
            A, saved = ctx.saved_tensors
            handle, t, l, omega_stream = ctx.meta
            dA, dtau = handle.backward(saved, A, t, l, omega_stream, dX.contiguous())
            return dA, dtau.reshape(()), None, None, None

    return FRSVTFunction


def frsvt_svt_autograd(A, tau, handle, l: int, omega_stream: int = 0):
    """Differentiable X = FRSVT_tau(A): gradients with respect to A and tau by the library's adjoint."""
    return _autograd_function().apply(A, tau, handle, l, omega_stream)


class LRR:
    """Low-rank representation (Table 6, Type A) by the inexact ALM on the GPU, the J step by
    FRSVT (include/frsvt.h, frsvt_lrr_*).  O: d x n float32 CUDA tensor, kept referenced."""

    def __init__(self, d_max: int, n_max: int, l: int, q: int = 1, seed: int = 0, range_prop: bool = True,
                 stream=None):
        h = _P()
        st = lib().frsvt_lrr_create(ctypes.byref(h), d_max, n_max, l, q, seed, 1 if range_prop else 0,
                                     _stream_ptr(stream))
        if st != FRSVT_OK:
            raise FrsvtError(st, "frsvt_lrr_create failed")
        self._h = h
        self._O = None

    def close(self):
        if getattr(self, "_h", None):
            lib().frsvt_lrr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, st):
        if st != FRSVT_OK:
            raise FrsvtError(st, lib().frsvt_lrr_last_error(self._h).decode())

    def init(self, O, lam: float, mu0: float = 1e-6, rho: float = 1.1, mu_max: float = 1e10):
        _check_f32_cuda(O, "O")
        self._O = O
        d, n = O.shape
        self._chk(lib().frsvt_lrr_init(self._h, _ptr(O), d, n, O.stride(0), lam, mu0, rho, mu_max))

    def step(self, sync_err: bool = False):
        """One iteration; with sync_err the max-norm residual (synchronizes)."""
        e = ctypes.c_double(0.0)
        self._chk(lib().frsvt_lrr_step(self._h, ctypes.byref(e) if sync_err else None))
        return e.value if sync_err else None

    def result(self):
        """(L, S, next mu, iterations) with L and S as new float32 CUDA tensors."""
        import torch
        d, n = self._O.shape
        L = torch.empty((n, n), dtype=torch.float32, device=self._O.device)
        S = torch.empty((d, n), dtype=torch.float32, device=self._O.device)
        mu = ctypes.c_double(0.0)
        it = ctypes.c_int32(0)
        self._chk(lib().frsvt_lrr_get(self._h, _ptr(L), n, _ptr(S), n, ctypes.byref(mu), ctypes.byref(it)))
        return L, S, mu.value, it.value
