"""frsvt_svt_noalloc: the allocation-free FRSVT entry point for callers that cannot allocate.

Plug-ins whose host framework owns every device allocation, real-time paths that must not
enter the allocator (cudaMalloc may synchronize the device), and services with a device-memory
budget fixed at start-up cannot call cudaMalloc; the entry point keeps its scratch in a static
device array instead.  These tests call it through the C ABI twice in a row per shape and compare
each result with the handle-based frsvt_svt on the same input, seed and Omega stream index,
within the parity tolerance of the other GPU tests (relative Frobenius error <= 1e-4).  The
shapes cover the largest size the scratch array serves (65536 x 256, l = 16), a row count that is
no multiple of any tile with a padded leading dimension, and q = 0.  The file name puts it last
in collection order.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
TOL = 1e-4


def _noalloc_fn():
    from paper_1509_00296_gb300 import build, frsvt
    build.build()
    fn = frsvt.lib().frsvt_svt_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_float, ctypes.c_int32,
                   ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return frsvt, fn


@pytest.mark.parametrize("m,n,ld,l,q", [(20000, 200, 200, 12, 2), (65536, 256, 256, 16, 1), (4099, 130, 136, 10, 0)])
def test_noalloc_matches_handle_path_two_calls(m, n, ld, l, q):
    import torch
    assert torch.cuda.is_available()
    frsvt, fn = _noalloc_fn()
    seed = 77
    rng = np.random.default_rng(4 + m)
    U, _ = np.linalg.qr(rng.standard_normal((m, 40)))
    V, _ = np.linalg.qr(rng.standard_normal((n, 40)))
    s = 30.0 * 0.85 ** np.arange(40)
    A0 = ((U * s) @ V.T).astype(np.float32)
    A1 = (A0 + 0.01 * rng.standard_normal((m, n))).astype(np.float32)
    tau = float(0.5 * (s[5] + s[6]))
    h = frsvt.Handle(m, n, 16, q=q, range_prop=False, seed=seed)
    stream = torch.cuda.current_stream()
    for counter, A in enumerate((A0, A1)):
        Abuf = torch.zeros((m, ld), dtype=torch.float32, device="cuda")
        Abuf[:, :n] = torch.from_numpy(A).cuda()
        Ag = Abuf[:, :n]
        Xr = torch.zeros((m, ld), dtype=torch.float32, device="cuda")[:, :n]
        X_ref = h.svt(Ag, tau, l, X=Xr).cpu().numpy()         # handle path, Omega stream index = counter
        Xbuf = torch.full((m, ld), float("nan"), dtype=torch.float32, device="cuda")
        st = fn(ctypes.c_void_p(Ag.data_ptr()), m, n, ld, tau, l, q, seed, counter,
                ctypes.c_void_p(Xbuf.data_ptr()), ld, ctypes.c_void_p(stream.cuda_stream))
        assert st == 0
        torch.cuda.synchronize()
        Xn = Xbuf[:, :n].cpu().numpy()
        assert np.all(np.isfinite(Xn))
        assert np.all(np.isnan(Xbuf[:, n:].cpu().numpy()))    # the padding columns are not written
        err = np.linalg.norm(Xn - X_ref) / np.linalg.norm(X_ref)
        assert err <= TOL, (counter, err)
    h.close()


def test_noalloc_rejects_sizes_beyond_the_scratch():
    import torch
    frsvt, fn = _noalloc_fn()
    A = torch.zeros((16, 8), device="cuda")
    X = torch.zeros_like(A)
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    assert fn(p(A), 70000, 8, 8, 1.0, 4, 1, 0, 0, p(X), 8, None) == 1      # m above the limit
    assert fn(p(A), 400, 300, 300, 1.0, 4, 1, 0, 0, p(X), 300, None) == 1  # n above the limit
    assert fn(p(A), 16, 8, 8, 1.0, 17, 1, 0, 0, p(X), 8, None) == 1        # l above 16
    assert fn(p(A), 16, 8, 8, float("inf"), 4, 1, 0, 0, p(X), 8, None) == 1  # tau not finite
    assert fn(p(A), 16, 8, 8, 1.0, 4, 1, 0, 2 ** 64 - 1, p(X), 8, None) == 1  # reserved stream index
    assert fn(p(A), 8, 16, 16, 1.0, 4, 1, 0, 0, p(X), 16, None) == 2       # wide: unsupported
