"""frsvt_svt_factors: the FRSVT in factored form X = U V^T (U = A Q, V = Q M), against the FP64
oracle's X and r, on the narrow tensor-core path, the CUDA-core path and the wide basis."""
import numpy as np
import pytest

from gpu_util import rel_fro, spectrum_matrix, to_gpu
from oracle import svt as osvt

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module")
def fr():
    import torch
    assert torch.cuda.is_available()
    from paper_1509_00296_gb300 import build, frsvt
    build.build()
    return frsvt


@pytest.mark.parametrize("m,n,l,q", [(3000, 120, 12, 2), (1500, 300, 16, 1), (2048, 700, 60, 2), (777, 333, 37, 0)])
def test_factors_reconstruct_the_oracle_svt(fr, m, n, l, q):
    A, s = spectrum_matrix(m, n, min(n, 3 * l), 0.93, 0.01, seed=m + n)
    A = A.astype(np.float32).astype(np.float64)
    tau = float(0.5 * (s[l // 2] + s[l // 2 + 1]))
    ref = osvt.frsvt(A, tau, l, q, seed=19, stream=0)
    h = fr.Handle(m, n, l, q=q, range_prop=False, seed=19)
    U, V, r = h.svt_factors(to_gpu(A), tau, l)
    X = (U.double() @ V.double().T).cpu().numpy()
    assert rel_fro(X, ref.X) <= TOL
    assert int(r.item()) == ref.r
    info = h.info()
    assert info.device_status == 0 and info.s == min(l, n)
    # the same handle's frsvt_svt on the next Omega stream agrees with the factors of that stream
    X2 = h.svt(to_gpu(A), tau, l, X=to_gpu(np.zeros_like(A))).cpu().numpy()
    ref2 = osvt.frsvt(A, tau, l, q, seed=19, stream=1)
    assert rel_fro(X2, ref2.X) <= TOL
    h.close()


def test_factors_reject_short_leading_dimensions(fr):
    import ctypes
    import torch
    h = fr.Handle(100, 40, 8, q=1, range_prop=False)
    A = torch.randn(100, 40, device="cuda")
    U = torch.empty(100, 8, device="cuda")
    V = torch.empty(40, 8, device="cuda")
    st = fr.lib().frsvt_svt_factors(h._h, ctypes.c_void_p(A.data_ptr()), 100, 40, 40, 0.5, 8,
                                    ctypes.c_void_p(U.data_ptr()), 4, ctypes.c_void_p(V.data_ptr()), 8, None)
    assert st == 1                                   # ldu < l: FRSVT_ERR_INVALID_ARG
    h.close()
