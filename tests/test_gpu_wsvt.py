"""Batched weighted SVT (WNNM patch groups) on the GPU against the FP64 oracle."""
import numpy as np
import pytest

from oracle import svt
from paper_1509_00296_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

C, EPS = 2.8, 1e-8


def _fr():
    from paper_1509_00296_gb300 import frsvt as fr
    return fr


def _rel(X, R):
    return np.linalg.norm(X - R) / max(np.linalg.norm(R), 1e-30)


def _mixed_batch(seed=7):
    """Patch groups of the WNNM shape with n_b below, at and above m = 64, edges 40 / 160."""
    mats, _ = synth.wnnm_batch(seed=seed, batch=24)
    rng = np.random.default_rng(seed)
    for n in (40, 63, 64, 65, 160, 41):
        A = rng.standard_normal((64, 4)) @ rng.standard_normal((4, n)) + 0.05 * rng.standard_normal((64, n))
        mats.append(A.astype(np.float32))
    return mats


@pytest.fixture(scope="module")
def handle():
    fr = _fr()
    return fr.Handle(64, 160, 16, q=1, seed=11)


@pytest.mark.parametrize("variant", ["exact", "frsvt"])
def test_wsvt_matches_oracle(handle, variant):
    fr = _fr()
    mats = _mixed_batch()
    dm = [torch.from_numpy(A).cuda() for A in mats]
    v = fr.WSVT_EXACT if variant == "exact" else fr.WSVT_FRSVT
    out = handle.wsvt(dm, C, EPS, variant=v, l=12)
    torch.cuda.synchronize()
    assert handle.info().device_status & fr.DEV_BAD_PROBLEM == 0
    ref = svt.wsvt_batch([A.astype(np.float64) for A in mats], C, EPS, variant, l=12, q=1, seed=11, stream=0)
    errs = [_rel(o.cpu().numpy().astype(np.float64), r) for o, r in zip(out, ref)]
    assert max(errs) < 1e-4, (variant, max(errs), int(np.argmax(errs)))
    # the weights remove the noise directions but keep the rank-4 signal
    assert all(0 < np.linalg.norm(r) < np.linalg.norm(A) for r, A in zip(ref, mats))


def test_wsvt_full_batch_sampled(handle):
    """16384 problems of 64 x n_i, n_i in [40, 160], one launch per variant; sampled vs the oracle."""
    fr = _fr()
    mats, ns = synth.wnnm_batch(seed=1004)
    dm = [torch.from_numpy(A).cuda() for A in mats]
    rng = np.random.default_rng(5)
    picks = rng.choice(len(mats), size=12, replace=False)
    for variant, v in (("exact", fr.WSVT_EXACT), ("frsvt", fr.WSVT_FRSVT)):
        out = handle.wsvt(dm, C, EPS, variant=v, l=12)
        torch.cuda.synchronize()
        assert handle.info().device_status & fr.DEV_BAD_PROBLEM == 0
        for b in picks:
            A = mats[b].astype(np.float64)
            w = svt.wnnm_weights(A.shape[1], C, EPS)
            R = svt.wsvt(A, w) if variant == "exact" else svt.frsvt(A, 0.0, 12, 1, 11, 0, problem=int(b),
                                                                    weights=w).X
            assert _rel(out[b].cpu().numpy().astype(np.float64), R) < 1e-4, (variant, b)


def test_wsvt_edge_weights(handle):
    fr = _fr()
    mats = _mixed_batch(seed=9)[:6]
    dm = [torch.from_numpy(A).cuda() for A in mats]
    # c = 0: no shrinkage, X = A
    out = handle.wsvt(dm, 0.0, EPS, variant=fr.WSVT_EXACT)
    for o, A in zip(out, mats):
        assert _rel(o.cpu().numpy(), A) < 1e-4
    # weights above every singular value: X = 0
    out = handle.wsvt(dm, 1e6, EPS, variant=fr.WSVT_FRSVT, l=12)
    for o in out:
        assert float(o.abs().max()) == 0.0


def test_wsvt_bad_problem_is_flagged(handle):
    fr = _fr()
    handle.info()                                      # clear the sticky status
    A = torch.randn(64, 100, device="cuda")
    n = torch.tensor([100, 200], dtype=torch.int32, device="cuda")   # 200 > n_max = 160
    X = [torch.full_like(A, 7.0), torch.full_like(A, 7.0)]
    a = torch.tensor([A.data_ptr(), A.data_ptr()], dtype=torch.int64, device="cuda")
    x = torch.tensor([t.data_ptr() for t in X], dtype=torch.int64, device="cuda")
    handle.wsvt_raw(a, n, 64, C, EPS, x, fr.WSVT_EXACT)
    torch.cuda.synchronize()
    assert handle.info().device_status & fr.DEV_BAD_PROBLEM
    assert float(X[1].min()) == 7.0 and float(X[1].max()) == 7.0     # skipped, untouched
    assert float(X[0].max()) != 7.0


def test_wsvt_invalid_args(handle):
    fr = _fr()
    A = torch.randn(64, 50, device="cuda")
    with pytest.raises(fr.FrsvtError):
        handle.wsvt([A], C, 0.0)                          # eps must be > 0
    with pytest.raises(fr.FrsvtError):
        handle.wsvt([torch.randn(65, 50, device="cuda")], C, EPS)   # m > 64
    assert handle.wsvt([], C, EPS) == []


def test_wsvt_graph_capture_and_tuner(handle):
    fr = _fr()
    mats = _mixed_batch(seed=3)
    dm = [torch.from_numpy(A).cuda() for A in mats]
    out = [torch.empty_like(t) for t in dm]
    a = torch.tensor([t.data_ptr() for t in dm], dtype=torch.int64, device="cuda")
    x = torch.tensor([t.data_ptr() for t in out], dtype=torch.int64, device="cuda")
    n = torch.tensor([t.shape[1] for t in dm], dtype=torch.int32, device="cuda")
    for v in (fr.WSVT_EXACT, fr.WSVT_FRSVT):
        handle.wsvt_raw(a, n, 64, C, EPS, x, v, 12, tune=True)
        nt, cps = handle.wsvt_tuning(v)
        assert nt in (128, 256, 512) and cps >= 1
        handle.wsvt_raw(a, n, 64, C, EPS, x, v, 12)
        torch.cuda.synchronize()
        eager = [t.clone() for t in out]
        for t in out:
            t.zero_()
        s = torch.cuda.Stream()
        handle.set_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            handle.wsvt_raw(a, n, 64, C, EPS, x, v, 12)
        g.replay()
        torch.cuda.synchronize()
        handle.set_stream(None)
        for e, t in zip(eager, out):
            assert torch.equal(e, t)
