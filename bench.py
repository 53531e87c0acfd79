#!/usr/bin/env python
"""Benchmark: inexact-ALM RPCA iterations per second with FRSVT on one GB300.

Workload (one "step" = one full iALM iteration of the hot path): the large
low-rank recovery input, O = 8192 x 8192 float32, rank 100 (Gaussian factors
scaled 1/sqrt(100)) plus 10 % additive corruption uniform in [-10, 10]; inexact
ALM with FRSVT at l = 120, q = 2 (the wide-basis path: FP32-accurate 3xTF32
passes on tcgen05, double-float Gram and Cholesky, l x l core), lambda =
1/sqrt(8192), rho = 1.5.  Data is synthetic (seeded), see synth.recovery_8192.

Default arm (--impl frsvt): the C-ABI library; each step is one iALM iteration
replayed from a captured CUDA graph.  Timing: CUDA events around each step on
the launching stream, the L2 cache flushed (a 256 MiB write) between steps
outside the events.  `value` = steps / summed device time, max over ranks.
Also reported: per-phase device times through the library's tracing hook (the
roofline of the dominant kernel), one exact SVT of the same iterate by cuSOLVER
on the same GPU, the end-to-end rate through the public API with host buffers,
the FP64 oracle on the host cores, SM clocks sampled by nvidia-smi during the
timed region, the BF16 / FP8 variants of the same workload, and the other
workloads (video-background RPCA, batched weighted SVT, unrolled RPCA, Type B
weather windows) as extra keys.

--impl reference times the FP64 CPU oracle (numpy) on the same workload.
Under torchrun each rank runs an independent replica (the path does not shard).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ALM iters/s & tensor-pipe % of FRSVT vs exact-SVD SVT, same GPU, ≤1e-4 rel err"
UNIT = "ALM iters/s"
RN, RL, RQ = 8192, 120, 2                 # recovery: n x n, l, q
RDATA_SEED, ROMEGA_SEED = 1003, 2004
RWORKLOAD = ("large low-rank recovery 8192x8192 rank 100 + 10% corruption in [-10,10], "
             "iALM with FRSVT l=120 q=2 (FP32-accurate passes)")
M, N, L_COLS, Q_POW = 76800, 200, 10, 2   # video-background extra
LP_COLS = 16                              # l rounded up to the 16-column panel
DATA_SEED, OMEGA_SEED = 1002, 2002
WORKLOAD = "video-background RPCA 76800x200 (320x240 px x 200 frames), FRSVT l=10 q=2 range propagation"

# Kernels that serve each phase of the wide-basis FP32 path: one kernel, except the sketch (Omega
# generation, a few percent of it) and the small dense tails (the Gram of a basis-side matrix on all
# SMs, then the Cholesky QR operand on one SM or the core on an 8-CTA cluster).
WIDE_PHASE_KERNEL = {"sketch": "k_wd_omega + k_wd_pass<1,0>", "power_AQ": "k_wd_pass<0,0>", "power_AtZ": "k_wd_pass<1,0>",
                     "project": "k_wd_pass<0,0>", "orth": "k_wd_gram + k_wd_orth", "apply": "k_wd_trsm / k_wd_apply",
                     "core": "k_wd_gram + k_wd_core", "epilogue": "k_wd_alm<true>"}
# ncu counters of the wide-basis kernels on this workload, per launch (NCU_PROFILE records the capture command
# and these figures; tests/test_bench_host.py checks that they match; None where no capture of the current
# kernel exists).  traffic:
# dram__bytes_read.sum + dram__bytes_write.sum; tensor_pct: sm__pipe_tensor_cycles_active (percent of elapsed).
NCU_PROFILE = "profiles/wide_passes_recovery_8192x8192.md"
NCU_WIDE = {"k_wd_pass<1,0>": {"traffic": 286.4e6, "tensor_pct": 55.2},
            "k_wd_pass<0,0>": {"traffic": 291.4e6, "tensor_pct": 57.4},
            "k_wd_alm<true>": {"traffic": 1328.4e6, "tensor_pct": None}}


def config_dict(ws: int):
    """The workload description printed by both arms."""
    return {"workload": RWORKLOAD, "m": RN, "n": RN, "l": RL, "q": RQ, "range_prop": False,
            "precision": "fp32 data, 3xTF32 tcgen05 passes, double-float Gram / Cholesky",
            "l2": "inputs (3 x 268 MB) exceed L2; L2 also flushed between steps (256 MiB write, outside the events)",
            "timing": "sum of per-step CUDA-event durations on the launching stream",
            "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max_ms(dev_ms: float, device) -> float:
    """Largest timed-region duration (ms) over the ranks of the process group (the local value on
    one rank): replicas are timed together, the slowest one counts."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([dev_ms], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(steps: int, ws: int, max_ms: float) -> float:
    """Whole-job throughput: every rank runs `steps` iterations of its own replica within max_ms."""
    return ws * steps / (max_ms / 1e3)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def host_norm2(O, iters: int = 30, seed: int = 0) -> float:
    """||O||_2 by the power method on the host (FP64), for the oracle's initialisation."""
    import numpy as np
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(O.shape[1])
    s = 0.0
    for _ in range(iters):
        u = O @ v
        v = O.T @ u
        s = float(np.linalg.norm(v))
        v /= s
    return float(np.sqrt(s))


def oracle_cores() -> int:
    try:
        import threadpoolctl
        return max(i.get("num_threads", 1) for i in threadpoolctl.threadpool_info()) or os.cpu_count()
    except Exception:
        return int(os.environ.get("OPENBLAS_NUM_THREADS", os.cpu_count() or 1))


def oracle_rate(O64, normO2: float, iters: int, **kw):
    """FP64 oracle iALM-FRSVT iterations per second on a bounded sample (host cores); the
    initialisation (||O||_2, given) is outside the timing."""
    from oracle import rpca as orpca
    args = dict(l=RL, q=RQ, seed=ROMEGA_SEED, range_prop=False)
    args.update(kw)
    t0 = time.perf_counter()
    orpca.ialm_rpca(O64, method="frsvt", fixed_iters=iters, normO2=normO2, **args)
    dt = time.perf_counter() - t0
    return iters / dt, oracle_cores(), dt


def recovery_input():
    import numpy as np
    from paper_1509_00296_gb300 import synth
    O, _, _ = synth.recovery_8192(seed=RDATA_SEED)
    return np.ascontiguousarray(O, dtype=np.float32)


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np
    O64 = recovery_input().astype(np.float64)
    nrm = host_norm2(O64)
    # the oracle keeps no state between runs, so the warm-up steps have nothing to warm: each timed
    # step is one iALM-FRSVT iteration of the full workload
    rate, cores, dt = oracle_rate(O64, nrm, max(1, args.steps))
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / rate, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(ws),
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} iALM-FRSVT iterations of the full 8192x8192 workload "
                                       f"({dt:.1f} s), FP64 numpy oracle"},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="frsvt", choices=["frsvt", "reference"])
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--oracle-iters", type=int, default=2)
    ap.add_argument("--skip-extras", action="store_true", help="only the main timed region")
    ap.add_argument("--profile-svt", choices=["fp32", "bf16", "fp8"], default=None,
                    help="only three FRSVT calls on the 8192 x 8192 recovery matrix (l = 120, q = 2), for ncu")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_svt:
        return profile_svt(args.profile_svt)

    import numpy as np
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_1509_00296_gb300 import build, frsvt
    build.build()

    O_np = recovery_input()
    lam = 1.0 / np.sqrt(RN)
    O = torch.from_numpy(O_np).to(dev)
    S = torch.empty_like(O)
    A = torch.empty_like(O)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    h = frsvt.Handle(RN, RN, RL, q=RQ, range_prop=False, seed=ROMEGA_SEED, stream=stream)
    h.rpca_init(O, S, A, lam, 1.5, 1e7)

    # one eager step first, its launches counted through the tracing hook
    h.enable_timing(True)
    h.timings()
    h.ialm_step(O, S, A, RL)
    groups_per_step = sum(v[1] for v in h.timings().values())
    h.enable_timing(False)
    h.ialm_step(O, S, A, RL)                     # captured by the library: its kernel nodes are counted
    kernels_per_step = h.step_kernels()
    if kernels_per_step <= 0:
        raise RuntimeError("the library did not capture the iALM step; kernel count unknown")
    graph = None
    if not args.no_graph:
        cap = torch.cuda.Stream()
        h.set_stream(cap)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=cap):
            h.ialm_step(O, S, A, RL)
        h.set_stream(stream)

    def step():
        if graph is not None:
            graph.replay()
        else:
            h.ialm_step(O, S, A, RL)

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(float(k))
            evs[k][0].record(stream)
            step()
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall0
    if ws > 1:
        torch.distributed.barrier()
    dev_ms = reduce_max_ms(sum(a.elapsed_time(b) for a, b in evs), dev)
    ms_per_step = dev_ms / args.steps
    value = aggregate_rate(args.steps, ws, dev_ms)
    clocks = clk.summary()
    info = h.info()

    extras = {}
    if not args.skip_extras and rank == 0:
        extras = run_extras(args, h, O, S, A, O_np, lam, dev, stream, flush)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(config_dict(ws), graph=graph is not None),
            "gpu_launches": kernels_per_step * args.steps,
            "clocks": clocks,
            "wall_s_timed_region": t_wall,
            "alm_state": {"iter": info.alm_iter, "residual": info.residual, "rank": info.r, "basis": info.s,
                          "jacobi_sweeps": info.sweeps, "device_status": info.device_status},
        }
        line.update(extras)
        if "exact_svd_same_gpu" in line:
            line["exact_svd_same_gpu"]["frsvt_speedup"] = value / line["exact_svd_same_gpu"]["value"]
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def profile_svt(prec: str):
    """Three frsvt_svt calls on the large low-rank recovery matrix: a fixed, short launch sequence
    for ncu captures (per call: six passes, each followed by its partial sum)."""
    import numpy as np
    import torch
    from paper_1509_00296_gb300 import build, frsvt, synth
    build.build()
    torch.cuda.set_device(0)
    n = 8192
    O_np, _, _ = synth.recovery_8192(seed=1003)
    A = torch.from_numpy(np.ascontiguousarray(O_np, dtype=np.float32)).cuda()
    X = torch.empty_like(A)
    h = frsvt.Handle(n, n, 120, q=2, range_prop=False, seed=5,
                     precision={"fp32": frsvt.PREC_FP32, "bf16": frsvt.PREC_BF16, "fp8": frsvt.PREC_FP8}[prec])
    for _ in range(3):
        h.svt(A, 300.0, 120, X=X)
    torch.cuda.synchronize()
    info = h.info()
    print(json.dumps({"profile_svt": prec, "r": info.r, "s": info.s, "sweeps": info.sweeps,
                      "device_status": info.device_status}))
    return 0


def fp32_alu_peak_tflops() -> float:
    """FP32 FMA rate of the whole chip from its unit counts and clock: 152 SMs x 128 lanes x 2 FLOP
    x the measured maximum SM clock (MEASURED_PEAKS.json, else 2070 MHz)."""
    mhz = 2070.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    except Exception:
        pass
    return 152 * 128 * 2 * mhz * 1e6 / 1e12


def fp32_issue_peak_tops() -> float:
    """FP32 lane-instruction issue peak of the GPU: 152 SMs x 128 FP32 lanes x max SM clock."""
    return fp32_alu_peak_tflops() / 2.0


def wide_roofline(tm, K, n, sweeps):
    """Rooflines of the wide-basis iALM step's kernel groups from the tracing hook's per-phase
    times (CUDA events on the launching stream), and the dominant one.  HBM-bound groups:
    algorithmic bytes per launch over the average launch time (a pass's launch group is the pass
    and its partial sum, k_wd_psum; the ncu traffic is the pass kernel's).  The small dense tails (Gram,
    Cholesky, Jacobi): FP32-pipe lane instructions per launch over time, against the GPU's FP32
    issue peak (a df64 product-accumulate is 9 FP32 instructions; a Jacobi pair rotation on
    128-long columns ~1000)."""
    peak, peak_kind = peaks()
    e = 4.0 * n * n                      # one float32 pass over A
    z = 4.0 * 128 * n                    # one 128-wide basis-side matrix
    kern = {}
    for ph, (ms, cnt) in tm.items():
        if cnt > 0 and ph in WIDE_PHASE_KERNEL:
            k = WIDE_PHASE_KERNEL[ph]
            t = kern.setdefault(k, [0.0, 0])
            t[0] += ms / K
            t[1] += cnt / K
    hbm_bytes = {"k_wd_pass<1,0>": e + 3 * z, "k_wd_pass<0,0>": e + 4 * z, "k_wd_alm<true>": 5 * e + 4 * z,
                 "k_wd_omega + k_wd_pass<1,0>": e + 5 * z,
                 "k_wd_trsm / k_wd_apply": 3 * z}
    gram_ops = 9.0 * n * 128 * 129 / 2
    chol_ops = 4.5e6
    alu_ops = {"k_wd_gram + k_wd_orth": gram_ops + chol_ops,
               "k_wd_gram + k_wd_core": gram_ops + chol_ops + sweeps * (128 * 127 / 2) * 1000.0}
    pk = fp32_issue_peak_tops()
    all_roofs = {}
    # the sketch phase is two launch groups (Omega^T, then the pass with its sum): one unit of work
    units_per_group = {"k_wd_omega + k_wd_pass<1,0>": 0.5}
    for k, (ms, cnt) in kern.items():
        per_launch_ms = ms / (cnt * units_per_group.get(k, 1.0))
        ncu = NCU_WIDE.get(k, {})
        if k in hbm_bytes:
            ach = hbm_bytes[k] / (per_launch_ms / 1e3) / 1e9
            r = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                 "traffic": ncu.get("traffic"), "algorithmic_bytes_per_launch": hbm_bytes[k],
                 "peak_kind": f"{peak_kind} (STREAM-style copy)"}
        elif k in alu_ops:
            ach = alu_ops[k] / (per_launch_ms / 1e3) / 1e12
            r = {"bound": "alu", "achieved": ach, "peak": pk, "unit": "T FP32 lane-instructions/s", "frac": ach / pk,
                 "traffic": None, "algorithmic_ops_per_launch": alu_ops[k],
                 "peak_kind": "derived: 152 SMs x 128 FP32 lanes x max SM clock (issue rate)"}
        else:
            continue
        r.update({"kernel": k, "avg_launch_ms": per_launch_ms, "launch_groups_per_step": cnt})
        all_roofs[k] = r
    dom = max(all_roofs, key=lambda k: kern[k][0])
    roof = dict(all_roofs[dom])
    roof["kernel_ms_per_step"] = {k: v[0] for k, v in kern.items()}
    roof["other_kernels"] = {k: {"bound": v["bound"], "frac": v["frac"], "achieved": v["achieved"], "unit": v["unit"]}
                             for k, v in all_roofs.items() if k != dom}
    return roof


def run_extras(args, h, O, S, A, O_np, lam, dev, stream, flush):
    import numpy as np
    import torch

    out = {}
    # ---- per-phase device times (tracing hook), same step, eager launches on the same stream
    K = max(5, min(args.steps, 20))
    h.enable_timing(True)
    h.timings()
    for k in range(K):
        flush.fill_(float(k))
        h.ialm_step(O, S, A, RL)
    tm = h.timings()
    h.enable_timing(False)
    out["phases_ms_per_step"] = {k: v[0] / K for k, v in tm.items() if v[1] > 0}
    out["roofline"] = wide_roofline(tm, K, RN, h.info().sweeps)
    out["tensor_pipe_pct"] = {k: v["tensor_pct"] for k, v in NCU_WIDE.items() if v.get("tensor_pct") is not None}
    out["tensor_pipe_pct"]["source"] = f"ncu capture of the passes on this workload, {NCU_PROFILE}"

    # ---- exact-SVD iALM on the same GPU: one iteration on the current iterate (cuSOLVER through
    # torch.linalg.svd, then the same shrinkage, reconstruction and multiplier update)
    info = h.info()
    mu = info.mu
    torch.linalg.svd(A[:1024, :1024], full_matrices=False, driver="gesvd")   # set-up outside the timing
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    U, sv, Vh = torch.linalg.svd(A, full_matrices=False, driver="gesvd")
    Le = (U * torch.clamp(sv - 1.0 / mu, min=0.0)) @ Vh
    T = A + S - Le
    Se = torch.sign(T) * torch.clamp(T.abs() - lam / mu, min=0.0)
    Ae = O - Se + (T - Se) / 1.5
    e1.record()
    torch.cuda.synchronize()
    ex_ms = e0.elapsed_time(e1)
    del U, sv, Vh, Le, T, Se, Ae
    torch.cuda.empty_cache()
    out["exact_svd_same_gpu"] = {
        "value": 1e3 / ex_ms, "unit": UNIT, "ms_per_step": ex_ms,
        "method": "one iALM iteration with exact SVT by torch.linalg.svd (cuSOLVER gesvd), float32, same GPU",
        "frsvt_speedup": None}

    # ---- end to end through the public API with host buffers: rpca_init from pinned host O, K2
    # iterations with the residual read back every step, S and L copied back; run twice, the
    # second is timed (the first captures the iteration graphs for these buffers)
    O_host = torch.from_numpy(O_np).pin_memory()
    S_host = torch.empty_like(O_host).pin_memory()
    L_host = torch.empty_like(O_host).pin_memory()
    K2 = max(5, min(args.steps, 20))
    Od, Sd, Ad, Ld = (torch.empty_like(O) for _ in range(4))

    def e2e_run():
        Od.copy_(O_host, non_blocking=True)
        h.rpca_init(Od, Sd, Ad, lam, 1.5, 1e7)
        for k in range(K2):
            h.ialm_step(Od, Sd, Ad, RL, L=Ld if k == K2 - 1 else None, sync_residual=True)
        S_host.copy_(Sd, non_blocking=True)
        L_host.copy_(Ld, non_blocking=True)
        torch.cuda.synchronize()

    e2e_run()
    w0 = time.perf_counter()
    e2e_run()
    w = time.perf_counter() - w0
    nbytes = 4 * RN * RN
    out["e2e"] = {"value": K2 / w, "unit": UNIT, "h2d_bytes_per_step": nbytes / K2,
                  "d2h_bytes_per_step": (8 * K2 + 2 * nbytes) / K2,
                  "what": f"rpca_init (spectral norm by 30 power steps) + {K2} rpca_ialm_step calls from pinned "
                          f"host O, residual read back every step, S and L copied back at the end; wall clock"}
    del Od, Sd, Ad, Ld, O_host, S_host, L_host

    # ---- FP64 oracle on the host cores (bounded sample)
    O64 = O_np.astype(np.float64)
    rate, cores, dt = oracle_rate(O64, host_norm2(O64), args.oracle_iters)
    del O64
    out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                           "sample": f"{args.oracle_iters} iALM-FRSVT iterations of the full 8192x8192 workload "
                                     f"({dt:.1f} s), FP64 numpy oracle"}
    out["recovery_8192_variants"] = bench_recovery(args, O, lam, dev, flush)
    out["video"] = bench_video(args, dev, flush)
    out["wsvt_batch"] = bench_wsvt(dev)
    out["unrolled_rpca"] = bench_unrolled(dev)
    out["weather_type_b"] = bench_weather()
    out["lrr_type_a"] = bench_lrr()
    return out


def bench_video(args, dev, flush):
    """The video-background workload (76800 x 200, l = 10, q = 2, range propagation; the narrow
    tensor-core path): graph-replayed iterations per second, per-phase times and the roofline of
    its dominant phase, exact-SVD iALM on the same GPU, and its BF16 / rank-prediction /
    orthonormalise-last variants."""
    import numpy as np
    import torch
    from paper_1509_00296_gb300 import frsvt, synth
    O_np, _, _ = synth.video(seed=DATA_SEED)
    lam = 1.0 / np.sqrt(max(M, N))
    O = torch.from_numpy(O_np).to(dev)
    S = torch.empty_like(O)
    A = torch.empty_like(O)
    h = frsvt.Handle(M, N, L_COLS, q=Q_POW, range_prop=True, seed=OMEGA_SEED, stream=torch.cuda.current_stream())
    h.rpca_init(O, S, A, lam, 1.5, 1e7)
    h.ialm_step(O, S, A, L_COLS)
    steps = max(10, min(args.steps, 50))
    ms = graph_rate(h, O, S, A, L_COLS, steps, flush)
    out = {"workload": WORKLOAD, "ms_per_step": ms, "value": 1e3 / ms, "unit": UNIT}
    K = 10
    h.enable_timing(True)
    h.timings()
    for k in range(K):
        flush.fill_(float(k))
        h.ialm_step(O, S, A, L_COLS)
    tm = h.timings()
    h.enable_timing(False)
    out["phases_ms_per_step"] = {k: v[0] / K for k, v in tm.items() if v[1] > 0}
    e = 4.0 * M * N
    z = 4.0 * M * LP_COLS
    alg_bytes = {"epilogue": 5 * e + z, "sketch": e, "power_AQ": e + z, "power_AtZ": e + z, "project": e + z,
                 "core": z}
    dom = max((k for k in alg_bytes if tm.get(k, (0, 0))[1] > 0), key=lambda k: tm[k][0])
    avg_ms = tm[dom][0] / tm[dom][1]
    peak, _ = peaks()
    ach = alg_bytes[dom] / (avg_ms / 1e3) / 1e9
    out["roofline"] = {"bound": "hbm", "phase": dom, "achieved": ach, "peak": peak, "unit": "GB/s",
                       "frac": ach / peak, "algorithmic_bytes_per_launch": alg_bytes[dom], "avg_launch_ms": avg_ms}
    # exact-SVD iALM on the same GPU, both cuSOLVER drivers (gesvd, gesvdj); the faster one counts
    normO2 = torch.linalg.matrix_norm(O, 2).item()
    per_driver = {}
    for drv in ("gesvd", "gesvdj"):
        Oe = O.clone()
        Se = torch.zeros_like(Oe)
        Ye = Oe / max(normO2, Oe.abs().max().item() / lam)
        mu = 1.25 / normO2
        torch.linalg.svd(Oe - Se + Ye / mu, full_matrices=False, driver=drv)   # set-up outside the timing
        torch.cuda.synchronize()
        ex_it = 3
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(ex_it):
            U, sv, Vh = torch.linalg.svd(Oe - Se + Ye / mu, full_matrices=False, driver=drv)
            Le = (U * torch.clamp(sv - 1.0 / mu, min=0.0)) @ Vh
            T = Oe - Le + Ye / mu
            Se = torch.sign(T) * torch.clamp(T.abs() - lam / mu, min=0.0)
            Ye = Ye + mu * (Oe - Le - Se)
            mu = min(1.5 * mu, 1e7 * 1.25 / normO2)
        t1.record()
        torch.cuda.synchronize()
        per_driver[drv] = t0.elapsed_time(t1) / ex_it
    best = min(per_driver, key=per_driver.get)
    out["exact_svd_same_gpu"] = {"ms_per_step": per_driver[best], "driver": best, "ms_by_driver": per_driver,
                                 "frsvt_speedup": per_driver[best] / ms}
    h.close()
    out["bf16"] = bench_video_bf16(args, O, O_np, lam, dev, flush)
    out["rank_prediction"] = bench_video_ap(args, O, lam, flush)
    out["orth_last"] = bench_video_orth_last(args, O, lam, flush)
    return out


def graph_rate(h, O, S, A, l, steps, flush):
    """Capture one iALM iteration in a CUDA graph and time `steps` replays (device time, L2 flushed
    between replays outside the events); returns ms per iteration."""
    return statistics.fmean(graph_replay_ms(h, O, S, A, l, steps, flush))


def graph_replay_ms(h, O, S, A, l, steps, flush):
    """The device time (ms) of each of `steps` replays of one captured iALM iteration."""
    import torch
    cap = torch.cuda.Stream()
    st = torch.cuda.current_stream()
    h.set_stream(cap)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=cap):
        h.ialm_step(O, S, A, l)
    h.set_stream(st)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.fill_(float(k))
        evs[k][0].record()
        g.replay()
        evs[k][1].record()
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def bench_video_bf16(args, O, O_np, lam, dev, flush):
    """The video workload with the BF16 passes (sketch and first q - 1 power steps on a BF16 shadow
    of A, FP32-accurate last power step and projection)."""
    import torch
    from paper_1509_00296_gb300 import frsvt
    S = torch.empty_like(O)
    A = torch.empty_like(O)
    h = frsvt.Handle(M, N, L_COLS, q=Q_POW, range_prop=True, seed=OMEGA_SEED, stream=torch.cuda.current_stream(),
                     precision=frsvt.PREC_BF16)
    h.rpca_init(O, S, A, lam, 1.5, 1e7)
    h.ialm_step(O, S, A, L_COLS)
    ms = graph_rate(h, O, S, A, L_COLS, max(10, min(args.steps, 50)), flush)
    h.close()
    return {"precision": "bf16 sketch + first q-1 power steps, FP32-accurate last power step and projection",
            "ms_per_step": ms, "value": 1e3 / ms, "unit": UNIT}


def bench_video_orth_last(args, O, lam, flush):
    """The video workload orthonormalising only after the last power step (Sec. 2.5,
    FRSVT_CFG_ORTH_LAST): the intermediate power step hands A^T Z on without its Cholesky QR tail.
    Reported with the relative difference of L and S from the default path after 20 iterations."""
    import torch
    from paper_1509_00296_gb300 import frsvt
    res = {}
    for orth_last in (False, True):
        S = torch.empty_like(O)
        A = torch.empty_like(O)
        Lm = torch.empty_like(O)
        h = frsvt.Handle(M, N, L_COLS, q=Q_POW, range_prop=True, seed=OMEGA_SEED,
                         stream=torch.cuda.current_stream(), orth_last=orth_last)
        h.rpca_init(O, S, A, lam, 1.5, 1e7)
        for k in range(20):
            h.ialm_step(O, S, A, L_COLS, L=Lm if k == 19 else None)
        torch.cuda.synchronize()
        res[orth_last] = (Lm.clone(), S.clone())
        if orth_last:
            ms = graph_rate(h, O, S, A, L_COLS, max(10, min(args.steps, 50)), flush)
        h.close()
    dl = float(torch.linalg.norm(res[True][0] - res[False][0]) / torch.linalg.norm(res[False][0]))
    ds = float(torch.linalg.norm(res[True][1] - res[False][1]) / torch.linalg.norm(res[False][1]))
    return {"variant": "orthonormalise only after the last power step (Sec. 2.5)", "ms_per_step": ms,
            "value": 1e3 / ms, "unit": UNIT, "rel_diff_L_vs_default_20_iters": dl,
            "rel_diff_S_vs_default_20_iters": ds}


def bench_video_ap(args, O, lam, flush):
    """The video workload with the adaptive rank prediction of Eq. 7 (a = 2, rho = 0.05,
    gamma = 0.08: b = 16): the sampling rate is chosen on the device each iteration, so the
    captured iteration replays without host involvement."""
    import torch
    from paper_1509_00296_gb300 import frsvt
    S = torch.empty_like(O)
    A = torch.empty_like(O)
    h = frsvt.Handle(M, N, 16, q=Q_POW, range_prop=True, seed=OMEGA_SEED, stream=torch.cuda.current_stream())
    h.set_rank_prediction(2, 0.05, 0.08)
    h.rpca_init(O, S, A, lam, 1.5, 1e7)
    ls = [h.rank_prediction()]
    for _ in range(8):
        h.ialm_step(O, S, A, L_COLS)
        ls.append(h.rank_prediction())
    ms = graph_rate(h, O, S, A, L_COLS, max(10, min(args.steps, 50)), flush)
    info = h.info()
    h.close()
    return {"rule": "l' = min(r + (r < l ? 2 : ceil(0.05 n)), b), b = ceil(0.08 n) = 16, l_0 = 2",
            "sampling_rates_first_iterations": ls, "rank": info.r, "ms_per_step": ms, "value": 1e3 / ms,
            "unit": UNIT}


def bench_lrr():
    """Low-rank representation (Table 6, Type A) on a face-sized union of subspaces (the paper's
    Yale B setting, 2016 x 640: 10 classes of 64 samples; here 9-dimensional subspaces, 10 % of
    the columns corrupted): the GPU iALM (FRSVT J step l = 128 with range propagation, q = 1;
    Newton-Schulz (I + Z^T Z)^{-1} formed once) timed over 30 iterations from the reading's
    defaults mu0 = 1e-6, rho = 1.1 (CUDA events on the stream, no synchronisation inside)."""
    import numpy as np
    import torch
    from paper_1509_00296_gb300 import frsvt, synth
    O, _, _, _ = synth.subspaces(seed=1012, d=2016, k=10, dim=9, per=64, frac=0.1)
    Og = torch.from_numpy(np.ascontiguousarray(O, dtype=np.float32)).cuda()
    d, n = O.shape
    h = frsvt.LRR(d, n, 128, q=1, seed=5, range_prop=True, stream=torch.cuda.current_stream())
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    h.init(Og, 0.3, mu0=1e-6, rho=1.1)
    t1.record()
    torch.cuda.synchronize()
    init_ms = t0.elapsed_time(t1)
    for _ in range(3):
        h.step()
    K = 30
    t0.record()
    for _ in range(K):
        h.step()
    t1.record()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / K
    err = h.step(sync_err=True)
    h.close()
    return {"workload": f"LRR {d} x {n} (10 subspaces of dim 9, 64 samples each, 10 % corrupted columns), "
                        "lam 0.3, FRSVT l = 128 q = 1 with range propagation",
            "ms_per_iteration": ms, "value": 1e3 / ms, "unit": "iALM iterations/s", "init_ms": init_ms,
            "stop_quantity_after_34": err,
            "paper_context": "44.59 s for the whole LRR on 640 faces (Table 7, LRR+FRSVT, Matlab, CPU)"}


def bench_weather():
    """Type B RPCA (truncated nuclear norm, k = 1) on windows of 5 frames of the synthetic snow
    video (384 x 288 pixels): per window rpca_init + 30 iALM iterations with partial FRSVT (l = 3,
    q = 2, range propagation), O copied in and L, S copied out; device time per window."""
    import numpy as np
    import torch
    from paper_1509_00296_gb300 import frsvt, synth
    O_np, _, _ = synth.snow_video(frames=20)
    m, F = O_np.shape
    nwin, win, iters = F // 5, 5, 30
    def padded():                                   # leading dimension 8 (TMA rows: multiples of 16 bytes)
        return torch.zeros((m, 8), dtype=torch.float32, device="cuda")[:, :win]

    Od, S, A, L = padded(), padded(), padded(), padded()
    h = frsvt.Handle(m, win, 3, q=2, range_prop=True, seed=8, stream=torch.cuda.current_stream())
    h.set_partial(1)
    host = [torch.from_numpy(np.ascontiguousarray(O_np[:, w * win:(w + 1) * win])).pin_memory() for w in range(nwin)]
    Lh = torch.empty((m, win), dtype=torch.float32).pin_memory()
    Sh = torch.empty((m, win), dtype=torch.float32).pin_memory()

    def window(w):
        Od.copy_(host[w], non_blocking=True)
        h.rpca_init(Od, S, A, 1.0 / np.sqrt(m), 1.5, 1e7)
        for k in range(iters):
            h.ialm_step(Od, S, A, 3, L=L if k == iters - 1 else None)
        Lh.copy_(L, non_blocking=True)
        Sh.copy_(S, non_blocking=True)

    window(0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record()
    for w in range(nwin):
        window(w)
    e1.record()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    info = h.info()
    h.close()
    ms = e0.elapsed_time(e1) / nwin
    return {"workload": "snow video 384 x 288, windows of 5 frames (110592 x 5), Type B iALM k = 1, l = 3, q = 2, "
                        "30 iterations per window", "ms_per_window": ms, "ms_per_frame": ms / win,
            "wall_ms_per_window": 1e3 * wall / nwin, "rank": info.r, "residual": info.residual,
            "paper_context": "65.5 ms per frame (n = 5 window, Matlab 2014a, one CPU thread, Sec. 4.2)"}


def bench_recovery(args, O, lam, dev, flush):
    """The headline workload in the BF16-shadow and FP8-shadow (E4M3, per-128 x 128-tile power-of-two
    scales) modes (sketch and first power step on the shadow, FP32-accurate last power step and
    projection), and at FP32 with range propagation (Alg. 1 steps 8-11) or with the intermediate
    power step left unnormalised (Sec. 2.5).  Iterations per second from a captured graph and
    per-phase device times (the "orth" phase shows the Cholesky QR each variant saves or keeps)."""
    import torch
    from paper_1509_00296_gb300 import frsvt
    out = {"workload": RWORKLOAD, "unit": UNIT, "hbm_floor_ms_fp32": 11 * 4.0 * RN * RN / (peaks()[0] * 1e9) * 1e3}
    S = torch.empty_like(O)
    A = torch.empty_like(O)
    variants = (("bf16", frsvt.PREC_BF16, False, False), ("fp8", frsvt.PREC_FP8, False, False),
                ("fp32_range_prop", frsvt.PREC_FP32, True, False), ("fp32_orth_last", frsvt.PREC_FP32, False, True))
    for name, prec, rp, ol in variants:
        h = frsvt.Handle(RN, RN, RL, q=RQ, range_prop=rp, seed=ROMEGA_SEED, stream=torch.cuda.current_stream(),
                         precision=prec, orth_last=ol)
        h.rpca_init(O, S, A, lam, 1.5, 1e7)
        for _ in range(3):
            h.ialm_step(O, S, A, RL)
        K = 5
        h.enable_timing(True)
        h.timings()
        for k in range(K):
            flush.fill_(float(k))
            h.ialm_step(O, S, A, RL)
        tm = h.timings()
        h.enable_timing(False)
        reps = graph_replay_ms(h, O, S, A, RL, 10, flush)
        ms = statistics.fmean(reps)
        info = h.info()
        out[name] = {"ms_per_step": ms, "value": 1e3 / ms,
                     "replay_ms_median": statistics.median(reps), "replay_ms_max": max(reps),
                     "phases_ms_per_step": {k: v[0] / K for k, v in tm.items() if v[1] > 0},
                     "launch_groups_per_step": sum(v[1] for v in tm.values()) / K, "jacobi_sweeps": info.sweeps,
                     "rank": info.r, "basis": info.s, "device_status": info.device_status}
        if rp:
            out[name]["propagated_columns"] = info.keep
        h.close()
    return out


def bench_wsvt(dev):
    """Batched weighted SVT: 16384 WNNM patch groups 64 x n_i, n_i in [40, 160], one launch per
    variant after the autotuner; problems per second (device time, CUDA events)."""
    import torch
    from paper_1509_00296_gb300 import frsvt, synth
    mats, _ = synth.wnnm_batch(seed=1004)
    dm = [torch.from_numpy(a).to(dev) for a in mats]
    out = [torch.empty_like(t) for t in dm]
    a = torch.tensor([t.data_ptr() for t in dm], dtype=torch.int64, device=dev)
    x = torch.tensor([t.data_ptr() for t in out], dtype=torch.int64, device=dev)
    n = torch.tensor([t.shape[1] for t in dm], dtype=torch.int32, device=dev)
    h = frsvt.Handle(64, 160, 16, q=1, seed=11, stream=torch.cuda.current_stream())
    res = {"workload": "16384 patch groups 64 x n_i, n_i uniform in [40, 160], rank 4 + N(0, 0.05^2), "
                       "w_j = 2.8 sqrt(n_i) / (sigma_j + 1e-8)", "unit": "problems/s"}
    for v, name in ((frsvt.WSVT_EXACT, "exact"), (frsvt.WSVT_FRSVT, "frsvt_l12_q1")):
        h.wsvt_raw(a, n, 64, 2.8, 1e-8, x, v, 12, tune=True)
        for _ in range(2):
            h.wsvt_raw(a, n, 64, 2.8, 1e-8, x, v, 12)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(5):
            h.wsvt_raw(a, n, 64, 2.8, 1e-8, x, v, 12)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 5
        res[name] = {"ms_per_batch": ms, "value": 16384 / ms * 1e3, "launch_shape": h.wsvt_tuning(v)}
    return res


def bench_unrolled(dev):
    """Unrolled RPCA training step: batch of 8 matrices 2048 x 512, 10 iALM steps with FRSVT
    (l = 16, q = 1), loss ||L_10 - L_true||^2, forward + backward (device time); the batch's y0
    scales are computed once per batch and reported on their own."""
    import numpy as np
    import torch
    from paper_1509_00296_gb300 import synth
    from paper_1509_00296_gb300.unrolled import RPCAUnrolled
    O, L, _ = synth.unrolled_batch(seed=1005)
    Ob = torch.from_numpy(O.astype(np.float32)).to(dev)
    Lb = torch.from_numpy(L.astype(np.float32)).to(dev)
    net = RPCAUnrolled(2048, 512, steps=10, l=16, q=1, mu0=1.25 / float(np.linalg.norm(O[0], 2)))

    def train_step():
        net.tau.grad = None
        net.mu.grad = None
        loss = net.loss(Ob, Lb)
        loss.backward()
        return loss

    train_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    net.dual_scales(Ob)                      # the per-batch y0 scales, timed on their own
    e1.record()
    torch.cuda.synchronize()
    scales_ms = e0.elapsed_time(e1)
    e0.record()
    reps = 3
    for _ in range(reps):
        loss = train_step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    return {"workload": "8 x (2048 x 512), rank 8 + 5 % outliers, 10 unrolled iALM steps, FRSVT l=16 q=1",
            "ms_per_training_step": ms, "loss": float(loss.detach()), "unit": "training steps/s", "value": 1e3 / ms,
            "y0_scales_ms_per_batch": scales_ms,
            "note": "forward + backward; the batch's y0 scales (data-only constants) are computed once per batch "
                    "tensor and timed separately"}


if __name__ == "__main__":
    sys.exit(main())
