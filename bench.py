#!/usr/bin/env python
"""Throughput of the fast damped Gauss-Newton (fLM) step on one GB300.

Workload (one decomposition per GPU; with --gpus N each rank runs its own
seeded problem, no data exchanged -- replicas, weak scaling):
  200 x 200 x 200 tensor, rank R = 20, float32 values stored as two bfloat16
  planes; factors with mode-1 collinearity 0.95 and modes 2-3 collinearity
  0.81; noise at SNR 40 dB; seeded N(0, 1) initial factors.
A "step" is one Levenberg-Marquardt trial: Gramians, damped inverses, w,
core build, float32 Gauss-Jordan inverse of the core + float64 refinement,
update, one pass over the tensor (MTTKRP and direct residual at the trial
point), gain ratio, damping update, normalisation, stop test -- captured once
in a CUDA graph and replayed.  Every 50 launches the run restarts from its
initial factors (outside the timed events) so every timed step is an ordinary
trial of an unconverged run.  The 32 MB tensor fits in L2, so L2 is flushed (a
256 MB write) between timed steps, outside the timed events.

Also reported: the plain float64 form (float64 tensor and float64 core
Cholesky) on the same problem, time-to-fit of both forms (stop when an
accepted step changes the relative error by < 1e-9), the float32 core
inverse and the MTTKRP pass alone against their rooflines, an end-to-end
figure through the public API (every step copies its float32 tensor from
pinned host memory on a copy stream, overlapping the previous step, splits
it and replays a captured one-step graph, then reads its status back), ALS
sweeps on the same tensor, the batched and served forms, and the CPU oracle
on the host cores.

--impl reference times the CPU oracle (the float64 numpy implementation in
oracle/) on the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fast-dGN iters/s & time-to-fit vs plain FP64 GPU form; p99 served latency"
DIMS = (200, 200, 200)
R = 20
WORKLOAD = "cp3-200^3-R20-collinear(0.95,0.81,0.81)-snr40"
L2_FLUSH_BYTES = 256 << 20
# DRAM traffic per launch, dram__bytes_read.sum + dram__bytes_write.sum from
# one ncu capture of the kernel (bytes); None where the kernel has changed
# since its counters were taken.
TRAFFIC_TC3_200 = 32.2932e6             # k_mttkrp_tc3, 200^3 R=20, two-plane tensor (mean of two launches)
TRAFFIC_TC3_512 = 539.4846e6            # k_mttkrp_tc3, 512^3 R=32 (mean of two launches)
TRAFFIC_TC_200 = 32.2857e6              # k_mttkrp_tc, 200^3 R=20, float32 tensor (mean of two launches)
TRAFFIC_TC_512 = 539.4094e6             # k_mttkrp_tc, 512^3 R=32, float32 tensor (mean of two launches)
# summed over the kernels of one float32 core inverse (n = 1200), every kernel
# with cold caches under ncu (bytes)
GJ_TRAFFIC = 84.523e6
# timed runs restart from their initial factors every this many launches
RESTART_EVERY = 50


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--no-batch", action="store_true", help="skip the 512-problem batched run")
    p.add_argument("--serve-seconds", type=float, default=60.0,
                   help="length of the served Poisson stream (0 = skip)")
    p.add_argument("--serve-rate", type=float, default=200.0)
    p.add_argument("--serve-slots", type=int, default=4,
                   help="large requests running at once on their own device States")
    p.add_argument("--no-extras", action="store_true",
                   help="only the timed steps (no float64 form, time-to-fit, oracle)")
    p.add_argument("--profile", default="", choices=["", "mttkrp", "step"],
                   help="profiling driver: run only this part (no JSON line)")
    p.add_argument("--dims", default="", help="tensor dims for --profile, e.g. 400,400,400")
    p.add_argument("--rank", type=int, default=R)
    p.add_argument("--dtype", default="f32", choices=["f64", "f32", "bf16", "bf16x2"])
    return p.parse_args()


def run_profile(args):
    """Run one part of the path a few times on a seeded device tensor (for ncu)."""
    import torch
    from paper_1205_2584_gb300 import cpdgn as cp
    torch.cuda.set_device(0)
    dims = tuple(int(x) for x in args.dims.split(",")) if args.dims else DIMS
    g = torch.Generator(device="cuda").manual_seed(args.seed)
    shape = cp.make_shape(dims, args.rank, args.dtype)
    J = 1
    for d in dims:
        J *= d
    Y = torch.randn(J, generator=g, device="cuda", dtype=torch.float32)
    Y = cp.tensor_split(Y) if args.dtype == "bf16x2" else Y.to(cp.TORCH_DTYPE[shape.y_dtype])
    a = torch.randn(args.rank * sum(dims), generator=g, device="cuda", dtype=torch.float64)
    with torch.cuda.stream(torch.cuda.Stream()):
        if args.profile == "mttkrp":
            ws = cp.alloc_workspace(shape)
            for _ in range(args.warmup + args.steps):
                cp.mttkrp_all(shape, Y, a, ws=ws)
        else:
            st = cp.State(shape, a, mu0=-1.0, mu_max=float("inf"), max_iter=10 ** 9,
                          core_mode=cp.CP_CORE_MIXED if args.dtype != "f64" else cp.CP_CORE_F64, refine_iters=8)
            st.init(Y)
            for _ in range(args.warmup + args.steps):
                st.step(Y)
        torch.cuda.synchronize()


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------

class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.t:
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def dist_init(args):
    import torch
    rank, world = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(x: float, world: int) -> float:
    """Largest value over the ranks (the slowest rank's time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(t_ms_local: float, steps: int, world: int):
    """Whole-job throughput of `world` replicas that each ran `steps` steps:
    all steps over the slowest rank's time (weak scaling).  Returns
    (iters/s, ms per step, max time in ms)."""
    t_ms = allmax(t_ms_local, world)
    return world * steps / (t_ms / 1e3), t_ms / steps, t_ms


def oracle_threads():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        n = [i.get("num_threads", 0) for i in info if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_rate(problem, seconds: float):
    """Oracle LM iterations per second on a bounded sample of the workload."""
    from oracle import cp_oracle as O
    t0 = time.perf_counter()
    res = O.lm_fit(problem.Y, problem.init, mu0=None, max_iter=1, tol=0.0)
    t1 = time.perf_counter()
    per = max(t1 - t0, 1e-3)
    k = max(2, int(seconds / per))
    t0 = time.perf_counter()
    res = O.lm_fit(problem.Y, problem.init, mu0=None, max_iter=k, tol=0.0)
    dt = time.perf_counter() - t0
    return res.iters / dt, res.iters, dt


# FP32 multiply-add lanes per SM and SM count of a GB300 (derived ALU peak:
# SMs x lanes x 2 flops x maximum SM clock)
FP32_FMA_PER_SM_CLK = 128
GB300_SMS = 152


def gj_inverse_flops(n: int, ident: int, b: int = 64) -> int:
    """Algorithmic flops of the blocked Gauss-Jordan inverse of an n x n
    matrix whose leading ident rows are the identity (eliminated at once):
    the identity step updates the (n - e)^2 trailing block with depth e;
    every later sweep with panel width w does the rank-w update of the n - w
    rows outside the panel (all n columns), the row panel P^{-1} A[k, :] and
    the inverse of its pivot block (w^3).  The library forms each next pivot
    block ahead of its sweep; those products repeat work counted here (one
    row-panel block and one update tile) and are not counted again."""
    nt = (n + b - 1) // b
    k0 = min(ident // b, nt - 1)
    e = k0 * b
    fma = (n - e) ** 2 * e
    for k in range(k0, nt):
        w = min(b, n - k * b)
        fma += (n - w) * n * w + w * w * (n - w) + w ** 3
    return 2 * fma


def core_cholesky_flops(N: int, R: int) -> float:
    """The method's algorithmic core work per trial (Sec. 4.4 complexity):
    one Cholesky of the N R^2 x N R^2 core, n^3 / 3 flops with n = N R^2."""
    n = N * R * R
    return n ** 3 / 3.0


def core_inverse_roofline(cp, torch, flush, peaks, peak_src, seed, reps=20):
    """cp_spd_invert_f32 timed live on an SPD matrix shaped like the
    benchmark's core (n = N R^2 = 1200, identity diagonal R^2 x R^2 blocks),
    L2 flushed and the input restored between launches (outside the events).
    The call is captured once in a CUDA graph and the replays are timed, as
    inside the step's graph (host launch overhead is not device time).

    `achieved` counts the method's core work, one Cholesky of the core
    (n^3 / 3 flops), over the time the library takes to solve the core system
    this way; the inverse's own flop count is reported beside it."""
    import numpy as np
    n, blk = len(DIMS) * R * R, R * R
    rng = np.random.default_rng(seed + 17)
    X = rng.standard_normal((n, n))
    X = X + X.T
    for b0 in range(0, n, blk):
        X[b0:b0 + blk, b0:b0 + blk] = 0.0
    X *= 0.45 / np.linalg.norm(X, 2)
    M = torch.from_numpy((np.eye(n) + X).astype(np.float32).ravel(order="F").copy()).cuda()
    A = torch.empty_like(M)
    inv = cp.SpdInverse(n, blk)
    for _ in range(3):
        A.copy_(M)
        inv.run(A)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    A.copy_(M)
    with torch.cuda.graph(g, stream=torch.cuda.current_stream()):
        inv.run(A)
    evs = []
    for _ in range(reps):
        A.copy_(M)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        evs.append((e0, e1))
    torch.cuda.synchronize()
    ms = statistics.mean(a.elapsed_time(b) for a, b in evs)
    alg = core_cholesky_flops(len(DIMS), R)
    own = gj_inverse_flops(n, blk)
    peak = GB300_SMS * FP32_FMA_PER_SM_CLK * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    achieved = alg / (ms * 1e-3) / 1e12
    return {"bound": "alu", "kernel": "k_gj_* (float32 Gauss-Jordan inverse of the core, one call)",
            "workload": f"n = N R^2 = {n}, identity {blk} x {blk} blocks, SPD", "achieved": achieved,
            "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": GJ_TRAFFIC,
            "traffic_note": "DRAM bytes of one inverse under ncu, every kernel with cold caches: an upper "
                            "bound; inside the step the core is L2-resident",
            "ms_per_launch": ms, "algorithmic_flops": alg,
            "algorithmic_count": "core Cholesky n^3/3, n = N R^2 (the method's core work, Sec. 4.4)",
            "inverse_own_flops": own, "inverse_own_tflops": own / (ms * 1e-3) / 1e12,
            "peak_source": "derived, not measured: 152 SMs x 128 FP32 FMA lanes x 2 flops x max SM clock "
                           "(MEASURED_PEAKS.json has no FP32 figure)",
            "note": "latency-bound pivot chain (13 sweeps of 64 dependent elimination steps)"}


def oracle_rate_one_thread(seed: int, seconds: float):
    """oracle_rate on one host thread: a child interpreter with the BLAS and
    OpenMP pools limited to one thread before numpy loads."""
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "from paper_1205_2584_gb300 import synth; "
            "p = synth.config2(%d, bench.DIMS, dtype='bf16x2'); "
            "print(json.dumps(bench.oracle_rate(p, %f)))") % (ROOT, seed, seconds)
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = "1"
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                           timeout=max(120.0, 10 * seconds))
        rate, iters, secs = json.loads(r.stdout.strip().splitlines()[-1])
        return {"value": rate, "unit": "iters/s", "cores": 1,
                "sample": f"first {iters} LM iterations, {secs:.1f} s"}
    except Exception as e:   # reported, never fatal
        return {"value": None, "error": str(e)[:200]}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(args):
    import torch
    rank, world, local = dist_init(args)
    # every launch goes to one non-default stream (CUDA graphs cannot capture
    # the legacy default stream)
    with torch.cuda.stream(torch.cuda.Stream()):
        _run_ours(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _run_ours(args, rank, world, local):
    import numpy as np
    import torch

    from paper_1205_2584_gb300 import cpdgn as cp
    from paper_1205_2584_gb300 import synth

    seed = args.seed + rank
    peaks, peak_src = measured_peaks()
    # the benchmark tensor: float32 values (config 2's "FP32" tensor); the
    # oracle and the float64 form see the same values in float64
    prob = synth.config2(seed, DIMS, dtype="f32")
    shape32 = cp.make_shape(DIMS, R, "f32")
    Y32 = cp.tensor_to_device(prob.Y, "f32")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def new_state(shape, mode, a0, tol=0.0, max_iter=10 ** 9, mu_max=float("inf"), mu0=-1.0,
                  normalize=True):
        a = cp.factors_to_device(a0)
        st = cp.State(shape, a, mu0=mu0, tau=1e-3, tol=tol, mu_max=mu_max, max_iter=max_iter,
                      core_mode=mode, refine_iters=8, normalize=normalize)
        return st, a

    def timed_steps(st, a, Y, K, W, period=RESTART_EVERY):
        """Time K graph-replayed steps after W warm-up steps.  Every `period`
        launches the run restarts from its initial factors (outside the timed
        events), so that every timed step is an ordinary trial of an
        unconverged run rather than a no-progress step at huge damping."""
        a0 = a.clone()
        nk = st.capture(Y, 1)
        launches = 0

        def rearm():
            if launches and launches % period == 0:
                a.copy_(a0)
                st.init(Y)

        for _ in range(W):
            rearm()
            st.launch()
            launches += 1
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        barrier(world)
        torch.cuda.synchronize()
        for i in range(K):
            rearm()
            flush.zero_()                     # L2 flush, outside the timed events
            ev[i][0].record()
            st.launch()
            ev[i][1].record()
            launches += 1
        torch.cuda.synchronize()
        barrier(world)
        return sum(a.elapsed_time(b) for a, b in ev), nk

    def time_pass(shape, Y, a_in, reps=20):
        """cp_mttkrp_all (MTTKRP + direct residual, one pass) timed alone, L2
        flushed.  The call is captured once in a CUDA graph and the replays are
        timed, as inside the step's graph: the host-side work of the call
        (tensor-map encoding, launch) is not device time."""
        ws = cp.alloc_workspace(shape)
        m = torch.empty_like(a_in)
        r2 = torch.empty(1, dtype=torch.float64, device="cuda")
        call = lambda: cp._check(cp._lib.cp_mttkrp_all(cp.ctypes.byref(shape), cp._ptr(Y), cp._ptr(a_in),
                                                       cp._ptr(m), cp._ptr(r2), cp._ptr(ws), ws.numel(),
                                                       cp._stream()), "cp_mttkrp_all")
        for _ in range(3):
            call()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=torch.cuda.current_stream()):
            call()
        for _ in range(3):
            g.replay()
        evs = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            g.replay()
            e1.record()
            evs.append((e0, e1))
        torch.cuda.synchronize()
        return statistics.mean(e0.elapsed_time(e1) for e0, e1 in evs)

    # --- timed region: mixed form on the float32 tensor (tensor-core pass,
    # float32 core inverse + float64 refinement, float64 control) ---
    st, a = new_state(shape32, cp.CP_CORE_MIXED, prob.init)
    st.init(Y32)
    with ClockSampler(local) as clk:
        t_ms, nk = timed_steps(st, a, Y32, args.steps, args.warmup)
    status = st.status()
    value, ms_per_step, t_ms = aggregate(t_ms, args.steps, world)

    out = {"metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "f32 tensor (bf16-piece tensor-core products, f32 accumulate), f32 core inverse + "
                    "f64 refinement, f64 control",
           "data": "synthetic",
           "config": {"workload": WORKLOAD, "dims": list(DIMS), "R": R,
                      "tensor_dtype": "f32",
                      "core": "f32 Gauss-Jordan inverse + f64 refinement (<= 8 sweeps, adaptive)",
                      "l2": "flushed between steps",
                      "parallelism": f"replicas x{world}", "global_batch": world},
           "gpu_launches": nk * args.steps, "clocks": clk.summary(),
           "state_after": {k: status[k] for k in ("iters", "accepted", "rel_err", "mu", "stop_reason",
                                                  "refine_resid", "refine_sweeps")}}

    if not args.no_extras and rank == 0:
        from oracle import cp_oracle as O
        prob2 = synth.config2(seed, DIMS, dtype="bf16x2")
        shape2 = cp.make_shape(DIMS, R, "bf16x2")
        Y2 = cp.tensor_to_device(prob2.Y, "bf16x2")
        shape64 = cp.make_shape(DIMS, R, "f64")
        Y64 = cp.tensor_to_device(prob.Y, "f64")          # the float32 values, stored as float64

        # --- the tensor pass alone against HBM: this workload and a large one ---
        a_in = cp.factors_to_device(prob.init)
        mt_ms = time_pass(shape32, Y32, a_in)
        bytes_alg = int(np.prod(DIMS)) * 4
        achieved = bytes_alg / (mt_ms * 1e-3) / 1e9
        out["roofline_tensor_pass"] = {"bound": "hbm", "kernel": "k_mttkrp_tc (all-mode MTTKRP + direct residual, "
                                                                 "one pass, float32 tensor)",
                                       "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                       "frac": achieved / peaks["hbm_gbs"], "traffic": TRAFFIC_TC_200,
                                       "peak_source": f"{peak_src} hbm_gbs", "ms_per_launch": mt_ms,
                                       "algorithmic_bytes": bytes_alg, "peak_kind": "burst (kernel timed alone)"}
        mt2_ms = time_pass(shape2, Y2, a_in)
        out["roofline_tensor_pass_bf16x2"] = {"bound": "hbm", "kernel": "k_mttkrp_tc3 (two-plane tensor)",
                                              "achieved": bytes_alg / (mt2_ms * 1e-3) / 1e9,
                                              "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                              "frac": bytes_alg / (mt2_ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
                                              "traffic": TRAFFIC_TC3_200, "ms_per_launch": mt2_ms}
        big = (512, 512, 512)
        gbig = torch.Generator(device="cuda").manual_seed(seed)
        Ybig = torch.randn(int(np.prod(big)), generator=gbig, device="cuda", dtype=torch.float32)
        abig = torch.randn(32 * sum(big), generator=gbig, device="cuda", dtype=torch.float64)
        bbig = int(np.prod(big)) * 4
        big_ms = time_pass(cp.make_shape(big, 32, "f32"), Ybig, abig)
        out["roofline_large"] = {"bound": "hbm", "kernel": "k_mttkrp_tc", "workload": "512^3, R=32, f32",
                                 "achieved": bbig / (big_ms * 1e-3) / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                 "frac": bbig / (big_ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
                                 "ms_per_launch": big_ms, "algorithmic_bytes": bbig, "traffic": TRAFFIC_TC_512}
        Ybig2 = cp.tensor_split(Ybig)
        del Ybig
        big2_ms = time_pass(cp.make_shape(big, 32, "bf16x2"), Ybig2, abig)
        out["roofline_large_bf16x2"] = {"bound": "hbm", "kernel": "k_mttkrp_tc3", "workload": "512^3, R=32, bf16x2",
                                        "achieved": bbig / (big2_ms * 1e-3) / 1e9, "peak": peaks["hbm_gbs"],
                                        "unit": "GB/s", "frac": bbig / (big2_ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
                                        "ms_per_launch": big2_ms, "algorithmic_bytes": bbig,
                                        "traffic": TRAFFIC_TC3_512}
        del Ybig2, abig
        # --- the dominant kernel sequence of the step: the float32 core inverse ---
        out["roofline"] = core_inverse_roofline(cp, torch, flush, peaks, peak_src, seed)

        # --- the two-plane tensor form of the same step ---
        st2, a2 = new_state(shape2, cp.CP_CORE_MIXED, prob2.init)
        st2.init(Y2)
        k2 = max(5, args.steps // 2)
        t2, _ = timed_steps(st2, a2, Y2, k2, 2)
        out["bf16x2_tensor_form"] = {"value": k2 / (t2 / 1e3), "unit": "iters/s", "ms_per_step": t2 / k2,
                                     "tensor_dtype": "bf16x2 (hi + lo bfloat16 planes, 16 significant bits)"}
        st2.close()

        # --- ALS sweeps (Sec. 3, Eq. ALS; the initialisation before fLM) on the
        # same tensor: N passes over Y per sweep, one per mode ---
        st_a, a_a = new_state(shape32, cp.CP_CORE_MIXED, prob.init)
        st_a.init(Y32)
        st_a.als(Y32, 2)
        torch.cuda.synchronize()
        ka = 10
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st_a.als(Y32, ka)
        e1.record()
        torch.cuda.synchronize()
        als_ms = e0.elapsed_time(e1) / ka
        out["als"] = {"value": 1e3 / als_ms, "unit": "sweeps/s", "ms_per_sweep": als_ms,
                      "passes_per_sweep": len(DIMS), "sweeps_timed": ka,
                      "status_error": st_a.status()["error"]}
        st_a.close()

        # --- end to end through the public API: float32 tensor on the host ---
        # Every step copies its own input (the pinned float32 tensor) to the
        # device, places it in the state's tensor buffer, runs the step (one
        # replay of a captured one-step graph) and reads its status back.  Two
        # staging buffers: step k + 1's host copy runs on a copy stream while
        # step k computes; a staging buffer is overwritten only after the
        # device copy that read it has run.
        Yh = torch.from_numpy(np.asarray(prob.Y, dtype=np.float32).ravel(order="F")).pin_memory()
        Yst = [torch.empty(Yh.numel(), dtype=torch.float32, device="cuda") for _ in range(2)]
        Yd = torch.empty(Yh.numel(), dtype=torch.float32, device="cuda")
        st_e, a_e = new_state(shape32, cp.CP_CORE_MIXED, prob.init)
        a_e0 = a_e.clone()
        Yd.copy_(Yh)
        st_e.init(Yd)
        st_e.capture(Yd, 1)
        for _ in range(args.warmup):
            st_e.launch()
        hst = torch.empty(128, dtype=torch.uint8).pin_memory()
        cur = torch.cuda.current_stream()
        cs = torch.cuda.Stream()
        ev_c = [torch.cuda.Event(), torch.cuda.Event()]     # host copy into staging buffer b done
        ev_s = [torch.cuda.Event(), torch.cuda.Event()]     # staging buffer b consumed
        torch.cuda.synchronize()
        e2e_ms, done = 0.0, 0
        while done < args.steps:
            a_e.copy_(a_e0)
            st_e.init(Yd)
            chunk = min(RESTART_EVERY, args.steps - done)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            cs.wait_stream(cur)
            with torch.cuda.stream(cs):
                Yst[0].copy_(Yh, non_blocking=True)
                ev_c[0].record(cs)
            for k in range(chunk):
                b = k & 1
                if k + 1 < chunk:
                    with torch.cuda.stream(cs):
                        if k >= 1:
                            cs.wait_event(ev_s[1 - b])
                        Yst[1 - b].copy_(Yh, non_blocking=True)
                        ev_c[1 - b].record(cs)
                cur.wait_event(ev_c[b])
                Yd.copy_(Yst[b])
                ev_s[b].record(cur)
                st_e.launch()
                hst.copy_(st_e.status_tensor(), non_blocking=True)
            e1.record()
            torch.cuda.synchronize()
            e2e_ms += e0.elapsed_time(e1)
            done += chunk
        out["e2e"] = {"value": args.steps / (e2e_ms / 1e3), "unit": "iters/s",
                      "h2d_bytes_per_step": Yh.numel() * Yh.element_size(), "d2h_bytes_per_step": 128,
                      "path": "pinned float32 host tensor -> device staging buffer (copy stream, two buffers: the "
                              "next step's copy overlaps this step) -> the state's tensor buffer, one captured "
                              "cp_dgn_step, status -> host"}
        st_e.close()
        del Yst, Yd

        # --- plain float64 form on the float64 tensor ---
        st64, a64 = new_state(shape64, cp.CP_CORE_F64, prob.init)
        st64.init(Y64)
        k64 = max(5, args.steps // 5)
        t64, _ = timed_steps(st64, a64, Y64, k64, 2)
        out["fp64_form"] = {"value": k64 / (t64 / 1e3), "unit": "iters/s", "ms_per_step": t64 / k64,
                            "tensor_dtype": "f64 (the float32 values)", "core": "f64 Cholesky", "steps": k64}
        out["speedup_vs_fp64_form"] = value / out["fp64_form"]["value"]
        st64.close()

        # --- time to fit, both forms, and every form against the FP64 oracle ---
        def ttf(shape, Y, init, mode, cap=3000, chunk=20):
            s, _ = new_state(shape, mode, init, tol=1e-9, max_iter=cap, mu_max=1e30)
            s.init(Y)
            s.capture(Y, chunk)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            while True:
                s.launch()
                d = s.status()
                if d["stop"] != 0:
                    break
            t = time.perf_counter() - t0
            s.close()
            return {"seconds": t, "iters": d["iters"], "accepted": d["accepted"], "rel_err": d["rel_err"],
                    "stop": d["stop_reason"], "error": d["error"]}
        ttf32 = ttf(shape32, Y32, prob.init, cp.CP_CORE_MIXED)
        ttf64 = ttf(shape64, Y64, prob.init, cp.CP_CORE_F64)
        ttf2 = ttf(shape2, Y2, prob2.init, cp.CP_CORE_MIXED)
        out["time_to_fit"] = {"mixed": ttf32, "plain_f64": ttf64, "mixed_bf16x2": ttf2,
                              "gain": ttf64["seconds"] / ttf32["seconds"],
                              "rel_err_diff": abs(ttf32["rel_err"] - ttf64["rel_err"]) / ttf64["rel_err"]}
        out["oracle_error"] = oracle_errors(cp, O, torch, prob, prob2, shape32, shape2, shape64, Y32, Y2, Y64,
                                            {"mixed_f32": ttf32, "plain_f64": ttf64, "mixed_bf16x2": ttf2})

        out["config1"] = bench_config1(cp, O, torch, seed)
        out["config3"] = bench_config3(cp, O, torch, seed, flush)
        out["next_rows"] = bench_next_rows(cp, O, torch, seed, prob, Y32)
        if not args.no_batch:
            out["batched"] = bench_batched(seed)
        if args.serve_seconds > 0:
            out["served"] = bench_served(seed, args.serve_seconds, args.serve_rate, args.serve_slots)

        # --- CPU oracle on the host cores (bounded sample) ---
        rate, iters, secs = oracle_rate(prob, args.cpu_seconds)
        out["cpu_baseline"] = {"value": rate, "unit": "iters/s", "cores": oracle_threads(),
                               "kind": "oracle",
                               "sample": f"first {iters} LM iterations of the same 200^3 R=20 problem "
                                         f"(the same float32 tensor values in float64), {secs:.1f} s",
                               "one_thread": oracle_rate_one_thread(seed, max(2.0, args.cpu_seconds / 3))}
    st.close()
    if rank == 0:
        print(json.dumps(out), flush=True)


def _rel(a, b):
    import numpy as np
    a = np.concatenate([np.ravel(np.asarray(x)) for x in a])
    b = np.concatenate([np.ravel(np.asarray(x)) for x in b])
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def gpu_step_delta(cp, torch, shape, Y, A, mu, mode):
    """One GPU trial from factors A at damping mu (no normalisation): its step."""
    a = cp.factors_to_device(A)
    st = cp.State(shape, a, mu0=float(mu), max_iter=10, core_mode=mode, normalize=False, refine_iters=8)
    st.init(Y)
    st.step(Y)
    torch.cuda.synchronize()
    dims = [x.shape[0] for x in A]
    Rr = A[0].shape[1]
    d = [x.numpy().copy() for x in cp.split_factors(st.buffer(cp.State.BUF_DELTA, Rr * sum(dims)).cpu(), dims, Rr)]
    s = st.status()
    st.close()
    return d, s


def core_kappa(O, A, mu):
    import numpy as np
    ev = np.linalg.eigvalsh(O.spd_core(A, mu))
    return float(ev[-1] / ev[0])


def oracle_errors(cp, O, torch, prob, prob2, shape32, shape2, shape64, Y32, Y2, Y64, ttfs):
    """Every form against the FP64 oracle: (1) one step from a fixed state of
    the oracle's own trajectory (after 20 LM iterations from the seeded start,
    where mu is already well below its start), relative to the oracle's
    fLM_a step, with kappa of the core there; (2) the final epsilon of the
    form's run to its stop rule (relative fit change < 1e-9) against the
    oracle's run to the same rule on the same tensor values."""
    out = {}
    t0 = time.perf_counter()
    ref32 = O.lm_fit(prob.Y, prob.init, mu0=None, max_iter=3000, tol=1e-9)
    ref2 = O.lm_fit(prob2.Y, prob2.init, mu0=None, max_iter=3000, tol=1e-9)
    mid32 = O.lm_fit(prob.Y, prob.init, mu0=None, max_iter=20, tol=0.0)
    mid2 = O.lm_fit(prob2.Y, prob2.init, mu0=None, max_iter=20, tol=0.0)
    for name, pr, ref, mid, shape, Y, mode in (
            ("plain_f64", prob, ref32, mid32, shape64, Y64, cp.CP_CORE_F64),
            ("mixed_f32", prob, ref32, mid32, shape32, Y32, cp.CP_CORE_MIXED),
            ("mixed_bf16x2", prob2, ref2, mid2, shape2, Y2, cp.CP_CORE_MIXED)):
        d, s = gpu_step_delta(cp, torch, shape, Y, mid.A, mid.mu, mode)
        ost = O.flm_step(pr.Y, mid.A, mid.mu)
        ttf = ttfs[name]
        out[name] = {"step_rel_err": _rel(d, ost.delta), "step_state": {"oracle_iter": 20, "mu": mid.mu,
                                                                        "kappa_core": core_kappa(O, mid.A, mid.mu)},
                     "refine_sweeps": s["refine_sweeps"], "refine_resid": s["refine_resid"],
                     "final_eps": ttf["rel_err"], "oracle_final_eps": ref.rel_err,
                     "final_eps_rel_err": abs(ttf["rel_err"] - ref.rel_err) / ref.rel_err,
                     "iters": ttf["iters"], "oracle_iters": ref.iters, "oracle_stop": ref.stop}
    out["oracle_seconds"] = time.perf_counter() - t0
    return out


def bench_config1(cp, O, torch, seed):
    """20^3, R = 5, float64, mu_0 = 1, 200 LM iterations (graph-captured in
    one launch): microseconds per step and the 200-iteration wall time, and
    the final epsilon against the oracle's 200 iterations from the same start."""
    from paper_1205_2584_gb300 import synth
    p = synth.config1(seed)
    shape = cp.make_shape(p.dims, p.R, "f64")
    Y = cp.tensor_to_device(p.Y, "f64")
    a = cp.factors_to_device(p.init)
    a0 = a.clone()
    st = cp.State(shape, a, mu0=1.0, max_iter=200, mu_max=float("inf"), core_mode=cp.CP_CORE_F64)
    st.capture(Y, 200)
    times = []
    for _ in range(4):
        a.copy_(a0)
        st.init(Y)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st.launch()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    s = st.status()
    st.close()
    ref = O.lm_fit(p.Y, p.init, mu0=1.0, max_iter=200, tol=0.0, mu_max=float("inf"))
    ms = statistics.median(times[1:])
    return {"workload": "cp3-20^3-R5-f64-snr30, mu0 = 1, 200 iterations", "us_per_step": 1e3 * ms / 200,
            "wall_ms_200_iters": ms, "iters": s["iters"], "rel_err": s["rel_err"],
            "oracle_rel_err": ref.rel_err, "final_eps_rel_err": abs(s["rel_err"] - ref.rel_err) / ref.rel_err,
            "core": "f64 Cholesky"}


def bench_config3(cp, O, torch, seed, flush):
    """60^4, R = 15 (core N R^2 = 900), column norms log-uniform over
    [1e-2, 1e2], SNR 30 dB, bfloat16 tensor: iterations/s of the mixed form
    and the float64 form (float64 tensor of the same values), their
    time-to-fit (relative fit change < 1e-9, at most 1500 trials), and one
    step of each against the oracle's step from the seeded start."""
    from paper_1205_2584_gb300 import synth
    p = synth.config3(seed)
    out = {"workload": "cp4-60^4-R15-lognorm(1e-2..1e2)-snr30, bf16 tensor"}
    forms = (("mixed_bf16", cp.make_shape(p.dims, p.R, "bf16"), cp.tensor_to_device(p.Y, "bf16"),
              cp.CP_CORE_MIXED),
             ("plain_f64", cp.make_shape(p.dims, p.R, "f64"), cp.tensor_to_device(p.Y, "f64"), cp.CP_CORE_F64))
    mu0 = O.initial_mu(p.init, 1e-3)
    ost = O.flm_step(p.Y, p.init, mu0)
    for name, shape, Y, mode in forms:
        a = cp.factors_to_device(p.init)
        a0 = a.clone()
        st = cp.State(shape, a, mu0=-1.0, tau=1e-3, max_iter=10 ** 9, mu_max=float("inf"), core_mode=mode,
                      refine_iters=8)
        st.init(Y)
        st.capture(Y, 1)
        for _ in range(3):
            st.launch()
        K = 20
        ev = []
        for i in range(K):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            st.launch()
            e1.record()
            ev.append((e0, e1))
        torch.cuda.synchronize()
        ms = sum(x.elapsed_time(y) for x, y in ev) / K
        st.close()
        # time to fit
        a.copy_(a0)
        st = cp.State(shape, a, mu0=-1.0, tau=1e-3, tol=1e-9, max_iter=1500, mu_max=1e30, core_mode=mode,
                      refine_iters=8)
        st.init(Y)
        st.capture(Y, 20)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        while True:
            st.launch()
            d = st.status()
            if d["stop"] != 0:
                break
        tf = time.perf_counter() - t0
        st.close()
        dl, _ = gpu_step_delta(cp, torch, shape, Y, p.init, mu0, mode)
        out[name] = {"iters_per_s": 1e3 / ms, "ms_per_step": ms, "time_to_fit_s": tf, "iters": d["iters"],
                     "accepted": d["accepted"], "rel_err": d["rel_err"], "stop": d["stop_reason"],
                     "step_rel_err_vs_oracle": _rel(dl, ost.delta)}
    out["iters_per_s_gain"] = out["mixed_bf16"]["iters_per_s"] / out["plain_f64"]["iters_per_s"]
    out["time_to_fit_gain"] = out["plain_f64"]["time_to_fit_s"] / out["mixed_bf16"]["time_to_fit_s"]
    out["final_eps_mixed_vs_f64"] = abs(out["mixed_bf16"]["rel_err"] - out["plain_f64"]["rel_err"]) / \
        out["plain_f64"]["rel_err"]
    out["step_state"] = {"mu": mu0, "kappa_core": core_kappa(O, p.init, mu0)}
    return out


def bench_next_rows(cp, O, torch, seed, prob, Y32):
    """The later rows of the method, each timed on the device and compared
    with the float64 oracle on the same inputs:
      hosvd     cp_hosvd (Algorithm 1 step 1) on the benchmark tensor
                (200^3, R = 20, float32 values), 30 subspace iterations;
      theorem4  cp_hinv_blocks + cp_hinv_diag (Theorem 4, Eq. fastblock) at
                the benchmark's start factors (N R^2 = 1200), mu = 1;
      sae       cp_sae (Eq. MedSAE: cosines, Hungarian matching) of the true
                factors against a perturbed, permuted copy, R = 20;
      complex   cp_cdgn_step (Theorems 5-8) on 70^4, R = 5 complex128 (the
                paper's complex experiments); the step error on 30^4, R = 5."""
    from paper_1205_2584_gb300 import synth
    import numpy as np
    out = {}

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best

    dims, R = prob.dims, prob.R
    shape = cp.make_shape(dims, R, "f32")
    a = torch.empty(R * sum(dims), dtype=torch.float64, device="cuda")
    ms = timed(lambda: cp.hosvd(shape, Y32, a, iters=30), 5)
    got = cp.split_factors(a.cpu(), dims, R)
    Yv = np.asarray(prob.Y, dtype=np.float32).astype(np.float64)
    ref = O.hosvd_factors(Yv, R)
    err = max(float(np.max(np.abs(got[n].numpy() - ref[n]))) for n in range(len(dims)))
    out["hosvd"] = {"workload": f"{dims[0]}^3, R={R}, float32 tensor, 30 subspace iterations", "ms": ms,
                    "max_abs_err_vs_oracle": err}

    shape64 = cp.make_shape(dims, R, "f64")
    a0 = cp.factors_to_device(prob.init)
    mu = 1.0
    res = {}

    def hb():
        res["b"] = cp.hinv_blocks(shape64, a0, mu)
    ms_b = timed(hb, 5)
    Gt, St, info = res["b"]
    ms_d = timed(lambda: cp.hinv_diag(shape64, a0, Gt, St), 5)
    Gt_ref, St_ref = O.hinv_blocks(prob.init, mu)
    n = len(dims) * R * R
    St_np = St.cpu().numpy().reshape(n, n, order="F")
    T = sum(dims)
    out["theorem4"] = {"workload": f"{dims[0]}^3, R={R} start factors, mu = 1 (N R^2 = {n})",
                       "blocks_ms": ms_b, "diag_ms": ms_d, "info": int(info.item()),
                       "St_rel_err_vs_oracle": _rel(St_np, St_ref),
                       "stored_doubles": len(dims) * R * R + n * n, "full_inverse_doubles": (R * T) ** 2}

    rng = np.random.default_rng(seed + 7)
    A = [np.asarray(f) for f in prob.true_factors]
    perm = rng.permutation(R)
    est = [(f + 0.05 * rng.standard_normal(f.shape))[:, perm] * rng.choice([-1.0, 1.0], R) for f in A]
    at, ae = cp.factors_to_device(A), cp.factors_to_device(est)
    res2 = {}

    def sf():
        res2["s"] = cp.sae(shape64, at, ae)
    us = 1e3 * timed(sf, 20)
    a2, pi = res2["s"]
    a2_ref, pi_ref = O.sae(A, est)
    out["sae"] = {"workload": f"N=3, R={R}, I_n={dims[0]}: true factors vs a perturbed, permuted copy",
                  "us_per_call": us, "max_abs_err_vs_oracle": float(np.max(np.abs(a2.cpu().numpy() - a2_ref))),
                  "permutation_equal": bool(np.array_equal(pi.cpu().numpy(), np.asarray(pi_ref))),
                  "medsae_db": cp.medsae_db([a2]), "oracle_medsae_db": O.medsae([a2_ref])}

    pc = synth.make_complex_problem(seed + 250, (70, 70, 70, 70), 5, snr_db=30)
    shc = cp.make_shape(pc.dims, pc.R, "c128")
    Yc = cp.ctensor_to_device(pc.Y)
    ac = cp.cfactors_to_device(pc.init)
    ac0 = ac.clone()
    st = cp.CState(shc, ac, mu0=-1.0, max_iter=100000, tol=0.0, normalize=True)
    k, best = 20, float("inf")
    for _ in range(4):                             # 20 trials from the start factors, the first run a warm-up
        ac.copy_(ac0)
        st.init(Yc)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(k):
            st.step(Yc)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    ms_c = best / k
    sc = st.status()
    st.close()
    del Yc
    ps = synth.make_complex_problem(seed + 251, (30, 30, 30, 30), 5, snr_db=30)
    shs = cp.make_shape(ps.dims, ps.R, "c128")
    Ys = cp.ctensor_to_device(ps.Y)
    asm = cp.cfactors_to_device(ps.init)
    mu_s = 0.5
    st = cp.CState(shs, asm, mu0=mu_s, max_iter=10, normalize=False)
    st.init(Ys)
    st.step(Ys)
    torch.cuda.synchronize()
    nA = ps.R * sum(ps.dims)
    d = st.buffer(cp.CState.BUF_DELTA, nA).cpu().numpy()
    st.close()
    ref_d = O.cflm_step(ps.Y, ps.init, mu_s)[0]
    ref_flat = np.concatenate([np.asarray(x).T.reshape(-1) for x in ref_d])
    out["complex"] = {"workload": "70^4, R=5, complex128, snr 30 (the paper's complex experiments)",
                      "iters_per_s": 1e3 / ms_c, "ms_per_step": ms_c, "iters": sc["iters"],
                      "rel_err_after": sc["rel_err"],
                      "step_rel_err_vs_oracle": float(np.linalg.norm(d - ref_flat) / np.linalg.norm(ref_flat)),
                      "step_case": "30^4, R=5, mu = 0.5, from the start factors"}
    return out


def _ttf_state(cp, shape, Y, a0, mode, tol, cap=1000, chunk=20):
    """Run one State to its stop rule in graph chunks; wall seconds + status."""
    import torch
    a = a0.clone() if torch.is_tensor(a0) else cp.factors_to_device(a0)
    st = cp.State(shape, a, mu0=-1.0, tau=1e-3, tol=tol, mu_max=1e30, max_iter=cap, core_mode=mode,
                  refine_iters=8)
    st.capture(Y, chunk)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st.init(Y)
    while True:
        st.launch()
        d = st.status()
        if d["stop"] != 0:
            break
    t = time.perf_counter() - t0
    st.close()
    return t, d


def bench_batched(seed):
    """512 independent problems (I_n ~ U{10..64}, R ~ U{3..12}, mode-1
    collinearity 0.8, SNR 30 dB, float32 tensors) run to their stop rule
    (relative error change < 1e-8, max 1000 trials) by one graph-captured
    persistent launch with the autotuned tile / queue order; against the
    plain float64 form run problem by problem on a sample."""
    import numpy as np
    import torch
    from paper_1205_2584_gb300 import autotune, synth
    from paper_1205_2584_gb300 import cpdgn as cp
    specs = synth.config4_specs(seed, 512)
    probs = [synth.config4_problem(s, dtype="f32") for s in specs]
    b = cp.Batch([(p.Y, p.init, None) for p in probs], tol=1e-8, max_iter=1000)
    cfg = autotune.tune_batch(b, trials=2, cache=False)
    order = None if cfg["order"] == "given" else "cost"
    g = b.capture(tile=cfg["tile"], order=order, ctas=cfg["ctas"])
    times = []
    for rep in range(3):
        b.reset()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    t = statistics.median(times)
    st = b.statuses()
    iters = sum(x["iters"] for x in st)
    stops = {}
    for x in st:
        stops[x["stop_reason"]] = stops.get(x["stop_reason"], 0) + 1
    # plain float64 form, one problem at a time, on a sample
    rng = np.random.default_rng(seed)
    sample = rng.choice(512, size=8, replace=False)
    t64, it64 = 0.0, 0
    for k in sample:
        p64 = synth.config4_problem(specs[k], dtype="f64")
        shape = cp.make_shape(p64.Y.shape, p64.R, "f64")
        Y = cp.tensor_to_device(p64.Y, "f64")
        dt, d = _ttf_state(cp, shape, Y, p64.init, cp.CP_CORE_F64, tol=1e-8)
        t64 += dt
        it64 += d["iters"]
    per64 = t64 / len(sample)
    # final epsilon of sampled problems against the oracle's run to the same
    # stop rule on the same float32 values
    from oracle import cp_oracle as O
    errs = []
    for k in sample[:4]:
        ref = O.lm_fit(probs[k].Y, probs[k].init, mu0=None, max_iter=1000, tol=1e-8)
        errs.append(abs(st[k]["rel_err"] - ref.rel_err) / ref.rel_err)
    return {"oracle_final_eps_rel_err": {"max": max(errs), "sample": [int(k) for k in sample[:4]]},
            "workload": "512 problems, I_n~U{10..64}, R~U{3..12}, mode-1 collinearity 0.8, snr30, f32",
            "value": iters / t, "unit": "iters/s", "seconds_all_512": t, "problems_per_s": 512 / t,
            "trials_total": iters, "stops": stops, "tile": cfg["tile"], "order": cfg["order"], "ctas": cfg["ctas"], "tuner_timings_ms": cfg["timings"],
            "graph": "one captured persistent launch",
            "fp64_form": {"iters_per_s": it64 / t64, "seconds_per_problem": per64,
                          "sample": f"{len(sample)} problems run one at a time (float64 tensor, float64 core)"},
            "iters_per_s_gain": (iters / t) / (it64 / t64),
            "time_to_fit_gain": per64 * 512 / t}


def bench_served(seed, seconds, rate, slots=4):
    """Poisson request stream (70 % 32^3 R=5, 25 % 128^3 R=16, 5 % 400^3
    R=30; float32 tensors; stop at relative error change < 1e-8) served by
    the continuous-batching loop in real time."""
    import torch
    from paper_1205_2584_gb300 import serve as S
    from paper_1205_2584_gb300 import cpdgn as cp
    budget = 64 << 30
    srv = S.Server(hbm_budget=budget, arena_bytes=8 << 30, large_slots=slots, tol=1e-8, max_iter=1000)
    classes = [((32, 32, 32), 5), ((128, 128, 128), 16), ((400, 400, 400), 30)]
    warm = [S.Request(rid=-1 - k, arrival=0.0, dims=d, R=R, seed=12345 + k, collinearity=0.5)
            for k, (d, R) in enumerate(classes)]
    srv.serve(warm, realtime=False)           # module load, one State per large shape
    reqs = S.poisson_requests(seed, rate, seconds)
    t0 = time.perf_counter()
    res = srv.serve(reqs, realtime=True)
    wall = time.perf_counter() - t0
    out = {"workload": f"Poisson {rate:g} req/s over {seconds:g} s: 70% 32^3 R5, 25% 128^3 R16, "
                       f"5% 400^3 R30, collinearity U[0,0.95], snr30, f32",
           "offered": len(reqs), **S.summarize(res, wall), "wall_s": wall,
           "hbm_budget_gb": budget / 2 ** 30, "peak_admitted_gb": srv.peak_bytes / 2 ** 30,
           "large_slots": slots,
           "lane_rounds": [ln.rounds for ln in srv.lanes], "state_rounds": srv.large_rounds}
    # the same request alone, mixed form vs plain float64 form, per class
    alone = {}
    for k, (d, R) in enumerate(classes):
        req = S.Request(rid=0, arrival=0.0, dims=d, R=R, seed=777 + k, collinearity=0.5)
        t32 = time.perf_counter()
        r = srv.serve([req], realtime=False)[0]
        t32 = time.perf_counter() - t32
        y64, a64 = S.synth_on_device(req, srv.device, torch.float64)
        if r.path == "lane":              # lanes run on the float32 values
            y64 = y64.float().double()
        elif S.two_plane_ok(d, R):        # a State request ran on the hi + lo values
            y2 = cp.tensor_split(y64.float())
            y64 = y2[:y64.numel()].double() + y2[y64.numel():].double()
        dt, d64 = _ttf_state(cp, cp.make_shape(d, R, "f64"), y64, a64, cp.CP_CORE_F64, tol=1e-8)
        entry = {"mixed_s": t32, "mixed_iters": r.status["iters"], "f64_s": dt, "f64_iters": d64["iters"],
                 "gain": dt / t32}
        if d[0] <= 128:            # the oracle's run to the same stop rule on the same values
            from oracle import cp_oracle as O
            Yh = y64.cpu().numpy().reshape(d, order="F")
            A0 = [x.numpy().copy() for x in cp.split_factors(a64.cpu(), d, R)]
            ref = O.lm_fit(Yh, A0, mu0=None, max_iter=1000, tol=1e-8)
            entry["oracle_final_eps_rel_err"] = abs(r.status["rel_err"] - ref.rel_err) / ref.rel_err
        alone["x".join(map(str, d)) + f"-R{R}"] = entry
        del y64, a64
    out["alone_vs_fp64_form"] = alone
    srv.close()
    return out


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle
# ---------------------------------------------------------------------------

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import cp_oracle as O
    from paper_1205_2584_gb300 import synth
    prob = synth.config2(args.seed, DIMS, dtype="f32")
    # warm-up iterations, then K timed LM iterations continuing from there
    w = O.lm_fit(prob.Y, prob.init, mu0=None, max_iter=max(1, args.warmup), tol=0.0)
    t0 = time.perf_counter()
    r = O.lm_fit(prob.Y, w.A, mu0=w.mu, max_iter=args.steps, tol=0.0)
    total = time.perf_counter() - t0
    times = [0.0] * r.iters
    value = r.iters / total
    out = {"metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": WORKLOAD, "dims": list(DIMS), "R": R,
                      "tensor_dtype": "f32 (the float32 tensor values in float64, f64 math)"},
           "cpu_baseline": {"value": value, "unit": "iters/s", "cores": oracle_threads(), "kind": "oracle",
                            "sample": f"{len(times)} consecutive LM iterations from the seeded start"},
           "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.profile:
        run_profile(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
