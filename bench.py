"""Throughput of one design step of the diffractive-storage hot path on GB300.

A step is one forward (every channel through all K layers and K+1 gaps), the
MSE objective with per-channel PSNR and dL/dI, and the adjoint gradient
dL/dh, over a design of 4096 wavelength channels, 5 layers of 200 x 200
thickness pixels padded to 400 x 400 (the massive workload).  The metric is
lambda-channel layer-propagations per second (N_w * (K+1) per step).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank runs its own
4096-channel shard of an N*4096-channel design (weak scaling) and the
gradient shards are summed with one all-reduce.  ``--impl reference`` times
the FP64 CPU oracle on the host cores on a bounded channel sample instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# DRAM bytes (read + write) per channel of one launch of a kernel kind (the
# average over the kind's launches of a step), from ncu captures of the same
# build on the 256-channel design, keyed by (kernel family, N, M, kernel kind);
# the bench scales them to the launch's channels.  An entry must be removed
# (traffic reported as null) when its kernel changes.
TRAFFIC_PER_CHANNEL = {
    # One capture of every bulk pass of a step (dram__bytes_read + write per
    # launch / 256 channels), each kind averaged over its launches.
    # 200 -> 400, K = 5: forward column 1.3875 / 1.3875 / 1.3887 / 1.3872 MB and
    # 1.0646 MB (last gap, field-of-view output rows); adjoint column 0.9075 MB
    # (first gap, field-of-view input rows) and 1.3876 / 1.3883 / 1.3874 / 1.3904 MB;
    # forward row 0.7277 MB (first pass, from the input-field table) and 1.3579 /
    # 1.3580 / 1.3577 / 1.3583 MB; adjoint row 1.4205 / 1.4195 / 1.4215 / 1.4203 MB
    # and 0.9861 MB (layer 1: no spectra written back)
    ("column_bulk", 200, 400, "column_forward"): ((1.3875e6 + 1.3875e6 + 1.3887e6 + 1.3872e6 + 1.0646e6) / 5,
                                                  "profiles/column_pass_bulk_batched.md"),
    ("column_bulk", 200, 400, "column_adjoint"): ((0.9075e6 + 1.3876e6 + 1.3883e6 + 1.3874e6 + 1.3904e6) / 5,
                                                  "profiles/column_pass_bulk_batched.md"),
    ("row_bulk", 200, 400, "row_forward"): ((0.7277e6 + 1.3579e6 + 1.3580e6 + 1.3577e6 + 1.3583e6) / 5,
                                            "profiles/row_passes_batched.md"),
    ("row_bulk", 200, 400, "row_adjoint"): ((1.4205e6 + 1.4195e6 + 1.4215e6 + 1.4203e6 + 0.9861e6) / 5,
                                            "profiles/row_passes_batched.md"),
    # 256 -> 512, K = 8 (the precision geometry with 256 channels): forward column
    # 2.4101 / 2.4105 / 2.4089 / 2.4096 / 2.4093 / 2.4098 / 2.4090 MB and 1.7779 MB;
    # adjoint column 1.6248 MB and 2.4096 / 2.4094 / 2.4101 / 2.4092 / 2.4092 /
    # 2.4092 / 2.4098 MB; forward row 1.3346 MB and 2.3736 / 2.3727 / 2.3729 /
    # 2.3733 / 2.3738 / 2.3720 / 2.3721 MB; adjoint row 2.4562 / 2.4547 / 2.4545 /
    # 2.4558 / 2.4562 / 2.4542 / 2.4540 MB and 1.6203 MB
    ("column_bulk", 256, 512, "column_forward"): (2.33064e6, "profiles/column_pass_m512_precision.md"),
    ("column_bulk", 256, 512, "column_adjoint"): (2.31141e6, "profiles/column_pass_m512_precision.md"),
    ("row_bulk", 256, 512, "row_forward"): (2.24313e6, "profiles/row_passes_m512_precision.md"),
    ("row_bulk", 256, 512, "row_adjoint"): (2.35074e6, "profiles/row_passes_m512_precision.md"),
}


def step_bytes(n, m, K, F, nw, bin_=1):
    """Algorithmic bytes of one step (forward + loss + adjoint) of nw channels:
    'design' = what the multi-pass kernels must move (complex64 = 8 B: the
    create-time v1 table read by the first row pass, the row spectra N x M in
    and out of every pass, the checkpoints, one transfer-table quadrant per
    column pass, the field-of-view rows of the last forward / first adjoint gap,
    output, loss and seed; the per-chunk gradient partials are left out), and
    'ideal' = 40 N^2 B per layer-propagation (read v, write v_next forward;
    read a and the checkpoint, write a_prev adjoint), the traffic of a design
    that keeps the spectra on chip."""
    hs = m // 2 + 1
    det = (F // bin_) ** 2
    fwd = (8 * n * n + 8 * n * m                                   # first row pass (v1 table)
           + (K - 1) * (16 * n * m + 8 * n * n)                     # forward row passes + checkpoints
           + (K - 1) * (16 * n * m + 8 * hs * hs)                   # column passes
           + (8 * n * m + 8 * F * m + 8 * hs * hs)                  # last gap: field-of-view rows out
           + (8 * F * m + 8 * F * F + 4 * F * F))                   # output row pass: o, I
    loss = 8 * F * F + 4 * det + 4 * F * F                          # o and T in, dL/dI out
    adj = ((8 * F * F + 4 * F * F + 8 * F * m)                      # seed row pass
           + (8 * F * m + 8 * n * m + 8 * hs * hs)                  # first adjoint gap: FOV rows in
           + (K - 1) * (16 * n * m + 8 * hs * hs)                   # adjoint column passes
           + (K - 1) * (16 * n * m + 8 * n * n)                     # adjoint row passes
           + (8 * n * m + 8 * n * n))                               # layer 1: no spectra written back
    return {"design": nw * (fwd + loss + adj), "ideal": nw * (K + 1) * 40 * n * n}


def method_bytes_per_launch(kind, nw, n, K):
    """The method's algorithmic bytes credited to one launch of a kernel kind:
    16 N^2 B per forward layer-propagation (read v, write
    v_next) and 24 N^2 B per adjoint one (read a and the checkpoint, write
    a_prev), complex64; a multi-pass launch advances every channel by one
    propagation, a fused sweep through all of its gaps."""
    return {"column_forward": nw * 16 * n * n, "row_forward": nw * 16 * n * n,
            "column_adjoint": nw * 24 * n * n, "row_adjoint": nw * 24 * n * n,
            "fused_forward": nw * (K + 1) * 16 * n * n, "fused_adjoint": nw * K * 24 * n * n}.get(kind)


def kernel_family(detail, kind):
    """Which kernel of a multi-pass kind ran ('column_bulk' / 'column_plain',
    'row_bulk' / 'row_plain'), from the configuration name dos_describe prints
    (multipass, multipass:bulk or multipass:bulk[col+row_fwd+...])."""
    name = detail.split("|")[0].strip().split()[0].removeprefix("path=")
    if not name.startswith("multipass"):
        return None
    tag = {"column_forward": "col", "column_adjoint": "col", "row_forward": "row_fwd",
           "row_adjoint": "row_adj"}.get(kind)
    if tag is None:
        return None
    bulk = name == "multipass:bulk" or (name.startswith("multipass:bulk[") and tag in name[15:].rstrip("]").split("+"))
    return ("column_" if kind.startswith("column") else "row_") + ("bulk" if bulk else "plain")


METRIC = "lambda-channel layer-propagations/s (fwd+adjoint, 4096 lambda)"
UNIT = "propagations/s"
WORKLOAD = "massive"


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=40)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default=WORKLOAD)
    p.add_argument("--n-lambda", type=int, default=0,
                   help="channels of the workload (0: its own count); smaller designs for profiling")
    p.add_argument("--path", default="auto")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-split", action="store_true", help="skip the split-BF16 DFT-GEMM comparison")
    return p.parse_args()


def _workload(name, rank, world, n_lambda=0):
    from paper_2604_02624_gb300 import sharding
    from paper_2604_02624_gb300 import workloads as W
    w = W.workload(name, n_lambda=n_lambda) if n_lambda else W.workload(name)
    if world > 1:
        # weak scaling: the design holds world * N_w channels, rank r owns one shard
        nw = w.n_lambda
        big = W.workload(name, n_lambda=nw * world) if name in ("batched", "massive", "precision") else w
        lo, hi = sharding.shard_range(big.n_lambda, rank, world)
        w = big.subset(np.arange(lo, hi))
    return w


def _config(w, world):
    return {"workload": f"{w.name}: {w.n_lambda} lambda x {w.n_layers} layers, {w.n}x{w.n} "
                        f"padded to {w.m}x{w.m}, FOV {w.fov}x{w.fov}",
            "n_lambda_per_gpu": int(w.n_lambda), "n_layers": int(w.n_layers), "n": int(w.n),
            "m": int(w.m), "fov": int(w.fov), "n_lambda_total": int(w.n_lambda * world),
            "l2": "inputs larger than L2 (row spectra and checkpoints are several GB)",
            "parallelism": f"lambda-shard x{world}" if world > 1 else "single GPU"}


# ----------------------------------------------------------------- oracle timing
# The FP64 oracle (as it stands) on the host cores: one process per core
# (spawn, so no worker inherits a CUDA context), each running whole channels
# (forward + MSE + adjoint) on one thread; numpy's FFT is single-threaded.
_ORACLE = {}


def _oracle_init(name, h, T):
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    sys.path.insert(0, ROOT)
    from paper_2604_02624_gb300 import workloads as W
    _ORACLE.update(w=W.workload(name), h=h, T=T)


def _oracle_channel(i):
    from oracle import dos_oracle as O
    w = _ORACLE["w"].subset([i])
    O.loss_and_grad(_ORACLE["h"], _ORACLE["T"][i:i + 1], lambdas=w.lambdas, gaps=w.gaps, pitch=w.pitch,
                    m=w.m, fov=w.fov, aperture=w.aperture, n_index=w.n_index, kappa=w.kappa)
    return i


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OraclePool:
    """A pool of oracle workers, one per host core, started once."""

    def __init__(self, w, h, T, cores=None):
        import multiprocessing as mp
        self.cores = cores or host_cores()
        self.w = w
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_oracle_init, initargs=(w.name, h, T))
        self.next = 0
        self.pool.map(_oracle_channel, [0] * self.cores)   # workers up and warm

    def sample(self, seconds):
        """Whole channels on every core until ``seconds`` of wall time; returns
        (propagations/s, channels, seconds)."""
        done = 0
        t0 = time.perf_counter()
        while True:
            idx = [((self.next + j) * 997) % self.w.n_lambda for j in range(self.cores)]
            self.next += self.cores
            self.pool.map(_oracle_channel, idx, chunksize=1)
            done += len(idx)
            el = time.perf_counter() - t0
            if el >= seconds:
                break
        return done * (self.w.n_layers + 1) / el, done, el

    def close(self):
        self.pool.close()
        self.pool.join()


# ----------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ----------------------------------------------------------------- reference arm
def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return 0
    from paper_2604_02624_gb300 import workloads as W
    w = _workload(a.workload, 0, 1, a.n_lambda)
    h = W.thickness(w, 0)
    T = W.targets(w, 1)
    pool = OraclePool(w, h, T)
    per_step = max(1.0, a.cpu_seconds / max(1, a.steps + a.warmup))
    for _ in range(a.warmup):
        pool.sample(0.0)
    vals, chans, secs = [], 0, 0.0
    for _ in range(a.steps):
        v, c, s = pool.sample(per_step)
        vals.append(v)
        chans += c
        secs += s
    pool.close()
    value = chans * (w.n_layers + 1) / secs
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * secs / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(w, 1),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
                             "sample": f"{chans} whole channels (fwd + MSE + adjoint, FP64) of the "
                                       f"{w.n_lambda}-channel design, one process per host core"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- our arm
def run_ours(a):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_2604_02624_gb300 import workloads as W
    from paper_2604_02624_gb300 import _lib as L
    from paper_2604_02624_gb300.api import DiffractiveStack

    w = _workload(a.workload, rank, world, a.n_lambda)
    h_np = W.thickness(w, 0)
    T_np = W.targets(w, 1)
    stack = DiffractiveStack.from_workload(w, device=dev, n_lambda_total=w.n_lambda * world,
                                           path=a.path)
    h = torch.tensor(h_np, dtype=torch.float32, device=dev)
    T = torch.tensor(T_np, dtype=torch.float32, device=dev)
    I = torch.empty((w.n_lambda, w.fov, w.fov), dtype=torch.float32, device=dev)
    g = torch.empty_like(h)
    stream = torch.cuda.current_stream(dev)
    launches = [0]

    def step():
        stack.forward(h, out=I)
        n1 = stack.last_launch_count
        _, psnr, dLdI = stack.loss(T, read=False)
        n2 = stack.last_launch_count
        stack.backward(dLdI, out=g)
        n3 = stack.last_launch_count
        if dist is not None:
            dist.all_reduce(g)
        launches[0] += n1 + n2 + n3

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    launches[0] = 0
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    # the timed region: no per-kernel events in it
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    timed_launches = launches[0]
    # a second pass of the same steps with CUDA events around every kernel
    # (on the library's stream) gives each kernel kind's launch duration
    L.dos_set_timing(stack.handle, True)
    for _ in range(a.steps):
        step()
    torch.cuda.synchronize()
    kernel = {}
    for kind, name in enumerate(L.KERNEL_KINDS):
        n, t = L.dos_kernel_time(stack.handle, kind)
        kernel[name] = (n, t)
    L.dos_set_timing(stack.handle, False)
    clk = clocks.stop()
    if dist is not None:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    ms_step = ms / a.steps
    units_per_step = w.n_lambda * (w.n_layers + 1) * world
    value = units_per_step / (ms_step * 1e-3)

    # ---- roofline of the dominant kernel (live CUDA-event times above)
    import json as _json
    peaks = {}
    try:
        peaks = _json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    dom = max(kernel, key=lambda k: kernel[k][1])
    n_l, t_l = kernel[dom]
    per_launch_ms = t_l / max(1, n_l)
    nw, n, m, K, F, hs = w.n_lambda, w.n, w.m, w.n_layers, w.fov, w.m // 2 + 1
    # Algorithmic bytes of the method (complex64 = 8 B): 16 N^2 per forward
    # layer-propagation (read v, write v_next) and 24 N^2 per adjoint one (read
    # a and the checkpoint, write a_prev).  A multi-pass launch advances every
    # channel by one propagation and is credited that propagation's bytes; a
    # fused sweep advances every channel through all its gaps.
    method = method_bytes_per_launch(dom, nw, n, K)
    # what the multi-pass design itself must move per launch (every channel once)
    algo = {
        # the last forward column pass writes, and the adjoint's first reads,
        # only the F field-of-view rows
        "column_forward": nw * ((K - 1) * (16 * n * m + 8 * hs * hs) + (8 * F * m + 8 * n * m + 8 * hs * hs)) / K,
        "column_adjoint": nw * ((K - 1) * (16 * n * m + 8 * hs * hs) + (8 * F * m + 8 * n * m + 8 * hs * hs)) / K,
        # the first forward row pass reads the v1 table (N x N) instead of
        # spectra; layer 1's adjoint row pass writes no spectra back
        "row_forward": nw * ((K - 1) * (16 * n * m + 8 * n * n) + (8 * n * n + 8 * n * m)) / K,
        "row_adjoint": nw * ((K - 1) * (16 * n * m + 8 * n * n) + (8 * n * m + 8 * n * n)) / K,
        # fused sweeps: checkpoints, transfer table, output field / seed
        "fused_forward": nw * (8 * K * n * n + 8 * hs * hs + 12 * F * F),
        "fused_adjoint": nw * (8 * K * n * n + 8 * hs * hs + 12 * F * F),
    }.get(dom)
    # algorithmic FP32 flops of a line DFT of M points: 5 M log2 M (radix-2 count);
    # a layer-propagation runs 2N row and 2M column line DFTs
    line = 5.0 * m * np.log2(m)
    flops = {"fused_forward": nw * (K + 1) * (2 * n + 2 * m) * line,
             "fused_adjoint": nw * K * (2 * n + 2 * m) * line}.get(dom)
    fp32_peak = 152 * 128 * 2 * 2.07e9 / 1e12   # SMs x FP32 lanes x 2 flop/FMA x max SM clock
    roof = None
    if flops:
        ach = flops / (per_launch_ms * 1e-3) / 1e12
        hbm = method / (per_launch_ms * 1e-3) / 1e9
        roof = {"bound": "alu", "kernel": dom, "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": ach / fp32_peak, "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz",
                "traffic": None, "algorithmic_flops_per_launch": flops,
                "hbm_achieved_gbs": hbm, "hbm_frac_of_measured": hbm / hbm_peak,
                "algorithmic_bytes_per_launch": method, "design_bytes_per_launch": algo,
                "ms_per_launch": per_launch_ms, "launches": n_l}
    elif algo:
        ach = method / (per_launch_ms * 1e-3) / 1e9
        tr = TRAFFIC_PER_CHANNEL.get((kernel_family(L.dos_describe(stack.handle), dom), w.n, w.m, dom))
        design = algo / (per_launch_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach / hbm_peak, "peak_source": peak_src,
                "traffic": tr[0] * nw if tr else None,
                "traffic_source": tr[1] if tr else None,
                "algorithmic_bytes_per_launch": method,
                "algorithmic_bytes_note": "16 N^2 B per forward, 24 N^2 B per adjoint layer-propagation, "
                                          "x the launch's channels",
                "design_bytes_per_launch": algo, "design_gbs": design, "design_frac": design / hbm_peak,
                "ms_per_launch": per_launch_ms, "launches": n_l,
                "timing": "kernel durations from a second pass of the same steps with CUDA events on the "
                          "library's stream; the headline time has no per-kernel events"}
        # the multi-pass kernels are also measured against the FP32 ALU peak (the
        # column pass is bound by its line-DFT arithmetic): 2 line DFTs per line
        # (5 M log2 M each) and the 6-flop complex multiply per point
        lines = {"column_forward": m, "column_adjoint": m, "row_forward": n, "row_adjoint": n}.get(dom)
        if lines:
            fl = nw * lines * (2 * line + 6 * m)
            roof["alu_achieved_tflops"] = fl / (per_launch_ms * 1e-3) / 1e12
            roof["alu_frac_of_derived_peak"] = roof["alu_achieved_tflops"] / fp32_peak
            roof["algorithmic_flops_per_launch"] = fl
    kernel_share = {k: {"launches": v[0], "ms": v[1], "share": v[1] / max(1e-9, sum(x[1] for x in kernel.values()))}
                    for k, v in kernel.items() if v[0]}

    # ---- the same step replayed as one CUDA graph (dos_step)
    graph_ms = None
    for _ in range(2):
        stack.step(h, T, grad_out=g, intensity_out=I)
    torch.cuda.synchronize()
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    for _ in range(a.steps):
        stack.step(h, T, grad_out=g, intensity_out=I)
    g1.record(stream)
    torch.cuda.synchronize()
    graph_ms = g0.elapsed_time(g1) / a.steps

    # ---- end to end through the public API with pinned host buffers
    e2e = None
    if not a.no_e2e:
        h_host = torch.tensor(h_np, dtype=torch.float32).pin_memory()
        T_host = torch.tensor(T_np, dtype=torch.float32).pin_memory()
        g_host = torch.empty(h.shape, dtype=torch.float32).pin_memory()
        loss_host = torch.empty(1, dtype=torch.float64).pin_memory()
        h_dev = torch.empty_like(h)
        T_dev = torch.empty_like(T)
        # the targets (the step's large input) are uploaded on a copy stream
        # while the forward pass runs; the loss waits for them, and the next
        # upload waits until this step's loss has read them
        main = torch.cuda.current_stream()
        copy_stream = torch.cuda.Stream()
        t_ready, t_free = torch.cuda.Event(), torch.cuda.Event()

        def e2e_step():
            h_dev.copy_(h_host, non_blocking=True)
            with torch.cuda.stream(copy_stream):
                copy_stream.wait_event(t_free)
                T_dev.copy_(T_host, non_blocking=True)
                t_ready.record(copy_stream)
            stack.forward(h_dev, out=I)
            main.wait_event(t_ready)
            _, _, dLdI = stack.loss(T_dev, read=False)
            t_free.record(main)
            stack.backward(dLdI, out=g)
            if dist is not None:
                dist.all_reduce(g)
            g_host.copy_(g, non_blocking=True)
            loss_host[0] = stack.read_loss()   # waits for the step

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        k2 = max(3, a.steps // 2)
        t0 = time.perf_counter()
        for _ in range(k2):
            e2e_step()
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        e2e = {"value": units_per_step * k2 / el, "unit": UNIT,
               "h2d_bytes_per_step": int(h_host.numel() * 4 + T_host.numel() * 4),
               "d2h_bytes_per_step": int(g_host.numel() * 4 + 8)}

    path_name = stack.path
    path_detail = L.dos_describe(stack.handle)
    # ---- split-BF16 DFT-GEMM form vs the FP32 path, on the precision workload
    split = None
    if rank == 0 and not a.no_split and world == 1:
        stack.close()
        split = _split_compare(dev, L, DiffractiveStack, W)

    cpu = None
    if rank == 0 and not a.no_cpu_baseline:
        pool = OraclePool(w, h_np, T_np)
        v, c, s = pool.sample(a.cpu_seconds)
        pool.close()
        cpu = {"value": v, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
               "sample": f"{c} whole channels (fwd + MSE + adjoint, FP64) of the {w.n_lambda}-channel "
                         f"design in {s:.1f} s, one process per host core"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": _config(w, world), "path": path_name,
            "path_detail": path_detail, "roofline": roof,
            "kernels": kernel_share, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": timed_launches, "clocks": clk,
            "graph_step": {"ms_per_step": graph_ms, "value": units_per_step / (graph_ms * 1e-3),
                           "note": "forward + loss + backward replayed as one CUDA graph (dos_step)"}}
    sb = step_bytes(w.n, w.m, w.n_layers, w.fov, w.n_lambda, getattr(w, "detector_bin", 1) or 1)
    line["step_traffic"] = {
        "design_bytes_per_step": sb["design"] * world, "ideal_bytes_per_step": sb["ideal"] * world,
        "design_gbs": sb["design"] / (ms_step * 1e-3) / 1e9,
        "design_frac_of_measured_hbm": sb["design"] / (ms_step * 1e-3) / 1e9 / hbm_peak,
        "ideal_gbs": sb["ideal"] / (ms_step * 1e-3) / 1e9,
        "ideal_frac_of_measured_hbm": sb["ideal"] / (ms_step * 1e-3) / 1e9 / hbm_peak,
        "note": "whole step on one GPU: the multi-pass kernels' design bytes, and the method's algorithmic "
                "40 N^2 B per layer-propagation (16 forward + 24 adjoint)"}
    line["split_bf16"] = split
    if rank == 0:
        print(json.dumps(line), flush=True)
    stack.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def _split_compare(dev, L, DiffractiveStack, W):
    """Speed and deviation of the split-BF16 tensor-core DFT-GEMM path against
    the FP32 path on the same GPU (precision workload: 4096 lambda, K = 8,
    256 -> 512).  Errors against the FP64 oracle are measured by the tests."""
    import torch
    w = W.workload("precision")
    h = torch.tensor(W.thickness(w, 0), dtype=torch.float32, device=dev)
    T = torch.tensor(W.targets(w, 1), dtype=torch.float32, device=dev)
    res = {}
    outs = {}
    for path in ("auto", "dft_gemm", "dft_gemm_x3"):
        st = DiffractiveStack.from_workload(w, device=dev, path=path)
        for _ in range(1):
            st.forward(h)
            _, _, dl = st.loss(T, read=False)
            st.backward(dl)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        reps = 2
        e0.record()
        for _ in range(reps):
            I = st.forward(h)
            _, _, dl = st.loss(T, read=False)
            g = st.backward(dl)
        e1.record()
        torch.cuda.synchronize()
        res[path] = {"ms_per_step": e0.elapsed_time(e1) / reps, "detail": L.dos_describe(st.handle)[:120]}
        outs[path] = (I.double(), g.double())
        st.close()
    dI = float(torch.linalg.vector_norm(outs["dft_gemm"][0] - outs["auto"][0]) / torch.linalg.vector_norm(outs["auto"][0]))
    dg = float(torch.linalg.vector_norm(outs["dft_gemm"][1] - outs["auto"][1]) / torch.linalg.vector_norm(outs["auto"][1]))
    # tensor-core work of the step: per propagation four real GEMMs of the padded
    # DFT matrices (rows x K) against the channels' data, three bf16 terms each
    pad = lambda v, q: (v + q - 1) // q * q
    n, m = w.n, w.m
    rp1, kp1, rp2, kp2 = pad(2 * m, 256), pad(2 * n, 64), pad(2 * n, 256), pad(2 * m, 64)
    per_channel = rp1 * n * kp1 + rp1 * m * kp1 + rp2 * m * kp2 + rp2 * n * kp2
    flops = 2.0 * 3 * (2 * w.n_layers + 1) * w.n_lambda * per_channel
    tf = flops / (res["dft_gemm"]["ms_per_step"] * 1e-3) / 1e12
    tf3 = 2 * flops / (res["dft_gemm_x3"]["ms_per_step"] * 1e-3) / 1e12  # six products instead of three
    peaks = {}
    try:
        import json as _json
        peaks = _json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    peak = peaks.get("bf16_tflops_sustained", 1700.0)
    return {"workload": "precision: 4096 lambda x 8 layers, 256x256 padded to 512x512",
            "fp32_path": res["auto"], "split_bf16_dft_gemm": res["dft_gemm"],
            "split_bf16_x3_dft_gemm": dict(res["dft_gemm_x3"], rel_l2_intensity_vs_fp32=float(
                torch.linalg.vector_norm(outs["dft_gemm_x3"][0] - outs["auto"][0]) / torch.linalg.vector_norm(outs["auto"][0]))),
            "speedup_vs_fp32": res["auto"]["ms_per_step"] / res["dft_gemm"]["ms_per_step"],
            "rel_l2_intensity_vs_fp32": dI, "rel_l2_gradient_vs_fp32": dg,
            "tensor": {"gemm_flops_per_step": flops, "achieved_tflops_whole_path": tf,
                       "peak_tflops": peak, "peak_source": "measured sustained bf16" if peaks else "fallback",
                       "frac_whole_path": tf / peak,
                       "x3_gemm_flops_per_step": 2 * flops, "x3_achieved_tflops_whole_path": tf3,
                       "x3_frac_whole_path": tf3 / peak,
                       "note": "whole-path time (GEMMs and the conversion kernels between them) in the denominator"}}


def main():
    a = _args()
    if a.impl == "reference":
        return run_reference(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
