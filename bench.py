#!/usr/bin/env python
"""Benchmark of the buoyancy-driven-cavity step on GB300.

Headline workload: the 128^3 cavity at Ra 1e5, Pr 0.71, initial T linear in
x plus U(-1e-3, 1e-3) noise (seed 0), split on one GPU into 2x2x2 blocks that
exchange ghost faces every step, FP64.  One bench step = one explicit step
of the whole hot path: fused residual + update with residual /
spectral-radius reductions, wall conditions + finalise (dt, centre pressure,
Nusselt), face pack and unpack.  Metric: grid-point updates per second
(interior nodes x steps / time), whole job.  The same line carries the
FP32-mixed form of the same workload and of the 256^3, Ra 1e6 cavity as
"variants".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--precision fp64|fp32] [--workload cfg2|cfg3] [--no-variants]

Under torchrun every rank advances its own independent cavity (replicas; the
step has no data-path collective); rank 0 prints one JSON line.
The reference arm times the FP64 CPU oracle on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "grid-point updates/s per step"
UNIT = "point-updates/s"
# FP64 operations per interior point of the fused FP64 step (adds, multiplies,
# compares = 1, FMA = 2, sqrt = 1), counted on the kernel's formulation: rates
# 144 (beta^2 7, dissipation weights 15, fourth differences 18, dissipation 5,
# divergence 8, continuity 2, advection-diffusion weights 24, u 16, v 17, w 17,
# T 13, buoyancy 2), update 11, residual sums 10, spectral radius of the new
# state 25
FP64_FLOP_PER_POINT = 190
# algorithmic HBM bytes per interior point-update of one fused pass: every
# stored array read once and written once (FP64: 5 x 8 B; FP32-mixed: 7 x 4 B,
# u, v, w and the hi/lo pairs of p and T)
BYTES_PER_POINT = {"fp64": 80, "fp32": 56}
# algorithmic HBM bytes per interior point of one launch of the adjoint's
# dominant kernel (the reverse of the rates, FP32 sweep): read the stored
# FP32-mixed state (7 x 4 B) and the adjoint of the state after the step
# (5 x 4 B), write the adjoint of the state before it (5 x 4 B)
ADJ_BYTES_PER_POINT = 68
# DRAM bytes (read + write) per launch of the dominant kernel from one ncu
# capture of the same workload and kernel shape, kept with the capture's
# summary; None where no capture of the current kernel exists.  Key:
# (precision, workload, blocks, shape); the FP32 shape is the autotuner's
# "TY,KC,R,form"
FP64_SHAPE = "32x4x8"
TRAFFIC = {("fp64", "cfg2", (2, 2, 2), FP64_SHAPE): 115.065344e6 + 55.689216e6,
           ("fp32", "cfg3", (1, 1, 1), "8,96,4,3"): 613.445632e6 + 434.552064e6,
           ("fp32", "cfg3", (1, 1, 1), "8,64,4,3"): 575.716096e6 + 435.488256e6,
           ("fp32", "cfg3", (1, 1, 1), "8,32,4,3"): 585.227776e6 + 434.474240e6,
           ("fp32", "cfg4", None, "8,64,4,3"): 612.079360e6 + 324.579072e6}
F32_FORMS = {3: "k_step_f32q (two nodes per thread, f32x2; z neighbours below the plane in registers)"}
# FP64 peak derived from the unit counts: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
L2_BYTES = 129e6
# the paper's timed single-GPU size (Section 4.6, Tables 3-4): 256^3 at Ra 1e5, FP64
CAVITY256_FP64 = dict(name="cavity256_ra1e5_fp64", n=(256, 256, 256), Ra=1e5, Pr=0.71, noise=1e-3, seed=0)
WORKLOADS = {"cfg2": workloads.CFG2, "cfg3": workloads.CFG3, "cav256": CAVITY256_FP64}


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "fp32"], default="fp64")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="cfg2")
    ap.add_argument("--blocks", default=None, help="px,py,pz (default 2,2,2 for cfg2, 1,1,1 for cfg3)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    return ap.parse_args(argv)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.lines: list[str] = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = max(smax, float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(values, world: int, device: str) -> list[float]:
    """Each of `values` maximised over the ranks: the slowest rank sets the
    job's time (all ranks call this; 1 rank: unchanged)."""
    if world == 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def job_value(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the (max) time."""
    return units_per_rank * world / seconds


def default_blocks(workload: str, blocks: str | None):
    if blocks:
        return tuple(int(v) for v in blocks.split(","))
    return (2, 2, 2) if workload == "cfg2" else (1, 1, 1)


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the CPU baseline."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_rate(cfg, blocks, min_seconds=10.0, max_steps=200):
    """Point-updates/s of the oracle as it stands: steps of the workload until
    about min_seconds of CPU work (threads: OMP_NUM_THREADS, default all cores)."""
    import oracle
    n = cfg["n"]
    o = oracle.OracleCavity(*n, dict(Ra=cfg["Ra"], Pr=cfg["Pr"]), blocks=blocks, noise=cfg["noise"], seed=cfg["seed"])
    o.step(1)
    t0 = time.perf_counter()
    steps = 0
    while steps < max_steps and time.perf_counter() - t0 < min_seconds:
        o.step(1)
        steps += 1
    dt = time.perf_counter() - t0
    return n[0] * n[1] * n[2] * steps / dt, steps, dt


def cpu_baseline(workload, blocks, min_seconds=10.0, max_steps=200):
    """The oracle on the host cores (all of them, OpenMP over k) on a bounded
    sample, plus the same oracle on one thread in a child process."""
    cfg = WORKLOADS[workload]
    value, steps, dt = oracle_rate(cfg, blocks, min_seconds, max_steps)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    n = cfg["n"]
    one = None
    code = ("import json, sys; sys.path.insert(0, %r); import bench, workloads; "
            "v, s, t = bench.oracle_rate(bench.WORKLOADS[%r], %r, %r, %r); "
            "print(json.dumps([v, s, t]))" % (ROOT, workload, tuple(blocks), min_seconds / 2, max_steps))
    try:
        env = dict(os.environ, OMP_NUM_THREADS="1")
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                           timeout=120 + 4 * min_seconds)
        v1, s1, t1 = json.loads(r.stdout.strip().splitlines()[-1])
        one = {"value": v1, "threads": 1, "sample": f"{s1} oracle steps ({t1:.1f} s)"}
    except (OSError, subprocess.SubprocessError, ValueError, IndexError):
        one = None
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": cpu_model(),
            "sample": f"{steps} oracle steps of the {n[0]}x{n[1]}x{n[2]} cavity in {blocks} blocks "
                      f"({dt:.1f} s, FP64, OpenMP over k on {cores} threads)",
            "one_thread": one}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    cfg = WORKLOADS[args.workload]
    n = cfg["n"]
    blocks = default_blocks(args.workload, args.blocks)
    import oracle
    o = oracle.OracleCavity(*n, dict(Ra=cfg["Ra"], Pr=cfg["Pr"]), blocks=blocks, noise=cfg["noise"], seed=cfg["seed"])
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    pts = n[0] * n[1] * n[2]
    value = pts * args.steps / dt
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded initial state; no dataset)",
        "config": {"workload": f"cavity {n[0]}^3 Ra {cfg['Ra']:g} Pr {cfg['Pr']} noise {cfg['noise']:g} seed "
                               f"{cfg['seed']}, blocks {blocks}, FP64 oracle", "blocks": list(blocks)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} timed oracle steps after {args.warmup} warm-up steps"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


_FP64_PEAK = {}


def fp64_peak(m, device: int):
    """FP64 FMA throughput of this GPU measured by the library's DFMA chains
    (cavity_measure_fp64_peak), once per process."""
    if device not in _FP64_PEAK:
        _FP64_PEAK[device] = m.cavity_measure_fp64_peak(device)
    return _FP64_PEAK[device]


def roofline_for(precision, pts, step_ms, hbm, traffic=None, form=3, fp64_measured=None):
    step_s = step_ms / 1e3
    bpp = BYTES_PER_POINT[precision]
    gbs = bpp * pts / step_s / 1e9
    hbm_obj = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": (gbs / hbm) if hbm else None,
               "bytes_per_point": bpp, "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    if precision == "fp32":
        return dict(kernel=F32_FORMS.get(form, f"FP32 step kernel form {form}") +
                    ": TMA-staged fused residual + update + partials", traffic=traffic, kernel_ms=step_ms, **hbm_obj)
    tf = FP64_FLOP_PER_POINT * pts / step_s / 1e12
    peak = fp64_measured or FP64_PEAK_TFLOPS
    return {"kernel": "k_step_f64 (fused residual + update + reductions)", "bound": "alu", "achieved": tf,
            "peak": peak, "unit": "TFLOP/s", "frac": tf / peak, "traffic": traffic,
            "peak_source": ("measured FP64 FMA throughput (cavity_measure_fp64_peak: independent DFMA chains on "
                            "every SM, of measured)" if fp64_measured else
                            "derived FP64 peak: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz"),
            "peak_derived": FP64_PEAK_TFLOPS, "frac_of_derived": tf / FP64_PEAK_TFLOPS,
            "kernel_ms": step_ms, "flop_per_point": FP64_FLOP_PER_POINT,
            "flop_per_point_note": "counted on the kernel's formulation; the oracle's plain formulation of "
                                   "Eqs. 1-3 counts about 212", "hbm_view": hbm_obj}


def measure(m, torch, precision, workload, blocks, steps, warmup, rank, world, local, stream, e2e=True,
            overlap=False):
    """Device time of `steps` steps (and optionally e2e) of one workload."""
    cfg = WORKLOADS[workload]
    n = cfg["n"]
    pts = n[0] * n[1] * n[2]
    prec = m.CAVITY_FP64 if precision == "fp64" else m.CAVITY_FP32_MIXED
    c = m.Cavity(*n, blocks=blocks, precision=prec, seed=cfg["seed"] + rank, noise_amp=cfg["noise"],
                 device=local, stream=stream.cuda_stream, Ra=cfg["Ra"], Pr=cfg["Pr"])
    nb = blocks[0] * blocks[1] * blocks[2]
    # FP64: step, walls, finalise; FP32-mixed: step, finalise; + pack, unpack when split
    launches_per_step = (3 if precision == "fp64" else 2) + (2 if nb > 1 else 0)
    if overlap:  # + the shell kernel
        m.cavity_set_overlap(c.h, True)
        launches_per_step += 1
    both_buffers = pts * BYTES_PER_POINT[precision]  # the two buffer sets of the state
    # one step reads one buffer set (half of both_buffers) and writes the
    # other, which the next step reads: flush L2 unless that set exceeds it
    flush = both_buffers / 2 < 1.2 * L2_BYTES
    scratch = torch.empty(int(2 * L2_BYTES) // 4, dtype=torch.float32, device=f"cuda:{local}") if flush else None

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    tuned = m.cavity_autotune(c.h, 20) if precision == "fp32" else None  # FP32: the autotuner picks the shape
    shape = (f"{tuned['tile_y']},{tuned['kc']},{tuned['ring']},{tuned['kernel_form']}" if tuned else FP64_SHAPE)
    c.step(warmup)
    c.sync()
    # per-kernel durations: CUDA events around every launch on the handle's
    # stream over 20 steps just before and 20 just after the timed region,
    # averaged (the FP64 step's cost drifts with the state along a run)
    kms_before = m.cavity_time_kernels(c.h, 20)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        if not flush:
            # K graph-replayed steps, inputs resident in HBM (state larger than L2)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            c.step(steps)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
        else:
            # state fits in L2: write a 2xL2 buffer before every timed step
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            with torch.cuda.stream(stream):
                for a, b in ev:
                    scratch.fill_(1.0)
                    a.record(stream)
                    c.step(1)
                    b.record(stream)
            torch.cuda.synchronize()
            ms = sum(a.elapsed_time(b) for a, b in ev)
    barrier()
    rc = c.sync()
    kms = [0.5 * (x + y) for x, y in zip(kms_before, m.cavity_time_kernels(c.h, 20))]
    ms, = max_over_ranks([ms], world, f"cuda:{local}")
    out = {"value": job_value(pts * steps, world, ms / 1e3), "ms_per_step": ms / steps, "steps": steps,
           "kernel_ms": {"step": kms[0], "bc_finalize": kms[1], "pack": kms[2], "unpack": kms[3]},
           "gpu_launches": launches_per_step * steps, "clocks": clk.summary(), "status": rc, "autotune": tuned,
           "l2": (f"L2 flushed (2 x L2 buffer written) before every timed step: a step reads one buffer set "
                  f"({both_buffers / 2e6:.0f} MB), which fits in the 129 MB L2" if flush else
                  f"no flush: a step reads one buffer set ({both_buffers / 2e6:.0f} MB), more than the 129 MB L2"),
           "roofline": roofline_for(precision, pts, kms[0], measured_peaks().get("hbm_gbs"),
                                    # the overlapped schedule's step kernel skips the shell
                                    # nodes: no capture of it
                                    None if overlap else TRAFFIC.get((precision, workload, tuple(blocks), shape)),
                                    tuned["kernel_form"] if tuned else 3,
                                    fp64_peak(m, local) if precision == "fp64" else None)}
    if e2e:
        # end to end through the public API with host buffers: initial state
        # from host; every step's residual + Nusselt record written by the
        # device into page-locked host memory (the step log) as the step
        # finishes, read on the host after the final synchronisation; final
        # fields back to host
        # the initial state and the final fields in page-locked host memory
        host0 = torch.empty(tuple(c.fields().shape), dtype=torch.float64, pin_memory=True).numpy()
        c.fields(out=host0)
        host1 = torch.empty(host0.shape, dtype=torch.float64, pin_memory=True).numpy()
        e2e_steps = max(1, min(steps, 500))
        log = m.StepLog(e2e_steps)
        m.cavity_set_step_log(c.h, log)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c.set_fields(host0)
        c.step(e2e_steps)
        res = c.fields(out=host1)  # synchronises: every record is in host memory
        recs = log.array.copy()
        t1 = time.perf_counter()
        barrier()
        m.cavity_set_step_log(c.h, None)
        log.close()
        steps_seen = np.sort(recs["step"])
        assert np.all(np.diff(steps_seen) == 1) and np.all(recs["flags"] == 0), "step log incomplete"
        e2e_s = t1 - t0
        e2e_s, = max_over_ranks([e2e_s], world, f"cuda:{local}")
        out["e2e"] = {"value": job_value(pts * e2e_steps, world, e2e_s), "unit": UNIT, "steps": e2e_steps,
                      "h2d_bytes_per_step": host0.nbytes / e2e_steps,
                      "d2h_bytes_per_step": res.nbytes / e2e_steps + m.STEP_RECORD.itemsize,
                      "per_step_result": "residual norms, Nusselt numbers, time and dt of every step, written "
                                         "by the device to page-locked host memory (step log)"}
    c.close()
    return out


def measure_batch(m, torch, steps, warmup, rank, world, local, stream):
    """The batched form: 64 cavities of uneven sizes and Ra (configuration 4),
    FP32-mixed, tile shape chosen by the autotuner, graph-replayed steps."""
    cavs = workloads.batch_cavities()
    sizes = [c["n"] for c in cavs]
    params = [m.cavity_default_params(Ra=c["Ra"], Pr=workloads.CFG4["Pr"]) for c in cavs]
    h = m.cavity_create_batch(sizes, params, precision=m.CAVITY_FP32_MIXED, seeds=[c["seed"] + 1000 * rank for c in cavs],
                              noise_amp=workloads.CFG4["noise"], device=local, stream=stream.cuda_stream)
    pts = sum(a * b * c for a, b, c in sizes)
    both_buffers = pts * BYTES_PER_POINT["fp32"]
    tuned = m.cavity_autotune(h, 20)
    m.cavity_step(h, warmup)
    m.cavity_sync(h)
    kms_before = m.cavity_time_kernels(h, 10)  # averaged with 10 steps after the timed region
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        m.cavity_step(h, steps)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    rc = m.cavity_sync(h)
    kms = [0.5 * (x + y) for x, y in zip(kms_before, m.cavity_time_kernels(h, 10))]
    ms, = max_over_ranks([ms], world, f"cuda:{local}")
    m.cavity_destroy(h)
    return {"value": job_value(pts * steps, world, ms / 1e3), "ms_per_step": ms / steps, "steps": steps,
            "kernel_ms": {"step": kms[0], "bc_finalize": kms[1], "pack": kms[2], "unpack": kms[3]},
            "gpu_launches": 2 * steps, "clocks": clk.summary(), "status": rc, "autotune": tuned,
            "roofline": roofline_for("fp32", pts, kms[0], measured_peaks().get("hbm_gbs"),
                                     TRAFFIC.get(("fp32", "cfg4", None, f"{tuned['tile_y']},{tuned['kc']},"
                                                  f"{tuned['ring']},{tuned['kernel_form']}")),
                                     tuned["kernel_form"]),
            "config": {"workload": f"batch of {len(cavs)} cavities, n_d in [24, 96], Ra log-uniform in [1e3, 1e6], "
                                   f"{pts} interior points, FP32-mixed, one graph launch per step",
                       "l2": (f"no flush: a step reads one buffer set ({both_buffers / 2e6:.0f} MB), more than "
                              f"the 129 MB L2" if both_buffers / 2 > 1.2 * L2_BYTES else
                              "state smaller than L2: not flushed")},
            "dtype": "f32 (p as f32 hi/lo pair, f64 reductions)"}


def measure_adjoint(m, torch, rank, world, local, stream):
    """Configuration 5: gradient of the mean hot-wall Nusselt number over 500
    FP32-mixed steps of a 128^3 cavity w.r.t. the 128x128 hot-wall temperature
    field and Ra, checkpoints every 50 steps.  Wall time of the checkpointed
    forward run and of the reverse sweep (segment recomputation + FP32
    adjoint kernels with FP64 reductions), through the public API."""
    cfg = workloads.CFG5
    n = cfg["n"]
    pts = n[0] * n[1] * n[2]
    theta = workloads.wall_temperature(n[1], n[2], seed=cfg["theta_seed"], sigma=cfg["theta_sigma"])
    c = m.Cavity(*n, precision=m.CAVITY_FP32_MIXED, seed=cfg["seed"] + rank, noise_amp=cfg["noise"], device=local,
                 stream=stream.cuda_stream, Ra=cfg["Ra"], Pr=cfg["Pr"])
    m.cavity_set_wall_temperature(c.h, 0, theta)
    tuned = m.cavity_autotune(c.h, 20)  # the FP32 step's tile shape (forward and recomputation)
    # warm-up with the timed run's own step count and checkpoint interval, so
    # that the timed run reuses the checkpoint and segment memory
    m.cavity_adjoint_forward(c.h, cfg["steps"], cfg["ckpt"])
    m.cavity_adjoint_backward(c.h, n[1], n[2])
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        J = m.cavity_adjoint_forward(c.h, cfg["steps"], cfg["ckpt"])
        t1 = time.perf_counter()
        g, gra = m.cavity_adjoint_backward(c.h, n[1], n[2])
        t2 = time.perf_counter()
    rc = c.sync()
    gather_ms = m.cavity_adjoint_kernel_ms(c.h)
    c.close()
    fwd, bwd = t1 - t0, t2 - t1
    fwd, bwd = max_over_ranks([fwd, bwd], world, f"cuda:{local}")
    steps = cfg["steps"]
    hbm = measured_peaks().get("hbm_gbs")
    gbs = ADJ_BYTES_PER_POINT * pts / (gather_ms / 1e3) / 1e9
    return {"metric": "gradient point-steps/s (forward + reverse sweep)", "value": job_value(pts * steps, world, fwd + bwd),
            "unit": "point-steps/s", "steps": steps, "checkpoint_every": cfg["ckpt"],
            "forward_ms_per_step": 1e3 * fwd / steps, "backward_ms_per_step": 1e3 * bwd / steps,
            "J": J, "dJ_dRa": gra, "grad_wall_norm": float(np.linalg.norm(g)), "clocks": clk.summary(), "status": rc,
            "autotune": tuned,
            "roofline": {"kernel": "k_adj_gather (reverse of the rates, FP32 gather form)", "bound": "hbm",
                         "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm if hbm else None,
                         "traffic": None, "kernel_ms": gather_ms, "bytes_per_point": ADJ_BYTES_PER_POINT,
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"},
            "config": {"workload": f"adjoint of {steps} steps, cavity {n[0]}^3 Ra {cfg['Ra']:g}, FP32-mixed forward, "
                                   f"FP32 reverse sweep (FP64 reductions), checkpoints every {cfg['ckpt']}"},
            "dtype": "f32 forward (p, T as f32 pairs), f32 adjoint sweep with f64 reductions"}


def summary(line) -> dict:
    """One short entry per measured workload (value, time per step, roofline
    fraction), printed last so that a truncated tail of the line still shows
    every workload."""
    out = {}
    for name, v in [("headline", line)] + list(line.get("variants", {}).items()):
        r = v.get("roofline") or {}
        out[name] = {"value": v.get("value"), "ms_per_step": v.get("ms_per_step", v.get("backward_ms_per_step")),
                     "bound": r.get("bound"), "frac": r.get("frac"), "kernel_ms": r.get("kernel_ms")}
    return out


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import paper_2006_02602_gb300 as m
    m.load_library()
    stream = torch.cuda.Stream(device=local)

    cfg = WORKLOADS[args.workload]
    n = cfg["n"]
    blocks = default_blocks(args.workload, args.blocks)
    r = measure(m, torch, args.precision, args.workload, blocks, args.steps, args.warmup, rank, world, local, stream)
    dtype = "f64" if args.precision == "fp64" else "f32 (p as f32 hi/lo pair, f64 reductions)"
    line = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": dtype, "data": "synthetic (seeded initial state; no dataset)",
        "config": {"workload": f"cavity {n[0]}^3 Ra {cfg['Ra']:g} Pr {cfg['Pr']} noise {cfg['noise']:g}, "
                               f"blocks {blocks}, {args.precision.upper()}, all hot-path rows per step",
                   "blocks": list(blocks), "parallelism": f"replicas x{world}", "l2": r["l2"]},
        "kernel_ms": r["kernel_ms"], "e2e": r["e2e"], "gpu_launches": r["gpu_launches"],
        "roofline": r["roofline"], "clocks": r["clocks"], "status": r["status"],
    }
    if r.get("autotune"):
        line["autotune"] = r["autotune"]
    if not args.no_variants and args.workload == "cfg2" and args.precision == "fp64":
        variants = {}
        for name, prec, wl, blk, steps in (("fp32_mixed_cfg2", "fp32", "cfg2", (2, 2, 2), min(args.steps, 500)),
                                           ("fp32_mixed_cfg3", "fp32", "cfg3", (1, 1, 1), min(args.steps, 500))):
            v = measure(m, torch, prec, wl, blk, steps, args.warmup, rank, world, local, stream, e2e=False)
            wcfg = WORKLOADS[wl]
            v["config"] = {"workload": f"cavity {wcfg['n'][0]}^3 Ra {wcfg['Ra']:g} blocks {blk} FP32-mixed",
                           "l2": v.pop("l2")}
            v["dtype"] = "f32 (p as f32 hi/lo pair, f64 reductions)"
            variants[name] = v
        v = measure(m, torch, "fp64", "cfg2", (2, 2, 2), min(args.steps, 1000), args.warmup, rank, world, local,
                    stream, e2e=False, overlap=True)
        v["config"] = {"workload": "cavity 128^3 Ra 1e+05 blocks (2, 2, 2) FP64, interior/shell split: shell nodes "
                                   "first, pack/unpack on a second stream while the interior is stepped",
                       "l2": v.pop("l2")}
        v["dtype"] = "f64"
        v["kernel_ms_note"] = "kernel_ms from the plain (non-overlapped) launch sequence"
        variants["fp64_cfg2_overlap"] = v
        v = measure(m, torch, "fp64", "cav256", (1, 1, 1), min(args.steps, 200), args.warmup, rank, world, local,
                    stream, e2e=False)
        v["config"] = {"workload": "cavity 256^3 Ra 1e+05 one block FP64: the paper's timed single-GPU size "
                                   "(Section 4.6, Tables 3-4)", "l2": v.pop("l2")}
        v["dtype"] = "f64"
        variants["fp64_cavity256"] = v
        variants["batch64_fp32"] = measure_batch(m, torch, min(args.steps, 500), args.warmup, rank, world, local,
                                                 stream)
        variants["adjoint_cfg5"] = measure_adjoint(m, torch, rank, world, local, stream)
        line["variants"] = variants
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload, blocks)
    if "variants" in line:
        line["summary"] = summary(line)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
