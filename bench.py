"""Benchmark: QLA site-update throughput on the 8192^2 three-cylinder workload.

A bench step = 100 QLA time steps (qla_step(100): fused passes of
steps_per_pass steps) followed by one diagnostics reduction (energy Eq. 27,
div B), i.e. one diagnostics interval of the workload. Inputs (the 1.6 GB FP32
state) are far larger than the 129 MB L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 (torchrun) every rank runs its own replica of the workload (the
lattices are independent: weak scaling, no data-path collective); value is the
sum of site-updates over ranks divided by the slowest rank's time.
--impl reference times the FP64 CPU oracle on the host cores on a bounded
window of the same workload (rank 0 only).
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# DRAM bytes per sweep launch (dram__bytes_read.sum + dram__bytes_write.sum) from an ncu capture
# (one pass) of two sweep launches of this benchmark's own command on the 8192^2 workload (its
# summary sits in profiles/ beside the launch list), valid while the sweep's code (comment lines
# excluded), the workload, the steps per pass and the launch form (balanced split, one launch per
# pass or all passes of a bench step in one persistent launch) match.
MEASURED_TRAFFIC = {"sweep_sha256_prefix": "677c90822e6ffdd2", "workload": "cylinders8192_fp32",
                    "steps_per_pass": 2, "chunk_rows": 0, "launch": "per_pass", "bytes_per_launch": 7.77284e9}

L2_BYTES = 129e6  # GB300 L2
METRIC = "site-updates/s per QLA step"
UNIT = "site-updates/s"
BYTES_PER_SITE_UPDATE = 60.0  # FP32 general kernel: 24 B state read + 24 B write + 12 B n_x, n_y, n_z
QLA_STEPS_PER_BENCH_STEP = 100
E2E_CONTEXTS = 3  # contexts in flight in the pipelined e2e leg


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.rows = []
        self.proc = None
        self.th = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.dev)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.th:
            self.th.join(timeout=2)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[0]) for r in self.rows if num(r[0]) is not None]
        mx = [num(r[1]) for r in self.rows if num(r[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[4 + k].strip() == "Active"})
        pw = [num(r[2]) for r in self.rows if num(r[2]) is not None]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows), "power_w_max": max(pw) if pw else None}


def sweep_code_hash() -> str:
    """sha256 prefix of the per-pass sweep kernel's sources (the kernel, its
    instantiations and launch split, the shared declarations) with their
    comment lines removed."""
    import hashlib

    code = []
    for name in ("qla_sweep.cuh", "qla_sweep_f32.cu", "qla_internal.h"):
        with open(os.path.join(ROOT, "paper_2301_13601_gb300", "csrc", name)) as f:
            code += [l for l in f.read().splitlines() if not l.lstrip().startswith("//")]
    return hashlib.sha256("\n".join(code).encode()).hexdigest()[:16]


def job_throughput(units: float, elapsed_ms: float, world: int, device=None):
    """Whole-job throughput over ranks: units summed over ranks divided by the
    slowest rank's elapsed time (the job ends when its last rank does).
    Returns (units per second, max elapsed ms). world == 1 needs no process group."""
    if world == 1:
        return units / (elapsed_ms / 1e3), elapsed_ms
    import torch
    import torch.distributed as dist

    t = torch.tensor([elapsed_ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / (float(t.item()) / 1e3), float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def cpu_baseline(seconds: float = 12.0, impl_steps: int = 0):
    """FP64 oracle on a bounded 1024^2 window of the workload (host cores)."""
    import oracle
    from paper_2301_13601_gb300 import media

    w = media.workload_cylinders_8192()
    N = 1024
    # window around the pulse and the first cylinder edge, taken as its own periodic lattice
    obj = min(w.objects, key=lambda o: o.cx)
    y0 = int(max(0, min(w.Ny - N, obj.cy - N // 2)))
    x0 = int(max(0, min(w.Nx - N, w.pulse.x0 - 256)))
    objs =[media.Ellipse(o.cx - x0, o.cy - y0, o.a, o.b, o.angle, o.n, o.w) for o in w.objects]
    nx, ny, nz = media.medium(N, N, objs)
    theta, beta = oracle.angles(nx, ny, nz, w.delta)
    q = oracle.init_pulse(N, N, w.pulse.pol, w.pulse.x0 - x0, w.pulse.sigma, w.pulse.amp)
    steps = 0
    t0 = time.perf_counter()
    chunk = 5
    while True:
        oracle.run(q, theta, beta, chunk)
        steps += chunk
        el = time.perf_counter() - t0
        if (impl_steps and steps >= impl_steps) or (not impl_steps and el >= seconds):
            break
    rate = N * N * steps / el
    return {"value": rate, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
            "sample": f"FP64 oracle, {N}x{N} window of the 8192^2 workload (pulse + cylinder), "
                      f"{steps} QLA steps, {el:.1f} s"}, el, N * N * steps


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2301_13601_gb300 import media

    w = media.workload_cylinders_8192()
    N, S = 1024, 10
    objs = [media.Ellipse(o.cx - 768, o.cy - 3584, o.a, o.b, o.angle, o.n, o.w) for o in w.objects]
    nx, ny, nz = media.medium(N, N, objs)
    theta, beta = oracle.angles(nx, ny, nz, w.delta)
    q = oracle.init_pulse(N, N, w.pulse.pol, 256.0, w.pulse.sigma, w.pulse.amp)
    for _ in range(args.warmup):
        oracle.run(q, theta, beta, S)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.run(q, theta, beta, S)
        oracle.energy(q)
        oracle.divB(q)
    el = time.perf_counter() - t0
    value = N * N * S * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "cylinders8192 (1024x1024 window)", "lattice": f"{N}x{N}", "delta": w.delta,
                       "qla_steps_per_bench_step": S, "precision": "fp64", "sequence": "interleaved",
                       "potential": "paper"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
                             "sample": f"{N}x{N} window, {S} QLA steps + diagnostics per bench step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2301_13601_gb300 import build as _build
    from paper_2301_13601_gb300 import media
    from paper_2301_13601_gb300.qla import Simulation

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    _build.build()
    w = {"cylinders8192": media.workload_cylinders_8192, "ellipse2048": media.workload_ellipse_2048,
         "cylinder256": media.workload_cylinder_256,
         "cylinders4096": lambda: media.workload_cylinders_8192(N=4096)}[args.workload]()
    n = w.medium()
    S = QLA_STEPS_PER_BENCH_STEP
    sim = Simulation(*n, w.delta, precision="fp32", steps_per_pass=args.steps_per_pass,
                     chunk_rows=args.chunk_rows, launch=args.launch)
    sim.init_pulse("Ez" if w.pulse.pol == media.POL_EZ else "Ey", w.pulse.x0, w.pulse.sigma, w.pulse.amp)
    stream = sim.stream
    sites = w.Nx * w.Ny

    def bench_step():
        sim.step(S)
        return sim.diagnostics()

    for _ in range(args.warmup):
        bench_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    e_begin = torch.cuda.Event(enable_timing=True)
    e_end = torch.cuda.Event(enable_timing=True)
    sweep_ms = 0.0
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    e_begin.record(stream)
    last = None
    for i in range(args.steps):
        ev[i][0].record(stream)
        sim.step(S)
        ev[i][1].record(stream)
        last = sim.diagnostics()
    e_end.record(stream)
    torch.cuda.synchronize()
    clocks.stop()
    total_ms = e_begin.elapsed_time(e_end)
    sweep_ms = sum(a.elapsed_time(b) for a, b in ev)
    value, total_ms = job_throughput(sites * S * args.steps, total_ms, world, device="cuda")
    if world > 1:
        dist.barrier()
    # one launch per pass, or every pass of a bench step in one persistent launch
    launch_form = sim.launch
    launches_per_step = 1 if launch_form == "persistent" else math.ceil(S / sim.steps_per_pass)
    # e2e through the public API with host buffers: pinned H2D state copy,
    # qla_step, diagnostics, D2H state copy, every bench step. Serial: one
    # context, each step's copies between its compute. Pipelined (the reported
    # value): E2E_CONTEXTS contexts on their own streams, each stepping its own
    # lattice of the workload, bench step i on context i mod E2E_CONTEXTS, so
    # that the host copies of one step overlap the compute of the others
    # (qla_set_fields_f32 and qla_step are asynchronous on the context's
    # stream; diagnostics and the read-back synchronise it) and a read-back
    # that the host stalls in (measured on GB300: now and then 25-70 ms for
    # the usual 8 ms) is covered by the steps queued behind it. The sweeps of
    # the contexts run one after the other (events order them): each pass of
    # the balanced split is one wave of CTAs sized for the whole GPU, so two
    # passes sharing the SMs would both run long.
    e2e_value = e2e_serial = h2d_gbs = d2h_gbs = None
    if not args.skip_extras:
        host = [torch.empty((6, w.Ny, w.Nx), dtype=torch.float32, pin_memory=True) for _ in range(2)]
        sim.get_fields_host_f32(host[0].data_ptr())
        host[1].copy_(host[0])
        e2e_steps = max(2, min(args.steps, 8))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            sim.set_fields_host_f32(host[0].data_ptr())
            sim.step(S)
            sim.diagnostics()
            sim.get_fields_host_f32(host[0].data_ptr())
        e2e_serial = sites * S * e2e_steps * world / (time.perf_counter() - t0)
        # the host copies alone (what the pipelined leg hides behind compute)
        t0 = time.perf_counter()
        for _ in range(3):
            sim.set_fields_host_f32(host[0].data_ptr())
            sim.synchronize()
        h2d_gbs = 3 * 24 * sites / (time.perf_counter() - t0) / 1e9
        t0 = time.perf_counter()
        for _ in range(3):
            sim.get_fields_host_f32(host[0].data_ptr())
        d2h_gbs = 3 * 24 * sites / (time.perf_counter() - t0) / 1e9
        sims = [sim] + [Simulation(*n, w.delta, precision="fp32", steps_per_pass=args.steps_per_pass,
                                   chunk_rows=args.chunk_rows, launch=args.launch) for _ in range(E2E_CONTEXTS - 1)]
        P = len(sims)
        host += [torch.empty_like(host[0], pin_memory=True) for _ in range(P - len(host))]
        for k in range(1, P):
            host[k].copy_(host[0])
            sims[k].set_fields_host_f32(host[k].data_ptr())
            sims[k].step(S)
            sims[k].diagnostics()
        torch.cuda.synchronize()
        done = [torch.cuda.Event() for _ in range(P)]
        nsteps = P * e2e_steps
        t0 = time.perf_counter()
        for i in range(nsteps + P - 1):
            if i < nsteps:  # queue bench step i: upload, then sweep after step i - 1's sweeps
                c = sims[i % P]
                c.set_fields_host_f32(host[i % P].data_ptr())
                if i > 0:
                    c.stream.wait_event(done[(i - 1) % P])
                c.step(S)
                done[i % P].record(c.stream)
            j = i - (P - 1)  # read back the oldest step in flight
            if j >= 0:
                d = sims[j % P]
                d.diagnostics()
                d.get_fields_host_f32(host[j % P].data_ptr())
        e2e_value = sites * S * nsteps * world / (time.perf_counter() - t0)
        for c in sims[1:]:
            c.close()
    sim.close()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    peak, peak_kind = measured_peaks()
    k = sim.steps_per_pass
    sha = sweep_code_hash()
    traffic = None
    if (sha == MEASURED_TRAFFIC["sweep_sha256_prefix"] and w.name == MEASURED_TRAFFIC["workload"]
            and k == MEASURED_TRAFFIC["steps_per_pass"] and sim.chunk_rows == MEASURED_TRAFFIC["chunk_rows"]
            and launch_form == MEASURED_TRAFFIC["launch"]):
        traffic = MEASURED_TRAFFIC["bytes_per_launch"]
    launch_ms = sweep_ms / (args.steps * launches_per_step)
    steps_per_launch = S / launches_per_step
    achieved = BYTES_PER_SITE_UPDATE * sites * steps_per_launch / (launch_ms / 1e3) / 1e9
    cb = None if args.skip_extras else cpu_baseline(seconds=args.cpu_seconds)[0]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "lattice": f"{w.Nx}x{w.Ny}", "delta": w.delta,
                   "qla_steps_per_bench_step": S, "steps_per_pass": k, "chunk_rows": sim.chunk_rows,
                   "launch": launch_form,
                   "precision": "fp32", "sequence": "interleaved", "potential": "paper",
                   "l2": (f"inputs {'larger' if 80 * sites > L2_BYTES else 'smaller'} than L2 (state "
                          f"{24 * sites / 1e9:.2f} GB + coefficients {56 * sites / 1e9:.2f} GB read per pass)"),
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "kernel": (f"sweep_persistent_kernel<float,{k}> ({S // k} passes per launch)"
                                if launch_form == "persistent" else f"sweep_kernel<float,{k}>"),
                     "bytes_per_site_update": BYTES_PER_SITE_UPDATE,
                     "note": "algorithmic bytes of the unfused step x steps per launch"},
        "cpu_baseline": cb,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 6 * sites * 4,
                "d2h_bytes_per_step": 6 * sites * 4 + 40, "serial_value": e2e_serial,
                "h2d_gbs_alone": h2d_gbs, "d2h_gbs_alone": d2h_gbs,
                "note": "public C ABI with pinned host buffers; every bench step uploads its state, runs "
                        "100 QLA steps + diagnostics and downloads the state; three contexts in flight (the copies "
                        "of one step overlap the compute of the others); serial_value: one context, copies in "
                        "line; *_gbs_alone: the host copies timed alone"},
        "clocks": clocks.summary(),
        "gpu_launches": args.steps * (launches_per_step + 2),
        "energy_last": last["energy"] if last else None,
    }
    if not args.skip_extras:
        line["single_family"] = single_family_report(w, args, peak, peak_kind)
        # the other polarisation: the same lattice and pulse, E_y instead of E_z
        line["single_family_other"] = single_family_report(w, args, peak, peak_kind, other=True)
        line["batch"] = batch_report(args, peak, peak_kind)
    if not args.skip_extras and not args.skip_surrogate:
        line["surrogate"] = surrogate_report()
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def single_family_report(w, args, peak, peak_kind, steps: int = 5, other: bool = False):
    """The same workload with only the pulse's polarisation family stored and
    advanced (qla_options.families): the other family's three components are
    zero at the start and stay exactly zero under every operator, so the result
    is the same state (bit for bit, tested) for half the work. Its algorithmic
    bytes per site-update are those of the family's kernel (TM: 24 B of state +
    4 B of n_z; TE: 24 B + 8 B of n_x, n_y). other: the pulse of the other
    polarisation (same position, width and amplitude) and its family."""
    import torch

    from paper_2301_13601_gb300 import media
    from paper_2301_13601_gb300.qla import Simulation

    fam, pol = ("TM", "Ez") if (w.pulse.pol == media.POL_EZ) != other else ("TE", "Ey")
    alg = 28.0 if fam == "TM" else 32.0
    S = QLA_STEPS_PER_BENCH_STEP
    with Simulation(*w.medium(), w.delta, precision="fp32", steps_per_pass=args.steps_per_pass,
                    chunk_rows=args.chunk_rows, families=fam, launch=args.launch) as sim:
        form = sim.launch
        sim.init_pulse(pol, w.pulse.x0, w.pulse.sigma, w.pulse.amp)
        sim.step(S)
        sim.diagnostics()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(sim.stream)
        for _ in range(steps):
            sim.step(S)
            sim.diagnostics()
        e1.record(sim.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
    value = w.Nx * w.Ny * S / (ms / 1e3)
    return {"families": fam, "value": value, "unit": UNIT, "ms_per_step": ms, "steps": steps, "launch": form,
            "bytes_per_site_update": alg, "bandwidth_equivalent_frac": value * alg / 1e9 / peak,
            "peak_kind": peak_kind, "note": "same bench step (100 QLA steps + diagnostics); the other family's "
            "planes are zero and stay zero (Eq. 17-22 never couple the families)"}


def batch_instances(args):
    """The 64-lattice workload (sides 256-2048, 2000-8000 steps each), every
    lattice's step count divided by --batch-step-scale (a bench step stays
    well under a second)."""
    from paper_2301_13601_gb300 import media

    ws = media.workload_batch64()
    inst = []
    for w in ws:
        steps = max(4, (w.steps // args.batch_step_scale) // 4 * 4)
        inst.append({"n": w.medium(), "delta": w.delta, "nsteps": steps,
                     "pulse": ("Ez" if w.pulse.pol == media.POL_EZ else "Ey", w.pulse.x0, w.pulse.sigma, 1.0)})
        if args.chunk_rows:
            inst[-1]["chunk_rows"] = args.chunk_rows
    return ws, inst


def batch_report(args, peak, peak_kind, steps: int = 3):
    """The batched workload in one persistent CUDA-graph launch per bench step,
    with the steps per pass and rows per tile chosen by the autotuner (timed
    candidates, cached per GPU, kernel version and batch shape)."""
    import torch

    from paper_2301_13601_gb300.qla import Batch

    ws, inst = batch_instances(args)
    t_tune = time.perf_counter()
    with Batch(inst, steps_per_pass=0) as b:
        t_tune = time.perf_counter() - t_tune
        info = b.info()
        b.run()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            b.run()
        el = time.perf_counter() - t0
        tuned = dict(b.tuned)
    value = info["site_updates"] * steps / el
    return {"workload": f"batch64: {len(inst)} lattices, sides {sorted({w.Nx for w in ws})}, "
                        f"{min(i['nsteps'] for i in inst)}-{max(i['nsteps'] for i in inst)} QLA steps each per run",
            "value": value, "unit": UNIT, "ms_per_run": 1e3 * el / steps, "runs": steps,
            "bandwidth_equivalent_frac": value * BYTES_PER_SITE_UPDATE / 1e9 / peak, "peak_kind": peak_kind,
            "steps_per_pass": info["steps_per_pass"], "chunk_rows": tuned.get("chunk_rows"),
            "autotuned": True, "autotune_seconds": t_tune, "work_items": info["work_items"],
            "launch": "one persistent kernel in a CUDA graph per run (synchronous)"}


SURROGATE_CHECKPOINT = os.path.join(ROOT, "paper_2301_13601_gb300", "checkpoints", "surrogate_k16.npz")
# the same network advancing 32 steps per call (trained from the 16-step weights)
SURROGATE_CHECKPOINT_K32 = os.path.join(ROOT, "paper_2301_13601_gb300", "checkpoints", "surrogate_k32.npz")


def surrogate_report(calls: int = 250, seed: int = 7):
    """The learned surrogate on the 1024^2 scattering workload: a rollout of
    `calls` x 16 steps (with its energy check and QLA fallback) against plain
    QLA, the error curve, the horizon within rel L2 1e-2 and the speedups, and
    the tensor-core conv kernel's throughput against the measured BF16 peak."""
    import numpy as np
    import torch

    from paper_2301_13601_gb300 import media
    from paper_2301_13601_gb300 import surrogate as S
    from paper_2301_13601_gb300 import surrogate_train as T

    if not os.path.exists(SURROGATE_CHECKPOINT):
        return {"unavailable": "no trained checkpoint"}
    params, meta = T.load_checkpoint(SURROGATE_CHECKPOINT)
    w = media.workload_surrogate_1024(seed)
    with S.Surrogate(w.Ny, w.Nx, nimg=1, K=meta["K"], out_scale=meta["out_scale"]) as sur:
        sur.set_params(params)
        r = T.evaluate(sur, w, calls, drift_tol=1e-3, checkpoints=calls // 5)
        flops = sur.info()["flops_per_call"]
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except (OSError, ValueError):
        pass
    bf16 = peaks.get("bf16_tflops") or 1900.0
    # algorithmic MACs per site of the network (first layer 9 x 9 x 64 with its 9 input channels,
    # four hidden 9 x 64 x 64, last 9 x 64 x 6); the kernels compute padded channels (16 in, 16 out)
    alg_flops = 2 * (9 * 9 * 64 + 4 * 9 * 64 * 64 + 9 * 64 * 6) * w.Nx * w.Ny
    achieved = alg_flops / r["forward_seconds_per_call"] / 1e12
    curve = [(c["steps"], round(c["rel_l2"], 5)) for c in r["curve"][4::5]]
    variants = []
    if os.path.exists(SURROGATE_CHECKPOINT_K32):
        p32, m32 = T.load_checkpoint(SURROGATE_CHECKPOINT_K32)
        calls32 = calls * meta["K"] // m32["K"]
        with S.Surrogate(w.Ny, w.Nx, nimg=1, K=m32["K"], out_scale=m32["out_scale"]) as sur:
            sur.set_params(p32)
            r32 = T.evaluate(sur, w, calls32, drift_tol=1e-3, checkpoints=calls32 // 5)
        variants.append({
            "K": m32["K"], "checkpoint": os.path.relpath(SURROGATE_CHECKPOINT_K32, ROOT),
            "trained": {k: m32[k] for k in ("trajectories", "iters", "noise", "final_loss", "train_seconds")},
            "rel_l2": r32["rel_l2"], "horizon_steps_rel_l2_1e-2": r32["horizon_steps_rel_l2_1e-2"],
            "speedup_at_rel_l2_1e-2": r32["speedup_at_rel_l2_1e-2"],
            "speedup_at_rel_l2_1e-2_serial": r32["speedup_at_rel_l2_1e-2_serial"], "speedup_rollout": r32["speedup_rollout"],
            "speedup_forward": r32["speedup_forward"], "surrogate_calls": r32["surrogate_calls"],
            "fallback_calls": r32["fallback_calls"]})
    return {
        "workload": f"surrogate1024 seed {seed}: 1024x1024, delta 0.05, {calls} calls x 16 steps",
        "checkpoint": os.path.relpath(SURROGATE_CHECKPOINT, ROOT),
        "trained": {k: meta[k] for k in ("trajectories", "steps", "lattice", "iters", "batch", "noise",
                                         "final_loss", "train_seconds")},
        "rel_l2": r["rel_l2"], "rel_l2_no_update": r["rel_l2_no_update"],
        "horizon_steps_rel_l2_1e-2": r["horizon_steps_rel_l2_1e-2"],
        "speedup_at_rel_l2_1e-2": r["speedup_at_rel_l2_1e-2"],
        "speedup_at_rel_l2_1e-2_serial": r["speedup_at_rel_l2_1e-2_serial"],
        "speedup_rollout": r["speedup_rollout"], "speedup_forward": r["speedup_forward"],
        "surrogate_calls": r["surrogate_calls"], "fallback_calls": r["fallback_calls"],
        "energy_drift": r["energy_drift"], "qla_energy_drift": r["qla_energy_drift"],
        "drift_check": "per call, |E_after/E_before - 1| <= 1e-3 (FP64 energy, Eq. 27)",
        "qla_ms_per_16_steps": 1e3 * r["qla_seconds_per_K"],
        "forward_ms_per_call": 1e3 * r["forward_seconds_per_call"],
        "rel_l2_curve": curve,
        # steps per call at which one forward costs as much as plain QLA for those steps
        "break_even_K": meta["K"] * r["forward_seconds_per_call"] / r["qla_seconds_per_K"],
        "variants": variants,
        "training_step_ms": time_training(params, meta),
        "training_batch": "4 x 512x256 (loss, full gradient on the tensor cores, Adam)",
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": bf16, "unit": "TFLOP/s",
                     "frac": achieved / bf16, "peak_kind": "measured" if peaks.get("bf16_tflops") else "fallback",
                     "kernel": "conv3x3_tc_kernel (6 layers, one forward call)",
                     "flops": "2 x algorithmic MACs: 9 x (9x64 + 4 x 64x64 + 64x6) = 156096 per site",
                     "achieved_padded": flops / r["forward_seconds_per_call"] / 1e12,
                     "flops_padded": "2 x padded MACs: 9 x (16x64 + 4 x 64x64 + 64x16) per site"},
    }


def time_training(params, meta, warmup: int = 3, steps: int = 10) -> float:
    """ms per surrogate training step (loss, full gradient and Adam on a batch
    of 4 lattices of 512x256), CUDA events on the surrogate's stream."""
    import torch

    from paper_2301_13601_gb300 import surrogate as S

    with S.Surrogate(256, 512, nimg=4, K=meta["K"], out_scale=meta["out_scale"], train=True) as tr:
        tr.set_params(params)
        qa = torch.randn((4, 6, 256, 512), device="cuda")
        na = torch.rand((4, 3, 256, 512), device="cuda") * 2 + 1
        qb = qa * 1.01
        for _ in range(warmup):
            tr.train_step(qa, na, qb, 1e-6)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(tr.stream)
        for _ in range(steps):
            tr.train_step(qa, na, qb, 1e-6)
        e1.record(tr.stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / steps


def run_surrogate(args):
    """The surrogate alone on the 1024^2 workload: forward calls (16 QLA steps
    each) on device-resident fields, and training steps (batch 4 of 512x256),
    timed with CUDA events; the conv kernel's throughput against the BF16 peak."""
    import numpy as np
    import torch

    from paper_2301_13601_gb300 import build as _build
    from paper_2301_13601_gb300 import media
    from paper_2301_13601_gb300 import surrogate as S
    from paper_2301_13601_gb300 import surrogate_train as T

    _build.build()
    params, meta = T.load_checkpoint(SURROGATE_CHECKPOINT)
    w = media.workload_surrogate_1024(7)
    n = torch.as_tensor(np.stack(w.medium()), dtype=torch.float32, device="cuda")[None].contiguous()
    q = [torch.randn((1, 6, w.Ny, w.Nx), device="cuda") * 0.5 for _ in range(2)]

    def ev():
        return torch.cuda.Event(enable_timing=True)

    with S.Surrogate(w.Ny, w.Nx, K=meta["K"], out_scale=meta["out_scale"]) as sur:
        sur.set_params(params)
        for i in range(args.warmup):
            sur.forward(q[i & 1], n, q[(i + 1) & 1])
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record(sur.stream)
        for i in range(args.steps):
            sur.forward(q[i & 1], n, q[(i + 1) & 1])
        e1.record(sur.stream)
        e1.synchronize()
        fwd_ms = e0.elapsed_time(e1) / args.steps
        flops = sur.info()["flops_per_call"]
    train_ms = time_training(params, meta, args.warmup, args.steps)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except (OSError, ValueError):
        pass
    bf16 = peaks.get("bf16_tflops") or 1900.0
    sites = w.Nx * w.Ny
    alg_flops = 2 * (9 * 9 * 64 + 4 * 9 * 64 * 64 + 9 * 64 * 6) * sites  # algorithmic MACs (see surrogate_report)
    achieved = alg_flops / (fwd_ms / 1e3) / 1e12
    line = {"metric": "QLA-equivalent site-updates/s of the surrogate forward", "value": sites * 16 / (fwd_ms / 1e3),
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": fwd_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16 (fp32 accumulate)",
            "data": "synthetic", "config": {"workload": "surrogate1024 seed 7", "lattice": "1024x1024",
                                            "steps_per_call": 16, "l2": "activations 128 MB per buffer"},
            "training_step_ms": train_ms, "training_batch": "4 x 512x256",
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": bf16, "unit": "TFLOP/s",
                         "frac": achieved / bf16, "kernel": "conv3x3_tc_kernel (6 layers per call)",
                         "flops": "2 x algorithmic MACs (156096 per site)",
                         "achieved_padded": flops / (fwd_ms / 1e3) / 1e12,
                         "peak_kind": "measured" if peaks.get("bf16_tflops") else "fallback"}}
    print(json.dumps(line), flush=True)


def run_batch(args):
    """64 lattices of uneven sizes in one persistent graph launch per bench step."""
    import torch

    from paper_2301_13601_gb300 import build as _build
    from paper_2301_13601_gb300.qla import Batch

    _build.build()
    ws, inst = batch_instances(args)
    # --steps-per-pass 0 (the default): the autotuner chooses steps per pass and tile rows
    with Batch(inst, steps_per_pass=args.steps_per_pass) as b:
        info = b.info()
        K = info["steps_per_pass"]
        tuned = b.tuned
        for _ in range(args.warmup):
            b.run()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            b.run()
        el = time.perf_counter() - t0
    value = info["site_updates"] * args.steps / el
    peak, peak_kind = measured_peaks()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch64", "lattices": len(inst), "sides": sorted({w.Nx for w in ws}),
                       "qla_steps_per_lattice": f"{min(i['nsteps'] for i in inst)}-{max(i['nsteps'] for i in inst)}",
                       "steps_per_pass": K, "chunk_rows": (tuned or {}).get("chunk_rows", args.chunk_rows),
                       "autotuned": tuned is not None, "work_items": info["work_items"],
                       "launch": "one persistent kernel in a CUDA graph"},
            "bandwidth_equivalent_frac": value * BYTES_PER_SITE_UPDATE / 1e9 / peak, "peak_kind": peak_kind}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--steps-per-pass", type=int, default=0)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--workload", choices=["cylinders8192", "cylinders4096", "ellipse2048", "cylinder256", "batch64",
                                           "surrogate1024"],
                    default="cylinders8192")
    ap.add_argument("--batch-step-scale", type=int, default=10, help="batch64: steps of each lattice divided by this")
    ap.add_argument("--chunk-rows", type=int, default=0)
    ap.add_argument("--launch", choices=["auto", "per_pass", "persistent"], default="auto",
                    help="sweep launch form: one launch per pass, or every pass of a bench step in one launch")
    ap.add_argument("--skip-extras", action="store_true", help="no e2e leg and no CPU baseline (profiling runs)")
    ap.add_argument("--skip-surrogate", action="store_true", help="no surrogate evaluation")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch64":
        run_batch(args)
    elif args.workload == "surrogate1024":
        run_surrogate(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
