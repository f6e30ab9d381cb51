"""Training data, training loop and evaluation of the QLA surrogate.

Data: plain-QLA trajectories computed on the GPU by qla_step, on periodic
lattices with the local statistics of the 1024^2 scattering workload
(delta 0.05, 1-3 tanh-edged ellipses with n_i in [1, 3] and 4-cell edges, a
pulse of random polarisation with sigma in [20, 60] cells). One snapshot is
kept every K steps; consecutive snapshots are the (input, target) pairs.
Training: Adam with a cosine learning-rate schedule on random batches of
pairs, every step through qla_surrogate_train_step. Evaluation: a rollout of
the surrogate (with its energy check and QLA fallback) against plain QLA on
the same lattice, relative L2 error, energy drift and time per K steps.
"""
from __future__ import annotations

import math
import os
import time
from typing import Dict, List, Optional

import numpy as np

from . import media
from .qla import Simulation
from .surrogate import Surrogate


def training_workload(rng: np.random.Generator, Nx: int = 512, Ny: int = 256, delta: float = 0.05,
                      steps: int = 1024) -> media.Workload:
    """One random training lattice: objects fully inside it, pulse clear of its x-boundary."""
    nobj = int(rng.integers(1, 4))
    objs = []
    for _ in range(nobj):
        a = float(rng.uniform(0.05, 0.25)) * Ny
        b = float(rng.uniform(0.05, 0.25)) * Ny
        r = max(a, b) + 8.0
        cx = float(rng.uniform(r, Nx - r))
        cy = float(rng.uniform(r, Ny - r))
        ang = float(rng.uniform(0.0, math.pi))
        n = tuple(float(v) for v in rng.uniform(1.0, 3.0, size=3))
        objs.append(media.Ellipse(cx, cy, a, b, ang, n, 4.0))
    pol = int(rng.integers(0, 2))
    sigma = float(rng.uniform(20.0, 60.0))
    lo, hi = 3.0 * sigma, Nx - 3.0 * sigma - delta * steps
    x0 = float(rng.uniform(lo, max(lo, hi)))
    return media.Workload(f"train_{Nx}x{Ny}", Nx, Ny, delta, steps, objs, media.Pulse(pol, x0, sigma, 1.0))


def _pol_name(pol: int) -> str:
    return "Ez" if pol == media.POL_EZ else "Ey"


def generate(workloads: List[media.Workload], K: int = 16, snapshots: Optional[int] = None) -> Dict:
    """Run plain QLA on each workload; keep (snapshots + 1) states K steps apart.

    Returns torch tensors on the GPU: q [n_traj][T+1][6][Ny][Nx], n [n_traj][3][Ny][Nx]."""
    import torch

    Ny, Nx = workloads[0].Ny, workloads[0].Nx
    T = snapshots if snapshots is not None else workloads[0].steps // K
    q = torch.empty((len(workloads), T + 1, 6, Ny, Nx), dtype=torch.float32, device="cuda")
    nf = torch.empty((len(workloads), 3, Ny, Nx), dtype=torch.float32, device="cuda")
    for i, w in enumerate(workloads):
        n = w.medium()
        nf[i] = torch.as_tensor(np.stack(n), dtype=torch.float32)
        with Simulation(*n, w.delta) as sim:
            sim.init_pulse(_pol_name(w.pulse.pol), w.pulse.x0, w.pulse.sigma, w.pulse.amp)
            for j in range(T + 1):
                if j:
                    sim.step(K)
                with torch.cuda.stream(sim.stream):
                    q[i, j].copy_(sim.state_tensor())
            sim.synchronize()
    torch.cuda.synchronize()
    return {"q": q, "n": nf, "K": K}


def train(sur: Surrogate, data: Dict, iters: int, lr: float = 1e-3, lr_min: float = 1e-5, warmup: int = 50,
          seed: int = 0, log_every: int = 100, time_limit: Optional[float] = None, noise: float = 0.0) -> List:
    """Adam steps on random batches of consecutive-snapshot pairs. Returns [(iter, loss)].

    noise > 0 perturbs each input state by Gaussian noise of that standard
    deviation relative to the batch RMS, keeping the target: the network then
    also learns to pull a slightly wrong state back toward the trajectory,
    which is what it meets in a rollout."""
    import torch

    q, nf = data["q"], data["n"]
    n_traj, T = q.shape[0], q.shape[1] - 1
    B = sur.nimg
    rng = np.random.default_rng(seed)
    q_in = torch.empty((B,) + tuple(q.shape[2:]), dtype=torch.float32, device="cuda")
    q_t = torch.empty_like(q_in)
    nb = torch.empty((B,) + tuple(nf.shape[1:]), dtype=torch.float32, device="cuda")
    hist = []
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    t0 = time.perf_counter()
    for it in range(iters):
        ti = torch.as_tensor(rng.integers(0, n_traj, B), device="cuda")
        tj = torch.as_tensor(rng.integers(0, T, B), device="cuda")
        q_in.copy_(q[ti, tj])
        q_t.copy_(q[ti, tj + 1])
        nb.copy_(nf[ti])
        if noise > 0.0:
            rms = q_in.square().mean().sqrt()
            q_in.add_(torch.randn(q_in.shape, device="cuda", generator=gen) * (noise * rms))
        if it < warmup:
            lr_it = lr * (it + 1) / warmup
        else:
            u = (it - warmup) / max(1, iters - warmup)
            lr_it = lr_min + 0.5 * (lr - lr_min) * (1.0 + math.cos(math.pi * u))
        want = (it % log_every == 0) or it == iters - 1
        loss = sur.train_step(q_in, nb, q_t, lr_it, want_loss=want)
        if want:
            hist.append((it, loss))
            if time_limit is not None and time.perf_counter() - t0 > time_limit:
                break
    sur.synchronize()
    return hist


def evaluate(sur: Surrogate, w: media.Workload, calls: int, drift_tol: float = 1e-3, checkpoints: int = 1,
             drift_mode: int = 0) -> Dict:
    """Rollout of `calls` surrogate calls (K steps each) against plain QLA.

    The rollout is split into `checkpoints` equal segments so that the error
    can be followed in time (a per-call energy check does not depend on the
    split; a check from the start keeps the initial energy as reference)."""
    import torch

    K = sur.K
    n = w.medium()
    nf = torch.as_tensor(np.stack(n), dtype=torch.float32, device="cuda").contiguous()
    pol = _pol_name(w.pulse.pol)
    seg = max(1, calls // checkpoints)
    out = {"calls": calls, "K": K, "steps": calls * K, "lattice": [w.Nx, w.Ny], "curve": []}
    with Simulation(*n, w.delta) as ref, Simulation(*n, w.delta) as sim:
        ref.init_pulse(pol, w.pulse.x0, w.pulse.sigma, w.pulse.amp)
        sim.init_pulse(pol, w.pulse.x0, w.pulse.sigma, w.pulse.amp)
        q0 = ref.get_fields(np.float32).astype(np.float64)
        e_ref = ref.energy()
        stats_tot = {"surrogate_calls": 0, "fallback_calls": 0, "max_drift": 0.0}
        t_sur = 0.0
        done = 0
        while done < calls:
            c = min(seg, calls - done)
            t0 = time.perf_counter()
            st = sur.rollout(sim, nf, c, drift_tol, drift_mode=drift_mode, energy_ref=e_ref)
            t_sur += time.perf_counter() - t0
            ref.step(c * K)
            done += c
            for k in ("surrogate_calls", "fallback_calls"):
                stats_tot[k] += st[k]
            stats_tot["max_drift"] = max(stats_tot["max_drift"], st["max_drift"])
            qr = ref.get_fields(np.float32).astype(np.float64)
            qs = sim.get_fields(np.float32).astype(np.float64)
            rel = float(np.linalg.norm(qs - qr) / np.linalg.norm(qr))
            persist = float(np.linalg.norm(q0 - qr) / np.linalg.norm(qr))
            out["curve"].append({"steps": done * K, "rollout_seconds": t_sur, "rel_l2": rel, "rel_l2_no_update": persist,
                                 "energy_drift": abs(sim.energy() / e_ref - 1.0),
                                 "qla_energy_drift": abs(ref.energy() / e_ref - 1.0),
                                 "fallbacks": stats_tot["fallback_calls"]})
        out.update(stats_tot)
        out["rel_l2"] = out["curve"][-1]["rel_l2"]
        out["rel_l2_no_update"] = out["curve"][-1]["rel_l2_no_update"]
        out["energy_drift"] = out["curve"][-1]["energy_drift"]
        out["qla_energy_drift"] = out["curve"][-1]["qla_energy_drift"]
        out["rollout_seconds"] = t_sur
        # wall time of plain QLA for the same number of steps (as the rollout's)
        ref.synchronize()
        t0 = time.perf_counter()
        ref.step(calls * K)
        ref.synchronize()
        out["qla_seconds"] = time.perf_counter() - t0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        # device time of the network alone (one call)
        qa = torch.as_tensor(qr, dtype=torch.float32, device="cuda")
        qb = torch.empty_like(qa)
        sur.forward(qa, nf, qb)
        e0.record(sur.stream)
        reps = 10
        for _ in range(reps):
            sur.forward(qa, nf, qb)
        e1.record(sur.stream)
        e1.synchronize()
        out["forward_seconds_per_call"] = e0.elapsed_time(e1) / 1e3 / reps
    out["qla_seconds_per_K"] = out["qla_seconds"] / calls
    out["speedup_rollout"] = out["qla_seconds"] / t_sur
    out["speedup_forward"] = out["qla_seconds_per_K"] / out["forward_seconds_per_call"]
    # horizon within the error bound, and the rollout's speedup over it
    tol = 1e-2
    horizon = 0
    for c in out["curve"]:
        if c["rel_l2"] > tol:
            break
        horizon = c["steps"]
    out["horizon_steps_rel_l2_1e-2"] = horizon
    out["speedup_at_rel_l2_1e-2"] = out["speedup_at_rel_l2_1e-2_serial"] = None
    if horizon:
        # the horizon advanced as one rollout from the initial state (the curve
        # above is taken in short segments, each of which restarts the
        # pipeline and synchronises twice), speculative and serial
        t_h = {}
        for serial in (False, True):
            with Simulation(*n, w.delta) as sim2:
                sim2.init_pulse(pol, w.pulse.x0, w.pulse.sigma, w.pulse.amp)
                sim2.synchronize()
                t0 = time.perf_counter()
                sur.rollout(sim2, nf, horizon // K, drift_tol, drift_mode=drift_mode, energy_ref=e_ref,
                            serial=serial)
                t_h[serial] = time.perf_counter() - t0
        out["speedup_at_rel_l2_1e-2"] = out["qla_seconds_per_K"] * (horizon // K) / t_h[False]
        out["speedup_at_rel_l2_1e-2_serial"] = out["qla_seconds_per_K"] * (horizon // K) / t_h[True]
    return out


DEFAULT_CHECKPOINT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "checkpoints", "surrogate_k16.npz")


def save_checkpoint(path: str, params, meta: Dict) -> None:
    import json

    np.savez_compressed(path, params=np.asarray(params, dtype=np.float32), meta=json.dumps(meta))


def load_checkpoint(path: str):
    import json

    z = np.load(path, allow_pickle=False)
    return z["params"], json.loads(str(z["meta"]))


def main(argv=None):
    """Generate plain-QLA trajectories, train the surrogate on the GPU and save a checkpoint."""
    import argparse
    import json

    import torch

    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--out", required=True)
    ap.add_argument("--trajectories", type=int, default=64)
    ap.add_argument("--steps", type=int, default=1024, help="QLA steps per trajectory")
    ap.add_argument("--nx", type=int, default=512)
    ap.add_argument("--ny", type=int, default=256)
    ap.add_argument("--iters", type=int, default=20000)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--noise", type=float, default=0.0)
    ap.add_argument("--seed", type=int, default=100)
    ap.add_argument("--init", default=None, help="start from this checkpoint")
    ap.add_argument("--K", type=int, default=16, help="QLA steps per surrogate call")
    a = ap.parse_args(argv)
    K = a.K
    # output scale K/256 (1/16 at K = 16): a checkpoint trained for K steps,
    # loaded for 2K steps, starts from twice its per-call update
    out_scale = K / 256.0
    rng = np.random.default_rng(a.seed)
    t0 = time.perf_counter()
    wl = [training_workload(rng, a.nx, a.ny, 0.05, a.steps) for _ in range(a.trajectories)]
    data = generate(wl, K)
    t1 = time.perf_counter()
    with Surrogate(a.ny, a.nx, nimg=a.batch, K=K, out_scale=out_scale, train=True, seed=a.seed) as sur:
        if a.init:
            sur.set_params(load_checkpoint(a.init)[0])
        hist = train(sur, data, a.iters, lr=a.lr, log_every=max(1, a.iters // 40), seed=a.seed, noise=a.noise)
        params = sur.get_params()
    t2 = time.perf_counter()
    meta = {"K": K, "out_scale": out_scale, "trajectories": a.trajectories, "steps": a.steps, "lattice": [a.nx, a.ny],
            "delta": 0.05, "iters": a.iters, "batch": a.batch, "lr": a.lr, "noise": a.noise, "seed": a.seed,
            "init": a.init, "final_loss": hist[-1][1], "data_seconds": t1 - t0, "train_seconds": t2 - t1,
            "gpu": torch.cuda.get_device_name()}
    save_checkpoint(a.out, params, meta)
    print(json.dumps({"meta": meta, "loss": hist}))


if __name__ == "__main__":
    main()
