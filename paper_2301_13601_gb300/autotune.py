"""Autotuner for the fused sweep: steps per HBM pass and rows per tile.

For a lattice (single context) or a set of lattices (batch), every candidate
configuration is timed on the GPU with CUDA events after warm-up, and the
fastest is cached in a JSON file keyed by the lattice shape, the step
variant and the GPU name. The cache lives in $QLA_AUTOTUNE_CACHE or
~/.cache/qla_gb300/autotune.json.
"""
from __future__ import annotations

import json
import os
import time
from typing import Callable, Dict, Iterable, List, Optional, Sequence, Tuple

CACHE_ENV = "QLA_AUTOTUNE_CACHE"


def cache_path() -> str:
    return os.environ.get(CACHE_ENV, os.path.join(os.path.expanduser("~"), ".cache", "qla_gb300", "autotune.json"))


def load_cache(path: Optional[str] = None) -> dict:
    p = path or cache_path()
    try:
        with open(p) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: Optional[str] = None) -> None:
    p = path or cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def kernel_version() -> str:
    """sha256 prefix of the sweep kernel's source: cached choices of an older
    kernel are not reused."""
    import hashlib

    src = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc", "qla_sweep.cuh")
    try:
        with open(src, "rb") as f:
            return hashlib.sha256(f.read()).hexdigest()[:12]
    except OSError:
        return "unknown"


def single_key(Nx: int, Ny: int, precision: str, sequence: str, potential: str, gpu: str) -> str:
    return f"single/{gpu}/{kernel_version()}/{precision}/{sequence}/{potential}/{Nx}x{Ny}"


def chunk_candidates(Ny: int, K: int) -> List[int]:
    """Rows per tile to try: 0 (the balanced split: one equal-cost share of
    each family's rows per resident CTA) and a few fixed tile heights between
    16 K (warm-up at most a third) and the whole lattice."""
    out = {0}
    for h in (128, 192, 256, 320, 384, 512, 768, 1024, 2048, 4096):
        if 16 * K <= h < Ny:
            out.add(h)
    out.add(Ny)
    return sorted(out)


def pick_best(results: Iterable[Tuple[dict, float]]) -> Tuple[dict, float]:
    """Fastest (config, seconds) pair; ties keep the first."""
    best = None
    for cfg, sec in results:
        if best is None or sec < best[1]:
            best = (cfg, sec)
    if best is None:
        raise ValueError("no candidate could be timed")
    return best


def tune_single(n_x, n_y, n_z, delta: float, precision: str = "fp32", sequence: str = "interleaved",
                potential: str = "paper", ks: Sequence[int] = (1, 2, 4), steps: int = 16, repeats: int = 3,
                use_cache: bool = True, timer: Optional[Callable] = None) -> dict:
    """Time qla_step(steps) for each (steps per pass, rows per tile) candidate."""
    import torch

    from .qla import QLAError, Simulation

    Ny, Nx = n_x.shape
    gpu = torch.cuda.get_device_name()
    key = single_key(Nx, Ny, precision, sequence, potential, gpu)
    cache = load_cache() if use_cache else {}
    if key in cache:
        return cache[key]
    results = []
    for K in ks:
        for ch in chunk_candidates(Ny, K):
            try:
                sim = Simulation(n_x, n_y, n_z, delta, precision=precision, sequence=sequence, potential=potential,
                                 steps_per_pass=K, chunk_rows=ch)
            except QLAError:
                continue
            with sim:
                sim.init_pulse("Ez", Nx / 4, max(2.0, Nx / 32), 1.0)
                s = steps - steps % K or K
                sim.step(s)  # warm-up
                sim.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(sim.stream)
                for _ in range(repeats):
                    sim.step(s)
                e1.record(sim.stream)
                e1.synchronize()
                sec = e0.elapsed_time(e1) / 1e3 / (repeats * s)
            results.append(({"steps_per_pass": K, "chunk_rows": ch}, sec))
    cfg, sec = pick_best(results)
    entry = dict(cfg, seconds_per_step=sec, site_updates_per_s=Nx * Ny / sec, tuned_at=time.time())
    if use_cache:
        cache[key] = entry
        save_cache(cache)
    return entry


def tune_batch(instances: List[dict], ks: Sequence[int] = (2, 4), chunks: Sequence[int] = (256, 512, 768, 1024),
               step_scale: int = 8, use_cache: bool = True, sequence: str = "interleaved",
               potential: str = "paper") -> dict:
    """Pick steps per pass and one rows-per-tile value for a batch by timing a
    shortened copy of it (every lattice run for nsteps/step_scale steps)."""
    import torch

    from .qla import Batch

    gpu = torch.cuda.get_device_name()
    sig = ",".join(f"{ins['n'][0].shape[1]}x{ins['n'][0].shape[0]}:{ins['nsteps']}" for ins in instances)
    import hashlib

    key = (f"batch/{gpu}/{kernel_version()}/{sequence}/{potential}/"
           f"{hashlib.sha256(sig.encode()).hexdigest()[:16]}")
    cache = load_cache() if use_cache else {}
    if key in cache:
        return cache[key]
    results = []
    for K in ks:
        for ch in chunks:
            short = []
            for ins in instances:
                d = dict(ins)
                s = max(K, (ins["nsteps"] // step_scale) // K * K)
                d["nsteps"] = s
                d["chunk_rows"] = ch
                short.append(d)
            with Batch(short, steps_per_pass=K, sequence=sequence, potential=potential) as b:
                b.run()  # warm-up (graph capture)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                b.run()
                sec = time.perf_counter() - t0
                su = b.info()["site_updates"]
            results.append(({"steps_per_pass": K, "chunk_rows": ch}, sec / su))
    cfg, spu = pick_best(results)
    entry = dict(cfg, site_updates_per_s=1.0 / spu, tuned_at=time.time())
    if use_cache:
        cache[key] = entry
        save_cache(cache)
    return entry
