"""Runs of the paper's scattering set-up (Sec. 3, Fig. 1; Sec. 4, Fig. 2) on the GPU path.

The object is the anisotropic one of Sec. 4 (media.cone_cylinder_medium: n_z
conical, n_x = n_y cylindrical, n_max = 3) centred on an N x N periodic
lattice, with a 1D Gaussian pulse travelling in +x. Fig. 1 of the paper shows
the total energy (Eq. 27) over the run for delta = 0.3 (20k steps) and 0.1
(60k steps), i.e. the same physical time delta * steps = 6000 cells on
8192^2; energy_history() records E(t)/E(0) - 1 and the divergence ratios for
any (delta, step sequence, potential variant).

    python -m paper_2301_13601_gb300.studies --N 8192 --deltas 0.3 0.1

prints one JSON record per run. Radii (not given in the paper): r_cone =
r_cyl = N/16; pulse x0 = N/4, sigma = N/80.
"""
from __future__ import annotations

import argparse
import json
import time
from typing import Dict, Iterable, List

from . import media
from .qla import Simulation


def energy_history(N: int, delta: float, sequence: str = "interleaved", potential: str = "paper",
                   polarization: str = "Ez", physical_time: float = None, samples: int = 20) -> Dict:
    """One run: E(t)/E(0) - 1 at `samples` evenly spaced times, and at the end
    max |div B|/max |B| and max |div D|/max |D|. Only the pulse's polarisation
    family is advanced (the other stays exactly zero)."""
    if physical_time is None:
        physical_time = 6000.0 * N / 8192
    steps = int(round(physical_time / delta))
    every = max(1, steps // samples)
    n = media.cone_cylinder_medium(N, N / 16, N / 16)
    family = "TM" if polarization == "Ez" else "TE"
    t0 = time.time()
    with Simulation(*n, delta, sequence=sequence, potential=potential, families=family) as sim:
        sim.init_pulse(polarization, N / 4, N / 80, -1.0 if polarization == "Ez" else 1.0)
        e0 = sim.energy()
        hist: List[List[float]] = []
        done = 0
        while done < steps:
            k = min(every, steps - done)
            sim.step(k)
            done += k
            hist.append([done, sim.energy() / e0 - 1.0])
        _, mb, b = sim.divB()
        _, md, d = sim.divD()
    return {"N": N, "delta": delta, "steps": steps, "sequence": sequence, "potential": potential,
            "polarization": polarization, "energy_rel_change": hist,
            "max_abs_energy_rel_change": max(abs(v) for _, v in hist),
            "divB_over_B": mb / b if b > 0 else 0.0, "divD_over_D": md / d if d > 0 else 0.0,
            "seconds": time.time() - t0}


def main(argv: Iterable[str] = None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--N", type=int, default=8192)
    ap.add_argument("--deltas", type=float, nargs="+", default=[0.3, 0.1])
    ap.add_argument("--sequences", nargs="+", default=["plain", "interleaved"])
    ap.add_argument("--potentials", nargs="+", default=["paper", "unitary"])
    ap.add_argument("--polarization", default="Ez", choices=["Ez", "Ey"])
    a = ap.parse_args(argv)
    for delta in a.deltas:
        for seq in a.sequences:
            for pot in a.potentials:
                r = energy_history(a.N, delta, seq, pot, a.polarization)
                print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
