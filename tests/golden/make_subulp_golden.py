"""Write oracle energies for the sub-resolution potential test.

Calls only the CPU oracle (``oracle/``) and the input generators
(``paper_2301_13601_gb300.media``); nothing here touches the CUDA path.

Workload: a 512^2 lattice, delta 0.05, one tanh-edged ellipse (semi-axes
60 x 36, rotated 30 deg, edge 8, indices (2.0, 1.4, 1.1)) at the centre, an
E_y pulse (sigma 12) at x0 = 110; interleaved step (Eq. 28) with the printed
potentials (Eq. 21-22), 3000 steps. Output ``ellipse512_subulp_potentials.npz``:
the energy (Eq. 27) every 250 steps of the plain run (``energy``) and of runs
whose potential angles beta (Eq. 25) are set to zero where |beta| < 2^-k
(``energy_k25``, ``energy_k24``, ``energy_k23``): a potential row then has no
effect where its increment beta * q would lie below FP32 resolution of a
target of the same size.

Usage: python tests/golden/make_subulp_golden.py
"""
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2301_13601_gb300 import media  # noqa: E402

N, DELTA, STEPS, EVERY = 512, 0.05, 3000, 250
X0, SIGMA = 110.0, 12.0


def workload_medium():
    objs = [media.Ellipse(256.0, 256.0, 60.0, 36.0, math.radians(30.0), (2.0, 1.4, 1.1), 8.0)]
    return media.medium(N, N, objs)


def energies(theta, beta):
    q = oracle.init_pulse(N, N, oracle.POL_EY, X0, SIGMA, 1.0)
    out = [oracle.energy(q)]
    for _ in range(EVERY, STEPS + 1, EVERY):
        oracle.run(q, theta, beta, EVERY, oracle.SEQ_INTERLEAVED, oracle.POT_PAPER)
        out.append(oracle.energy(q))
        print(f"step {len(out) * EVERY - EVERY} energy {out[-1]:.15e}", flush=True)
    return np.array(out)


def main():
    theta, beta = oracle.angles(*workload_medium(), DELTA)
    res = {"steps": np.arange(0, STEPS + 1, EVERY), "energy": energies(theta, beta)}
    for k in (25, 24, 23):
        b = beta.copy()
        b[np.abs(b) < 2.0 ** -k] = 0.0
        res[f"energy_k{k}"] = energies(theta, b)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ellipse512_subulp_potentials.npz")
    np.savez_compressed(out, **res)
    print("wrote", out)


if __name__ == "__main__":
    main()
