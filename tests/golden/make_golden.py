"""Write oracle-computed expected values for the long parity tests.

Calls only the CPU oracle (``oracle/``) and the input generators
(``paper_2301_13601_gb300.media``); nothing here touches the CUDA path.

Output ``ellipse2048_interleaved_paper.npz`` (2048^2 lattice, delta 0.05, E_y
pulse, tanh-edged ellipse; interleaved step Eq. 28 with the printed potentials
Eq. 21-22): energy (Eq. 27) and div B statistics every 100 steps for 10000
steps, and the full state at steps 0, 1000 and 10000 sampled on every 16th
site in x and y (``q_s{step}``, shape (6, 128, 128)).

Usage: python tests/golden/make_golden.py [--threads N]
"""
import argparse
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2301_13601_gb300 import media  # noqa: E402

SAMPLE = 16


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                  "ellipse2048_interleaved_paper.npz"))
    args = ap.parse_args()
    if args.threads:
        oracle.set_threads(args.threads)
    w = media.workload_ellipse_2048()
    nx, ny, nz = w.medium()
    theta, beta = oracle.angles(nx, ny, nz, w.delta)
    q = oracle.init_pulse(w.Nx, w.Ny, w.pulse.pol, w.pulse.x0, w.pulse.sigma, w.pulse.amp)
    every = 100
    steps, energy, div = [0], [oracle.energy(q)], [oracle.divB(q)]
    snaps = {"q_s0": q[:, ::SAMPLE, ::SAMPLE].copy()}
    t0 = time.time()
    for s in range(every, w.steps + 1, every):
        oracle.run(q, theta, beta, every, oracle.SEQ_INTERLEAVED, oracle.POT_PAPER)
        steps.append(s)
        energy.append(oracle.energy(q))
        div.append(oracle.divB(q))
        if s in (1000, w.steps):
            snaps[f"q_s{s}"] = q[:, ::SAMPLE, ::SAMPLE].copy()
        print(f"step {s} energy {energy[-1]:.15e} elapsed {time.time() - t0:.0f}s", flush=True)
    np.savez_compressed(args.out, steps=np.array(steps), energy=np.array(energy),
                        divB=np.array(div), sample=SAMPLE, delta=w.delta, **snaps)
    print("wrote", args.out)


if __name__ == "__main__":
    main()
