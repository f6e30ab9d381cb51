"""The stored oracle values are what the committed scripts produce.

tests/golden/*.npz hold expected values written by tests/golden/make_*.py,
which call only the CPU oracle. These checks rerun the first stretch of each
script's runs with the current oracle and compare it with the stored values,
so that a change to the oracle's arithmetic or to an input generator cannot
leave a stale file behind. (CPU only, about twenty seconds.)
"""
import importlib.util
import os

import numpy as np
import pytest

import oracle
from paper_2301_13601_gb300 import media

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_script(name):
    spec = importlib.util.spec_from_file_location(name, os.path.join(GOLDEN, name + ".py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_ellipse2048_golden_inputs_reproduce():
    # the input generators and the pulse (the step's arithmetic is rechecked
    # on the 512^2 file below, whose runs take the same code path)
    g = np.load(os.path.join(GOLDEN, "ellipse2048_interleaved_paper.npz"))
    w = media.workload_ellipse_2048()
    q = oracle.init_pulse(w.Nx, w.Ny, w.pulse.pol, w.pulse.x0, w.pulse.sigma, w.pulse.amp)
    assert np.array_equal(q[:, ::int(g["sample"]), ::int(g["sample"])], g["q_s0"])
    assert oracle.energy(q) == pytest.approx(g["energy"][0], rel=1e-15)
    theta, beta = oracle.angles(*w.medium(), w.delta)
    assert np.all(np.isfinite(theta)) and np.all(np.isfinite(beta))


def test_subulp_golden_reproduces():
    g = np.load(os.path.join(GOLDEN, "ellipse512_subulp_potentials.npz"))
    m = load_script("make_subulp_golden")
    theta, beta = oracle.angles(*m.workload_medium(), m.DELTA)
    cut = beta.copy()
    cut[np.abs(cut) < 2.0 ** -24] = 0.0
    for b, key in ((beta, "energy"), (cut, "energy_k24")):
        q = oracle.init_pulse(m.N, m.N, oracle.POL_EY, m.X0, m.SIGMA, 1.0)
        oracle.run(q, theta, b, m.EVERY, oracle.SEQ_INTERLEAVED, oracle.POT_PAPER)
        assert oracle.energy(q) == pytest.approx(g[key][1], rel=1e-14), key
    # the cuts remove energy in the order of their thresholds
    d = [g[k][-1] - g["energy"][-1] for k in ("energy_k25", "energy_k24", "energy_k23")]
    assert 0 > d[0] > d[1] > d[2]
