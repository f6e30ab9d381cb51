"""Full-length parity on the 2048^2 ellipse workload against stored oracle values.

tests/golden/ellipse2048_interleaved_paper.npz is written by
tests/golden/make_golden.py, which calls only the FP64 CPU oracle: energy
(Eq. 27) and div B every 100 steps for 10000 steps, and the state at steps
1000 and 10000 sampled on every 16th site.

Targets: FP32 state vs the FP64 oracle, relative L2 <= 1e-4 after 1e4 steps;
|E_gpu - E_oracle| / E(0) <= 1e-6 at every diagnostic step; the FP64 GPU mode
to relative L2 <= 1e-12.
"""
import os

import numpy as np
import pytest

from paper_2301_13601_gb300 import media
from paper_2301_13601_gb300.qla import Simulation

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "ellipse2048_interleaved_paper.npz")


@pytest.fixture(scope="module")
def golden():
    if not os.path.exists(GOLDEN):
        pytest.fail(f"missing {GOLDEN}; run tests/golden/make_golden.py")
    return np.load(GOLDEN)


def run_gpu(golden, precision):
    w = media.workload_ellipse_2048()
    n = w.medium()
    S = int(golden["sample"])
    steps = golden["steps"]
    out = {"energy": [], "div": []}
    with Simulation(*n, w.delta, precision=precision) as sim:
        sim.init_pulse("Ey", w.pulse.x0, w.pulse.sigma, w.pulse.amp)
        d = sim.diagnostics()
        out["energy"].append(d["energy"])
        out["div"].append((d["div_l2_sq"], d["div_max"], d["b_max"]))
        for k in range(1, len(steps)):
            sim.step(int(steps[k] - steps[k - 1]))
            d = sim.diagnostics()
            out["energy"].append(d["energy"])
            out["div"].append((d["div_l2_sq"], d["div_max"], d["b_max"]))
            if int(steps[k]) in (1000, w.steps):
                out[f"q_s{int(steps[k])}"] = sim.get_fields()[:, ::S, ::S]
    return out


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_ellipse_2048_fp32_full_length(golden):
    got = run_gpu(golden, "fp32")
    E = np.array(got["energy"])
    Eo = golden["energy"]
    drift = np.abs(E - Eo) / Eo[0]
    assert drift.max() <= 1e-6, f"max |E_gpu - E_oracle|/E(0) = {drift.max():.3e}"
    for s in (1000, 10000):
        r = rel_l2(got[f"q_s{s}"], golden[f"q_s{s}"])
        assert r <= 1e-4, f"step {s}: rel L2 {r:.3e}"


def test_ellipse_2048_fp64_full_length(golden):
    got = run_gpu(golden, "fp64")
    for s in (1000, 10000):
        r = rel_l2(got[f"q_s{s}"], golden[f"q_s{s}"])
        assert r <= 1e-12, f"step {s}: rel L2 {r:.3e}"
    E = np.array(got["energy"])
    assert (np.abs(E - golden["energy"]) / golden["energy"][0]).max() <= 1e-12
