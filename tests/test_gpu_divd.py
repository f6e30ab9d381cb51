"""div D on the GPU (qla_divD) against the oracle, and the behaviour the paper
describes for the E_y polarisation (Sec. 4.2): the QLA generates an E_x field
that keeps div D small where the medium makes D_y vary along y.

The oracle's div D is pinned on the CPU (a discrete curl in an anisotropic
medium has zero divergence; a closed form), tests/test_oracle_pins.py.
"""
import numpy as np
import pytest

import oracle
from paper_2301_13601_gb300 import media
from paper_2301_13601_gb300.qla import Simulation

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_divD_matches_oracle(precision):
    Nx, Ny = 333, 121
    q = np.random.default_rng(6).standard_normal((6, Ny, Nx))
    if precision == "fp32":
        q = q.astype(np.float32).astype(np.float64)
    n = media.smooth_periodic_medium(Nx, Ny, seed=5, amp=0.4)
    with Simulation(*n, 0.1, precision=precision) as sim:
        sim.set_fields(q)
        s, m, d = sim.divD()
    rs, rm, rd = oracle.divD(q, *n)
    assert abs(s - rs) <= 1e-13 * rs
    assert abs(m - rm) <= 1e-14 * rm
    assert abs(d - rd) <= 1e-14 * rd


def test_ey_pulse_generates_ex_that_cancels_div_D():
    """E_y pulse through an anisotropic ellipse with the unitary potentials:
    div D with the generated E_x is far below what D_y alone would give.
    (Oracle, 256^2 at 800 steps: 3.2e-3 against 4.2e-2 of max |D|.)"""
    Nx = Ny = 256
    n = media.medium(Nx, Ny, [media.Ellipse(150, 128, 40, 25, 0.5, (2.0, 1.4, 1.1), 4.0)])
    with Simulation(*n, 0.1, potential="unitary") as sim:
        sim.init_pulse("Ey", 60.0, 10.0, 1.0)
        sim.step(800)
        s, m, d = sim.divD()
        q = sim.get_fields()
        q[0] = 0.0
        sim.set_fields(q)
        s0, m0, d0 = sim.divD()
    ratio, ratio_no_ex = m / d, m0 / d0
    print(f"max|div D|/max|D| = {ratio:.3e}; without E_x {ratio_no_ex:.3e}")
    assert ratio < 1e-2 and ratio < 0.2 * ratio_no_ex
