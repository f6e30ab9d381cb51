"""Each operator of the step on the GPU (qla_debug_apply) against the oracle's
function for that operator: collisions C_X, C_Y and their transposes (Eq. 17,
Eq. 19), the eight streaming shifts (Eq. 18, Eq. 20) and the potentials V_X,
V_Y (Eq. 21-22) in both variants. The GPU evaluates each operator with the
sweep's per-site arithmetic and coefficient pairs; a mistake in one factor
(a sign, a partner component, a shift direction) fails its own case here.

Tolerances: FP64 contexts store (cos a - 1, sin a) computed in double, the
oracle rounds cos a and sin a separately: one rotation agrees to a few ulp
(1e-14 relative); streaming is a permutation and compared bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_2301_13601_gb300 import media
from paper_2301_13601_gb300.qla import OPS, QLAError, Simulation

pytestmark = pytest.mark.gpu

Nx, Ny = 136, 50


def setup(potential="paper", sequence="interleaved", precision="fp64"):
    n = media.smooth_periodic_medium(Nx, Ny, seed=11, amp=0.4)
    q = np.random.default_rng(12).standard_normal((6, Ny, Nx))
    if precision == "fp32":
        q = q.astype(np.float32).astype(np.float64)
    sim = Simulation(*n, 0.2, precision=precision, potential=potential, sequence=sequence)
    sim.set_fields(q)
    theta, beta = oracle.angles(*n, 0.2)
    return sim, q, theta, beta


STREAMS = {"S14+x": (1, 4, 0, +1), "S14-x": (1, 4, 0, -1), "S25+x": (2, 5, 0, +1), "S25-x": (2, 5, 0, -1),
           "S03+y": (0, 3, 1, +1), "S03-y": (0, 3, 1, -1), "S25+y": (2, 5, 1, +1), "S25-y": (2, 5, 1, -1)}


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("op", ["CX", "CX_T", "CY", "CY_T"])
def test_collisions(op):
    sim, q, theta, beta = setup()
    with sim:
        sim.debug_apply(op)
        got = sim.get_fields()
    ref = q.copy()
    (oracle.collide_x if op.startswith("CX") else oracle.collide_y)(ref, theta, dagger=op.endswith("_T"))
    assert rel(got, ref) < 1e-14
    assert not np.array_equal(got, q)


@pytest.mark.parametrize("op", list(STREAMS))
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_streaming_is_the_permutation(op, precision):
    sim, q, theta, beta = setup(precision=precision)
    with sim:
        sim.debug_apply(op, 3)
        got = sim.get_fields()
    ref = q.copy()
    ca, cb, axis, d = STREAMS[op]
    for _ in range(3):
        oracle.stream(ref, ca, cb, axis, d)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("op", ["VX", "VY"])
@pytest.mark.parametrize("potential", ["paper", "unitary"])
@pytest.mark.parametrize("sequence", ["interleaved", "plain"])
def test_potentials(op, potential, sequence):
    sim, q, theta, beta = setup(potential=potential, sequence=sequence)
    with sim:
        sim.debug_apply(op)
        got = sim.get_fields()
    ref = q.copy()
    scale = 0.5 if sequence == "interleaved" else 1.0
    mode = oracle.POT_PAPER if potential == "paper" else oracle.POT_UNITARY
    (oracle.potential_x if op == "VX" else oracle.potential_y)(ref, beta, scale, mode)
    assert rel(got, ref) < 1e-14


def test_fp32_collision_and_transpose_cancel():
    """C followed by its transpose is the identity up to FP32 rounding."""
    sim, q, theta, beta = setup(precision="fp32")
    with sim:
        sim.debug_apply("CY")
        sim.debug_apply("CY_T")
        got = sim.get_fields()
    assert rel(got, q) < 1e-6


def test_bad_arguments():
    sim, q, theta, beta = setup()
    with sim:
        with pytest.raises(ValueError):
            sim.debug_apply("CZ")
        with pytest.raises(QLAError):
            sim.debug_apply("CX", -1)
        sim.debug_apply("CX", 0)
        assert np.array_equal(sim.get_fields(), q)
        assert len(OPS) == 14
