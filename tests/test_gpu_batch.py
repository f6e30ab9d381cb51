"""Batched lattices in one persistent graph launch (qla_batch_*).

The batched kernel runs the same per-tile arithmetic as the single-lattice
sweep, so each lattice must come out bit-identical to qla_step with the same
steps per pass; one lattice is also checked against the FP64 oracle. The
dependency waits are bounded: withholding one completion must end the run with
QLA_ETIMEOUT instead of hanging.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2301_13601_gb300 import media
from paper_2301_13601_gb300.qla import Batch, Simulation

pytestmark = pytest.mark.gpu

# (Nx, Ny, nsteps, polarisation, chunk_rows): uneven sizes, several strips and
# chunks, steps multiples of 4, a lattice narrower than a strip; Nx a multiple
# of 8 from 256 up (256, 512, 776) sweeps in the seam layout (strip 0 across
# x = 0, every strip on TMA), the others in the plain layout
CASES = [(64, 48, 8, "Ez", 0), (128, 100, 12, "Ey", 24), (200, 64, 16, "Ez", 0), (256, 256, 4, "Ey", 96),
         (300, 70, 20, "Ez", 16), (96, 96, 24, "Ey", 0), (512, 64, 8, "Ez", 0), (776, 40, 12, "Ey", 16)]


def make_instances(K=4):
    inst = []
    for k, (Nx, Ny, steps, pol, ch) in enumerate(CASES):
        objs = [media.Ellipse(0.6 * Nx, 0.5 * Ny, 0.2 * Nx, 0.15 * Ny, 0.3 * k, (1.5, 1.3, 2.2), 3.0)]
        inst.append({"n": media.medium(Nx, Ny, objs), "delta": 0.2, "nsteps": steps,
                     "pulse": (pol, Nx / 4, Nx / 16, 1.0), "chunk_rows": ch})
    return inst


@pytest.mark.parametrize("K", [4, 2])
def test_batch_bit_identical_to_single_lattice(K):
    inst = make_instances()
    with Batch(inst, steps_per_pass=K) as b:
        b.run()
        b.run()  # graph replay: a second run continues from the first
        got = [b.get_fields(i) for i in range(len(inst))]
        diags = [b.diagnostics(i) for i in range(len(inst))]
    for i, ins in enumerate(inst):
        with Simulation(*ins["n"], ins["delta"], steps_per_pass=K) as sim:
            pol, x0, sig, amp = ins["pulse"]
            sim.init_pulse(pol, x0, sig, amp)
            sim.step(2 * ins["nsteps"])
            ref = sim.get_fields(dtype=np.float32)
            e = sim.energy()
        assert np.array_equal(got[i], ref), f"instance {i}"
        assert diags[i]["energy"] == e


def test_batch_matches_oracle():
    inst = make_instances()
    with Batch(inst) as b:
        b.run()
        got = [b.get_fields(i).astype(np.float64) for i in range(len(inst))]
    for i in (1, 4):
        ins = inst[i]
        theta, beta = oracle.angles(*ins["n"], ins["delta"])
        Ny, Nx = ins["n"][0].shape
        pol, x0, sig, amp = ins["pulse"]
        ref = oracle.init_pulse(Nx, Ny, 0 if pol == "Ez" else 1, x0, sig, amp)
        oracle.run(ref, theta, beta, ins["nsteps"])
        assert np.linalg.norm(got[i] - ref) / np.linalg.norm(ref) < 3e-6


def test_batch_wait_times_out_instead_of_hanging():
    inst = make_instances()
    with Batch(inst) as b:
        b.set_wait_limit(50_000_000, withhold=1)  # 50 ms; one completion that never comes
        t0 = time.time()
        st = b.run_status()
        dt = time.time() - t0
        assert st == 4  # QLA_ETIMEOUT
        assert dt < 30.0
        # the batch stays usable once the hook is removed (states are discarded)
        b.set_wait_limit(4_000_000_000, withhold=0)
        assert b.run_status() == 0


def test_batch_rejects_bad_descriptors():
    from paper_2301_13601_gb300.qla import QLAError

    inst = make_instances()
    inst[0]["nsteps"] = 6  # not a multiple of steps_per_pass = 4
    with pytest.raises(QLAError):
        Batch(inst)
    inst = make_instances()
    with pytest.raises(QLAError):
        Batch(inst, steps_per_pass=3)
