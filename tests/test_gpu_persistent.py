"""The persistent launch form (qla_options.launch) against one launch per pass.

Both forms run the same per-pass arithmetic over the same shares, so the
states must agree bit for bit after any number of steps and calls: a share
that started a pass before the shares it reads had finished theirs (a missing
dependency), or that overwrote rows a neighbour had not yet read, would show
as a difference here. Cases: the bench-like lattice shape, the seam strip with
one clamped strip, rows fewer than a dependency window, shares over several
strips, a ragged last strip, both families, one family, both step orders and
potential variants, step counts with a shorter tail pass, several calls in a
row with diagnostics between them; once against the FP64 oracle.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2301_13601_gb300 import media
from paper_2301_13601_gb300.qla import Simulation

pytestmark = pytest.mark.gpu


def fields(Nx, Ny, seed, family="both"):
    q = media.smooth_periodic_field(Nx, Ny, seed)
    q += 0.05 * np.random.default_rng(seed).standard_normal(q.shape)
    if family == "TM":
        q[[0, 1, 5]] = 0.0
    elif family == "TE":
        q[[2, 3, 4]] = 0.0
    return q


def run(Nx, Ny, launch, calls, family="both", sequence="interleaved", potential="paper", seed=1):
    n = media.smooth_periodic_medium(Nx, Ny, seed=seed + 10, amp=0.3)
    with Simulation(*n, 0.1, launch=launch, families=family, sequence=sequence, potential=potential) as sim:
        sim.set_fields(fields(Nx, Ny, seed, family))
        energies = []
        for steps in calls:
            sim.step(steps)
            energies.append(sim.diagnostics()["energy"])
        return sim.launch, sim.get_fields(np.float32), energies


@pytest.mark.parametrize("Nx,Ny,family,calls", [
    (2048, 2048, "both", (10,)),
    (256, 300, "both", (7, 4)),        # the seam strip and one clamped strip; a tail pass
    (1000, 64, "TE", (6, 6, 1)),       # windows wrapping around y
    (520, 7, "both", (8,)),            # fewer rows than a dependency window
    (4096, 32, "TM", (12,)),           # shares over several strips
    (2056, 1500, "both", (3, 9, 2)),   # ragged last strip
])
def test_persistent_bit_identical_to_per_pass(Nx, Ny, family, calls):
    form, got, e_got = run(Nx, Ny, "persistent", calls, family)
    assert form == "persistent"
    form_ref, ref, e_ref = run(Nx, Ny, "per_pass", calls, family)
    assert form_ref == "per_pass"
    assert np.array_equal(got, ref)
    assert e_got == e_ref


@pytest.mark.parametrize("sequence,potential", [("plain", "paper"), ("interleaved", "unitary"),
                                                ("plain", "unitary")])
def test_persistent_step_orders_and_potentials(sequence, potential):
    _, got, _ = run(768, 200, "persistent", (9,), sequence=sequence, potential=potential)
    _, ref, _ = run(768, 200, "per_pass", (9,), sequence=sequence, potential=potential)
    assert np.array_equal(got, ref)


def test_persistent_many_passes_in_one_launch():
    """200 passes in one launch (the counters run on across calls)."""
    _, got, _ = run(1024, 1024, "persistent", (400, 2, 400))
    _, ref, _ = run(1024, 1024, "per_pass", (400, 2, 400))
    assert np.array_equal(got, ref)


def test_the_persistent_form_applies_where_documented():
    n = media.uniform_medium(512, 64, (1.2, 1.3, 1.4))
    with Simulation(*n, 0.1, launch="persistent") as sim:
        assert sim.launch == "persistent"
    with Simulation(*n, 0.1) as sim:  # automatic: one launch per pass
        assert sim.launch == "per_pass"
    with Simulation(*n, 0.1, chunk_rows=32, launch="persistent") as sim:  # fixed tiles
        assert sim.launch == "per_pass"
    with Simulation(*n, 0.1, precision="fp64", launch="persistent") as sim:
        assert sim.launch == "per_pass"
    with Simulation(*n, 0.1, steps_per_pass=4, launch="persistent") as sim:
        assert sim.launch == "per_pass"
    m = media.uniform_medium(500, 64, (1.2, 1.3, 1.4))  # Nx not a multiple of 8
    with Simulation(*m, 0.1, launch="persistent") as sim:
        assert sim.launch == "per_pass"


def test_persistent_matches_oracle():
    Nx, Ny, steps = 512, 200, 12
    n = media.medium(Nx, Ny, [media.Ellipse(300, 100, 60, 40, 0.3, (1.6, 2.1, 2.7), 4.0)])
    with Simulation(*n, 0.1, launch="persistent") as sim:
        assert sim.launch == "persistent"
        sim.init_pulse("Ey", 150.0, 25.0, 0.9)
        sim.step(steps)
        got = sim.get_fields(np.float64)
    theta, beta = oracle.angles(*n, 0.1)
    q = oracle.init_pulse(Nx, Ny, oracle.POL_EY, 150.0, 25.0, 0.9)
    oracle.run(q, theta, beta, steps, oracle.SEQ_INTERLEAVED, oracle.POT_PAPER)
    assert np.linalg.norm(got - q) <= 3e-6 * np.linalg.norm(q)


def test_persistent_wait_times_out_instead_of_hanging():
    """Every wait of a persistent pass for its neighbours is bounded: with the
    test hook demanding one pass more than any share will publish, the first
    waits run out after 50 ms, every CTA stops, and the call's
    synchronisation reports QLA_ETIMEOUT instead of hanging. The device stays
    usable: a fresh context then agrees with one launch per pass."""
    from paper_2301_13601_gb300.qla import QLAError

    Nx, Ny = 1024, 512
    n = media.smooth_periodic_medium(Nx, Ny, seed=3, amp=0.3)
    with Simulation(*n, 0.1, launch="persistent") as sim:
        assert sim.launch == "persistent"
        sim.set_fields(fields(Nx, Ny, 1))
        sim.set_wait_limit(50_000_000, withhold=1)  # a pass that never comes
        t0 = time.time()
        sim.step(10)
        with pytest.raises(QLAError) as err:
            sim.synchronize()
        assert err.value.status == 4  # QLA_ETIMEOUT
        assert time.time() - t0 < 30.0
    _, got, _ = run(512, 200, "persistent", (6,))
    _, ref, _ = run(512, 200, "per_pass", (6,))
    assert np.array_equal(got, ref)
