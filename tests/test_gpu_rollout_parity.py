"""The surrogate rollout's energy check against the FP64 oracle (row a11:
plain QLA stays the judge of every surrogate call).

qla_surrogate_rollout computes the energy (Eq. 27) of the state a call starts
from and of the network's proposal with a light reduction (FP32 squares, FP64
sums; its header states ~1e-6 relative) and accepts the proposal when
|E(proposal)/E(start) - 1| <= drift_tol. Here the same proposal is computed by
a separate forward call (the same kernels and weights, so bit-identical), its
energy and the start energy are taken by the oracle in FP64, and:
  * the rollout's two energies agree with the oracle's to 1e-6;
  * with drift_tol just above the oracle's drift the call is accepted and the
    state becomes the proposal bit for bit; just below, it is rejected and the
    state is K plain QLA steps from the start, bit for bit. "Just" is 5e-6 in
    drift, twice the error the 1e-6 energy accuracy allows on a ratio of two
    energies, so the decision is the oracle's.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_13601_gb300 import media
from paper_2301_13601_gb300 import surrogate as S
from paper_2301_13601_gb300 import surrogate_train as T
from paper_2301_13601_gb300.qla import Simulation

pytestmark = pytest.mark.gpu

H, W, DELTA = 128, 256, 0.05


def start_state():
    """A pulse that has entered an anisotropic ellipse (plain QLA, FP32)."""
    n = media.medium(W, H, [media.Ellipse(150.0, 64.0, 30.0, 20.0, 0.5, (2.0, 1.5, 2.5), 4.0)])
    with Simulation(*n, DELTA, precision="fp32") as sim:
        sim.init_pulse("Ez", 100.0, 20.0, 1.0)
        sim.step(640)
        q = sim.get_fields(dtype=np.float32)
    return n, q


@pytest.fixture(scope="module")
def setup():
    params, meta = T.load_checkpoint(T.DEFAULT_CHECKPOINT)
    n, q = start_state()
    nf = torch.as_tensor(np.stack(n), dtype=torch.float32, device="cuda").contiguous()
    with S.Surrogate(H, W, K=meta["K"], out_scale=meta["out_scale"]) as sur:
        sur.set_params(params)
        qi = torch.as_tensor(q[None], device="cuda").contiguous()
        qo = torch.empty_like(qi)
        sur.forward(qi, nf, qo)
        sur.synchronize()
        prop = qo[0].cpu().numpy()
    e_start = oracle.energy(q.astype(np.float64))
    e_prop = oracle.energy(prop.astype(np.float64))
    return params, meta, n, nf, q, prop, e_start, e_prop


def rollout_once(setup, tol):
    params, meta, n, nf, q, prop, e_start, e_prop = setup
    with Simulation(*n, DELTA, precision="fp32") as sim, \
            S.Surrogate(H, W, K=meta["K"], out_scale=meta["out_scale"]) as sur:
        sur.set_params(params)
        sim.set_fields(q)
        st = sur.rollout(sim, nf, 1, drift_tol=tol)
        got = sim.get_fields(dtype=np.float32)
    return st, got


def test_rollout_energies_match_the_oracle(setup):
    params, meta, n, nf, q, prop, e_start, e_prop = setup
    drift = abs(e_prop / e_start - 1)
    assert drift > 2e-5  # the network changes the energy measurably on this state
    st, got = rollout_once(setup, 1.0)
    assert st["surrogate_calls"] == 1
    print(f"oracle E(start) {e_start:.12e} E(proposal) {e_prop:.12e} drift {drift:.3e}; "
          f"rollout E(start) {st['energy_ref']:.12e} E(final) {st['energy_final']:.12e}")
    assert abs(st["energy_ref"] / e_start - 1) <= 1e-6
    assert abs(st["energy_final"] / e_prop - 1) <= 1e-6
    assert abs(st["max_drift"] - drift) <= 2e-6


def test_accept_reject_decision_is_the_oracles(setup):
    params, meta, n, nf, q, prop, e_start, e_prop = setup
    drift = abs(e_prop / e_start - 1)
    st, got = rollout_once(setup, drift + 5e-6)
    assert st["surrogate_calls"] == 1 and st["fallback_calls"] == 0
    assert np.array_equal(got, prop)
    st, got = rollout_once(setup, drift - 5e-6)
    assert st["surrogate_calls"] == 0 and st["fallback_calls"] == 1
    with Simulation(*n, DELTA, precision="fp32") as sim:
        sim.set_fields(q)
        sim.step(meta["K"])
        qla = sim.get_fields(dtype=np.float32)
    assert np.array_equal(got, qla)


@pytest.mark.parametrize("mode", [S.DRIFT_PER_CALL, S.DRIFT_FROM_START])
def test_speculative_rollout_equals_the_serial_loop(setup, mode):
    """The default rollout runs the next call's network pass while the host
    reads the current call's energy (a third state buffer) and discards it on
    a rejection; its states, decisions and statistics must be the serial
    loop's, bit for bit, on a run that mixes accepted and rejected calls."""
    params, meta, n, nf, q, prop, e_start, e_prop = setup
    calls = 12

    def run(tol, serial):
        with Simulation(*n, DELTA, precision="fp32") as sim, \
                S.Surrogate(H, W, K=meta["K"], out_scale=meta["out_scale"]) as sur:
            sur.set_params(params)
            sim.set_fields(q)
            st = sur.rollout(sim, nf, calls, drift_tol=tol, drift_mode=mode, serial=serial)
            return st, sim.get_fields(dtype=np.float32), sim.step_count

    chosen = None
    for tol in np.geomspace(1e-4, 3e-2, 25):  # the network's drift per call is ~1e-2 on this state
        st, got, steps = run(tol, True)
        if 0 < st["fallback_calls"] < calls:
            chosen = (float(tol), st, got, steps)
            break
    assert chosen, "no tolerance gives a mix of accepted and rejected calls"
    tol, st_s, got_s, steps_s = chosen
    st_p, got_p, steps_p = run(tol, False)
    print(f"tol {tol}: serial {st_s}, speculative {st_p}")
    assert steps_p == steps_s == calls * meta["K"]
    assert st_p == st_s
    assert np.array_equal(got_p, got_s)
    for tol in (0.0, 1.0):  # all rejected / all accepted
        a, b = run(tol, True), run(tol, False)
        assert a[0] == b[0] and np.array_equal(a[1], b[1]) and a[2] == b[2]
