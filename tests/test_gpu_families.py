"""Advancing one polarisation family (qla_options.families).

No operator of Eq. 17-22 couples TM = (q2, q3, q4) with TE = (q0, q1, q5), so a
field with one family zero keeps it at exactly zero: a context that stores and
advances only the other family must give the same state bit for bit. The
oracle side of this fact is pinned on the CPU (TE/TM decoupling in
tests/test_oracle_pins.py); here the two GPU paths are compared with each other
and, once, with the oracle.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2301_13601_gb300 import media
from paper_2301_13601_gb300 import qla as Q
from paper_2301_13601_gb300.qla import QLAError, Simulation

pytestmark = pytest.mark.gpu

TM = (2, 3, 4)
TE = (0, 1, 5)


def medium(Nx=520, Ny=90):
    return media.medium(Nx, Ny, [media.Ellipse(300, 45, 60, 30, 0.4, (1.6, 2.1, 2.7), 4.0)])


def run(n, family, pol, precision, K, steps, chunk=0):
    with Simulation(*n, 0.1, precision=precision, steps_per_pass=K, chunk_rows=chunk, families=family) as sim:
        sim.init_pulse(pol, 150.0, 25.0, 0.9)
        sim.step(steps)
        return sim.get_fields(np.float64)


@pytest.mark.parametrize("precision, K", [("fp32", 2), ("fp32", 4), ("fp32", 1), ("fp64", 2)])
@pytest.mark.parametrize("family, pol", [("TM", "Ez"), ("TE", "Ey")])
def test_single_family_bit_identical(precision, K, family, pol):
    n = medium()
    steps = 3 * K + 1  # fused passes and a shorter tail pass
    both = run(n, "both", pol, precision, K, steps, chunk=40)
    one = run(n, family, pol, precision, K, steps, chunk=40)
    assert np.array_equal(both, one)
    other = TE if family == "TM" else TM
    assert not np.any(one[list(other)])
    assert np.any(one[list(TM if family == "TM" else TE)])


def test_single_family_matches_oracle():
    n = medium(264, 70)
    steps = 9
    got = run(n, "TM", "Ez", "fp64", 2, steps)
    theta, beta = oracle.angles(*n, 0.1)
    q = oracle.init_pulse(264, 70, 0, 150.0, 25.0, 0.9)
    oracle.run(q, theta, beta, steps, oracle.SEQ_INTERLEAVED, oracle.POT_PAPER)
    assert np.linalg.norm(got - q) <= 1e-12 * np.linalg.norm(q)


def test_set_fields_ignores_the_other_family():
    n = medium()
    rng = np.random.default_rng(4)
    q = rng.standard_normal((6, 90, 520))
    q_tm = q.copy()
    q_tm[list(TE)] = 0.0
    with Simulation(*n, 0.1, families="TM") as one, Simulation(*n, 0.1) as both:
        one.set_fields(q)  # TE planes ignored
        both.set_fields(q_tm)
        back = one.get_fields(np.float32)
        assert not np.any(back[list(TE)])
        one.step(5)
        both.step(5)
        assert np.array_equal(one.get_fields(np.float32), both.get_fields(np.float32))
        # the FP32 host path as well
        host = torch.tensor(q.astype(np.float32)).pin_memory()
        one.set_fields_host_f32(host.data_ptr())
        one.synchronize()
        assert not np.any(one.get_fields(np.float32)[list(TE)])


def test_mismatched_pulse_and_bad_option_rejected():
    n = medium(264, 40)
    with Simulation(*n, 0.1, families="TE") as sim:
        with pytest.raises(QLAError) as e:
            sim.init_pulse("Ez", 100.0, 10.0, 1.0)
        assert e.value.status == 1  # QLA_EINVAL; the context stays usable
        sim.init_pulse("Ey", 100.0, 10.0, 1.0)
        sim.step(2)
    with pytest.raises(ValueError):
        Simulation(*n, 0.1, families="TEM")


def test_batch_rejects_a_single_family():
    L = Q.load_library()
    opt = Q.Options()
    L.qla_default_options(ctypes.byref(opt))
    opt.families = Q.FAMILY_TM
    opt.device = torch.cuda.current_device()
    n = medium(128, 16)
    d = Q.InstanceDesc()
    d.Nx, d.Ny = 128, 16
    keep = [np.ascontiguousarray(a, dtype=np.float64) for a in n]
    d.n_x, d.n_y, d.n_z = (a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for a in keep)
    d.delta, d.nsteps, d.pulse_polarization, d.chunk_rows = 0.1, 4, -1, 0
    b = ctypes.c_void_p()
    assert L.qla_batch_create(1, ctypes.byref(d), ctypes.byref(opt), ctypes.byref(b)) == 6  # QLA_EUNSUPPORTED


def test_rollout_needs_both_families():
    from paper_2301_13601_gb300 import surrogate as S

    Nx, Ny = 128, 64
    n = media.medium(Nx, Ny, [media.Ellipse(70, 30, 20, 12, 0.3, (1.5, 2.0, 2.5), 3.0)])
    nf = torch.as_tensor(np.stack(n), dtype=torch.float32, device="cuda")
    with S.Surrogate(Ny, Nx, K=16, seed=10) as sur, Simulation(*n, 0.05, families="TM") as sim:
        sim.init_pulse("Ez", 40, 10)
        with pytest.raises(QLAError) as e:
            sur.rollout(sim, nf, 1, drift_tol=1e-3)
        assert e.value.status == 6
