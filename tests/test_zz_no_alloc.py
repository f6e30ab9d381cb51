"""qla_diagnostics_noalloc: the diagnostics entry point that allocates nothing.

It serves callers that may not call cudaMalloc when they need the energy and
div B of a state they already hold on the device (their memory belongs to
another allocator, or the loop must not block on or fail in the allocator).
Its scratch lives in a fixed device array inside the library. These tests call
it through the C ABI and compare it with the context-based qla_diagnostics on
the same device state, twice in a row (the shared array keeps the previous
call's contents, which must not leak into the next result).

This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from paper_2301_13601_gb300 import media
from paper_2301_13601_gb300.qla import FP32, FP64, Diag, Simulation, load_library

pytestmark = pytest.mark.gpu


def noalloc(sim):
    L = load_library()
    d = Diag()
    st = L.qla_diagnostics_noalloc(L.qla_state_device_ptr(sim._ctx), sim.precision, sim.Nx, sim.Ny,
                                   ctypes.c_void_p(sim.stream.cuda_stream), ctypes.byref(d))
    return st, {"energy": d.energy, "div_l2_sq": d.div_l2_sq, "div_max": d.div_max, "b_max": d.b_max,
                "nonfinite": d.nonfinite}


def assert_close(a, b):
    # tolerances of the diagnostics parity tests (compensated FP64 sums in a
    # different but fixed order)
    assert a["nonfinite"] == b["nonfinite"]
    assert abs(a["energy"] - b["energy"]) <= 1e-14 * abs(b["energy"])
    assert abs(a["div_l2_sq"] - b["div_l2_sq"]) <= 1e-13 * abs(b["div_l2_sq"])
    assert abs(a["div_max"] - b["div_max"]) <= 1e-14 * abs(b["div_max"])
    assert abs(a["b_max"] - b["b_max"]) <= 1e-14 * abs(b["b_max"])


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_noalloc_matches_context_diagnostics_twice(precision):
    Nx, Ny = 700, 333
    n = media.smooth_periodic_medium(Nx, Ny, seed=4, amp=0.3)
    q = media.smooth_periodic_field(Nx, Ny, 21)
    q += 0.1 * np.random.default_rng(2).standard_normal(q.shape)
    with Simulation(*n, 0.1, precision=precision) as sim:
        sim.set_fields(q)
        st, got = noalloc(sim)
        assert st == 0
        assert_close(got, sim.diagnostics())
        # second call on a different state: nothing of the first call may remain
        sim.step(9)
        st, got2 = noalloc(sim)
        assert st == 0
        ref2 = sim.diagnostics()
        assert_close(got2, ref2)
        assert got2["energy"] != got["energy"]


def test_noalloc_after_a_larger_call_and_nonfinite():
    """A small lattice after a tall one reads only records it wrote itself."""
    big = Simulation(*media.uniform_medium(64, 4000, (1.2, 1.3, 1.4)), 0.1)
    big.set_fields(np.random.default_rng(1).standard_normal((6, 4000, 64)))
    st, _ = noalloc(big)
    assert st == 0
    big.close()
    Nx, Ny = 96, 10
    q = np.random.default_rng(3).standard_normal((6, Ny, Nx))
    q[4, 2, 5] = np.nan
    with Simulation(*media.uniform_medium(Nx, Ny, (1.2, 1.3, 1.4)), 0.1) as sim:
        sim.set_fields(q)
        st, got = noalloc(sim)
        ref = sim.diagnostics()
    assert st == 5 and got["nonfinite"] == 1 == ref["nonfinite"]


def test_noalloc_rejects_sizes_beyond_its_scratch():
    """Size and argument checks come before any use of the device (run with no
    visible GPU, so that a missing check cannot reach one)."""
    import host_checks

    host_checks.run_without_gpu("noalloc_rejects_sizes_beyond_its_scratch")
