"""Host-side checks of the balanced split of a sweep pass (qla_sweep_split).

With chunk_rows = 0 a pass launches one CTA per resident slot and family;
CTA b sweeps the row units [bounds[b], bounds[b + 1]) (u = strip * Ny + y) as
one segment per strip it touches. The bounds come from the library's host
arithmetic, the same code the kernel runs per CTA. These tests check, with no
GPU visible, that the shares tile the units exactly and that their costs
under the documented model agree: 16 per row of a strip copied by TMA, more
per row of an FP32 strip that wraps around x (copied with cp.async), and the
warm-up rows 8K + R (K - 1) at each strip start.
"""
import numpy as np
import pytest

import host_checks
from paper_2301_13601_gb300 import qla

W_IN = 256


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


def model(Nx, Ny, K, precision):
    """Per-strip row costs and the warm-up rows of the documented model. The
    slow-strip weights (32 at K = 1, 2; 26 at K = 4) are the library's
    measured constants."""
    wv = W_IN - 8 * K
    nsx = -(-Nx // wv)
    R = 8 if (precision == "fp32" and K == 1) else 4
    tma_ok = precision == "fp32" and Nx % 8 == 0
    w = []
    for s in range(nsx):
        xbase = s * wv - 4 * K
        uses_tma = tma_ok and xbase >= 0 and xbase + W_IN <= Nx and xbase % 8 == 0
        w.append(16 if (uses_tma or not tma_ok) else (26 if K >= 4 else 32))
    return nsx, w, 8 * K + R * (K - 1)


def share_costs(b, Ny, w, warm):
    """Cost of each share: its rows at their strip's row cost, plus the warm-up
    of every strip start it holds."""
    costs = []
    for u0, u1 in zip(b[:-1], b[1:]):
        c, u = 0, u0
        while u < u1:
            s, y0 = divmod(int(u), Ny)
            y1 = min(Ny, y0 + int(u1 - u))
            c += w[s] * (y1 - y0) + (16 * warm if y0 == 0 else 0)
            u += y1 - y0
        costs.append(c)
    return np.array(costs)


@pytest.mark.parametrize("Nx,Ny,K,G,precision", [(8192, 8192, 2, 304, "fp32"), (4096, 4096, 4, 152, "fp32"),
                                                 (1024, 1024, 4, 152, "fp32"), (1000, 777, 2, 304, "fp32"),
                                                 (8192, 8192, 2, 304, "fp64"), (300, 40, 1, 152, "fp32"),
                                                 (240, 3, 2, 5, "fp32"), (7, 5, 2, 1, "fp64")])
def test_shares_tile_the_units_with_equal_cost(Nx, Ny, K, G, precision):
    b = qla.sweep_split(Nx, Ny, K, G, precision)
    nsx, w, warm = model(Nx, Ny, K, precision)
    assert b.size == G + 1 and b[0] == 0 and b[-1] == nsx * Ny and np.all(np.diff(b) >= 0)
    costs = share_costs(b, Ny, w, warm)
    total = sum(16 * warm + w[s] * Ny for s in range(nsx))
    assert costs.sum() == total
    # a bound lands on the first unit whose cost prefix reaches its ideal
    # position: off by less than one row's cost, or by a strip's warm-up
    slack = max(w) + 16 * warm
    assert np.all(np.abs(costs - total / G) <= 2 * slack), (costs.min(), costs.max(), total / G)


def test_slow_strips_are_the_ones_that_wrap():
    # 8192 columns at K = 2: strips of 240 outputs; strip 0 starts at column
    # -8 and strip 34 ends past 8192, so both copy with cp.async
    nsx, w, _ = model(8192, 8192, 2, "fp32")
    assert nsx == 35 and w[0] == w[34] == 32 and all(x == 16 for x in w[1:34])
    b = qla.sweep_split(8192, 8192, 2, 304)
    first = b[1] - b[0]
    mid = np.median(np.diff(b))
    assert first < 0.6 * mid  # a slow strip's share holds about half the rows


def test_rejects_bad_arguments():
    with pytest.raises(qla.QLAError):
        qla.sweep_split(0, 8, 2, 4)
    with pytest.raises(qla.QLAError):
        qla.sweep_split(64, 64, 3, 4)  # K = 3 is not instantiated
    with pytest.raises(qla.QLAError):
        qla.sweep_split(64, 64, 4, 4, "fp64")  # FP64 has K = 1, 2
    with pytest.raises(qla.QLAError):
        qla.sweep_split(64, 64, 2, 0)


def test_split_needs_no_gpu():
    host_checks.run_without_gpu("sweep_split_is_host_arithmetic")
