"""Host-side checks of the strips and balanced split of a sweep pass
(qla_sweep_split).

With chunk_rows = 0 a pass launches one CTA per resident slot and family;
CTA b sweeps the row units [bounds[b], bounds[b + 1]) (u = strip * Ny + y) as
one segment per strip it touches. The bounds come from the library's host
arithmetic, the same code the kernel runs per CTA. These tests check, with no
GPU visible, the strip count of both layouts (FP32 with K >= 2, Nx a multiple
of 8 and at least 256: strip 0 straddles the periodic seam and strips of
256 - 8K outputs cover the columns between; otherwise strips of 256 - 8K
outputs from column 0), that the shares tile the units exactly, and that
their costs (one per row, plus the warm-up rows 8K + R (K - 1) at each strip
start) agree within one strip start's warm-up.
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
    """Strip count and warm-up rows of the documented layout."""
    wv = W_IN - 8 * K
    R = 8 if (precision == "fp32" and K == 1) else 4
    seam = precision == "fp32" and Nx % 8 == 0 and Nx >= W_IN and K >= 2
    nsx = 1 + -(-(Nx - W_IN + 8 * K) // wv) if seam else -(-Nx // wv)
    return nsx, 8 * K + R * (K - 1)


def share_costs(b, Ny, warm):
    """Cost of each share: its rows, plus the warm-up of every strip start it holds."""
    costs = []
    for u0, u1 in zip(b[:-1], b[1:]):
        c, u = 0, int(u0)
        while u < u1:
            s, y0 = divmod(u, Ny)
            y1 = min(Ny, y0 + int(u1 - u))
            c += (y1 - y0) + (warm if y0 == 0 else 0)
            u += y1 - y0
        costs.append(c)
    return np.array(costs)


@pytest.mark.parametrize("Nx,Ny,K,G,precision", [(8192, 8192, 2, 304, "fp32"), (4096, 4096, 4, 152, "fp32"),
                                                 (1024, 1024, 4, 152, "fp32"), (1000, 777, 2, 304, "fp32"),
                                                 (8192, 8192, 2, 304, "fp64"), (300, 40, 1, 152, "fp32"),
                                                 (240, 3, 2, 5, "fp32"), (7, 5, 2, 1, "fp64"),
                                                 (256, 64, 2, 304, "fp32"), (1004, 50, 2, 40, "fp32")])
def test_shares_tile_the_units_with_equal_cost(Nx, Ny, K, G, precision):
    b = qla.sweep_split(Nx, Ny, K, G, precision)
    nsx, warm = model(Nx, Ny, K, precision)
    assert b.size == G + 1 and b[0] == 0 and b[-1] == nsx * Ny and np.all(np.diff(b) >= 0)
    costs = share_costs(b, Ny, warm)
    total = nsx * (Ny + warm)
    assert costs.sum() == total
    # a bound lands where its ideal cost position falls, except inside a
    # strip's warm-up, where it moves to the strip's first row
    assert np.all(np.abs(costs - total / G) <= warm + 1), (costs.min(), costs.max(), total / G)


def test_seam_layout_strip_count():
    # 8192 columns at K = 2: the seam strip writes [8072, 8192) and [0, 120);
    # 34 strips of 240 cover the 7952 columns between
    assert model(8192, 8192, 2, "fp32")[0] == 35
    assert qla.sweep_split(8192, 8192, 2, 1)[-1] == 35 * 8192
    # the plain layout: 8192 / 240 -> 35 strips as well; 1000 columns (not a
    # multiple of 8) -> 5 strips; 1000 + 4 -> seam strip + 4
    assert qla.sweep_split(1000, 10, 2, 1)[-1] == 5 * 10
    assert qla.sweep_split(1004, 10, 2, 1)[-1] == (1 + 4) * 10


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
