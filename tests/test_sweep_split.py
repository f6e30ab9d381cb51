"""Host-side checks of the strips and balanced split of a sweep pass
(qla_sweep_split).

With chunk_rows = 0 a pass launches one CTA per resident slot and family;
the CTA holding share b sweeps the row units [bounds[b], bounds[b + 1])
(u = strip * Ny + y) as one segment per strip it touches. The bounds come
from the library's host arithmetic, the same code the kernel runs per CTA.
These tests check, with no GPU visible, the strip count of both layouts (FP32
with K >= 2, Nx a multiple of 8 and at least 256: strip 0 straddles the
periodic seam and strips of 256 - 8K outputs cover the columns between;
otherwise strips of 256 - 8K outputs from column 0), that the shares tile
the units exactly, and the bounds against a Python restatement of the
documented cost model: 16 per row (the seam strip's rows 18 for TM, 19 for
TE), 16 x (8K + R (K - 1)) warm-up at each strip start, shares weighted by
profile (one layer or the first of two: the first half 1 + 3/64, the second
1 - 3/64; the second of two layers: linearly from 1 + 6/64 down to 1 - 6/64),
the constants the library measured.
"""
import numpy as np
import pytest

import host_checks
from paper_2301_13601_gb300 import qla

W_IN = 256
SEAM_COST = {"TM": 18, "TE": 19}
OLDER64, SLOPE64 = 3, 6


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


def layout(Nx, K, precision):
    wv = W_IN - 8 * K
    seam = precision == "fp32" and Nx % 8 == 0 and Nx >= W_IN and K >= 2
    nsx = 1 + -(-(Nx - W_IN + 8 * K) // wv) if seam else -(-Nx // wv)
    R = 8 if (precision == "fp32" and K == 1) else 4
    return seam, nsx, 8 * K + R * (K - 1)


def model_bounds(Nx, Ny, K, G, precision, family, layers):
    """The documented split, in integer arithmetic."""
    seam, nsx, warm = layout(Nx, K, precision)
    w0 = SEAM_COST[family] if seam else 16
    c0 = 16 * warm + w0 * Ny
    per = 16 * (Ny + warm)
    C = c0 + (nsx - 1) * per
    profile = 2 if (layers == 2 and family == "TE") else 1

    def unit(c):
        if c < c0:
            r = c - 16 * warm
            return 0 if r <= 0 else r // w0
        s = 1 + (c - c0) // per
        if s >= nsx:
            return nsx * Ny
        r = c - c0 - (s - 1) * per - 16 * warm
        return s * Ny + (0 if r <= 0 else r // 16)

    out = []
    for b in range(G + 1):
        num, den = b, G
        if profile == 1 and G % 2 == 0:
            H = G // 2
            num = b * (64 + OLDER64) if b <= H else H * (64 + OLDER64) + (b - H) * (64 - OLDER64)
            den = 64 * G
        elif profile == 2 and G >= 2:
            num = 64 * (G - 1) * b + SLOPE64 * b * (G - b)
            den = 64 * G * (G - 1)
        out.append(unit(C // den * num + C % den * num // den))
    return np.array(out)


CASES = [(8192, 8192, 2, 304, "fp32"), (4096, 4096, 4, 152, "fp32"), (1024, 1024, 4, 152, "fp32"),
         (1000, 777, 2, 304, "fp32"), (8192, 8192, 2, 304, "fp64"), (300, 40, 1, 152, "fp32"),
         (240, 3, 2, 5, "fp32"), (7, 5, 2, 1, "fp64"), (256, 64, 2, 304, "fp32"), (1004, 50, 2, 40, "fp32")]


@pytest.mark.parametrize("Nx,Ny,K,G,precision", CASES)
@pytest.mark.parametrize("family,layers", [("TM", 2), ("TE", 2), ("TM", 1), ("TE", 1)])
def test_shares_tile_the_units_as_documented(Nx, Ny, K, G, precision, family, layers):
    b = qla.sweep_split(Nx, Ny, K, G, precision, family, layers)
    _, nsx, _ = layout(Nx, K, precision)
    assert b.size == G + 1 and b[0] == 0 and b[-1] == nsx * Ny and np.all(np.diff(b) >= 0)
    assert np.array_equal(b, model_bounds(Nx, Ny, K, G, precision, family, layers))


def test_share_profiles_at_8192():
    N = 8192
    tm = np.diff(qla.sweep_split(N, N, 2, 304, "fp32", "TM", 2)).astype(float)
    te = np.diff(qla.sweep_split(N, N, 2, 304, "fp32", "TE", 2)).astype(float)
    # first layer: the first 152 shares (past the seam strip's) 67/61 of the last 152
    assert abs(np.median(tm[20:152]) / np.median(tm[152:]) - 67 / 61) < 0.01
    # second layer: rows fall linearly with the start order (weights 1 + a (1 - 2b / 303), a = 6/64)
    w = lambda b: 1 + (1 - 2 * b / 303) * 6 / 64
    assert abs(np.median(te[20:30]) / np.median(te[290:300]) - w(25) / w(295)) < 0.02
    # the seam strip's shares (strip 0, the first shares) hold 16/18 (TM) of the rows per cost
    assert abs(np.median(tm[1:8]) / np.median(tm[20:30]) - 16 / 18) < 0.02


def test_seam_layout_strip_count():
    # 8192 columns at K = 2: the seam strip writes [8072, 8192) and [0, 120);
    # 34 strips of 240 cover the 7952 columns between
    assert layout(8192, 2, "fp32")[1] == 35
    assert qla.sweep_split(8192, 8192, 2, 1)[-1] == 35 * 8192
    # the plain layout: 1000 columns (not a multiple of 8) -> 5 strips;
    # 1000 + 4 -> the seam strip + 4
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
    with pytest.raises(qla.QLAError):
        qla.sweep_split(64, 64, 2, 4, layers=3)


def test_split_needs_no_gpu():
    host_checks.run_without_gpu("sweep_split_is_host_arithmetic")
