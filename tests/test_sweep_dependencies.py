"""Host-side checks of the persistent launch form's dependency lists
(qla_sweep_dependencies), with no GPU.

In the persistent form CTA b sweeps share b of a family in every pass and,
before a pass, waits only for the shares listed here instead of for the whole
previous pass. The list must hold every share whose previous pass wrote a
cell that share b reads (read after write) or read a cell that share b
overwrites (write after read, the two state buffers alternating). These tests
build, cell by cell, which share writes each cell and which cells each share
reads, from the kernel's strip geometry (the seam layout: strip 0 reads
columns [Nx - 128, Nx + 128) mod Nx and writes the 256 - 8K in their middle;
strip s >= 1 writes 240 columns from 128 - 4K + 240 (s - 1), up to
Nx - 128 + 4K, and reads 256 from 4K before them, moved left to end at Nx at
the latest) and its row reach (a segment of rows [y0, y1) reads rows
[y0 - 4K, y1 + 4K + R - 1), R = 4, periodic), and check that every pair of
shares that meet this way lists each other. They also check that the writes
tile the lattice exactly once and that the lists stay local (a share waits
for its halo neighbours, not for the lattice).
"""
import numpy as np
import pytest

from paper_2301_13601_gb300 import qla

K, R, W_IN = 2, 4, 256
H = 4 * K


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


def strip_geometry(Nx, s):
    """(read columns, written columns) of strip s as index arrays mod Nx."""
    wv = W_IN - 2 * H
    if s == 0:
        rd = (Nx - W_IN // 2 + np.arange(W_IN)) % Nx
        wr = (Nx - W_IN // 2 + H + np.arange(W_IN - 2 * H)) % Nx
    else:
        o_lo = W_IN // 2 - H + (s - 1) * wv
        o_hi = min(o_lo + wv, Nx - W_IN // 2 + H)
        xb = min(o_lo - H, Nx - W_IN)
        rd = (xb + np.arange(W_IN)) % Nx
        wr = np.arange(o_lo, o_hi) % Nx
    return rd, wr


def segments(b0, b1, Ny):
    u = b0
    while u < b1:
        s, y0 = divmod(u, Ny)
        y1 = min(Ny, y0 + (b1 - u))
        yield s, y0, y1
        u += y1 - y0


def check(Nx, Ny, G, family, max_deps=None):
    nsx = 1 + -(-(Nx - W_IN + 2 * H) // (W_IN - 2 * H))
    bounds = qla.sweep_split(Nx, Ny, K, G, "fp32", family, layers=1)
    assert bounds[0] == 0 and bounds[-1] == nsx * Ny
    writer = np.full((Ny, Nx), -1, dtype=np.int32)
    for b in range(G):
        for s, y0, y1 in segments(int(bounds[b]), int(bounds[b + 1]), Ny):
            _, wr = strip_geometry(Nx, s)
            block = writer[y0:y1][:, wr]
            assert np.all(block == -1), "a cell written twice"
            writer[np.ix_(np.arange(y0, y1), wr)] = b
    assert np.all(writer >= 0), "a cell nobody writes"
    deps = [set(qla.sweep_dependencies(Nx, Ny, K, G, b, family).tolist()) for b in range(G)]
    for b in range(G):
        assert b not in deps[b]
        for d in deps[b]:
            assert b in deps[d], "the relation is symmetric"
        if max_deps is not None:
            assert len(deps[b]) <= max_deps
    for d in range(G):
        readers_of = set()
        for s, z0, z1 in segments(int(bounds[d]), int(bounds[d + 1]), Ny):
            rd, _ = strip_geometry(Nx, s)
            rows = np.arange(z0 - H, z1 + H + R - 1) % Ny
            readers_of |= set(np.unique(writer[np.ix_(rows, rd)]).tolist())
        readers_of.discard(d)
        missing = readers_of - deps[d]
        assert not missing, f"share {d} reads cells of shares {sorted(missing)} it does not wait for"
    return deps


@pytest.mark.parametrize("family", ["TM", "TE"])
def test_dependencies_cover_every_halo_neighbour_2048(family):
    deps = check(2048, 2048, 304, family, max_deps=12)
    assert max(len(d) for d in deps) >= 3


def test_dependencies_8192_stay_local():
    # the bench lattice: 35 strips of 8192 rows, 304 shares of ~943 rows
    check(8192, 8192, 304, "TM", max_deps=12)


@pytest.mark.parametrize("Nx,Ny,G", [
    (256, 300, 304),   # the seam strip and one clamped strip
    (1000, 64, 304),   # short strips: windows wrap around y
    (520, 7, 13),      # fewer rows than a window: whole strips depend
    (4096, 32, 304),   # shares spanning several strips
    (2056, 1500, 77),  # ragged last strip, few shares
])
def test_dependencies_edge_lattices(Nx, Ny, G):
    check(Nx, Ny, G, "TE")


def test_dependencies_argument_checks():
    with pytest.raises(qla.QLAError):
        qla.sweep_dependencies(1000, 100, 4, 304, 0)  # only 2 steps per pass are built
    with pytest.raises(qla.QLAError):
        qla.sweep_dependencies(1004, 100, 2, 304, 0)  # Nx not a multiple of 8: no seam layout
    with pytest.raises(qla.QLAError):
        qla.sweep_dependencies(1000, 100, 2, 304, 304)  # share out of range
    with pytest.raises(qla.QLAError):
        qla.sweep_dependencies(1000, 100, 2, 5000, 0)  # more shares than the counters hold
