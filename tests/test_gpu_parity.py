"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances:
  FP64 mode: relative L2 <= 1e-12 (the GPU evaluates the same rotations in a
             different rounding order: ~1e-16 per operation).
  FP32 mode: per step ~64 roundings of relative size 2^-24 per component, so
             the relative L2 error grows like sqrt(steps) * 1e-7 to 1e-6;
             bounds below are stated per test.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2301_13601_gb300 import media
from paper_2301_13601_gb300.qla import QLAError, Simulation

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def gpu_run(n, q0, delta, steps, **kw):
    with Simulation(*n, delta, **kw) as sim:
        sim.set_fields(q0)
        sim.step(steps)
        return sim.get_fields()


def oracle_run(n, q0, delta, steps, sequence="interleaved", potential="paper"):
    theta, beta = oracle.angles(*n, delta)
    q = np.array(q0, dtype=np.float64, copy=True)
    oracle.run(q, theta, beta, steps, oracle.SEQ_INTERLEAVED if sequence == "interleaved" else oracle.SEQ_PLAIN,
               oracle.POT_PAPER if potential == "paper" else oracle.POT_UNITARY)
    return q


# lattice shapes (Nx, Ny, rows per tile; 0 = the balanced split): several
# strips with a ragged tail and several row chunks, the same under the
# balanced split (shares spanning strips), odd sizes (scalar-load path), a
# tiny lattice narrower than a strip (fewer row units than CTA slots)
SHAPES = [(500, 70, 24), (500, 70, 0), (37, 53, 0), (8, 5, 0), (64, 64, 16)]


def problem(Nx, Ny, seed=3):
    n = media.smooth_periodic_medium(Nx, Ny, seed=seed, amp=0.3)
    q0 = media.smooth_periodic_field(Nx, Ny, seed + 10)
    # add small-scale structure so that every shift matters
    q0 += 0.1 * np.random.default_rng(seed).standard_normal(q0.shape)
    return n, q0


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("K", [1, 2])
@pytest.mark.parametrize("sequence", ["interleaved", "plain"])
@pytest.mark.parametrize("potential", ["paper", "unitary"])
def test_fp64_matches_oracle(shape, K, sequence, potential):
    Nx, Ny, chunk = shape
    n, q0 = problem(Nx, Ny)
    delta, steps = 0.2, 2 * K + 1
    got = gpu_run(n, q0, delta, steps, precision="fp64", steps_per_pass=K, chunk_rows=chunk,
                  sequence=sequence, potential=potential)
    ref = oracle_run(n, q0, delta, steps, sequence, potential)
    assert rel_l2(got, ref) < 1e-12


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("K", [1, 2, 4])
@pytest.mark.parametrize("sequence", ["interleaved", "plain"])
@pytest.mark.parametrize("potential", ["paper", "unitary"])
def test_fp32_matches_oracle(shape, K, sequence, potential):
    Nx, Ny, chunk = shape
    n, q0 = problem(Nx, Ny)
    delta, steps = 0.2, 3 * K + 1
    got = gpu_run(n, q0, delta, steps, precision="fp32", steps_per_pass=K, chunk_rows=chunk,
                  sequence=sequence, potential=potential)
    ref = oracle_run(n, q0, delta, steps, sequence, potential)
    assert rel_l2(got, ref) < 3e-6


@pytest.mark.parametrize("K", [2, 4])
@pytest.mark.parametrize("sequence", ["interleaved", "plain"])
@pytest.mark.parametrize("potential", ["paper", "unitary"])
@pytest.mark.parametrize("chunk", [40, 0])
def test_fp32_tma_strips_match_oracle(K, sequence, potential, chunk):
    """Nx a multiple of 8 and several strips: the inner strips load their rows
    with TMA, the two that wrap around x with cp.async; both must agree with
    the oracle (rows in tiles of 40 with a ragged last tile, or the balanced
    split: shares that start and end inside strips and span strip ends)."""
    Nx, Ny = 1024, 96
    n, q0 = problem(Nx, Ny, seed=5)
    delta, steps = 0.2, 3 * K + 1
    got = gpu_run(n, q0, delta, steps, precision="fp32", steps_per_pass=K, chunk_rows=chunk,
                  sequence=sequence, potential=potential)
    ref = oracle_run(n, q0, delta, steps, sequence, potential)
    assert rel_l2(got, ref) < 3e-6


@pytest.mark.parametrize("K", [2, 4])
@pytest.mark.parametrize("Ny, chunk", [(100, 40), (96, 37), (98, 24)])
def test_fp32_tma_block_boxes_match_oracle(K, Ny, chunk):
    """The TMA copies load whole R-row blocks, and one box for the blocks of
    all levels of a coefficient plane when they lie in one group of R + 4
    rows. Cases: Ny not a multiple of R + 4 (no merged view: one box per
    level), tiles of 37 rows (level blocks straddling a row group in every
    other iteration), Ny not a multiple of R (blocks at the y-wrap loaded
    row by row)."""
    Nx = 1024
    n, q0 = problem(Nx, Ny, seed=7)
    delta, steps = 0.2, 3 * K + 1
    got = gpu_run(n, q0, delta, steps, precision="fp32", steps_per_pass=K, chunk_rows=chunk)
    ref = oracle_run(n, q0, delta, steps, "interleaved", "paper")
    assert rel_l2(got, ref) < 3e-6


@pytest.mark.parametrize("Nx, Ny, chunk, K", [(256, 40, 0, 2), (264, 30, 0, 2), (512, 37, 0, 4), (744, 50, 16, 2),
                                              (2048, 21, 0, 2), (496, 64, 24, 4)])
@pytest.mark.parametrize("sequence", ["interleaved", "plain"])
def test_fp32_seam_layout_matches_oracle(Nx, Ny, chunk, K, sequence):
    """FP32, Nx a multiple of 8 and at least 256, K >= 2: strip 0 straddles
    the periodic seam and loads its two 128-column halves with one TMA box
    each (landing swapped in shared memory); the last strip's input is moved
    left to end at Nx. Cases: Nx = 256 (the seam strip and one strip over 16
    columns), a last strip clamped against the right edge, Ny not a multiple
    of R (boxes at the y-wrap loaded row by row), tiles and the balanced split."""
    n, q0 = problem(Nx, Ny, seed=13)
    delta, steps = 0.2, 3 * K + 1
    got = gpu_run(n, q0, delta, steps, precision="fp32", steps_per_pass=K, chunk_rows=chunk, sequence=sequence)
    ref = oracle_run(n, q0, delta, steps, sequence, "paper")
    assert rel_l2(got, ref) < 3e-6


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("Nx, Ny", [(1000, 777), (2048, 300)])
def test_balanced_split_equals_tiles_bit_exact(precision, Nx, Ny):
    """Every output site is computed by the same operations in the same order
    whichever CTA sweeps it (a tile or a share of the balanced split, warm-up
    rows included), so the two launch forms agree bit for bit."""
    n, q0 = problem(Nx, Ny, seed=11)
    K = 2
    a = gpu_run(n, q0, 0.2, 4 * K, precision=precision, steps_per_pass=K, chunk_rows=0)
    b = gpu_run(n, q0, 0.2, 4 * K, precision=precision, steps_per_pass=K, chunk_rows=56)
    assert np.array_equal(a, b)


def test_balanced_split_covers_the_units():
    """The context's split: one share per resident slot (two 112 KB CTAs per
    SM at 2 steps per pass), bounds tiling the strips x rows, and a context
    with chunk_rows set reports no split."""
    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n, q0 = problem(2048, 300, seed=2)
    with Simulation(*n, 0.2, precision="fp32", steps_per_pass=2) as sim:
        b = sim.sweep_split()
        nsx = 1 + -(-(2048 - 256 + 16) // 240)  # the seam strip and the strips between
        assert b is not None and b[0] == 0 and b[-1] == nsx * 300 and np.all(np.diff(b) >= 0)
        assert b.size - 1 == 2 * sms
    with Simulation(*n, 0.2, precision="fp32", steps_per_pass=2, chunk_rows=64) as sim:
        assert sim.sweep_split() is None and sim.chunk_rows == 64


def test_pulse_init_matches_oracle():
    for pol, name in ((0, "Ez"), (1, "Ey")):
        Nx, Ny = 300, 20
        n = media.uniform_medium(Nx, Ny, (1.0, 1.0, 1.0))
        with Simulation(*n, 0.1, precision="fp64") as sim:
            sim.init_pulse(name, 250.5, 30.0, -0.8)
            got = sim.get_fields()
        ref = oracle.init_pulse(Nx, Ny, pol, 250.5, 30.0, -0.8)
        assert np.abs(got - ref).max() < 1e-15


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_cylinder_256_full_run(precision):
    """256^2, delta 0.1, 400 steps, cylinder R 30, E_z pulse: the full workload."""
    w = media.workload_cylinder_256()
    n = w.medium()
    theta, beta = oracle.angles(*n, w.delta)
    ref = oracle.init_pulse(w.Nx, w.Ny, w.pulse.pol, w.pulse.x0, w.pulse.sigma, w.pulse.amp)
    oracle.run(ref, theta, beta, w.steps)
    with Simulation(*n, w.delta, precision=precision) as sim:
        sim.init_pulse("Ez", w.pulse.x0, w.pulse.sigma, w.pulse.amp)
        sim.step(w.steps)
        got = sim.get_fields()
        e = sim.energy()
        dv = sim.divB()
    E0 = oracle.energy(oracle.init_pulse(w.Nx, w.Ny, 0, w.pulse.x0, w.pulse.sigma, w.pulse.amp))
    if precision == "fp64":
        assert rel_l2(got, ref) < 1e-12
        # energy is quadratic in the fields: twice the field tolerance
        assert abs(e - oracle.energy(ref)) / E0 < 2e-12
        od = oracle.divB(ref)
        assert abs(dv[0] - od[0]) <= 1e-10 * od[0] and abs(dv[1] - od[1]) <= 1e-12 and abs(dv[2] - od[2]) <= 1e-12
    else:
        assert rel_l2(got, ref) < 2e-5
        assert abs(e - oracle.energy(ref)) / E0 < 2e-6


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_diagnostics_match_oracle(precision):
    Nx, Ny = 333, 121
    rng = np.random.default_rng(5)
    q = rng.standard_normal((6, Ny, Nx))
    if precision == "fp32":
        q = q.astype(np.float32).astype(np.float64)
    n = media.uniform_medium(Nx, Ny, (1.2, 1.3, 1.4))
    with Simulation(*n, 0.1, precision=precision) as sim:
        sim.set_fields(q)
        d = sim.diagnostics()
    assert d["nonfinite"] == 0
    assert abs(d["energy"] - oracle.energy(q)) <= 1e-14 * oracle.energy(q)
    s, m, b = oracle.divB(q)
    assert abs(d["div_l2_sq"] - s) <= 1e-13 * s
    assert abs(d["div_max"] - m) <= 1e-14 * m
    assert abs(d["b_max"] - b) <= 1e-14 * b


@pytest.mark.parametrize("scale", [1e-30, 1e25, "mixed"])
def test_diagnostics_extreme_values_fp32(scale):
    """FP32 states whose values leave [2^-60, 2^60) (where FP32 squares would
    underflow or overflow) are reduced with FP64 squares: the energy and the
    other statistics still agree with the oracle."""
    Nx, Ny = 300, 77
    rng = np.random.default_rng(15)
    q = rng.standard_normal((6, Ny, Nx))
    if scale == "mixed":
        q[:, ::7, ::5] *= 1e22
        q[:, 1::9, ::3] *= 1e-24
    else:
        q *= scale
    q = q.astype(np.float32).astype(np.float64)
    n = media.uniform_medium(Nx, Ny, (1.2, 1.3, 1.4))
    with Simulation(*n, 0.1, precision="fp32") as sim:
        sim.set_fields(q)
        d = sim.diagnostics()
    assert d["nonfinite"] == 0
    assert abs(d["energy"] - oracle.energy(q)) <= 1e-14 * oracle.energy(q)
    s, m, b = oracle.divB(q)
    assert abs(d["div_l2_sq"] - s) <= 1e-13 * s
    assert abs(d["div_max"] - m) <= 1e-14 * m
    assert abs(d["b_max"] - b) <= 1e-14 * b


def test_diagnostics_deterministic():
    Nx, Ny = 1000, 700
    q = np.random.default_rng(9).standard_normal((6, Ny, Nx))
    n = media.uniform_medium(Nx, Ny, (1.2, 1.3, 1.4))
    with Simulation(*n, 0.1) as sim:
        sim.set_fields(q)
        a = [sim.diagnostics()["energy"] for _ in range(3)]
    assert a[0] == a[1] == a[2]


@pytest.mark.parametrize("family", ["TE", "TM"])
def test_families_never_couple_bit_exact(family):
    Nx, Ny = 300, 90
    n, q0 = problem(Nx, Ny, seed=7)
    te, tm = [0, 1, 5], [2, 3, 4]
    zero = tm if family == "TE" else te
    q0[zero] = 0.0
    for pot in ("paper", "unitary"):
        got = gpu_run(n, q0, 0.2, 17, precision="fp32", potential=pot)
        assert all(np.abs(got[c]).max() == 0.0 for c in zero)


def test_unitary_fp32_energy_drift_small():
    """All operators orthogonal: FP32 energy drift is rounding only."""
    w = media.workload_cylinder_256()
    n = w.medium()
    with Simulation(*n, w.delta, precision="fp32", potential="unitary") as sim:
        sim.init_pulse("Ez", w.pulse.x0, w.pulse.sigma, 1.0)
        e0 = sim.energy()
        sim.step(2000)
        e1 = sim.energy()
    assert abs(e1 / e0 - 1) < 2e-6


def test_nonfinite_state_is_reported():
    Nx, Ny = 64, 32
    n = media.uniform_medium(Nx, Ny, (1.2, 1.3, 1.4))
    q = np.zeros((6, Ny, Nx))
    q[3, 5, 7] = np.nan
    q[1, 2, 3] = np.inf
    with Simulation(*n, 0.1) as sim:
        sim.set_fields(q)
        d = sim.diagnostics()
        assert d["status"] == "QLA_ENONFINITE" and d["nonfinite"] == 2
        sim.step(4)  # the context stays usable (not sticky)
        sim.set_fields(np.zeros((6, Ny, Nx)))
        assert sim.diagnostics()["status"] == "QLA_OK"


def test_invalid_arguments_raise():
    Nx, Ny = 16, 16
    n = media.uniform_medium(Nx, Ny, (1.2, 1.3, 1.4))
    with pytest.raises(QLAError):
        Simulation(*n, 0.0)
    with pytest.raises(QLAError):
        Simulation(*n, 0.1, steps_per_pass=3)
    with Simulation(*n, 0.1) as sim:
        with pytest.raises(QLAError):
            sim.step(-1)
        with pytest.raises(QLAError):
            sim.init_pulse("Ez", 3.0, -1.0)
        sim.step(1)


def test_step_count_and_zero_steps():
    n, q0 = problem(40, 40)
    with Simulation(*n, 0.2) as sim:
        sim.set_fields(q0)
        sim.step(0)
        assert sim.step_count == 0
        assert rel_l2(sim.get_fields(), q0.astype(np.float32).astype(np.float64)) == 0.0
        sim.step(7)
        assert sim.step_count == 7


# ---------------------------------------------------------------------------
# Full-size workload, in the launch configuration the benchmark times, on
# sampled sites the oracle computes from a local window (the dependency radius
# of one step is 4 sites along each axis, so after s steps a site depends only
# on the (8s+1)^2 window around it).
# ---------------------------------------------------------------------------

def window(a, yc, xc, H):
    Ny, Nx = a.shape[-2:]
    ys = np.arange(yc - H, yc + H + 1) % Ny
    xs = np.arange(xc - H, xc + H + 1) % Nx
    return np.ascontiguousarray(a[..., ys[:, None], xs[None, :]])


def share_seams(sim, Ny, shares, W=240):
    """(row, column) sites on the seam between share b - 1 and share b of the
    balanced split, for each b in shares: the first row of share b, in the
    middle of its strip's columns. Seam layout at 2 steps per pass: strip 0
    writes columns [Nx - 120, Nx) and [0, 120), strip s >= 1 the W = 240
    columns from 120 + (s - 1) W, so strip s is centred on column s W."""
    bounds = sim.sweep_split()
    out = []
    for b in shares:
        s, y = divmod(int(bounds[b]), Ny)
        out.append((y, s * W))
    return out


def test_cylinders_8192_sampled_parity():
    w = media.workload_cylinders_8192()
    n = w.medium()
    steps = 8  # four fused passes of 2 steps, the automatic configuration at this size
    with Simulation(*n, w.delta, precision="fp32") as sim:
        assert sim.steps_per_pass == 2 and sim.chunk_rows == 0
        seams = share_seams(sim, 8192, [1, 2, 40, 157, 303])
        sim.init_pulse("Ez", w.pulse.x0, w.pulse.sigma, w.pulse.amp)
        q0 = sim.get_fields()
        sim.step(steps)
        got = sim.get_fields(dtype=np.float32)
    H = 4 * steps + 8
    # sample sites: pulse flank, object edges, lattice corners (periodic wrap,
    # inside the seam strip), strip seams (strip s >= 1 writes the 240 columns
    # from 120 + 240 (s - 1); the seam strip the 120 either side of x = 0) and
    # the seams between the CTA shares of the balanced split
    obj = w.objects[0]
    samples = [(4096, 1024 + 100), (0, 0), (8191, 8191), (int(obj.cy), int(obj.cx - obj.a)),
               (int(obj.cy + obj.b), int(obj.cx)), (1234, 360), (4096, 359), (8000, 8180), (5000, 8072),
               (6000, 119)] + seams
    for yc, xc in samples:
        nw = tuple(window(a, yc, xc, H) for a in n)
        qw = window(q0, yc, xc, H)
        ref = oracle_run(nw, qw, w.delta, steps)
        r = 3
        a = window(got, yc, xc, r)
        b = ref[:, H - r:H + r + 1, H - r:H + r + 1]
        scale = max(np.abs(b).max(), 1e-3)
        assert np.abs(a - b).max() <= 2e-6 * scale + 1e-12, (yc, xc)


def test_cylinders_8192_sampled_parity_200_steps():
    """The first 200 steps of the 8192^2 workload in the benchmark's launch
    configuration, on five sampled windows where the pulse is (the dependency
    window after 200 steps is 1601^2 sites): the pulse flank, a share seam, a
    strip seam, the periodic y-wrap and the pulse's far flank. FP32 bound:
    about 64 roundings of 2^-24 per component and step, a random walk of
    6e-8 * sqrt(64 * 200) = 7e-6 of the local amplitude; 1e-5 is asserted."""
    w = media.workload_cylinders_8192()
    n = w.medium()
    steps = 200
    with Simulation(*n, w.delta, precision="fp32") as sim:
        assert sim.steps_per_pass == 2
        bounds = sim.sweep_split()
        sim.init_pulse("Ez", w.pulse.x0, w.pulse.sigma, w.pulse.amp)
        q0 = sim.get_fields()
        sim.step(steps)
        got = sim.get_fields(dtype=np.float32)
    H = 4 * steps + 8
    x0 = int(w.pulse.x0)
    # a share seam inside the pulse's strip: the first share that starts in it below row 4096
    strip = (x0 - 40 + 120) // 240  # seam layout (see share_seams)
    seam = next(int(u) % 8192 for u in bounds if int(u) // 8192 == strip and int(u) % 8192 > 4096)
    samples = [(4096, x0 + 60), (seam, x0 - 40), (3000, 1080), (0, x0 + 10), (8191, x0 - 120)]
    for yc, xc in samples:
        nw = tuple(window(a, yc, xc, H) for a in n)
        qw = window(q0, yc, xc, H)
        ref = oracle_run(nw, qw, w.delta, steps)
        r = 3
        a = window(got, yc, xc, r)
        b = ref[:, H - r:H + r + 1, H - r:H + r + 1]
        scale = max(np.abs(b).max(), 1e-3)
        err = np.abs(a - b).max() / scale
        print(f"window ({yc}, {xc}): max error {err:.2e} of the local amplitude {scale:.3e}")
        assert err <= 1e-5, (yc, xc)
