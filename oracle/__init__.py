"""ctypes binding of the plain FP64 CPU oracle (``qla_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers. The CUDA product path
never imports this package and shares no code with it.

Every function follows one equation of arXiv 2301.13601; the docstrings name it.
Arrays are float64, C-contiguous; state ``q`` has shape (6, Ny, Nx) holding
Q = (n_x E_x, n_y E_y, n_z E_z, B_x, B_y, B_z) (Eq. 15).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

# Idle OpenMP threads sleep instead of spinning, so that the oracle does not
# starve (or get starved by) other processes sharing the host cores.
os.environ.setdefault("OMP_WAIT_POLICY", "PASSIVE")

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qla_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

POT_PAPER = 0
POT_UNITARY = 1
SEQ_INTERLEAVED = 0
SEQ_PLAIN = 1
POL_EZ = 0
POL_EY = 1

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
               "-shared", "-std=c11", "-Wall", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            d = ctypes.POINTER(ctypes.c_double)
            i = ctypes.c_int
            L.orc_version.restype = i
            L.orc_set_threads.argtypes = [i]
            L.orc_get_threads.restype = i
            L.orc_angles.argtypes = [i, i, d, d, d, ctypes.c_double, d, d]
            L.orc_collide_x.argtypes = [i, i, d, d, i]
            L.orc_collide_y.argtypes = [i, i, d, d, i]
            L.orc_stream.argtypes = [i, i, d, i, i, i, i]
            L.orc_potential_x.argtypes = [i, i, d, d, ctypes.c_double, i]
            L.orc_potential_y.argtypes = [i, i, d, d, ctypes.c_double, i]
            L.orc_collide_stream.argtypes = [i, i, i, d, d, d, i, ctypes.c_double, i]
            L.orc_step.argtypes = [i, i, d, d, d, i, i]
            L.orc_run.argtypes = [i, i, d, d, d, i, i, ctypes.c_longlong]
            L.orc_energy.argtypes = [i, i, d]
            L.orc_energy.restype = ctypes.c_double
            L.orc_divB.argtypes = [i, i, d, d]
            L.orc_divD.argtypes = [i, i, d, d, d, d, d]
            L.orc_init_pulse.argtypes = [i, i, d, i, ctypes.c_double, ctypes.c_double, ctypes.c_double]
            L.orc_yee_run.argtypes = [i, i, ctypes.c_double, ctypes.c_double, ctypes.c_longlong, d, d, d]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def angles(n_x, n_y, n_z, delta: float):
    """Eq. 24 (theta, 3 planes) and Eq. 25 (beta, 4 planes) from the index fields."""
    n_x, n_y, n_z = _f64(n_x), _f64(n_y), _f64(n_z)
    Ny, Nx = n_x.shape
    theta = np.empty((3, Ny, Nx))
    beta = np.empty((4, Ny, Nx))
    lib().orc_angles(Nx, Ny, _p(n_x), _p(n_y), _p(n_z), float(delta), _p(theta), _p(beta))
    return theta, beta


def collide_x(q: np.ndarray, theta: np.ndarray, dagger: bool = False) -> None:
    """Eq. 17 applied at every site, in place."""
    lib().orc_collide_x(q.shape[2], q.shape[1], _p(q), _p(theta), int(dagger))


def collide_y(q: np.ndarray, theta: np.ndarray, dagger: bool = False) -> None:
    """Eq. 19 (row 2 read with sin in column 3) applied at every site, in place."""
    lib().orc_collide_y(q.shape[2], q.shape[1], _p(q), _p(theta), int(dagger))


def stream(q: np.ndarray, ca: int, cb: int, axis: int, direction: int) -> None:
    """S^{+/-axis}_{ca cb} (Eq. 18/20): q_c(r) <- q_c(r + direction e_axis) for c in {ca, cb}."""
    lib().orc_stream(q.shape[2], q.shape[1], _p(q), int(ca), int(cb), int(axis), int(direction))


def potential_x(q, beta, scale: float = 1.0, mode: int = POT_PAPER) -> None:
    """Eq. 21 with angles scale*beta (POT_PAPER) or its unitary variant (POT_UNITARY)."""
    lib().orc_potential_x(q.shape[2], q.shape[1], _p(q), _p(beta), float(scale), int(mode))


def potential_y(q, beta, scale: float = 1.0, mode: int = POT_PAPER) -> None:
    """Eq. 22 (row 3 read as sin, cos) with angles scale*beta, or its unitary variant."""
    lib().orc_potential_y(q.shape[2], q.shape[1], _p(q), _p(beta), float(scale), int(mode))


def collide_stream(q, theta, beta, axis: int, mid_v: bool = False, vscale: float = 0.5,
                   mode: int = POT_PAPER) -> None:
    """U_X (Eq. 18) for axis 0 or U_Y (Eq. 20) for axis 1; with mid_v, V' inserted as in Eq. 28."""
    lib().orc_collide_stream(int(axis), q.shape[2], q.shape[1], _p(q), _p(theta), _p(beta),
                             int(mid_v), float(vscale), int(mode))


def step(q, theta, beta, sequence: int = SEQ_INTERLEAVED, mode: int = POT_PAPER) -> None:
    """One time step: Eq. 23 (SEQ_PLAIN) or Eq. 28 (SEQ_INTERLEAVED), in place."""
    lib().orc_step(q.shape[2], q.shape[1], _p(q), _p(theta), _p(beta), int(sequence), int(mode))


def run(q, theta, beta, nsteps: int, sequence: int = SEQ_INTERLEAVED, mode: int = POT_PAPER) -> None:
    """nsteps time steps in place."""
    lib().orc_run(q.shape[2], q.shape[1], _p(q), _p(theta), _p(beta), int(sequence), int(mode),
                  int(nsteps))


def energy(q) -> float:
    """Eq. 27: mean over sites of Q.Q (compensated summation)."""
    q = _f64(q)
    return float(lib().orc_energy(q.shape[2], q.shape[1], _p(q)))


def divB(q):
    """(sum div^2, max |div|, max |B|) of B = (q3, q4, q5) with central differences."""
    q = _f64(q)
    out = np.zeros(3)
    lib().orc_divB(q.shape[2], q.shape[1], _p(q), _p(out))
    return float(out[0]), float(out[1]), float(out[2])


def divD(q, n_x, n_y, n_z):
    """(sum div^2, max |div|, max |D|) of D = (n_x q0, n_y q1, n_z q2) (eps_i = n_i^2)
    with central differences."""
    q = _f64(q)
    nx, ny, nz = _f64(n_x), _f64(n_y), _f64(n_z)
    out = np.zeros(3)
    lib().orc_divD(q.shape[2], q.shape[1], _p(q), _p(nx), _p(ny), _p(nz), _p(out))
    return float(out[0]), float(out[1]), float(out[2])


def init_pulse(Nx: int, Ny: int, pol: int, x0: float, sigma: float, amp: float) -> np.ndarray:
    """1D Gaussian pulse travelling in +x, polarisation E_z (pol 0) or E_y (pol 1)."""
    q = np.empty((6, Ny, Nx))
    lib().orc_init_pulse(Nx, Ny, _p(q), int(pol), float(x0), float(sigma), float(amp))
    return q


def yee_run(eps: np.ndarray, E: np.ndarray, B: np.ndarray, h: float, dt: float, nsteps: int):
    """Brute-force Yee FDTD of curl Maxwell (eps dE/dt = curl B, dB/dt = -curl E); in place."""
    eps, E, B = _f64(eps), E, B
    assert E.dtype == np.float64 and B.dtype == np.float64
    Ny, Nx = eps.shape[1:]
    lib().orc_yee_run(Nx, Ny, float(h), float(dt), int(nsteps), _p(eps), _p(E), _p(B))
    return E, B


def simulate(n_x, n_y, n_z, delta: float, q0: np.ndarray, nsteps: int,
             sequence: int = SEQ_INTERLEAVED, mode: int = POT_PAPER) -> np.ndarray:
    """Convenience: angles from the index fields, then nsteps steps on a copy of q0."""
    theta, beta = angles(n_x, n_y, n_z, delta)
    q = np.array(q0, dtype=np.float64, order="C", copy=True)
    run(q, theta, beta, nsteps, sequence, mode)
    return q
