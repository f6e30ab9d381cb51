"""Python binding of libqla (the C ABI in include/qla.h).

Argument marshalling only: every step of the method runs in the CUDA library.
PyTorch provides the device memory (the context's buffers are torch tensors
handed to qla_create) and the CUDA stream. The library must be built
(``__graft_entry__.build()``); loading fails loudly otherwise, and there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libqla.so")

FP32, FP64 = 0, 1
SEQ_INTERLEAVED, SEQ_PLAIN = 0, 1
POT_PAPER, POT_UNITARY = 0, 1
POL_EZ, POL_EY = 0, 1
FAMILIES_BOTH, FAMILY_TM, FAMILY_TE = 0, 1, 2
LAUNCH_AUTO, LAUNCH_PER_PASS, LAUNCH_PERSISTENT = 0, 1, 2
LAUNCHES = {"auto": LAUNCH_AUTO, "per_pass": LAUNCH_PER_PASS, "persistent": LAUNCH_PERSISTENT}
# single operators for qla_debug_apply: collisions (Eq. 17, Eq. 19), streaming
# shifts S^{+-axis}_{components} (Eq. 18, Eq. 20), potentials (Eq. 21-22)
OPS = {"CX": 0, "CX_T": 1, "CY": 2, "CY_T": 3, "S14+x": 4, "S14-x": 5, "S25+x": 6, "S25-x": 7,
       "S03+y": 8, "S03-y": 9, "S25+y": 10, "S25-y": 11, "VX": 12, "VY": 13}

STATUS = {0: "QLA_OK", 1: "QLA_EINVAL", 2: "QLA_ENOMEM", 3: "QLA_ECUDA", 4: "QLA_ETIMEOUT",
          5: "QLA_ENONFINITE", 6: "QLA_EUNSUPPORTED", 7: "QLA_ESTATE"}

# Every symbol include/qla.h declares (checked by the tests).
EXPORTS = [
    "qla_default_options", "qla_query_buffer_sizes", "qla_create", "qla_init_pulse", "qla_set_fields",
    "qla_set_fields_f32", "qla_step", "qla_debug_apply", "qla_energy", "qla_divB", "qla_divD", "qla_diagnostics",
    "qla_get_fields",
    "qla_get_fields_f32", "qla_state_device_ptr", "qla_synchronize", "qla_step_count", "qla_get_config",
    "qla_last_error", "qla_status_string", "qla_destroy", "qla_diagnostics_noalloc", "qla_sweep_split",
    "qla_get_sweep_split", "qla_sweep_dependencies", "qla_get_launch", "qla_set_wait_limit",
    "qla_batch_create", "qla_batch_run", "qla_batch_get_fields_f32", "qla_batch_diagnostics", "qla_batch_info",
    "qla_batch_set_wait_limit", "qla_batch_last_error", "qla_batch_destroy",
]


class QLAError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}" + (f" ({detail})" if detail else ""))


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("sequence", ctypes.c_int), ("potential", ctypes.c_int),
                ("steps_per_pass", ctypes.c_int), ("chunk_rows", ctypes.c_int), ("device", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("families", ctypes.c_int), ("launch", ctypes.c_int)]


class BufferSizes(ctypes.Structure):
    _fields_ = [("state_bytes", ctypes.c_size_t), ("coeff_bytes", ctypes.c_size_t),
                ("index_bytes", ctypes.c_size_t), ("scratch_bytes", ctypes.c_size_t)]


class DeviceBuffers(ctypes.Structure):
    _fields_ = [("state", ctypes.c_void_p * 2), ("coeff", ctypes.c_void_p), ("index", ctypes.c_void_p),
                ("scratch", ctypes.c_void_p)]


class Diag(ctypes.Structure):
    _fields_ = [("energy", ctypes.c_double), ("div_l2_sq", ctypes.c_double), ("div_max", ctypes.c_double),
                ("b_max", ctypes.c_double), ("nonfinite", ctypes.c_longlong)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libqla.so and declare its C signatures. Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(path)
    P = ctypes.POINTER
    d, i, v, st = ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_int
    L.qla_default_options.argtypes = [P(Options)]
    L.qla_default_options.restype = None
    L.qla_query_buffer_sizes.argtypes = [i, i, P(Options), P(BufferSizes)]
    L.qla_query_buffer_sizes.restype = st
    L.qla_create.argtypes = [i, i, P(d), P(d), P(d), d, P(Options), P(DeviceBuffers), P(v)]
    L.qla_create.restype = st
    L.qla_init_pulse.argtypes = [v, i, d, d, d]
    L.qla_init_pulse.restype = st
    L.qla_set_fields.argtypes = [v, P(d)]
    L.qla_set_fields.restype = st
    L.qla_set_fields_f32.argtypes = [v, P(ctypes.c_float)]
    L.qla_set_fields_f32.restype = st
    L.qla_step.argtypes = [v, ctypes.c_longlong]
    L.qla_step.restype = st
    L.qla_debug_apply.argtypes = [v, i, i]
    L.qla_debug_apply.restype = st
    L.qla_energy.argtypes = [v, P(d)]
    L.qla_energy.restype = st
    L.qla_divB.argtypes = [v, P(d), P(d), P(d)]
    L.qla_divB.restype = st
    L.qla_divD.argtypes = [v, P(d), P(d), P(d)]
    L.qla_divD.restype = st
    L.qla_diagnostics.argtypes = [v, P(Diag)]
    L.qla_diagnostics.restype = st
    L.qla_get_fields.argtypes = [v, P(d)]
    L.qla_get_fields.restype = st
    L.qla_get_fields_f32.argtypes = [v, P(ctypes.c_float)]
    L.qla_get_fields_f32.restype = st
    L.qla_state_device_ptr.argtypes = [v]
    L.qla_state_device_ptr.restype = v
    L.qla_synchronize.argtypes = [v]
    L.qla_synchronize.restype = st
    L.qla_step_count.argtypes = [v]
    L.qla_step_count.restype = ctypes.c_longlong
    L.qla_get_config.argtypes = [v, P(i), P(i), P(i)]
    L.qla_get_config.restype = st
    L.qla_last_error.argtypes = [v]
    L.qla_last_error.restype = ctypes.c_char_p
    L.qla_status_string.argtypes = [st]
    L.qla_status_string.restype = ctypes.c_char_p
    L.qla_destroy.argtypes = [v]
    L.qla_destroy.restype = None
    L.qla_diagnostics_noalloc.argtypes = [v, i, i, i, v, P(Diag)]
    L.qla_diagnostics_noalloc.restype = st
    L.qla_sweep_split.argtypes = [i, i, i, i, i, i, i, P(ctypes.c_longlong), i]
    L.qla_sweep_split.restype = st
    L.qla_get_sweep_split.argtypes = [v, i, i, P(i), P(ctypes.c_longlong), i]
    L.qla_get_sweep_split.restype = st
    L.qla_sweep_dependencies.argtypes = [i, i, i, i, i, i, P(i), i, P(i)]
    L.qla_sweep_dependencies.restype = st
    L.qla_get_launch.argtypes = [v, P(i)]
    L.qla_get_launch.restype = st
    L.qla_set_wait_limit.argtypes = [v, ctypes.c_longlong, i]
    L.qla_set_wait_limit.restype = st
    _lib = L
    return L


def sweep_split(Nx: int, Ny: int, steps_per_pass: int, ctas: int, precision: str = "fp32", family: str = "TM",
                layers: int = 2) -> np.ndarray:
    """Share bounds of the balanced split of an Nx x Ny pass of steps_per_pass
    steps over `ctas` CTAs of a family's layer, in a pass of `layers` family
    layers (host arithmetic of the library; no GPU)."""
    L = load_library()
    out = np.zeros(int(ctas) + 1, dtype=np.int64)
    st = L.qla_sweep_split(int(Nx), int(Ny), _code("precision", {"fp32": FP32, "fp64": FP64}, precision),
                           int(steps_per_pass), int(ctas), _code("family", {"TM": FAMILY_TM, "TE": FAMILY_TE}, family),
                           int(layers), out.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), out.size)
    if st != 0:
        raise QLAError(st, "qla_sweep_split")
    return out


def sweep_dependencies(Nx: int, Ny: int, steps_per_pass: int, ctas: int, share: int,
                       family: str = "TM") -> np.ndarray:
    """Shares that share `share` of the persistent launch form waits for
    before its passes after the first (host arithmetic of the library; no
    GPU)."""
    L = load_library()
    out = np.zeros(int(ctas), dtype=np.int32)
    n = ctypes.c_int()
    st = L.qla_sweep_dependencies(int(Nx), int(Ny), int(steps_per_pass), int(ctas),
                                  _code("family", {"TM": FAMILY_TM, "TE": FAMILY_TE}, family), int(share),
                                  out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), out.size, ctypes.byref(n))
    if st != 0:
        raise QLAError(st, "qla_sweep_dependencies")
    return out[:n.value].copy()


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _fptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _code(name: str, table: dict, value):
    if isinstance(value, str):
        if value not in table:
            raise ValueError(f"{name} must be one of {list(table)}")
        return table[value]
    return int(value)


class Simulation:
    """One QLA lattice on one GPU (a qla_ctx).

    n_x, n_y, n_z: float64 arrays (Ny, Nx) of principal refractive indices.
    precision: 'fp32' (default) or 'fp64'; sequence: 'interleaved' (Eq. 28) or
    'plain' (Eq. 23); potential: 'paper' (Eq. 21-22 as printed) or 'unitary'.
    """

    def __init__(self, n_x, n_y, n_z, delta: float, precision="fp32", sequence="interleaved",
                 potential="paper", steps_per_pass: int = 0, chunk_rows: int = 0,
                 device: Optional[int] = None, stream=None, families="both", launch="auto"):
        import torch  # device memory and streams

        if not torch.cuda.is_available():
            raise RuntimeError("libqla needs a CUDA GPU; no CPU fallback exists")
        L = load_library()
        self._L = L
        self._ctx = None
        n_x, n_y, n_z = (np.ascontiguousarray(a, dtype=np.float64) for a in (n_x, n_y, n_z))
        if not (n_x.shape == n_y.shape == n_z.shape) or n_x.ndim != 2:
            raise ValueError("n_x, n_y, n_z must be 2D arrays of one shape (Ny, Nx)")
        self.Ny, self.Nx = n_x.shape
        dev = torch.cuda.current_device() if device is None else int(device)
        self.device = torch.device("cuda", dev)
        if stream is None:
            # a dedicated torch stream: the library's work and any events the
            # caller records on sim.stream are then ordered on one queue
            stream = torch.cuda.Stream(device=self.device)
        self.stream = stream
        opt = Options()
        L.qla_default_options(ctypes.byref(opt))
        opt.precision = _code("precision", {"fp32": FP32, "fp64": FP64}, precision)
        opt.sequence = _code("sequence", {"interleaved": SEQ_INTERLEAVED, "plain": SEQ_PLAIN}, sequence)
        opt.potential = _code("potential", {"paper": POT_PAPER, "unitary": POT_UNITARY}, potential)
        opt.steps_per_pass = int(steps_per_pass)
        opt.chunk_rows = int(chunk_rows)
        opt.device = dev
        opt.stream = ctypes.c_void_p(stream.cuda_stream)
        # "TM": only (q2, q3, q4), the E_z polarisation; "TE": only (q0, q1, q5), E_y
        opt.families = _code("families", {"both": FAMILIES_BOTH, "TM": FAMILY_TM, "TE": FAMILY_TE}, families)
        self.families = families
        # "per_pass": one kernel launch per pass; "persistent": the full passes
        # of a step() call in one cooperative launch; "auto": one launch per pass
        opt.launch = _code("launch", LAUNCHES, launch)
        self.precision = opt.precision
        sizes = BufferSizes()
        self._check(L.qla_query_buffer_sizes(self.Nx, self.Ny, ctypes.byref(opt), ctypes.byref(sizes)),
                    "qla_query_buffer_sizes")
        u8 = torch.uint8
        with torch.cuda.device(dev):
            self._bufs = {
                "state0": torch.empty(sizes.state_bytes, dtype=u8, device=self.device),
                "state1": torch.empty(sizes.state_bytes, dtype=u8, device=self.device),
                "coeff": torch.empty(sizes.coeff_bytes, dtype=u8, device=self.device),
                "index": torch.empty(sizes.index_bytes, dtype=u8, device=self.device),
                "scratch": torch.empty(sizes.scratch_bytes, dtype=u8, device=self.device),
            }
        db = DeviceBuffers()
        db.state[0] = self._bufs["state0"].data_ptr()
        db.state[1] = self._bufs["state1"].data_ptr()
        db.coeff = self._bufs["coeff"].data_ptr()
        db.index = self._bufs["index"].data_ptr()
        db.scratch = self._bufs["scratch"].data_ptr()
        torch.cuda.synchronize(self.device)  # allocations visible before the library's stream uses them
        ctx = ctypes.c_void_p()
        self._check(L.qla_create(self.Nx, self.Ny, _dptr(n_x), _dptr(n_y), _dptr(n_z), float(delta),
                                 ctypes.byref(opt), ctypes.byref(db), ctypes.byref(ctx)), "qla_create")
        self._ctx = ctx
        k, ch, pr = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        L.qla_get_config(ctx, ctypes.byref(k), ctypes.byref(ch), ctypes.byref(pr))
        self.steps_per_pass, self.chunk_rows = k.value, ch.value

    def set_wait_limit(self, timeout_ns: int, withhold: int = 0):
        """Test hook of the persistent form's waits (qla_set_wait_limit)."""
        self._check(self._L.qla_set_wait_limit(self._ctx, int(timeout_ns), int(withhold)), "qla_set_wait_limit")

    @property
    def launch(self) -> str:
        """The launch form the context's passes take: 'persistent' or 'per_pass'."""
        v = ctypes.c_int()
        self._check(self._L.qla_get_launch(self._ctx, ctypes.byref(v)), "qla_get_launch")
        return "persistent" if v.value == LAUNCH_PERSISTENT else "per_pass"

    # -- plumbing ---------------------------------------------------------
    def _check(self, status: int, where: str):
        if status != 0:
            detail = ""
            if self._ctx is not None:
                detail = (self._L.qla_last_error(self._ctx) or b"").decode()
            raise QLAError(status, where, detail)

    @property
    def shape(self):
        return (6, self.Ny, self.Nx)

    # -- API --------------------------------------------------------------
    def init_pulse(self, polarization, x0: float, sigma: float, amplitude: float = 1.0):
        pol = _code("polarization", {"Ez": POL_EZ, "Ey": POL_EY}, polarization)
        self._check(self._L.qla_init_pulse(self._ctx, pol, float(x0), float(sigma), float(amplitude)),
                    "qla_init_pulse")

    def set_fields(self, q: np.ndarray):
        q = np.asarray(q)
        if q.shape != self.shape:
            raise ValueError(f"state must have shape {self.shape}")
        if q.dtype == np.float32:
            q = np.ascontiguousarray(q)
            self._check(self._L.qla_set_fields_f32(self._ctx, _fptr(q)), "qla_set_fields_f32")
            self.synchronize()
        else:
            q = np.ascontiguousarray(q, dtype=np.float64)
            self._check(self._L.qla_set_fields(self._ctx, _dptr(q)), "qla_set_fields")

    def set_fields_host_f32(self, q_ptr: int):
        """Asynchronous copy from a pinned float32 host buffer (address)."""
        self._check(self._L.qla_set_fields_f32(self._ctx, ctypes.cast(q_ptr, ctypes.POINTER(ctypes.c_float))),
                    "qla_set_fields_f32")

    def get_fields(self, dtype=np.float64) -> np.ndarray:
        if np.dtype(dtype) == np.float32:
            out = np.empty(self.shape, dtype=np.float32)
            self._check(self._L.qla_get_fields_f32(self._ctx, _fptr(out)), "qla_get_fields_f32")
        else:
            out = np.empty(self.shape, dtype=np.float64)
            self._check(self._L.qla_get_fields(self._ctx, _dptr(out)), "qla_get_fields")
        return out

    def get_fields_host_f32(self, q_ptr: int):
        self._check(self._L.qla_get_fields_f32(self._ctx, ctypes.cast(q_ptr, ctypes.POINTER(ctypes.c_float))),
                    "qla_get_fields_f32")

    def step(self, nsteps: int):
        self._check(self._L.qla_step(self._ctx, int(nsteps)), "qla_step")

    def debug_apply(self, op: str, count: int = 1):
        """Apply one operator of the step (see OPS) `count` times."""
        self._check(self._L.qla_debug_apply(self._ctx, _code("op", OPS, op), int(count)), "qla_debug_apply")

    def diagnostics(self) -> dict:
        d = Diag()
        st = self._L.qla_diagnostics(self._ctx, ctypes.byref(d))
        if st not in (0, 5):
            self._check(st, "qla_diagnostics")
        return {"energy": d.energy, "div_l2_sq": d.div_l2_sq, "div_max": d.div_max, "b_max": d.b_max,
                "nonfinite": d.nonfinite, "status": STATUS[st]}

    def energy(self) -> float:
        e = ctypes.c_double()
        st = self._L.qla_energy(self._ctx, ctypes.byref(e))
        if st not in (0, 5):
            self._check(st, "qla_energy")
        return e.value

    def divB(self):
        a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        st = self._L.qla_divB(self._ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
        if st not in (0, 5):
            self._check(st, "qla_divB")
        return a.value, b.value, c.value

    def divD(self):
        """(sum div^2, max |div|, max |D|) of D = (n_x q0, n_y q1, n_z q2)."""
        a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        st = self._L.qla_divD(self._ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
        if st not in (0, 5):
            self._check(st, "qla_divD")
        return a.value, b.value, c.value

    def synchronize(self):
        self._check(self._L.qla_synchronize(self._ctx), "qla_synchronize")

    def sweep_split(self, steps_per_pass: Optional[int] = None, family: str = "TM") -> Optional[np.ndarray]:
        """Share bounds (row units u = strip * Ny + y, one share per CTA of the
        family's layer) of the balanced split that passes of steps_per_pass
        steps use (default: the configured steps per pass); None when the
        context sweeps fixed tiles of chunk_rows rows or does not advance the
        family."""
        K = int(steps_per_pass or self.steps_per_pass)
        fam = _code("family", {"TM": FAMILY_TM, "TE": FAMILY_TE}, family)
        n = ctypes.c_int()
        self._check(self._L.qla_get_sweep_split(self._ctx, K, fam, ctypes.byref(n), None, 0), "qla_get_sweep_split")
        if n.value == 0:
            return None
        out = np.zeros(n.value + 1, dtype=np.int64)
        self._check(self._L.qla_get_sweep_split(self._ctx, K, fam, ctypes.byref(n),
                                                out.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), out.size),
                    "qla_get_sweep_split")
        return out

    @property
    def step_count(self) -> int:
        return int(self._L.qla_step_count(self._ctx))

    def state_tensor(self):
        """The current device state as a torch view (6, Ny, Nx); valid until the next step."""
        import torch

        ptr = self._L.qla_state_device_ptr(self._ctx)
        buf = self._bufs["state0"] if ptr == self._bufs["state0"].data_ptr() else self._bufs["state1"]
        dt = torch.float32 if self.precision == FP32 else torch.float64
        n = 6 * self.Ny * self.Nx
        return buf[: n * (4 if dt == torch.float32 else 8)].view(dt).view(6, self.Ny, self.Nx)

    def close(self):
        if self._ctx is not None:
            self._L.qla_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class InstanceDesc(ctypes.Structure):
    _fields_ = [("Nx", ctypes.c_int), ("Ny", ctypes.c_int), ("n_x", ctypes.POINTER(ctypes.c_double)),
                ("n_y", ctypes.POINTER(ctypes.c_double)), ("n_z", ctypes.POINTER(ctypes.c_double)),
                ("delta", ctypes.c_double), ("nsteps", ctypes.c_longlong), ("pulse_polarization", ctypes.c_int),
                ("pulse_x0", ctypes.c_double), ("pulse_sigma", ctypes.c_double),
                ("pulse_amplitude", ctypes.c_double), ("chunk_rows", ctypes.c_int)]


def _batch_sigs(L):
    P = ctypes.POINTER
    v, i, st = ctypes.c_void_p, ctypes.c_int, ctypes.c_int
    L.qla_batch_create.argtypes = [i, P(InstanceDesc), P(Options), P(v)]
    L.qla_batch_create.restype = st
    L.qla_batch_run.argtypes = [v]
    L.qla_batch_run.restype = st
    L.qla_batch_get_fields_f32.argtypes = [v, i, P(ctypes.c_float)]
    L.qla_batch_get_fields_f32.restype = st
    L.qla_batch_diagnostics.argtypes = [v, i, P(Diag)]
    L.qla_batch_diagnostics.restype = st
    L.qla_batch_info.argtypes = [v, P(ctypes.c_longlong), P(i), P(ctypes.c_longlong)]
    L.qla_batch_info.restype = st
    L.qla_batch_set_wait_limit.argtypes = [v, ctypes.c_longlong, i]
    L.qla_batch_set_wait_limit.restype = st
    L.qla_batch_last_error.argtypes = [v]
    L.qla_batch_last_error.restype = ctypes.c_char_p
    L.qla_batch_destroy.argtypes = [v]
    L.qla_batch_destroy.restype = None


class Batch:
    """Many independent lattices advanced by one persistent graph launch (FP32).

    instances: list of dicts with keys n (tuple of three (Ny, Nx) arrays), delta,
    nsteps, and optionally pulse=(polarization 'Ez'/'Ey', x0, sigma, amplitude)
    and chunk_rows.
    steps_per_pass = 0 lets the autotuner (autotune.tune_batch, cached per GPU
    and batch shape) choose the steps per pass and the rows per tile of the
    instances that do not set chunk_rows; the choice is kept in self.tuned.
    """

    def __init__(self, instances, steps_per_pass: int = 4, sequence="interleaved", potential="paper",
                 device: Optional[int] = None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("libqla needs a CUDA GPU; no CPU fallback exists")
        self.tuned = None
        if int(steps_per_pass) == 0:
            from .autotune import tune_batch

            self.tuned = tune_batch(instances, sequence=sequence, potential=potential)
            steps_per_pass = int(self.tuned["steps_per_pass"])
            instances = [dict(ins, chunk_rows=ins.get("chunk_rows") or int(self.tuned["chunk_rows"]))
                         for ins in instances]
        L = load_library()
        _batch_sigs(L)
        self._L = L
        self._b = None
        self._keep = []
        descs = (InstanceDesc * len(instances))()
        self.shapes = []
        for k, ins in enumerate(instances):
            n = [np.ascontiguousarray(a, dtype=np.float64) for a in ins["n"]]
            self._keep.append(n)
            Ny, Nx = n[0].shape
            self.shapes.append((6, Ny, Nx))
            d = descs[k]
            d.Nx, d.Ny = Nx, Ny
            d.n_x, d.n_y, d.n_z = (_dptr(a) for a in n)
            d.delta = float(ins["delta"])
            d.nsteps = int(ins["nsteps"])
            pulse = ins.get("pulse")
            if pulse is None:
                d.pulse_polarization = -1
            else:
                d.pulse_polarization = _code("polarization", {"Ez": POL_EZ, "Ey": POL_EY}, pulse[0])
                d.pulse_x0, d.pulse_sigma, d.pulse_amplitude = float(pulse[1]), float(pulse[2]), float(pulse[3])
            d.chunk_rows = int(ins.get("chunk_rows", 0))
        opt = Options()
        L.qla_default_options(ctypes.byref(opt))
        opt.steps_per_pass = int(steps_per_pass)
        opt.sequence = _code("sequence", {"interleaved": SEQ_INTERLEAVED, "plain": SEQ_PLAIN}, sequence)
        opt.potential = _code("potential", {"paper": POT_PAPER, "unitary": POT_UNITARY}, potential)
        opt.device = torch.cuda.current_device() if device is None else int(device)
        b = ctypes.c_void_p()
        st = L.qla_batch_create(len(instances), descs, ctypes.byref(opt), ctypes.byref(b))
        if st != 0:
            raise QLAError(st, "qla_batch_create")
        self._b = b

    def run(self):
        st = self._L.qla_batch_run(self._b)
        if st != 0:
            raise QLAError(st, "qla_batch_run", (self._L.qla_batch_last_error(self._b) or b"").decode())

    def run_status(self) -> int:
        return int(self._L.qla_batch_run(self._b))

    def set_wait_limit(self, timeout_ns: int, withhold: int = 0):
        st = self._L.qla_batch_set_wait_limit(self._b, int(timeout_ns), int(withhold))
        if st != 0:
            raise QLAError(st, "qla_batch_set_wait_limit")

    def get_fields(self, i: int) -> np.ndarray:
        out = np.empty(self.shapes[i], dtype=np.float32)
        st = self._L.qla_batch_get_fields_f32(self._b, int(i), _fptr(out))
        if st != 0:
            raise QLAError(st, "qla_batch_get_fields_f32")
        return out

    def diagnostics(self, i: int) -> dict:
        d = Diag()
        st = self._L.qla_batch_diagnostics(self._b, int(i), ctypes.byref(d))
        if st not in (0, 5):
            raise QLAError(st, "qla_batch_diagnostics")
        return {"energy": d.energy, "div_l2_sq": d.div_l2_sq, "div_max": d.div_max, "b_max": d.b_max,
                "nonfinite": d.nonfinite}

    def info(self):
        t, k, s = ctypes.c_longlong(), ctypes.c_int(), ctypes.c_longlong()
        self._L.qla_batch_info(self._b, ctypes.byref(t), ctypes.byref(k), ctypes.byref(s))
        return {"work_items": t.value, "steps_per_pass": k.value, "site_updates": s.value}

    def close(self):
        if self._b is not None:
            self._L.qla_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
