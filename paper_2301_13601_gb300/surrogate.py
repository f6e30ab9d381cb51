"""Python binding of the surrogate's C ABI (include/qla_surrogate.h).

Argument marshalling only: the convolutions, losses, gradients and optimiser
steps run in libqla's kernels; torch tensors provide the device memory and
the stream. There is no CPU fallback.
"""
from __future__ import annotations

import ctypes

from .qla import QLAError, STATUS, load_library

EPI_GELU, EPI_LINEAR, EPI_DGRAD, EPI_QUPDATE = 0, 1, 2, 3
DRIFT_PER_CALL, DRIFT_FROM_START = 0, 1
ROLLOUT_SERIAL = 16  # flag: no speculative next call in qla_surrogate_rollout

EXPORTS = ["qla_conv3x3_bf16", "qla_pack_conv_weights", "qla_conv_schedule"]
CONV_SCHEDULE_FIELDS = 14  # ints per record of qla_conv_schedule

_sigs_done = False


def lib():
    global _sigs_done
    L = load_library()
    if not _sigs_done:
        v, i, f = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
        L.qla_conv3x3_bf16.argtypes = [v, i, i, i, i, v, v, i, i, v, v, v, v, f, v, v]
        L.qla_conv3x3_bf16.restype = i
        L.qla_pack_conv_weights.argtypes = [v, i, i, i, i, i, v, v]
        L.qla_pack_conv_weights.restype = i
        L.qla_conv_schedule.argtypes = [i, i, i, i, i, i, i, v, ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong)]
        L.qla_conv_schedule.restype = i
        _sigs_done = True
    return L


def conv_schedule(cin: int, nout: int, nimg: int, H: int, W: int, grid: int, cta: int):
    """The MMA issue schedule of one CTA of the conv kernel, enumerated on the
    host by the code the kernel runs (see qla_conv_schedule): an int array
    [records][CONV_SCHEDULE_FIELDS]. Touches no GPU."""
    import numpy as np

    L = lib()
    count = ctypes.c_longlong()
    st = L.qla_conv_schedule(cin, nout, nimg, H, W, grid, cta, None, 0, ctypes.byref(count))
    if st != 0:
        raise ValueError(f"qla_conv_schedule: status {st}")
    rec = np.zeros((count.value, CONV_SCHEDULE_FIELDS), dtype=np.int32)
    st = L.qla_conv_schedule(cin, nout, nimg, H, W, grid, cta, rec.ctypes.data_as(ctypes.c_void_p), count.value,
                             ctypes.byref(count))
    if st != 0 or count.value != rec.shape[0]:
        raise ValueError(f"qla_conv_schedule: status {st}")
    return rec


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    return ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)


def _check(st, where):
    if st != 0:
        raise QLAError(st, where, STATUS.get(st, str(st)))


def conv3x3(x, w_packed, nout, epilogue, out0, out1=None, bias=None, aux0=None, zprev=None, scale=1.0,
            error_flag=None, stream=None):
    """qla_conv3x3_bf16 on torch CUDA tensors; x is BF16 [H][W][cin] or [nimg][H][W][cin]."""
    nimg, H, W, cin = x.shape if x.dim() == 4 else (1, *x.shape)
    st = lib().qla_conv3x3_bf16(_ptr(x), nimg, H, W, cin, _ptr(w_packed), _ptr(bias), nout, epilogue, _ptr(aux0),
                                _ptr(zprev), _ptr(out0), _ptr(out1), float(scale), _ptr(error_flag),
                                _stream(stream))
    _check(st, "qla_conv3x3_bf16")


def pack_weights(w, out, nout_pad, cin_pad, transpose_flip=False, stream=None):
    """qla_pack_conv_weights: FP32 w [nout][cin][3][3] -> BF16 [9][cin_pad/8][nout_pad][8]."""
    nout, cin = w.shape[0], w.shape[1]
    st = lib().qla_pack_conv_weights(_ptr(w), nout, cin, nout_pad, cin_pad, int(bool(transpose_flip)), _ptr(out),
                                     _stream(stream))
    _check(st, "qla_pack_conv_weights")


# ---------------------------------------------------------------------------
# The surrogate network (qla_surrogate_*)
# ---------------------------------------------------------------------------
EXPORTS += ["qla_surrogate_param_count", "qla_surrogate_create", "qla_surrogate_init_params",
            "qla_surrogate_set_params", "qla_surrogate_get_params", "qla_surrogate_forward",
            "qla_surrogate_loss_grad", "qla_surrogate_adam_step", "qla_surrogate_train_step",
            "qla_surrogate_synchronize", "qla_surrogate_rollout", "qla_surrogate_info",
            "qla_surrogate_last_error", "qla_surrogate_destroy"]

# logical layer shapes (cin, nout): parameters are W_l [nout][cin][3][3] then b_l [nout]
LAYERS = [(9, 64), (64, 64), (64, 64), (64, 64), (64, 64), (64, 6)]


class Config(ctypes.Structure):
    _fields_ = [("nimg", ctypes.c_int), ("H", ctypes.c_int), ("W", ctypes.c_int), ("K", ctypes.c_int),
                ("out_scale", ctypes.c_float), ("train", ctypes.c_int), ("stream", ctypes.c_void_p)]


class RolloutStats(ctypes.Structure):
    _fields_ = [("calls", ctypes.c_longlong), ("surrogate_calls", ctypes.c_longlong),
                ("fallback_calls", ctypes.c_longlong), ("energy_ref", ctypes.c_double),
                ("energy_final", ctypes.c_double), ("max_drift", ctypes.c_double)]


_net_sigs_done = False


def _net_lib():
    global _net_sigs_done
    L = lib()
    if not _net_sigs_done:
        v, i, d, f, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_float, ctypes.c_longlong
        P = ctypes.POINTER
        L.qla_surrogate_param_count.argtypes = []
        L.qla_surrogate_param_count.restype = ll
        L.qla_surrogate_create.argtypes = [P(Config), P(v)]
        L.qla_surrogate_create.restype = i
        L.qla_surrogate_init_params.argtypes = [v, ctypes.c_ulonglong]
        L.qla_surrogate_init_params.restype = i
        L.qla_surrogate_set_params.argtypes = [v, P(f)]
        L.qla_surrogate_set_params.restype = i
        L.qla_surrogate_get_params.argtypes = [v, P(f)]
        L.qla_surrogate_get_params.restype = i
        L.qla_surrogate_forward.argtypes = [v, v, v, v]
        L.qla_surrogate_forward.restype = i
        L.qla_surrogate_loss_grad.argtypes = [v, v, v, v, P(d), P(f)]
        L.qla_surrogate_loss_grad.restype = i
        L.qla_surrogate_adam_step.argtypes = [v, f, f, f, f]
        L.qla_surrogate_adam_step.restype = i
        L.qla_surrogate_train_step.argtypes = [v, v, v, v, f, P(d)]
        L.qla_surrogate_train_step.restype = i
        L.qla_surrogate_synchronize.argtypes = [v]
        L.qla_surrogate_synchronize.restype = i
        L.qla_surrogate_rollout.argtypes = [v, v, v, i, d, i, d, P(RolloutStats)]
        L.qla_surrogate_rollout.restype = i
        L.qla_surrogate_info.argtypes = [v, P(ll), P(ll)]
        L.qla_surrogate_info.restype = i
        L.qla_surrogate_last_error.argtypes = [v]
        L.qla_surrogate_last_error.restype = ctypes.c_char_p
        L.qla_surrogate_destroy.argtypes = [v]
        L.qla_surrogate_destroy.restype = None
        _net_sigs_done = True
    return L


def param_count() -> int:
    return int(_net_lib().qla_surrogate_param_count())


def param_slices():
    """(weight slice, weight shape, bias slice) of every layer in the flat vector."""
    out, off = [], 0
    for cin, nout in LAYERS:
        nw = nout * cin * 9
        out.append((slice(off, off + nw), (nout, cin, 3, 3), slice(off + nw, off + nw + nout)))
        off += nw + nout
    return out


class Surrogate:
    """A surrogate network on the GPU. Its work runs on its own torch stream;
    every call first waits for torch's current stream (where the caller made
    its tensors) and makes the current stream wait for it afterwards."""

    def __init__(self, H: int, W: int, nimg: int = 1, K: int = 16, out_scale: float = 1.0 / 16, train: bool = False,
                 seed=None, stream=None):
        import torch

        self._L = _net_lib()
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.H, self.W, self.nimg, self.K, self.out_scale = H, W, nimg, K, out_scale
        cfg = Config(nimg, H, W, K, out_scale, int(bool(train)), self.stream.cuda_stream)
        h = ctypes.c_void_p()
        st = self._L.qla_surrogate_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != 0:
            raise QLAError(st, "qla_surrogate_create")
        self._h = h
        if seed is not None:
            self.init_params(seed)

    def _check(self, st, where):
        if st != 0:
            raise QLAError(st, where, self._L.qla_surrogate_last_error(self._h).decode())

    def _enter(self):
        import torch

        self.stream.wait_stream(torch.cuda.current_stream())

    def _leave(self):
        import torch

        torch.cuda.current_stream().wait_stream(self.stream)

    def init_params(self, seed: int):
        self._check(self._L.qla_surrogate_init_params(self._h, int(seed)), "init_params")

    def set_params(self, p):
        import numpy as np

        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == param_count()
        self._check(self._L.qla_surrogate_set_params(self._h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
                    "set_params")

    def get_params(self):
        import numpy as np

        p = np.empty(param_count(), dtype=np.float32)
        self._check(self._L.qla_surrogate_get_params(self._h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
                    "get_params")
        return p

    def forward(self, q_in, n, q_out):
        self._enter()
        self._check(self._L.qla_surrogate_forward(self._h, _ptr(q_in), _ptr(n), _ptr(q_out)), "forward")
        self._leave()

    def loss_grad(self, q_in, n, q_target, want_loss=True, want_grad=False):
        import numpy as np

        loss = ctypes.c_double() if want_loss else None
        g = np.empty(param_count(), dtype=np.float32) if want_grad else None
        self._enter()
        st = self._L.qla_surrogate_loss_grad(self._h, _ptr(q_in), _ptr(n), _ptr(q_target),
                                             ctypes.byref(loss) if loss is not None else None,
                                             g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) if g is not None else None)
        self._check(st, "loss_grad")
        self._leave()
        return (loss.value if loss is not None else None), g

    def adam_step(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        self._enter()
        self._check(self._L.qla_surrogate_adam_step(self._h, lr, beta1, beta2, eps), "adam_step")

    def train_step(self, q_in, n, q_target, lr, want_loss=False):
        loss = ctypes.c_double() if want_loss else None
        self._enter()
        st = self._L.qla_surrogate_train_step(self._h, _ptr(q_in), _ptr(n), _ptr(q_target), lr,
                                              ctypes.byref(loss) if loss is not None else None)
        self._check(st, "train_step")
        self._leave()
        return loss.value if loss is not None else None

    def synchronize(self):
        self._check(self._L.qla_surrogate_synchronize(self._h), "synchronize")

    def rollout(self, sim, n, calls: int, drift_tol: float = 1e-3, drift_mode: int = DRIFT_PER_CALL,
                energy_ref: float = 0.0, serial: bool = False) -> dict:
        """Advance a Simulation (FP32) by calls x K steps; see qla_surrogate_rollout
        (serial=True: no speculative next call)."""
        import torch

        torch.cuda.synchronize()
        st = RolloutStats()
        mode = drift_mode | (ROLLOUT_SERIAL if serial else 0)
        self._check(self._L.qla_surrogate_rollout(self._h, sim._ctx, _ptr(n), calls, drift_tol, mode,
                                                  energy_ref, ctypes.byref(st)), "rollout")
        return {k: getattr(st, k) for k, _ in RolloutStats._fields_}

    def info(self):
        npar, fl = ctypes.c_longlong(), ctypes.c_longlong()
        self._check(self._L.qla_surrogate_info(self._h, ctypes.byref(npar), ctypes.byref(fl)), "info")
        return {"params": npar.value, "flops_per_call": fl.value}

    def close(self):
        if getattr(self, "_h", None):
            self._L.qla_surrogate_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
