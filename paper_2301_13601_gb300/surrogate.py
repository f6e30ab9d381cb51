"""Python binding of the surrogate's C ABI (include/qla_surrogate.h).

Argument marshalling only: the convolutions, losses, gradients and optimiser
steps run in libqla's kernels; torch tensors provide the device memory and
the stream. There is no CPU fallback.
"""
from __future__ import annotations

import ctypes

from .qla import QLAError, STATUS, load_library

EPI_GELU, EPI_LINEAR, EPI_DGRAD, EPI_QUPDATE = 0, 1, 2, 3

EXPORTS = ["qla_conv3x3_bf16", "qla_pack_conv_weights"]

_sigs_done = False


def lib():
    global _sigs_done
    L = load_library()
    if not _sigs_done:
        v, i, f = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
        L.qla_conv3x3_bf16.argtypes = [v, i, i, i, v, v, i, i, v, v, v, v, f, v, v]
        L.qla_conv3x3_bf16.restype = i
        L.qla_pack_conv_weights.argtypes = [v, i, i, i, i, i, v, v]
        L.qla_pack_conv_weights.restype = i
        _sigs_done = True
    return L


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    return ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)


def _check(st, where):
    if st != 0:
        raise QLAError(st, where, STATUS.get(st, str(st)))


def conv3x3(x, w_packed, nout, epilogue, out0, out1=None, bias=None, aux0=None, zprev=None, scale=1.0,
            error_flag=None, stream=None):
    """qla_conv3x3_bf16 on torch CUDA tensors; x is BF16 [H][W][cin]."""
    H, W, cin = x.shape
    st = lib().qla_conv3x3_bf16(_ptr(x), H, W, cin, _ptr(w_packed), _ptr(bias), nout, epilogue, _ptr(aux0),
                                _ptr(zprev), _ptr(out0), _ptr(out1), float(scale), _ptr(error_flag),
                                _stream(stream))
    _check(st, "qla_conv3x3_bf16")


def pack_weights(w, out, nout_pad, cin_pad, transpose_flip=False, stream=None):
    """qla_pack_conv_weights: FP32 w [nout][cin][3][3] -> BF16 [9][cin_pad/8][nout_pad][8]."""
    nout, cin = w.shape[0], w.shape[1]
    st = lib().qla_pack_conv_weights(_ptr(w), nout, cin, nout_pad, cin_pad, int(bool(transpose_flip)), _ptr(out),
                                     _stream(stream))
    _check(st, "qla_pack_conv_weights")
