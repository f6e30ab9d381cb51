"""The C-ABI library loads on any machine and exports every symbol include/*.h declares."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = "".join(open(h).read() for h in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))))
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qla_[A-Za-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2301_13601_gb300 import qla

    return ctypes.CDLL(qla.LIB_PATH)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("qla_create", "qla_init_pulse", "qla_step", "qla_energy", "qla_divB", "qla_get_fields",
                     "qla_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2301_13601_gb300 import qla, surrogate

    assert sorted(qla.EXPORTS + surrogate.EXPORTS) == declared_functions()


def test_status_strings_without_gpu(lib):
    lib.qla_status_string.restype = ctypes.c_char_p
    assert lib.qla_status_string(0) == b"QLA_OK"
    assert lib.qla_status_string(4) == b"QLA_ETIMEOUT"


def test_buffer_size_query_without_gpu(lib):
    from paper_2301_13601_gb300 import qla

    L = qla.load_library()
    sizes = qla.BufferSizes()
    assert L.qla_query_buffer_sizes(100, 50, None, ctypes.byref(sizes)) == 0
    assert sizes.state_bytes >= 6 * 100 * 50 * 4 and sizes.state_bytes % 256 == 0
    assert sizes.coeff_bytes >= 14 * 100 * 50 * 4
    assert L.qla_query_buffer_sizes(0, 50, None, ctypes.byref(sizes)) == 1
    assert L.qla_query_buffer_sizes(70000, 70000, None, ctypes.byref(sizes)) == 1


def test_create_rejects_bad_arguments_before_touching_a_gpu(lib):
    import numpy as np

    from paper_2301_13601_gb300 import qla

    L = qla.load_library()
    n = np.ones((4, 4))
    bad = n.copy()
    bad[1, 2] = -1.0
    ctx = ctypes.c_void_p()
    P = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert L.qla_create(4, 4, P(n), P(n), P(bad), 0.1, None, None, ctypes.byref(ctx)) == 1
    nan = n.copy()
    nan[0, 0] = np.nan
    assert L.qla_create(4, 4, P(nan), P(n), P(n), 0.1, None, None, ctypes.byref(ctx)) == 1
    assert L.qla_create(4, 4, P(n), P(n), P(n), 0.0, None, None, ctypes.byref(ctx)) == 1
    assert L.qla_create(4, 4, P(n), P(n), P(n), 0.7, None, None, ctypes.byref(ctx)) == 1
    assert not ctx.value


def test_conv_rejects_bad_arguments_without_gpu(lib):
    """qla_conv3x3_bf16 checks sizes, channel pairs and epilogue operands on the
    host and returns before any launch (the pointers below are never read)."""
    from paper_2301_13601_gb300 import surrogate as S

    L = S.lib()
    p = ctypes.c_void_p(256)  # stand-in device pointer, never dereferenced on these paths
    N = None

    def call(x=p, nimg=1, H=4, W=128, cin=64, nout=64, epi=S.EPI_LINEAR, aux0=N, zprev=N, out0=p, out1=N, err=p):
        return L.qla_conv3x3_bf16(x, nimg, H, W, cin, p, N, nout, epi, aux0, zprev, out0, out1, 1.0, err, N)

    EINVAL, EUNSUPPORTED = 1, 6
    assert call(x=N) == EINVAL
    assert call(err=N) == EINVAL
    assert call(nimg=0) == EINVAL
    assert call(H=0) == EINVAL
    assert call(W=100) == EINVAL and call(W=64) == EINVAL
    assert call(nimg=2, H=1 << 15, W=1 << 15) == EINVAL  # more than 2^31 - 1 pixels
    assert call(cin=32, nout=64) == EUNSUPPORTED and call(cin=16, nout=16) == EUNSUPPORTED
    assert call(epi=4) == EINVAL and call(epi=-1) == EINVAL
    assert call(out0=N) == EINVAL  # LINEAR writes out0
    assert call(epi=S.EPI_GELU, out0=N, out1=N) == EINVAL  # GELU needs the activation output
    assert call(epi=S.EPI_DGRAD, out1=p) == EINVAL  # DGRAD needs z_prev
    assert call(epi=S.EPI_QUPDATE, nout=16) == EINVAL  # QUPDATE needs q_in


def test_pack_and_surrogate_create_reject_bad_arguments_without_gpu(lib):
    """Host-side checks of qla_pack_conv_weights and qla_surrogate_create."""
    from paper_2301_13601_gb300 import surrogate as S

    L = S._net_lib()
    p = ctypes.c_void_p(256)  # never dereferenced on these paths
    EINVAL = 1
    assert L.qla_pack_conv_weights(None, 64, 64, 64, 64, 0, p, None) == EINVAL
    assert L.qla_pack_conv_weights(p, 64, 64, 64, 60, 0, p, None) == EINVAL  # padding not a multiple of 8
    assert L.qla_pack_conv_weights(p, 64, 72, 64, 64, 0, p, None) == EINVAL  # cin above its padding
    assert L.qla_pack_conv_weights(p, 6, 64, 16, 16, 1, p, None) == EINVAL  # adjoint: cin above nout_pad
    assert L.qla_pack_conv_weights(p, 0, 64, 64, 64, 0, p, None) == EINVAL
    h = ctypes.c_void_p()
    assert L.qla_surrogate_create(None, ctypes.byref(h)) == EINVAL
    for bad in (dict(W=100), dict(W=0), dict(H=0), dict(nimg=0), dict(K=0), dict(out_scale=0.0),
                dict(out_scale=float("nan")), dict(out_scale=-1.0), dict(nimg=4, H=1 << 14, W=1 << 15)):
        c = dict(nimg=1, H=64, W=128, K=16, out_scale=1.0 / 16, train=0, stream=None)
        c.update(bad)
        cfg = S.Config(**c)
        assert L.qla_surrogate_create(ctypes.byref(cfg), ctypes.byref(h)) == EINVAL, bad
        assert not h.value
