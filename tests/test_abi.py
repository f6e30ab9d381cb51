"""The C-ABI library loads on any machine and exports every symbol include/*.h declares."""
import ctypes
import glob
import os
import re

import pytest

import host_checks

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
    opt = qla.Options()
    L.qla_default_options(ctypes.byref(opt))
    assert opt.launch == qla.LAUNCH_AUTO
    for bad_launch in (-1, 3):  # launch forms: automatic, one launch per pass, persistent
        opt.launch = bad_launch
        assert L.qla_create(4, 4, P(n), P(n), P(n), 0.1, ctypes.byref(opt), None, ctypes.byref(ctx)) == 1
    assert not ctx.value
    # the persistent form's wait hook and launch query reject a missing context
    assert L.qla_set_wait_limit(None, 1000, 0) == 1
    launch = ctypes.c_int()
    assert L.qla_get_launch(None, ctypes.byref(launch)) == 1


def test_conv_rejects_bad_arguments_without_gpu(lib):
    """qla_conv3x3_bf16 checks sizes, channel pairs and epilogue operands on the
    host and returns before any launch. Run with no visible GPU: the stand-in
    device pointers can then reach no device even if a check were missing."""
    host_checks.run_without_gpu("conv_rejects_bad_arguments")


def test_pack_and_surrogate_create_reject_bad_arguments_without_gpu(lib):
    """Host-side checks of qla_pack_conv_weights and qla_surrogate_create (no
    visible GPU, as above)."""
    host_checks.run_without_gpu("pack_and_surrogate_create_reject_bad_arguments")
