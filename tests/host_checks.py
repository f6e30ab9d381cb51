"""Host-side argument checks of the C ABI that must fail before any launch.

They pass stand-in device pointers that must never be dereferenced. The
tests run each function here in a child process whose CUDA_VISIBLE_DEVICES is
empty: if a check were missing, the call would fail with a CUDA error instead
of launching a kernel on a bogus address of a real GPU.
"""
import ctypes
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def run_without_gpu(name: str) -> None:
    env = dict(os.environ)
    env["CUDA_VISIBLE_DEVICES"] = ""
    env["PYTHONPATH"] = os.pathsep.join([ROOT, HERE] + ([env["PYTHONPATH"]] if env.get("PYTHONPATH") else []))
    r = subprocess.run([sys.executable, "-c", f"import host_checks; host_checks.{name}()"], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, f"{name} failed:\n{r.stdout}\n{r.stderr}"


def conv_rejects_bad_arguments():
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


def pack_and_surrogate_create_reject_bad_arguments():
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


def noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2301_13601_gb300.qla import FP32, FP64, Diag, load_library

    L = load_library()
    d = Diag()
    dummy = ctypes.c_void_p(16)  # never dereferenced: the size check comes first
    assert L.qla_diagnostics_noalloc(dummy, FP32, 8, 16385, None, ctypes.byref(d)) == 1
    assert L.qla_diagnostics_noalloc(dummy, FP64, 70000, 70000, None, ctypes.byref(d)) == 1
    assert L.qla_diagnostics_noalloc(dummy, 7, 8, 8, None, ctypes.byref(d)) == 1
    assert L.qla_diagnostics_noalloc(None, FP32, 8, 8, None, ctypes.byref(d)) == 1


def sweep_split_is_host_arithmetic():
    import numpy as np

    from paper_2301_13601_gb300 import qla

    b = qla.sweep_split(8192, 8192, 2, 304)
    assert b[0] == 0 and b[-1] == 35 * 8192 and np.all(np.diff(b) > 0)
    b64 = qla.sweep_split(8192, 8192, 2, 304, "fp64")
    assert b64[-1] == b[-1]
