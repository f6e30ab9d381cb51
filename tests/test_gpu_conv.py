"""tcgen05 BF16 convolution (qla_conv3x3_bf16) against the FP64 numpy reference.

Inputs and weights are rounded to BF16 first, so the reference sees exactly the
operands the tensor cores multiply; the remaining difference is FP32
accumulation order over K = 9 * cin products (relative ~1e-6) plus, for BF16
outputs, one rounding (2^-8 relative).
"""
import numpy as np
import pytest
import torch

from oracle import cnn
from paper_2301_13601_gb300 import surrogate as S

pytestmark = pytest.mark.gpu

dev = "cuda"


def bf16_round(a):
    return torch.as_tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()


def make_case(H, W, cin, nout, seed):
    rng = np.random.default_rng(seed)
    x = bf16_round(rng.standard_normal((H, W, cin)))
    w = rng.standard_normal((nout, cin, 3, 3)) / np.sqrt(9 * cin)
    wq = bf16_round(w)
    b = rng.standard_normal(nout) * 0.1
    return x, w, wq, b


def to_dev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=dev)


def packed(w, cin_pad, nout_pad, flip=False):
    wt = to_dev(w, torch.float32)
    out = torch.empty(9 * cin_pad * nout_pad, dtype=torch.bfloat16, device=dev)
    S.pack_weights(wt, out, nout_pad, cin_pad, transpose_flip=flip)
    return out


SHAPES = [(1, 128), (3, 128), (5, 256), (160, 256)]  # one row (all taps wrap), x-wrap in one tile, >1 tile per CTA


@pytest.mark.parametrize("cin,nout", [(16, 64), (64, 64), (64, 16)])
@pytest.mark.parametrize("H,W", SHAPES)
def test_conv_linear_matches_reference(cin, nout, H, W):
    x, w, wq, b = make_case(H, W, cin, nout, seed=H * 7 + cin + nout)
    ref = cnn.conv3x3(x, wq, b)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    out = torch.empty((H, W, nout), dtype=torch.float32, device=dev)
    S.conv3x3(to_dev(x, torch.bfloat16), packed(w, cin, nout), nout, S.EPI_LINEAR, out,
              bias=to_dev(b, torch.float32), error_flag=err)
    torch.cuda.synchronize()
    assert err.item() == 0
    got = out.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - ref)) <= 2e-5 * np.max(np.abs(ref)) + 1e-6


@pytest.mark.parametrize("residual", [False, True])
def test_conv_gelu_epilogue(residual):
    H, W, cin, nout = 4, 256, 64, 64
    x, w, wq, b = make_case(H, W, cin, nout, seed=11)
    res = bf16_round(np.random.default_rng(12).standard_normal((H, W, nout))) if residual else None
    z = cnn.conv3x3(x, wq, b)
    act = cnn.gelu(z) + (res if residual else 0.0)
    zo = torch.empty((H, W, nout), dtype=torch.bfloat16, device=dev)
    ao = torch.empty_like(zo)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    S.conv3x3(to_dev(x, torch.bfloat16), packed(w, cin, nout), nout, S.EPI_GELU, zo, ao,
              bias=to_dev(b, torch.float32), aux0=to_dev(res, torch.bfloat16) if residual else None, error_flag=err)
    torch.cuda.synchronize()
    assert err.item() == 0
    zg = zo.float().cpu().numpy()
    ag = ao.float().cpu().numpy()
    assert np.max(np.abs(zg - z) / (np.abs(z) + 1e-3)) < 2 ** -8 * 1.01
    assert np.max(np.abs(ag - act)) < 2 ** -8 * (np.abs(act).max() + 1.0) * 1.5


# Long runs of rows per CTA (152 CTAs): more rows than the TMEM accumulator ring
# holds (8 blocks for 64 outputs, 32 for 16), runs that cross column blocks and
# images, and, for 64 -> 64, the residual read from the staged input rows.
@pytest.mark.parametrize("cin,nout,nimg,H,W", [(64, 16, 2, 320, 1024), (64, 64, 2, 200, 1024), (16, 64, 1, 400, 512)])
def test_conv_long_runs_match_reference(cin, nout, nimg, H, W):
    rng = np.random.default_rng(cin * 3 + nout + H)
    x = bf16_round(rng.standard_normal((nimg, H, W, cin)))
    w = rng.standard_normal((nout, cin, 3, 3)) / np.sqrt(9 * cin)
    wq = bf16_round(w)
    b = rng.standard_normal(nout) * 0.1
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    xd = to_dev(x, torch.bfloat16)
    if cin == nout:
        ao = torch.empty((nimg, H, W, nout), dtype=torch.bfloat16, device=dev)
        S.conv3x3(xd, packed(w, cin, nout), nout, S.EPI_GELU, None, ao, bias=to_dev(b, torch.float32), aux0=xd,
                  error_flag=err)
    else:
        out = torch.empty((nimg, H, W, nout), dtype=torch.float32, device=dev)
        S.conv3x3(xd, packed(w, cin, nout), nout, S.EPI_LINEAR, out, bias=to_dev(b, torch.float32), error_flag=err)
    torch.cuda.synchronize()
    assert err.item() == 0
    for i in range(nimg):
        z = cnn.conv3x3(x[i], wq, b)
        if cin == nout:
            act = cnn.gelu(z) + x[i]
            got = ao[i].float().cpu().numpy()
            assert np.max(np.abs(got - act)) < 2 ** -8 * (np.abs(act).max() + 1.0) * 1.5
        else:
            got = out[i].cpu().numpy().astype(np.float64)
            assert np.max(np.abs(got - z)) <= 2e-5 * np.max(np.abs(z)) + 1e-6


def test_transpose_flip_is_the_input_gradient():
    """Packing with transpose_flip turns the conv into its adjoint (dgrad)."""
    H, W, cin, nout = 3, 128, 64, 16  # forward layer 64 -> 16; dgrad maps 16 -> 64
    _, w, wq, _ = make_case(H, W, cin, nout, seed=21)
    g = bf16_round(np.random.default_rng(22).standard_normal((H, W, nout)))
    ref = cnn.conv3x3_input_grad(g, wq)
    out = torch.empty((H, W, cin), dtype=torch.float32, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    S.conv3x3(to_dev(g, torch.bfloat16), packed(w, cin_pad=16, nout_pad=64, flip=True), cin, S.EPI_LINEAR, out,
              error_flag=err)
    torch.cuda.synchronize()
    assert err.item() == 0
    got = out.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 2e-5 * np.max(np.abs(ref)) + 1e-6


def test_dgrad_epilogue():
    H, W, c = 3, 128, 64
    _, w, wq, _ = make_case(H, W, c, c, seed=31)
    rng = np.random.default_rng(32)
    dz = bf16_round(rng.standard_normal((H, W, c)))
    gin = rng.standard_normal((H, W, c)).astype(np.float32).astype(np.float64)
    zprev = bf16_round(rng.standard_normal((H, W, c)))
    g = cnn.conv3x3_input_grad(dz, wq) + gin
    dzp = g * cnn.gelu_grad(zprev)
    go = torch.empty((H, W, c), dtype=torch.float32, device=dev)
    dzo = torch.empty((H, W, c), dtype=torch.bfloat16, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    S.conv3x3(to_dev(dz, torch.bfloat16), packed(w, c, c, flip=True), c, S.EPI_DGRAD, go, dzo,
              aux0=to_dev(gin, torch.float32), zprev=to_dev(zprev, torch.bfloat16), error_flag=err)
    torch.cuda.synchronize()
    assert err.item() == 0
    assert np.max(np.abs(go.cpu().numpy() - g)) <= 2e-5 * np.abs(g).max()
    d = dzo.float().cpu().numpy()
    assert np.max(np.abs(d - dzp)) <= 2 ** -8 * 1.5 * np.abs(dzp).max() + 1e-5


def test_qupdate_epilogue():
    H, W, cin, nout = 2, 256, 64, 16
    x, w, wq, b = make_case(H, W, cin, nout, seed=41)
    q = np.random.default_rng(42).standard_normal((6, H, W)).astype(np.float32)
    scale = 0.0625
    acc = cnn.conv3x3(x, wq, b)
    ref = q + scale * np.moveaxis(acc[:, :, :6], 2, 0)
    qo = torch.empty((6, H, W), dtype=torch.float32, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    S.conv3x3(to_dev(x, torch.bfloat16), packed(w, cin, nout), nout, S.EPI_QUPDATE, qo,
              bias=to_dev(b, torch.float32), aux0=to_dev(q, torch.float32), scale=scale, error_flag=err)
    torch.cuda.synchronize()
    assert err.item() == 0
    assert np.max(np.abs(qo.cpu().numpy() - ref)) <= 1e-5 * np.abs(ref).max()


def test_conv_rejects_bad_arguments():
    from paper_2301_13601_gb300.qla import QLAError

    x = torch.zeros((2, 100, 64), dtype=torch.bfloat16, device=dev)  # W not a multiple of 128
    w = torch.zeros(9 * 64 * 64, dtype=torch.bfloat16, device=dev)
    out = torch.zeros((2, 100, 64), dtype=torch.float32, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    with pytest.raises(QLAError):
        S.conv3x3(x, w, 64, S.EPI_LINEAR, out, error_flag=err)
    x = torch.zeros((2, 128, 32), dtype=torch.bfloat16, device=dev)  # unsupported channel count
    with pytest.raises(QLAError):
        S.conv3x3(x, w, 64, S.EPI_LINEAR, out, error_flag=err)


def test_images_wrap_on_their_own():
    """nimg stacked images: each is periodic by itself (no leakage between images)."""
    nimg, H, W, cin, nout = 3, 2, 128, 64, 16
    rng = np.random.default_rng(51)
    x = bf16_round(rng.standard_normal((nimg, H, W, cin)))
    w = rng.standard_normal((nout, cin, 3, 3)) / np.sqrt(9 * cin)
    wq = bf16_round(w)
    b = rng.standard_normal(nout) * 0.1
    q = rng.standard_normal((nimg, 6, H, W)).astype(np.float32)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    out = torch.empty((nimg, H, W, nout), dtype=torch.float32, device=dev)
    xd = to_dev(x, torch.bfloat16)
    wp = packed(w, cin, nout)
    S.conv3x3(xd, wp, nout, S.EPI_LINEAR, out, bias=to_dev(b, torch.float32), error_flag=err)
    qo = torch.empty((nimg, 6, H, W), dtype=torch.float32, device=dev)
    S.conv3x3(xd, wp, nout, S.EPI_QUPDATE, qo, bias=to_dev(b, torch.float32), aux0=to_dev(q, torch.float32),
              scale=0.5, error_flag=err)
    torch.cuda.synchronize()
    assert err.item() == 0
    got = out.cpu().numpy()
    for i in range(nimg):
        ref = cnn.conv3x3(x[i], wq, b)
        assert np.max(np.abs(got[i] - ref)) <= 2e-5 * np.max(np.abs(ref))
        refq = q[i] + 0.5 * np.moveaxis(ref[:, :, :6], 2, 0)
        assert np.max(np.abs(qo[i].cpu().numpy() - refq)) <= 1e-5 * np.abs(refq).max()


def test_gelu_without_z_store():
    H, W, cin, nout = 2, 128, 16, 64
    x, w, wq, b = make_case(H, W, cin, nout, seed=61)
    act = cnn.gelu(cnn.conv3x3(x, wq, b))
    ao = torch.empty((H, W, nout), dtype=torch.bfloat16, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    S.conv3x3(to_dev(x, torch.bfloat16), packed(w, cin, nout), nout, S.EPI_GELU, None, ao,
              bias=to_dev(b, torch.float32), error_flag=err)
    torch.cuda.synchronize()
    assert err.item() == 0
    assert np.max(np.abs(ao.float().cpu().numpy() - act)) < 2 ** -8 * 1.5 * (np.abs(act).max() + 1.0)


@pytest.mark.parametrize("cin,nout", [(64, 64), (16, 64)])
def test_long_row_segments(cin, nout):
    """Many rows per CTA: the rolling window crosses column blocks and images."""
    nimg, H, W = 2, 700, 256
    rng = np.random.default_rng(71)
    x = bf16_round(rng.standard_normal((nimg, H, W, cin)))
    w = rng.standard_normal((nout, cin, 3, 3)) / np.sqrt(9 * cin)
    wq = bf16_round(w)
    b = rng.standard_normal(nout) * 0.1
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    out = torch.empty((nimg, H, W, nout), dtype=torch.float32, device=dev)
    S.conv3x3(to_dev(x, torch.bfloat16), packed(w, cin, nout), nout, S.EPI_LINEAR, out,
              bias=to_dev(b, torch.float32), error_flag=err)
    torch.cuda.synchronize()
    assert err.item() == 0
    got = out.cpu().numpy()
    for i in range(nimg):
        ref = cnn.conv3x3(x[i], wq, b)
        assert np.max(np.abs(got[i] - ref)) <= 2e-5 * np.max(np.abs(ref))


def test_residual_from_global_memory():
    """EPI_GELU with a residual tensor other than the input (read from global memory)."""
    H, W, c = 3, 128, 64
    x, w, wq, b = make_case(H, W, c, c, seed=81)
    res = bf16_round(np.random.default_rng(82).standard_normal((H, W, c)))
    act = cnn.gelu(cnn.conv3x3(x, wq, b)) + res
    ao = torch.empty((H, W, c), dtype=torch.bfloat16, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    S.conv3x3(to_dev(x, torch.bfloat16), packed(w, c, c), c, S.EPI_GELU, None, ao, bias=to_dev(b, torch.float32),
              aux0=to_dev(res, torch.bfloat16), error_flag=err)
    torch.cuda.synchronize()
    assert err.item() == 0
    assert np.max(np.abs(ao.float().cpu().numpy() - act)) < 2 ** -8 * 1.5 * (np.abs(act).max() + 1.0)


def test_residual_from_staged_input():
    """EPI_GELU with the residual equal to the input: read from the staged rows."""
    H, W, c = 5, 256, 64
    x, w, wq, b = make_case(H, W, c, c, seed=91)
    act = cnn.gelu(cnn.conv3x3(x, wq, b)) + x
    xd = to_dev(x, torch.bfloat16)
    zo = torch.empty((H, W, c), dtype=torch.bfloat16, device=dev)
    ao = torch.empty_like(zo)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    S.conv3x3(xd, packed(w, c, c), c, S.EPI_GELU, zo, ao, bias=to_dev(b, torch.float32), aux0=xd, error_flag=err)
    torch.cuda.synchronize()
    assert err.item() == 0
    assert np.max(np.abs(ao.float().cpu().numpy() - act)) < 2 ** -8 * 1.5 * (np.abs(act).max() + 1.0)
