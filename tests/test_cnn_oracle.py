"""Pins of the surrogate's numpy reference (oracle/cnn.py) against things other than itself."""
import numpy as np
import pytest
from scipy import ndimage, special

from oracle import cnn


def test_conv3x3_is_wrap_mode_correlation():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((5, 7, 3))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = cnn.conv3x3(x, w, b)
    for n in range(4):
        ref = b[n] + sum(ndimage.correlate(x[:, :, c], w[n, c], mode="wrap") for c in range(3))
        assert np.allclose(y[:, :, n], ref, atol=1e-12)


def test_conv3x3_brute_force_tiny():
    rng = np.random.default_rng(1)
    H, W = 3, 4
    x = rng.standard_normal((H, W, 2))
    w = rng.standard_normal((2, 2, 3, 3))
    y = cnn.conv3x3(x, w)
    for i in range(H):
        for j in range(W):
            for n in range(2):
                s = 0.0
                for ky in range(3):
                    for kx in range(3):
                        for c in range(2):
                            s += w[n, c, ky, kx] * x[(i + ky - 1) % H, (j + kx - 1) % W, c]
                assert abs(y[i, j, n] - s) < 1e-12


def test_input_and_weight_grads_are_adjoints():
    """<conv(x, w), g> = <x, dgrad(g, w)> = <w, wgrad(g, x)>."""
    rng = np.random.default_rng(2)
    x = rng.standard_normal((6, 5, 3))
    w = rng.standard_normal((4, 3, 3, 3))
    g = rng.standard_normal((6, 5, 4))
    lhs = np.sum(cnn.conv3x3(x, w) * g)
    assert abs(lhs - np.sum(x * cnn.conv3x3_input_grad(g, w))) < 1e-10
    assert abs(lhs - np.sum(w * cnn.conv3x3_weight_grad(g, x))) < 1e-10


def test_gelu_tanh_form_close_to_erf_form():
    x = np.linspace(-6, 6, 1001)
    exact = 0.5 * x * (1 + special.erf(x / np.sqrt(2)))
    assert np.max(np.abs(cnn.gelu(x) - exact)) < 1e-3
    assert cnn.gelu(0.0) == 0.0
    h = 1e-6
    fd = (cnn.gelu(x + h) - cnn.gelu(x - h)) / (2 * h)
    assert np.max(np.abs(fd - cnn.gelu_grad(x))) < 1e-8


@pytest.mark.parametrize("k,idx", [(0, (1, 2, 0, 1)), (2, (3, 1, 2, 2)), (5, (4, 0, 1, 0))])
def test_backward_matches_finite_differences(k, idx):
    rng = np.random.default_rng(3)
    ch = [9, 4, 4, 4, 4, 4, 6]
    ws = [rng.standard_normal((ch[i + 1], ch[i], 3, 3)) * 0.3 for i in range(6)]
    bs = [rng.standard_normal(ch[i + 1]) * 0.1 for i in range(6)]
    x = rng.standard_normal((5, 6, 9))
    dout = rng.standard_normal((5, 6, 6))
    _, cache = cnn.forward(x, ws, bs, 0.7)
    dW, dB = cnn.backward(dout, ws, cache, 0.7)

    def f():
        return np.sum(dout * cnn.forward(x, ws, bs, 0.7)[0])

    e = 1e-6
    ws[k][idx] += e
    fp = f()
    ws[k][idx] -= 2 * e
    fm = f()
    ws[k][idx] += e
    assert abs((fp - fm) / (2 * e) - dW[k][idx]) < 1e-6 * max(1.0, abs(dW[k][idx]))
    bs[k][0] += e
    fp = f()
    bs[k][0] -= 2 * e
    fm = f()
    bs[k][0] += e
    assert abs((fp - fm) / (2 * e) - dB[k][0]) < 1e-6 * max(1.0, abs(dB[k][0]))
