"""Pins of the FP64 U-Net oracle (no GPU): the convolution's orientation against shifted
inputs, pooling/upsampling identities, and every gradient against central finite differences.
The second half plants slips in the oracle and checks that one of these pins catches each."""
import numpy as np
import pytest

from oracle import unet_oracle as U


def test_parameter_count():
    assert U.num_params() == 274213


def test_conv3x3_orientation_by_shifts():
    # a kernel with a single 1 at (dy, dx) copies the input shifted by (dy-1, dx-1)
    rng = np.random.default_rng(0)
    x = rng.standard_normal((1, 6, 7, 1))
    for dy in range(3):
        for dx in range(3):
            W = np.zeros((1, 3, 3, 1))
            W[0, dy, dx, 0] = 1.0
            y = U.conv3x3(x, W, np.zeros(1))
            xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
            assert np.array_equal(y, xp[:, dy:dy + 6, dx:dx + 7, :])


def test_conv3x3_channel_mixing():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 4, 4, 3))
    W = np.zeros((2, 3, 3, 3))
    W[1, 1, 1, 2] = 2.0  # output 1 = 2 * input channel 2, output 0 = bias
    y = U.conv3x3(x, W, np.array([0.5, -1.0]))
    assert np.allclose(y[..., 0], 0.5) and np.allclose(y[..., 1], 2 * x[..., 2] - 1.0)


def test_pool_upsample_identities():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 8, 8, 3))
    assert np.allclose(U.avgpool2(U.upsample2(x)), x)
    c = np.full((1, 4, 4, 2), 3.5)
    assert np.allclose(U.avgpool2(c), 3.5)


def test_bf16_rounding():
    assert U.bf16_round(1.0) == 1.0
    assert U.bf16_round(1.0 + 2 ** -9) == 1.0            # tie -> even
    assert U.bf16_round(1.0 + 3 * 2 ** -9) == 1.0 + 2 ** -7
    assert U.bf16_round(-2.5) == -2.5


def _loss(theta, x, dout):
    out, _ = U.forward(theta, x)
    return float(np.sum(out * dout))


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    # He-scaled weights keep activations O(1), so a small step rarely crosses a ReLU kink
    theta = np.concatenate([np.concatenate([rng.standard_normal(co * k * k * ci) * np.sqrt(2.0 / (k * k * ci)),
                                            rng.standard_normal(co) * 0.1]) for ci, co, k in U.SPEC])
    x = rng.standard_normal((1, 16, 16, 2))
    dout = rng.standard_normal((1, 16, 16))
    g = U.backward(theta, x, dout)
    idx = rng.choice(theta.size, 40, replace=False)
    # make sure every layer's weights and the biases are probed
    offs = np.cumsum([0] + [co * k * k * ci + co for ci, co, k in U.SPEC])
    idx = np.concatenate([idx, offs[:-1], offs[1:] - 1])
    eps = 1e-6
    gmax = float(np.max(np.abs(g)))
    for i in idx:
        t1, t2 = theta.copy(), theta.copy()
        t1[i] += eps
        t2[i] -= eps
        fd = (_loss(t1, x, dout) - _loss(t2, x, dout)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-5 * abs(fd) + 1e-8 * gmax, (i, fd, g[i])


def test_features_scale_invariant():
    rng = np.random.default_rng(4)
    f = rng.standard_normal(16 * 16)
    a, rl = U.features(f, 16)
    b, rl2 = U.features(7.0 * f, 16)
    assert np.allclose(a, b) and np.isclose(rl2, 7.0 * rl)
    assert np.isclose(np.sqrt(np.mean(a[..., 0] ** 2)), 1.0)


# --- Planted slips in the U-Net oracle, each caught by one of the pins above -----------------

def _fails(pin):
    try:
        pin()
    except AssertionError:
        return True
    return False


def test_slip_flipped_forward_kernel_is_caught(monkeypatch):
    # convolution (kernel flipped) instead of the cross-correlation the layout defines
    orig = U.conv3x3
    monkeypatch.setattr(U, "conv3x3", lambda x, W, b: orig(x, W[:, ::-1, ::-1, :], b))
    assert _fails(test_conv3x3_orientation_by_shifts)
    assert _fails(test_gradient_matches_central_differences)


def test_slip_unflipped_data_gradient_is_caught(monkeypatch):
    # the data gradient must run the kernel the other way round; reading it as the forward
    # direction (offsets not mirrored) is a classic slip
    def bad(x, W, dout):
        B, H, Wd, C = x.shape
        xp = np.zeros((B, H + 2, Wd + 2, C))
        xp[:, 1:-1, 1:-1, :] = x
        dW = np.zeros_like(W)
        dxp = np.zeros_like(xp)
        for dy in range(3):
            for dx in range(3):
                dW[:, dy, dx, :] = np.einsum("bhwo,bhwi->oi", dout, xp[:, dy:dy + H, dx:dx + Wd, :])
                dxp[:, 2 - dy:2 - dy + H, 2 - dx:2 - dx + Wd, :] += dout @ W[:, dy, dx, :]
        return dxp[:, 1:-1, 1:-1, :], dW, dout.sum(axis=(0, 1, 2))
    monkeypatch.setattr(U, "conv3x3_backward", bad)
    assert _fails(test_gradient_matches_central_differences)


def test_slip_pooling_gradient_scale_is_caught(monkeypatch):
    # the 1/4 of the 2x2 average dropped from its gradient
    monkeypatch.setattr(U, "avgpool2_backward", lambda d: np.repeat(np.repeat(d, 2, axis=1), 2, axis=2))
    assert _fails(test_gradient_matches_central_differences)


def test_slip_upsampling_gradient_averaged_is_caught(monkeypatch):
    # nearest upsampling copies each value four times, so its gradient sums the four (not averages)
    orig = U.upsample2_backward
    monkeypatch.setattr(U, "upsample2_backward", lambda d: 0.25 * orig(d))
    assert _fails(test_gradient_matches_central_differences)


def test_slip_bf16_truncation_is_caught(monkeypatch):
    # chopping the low 16 bits instead of rounding to nearest even
    def chop(a):
        x = np.asarray(a, dtype=np.float32)
        return (x.view(np.uint32) & np.uint32(0xFFFF0000)).view(np.float32).astype(np.float64)
    monkeypatch.setattr(U, "bf16_round", chop)
    assert _fails(test_bf16_rounding)


def test_features_laplacian_stencil():
    # the second input channel is the 5-point stencil 4 f - (four neighbours): on the quadratic
    # f(i, j) = i^2 + j^2 every interior value is -4 (each axis' second difference is 2), and the
    # replicated edge makes the outward second difference along a boundary row i = 0 equal to 1
    # (f(1) - f(0) = 1 on that axis) instead of 2
    n = 12
    i, j = np.meshgrid(np.arange(n, dtype=np.float64), np.arange(n, dtype=np.float64), indexing="ij")
    f = (i * i + j * j).reshape(-1)
    a, rl = U.features(f, n)
    lap = a[0, :, :, 1] * rl
    assert np.allclose(lap[1:-1, 1:-1], -4.0, rtol=0, atol=1e-12)
    assert np.allclose(lap[0, 1:-1], -3.0, rtol=0, atol=1e-12)
