"""Pins of the learned-predictor oracle (CPU): loop convolution, finite-difference gradients,
and the identity of the prediction formula."""
import numpy as np
import pytest

from oracle import nn_oracle as N


def _rand_params(seed, scale=0.2):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(N.NPARAMS) * scale


def _loop_conv(x, W, b, periodic):
    ci_n, nz, ny, nx = x.shape
    y = np.zeros((W.shape[0], nz, ny, nx))
    offs = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    for co in range(W.shape[0]):
        for z in range(nz):
            for yy in range(ny):
                for xx in range(nx):
                    acc = b[co]
                    for kk, (dz, dy, dx) in enumerate(offs):
                        zz, y2, x2 = z + dz, yy + dy, xx + dx
                        if periodic:
                            zz, y2, x2 = zz % nz, y2 % ny, x2 % nx
                        elif not (0 <= zz < nz and 0 <= y2 < ny and 0 <= x2 < nx):
                            continue
                        acc += W[co, :, kk] @ x[:, zz, y2, x2]
                    y[co, z, yy, xx] = acc
    return y


@pytest.mark.parametrize("periodic", [True, False])
def test_conv_against_loops(periodic):
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, 4, 5, 6))
    W = rng.standard_normal((2, 3, 27))
    b = rng.standard_normal(2)
    assert np.allclose(N.conv(x, W, b, periodic), _loop_conv(x, W, b, periodic), atol=1e-12)


@pytest.mark.parametrize("periodic", [True, False])
def test_gradient_finite_difference(periodic):
    rng = np.random.default_rng(2)
    x = rng.standard_normal((4, 4, 5, 6))
    t = rng.standard_normal((4, 5, 6))
    p = _rand_params(3)
    _, g = N.loss_and_grad(p, x, t, periodic)
    idx = rng.choice(N.NPARAMS, 40, replace=False)
    idx = np.concatenate([idx, [N.NPARAMS - 1, 16 * 4 * 27 + 3, N.NPARAMS - 433]])   # biases too
    eps = 1e-6
    for i in idx:
        e = np.zeros(N.NPARAMS)
        e[i] = eps
        fd = (N.loss_and_grad(p + e, x, t, periodic)[0] - N.loss_and_grad(p - e, x, t, periodic)[0]) / (2 * eps)
        assert abs(fd - g[i]) < 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_silu_derivative():
    y = np.linspace(-6, 6, 101)
    h = 1e-6
    assert np.allclose((N.silu(y + h) - N.silu(y - h)) / (2 * h), N.dsilu(y), atol=1e-8)


def test_zero_network_is_cubic_extrapolation():
    """With all weights zero the prediction is the cubic through the four potentials; a potential
    cubic in time is predicted exactly (target 0), and its vanishing fourth difference is not
    amplified by the normalisation (floored scales)."""
    rng = np.random.default_rng(4)
    V0, D, Q, R = rng.standard_normal((4, 4, 5, 6))
    V = [V0 - k * D + 0.5 * k * k * Q - k ** 3 * R / 6 for k in range(5)]     # V(t - k dt), k = -1..3 below
    Vnext = V0 + D + 0.5 * Q + R / 6
    p = np.zeros(N.NPARAMS)
    assert np.allclose(N.predict(p, *V[:4], True), N.cubic_extrapolation(*V[:4]))
    assert np.allclose(N.cubic_extrapolation(*V[:4]), Vnext)
    x, s3 = N.inputs(*V[:4])
    assert np.all(np.isfinite(x)) and np.max(np.abs(x)) < 50
    assert np.max(np.abs(N.target(*V[:4], Vnext, s3))) < 1e-10


def test_scales_and_channels():
    """Channels are the backward differences over their root mean squares; a quadratic potential has
    a third difference at rounding level, which the floor keeps from being blown up to O(1)."""
    rng = np.random.default_rng(8)
    V = rng.standard_normal((4, 4, 5, 6))
    x, s3 = N.inputs(*V)
    D2 = V[0] - 2 * V[1] + V[2]
    D3 = V[0] - 3 * V[1] + 3 * V[2] - V[3]
    assert np.allclose(x[1] * N.rms(D2), D2) and abs(s3 - N.rms(D3)) < 1e-14
    V0, D, Q = rng.standard_normal((3, 4, 5, 6))
    Vq = [V0 - k * D + 0.5 * k * k * Q for k in range(4)]
    xq, _ = N.inputs(*Vq)
    assert np.max(np.abs(xq[2])) < 0.1
