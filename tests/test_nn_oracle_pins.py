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


def test_zero_network_is_linear_extrapolation():
    """With all weights zero the prediction is exactly 2 V(t) - V(t-dt), and the target of a
    potential that moves linearly in time is zero."""
    rng = np.random.default_rng(4)
    V0, D = rng.standard_normal((2, 4, 5, 6))
    V1, V2, V3 = V0 - D, V0 - 2 * D, V0 - 3 * D
    p = np.zeros(N.NPARAMS)
    assert np.allclose(N.predict(p, V0, V1, V2, V3, True), 2 * V0 - V1)
    x, s = N.inputs(V0, V1, V2, V3)
    assert np.allclose(N.target(V0, V1, V0 + D, s), 0.0)
    assert abs(s - np.sqrt(np.mean(D ** 2))) < 1e-14
