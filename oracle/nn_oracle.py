"""FP64 CPU oracle of the learned potential predictor (test infrastructure, not product code).

The network replaces the predictor half-step of the predictor-corrector scheme (Program summary:
"a predictor-corrector step when necessary"): from the last four Hartree-exchange potentials it
predicts the next one.  Inputs (channels, normalised per sample):
    x0 = (V(t) - V(t-dt)) / s,  x1 = (V(t-dt) - V(t-2dt)) / s,  x2 = (V(t-2dt) - V(t-3dt)) / s,
    x3 = (V(t) - <V(t)>) / s_V,
with s = rms(V(t) - V(t-dt)) and s_V = rms(V(t) - <V(t)>).  Output y: the correction to the linear
extrapolation, V~(t+dt) = 2 V(t) - V(t-dt) + s * y.
Network: conv3d 4->16, SiLU, conv3d 16->16, SiLU, conv3d 16->1, 3^3 kernels with bias, periodic
(circular) padding for periodic cells, zero padding for isolated ones.  Loss: mean squared error.

Only the tests may import this module.  Parity status: the forward pass is pinned against an
explicit-loop convolution and the backward pass against central finite differences (CPU tests).
"""
from __future__ import annotations

import numpy as np

C1, C2 = 16, 16
SHAPES = [(C1, 4, 27), (C1,), (C2, C1, 27), (C2,), (1, C2, 27), (1,)]
NPARAMS = int(sum(np.prod(s) for s in SHAPES))


def unpack(params):
    out, o = [], 0
    for s in SHAPES:
        n = int(np.prod(s))
        out.append(np.asarray(params[o:o + n], np.float64).reshape(s))
        o += n
    return out


def pack(arrs):
    return np.concatenate([np.asarray(a, np.float64).ravel() for a in arrs])


def _offsets():
    return [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def shift(x, d, periodic):
    """Array whose value at grid point r is x at r + d (d = (dz, dy, dx)); zero outside if isolated."""
    if periodic:
        return np.roll(x, shift=(-d[0], -d[1], -d[2]), axis=(-3, -2, -1))
    out = np.zeros_like(x)
    src, dst = [Ellipsis], [Ellipsis]
    for k, n in zip(d, x.shape[-3:]):
        if k >= 0:
            src.append(slice(k, n)); dst.append(slice(0, n - k))
        else:
            src.append(slice(0, n + k)); dst.append(slice(-k, n))
    out[tuple(dst)] = x[tuple(src)]
    return out


def conv(x, W, b, periodic):
    """y[co, r] = b[co] + sum_ci sum_kk W[co, ci, kk] x[ci, r + off(kk)], x: [ci, nz, ny, nx]."""
    y = np.broadcast_to(b[:, None, None, None], (W.shape[0],) + x.shape[1:]).copy()
    for kk, d in enumerate(_offsets()):
        xs = shift(x, d, periodic)
        y += np.einsum("oc,czyx->ozyx", W[:, :, kk], xs)
    return y


def conv_bwd(x, W, dy, periodic):
    """Gradients of sum(dy * conv(x, W, b)) with respect to x, W and b."""
    dW = np.zeros_like(W)
    dx = np.zeros_like(x)
    for kk, d in enumerate(_offsets()):
        xs = shift(x, d, periodic)
        dW[:, :, kk] = np.einsum("ozyx,czyx->oc", dy, xs)
        back = np.einsum("oc,ozyx->czyx", W[:, :, kk], dy)
        dx += shift(back, (-d[0], -d[1], -d[2]), periodic)
    return dx, dW, dy.sum(axis=(1, 2, 3))


def silu(y):
    return y / (1.0 + np.exp(-y))


def dsilu(y):
    s = 1.0 / (1.0 + np.exp(-y))
    return s * (1.0 + y * (1.0 - s))


def forward(params, x, periodic):
    W1, b1, W2, b2, W3, b3 = unpack(params)
    y1 = conv(x, W1, b1, periodic)
    a1 = silu(y1)
    y2 = conv(a1, W2, b2, periodic)
    a2 = silu(y2)
    out = conv(a2, W3, b3, periodic)[0]
    return out, (x, y1, a1, y2, a2)


def loss_and_grad(params, x, target, periodic):
    """MSE loss mean((out - target)^2) and its gradient with respect to all parameters."""
    W1, b1, W2, b2, W3, b3 = unpack(params)
    out, (x, y1, a1, y2, a2) = forward(params, x, periodic)
    n = out.size
    loss = float(np.mean((out - target) ** 2))
    dout = (2.0 / n) * (out - target)
    da2, dW3, db3 = conv_bwd(a2, W3, dout[None], periodic)
    dy2 = da2 * dsilu(y2)
    da1, dW2, db2 = conv_bwd(a1, W2, dy2, periodic)
    dy1 = da1 * dsilu(y1)
    _, dW1, db1 = conv_bwd(x, W1, dy1, periodic)
    return loss, pack([dW1, db1, dW2, db2, dW3, db3])


def inputs(V0, V1, V2, V3):
    """Normalised input channels and the scale s (see module docstring)."""
    s = np.sqrt(np.mean((V0 - V1) ** 2))
    m = V0.mean()
    sv = np.sqrt(np.mean((V0 - m) ** 2))
    x = np.stack([(V0 - V1) / s, (V1 - V2) / s, (V2 - V3) / s, (V0 - m) / sv])
    return x, s


def predict(params, V0, V1, V2, V3, periodic):
    x, s = inputs(V0, V1, V2, V3)
    out, _ = forward(params, x, periodic)
    return 2.0 * V0 - V1 + s * out


def target(V0, V1, Vnext, s):
    return (Vnext - (2.0 * V0 - V1)) / s


def residual(Vnew, Vpred):
    """||V_new - V~||_2 / ||V_new||_2 (the self-consistency misfit of the predicted potential)."""
    return float(np.linalg.norm(Vnew - Vpred) / np.linalg.norm(Vnew))
