"""FP64 CPU oracle of the learned potential predictor (test infrastructure, not product code).

The network replaces the predictor half-step of the predictor-corrector scheme (Program summary:
"a predictor-corrector step when necessary"): from the last four Hartree-exchange potentials it
predicts the next one.  With the backward differences of V0..V3 = V(t), V(t-dt), V(t-2dt), V(t-3dt)
    D1 = V0 - V1,  D2 = V0 - 2 V1 + V2,  D3 = V0 - 3 V1 + 3 V2 - V3,
the input channels (normalised per sample by their root mean square) are
    x0 = D1 / s1,  x1 = D2 / s2,  x2 = D3 / s3,  x3 = (V0 - <V0>) / s_V,
and the output y is a learned correction to the cubic extrapolation through the four potentials,
in units of s3:
    V~(t+dt) = 4 V0 - 6 V1 + 4 V2 - V3 + s3 * y.
A network that outputs zero reproduces the cubic, the best no-network baseline.  Each scale is
floored at 1e-13 rms(V0), so a difference that vanishes to rounding is not amplified.
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


FLOOR = 1e-13


def rms(a):
    return float(np.sqrt(np.mean(a * a)))


def cubic_extrapolation(V0, V1, V2, V3):
    """No-network baseline: the cubic through the last four potentials, evaluated at t + dt."""
    return 4.0 * V0 - 6.0 * V1 + 4.0 * V2 - V3


def inputs(V0, V1, V2, V3):
    """Normalised input channels and the output scale s3 (see module docstring)."""
    D1, D2, D3 = V0 - V1, V0 - 2.0 * V1 + V2, V0 - 3.0 * V1 + 3.0 * V2 - V3
    m = V0.mean()
    fl = FLOOR * rms(V0) + 1e-300
    s1, s2, s3, sv = (max(rms(D), fl) for D in (D1, D2, D3, V0 - m))
    x = np.stack([D1 / s1, D2 / s2, D3 / s3, (V0 - m) / sv])
    return x, s3


def predict(params, V0, V1, V2, V3, periodic):
    x, s3 = inputs(V0, V1, V2, V3)
    out, _ = forward(params, x, periodic)
    return cubic_extrapolation(V0, V1, V2, V3) + s3 * out


def bf16(x):
    """Round to the nearest bfloat16 (8-bit significand, ties to even), returned as float64.  The
    network stores its weights, inputs and activations in this format and accumulates in FP32; the
    rounding is done on the FP32 value, as a device does when it narrows FP32 to BF16."""
    f = np.asarray(x, np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16(params, x, periodic):
    """The forward pass at the network's storage precision: weights, biases, inputs and the two
    hidden activations rounded to BF16, every sum in FP64 (the device sums in FP32; the difference
    is its accumulation rounding and, rarely, a BF16 rounding decision that it flips)."""
    W1, b1, W2, b2, W3, b3 = unpack(bf16(params))
    a1 = bf16(silu(conv(bf16(x), W1, b1, periodic)))
    a2 = bf16(silu(conv(a1, W2, b2, periodic)))
    return conv(a2, W3, b3, periodic)[0]


def predict_bf16(params, V0, V1, V2, V3, periodic):
    """V~(t+dt) of the network as stored (forward_bf16), the scales and the cubic in FP64."""
    x, s3 = inputs(V0, V1, V2, V3)
    return cubic_extrapolation(V0, V1, V2, V3) + s3 * forward_bf16(params, x, periodic)


def target(V0, V1, V2, V3, Vnext, s3):
    return (Vnext - cubic_extrapolation(V0, V1, V2, V3)) / s3


def residual(Vnew, Vpred):
    """||V_new - V~||_2 / ||V_new||_2 (the self-consistency misfit of the predicted potential)."""
    return float(np.linalg.norm(Vnew - Vpred) / np.linalg.norm(Vnew))
