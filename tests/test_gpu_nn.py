"""Learned potential predictor on the GPU against its FP64 oracle, and the predicted step modes.

The GPU network stores weights and activations as BF16 and accumulates in FP32.  The oracle is
evaluated on the same BF16-rounded weights, inputs and activations (the rounding is emulated here
with round-to-nearest-even), so the remaining differences are FP32 accumulation order and the
rare BF16 rounding decision it flips: 1e-3 relative (L2) is required.
"""
import numpy as np
import pytest

from oracle import nn_oracle as N
from oracle import tdks_oracle as O
from paper_1804_01404_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def bf16(x):
    f = np.asarray(x, np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _ctx(s, precision="f64"):
    from paper_1804_01404_gb300.tdks import Context
    return Context(s, precision=precision)


def _hist(s, seed):
    """Five consecutive potentials with generic (non-polynomial) time dependence."""
    rng = np.random.default_rng(seed)
    shape = (s.n[2], s.n[1], s.n[0])
    base, d, c, e = (rng.standard_normal(shape) for _ in range(4))
    V = [base + 0.01 * np.sin(0.3 * k) * d + 0.002 * np.cos(0.7 * k) * c + 0.001 * np.sin(1.3 * k) * e
         for k in range(5)]                                 # V(t-3dt) .. V(t+dt)
    return V[3], V[2], V[1], V[0], V[4]


def _emulated_forward(params, V0, V1, V2, V3, periodic):
    x, s = N.inputs(V0, V1, V2, V3)
    x = bf16(x)
    W1, b1, W2, b2, W3, b3 = N.unpack(bf16(params))
    y1 = N.conv(x, W1, b1, periodic)
    a1 = bf16(N.silu(y1))
    y2 = N.conv(a1, W2, b2, periodic)
    a2 = bf16(N.silu(y2))
    out = N.conv(a2, W3, b3, periodic)[0]
    return out, s, (x, y1, a1, y2, a2)


# tiny grids, the bench crystal's 20^3 grid, and the 48^3 isolated grid of the cluster variant the
# predictor is meant for
SYS = {"periodic": W.tiny(periodic=True, n=(8, 9, 10)), "isolated": W.tiny(periodic=False, n=(9, 8, 7)),
       "crystal20": W.tiny(periodic=True, n=(20, 20, 20)), "cluster48": W.tiny(periodic=False, n=(48, 48, 48))}


@pytest.mark.parametrize("name", list(SYS))
def test_nn_forward_parity(name):
    s = SYS[name]
    ctx = _ctx(s)
    ctx.nn_init(3)
    rng = np.random.default_rng(1)
    params = rng.standard_normal(N.NPARAMS) * 0.15
    ctx.nn_params(params)
    V0, V1, V2, V3, _ = _hist(s, 2)
    vh = torch.from_numpy(np.stack([V0, V1, V2, V3])).to("cuda")
    vp = torch.empty_like(vh[0])
    ctx.nn_predict(vh, vp, mode=2)
    got = (vp.cpu().numpy() - N.cubic_extrapolation(V0, V1, V2, V3))
    out, sc, _ = _emulated_forward(params, V0, V1, V2, V3, s.periodic)
    ref = sc * out
    assert np.linalg.norm(got - ref) < 1e-3 * np.linalg.norm(ref)
    ctx.nn_predict(vh, vp, mode=0)
    assert np.max(np.abs(vp.cpu().numpy() - (2 * V0 - V1))) < 1e-14 * np.max(np.abs(V0))
    ctx.nn_predict(vh, vp, mode=1)
    assert np.max(np.abs(vp.cpu().numpy() - N.cubic_extrapolation(V0, V1, V2, V3))) < 1e-13 * np.max(np.abs(V0))


@pytest.mark.parametrize("name", list(SYS))
def test_nn_gradient_parity(name):
    s = SYS[name]
    ctx = _ctx(s)
    ctx.nn_init(4)
    rng = np.random.default_rng(5)
    params = rng.standard_normal(N.NPARAMS) * 0.15
    ctx.nn_params(params)
    V0, V1, V2, V3, V4 = _hist(s, 6)
    vh = torch.from_numpy(np.stack([V0, V1, V2, V3])).to("cuda")
    vn = torch.from_numpy(V4).to("cuda")
    loss, g = ctx.nn_gradient(vh, vn)
    # oracle gradient through the same BF16-rounded tensors
    out, sc, (x, y1, a1, y2, a2) = _emulated_forward(params, V0, V1, V2, V3, s.periodic)
    W1, b1, W2, b2, W3, b3 = N.unpack(bf16(params))
    t = N.target(V0, V1, V2, V3, V4, sc)
    n = out.size
    dout = (2.0 / n) * (out - t)
    da2, dW3, db3 = N.conv_bwd(a2, W3, dout[None], s.periodic)
    dy2 = da2 * N.dsilu(y2)
    da1, dW2, db2 = N.conv_bwd(a1, W2, dy2, s.periodic)
    dy1 = da1 * N.dsilu(y1)
    _, dW1, db1 = N.conv_bwd(x, W1, dy1, s.periodic)
    ref = N.pack([dW1, db1, dW2, db2, dW3, db3])
    assert abs(loss - np.mean((out - t) ** 2)) < 1e-4 * abs(loss)
    assert np.linalg.norm(g - ref) < 2e-3 * np.linalg.norm(ref)
    for sl in (slice(0, 1728), slice(1744, 8656), slice(8672, 9104)):     # each layer on its own
        assert np.linalg.norm(g[sl] - ref[sl]) < 5e-3 * np.linalg.norm(ref[sl])


def test_nn_training_reduces_loss():
    """A potential whose steps follow a fixed quadratic-in-time pattern: the network learns the
    curvature correction that linear extrapolation misses."""
    s = W.tiny(periodic=True, n=(8, 8, 8))
    ctx = _ctx(s)
    ctx.nn_init(1)
    rng = np.random.default_rng(7)
    shape = (8, 8, 8)
    base, d, c = rng.standard_normal(shape), 0.01 * rng.standard_normal(shape), 0.001 * rng.standard_normal(shape)
    seq = np.stack([base + np.sin(0.2 * k) * d + np.cos(0.35 * k) * c for k in range(40)])
    vseq = torch.from_numpy(seq).to("cuda")
    loss = ctx.nn_train(vseq, epochs=30, batch=4, lr=3e-3, seed=2)
    assert np.all(np.isfinite(loss))
    assert loss[-1] < 0.3 * loss[0], loss


def _steps(s, psi0, n, mode, thr, precision="f64", init_nn=False):
    from paper_1804_01404_gb300 import tdks as T
    ctx = _ctx(s, precision)
    u = torch.from_numpy(psi0).to("cuda", torch.complex128 if precision == "f64" else torch.complex64)
    ctx.update_potential(u)
    if init_nn:
        ctx.nn_init(0)
    if mode != T.PRED_PC:
        ctx.set_predictor(mode, thr)
    J, res = [], []
    t = 0.0
    for _ in range(n):
        ctx.step(u, t, s.dt)
        t += s.dt
        o = ctx.read_step_observables()
        J.append(o["J"])
        res.append(o["residual"])
    return np.array(J), np.array(res), o["fallbacks"], u.cpu().numpy()


def test_predicted_step_fallback_equals_pc():
    """With a threshold no prediction can meet, every predicted step is undone and redone with the
    plain PC: the run must equal the PC run."""
    from paper_1804_01404_gb300 import tdks as T
    s = W.small_periodic(nsteps=12)
    psi0 = W.initial_orbitals(s, 0)
    J0, _, _, u0 = _steps(s, psi0, 12, T.PRED_PC, 1e-5)
    J1, _, fb, u1 = _steps(s, psi0, 12, T.PRED_EXTRAP, 1e-300)
    assert fb == 12 - 3                   # the first three steps build the history
    assert np.max(np.abs(J1 - J0)) < 1e-12 * np.max(np.abs(J0))
    assert np.linalg.norm(u1 - u0) < 1e-12 * np.linalg.norm(u0)


def test_trained_network_beats_cubic_extrapolation_on_held_out_trajectory():
    """What the network gains over the method without it: trained on V_Hxc histories the method
    itself generates (plain predictor-corrector, small periodic cell, seeds 1-3), it predicts the
    next potential of a held-out trajectory (seed 11) better than the cubic extrapolation it
    corrects, and far better than the linear one."""
    from paper_1804_01404_gb300 import learned as L
    s = W.small_periodic(nsteps=200)
    trajs = [L.trajectory(s, W.initial_orbitals(s, seed), 150, "f32") for seed in (1, 2, 3)]
    held = L.trajectory(s, W.initial_orbitals(s, 11), 60, "f32")
    ctx = _ctx(s, "f32")
    ctx.nn_init(1)
    before = np.mean(L.misfits(ctx, held, 2))
    loss = L.train(ctx, trajs, epochs=4, batch=8, lr=1e-3, seed=3)
    lin, cub, net = (np.mean(L.misfits(ctx, held, m)) for m in (0, 1, 2))
    assert np.all(np.isfinite(loss)) and loss[-1] < loss[0]
    assert net < 0.95 * cub, (lin, cub, net, before)
    assert net < 0.1 * lin
