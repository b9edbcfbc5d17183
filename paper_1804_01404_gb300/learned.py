"""Training and evaluation of the learned potential predictor (host orchestration only).

Every computation runs in libtdks kernels through the C ABI: the trajectories that train the network
are produced by the method itself (tdks_step with the plain predictor-corrector), the network is
trained by tdks_nn_train, and evaluation runs tdks_step with each predictor mode.  This module only
moves device buffers between those calls and collects numbers.
"""
from __future__ import annotations

import time

import numpy as np


def trajectory(system, psi0, nsteps, precision="f32", t0=0.0, kick=None):
    """V_Hxc(t) for t = t0 .. t0 + nsteps dt along a plain predictor-corrector run, as a CUDA float64
    tensor [nsteps + 1, nz, ny, nx].  kick: optional impulse exp(i kappa.r) applied first (tdks_kick)."""
    import torch
    from .tdks import Context
    ctx = Context(system, precision=precision)
    dt = torch.complex64 if precision == "f32" else torch.complex128
    u = torch.from_numpy(np.ascontiguousarray(psi0)).to("cuda", dt)
    if kick is not None:
        ctx.kick(u, kick)
    ctx.update_potential(u)
    out = torch.empty((nsteps + 1, system.n[2], system.n[1], system.n[0]), dtype=torch.float64, device="cuda")
    out[0] = ctx.grid_array(1)
    t = t0
    for i in range(nsteps):
        ctx.step(u, t, system.dt)
        t += system.dt
        out[i + 1] = ctx.grid_array(1)
    ctx.check()
    ctx.close()
    return out


def train(ctx, trajectories, epochs=3, batch=8, lr=1e-3, seed=0):
    """Train the context's network on several trajectories; returns the mean loss per epoch."""
    losses = []
    for ep in range(epochs):
        tot, n = 0.0, 0
        for i, tr in enumerate(trajectories):
            l = ctx.nn_train(tr, epochs=1, batch=batch, lr=lr, seed=seed * 1000 + ep * 100 + i)
            tot += float(l[0]) * (tr.shape[0] - 4)
            n += tr.shape[0] - 4
        losses.append(tot / max(n, 1))
    return np.array(losses)


def misfits(ctx, vseq, mode):
    """Relative misfit ||V(t+dt) - V~|| / ||V(t+dt)|| of a predictor along a recorded trajectory
    (mode 0 linear, 1 cubic, 2 network)."""
    import torch
    out = []
    vp = torch.empty_like(vseq[0])
    for t in range(3, vseq.shape[0] - 1):
        hist = torch.stack([vseq[t], vseq[t - 1], vseq[t - 2], vseq[t - 3]]).contiguous()
        ctx.nn_predict(hist, vp, mode=mode)
        out.append(((vseq[t + 1] - vp).norm() / vseq[t + 1].norm()).item())
    return np.array(out)


def run(system, psi0, nsteps, precision, mode, threshold=1e-5, params=None, t0=0.0):
    """Propagate with a predictor mode; returns J(t), steps/s (host-synchronised every step), the
    per-step misfit and the number of fallbacks."""
    import torch
    from . import tdks as T
    ctx = T.Context(system, precision=precision)
    dt = torch.complex64 if precision == "f32" else torch.complex128
    u = torch.from_numpy(np.ascontiguousarray(psi0)).to("cuda", dt)
    ctx.update_potential(u)
    if mode != T.PRED_PC:
        ctx.nn_init(0)
        if params is not None:
            ctx.nn_params(params)
        ctx.set_predictor(mode, threshold)
    J, res = [], []
    torch.cuda.synchronize()
    tic = time.perf_counter()
    t = t0
    o = None
    for _ in range(nsteps):
        ctx.step(u, t, system.dt)
        t += system.dt
        o = ctx.read_step_observables()
        J.append(o["J"])
        res.append(o["residual"])
    torch.cuda.synchronize()
    sps = nsteps / (time.perf_counter() - tic)
    ctx.check()
    fb = o["fallbacks"] if o else 0.0
    ctx.close()
    return dict(J=np.array(J), steps_per_s=sps, residual=np.array(res), fallbacks=fb)
