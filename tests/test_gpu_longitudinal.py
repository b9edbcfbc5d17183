"""Longitudinal geometry on the GPU (tdks_set_longitudinal): the induced vector potential of a thin
film, d^2 A'_ind/dt^2 = 4 pi J, advanced on the device every step, against the oracle's
longitudinal run -- the plasma oscillation of a free electron gas and a cell with atoms under a
pulse -- plus the argument checks and a checkpoint / restart in the middle of a run."""
import math

import numpy as np
import pytest

from oracle import tdks_oracle as O
from paper_1804_01404_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _electron_gas(n=6, L=7.0):
    s = W.tiny(periodic=True, n=(n, n, n), natom=0, nk=1, norb=1)
    s.h = (L / n,) * 3
    s.kpts = np.zeros((1, 3))
    s.kw = np.ones(1)
    psi = np.full((1, 1, n, n, n), 1.0 / math.sqrt(O.cell_volume(s)), complex)
    return s, psi


def _gpu_run(s, psi0, nsteps, t0, precision="f64"):
    from paper_1804_01404_gb300.tdks import Context
    ctx = Context(s, precision=precision)
    u = torch.from_numpy(psi0).to("cuda", torch.complex128 if precision == "f64" else torch.complex64)
    ctx.update_potential(u)
    ctx.set_longitudinal(1, u, t0)
    J, A = [], []
    t = t0
    for _ in range(nsteps):
        ctx.step(u, t, s.dt)
        t += s.dt
        J.append(ctx.read_step_observables()["J"])
        A.append(ctx.longitudinal_A())
    ctx.check()
    return u, np.array(J), np.array(A), ctx


def test_plasma_oscillation():
    s, psi = _electron_gas()
    A0, t0 = 1e-3, 1e-12
    s.field = W.Field("step", (0.0, 0.0, A0))
    wp = math.sqrt(4.0 * math.pi * 2.0 / O.cell_volume(s))
    n = int(round(1.5 * (2 * math.pi / wp) / s.dt))
    u, J, A, ctx = _gpu_run(s, psi, n, t0)
    _, hist = O.longitudinal_run(s, psi, n, t0=t0)
    assert np.max(np.abs(A - hist["A_ind"])) < 1e-10 * A0
    assert np.max(np.abs(J - hist["J"])) < 1e-10 * np.max(np.abs(hist["J"]))
    t = np.arange(1, n + 1) * s.dt
    assert np.max(np.abs(A0 + A[:, 2] - A0 * np.cos(wp * t))) < 0.01 * A0      # the plasma oscillation
    ctx.close()


@pytest.mark.parametrize("precision,tol", [("f64", 1e-10), ("f32", 1e-4)])
def test_longitudinal_cell_with_atoms(precision, tol):
    s = W.tiny(periodic=True, n=(6, 7, 8), natom=2, nk=2, norb=2)
    s.field = W.Field("pulse", (0.0, 0.0, 0.05), 0.5, 6.0, 0.0)
    psi0 = W.initial_orbitals(s, 3)
    n = 25
    u, J, A, ctx = _gpu_run(s, psi0, n, 0.5, precision)
    ref, hist = O.longitudinal_run(s, psi0, n, t0=0.5)
    got = u.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(got - ref) < tol * np.linalg.norm(ref)
    assert np.max(np.abs(J - hist["J"])) < tol * np.max(np.abs(hist["J"]))
    assert np.max(np.abs(A - hist["A_ind"])) < tol * np.max(np.abs(hist["A_ind"]))
    assert np.max(np.abs(hist["A_ind"])) > 1e-8                                   # the film responds
    ctx.close()


def test_longitudinal_argument_checks():
    from paper_1804_01404_gb300.tdks import Context, TdksError
    s = W.tiny(periodic=True, n=(6, 7, 8), natom=1, nk=1, norb=1)
    u = torch.from_numpy(W.initial_orbitals(s, 1)).cuda()
    ctx = Context(s, precision="f64", obs_at_start=True)
    with pytest.raises(TdksError) as e:
        ctx.set_longitudinal(1, u, 0.0)
    assert e.value.status == 6                       # TDKS_EUNSUPPORTED
    ctx.close()
    iso = W.tiny(periodic=False, n=(7, 8, 9), natom=1, norb=1)
    ctx = Context(iso, precision="f64")
    with pytest.raises(TdksError):
        ctx.set_longitudinal(1, torch.from_numpy(W.initial_orbitals(iso, 1)).cuda(), 0.0)
    ctx.close()


def test_longitudinal_restart():
    """A checkpoint after 4 steps restores A'_ind, its previous level and the current the next step
    reads: the restored context continues like the original."""
    from paper_1804_01404_gb300.tdks import Context
    s = W.tiny(periodic=True, n=(6, 7, 8), natom=2, nk=2, norb=2)
    s.field = W.Field("pulse", (0.0, 0.0, 0.05), 0.5, 6.0, 0.0)
    psi0 = W.initial_orbitals(s, 5)
    a = Context(s, precision="f64")
    u = torch.from_numpy(psi0).cuda()
    a.update_potential(u)
    a.set_longitudinal(1, u, 0.5)
    t = 0.5
    for _ in range(4):
        a.step(u, t, s.dt)
        t += s.dt
    state = a.get_state()
    mid = u.clone()
    t_mid = t
    for _ in range(4):
        a.step(u, t, s.dt)
        t += s.dt
    b = Context(s, precision="f64")
    b.set_state(state)
    t = t_mid
    for _ in range(4):
        b.step(mid, t, s.dt)
        t += s.dt
    assert (mid - u).abs().max().item() < 1e-12 * u.abs().max().item()
    assert np.max(np.abs(b.longitudinal_A() - a.longitudinal_A())) < 1e-12 * np.max(np.abs(a.longitudinal_A()))
    a.close()
    b.close()
