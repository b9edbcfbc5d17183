"""Observables of the input state (options.obs_at_start = 1) against the end-of-step form.

With obs_at_start the first Taylor stage of step n forms J(t_n) from the derivative sums it computes
anyway, and the step leaves the dipole of rho(t_n); the default form leaves J(t_{n+1}) and the dipole
of rho(t_{n+1}) from an extra pass.  The propagation itself is the same, so after step n the first
form must equal what the second left after step n-1, and step 0 must give the oracle's current of the
initial orbitals.  Covered: plain predictor-corrector, single Taylor steps (pc = 0, so the corrector
kernel forms them), and cubic-extrapolation predicted steps."""
import numpy as np
import pytest

from oracle import tdks_oracle as O
from paper_1804_01404_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _system():
    s = W.diamond_crystal()
    s.kpts = s.kpts[:2]
    s.kw = np.full(2, 0.5)
    s.norb = 4
    return s


def _run(s, psi0, precision, at_start, nsteps, t0, pc=True, extrap=False):
    from paper_1804_01404_gb300 import tdks as T
    ctx = T.Context(s, precision=precision, pc=pc, obs_at_start=at_start)
    u = torch.from_numpy(psi0).to("cuda", torch.complex128 if precision == "f64" else torch.complex64)
    ctx.update_potential(u)
    if extrap:
        ctx.set_predictor(T.PRED_EXTRAP, 1.0)   # always accept, so every step after 4 is predicted
    J, d = [], []
    t = t0
    for _ in range(nsteps):
        ctx.step(u, t, s.dt)
        t += s.dt
        o = ctx.read_step_observables()
        J.append(o["J"])
        d.append(o["dipole"])
    ctx.check()
    return np.array(J), np.array(d), u.cpu().numpy()


@pytest.mark.parametrize("precision,tol", [("f64", 1e-11), ("f32", 2e-5)])
@pytest.mark.parametrize("pc,extrap", [(True, False), (False, False), (True, True)])
def test_obs_at_start_is_previous_end(precision, tol, pc, extrap):
    s = _system()
    psi0 = W.initial_orbitals(s, 3)
    t0 = 200.0
    n = 8
    Je, de, ue = _run(s, psi0, precision, False, n, t0, pc, extrap)
    Js, ds, us = _run(s, psi0, precision, True, n, t0, pc, extrap)
    # the observables do not change the propagation (up to the order of the density atomics)
    assert np.linalg.norm(ue - us) < tol * np.linalg.norm(ue)
    scale = np.max(np.abs(Je))
    assert np.max(np.abs(Js[1:] - Je[:-1])) < tol * scale
    assert np.max(np.abs(ds[1:] - de[:-1])) <= tol * max(np.max(np.abs(de)), 1e-30)
    J0 = O.current(s, O.projector_tables(s), psi0, O.field_Aprime(s.field, t0))
    assert np.max(np.abs(Js[0] - J0)) < tol * scale
    assert np.max(np.abs(ds[0])) < 1e-12          # rho(t0) is the reference density rho0
