"""TB-mBJ exchange on the GPU (tdks_options.xc = 3, tdks_set_mbj) against the oracle.

The potential of a set of orbitals (c fixed and c from the density; periodic with several
k-points, a 16^3 cell with several orbital chunks, a ragged isolated box), predictor-corrector
steps in FP64 and FP32 (the predictor's own orbitals feed the predicted potential), predicted
steps with the extrapolated potential, the tiled path of large isolated grids, the ground state with
TB-mBJ, and the argument checks."""
import math

import numpy as np
import pytest

from oracle import tdks_oracle as O
from paper_1804_01404_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _systems():
    a = W.tiny(periodic=True, n=(6, 7, 8), natom=2, nk=2, norb=2)
    a.field = W.Field("pulse", (0.0, 0.0, 0.03), 0.4, 5.0, 0.0)
    b = W.small_periodic()
    c = W.tiny(periodic=False, n=(7, 9, 11), natom=2, norb=2)
    d = W.tiny(periodic=False, n=(8, 9, 10), natom=2, norb=2)    # even nx: the paired FP32 kinetic sums
    return {"periodic-2k": a, "periodic-16": b, "isolated-ragged": c, "isolated-even": d}


SYSTEMS = _systems()


def _dev(psi, precision="f64"):
    return torch.from_numpy(np.ascontiguousarray(psi)).to(
        "cuda", torch.complex128 if precision == "f64" else torch.complex64)


@pytest.mark.parametrize("name", list(SYSTEMS))
@pytest.mark.parametrize("cval", [None, 0.93])
def test_mbj_potential(name, cval):
    from paper_1804_01404_gb300.tdks import Context
    s = SYSTEMS[name]
    psi = W.initial_orbitals(s, 2)
    ctx = Context(s, precision="f64", xc=3, mbj_c=cval)
    ctx.update_potential(_dev(psi))
    got = ctx.grid_array(1).cpu().numpy()
    rho = O.density(s, psi)
    ref = O.hxc(s, rho, True, 3, psi, cval)
    assert np.max(np.abs(got - ref)) < 1e-10 * np.max(np.abs(ref))
    # the mBJ exchange is really there: it differs from the LDA exchange by far more than the tolerance
    assert np.max(np.abs(ref - O.hxc(s, rho, True, 2))) > 1e-2 * np.max(np.abs(ref))
    c_ref = cval if cval is not None else O.mbj_c(s, rho)
    assert abs(ctx.mbj_c() - c_ref) < 1e-12 * c_ref
    ctx.close()


@pytest.mark.parametrize("name", ["periodic-2k", "isolated-ragged", "isolated-even"])
@pytest.mark.parametrize("precision,tol", [("f64", 1e-10), ("f32", 1e-4)])
def test_mbj_pc_steps(name, precision, tol):
    from paper_1804_01404_gb300.tdks import Context
    s = SYSTEMS[name]
    psi0 = W.initial_orbitals(s, 3)
    if not s.periodic:
        psi0 = O.apply_kick(s, psi0, (0.0, 0.0, 0.05))
    n = 4
    ref, vref, _ = O.run(s, psi0, n, xc_on=3)
    ctx = Context(s, precision=precision, xc=3)
    u = _dev(psi0, precision)
    ctx.update_potential(u)
    t = 0.0
    for _ in range(n):
        ctx.step(u, t, s.dt)
        t += s.dt
    ctx.check()
    got = u.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(got - ref) < tol * np.linalg.norm(ref)
    assert np.max(np.abs(ctx.grid_array(1).cpu().numpy() - vref)) < 10 * tol * np.max(np.abs(vref))
    # the TB-mBJ run differs from the LDA one by far more than the tolerance
    ref2, _, _ = O.run(s, psi0, n, xc_on=2)
    assert np.linalg.norm(ref2 - ref) > 100 * tol * np.linalg.norm(ref)
    ctx.close()


def test_mbj_tiled_steps():
    """Large isolated grid (tile kernels): the predictor's orbitals come from the tiled Horner
    stages; two PC steps with c fixed against the oracle."""
    from paper_1804_01404_gb300.tdks import Context
    s = W.isolated_cluster(n=24, natom=5, norb=3, radius=3.5, seed=4)
    s.n = (40, 30, 28)
    s.h = (0.45, 0.5, 0.55)
    psi0 = O.apply_kick(s, W.initial_orbitals(s, 3), (0.0, 0.0, 0.01))
    ref, vref, _ = O.run(s, psi0, 2, xc_on=3, mbj_c=1.1)
    ctx = Context(s, precision="f64", xc=3, mbj_c=1.1)
    ctx.tile_variant()                               # raises unless the context uses the tile kernels
    u = _dev(psi0)
    ctx.update_potential(u)
    t = 0.0
    for _ in range(2):
        ctx.step(u, t, s.dt)
        t += s.dt
    ctx.check()
    got = u.cpu().numpy()
    assert np.linalg.norm(got - ref) < 1e-10 * np.linalg.norm(ref)
    assert np.max(np.abs(ctx.grid_array(1).cpu().numpy() - vref)) < 1e-9 * np.max(np.abs(vref))
    ctx.close()


def test_mbj_ground_state():
    """The self-consistent ground state with TB-mBJ exchange (c from the density at every
    iteration) against the oracle's dense SCF."""
    from paper_1804_01404_gb300.tdks import Context
    s = W.tiny(periodic=True, n=(6, 6, 6), natom=1, nk=1, norb=2)
    s.field = W.Field("none")
    psi_ref, eig_ref, v_ref, _ = O.ground_state(s, xc_on=3, tol=1e-11)
    ctx = Context(s, precision="f64", xc=3)
    u = _dev(W.initial_orbitals(s, 7))
    its, resid, eband = ctx.ground_state(u, max_iter=20000, tol=1e-9)
    ctx.check()
    assert resid < 1e-9 and its < 20000, (its, resid)
    rho_ref = O.density(s, psi_ref)
    assert np.max(np.abs(ctx.grid_array(2).cpu().numpy() - rho_ref)) < 1e-7 * rho_ref.max()
    assert np.max(np.abs(ctx.grid_array(1).cpu().numpy() - v_ref)) < 1e-7 * np.max(np.abs(v_ref))
    eb_ref = float(np.sum(2.0 * np.asarray(s.kw)[:, None] * eig_ref))
    assert abs(eband - eb_ref) < 1e-7 * abs(eb_ref)
    ctx.close()


def test_mbj_argument_checks():
    from paper_1804_01404_gb300.tdks import Context, TdksError
    s = SYSTEMS["periodic-2k"]
    ctx = Context(s, precision="f64", xc=2)
    with pytest.raises(TdksError) as e:
        ctx.set_mbj(1.0)
    assert e.value.status == 6                       # TDKS_EUNSUPPORTED
    with pytest.raises(TdksError):
        ctx.mbj_c()
    ctx.close()
    ctx = Context(s, precision="f64", xc=3)
    with pytest.raises(TdksError) as e:
        ctx.set_mbj(math.nan)
    assert e.value.status == 1                       # TDKS_EINVAL
    ctx.set_mbj(0.0)                                  # back to c from the density
    ctx.close()


def test_mbj_extrapolated_predictor_steps():
    """Predicted steps with TB-mBJ (cubic extrapolation of V_Hxc, every prediction accepted): the
    corrector's potential comes from the propagated orbitals' own kinetic energy density.  Against an
    oracle loop of the same scheme (plain PC while the history fills, then the predicted step)."""
    from oracle import nn_oracle as N
    from paper_1804_01404_gb300 import tdks as T
    s = SYSTEMS["periodic-2k"]
    psi0 = W.initial_orbitals(s, 5)
    n = 7
    tabs, Vloc = O.projector_tables(s), O.local_potential(s)
    psi = psi0.copy()
    v = O.hxc(s, O.density(s, psi), True, 3, psi)
    hist = [v]
    for i in range(n):
        t = i * s.dt
        if len(hist) >= 4:
            vt = N.cubic_extrapolation(hist[-1], hist[-2], hist[-3], hist[-4])
            Ap = O.field_Aprime(s.field, t + 0.5 * s.dt)
            psi = O.propagate_all(s, tabs, Vloc + 0.5 * (v + vt), psi, Ap, s.dt)
            v = O.hxc(s, O.density(s, psi), True, 3, psi)
        else:
            psi, v, _ = O.pc_step(s, tabs, Vloc, psi, v, t, s.dt, xc_on=3)
        hist.append(v)
    ctx = T.Context(s, precision="f64", xc=3)
    u = _dev(psi0)
    ctx.update_potential(u)
    ctx.set_predictor(T.PRED_EXTRAP, 1.0)
    t = 0.0
    for _ in range(n):
        ctx.step(u, t, s.dt)
        t += s.dt
    ctx.check()
    assert ctx.read_step_observables()["fallbacks"] == 0
    got = u.cpu().numpy()
    assert np.linalg.norm(got - psi) < 1e-10 * np.linalg.norm(psi)
    assert np.max(np.abs(ctx.grid_array(1).cpu().numpy() - v)) < 1e-9 * np.max(np.abs(v))
    ctx.close()


@pytest.mark.parametrize("precision,tol,ctol", [("f64", 1e-5, 1e-6), ("f32", 3e-2, 2e-3)])
def test_mbj_plane_wave_edge_case(precision, tol, ctol):
    """The degenerate case of the Becke-Roussel equation: one plane wave gives a uniform density and
    tau - |j|^2/(2 rho) = 0, so Q = 0 up to rounding and the root is x = 2; g = 0 gives c = alpha.
    The GPU potential against the closed form -alpha (1 - 2 e^-2)(pi e^2 rho/2)^(1/3) plus the PZ
    correlation.  Tolerances: the square roots of g and t_s lift the rounding of their vanishing
    arguments to ~1e-8 in FP64; FP32 orbitals leave ~1e-7 relative noise in rho and tau, lifted to
    ~1e-2 of the potential (the FP32 case checks that the degenerate root stays finite and near
    the closed form)."""
    from paper_1804_01404_gb300.tdks import Context
    s = W.tiny(periodic=True, n=(8, 9, 10), natom=0, nk=1, norb=1)
    s.h = (0.5, 0.45, 0.4)
    s.kpts = np.zeros((1, 3))
    s.kw = np.ones(1)
    x, y, z = O.coords(s)
    L = [s.n[a] * s.h[a] for a in range(3)]
    u = np.exp(1j * (2 * np.pi / L[0] * x[None, None, :] + 4 * np.pi / L[1] * y[None, :, None] + 0 * z[:, None, None]))
    psi = (u / math.sqrt(O.cell_volume(s)))[None, None]
    ctx = Context(s, precision=precision, hartree=False, xc=3)
    ctx.update_potential(_dev(psi, precision))
    got = ctx.grid_array(1).cpu().numpy()
    rho = O.density(s, psi)
    rs = rho.mean() / 2
    exact = 0.012 * (1 - 2 * math.exp(-2.0)) * (math.pi * math.e ** 2 * rs) ** (1 / 3) + O.lda_c(rho)[0]
    assert np.all(np.isfinite(got))
    assert np.max(np.abs(got - exact)) < tol * np.max(np.abs(exact))
    assert abs(ctx.mbj_c() - (-0.012)) < ctol
    ctx.close()
