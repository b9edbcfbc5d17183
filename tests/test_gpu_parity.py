"""GPU parity: libtdks (through the C ABI) against the FP64 CPU oracle on the same seeded inputs.

Tolerances: the FP64 path must agree with the oracle to 1e-10 relative (L2 over orbitals, max-norm
over observable histories); in practice single operations agree to ~1e-13.  The FP32 path stores
and stencils orbitals in FP32 (unit roundoff 6e-8), so one H application or Taylor step agrees to
~1e-6 relative; 2e-5 is used.  Observables of the FP32 path after many steps: 1e-4 of max|X|.
"""
import numpy as np
import pytest

from oracle import tdks_oracle as O
from paper_1804_01404_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _ctx(s, precision="f64", **kw):
    from paper_1804_01404_gb300.tdks import Context
    return Context(s, precision=precision, **kw)


def _dev(psi, precision):
    dt = torch.complex128 if precision == "f64" else torch.complex64
    return torch.from_numpy(np.ascontiguousarray(psi)).to("cuda", dt)


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(np.asarray(b).ravel()), 1e-300))


def _systems():
    a = W.tiny(periodic=True, n=(6, 7, 5), natom=2, nk=2, norb=3)
    b = W.tiny(periodic=False, n=(7, 9, 11), natom=2, norb=2)
    c = W.small_periodic()
    d = W.diamond_crystal(nkdiv=1, norb=4)
    d.kpts = np.array([[0.11, -0.23, 0.37], [-0.3, 0.05, 0.2]])
    d.kw = np.array([0.5, 0.5])
    e = W.isolated_cluster(n=22, natom=6, norb=4, radius=3.8, seed=3)
    e.atoms = [W.Atom(at.R, at.Z) for at in e.atoms]
    f = W.tiny(periodic=True, n=(4, 5, 9), natom=1, norb=1)   # smallest allowed axis (4)
    f.h = (0.8, 0.7, 0.5)
    # odd x extent (the Hermitian rebuild of the Hartree solve mirrors kx = 1..4 to 8..5) and radix
    # 3 and 7 lines in the FFT of one periodic cell
    g = W.tiny(periodic=True, n=(9, 6, 7), natom=1, norb=2)
    return {"tiny-periodic": a, "tiny-isolated-ragged": b, "small-periodic": c,
            "diamond-2k": d, "cluster-22": e, "min-axis": f, "odd-periodic": g}


SYSTEMS = _systems()


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_local_potential(name):
    s = SYSTEMS[name]
    ctx = _ctx(s)
    got = ctx.grid_array(0).cpu().numpy()
    ref = O.local_potential(s)
    assert np.max(np.abs(got - ref)) < 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_hxc_potential(name):
    s = SYSTEMS[name]
    psi = W.initial_orbitals(s, 1)
    ctx = _ctx(s)
    ctx.update_potential(_dev(psi, "f64"))
    got = ctx.grid_array(1).cpu().numpy()
    ref = O.hxc(s, O.density(s, psi))
    assert np.max(np.abs(got - ref)) < 1e-11 * np.max(np.abs(ref))
    assert np.max(np.abs(ctx.grid_array(2).cpu().numpy() - O.density(s, psi))) < 1e-13 * O.density(s, psi).max()


def _oracle_full_V(s, psi):
    return O.local_potential(s) + O.hxc(s, O.density(s, psi))


@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("f32", 2e-5)])
@pytest.mark.parametrize("name", list(SYSTEMS))
def test_hpsi(name, precision, tol):
    s = SYSTEMS[name]
    psi = W.initial_orbitals(s, 2)
    rng = np.random.default_rng(5)
    u = psi + 0.3 * (rng.standard_normal(psi.shape) + 1j * rng.standard_normal(psi.shape)) * np.abs(psi).max()
    Ap = np.array([0.013, -0.021, 0.034]) if s.periodic else np.zeros(3)
    ctx = _ctx(s, precision)
    ctx.update_potential(_dev(psi, precision))
    ud = _dev(u, precision)
    hu = torch.empty_like(ud)
    ctx.hpsi(ud, hu, Ap)
    got = hu.cpu().numpy().astype(np.complex128)
    tabs = O.projector_tables(s)
    V = _oracle_full_V(s, psi)
    for k in range(s.nk):
        ref = O.hpsi(s, tabs, V, np.asarray(s.kpts[k]) + Ap, u[k])
        assert _rel(got[k], ref) < tol, (k, _rel(got[k], ref))


@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("f32", 2e-5)])
@pytest.mark.parametrize("name", list(SYSTEMS))
def test_taylor_step(name, precision, tol):
    s = SYSTEMS[name]
    psi = W.initial_orbitals(s, 3)
    Ap = np.array([0.0, 0.01, -0.02]) if s.periodic else np.zeros(3)
    ctx = _ctx(s, precision)
    ud = _dev(psi, precision)
    ctx.update_potential(ud)
    ctx.taylor_step(ud, 0.02, Ap)
    got = ud.cpu().numpy().astype(np.complex128)
    tabs = O.projector_tables(s)
    V = _oracle_full_V(s, psi)
    for k in range(s.nk):
        ref = O.taylor4(s, tabs, V, np.asarray(s.kpts[k]) + Ap, psi[k], 0.02)
        assert _rel(got[k], ref) < tol


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_observables(name):
    s = SYSTEMS[name]
    psi = W.initial_orbitals(s, 4)
    psi[:, 0] *= 1.01                                # norms differ from 1
    Ap = np.array([0.02, 0.0, -0.01]) if s.periodic else np.zeros(3)
    ctx = _ctx(s)
    ud = _dev(psi, "f64")
    rho0_psi = W.initial_orbitals(s, 9)
    ctx.update_potential(_dev(rho0_psi, "f64"))       # sets rho0
    rho = torch.full((s.n[2], s.n[1], s.n[0]), float("nan"), dtype=torch.float64, device="cuda")
    o = ctx.observables(ud, Ap, rho=rho)
    rho_ref = O.density(s, psi)
    assert np.max(np.abs(rho.cpu().numpy() - rho_ref)) < 1e-13 * np.max(rho_ref)
    tabs = O.projector_tables(s)
    nrm = O.norms(s, psi)
    assert abs(o["norm_min"] - nrm.min()) < 1e-13 and abs(o["norm_max"] - nrm.max()) < 1e-13
    d_ref = O.dipole(s, O.density(s, psi), O.density(s, rho0_psi))
    assert np.max(np.abs(o["dipole"] - d_ref)) < 1e-11 * max(1.0, np.max(np.abs(d_ref)))
    eb = O.band_energy(s, tabs, O.local_potential(s), psi, Ap)
    assert abs(o["e_band"] - eb) < 1e-11 * abs(eb)
    if s.periodic:
        J = O.current(s, tabs, psi, Ap)
        assert np.max(np.abs(o["J"] - J)) < 1e-11 * np.max(np.abs(J))


def _run_gpu(s, psi0, nsteps, precision, pc=True, hartree=True, xc=True):
    ctx = _ctx(s, precision, pc=pc, hartree=hartree, xc=xc)
    ud = _dev(psi0, precision)
    ctx.update_potential(ud)
    J, d = [], []
    t = 0.0
    for _ in range(nsteps):
        ctx.step(ud, t, s.dt)
        t += s.dt
        o = ctx.read_step_observables()
        J.append(o["J"])
        d.append(o["dipole"])
    return ud.cpu().numpy().astype(np.complex128), np.array(J), np.array(d), ctx


@pytest.fixture(scope="module")
def config1_oracle():
    s = W.small_periodic(nsteps=100)
    psi0 = W.initial_orbitals(s, 0)
    psi, vhxc, hist = O.run(s, psi0, s.nsteps)
    return s, psi0, psi, vhxc, hist


def test_periodic_cell_100_steps_f64(config1_oracle):
    """16^3 periodic cell, 2 atoms, 8 orbitals, A'-step kick, PC + Hartree + LDA, 100 steps:
    orbitals, V_Hxc, J(t) and d(t) within 1e-10 of the oracle."""
    s, psi0, psi, vhxc, hist = config1_oracle
    got, J, d, ctx = _run_gpu(s, psi0, s.nsteps, "f64")
    assert _rel(got, psi) < 1e-10
    assert np.max(np.abs(ctx.grid_array(1).cpu().numpy() - vhxc)) < 1e-10 * np.max(np.abs(vhxc))
    assert np.max(np.abs(J - hist["J"])) < 1e-10 * np.max(np.abs(hist["J"]))
    assert np.max(np.abs(d - hist["d"])) < 1e-10 * np.max(np.abs(hist["d"]))


def test_periodic_cell_100_steps_f32(config1_oracle):
    """FP32 orbitals with FP64 reductions and Poisson: J(t), d(t) within 1e-4 of max|X64|."""
    s, psi0, psi, vhxc, hist = config1_oracle
    got, J, d, _ = _run_gpu(s, psi0, s.nsteps, "f32")
    assert np.max(np.abs(J - hist["J"])) < 1e-4 * np.max(np.abs(hist["J"]))
    assert np.max(np.abs(d - hist["d"])) < 1e-4 * np.max(np.abs(hist["d"]))
    assert _rel(got, psi) < 1e-4


@pytest.mark.parametrize("pc,hartree,xc", [(True, True, True), (False, True, True), (True, False, False)])
def test_isolated_ragged_steps(pc, hartree, xc):
    """Isolated 7x9x11 box, kick, 5 steps, each switch of the step: orbitals and dipole match."""
    s = W.tiny(periodic=False, n=(7, 9, 11), natom=2, norb=2)
    psi0 = O.apply_kick(s, W.initial_orbitals(s, 5), (0.0, 0.0, 0.05))
    ref, _, hist = O.run(s, psi0, 5, pc=pc, hartree_on=hartree, xc_on=xc)
    got, J, d, _ = _run_gpu(s, psi0, 5, "f64", pc=pc, hartree=hartree, xc=xc)
    assert _rel(got, ref) < 1e-11
    assert np.max(np.abs(d - hist["d"])) < 1e-10 * np.max(np.abs(hist["d"]))


def test_kick_parity():
    s = W.isolated_cluster(n=22, natom=4, norb=3, radius=3.8)
    psi0 = W.initial_orbitals(s, 7)
    ctx = _ctx(s)
    ud = _dev(psi0, "f64")
    ctx.kick(ud, (0.01, -0.02, 0.03))
    assert _rel(ud.cpu().numpy(), O.apply_kick(s, psi0, (0.01, -0.02, 0.03))) < 1e-14


def test_diamond_full_size_first_steps():
    """Diamond cell at the bench configuration (20^3 grid, 16 orbitals x 64 k-points), the first three
    PC steps with the pulse on, in both precisions, against the oracle (all orbitals): these tie the
    FP64 GPU run that the bench's long-window FP32 errors are measured against to the oracle."""
    s = W.diamond_crystal()
    psi0 = W.initial_orbitals(s, 0)
    t0 = 200.0                                        # inside the pulse, A' != 0
    nsteps = 3
    tabs = O.projector_tables(s)
    Vloc = O.local_potential(s)
    vhxc = O.hxc(s, O.density(s, psi0))
    ref, t, Jref = psi0, t0, []
    for _ in range(nsteps):
        ref, vhxc, rho = O.pc_step(s, tabs, Vloc, ref, vhxc, t, s.dt)
        t += s.dt
        Jref.append(O.current(s, tabs, ref, O.field_Aprime(s.field, t)))
    Jref = np.array(Jref)
    for precision, tol, jtol in (("f64", 1e-11, 1e-11), ("f32", 2e-5, 1e-4)):
        ctx = _ctx(s, precision)
        ud = _dev(psi0, precision)
        ctx.update_potential(ud)
        J, t = [], t0
        for _ in range(nsteps):
            ctx.step(ud, t, s.dt)
            t += s.dt
            J.append(ctx.read_step_observables()["J"])
        assert _rel(ud.cpu().numpy().astype(np.complex128), ref) < tol
        assert np.max(np.abs(np.array(J) - Jref)) < jtol * np.max(np.abs(Jref))
        ctx.close()


def test_norm_monitor_reports_nonfinite():
    """A NaN planted in one orbital on the host is reported by the norm monitor as
    TDKS_ENONFINITE; the context stays usable afterwards."""
    from paper_1804_01404_gb300.tdks import TdksError
    s = W.small_periodic()
    psi = W.initial_orbitals(s, 0)
    ctx = _ctx(s)
    ctx.update_potential(_dev(psi, "f64"))
    bad = psi.copy()
    bad[0, 3, 5, 6, 7] = np.nan
    with pytest.raises(TdksError) as ei:
        ctx.observables(_dev(bad, "f64"))
    assert ei.value.status == 5
    o = ctx.observables(_dev(psi, "f64"))
    assert abs(o["norm_max"] - 1.0) < 1e-12


def test_orbital_shard():
    """A context that holds one shard of the orbitals (options.norb_offset / norb_total): H u and a
    Taylor step of its orbitals equal the oracle's for the same orbitals with V_loc (no density is
    formed on a shard), and the calls that form the potential from the orbitals are refused."""
    from paper_1804_01404_gb300.tdks import Context, TdksError
    s = W.small_periodic()
    psi = W.initial_orbitals(s, 6)[:, 4:]                 # orbitals 4..7 of 8
    s.norb = 4
    Ap = np.array([0.01, -0.02, 0.005])
    ctx = Context(s, precision="f64", norb_offset=4, norb_total=8)
    ud = _dev(psi, "f64")
    hu = torch.empty_like(ud)
    ctx.hpsi(ud, hu, Ap)
    tabs, Vloc = O.projector_tables(s), O.local_potential(s)
    q = np.asarray(s.kpts[0]) + Ap
    assert _rel(hu.cpu().numpy()[0], O.hpsi(s, tabs, Vloc, q, psi[0])) < 1e-12
    ctx.taylor_step(ud, 0.02, Ap)
    assert _rel(ud.cpu().numpy()[0], O.taylor4(s, tabs, Vloc, q, psi[0], 0.02)) < 1e-12
    for call in (lambda: ctx.update_potential(ud), lambda: ctx.step(ud, 0.0, 0.02)):
        with pytest.raises(TdksError) as e:
            call()
        assert e.value.status == 6 and "shard" in str(e.value)
    ctx.close()
