"""Ground state on the GPU (tdks_ground_state) against the oracle's dense self-consistent solution:
the occupied subspace (overlap with the oracle's states), the density, the band energy, and
stationarity of the result under the GPU's own time steps; the orbital energies (Ritz values and
vectors, tdks_orbital_energies) and the density of states (tdks_dos)."""
import numpy as np
import pytest

from oracle import tdks_oracle as O
from paper_1804_01404_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _systems():
    a = W.tiny(periodic=True, n=(6, 6, 6), natom=1, nk=1, norb=2)
    b = W.tiny(periodic=True, n=(6, 7, 5), natom=2, nk=2, norb=3)
    c = W.tiny(periodic=False, n=(7, 6, 8), natom=2, norb=2)
    for s in (a, b, c):
        s.field = W.Field("none")
    return {"periodic-1k": a, "periodic-2k": b, "isolated": c}


SYSTEMS = _systems()


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_ground_state_matches_oracle(name):
    from paper_1804_01404_gb300.tdks import Context
    s = SYSTEMS[name]
    psi_ref, eig_ref, v_ref, _ = O.ground_state(s, tol=1e-11)
    ctx = Context(s, precision="f64")
    u = torch.from_numpy(W.initial_orbitals(s, 7)).cuda()
    its, resid, eband = ctx.ground_state(u, max_iter=20000, tol=1e-9)
    ctx.check()
    assert resid < 1e-9 and its < 20000, (its, resid)
    got = u.cpu().numpy()
    for k in range(s.nk):          # same occupied subspace: the overlap matrix is unitary
        Ov = (got[k].reshape(s.norb, -1).conj() @ psi_ref[k].reshape(s.norb, -1).T) * s.dV
        assert np.max(np.abs(Ov.conj().T @ Ov - np.eye(s.norb))) < 1e-7
    rho = ctx.grid_array(2).cpu().numpy()
    rho_ref = O.density(s, psi_ref)
    assert np.max(np.abs(rho - rho_ref)) < 1e-7 * rho_ref.max()
    assert np.max(np.abs(ctx.grid_array(1).cpu().numpy() - v_ref)) < 1e-7 * np.max(np.abs(v_ref))
    eb_ref = float(np.sum(2.0 * np.asarray(s.kw)[:, None] * eig_ref))
    assert abs(eband - eb_ref) < 1e-7 * abs(eb_ref)
    # stationary under the GPU's own predictor-corrector steps
    t = 0.0
    for _ in range(10):
        ctx.step(u, t, s.dt)
        t += s.dt
    assert np.max(np.abs(ctx.grid_array(2).cpu().numpy() - rho)) < 1e-7 * rho.max()
    ctx.close()


def test_ground_state_argument_checks():
    from paper_1804_01404_gb300.tdks import Context, TdksError
    s = SYSTEMS["periodic-1k"]
    ctx = Context(s, precision="f64")
    u = torch.from_numpy(W.initial_orbitals(s, 1)).cuda()
    with pytest.raises(TdksError):
        ctx.ground_state(u, mix=1.5)
    with pytest.raises(TdksError):
        ctx.ground_state(torch.zeros_like(u))        # linearly dependent (zero) orbitals
    ctx.close()


def test_excited_pairs_after_a_pulse():
    """From the GPU ground state, a pulse excites electron-hole pairs: tdks_excited_pairs against the
    oracle's count on the same orbitals, zero before the pulse, positive after it."""
    from paper_1804_01404_gb300.tdks import Context, FIELD_PULSE
    s = SYSTEMS["periodic-2k"]
    ctx = Context(s, precision="f64")
    u = torch.from_numpy(W.initial_orbitals(s, 7)).cuda()
    ctx.ground_state(u, max_iter=20000, tol=1e-9)
    u_gs = u.clone()
    assert abs(ctx.excited_pairs(u, u_gs)) < 1e-12
    ctx.set_field(FIELD_PULSE, (0.0, 0.0, 0.2), 0.8, 3.0, 0.0)
    t = 0.0
    for _ in range(200):
        ctx.step(u, t, s.dt)
        t += s.dt
    ctx.check()
    n = ctx.excited_pairs(u, u_gs)
    ref = O.excited_pairs(s, u.cpu().numpy(), u_gs.cpu().numpy())
    assert abs(n - ref) < 1e-10 * abs(ref) and ref > 1e-8, (n, ref)
    ctx.close()


@pytest.mark.parametrize("name", ["periodic-2k", "isolated"])
def test_orbital_energies_and_dos_of_the_ground_state(name):
    """tdks_orbital_energies of the GPU ground state: the Ritz values equal the oracle's occupied
    eigenvalues, the rotated orbitals are eigenvectors of the GPU's own H (H u = e u), and tdks_dos
    of those energies equals the oracle's DOS."""
    from paper_1804_01404_gb300 import tdks as T
    s = SYSTEMS[name]
    _, eig_ref, _, _ = O.ground_state(s, tol=1e-11)
    ctx = T.Context(s, precision="f64")
    u = torch.from_numpy(W.initial_orbitals(s, 7)).cuda()
    ctx.ground_state(u, max_iter=20000, tol=1e-9)
    eps = ctx.orbital_energies(u, rotate=True)
    assert np.max(np.abs(eps - eig_ref)) < 1e-7 * np.max(np.abs(eig_ref))
    hu = torch.empty_like(u)
    ctx.hpsi(u, hu)
    ctx.check()
    for k in range(s.nk):
        for n in range(s.norb):
            r = (hu[k, n] - eps[k, n] * u[k, n]).abs().max().item()
            assert r < 1e-6 * u[k, n].abs().max().item(), (k, n, r)
    E = np.linspace(eps.min() - 0.5, eps.max() + 0.5, 777)
    d = T.dos(eps, s.kw, E, 0.03)
    assert np.max(np.abs(d - O.dos(eps, s.kw, E, 0.03))) < 1e-12 * np.max(d)
    ctx.close()


@pytest.mark.parametrize("precision,tol", [("f64", 1e-10), ("f32", 2e-5)])
def test_ritz_values_of_random_orbitals(precision, tol):
    """Ritz values of non-orthonormal random orbitals under V_loc + V_Hxc and a nonzero A', against
    the oracle's generalised eigenproblem; without rotation u is left unchanged."""
    from paper_1804_01404_gb300.tdks import Context
    s = W.tiny(periodic=True, n=(6, 7, 8), natom=2, nk=2, norb=3)
    psi = W.initial_orbitals(s, 3)
    psi = psi + 0.3 * np.roll(psi, 1, axis=1) * (1 + 0.5j)            # not orthonormal
    Ap = np.array([0.05, -0.02, 0.04])
    ctx = Context(s, precision=precision)
    u = torch.from_numpy(psi).to("cuda", torch.complex128 if precision == "f64" else torch.complex64)
    ctx.update_potential(u)
    before = u.clone()
    eps = ctx.orbital_energies(u, Ap=Ap)
    assert torch.equal(u, before)
    ctx.check()
    got_psi = u.cpu().numpy().astype(np.complex128)
    V = O.local_potential(s) + O.hxc(s, O.density(s, got_psi))
    ref, _ = O.orbital_energies(s, O.projector_tables(s), V, got_psi, Ap)
    assert np.max(np.abs(eps - ref)) < tol * np.max(np.abs(ref))
    ctx.close()


def test_ground_state_of_the_small_periodic_cell_converges():
    """The 16^3 cell with two pseudo-atoms and 8 orbitals (the small periodic workload): the
    Chebyshev-filtered iteration reaches a residual below 1e-8 in under 500 iterations, and the result
    is checked with the oracle's own operator at the density of the returned orbitals: they are
    eigenvectors of H[rho(u)] (|H u - e u| small), and their energies are the lowest eigenvalues of that
    operator (sparse Lanczos on the oracle's hpsi)."""
    spla = pytest.importorskip("scipy.sparse.linalg")
    from paper_1804_01404_gb300.tdks import Context
    s = W.small_periodic()
    s.field = W.Field("none")
    ctx = Context(s, precision="f64")
    u = torch.from_numpy(W.initial_orbitals(s, 2)).cuda()
    its, resid, eband = ctx.ground_state(u, max_iter=500, tol=1e-8)
    ctx.check()
    assert resid < 1e-8 and its < 500, (its, resid)
    psi = u.cpu().numpy()
    tabs = O.projector_tables(s)
    V = O.local_potential(s) + O.hxc(s, O.density(s, psi))
    q = np.asarray(s.kpts[0])
    eps, _ = O.orbital_energies(s, tabs, V, psi, np.zeros(3))
    for n in range(s.norb):
        hu = O.hpsi(s, tabs, V, q, psi[0, n:n + 1])[0]
        e = float(np.real(np.vdot(psi[0, n], hu) * s.dV))
        r = np.sqrt(np.sum(np.abs(hu - e * psi[0, n]) ** 2) * s.dV)
        assert r < 1e-6, (n, r)
    shape = (s.n[2], s.n[1], s.n[0])
    op = spla.LinearOperator((s.npts, s.npts), dtype=np.complex128,
                             matvec=lambda x: O.hpsi(s, tabs, V, q, x.reshape((1,) + shape))[0].ravel())
    low = np.sort(spla.eigsh(op, k=s.norb + 2, which="SA", tol=1e-12)[0])
    assert np.max(np.abs(np.sort(eps[0]) - low[:s.norb])) < 1e-7 * np.max(np.abs(low)), (eps, low)
    assert abs(eband - 2.0 * np.sum(low[:s.norb])) < 1e-7 * abs(eband)
    ctx.close()
