"""The buffer schemes of the shared-memory cell kernels' Taylor launches (tdks_cell_variant):
0 = two orbital copies, 1 = one copy swept in place plane by plane, 2 = scheme 0 compiled for the
periodic 20^3 and 16^3 grids (column segments unrolled over their planes), 3 = scheme 1 compiled for
those grids (FP32, two points per thread).

Each scheme is checked against the oracle's 4th-order Taylor step (Eq. taylor) and predictor-corrector
steps, on periodic and isolated grids, in FP64 and FP32, including the smallest allowed z extent
(4 planes, where every periodic z-neighbour of the sweep's last planes is an already replaced
plane's saved input) and batched multiscale cells.  The arithmetic per grid point and per projection
is the same in both schemes, so one Taylor step agrees between them (up to rounding in the potential,
whose density each context forms on its own)."""
import numpy as np
import pytest

from oracle import tdks_oracle as O
from paper_1804_01404_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(np.asarray(b).ravel()), 1e-300))


def _dev(psi, precision):
    return torch.from_numpy(np.ascontiguousarray(psi)).to(
        "cuda", torch.complex128 if precision == "f64" else torch.complex64)


def _systems():
    a = W.tiny(periodic=True, n=(6, 7, 5), natom=2, nk=2, norb=3)
    b = W.tiny(periodic=False, n=(7, 9, 11), natom=2, norb=2)
    c = W.tiny(periodic=True, n=(5, 6, 4), natom=1, nk=2, norb=2)      # nz = 4
    c.h = (0.6, 0.55, 0.7)
    d = W.diamond_crystal(nkdiv=1, norb=4)
    d.kpts = np.array([[0.11, -0.23, 0.37], [-0.3, 0.05, 0.2]])
    d.kw = np.array([0.5, 0.5])
    e = W.tiny(periodic=False, n=(9, 8, 4), natom=1, norb=2)            # isolated, nz = 4
    return {"tiny-periodic": a, "isolated-ragged": b, "periodic-nz4": c, "diamond-2k": d,
            "isolated-nz4": e}


SYSTEMS = _systems()


@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("f32", 2e-5)])
@pytest.mark.parametrize("name", list(SYSTEMS))
def test_taylor_step_both_schemes(name, precision, tol):
    from paper_1804_01404_gb300.tdks import Context
    s = SYSTEMS[name]
    psi = W.initial_orbitals(s, 3)
    Ap = np.array([0.0, 0.01, -0.02]) if s.periodic else np.zeros(3)
    tabs = O.projector_tables(s)
    V = O.local_potential(s) + O.hxc(s, O.density(s, psi))
    out = []
    for scheme in (0, 1):
        ctx = Context(s, precision=precision)
        ctx.cell_variant(scheme)
        assert ctx.cell_variant()[0] == scheme
        u = _dev(psi, precision)
        ctx.update_potential(u)
        ctx.taylor_step(u, 0.02, Ap)
        ctx.check()
        got = u.cpu().numpy()
        out.append(got)
        for k in range(s.nk):
            ref = O.taylor4(s, tabs, V, np.asarray(s.kpts[k]) + Ap, psi[k], 0.02)
            assert _rel(got[k].astype(np.complex128), ref) < tol, (scheme, k)
        ctx.close()
    assert _rel(out[1].astype(np.complex128), out[0].astype(np.complex128)) < (1e-14 if precision == "f64" else 1e-6)


@pytest.mark.parametrize("at_start", [False, True])
@pytest.mark.parametrize("name", ["tiny-periodic", "periodic-nz4", "isolated-ragged"])
def test_pc_steps_in_place_scheme(name, at_start):
    """Five predictor-corrector steps (FP64) with the in-place sweep: orbitals, J(t) and d(t) against
    the oracle, with the observables from the end-of-step pass or from the first stage."""
    from paper_1804_01404_gb300.tdks import Context
    s = SYSTEMS[name]
    psi0 = W.initial_orbitals(s, 5)
    if not s.periodic:
        psi0 = O.apply_kick(s, psi0, (0.0, 0.0, 0.05))
    n = 5
    ref, _, hist = O.run(s, psi0, n)
    ctx = Context(s, precision="f64", obs_at_start=at_start)
    ctx.cell_variant(1)
    u = _dev(psi0, "f64")
    ctx.update_potential(u)
    J, d = [], []
    t = 0.0
    for _ in range(n):
        ctx.step(u, t, s.dt)
        t += s.dt
        o = ctx.read_step_observables()
        J.append(o["J"])
        d.append(o["dipole"])
    ctx.check()
    J, d = np.array(J), np.array(d)
    assert _rel(u.cpu().numpy(), ref) < 1e-11
    dref = hist["d"]
    if at_start:       # step n reports the state it started from: the oracle's record of step n-1
        d, dref = d[1:], dref[:-1]
    assert np.max(np.abs(d - dref)) <= 1e-10 * max(np.max(np.abs(dref)), 1e-30)
    if s.periodic:
        Jref = hist["J"]
        if at_start:
            J, Jref = J[1:], Jref[:-1]
        assert np.max(np.abs(J - Jref)) < 1e-10 * np.max(np.abs(Jref))


@pytest.mark.parametrize("precision,tol", [("f64", 1e-11), ("f32", 1e-4)])
def test_multiscale_in_place_scheme(precision, tol):
    """Three cells with their own A' on a short Maxwell grid: two coupled steps with each scheme
    agree (the density atomics may sum in another order), and the in-place cells match the oracle's
    single-cell steps."""
    from paper_1804_01404_gb300.tdks import Context
    s = W.tiny(periodic=True, n=(6, 7, 8), natom=1, nk=2, norb=2)
    s.field = W.Field("none")
    ncell, m0, nX, dX = 3, 2, 8, 40.0
    X = np.arange(nX)
    A_now = 0.3 * np.exp(-((X - 2.5) / 1.5) ** 2)
    A_prev = 0.3 * np.exp(-((X - 2.4) / 1.5) ** 2)
    psis = np.stack([W.initial_orbitals(s, 30 + c) for c in range(ncell)])
    res = []
    for scheme in (0, 1):
        ctx = Context(s, precision=precision, ncell=ncell)
        ctx.cell_variant(scheme)
        u = _dev(psis, precision)
        ctx.update_potential(u)
        ctx.ms_init(dX, m0, A_now, A_prev)
        for i in range(2):
            ctx.ms_step(u, i * s.dt, s.dt)
        A, I = ctx.ms_read()
        ctx.check()
        res.append((u.cpu().numpy().astype(np.complex128), A, I))
        ctx.close()
    assert _rel(res[1][0], res[0][0]) < tol
    assert np.max(np.abs(res[1][1] - res[0][1])) <= tol * np.max(np.abs(res[0][1]))
    assert np.max(np.abs(res[1][2] - res[0][2])) <= tol * max(np.max(np.abs(res[0][2])), 1e-30)
    # against the oracle's coupled step
    tabs = O.projector_tables(s)
    Vloc = O.local_potential(s)
    cells = [(p, O.hxc(s, O.density(s, p))) for p in psis]
    An, Ap, I = A_now.copy(), A_prev.copy(), np.zeros(nX)
    for i in range(2):
        cells, An_next, Ap, I = O.multiscale_step(s, tabs, Vloc, cells, An, Ap, I, m0, dX, i * s.dt, s.dt)
        An = An_next
    for c in range(ncell):
        assert _rel(res[1][0][c], cells[c][0]) < tol, c
    assert np.max(np.abs(res[1][1] - An)) <= tol * np.max(np.abs(An))


def test_scheme_selection_and_errors():
    from paper_1804_01404_gb300.tdks import Context, TdksError
    s = SYSTEMS["diamond-2k"]                       # periodic 20^3: all four schemes apply in FP32
    ctx = Context(s, precision="f32")
    v, ms = ctx.cell_variant()
    assert v in (0, 1, 2, 3) and min(ms) > 0       # all timed at init; the fastest is kept
    assert ms[v] == min(ms)
    with pytest.raises(TdksError):
        ctx.cell_variant(4)
    ctx.close()
    c64 = Context(s, precision="f64")               # FP64: no scheme 3 (nor 2: two copies do not fit)
    assert c64.cell_variant()[1][3] == -1.0
    with pytest.raises(TdksError):
        c64.cell_variant(3)
    c64.close()
    t = SYSTEMS["tiny-periodic"]                    # 6 x 7 x 5: no built-in geometry
    ctx = Context(t, precision="f64")
    v, ms = ctx.cell_variant()
    assert v in (0, 1) and ms[2] == -1.0 and ms[3] == -1.0
    with pytest.raises(TdksError) as ei:
        ctx.cell_variant(2)
    assert "built-in" in str(ei.value)
    ctx.close()
    big = W.isolated_cluster(n=22, natom=4, norb=2, radius=3.8)      # 22 x 22 = 484 columns
    ctx = Context(big, precision="f32")
    v, ms = ctx.cell_variant()
    assert v == 0 and ms == [-1.0, -1.0, -1.0, -1.0]
    with pytest.raises(TdksError) as ei:
        ctx.cell_variant(1)
    assert "in-place" in str(ei.value)
    ctx.close()


GEOM_SYSTEMS = {"diamond-20^3": SYSTEMS["diamond-2k"], "periodic-16^3": W.small_periodic()}


@pytest.mark.parametrize("name,precision,tol", [("diamond-20^3", "f32", 2e-5), ("periodic-16^3", "f32", 2e-5),
                                                ("periodic-16^3", "f64", 1e-12)])
def test_taylor_step_built_in_geometry(name, precision, tol):
    """Schemes 2 and 3 (FP32) on the built-in grids against the oracle's Taylor step, and against
    scheme 0, whose arithmetic they repeat point by point.  (Two FP64 copies of a 20^3 orbital do not
    fit in shared memory: scheme 2 is refused there.)"""
    from paper_1804_01404_gb300.tdks import Context, TdksError
    s = GEOM_SYSTEMS[name]
    if name == "diamond-20^3":
        c64 = Context(s, precision="f64")
        assert c64.cell_variant()[1][2] == -1.0
        with pytest.raises(TdksError):
            c64.cell_variant(2)
        c64.close()
    psi = W.initial_orbitals(s, 4)
    Ap = np.array([0.02, -0.01, 0.015])
    tabs = O.projector_tables(s)
    V = O.local_potential(s) + O.hxc(s, O.density(s, psi))
    out = []
    schemes = (0, 2, 3) if precision == "f32" else (0, 2)
    for scheme in schemes:
        ctx = Context(s, precision=precision)
        ctx.cell_variant(scheme)
        assert ctx.cell_variant()[0] == scheme
        u = _dev(psi, precision)
        ctx.update_potential(u)
        ctx.taylor_step(u, 0.02, Ap)
        ctx.check()
        got = u.cpu().numpy()
        out.append(got)
        for k in range(s.nk):
            ref = O.taylor4(s, tabs, V, np.asarray(s.kpts[k]) + Ap, psi[k], 0.02)
            assert _rel(got[k].astype(np.complex128), ref) < tol, (scheme, k)
        ctx.close()
    for o in out[1:]:
        assert _rel(o.astype(np.complex128), out[0].astype(np.complex128)) < (1e-14 if precision == "f64" else 1e-6)


@pytest.mark.parametrize("precision,tol_u,tol_o,scheme", [("f64", 1e-11, 1e-10, 2), ("f32", 2e-5, 1e-4, 2),
                                                          ("f32", 2e-5, 1e-4, 3)])
@pytest.mark.parametrize("at_start", [False, True])
def test_pc_steps_built_in_geometry(at_start, precision, tol_u, tol_o, scheme):
    """Five predictor-corrector steps of the small periodic cell with scheme 2: orbitals, J(t) and
    d(t) against the oracle, with the observables from the end-of-step pass or from the first stage
    (FP32: two points per thread in the stages and in the final pass)."""
    from paper_1804_01404_gb300.tdks import Context
    s = GEOM_SYSTEMS["periodic-16^3"]
    psi0 = W.initial_orbitals(s, 5)
    n = 5
    ref, _, hist = O.run(s, psi0, n)
    ctx = Context(s, precision=precision, obs_at_start=at_start)
    ctx.cell_variant(scheme)
    u = _dev(psi0, precision)
    ctx.update_potential(u)
    J, d = [], []
    t = 0.0
    for _ in range(n):
        ctx.step(u, t, s.dt)
        t += s.dt
        o = ctx.read_step_observables()
        J.append(o["J"])
        d.append(o["dipole"])
    ctx.check()
    J, d = np.array(J), np.array(d)
    assert _rel(u.cpu().numpy().astype(np.complex128), ref) < tol_u
    Jref, dref = hist["J"], hist["d"]
    if at_start:       # step n reports the state it started from: the oracle's record of step n-1
        J, Jref, d, dref = J[1:], Jref[:-1], d[1:], dref[:-1]
    assert np.max(np.abs(d - dref)) <= tol_o * max(np.max(np.abs(dref)), 1e-30)
    assert np.max(np.abs(J - Jref)) < tol_o * np.max(np.abs(Jref))
