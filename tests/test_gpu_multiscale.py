"""Batches of microscopic cells and the coupled Maxwell + TDKS step (Sec. 5) against the oracle."""
import numpy as np
import pytest

from oracle import tdks_oracle as O
from paper_1804_01404_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _sys():
    s = W.tiny(periodic=True, n=(6, 7, 8), natom=1, nk=2, norb=2)
    s.field = W.Field("none")
    return s


@pytest.mark.parametrize("precision,tol", [("f64", 1e-11), ("f32", 1e-4)])
def test_batched_cells_equal_independent_cells(precision, tol):
    """Three cells with different orbitals and a common step field: each cell evolves exactly as the
    same cell alone (separate densities and potentials per cell)."""
    from paper_1804_01404_gb300.tdks import Context
    s = _sys()
    s.field = W.Field("step", (0.0, 0.0, 0.01))
    psis = [W.initial_orbitals(s, 10 + c) for c in range(3)]
    ctx = Context(s, precision=precision, ncell=3)
    dt_ = torch.complex128 if precision == "f64" else torch.complex64
    u = torch.from_numpy(np.stack(psis)).to("cuda", dt_)
    ctx.update_potential(u)
    t = 0.0
    for _ in range(3):
        ctx.step(u, t, s.dt)
        t += s.dt
    ctx.check()
    got = u.cpu().numpy().astype(np.complex128)
    for c in range(3):
        ref, _, _ = O.run(s, psis[c], 3, record=False)
        assert np.linalg.norm(got[c] - ref) < tol * np.linalg.norm(ref), c


@pytest.mark.parametrize("precision,tol", [("f64", 1e-10), ("f32", 1e-4)])
def test_multiscale_steps_against_oracle(precision, tol):
    """8-point Maxwell grid, two cells at X = 3, 4, an incident A profile: A(X) and the cell currents
    after 4 coupled steps match the oracle."""
    from paper_1804_01404_gb300.tdks import Context
    s = _sys()
    tabs = O.projector_tables(s)
    Vloc = O.local_potential(s)
    nX, m0, dX, dt = 8, 3, 40.0, s.dt
    X = np.arange(nX)
    A_now = 0.3 * np.exp(-((X - 2.0) / 1.5) ** 2)
    A_prev = 0.3 * np.exp(-((X - 1.9) / 1.5) ** 2)
    psis = [W.initial_orbitals(s, 20 + c) for c in range(2)]
    cells = [(p, O.hxc(s, O.density(s, p))) for p in psis]
    An, Ap, I = A_now.copy(), A_prev.copy(), np.zeros(nX)
    t = 0.0
    for _ in range(4):
        cells, An_next, Ap, I = O.multiscale_step(s, tabs, Vloc, cells, An, Ap, I, m0, dX, t, dt)
        An = An_next
        t += dt
    ctx = Context(s, precision=precision, ncell=2)
    dt_ = torch.complex128 if precision == "f64" else torch.complex64
    u = torch.from_numpy(np.stack(psis)).to("cuda", dt_)
    ctx.update_potential(u)
    ctx.ms_init(dX, m0, A_now, A_prev)
    for _ in range(4):
        ctx.ms_step(u, 0.0, dt)
    A_got, I_got = ctx.ms_read()
    ctx.check()
    assert np.max(np.abs(A_got - An)) < tol * np.max(np.abs(An))
    assert np.max(np.abs(I_got - I)) < tol * np.max(np.abs(I))
    got = u.cpu().numpy().astype(np.complex128)
    for c in range(2):
        assert np.linalg.norm(got[c] - cells[c][0]) < tol * np.linalg.norm(cells[c][0])


@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_multiscale_step_graphs_equal_stream_launches(precision, tol):
    """From the second step on tdks_ms_step replays a CUDA graph (one per rotation of the three A
    levels); seven steps with the graphs (each graph built once and replayed) and seven with the
    kernels launched one by one give the same A(X), currents and orbitals (up to the order of the
    density atomics), and count the same kernel launches.  Then the oracle's steps."""
    from paper_1804_01404_gb300.tdks import Context
    s = _sys()
    nX, m0, dX, dt = 9, 3, 40.0, s.dt
    X = np.arange(nX)
    A_now = 0.3 * np.exp(-((X - 2.0) / 1.5) ** 2)
    A_prev = 0.3 * np.exp(-((X - 1.9) / 1.5) ** 2)
    psis = [W.initial_orbitals(s, 40 + c) for c in range(3)]
    dt_ = torch.complex128 if precision == "f64" else torch.complex64
    res = []
    for graphs in (True, False):
        ctx = Context(s, precision=precision, ncell=3)
        ctx.set_step_graph(graphs)
        u = torch.from_numpy(np.stack(psis)).to("cuda", dt_)
        ctx.update_potential(u)
        ctx.ms_init(dX, m0, A_now, A_prev)
        ctx.stats(reset=True)
        for _ in range(7):
            ctx.ms_step(u, 0.0, dt)
        launches = ctx.stats(reset=True)["launches"]
        A, I = ctx.ms_read()
        ctx.check()
        res.append((u.cpu().numpy().astype(np.complex128), A, I, launches))
        ctx.close()
    (ug, Ag, Ig, lg), (us, As, Is, ls) = res
    assert lg == ls
    assert np.linalg.norm(ug - us) < tol * np.linalg.norm(us)
    assert np.max(np.abs(Ag - As)) <= tol * np.max(np.abs(As))
    assert np.max(np.abs(Ig - Is)) <= tol * max(np.max(np.abs(Is)), 1e-30)
    tabs = O.projector_tables(s)
    Vloc = O.local_potential(s)
    cells = [(p, O.hxc(s, O.density(s, p))) for p in psis]
    An, Ap, I = A_now.copy(), A_prev.copy(), np.zeros(nX)
    t = 0.0
    for _ in range(7):
        cells, An_next, Ap, I = O.multiscale_step(s, tabs, Vloc, cells, An, Ap, I, m0, dX, t, dt)
        An = An_next
        t += dt
    otol = 1e-10 if precision == "f64" else 1e-4
    assert np.max(np.abs(Ag - An)) < otol * np.max(np.abs(An))
    for c in range(3):
        assert np.linalg.norm(ug[c] - cells[c][0]) < otol * np.linalg.norm(cells[c][0])
