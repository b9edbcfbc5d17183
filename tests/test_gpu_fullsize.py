"""Parity at the full workload sizes, on outputs the oracle can compute one at a time.

* Isolated cluster: 96^3 grid (h = 0.4), 128 atoms, all 256 orbitals on the GPU, FP32 orbitals, in
  the launch configuration the bench times (tile kernels, tuned variant).  The Hartree + exchange
  potential (Hockney, 192^3 FFTs) is compared on the whole grid; H u and one Taylor step on sampled
  orbitals.
* Multiscale: 256 microscopic cells (16^3, 16 orbitals x 8 k each) on a 1D Maxwell grid, one coupled
  step; the Maxwell field on the whole grid, and the orbitals and current of sampled cells, each
  against the oracle's single-cell step with that cell's vector potential.
"""
import numpy as np
import pytest

from oracle import tdks_oracle as O
from paper_1804_01404_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
torch = pytest.importorskip("torch")


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


def test_cluster_full_size():
    from paper_1804_01404_gb300.tdks import Context
    s = W.isolated_cluster()
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    shape = (s.nk, s.norb, s.n[2], s.n[1], s.n[0])
    u = torch.randn(shape, dtype=torch.complex64, device="cuda", generator=g)
    u *= 1.0 / np.sqrt(s.npts * s.dV)
    ctx = Context(s, precision="f32")
    ctx.update_potential(u)
    V_gpu = (ctx.grid_array(0) + ctx.grid_array(1)).cpu().numpy()
    host = u.cpu().numpy()
    rho = np.zeros(s.n[::-1])
    for b0 in range(0, s.norb, 16):                  # the density is additive over orbitals
        rho += O.density(s, host[:, b0:b0 + 16].astype(np.complex128))
    Vloc = O.local_potential(s)
    V = Vloc + O.hxc(s, rho)
    assert np.max(np.abs(V_gpu - V)) < 1e-6 * np.max(np.abs(V))
    tabs = O.projector_tables(s)
    hu = torch.empty_like(u)
    ctx.hpsi(u, hu)
    hu_h = hu.cpu().numpy()
    sample = (0, 137, s.norb - 1)
    for b in sample:
        ref = O.hpsi(s, tabs, V, np.zeros(3), host[0, b].astype(np.complex128))
        assert _rel(hu_h[0, b].astype(np.complex128), ref) < 2e-5, b
    ctx.taylor_step(u, s.dt)
    ctx.check()
    out = u.cpu().numpy()
    for b in sample:
        ref = O.taylor4(s, tabs, V, np.zeros(3), host[0, b].astype(np.complex128), s.dt)
        assert _rel(out[0, b].astype(np.complex128), ref) < 2e-5, b


def test_multiscale_256_cells_one_step():
    from paper_1804_01404_gb300.tdks import Context
    s = W.multiscale_cell()
    ncell, m0, dX, dt = 256, 4, 250.0, s.dt
    nX = m0 + ncell + 4
    X = np.arange(nX)
    A_now = 0.3 * np.sin(2 * np.pi * X / 64.0)
    A_prev = 0.3 * np.sin(2 * np.pi * (X + 0.5) / 64.0)
    psi = W.initial_orbitals(s, 3)
    ctx = Context(s, precision="f32", ncell=ncell)
    u = torch.from_numpy(np.ascontiguousarray(np.broadcast_to(psi.astype(np.complex64), (ncell,) + psi.shape))).cuda()
    ctx.update_potential(u)
    ctx.ms_init(dX, m0, A_now, A_prev)
    ctx.ms_step(u, 0.0, dt)
    A_gpu, I_gpu = ctx.ms_read()
    ctx.check()
    c = O.C_LIGHT
    k = c * dt / dX
    A_next = O.mur_boundary(O.maxwell_step(A_now, A_prev, np.zeros(nX), k, dt, c), A_now, k)
    assert np.max(np.abs(A_gpu - A_next)) < 1e-12 * np.max(np.abs(A_next))
    tabs = O.projector_tables(s)
    Vloc = O.local_potential(s)
    vhxc = O.hxc(s, O.density(s, psi))
    got = u.cpu().numpy()
    for j in (0, 137, ncell - 1):
        Xj = m0 + j
        Amid = np.array([0.0, 0.0, 0.5 * (A_now[Xj] + A_next[Xj]) / c])
        ref, _, _ = O.pc_step(s, tabs, Vloc, psi, vhxc, 0.0, dt, Ap=Amid)
        assert _rel(got[j].astype(np.complex128), ref) < 1e-4, j
        Iref = O.current(s, tabs, ref, np.array([0.0, 0.0, A_next[Xj] / c]))[2]
        assert abs(I_gpu[Xj] - Iref) < 1e-4 * abs(Iref) + 1e-12, (j, I_gpu[Xj], Iref)
