"""GPU parity of the large-grid (TMA tile) path against the FP64 oracle.

An isolated 40 x 30 x 28 grid does not fit the shared-memory cell kernels in either precision,
so every call goes through the tile kernels; the tiles are ragged in x (40 = 32 + 8) and y
(30 = 3 x 8 + 6).  Tolerances as in test_gpu_parity.py.
"""
import numpy as np
import pytest

from oracle import tdks_oracle as O
from paper_1804_01404_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _system():
    s = W.isolated_cluster(n=24, natom=5, norb=3, radius=3.5, seed=4)
    s.n = (40, 30, 28)
    s.h = (0.45, 0.5, 0.55)
    return s


S = _system()


def _ctx(s, precision, **kw):
    from paper_1804_01404_gb300.tdks import Context
    return Context(s, precision=precision, **kw)


def _dev(psi, precision):
    return torch.from_numpy(np.ascontiguousarray(psi)).to(
        "cuda", torch.complex128 if precision == "f64" else torch.complex64)


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


def test_uses_tiled_path():
    from paper_1804_01404_gb300.tdks import Context
    for prec in ("f32", "f64"):
        ctx = Context(S, precision=prec)
        assert ctx.query()["npts"] == 40 * 30 * 28


@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("f32", 2e-5)])
def test_tiled_hpsi(precision, tol):
    psi = W.initial_orbitals(S, 1)
    ctx = _ctx(S, precision)
    ctx.update_potential(_dev(psi, precision))
    ud = _dev(psi, precision)
    hu = torch.empty_like(ud)
    ctx.hpsi(ud, hu)
    ctx.check()
    tabs = O.projector_tables(S)
    V = O.local_potential(S) + O.hxc(S, O.density(S, psi))
    ref = O.hpsi(S, tabs, V, np.zeros(3), psi[0])
    assert _rel(hu.cpu().numpy()[0].astype(np.complex128), ref) < tol


@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("f32", 2e-5)])
def test_tiled_taylor(precision, tol):
    psi = W.initial_orbitals(S, 2)
    ctx = _ctx(S, precision)
    ud = _dev(psi, precision)
    ctx.update_potential(ud)
    ctx.taylor_step(ud, 0.02)
    ctx.check()
    tabs = O.projector_tables(S)
    V = O.local_potential(S) + O.hxc(S, O.density(S, psi))
    ref = O.taylor4(S, tabs, V, np.zeros(3), psi[0], 0.02)
    assert _rel(ud.cpu().numpy()[0].astype(np.complex128), ref) < tol


@pytest.mark.parametrize("precision,tol,dtol", [("f64", 1e-11, 1e-10), ("f32", 1e-4, 1e-4)])
def test_tiled_pc_steps(precision, tol, dtol):
    psi0 = O.apply_kick(S, W.initial_orbitals(S, 3), (0.0, 0.0, 0.01))
    ref, _, hist = O.run(S, psi0, 3)
    ctx = _ctx(S, precision)
    ud = _dev(psi0, precision)
    ctx.update_potential(ud)
    d = []
    t = 0.0
    for _ in range(3):
        ctx.step(ud, t, S.dt)
        t += S.dt
        d.append(ctx.read_step_observables()["dipole"])
    ctx.check()
    assert _rel(ud.cpu().numpy().astype(np.complex128), ref) < tol
    assert np.max(np.abs(np.array(d) - hist["d"])) < dtol * np.max(np.abs(hist["d"]))


def test_tiled_observables():
    psi = W.initial_orbitals(S, 4)
    psi[0, 1] *= 1.02
    ctx = _ctx(S, "f64")
    ctx.update_potential(_dev(W.initial_orbitals(S, 5), "f64"))
    o = ctx.observables(_dev(psi, "f64"))
    nrm = O.norms(S, psi)
    assert abs(o["norm_max"] - nrm.max()) < 1e-12 and abs(o["norm_min"] - nrm.min()) < 1e-12
    eb = O.band_energy(S, O.projector_tables(S), O.local_potential(S), psi, np.zeros(3))
    assert abs(o["e_band"] - eb) < 1e-11 * abs(eb)


@pytest.mark.parametrize("precision,variant", [("f32", 0), ("f32", 1), ("f32", 2), ("f32", 3), ("f32", 4), ("f32", 5),
                                               ("f32", 6), ("f64", 0), ("f64", 1)])
def test_tiled_variants_hpsi_and_taylor(precision, variant):
    """Every stencil variant (one point per thread for 3 CTAs per SM, or for 2 with L2 prefetch; FP32
    2 x 2 and 2 x 1 blocks) against the oracle, on the anisotropic ragged grid (h differs per axis, so
    the per-axis coefficient ratios of the blocked variants are exercised)."""
    psi = W.initial_orbitals(S, 6)
    ctx = _ctx(S, precision)
    v, ms = ctx.tile_variant(variant)
    nvar = 7 if precision == "f32" else 2
    assert v == [variant, variant] and all(m > 0 for row in ms for m in row[:nvar])
    tol = 2e-5 if precision == "f32" else 1e-12
    ctx.update_potential(_dev(psi, precision))
    ud = _dev(psi, precision)
    hu = torch.empty_like(ud)
    ctx.hpsi(ud, hu)
    tabs = O.projector_tables(S)
    V = O.local_potential(S) + O.hxc(S, O.density(S, psi))
    for b in range(psi.shape[0]):
        ref = O.hpsi(S, tabs, V, np.zeros(3), psi[b])
        assert _rel(hu.cpu().numpy()[b].astype(np.complex128), ref) < tol
    ctx.taylor_step(ud, 0.02)
    ctx.check()
    for b in range(psi.shape[0]):
        ref = O.taylor4(S, tabs, V, np.zeros(3), psi[b], 0.02)
        assert _rel(ud.cpu().numpy()[b].astype(np.complex128), ref) < tol


@pytest.mark.parametrize("schedule", [0, 1, 2])
def test_projection_schedules(schedule):
    """The three schedules of the FP32 tensor-core projection (2, 4, 8 warps per CTA over the sphere
    points) give H u and a Taylor step within the FP32 bound of the oracle; all three are timed at
    init and the fastest is kept; FP64 contexts (CUDA-core projection) refuse the call."""
    from paper_1804_01404_gb300.tdks import TdksError
    psi = W.initial_orbitals(S, 7)
    ctx = _ctx(S, "f32")
    v0, ms = ctx.project_variant()
    assert min(ms) > 0 and ms[v0] == min(ms)
    assert ctx.project_variant(schedule)[0] == schedule
    ctx.update_potential(_dev(psi, "f32"))
    ud = _dev(psi, "f32")
    hu = torch.empty_like(ud)
    ctx.hpsi(ud, hu)
    tabs = O.projector_tables(S)
    V = O.local_potential(S) + O.hxc(S, O.density(S, psi))
    for b in range(psi.shape[0]):
        ref = O.hpsi(S, tabs, V, np.zeros(3), psi[b])
        assert _rel(hu.cpu().numpy()[b].astype(np.complex128), ref) < 2e-5
    ctx.taylor_step(ud, 0.02)
    ctx.check()
    for b in range(psi.shape[0]):
        ref = O.taylor4(S, tabs, V, np.zeros(3), psi[b], 0.02)
        assert _rel(ud.cpu().numpy()[b].astype(np.complex128), ref) < 2e-5
    with pytest.raises(TdksError):
        ctx.project_variant(3)
    with pytest.raises(TdksError):
        _ctx(S, "f64").project_variant()


def test_tile_variant_rules():
    from paper_1804_01404_gb300.tdks import TdksError
    c64 = _ctx(S, "f64")
    assert all(v in (0, 1) for v in c64.tile_variant()[0])
    with pytest.raises(TdksError):
        c64.tile_variant(2)
    with pytest.raises(TdksError):
        c64.tile_variant(3)
    with pytest.raises(TdksError):
        _ctx(S, "f32").tile_variant(7)


def test_staged_variants_need_nx_divisible_by_4():
    """Variants 5 and 6 (potential rows as a tensor map of floats) apply only when nx % 4 == 0: on an
    nx = 38 grid the tuner skips them and forcing one is refused; the others still run there."""
    from paper_1804_01404_gb300.tdks import TdksError
    s = W.isolated_cluster(n=24, natom=3, norb=2, radius=3.5, seed=5)
    s.n = (38, 34, 30)                                    # too large for one orbital in shared memory
    ctx = _ctx(s, "f32")
    v, ms = ctx.tile_variant()
    assert ms[0][5] == -1.0 and ms[0][6] == -1.0 and ms[1][5] == -1.0 and v[0] not in (5, 6)
    assert all(m > 0 for m in ms[0][:5])
    with pytest.raises(TdksError):
        ctx.tile_variant(5)
    psi = W.initial_orbitals(s, 2)
    ud = _dev(psi, "f32")
    ctx.update_potential(ud)
    ctx.tile_variant(3)
    hu = torch.empty_like(ud)
    ctx.hpsi(ud, hu)
    ctx.check()
    tabs = O.projector_tables(s)
    V = O.local_potential(s) + O.hxc(s, O.density(s, psi))
    ref = O.hpsi(s, tabs, V, np.zeros(3), psi[0])
    assert _rel(hu.cpu().numpy()[0].astype(np.complex128), ref) < 2e-5


def test_wait_timeout_is_reported_and_context_recovers():
    """The failure path of the tile kernels without a GPU fault: the copy producer stops after two
    planes, the stencil warps wait for a third that never arrives, give up after a short poll limit
    and report TDKS_ETIMEOUT through tdks_check; the same context then computes H u correctly."""
    from paper_1804_01404_gb300.tdks import TdksError
    psi = W.initial_orbitals(S, 7)
    for precision, tol in (("f32", 2e-5), ("f64", 1e-12)):
        ctx = _ctx(S, precision)
        ud = _dev(psi, precision)
        ctx.update_potential(ud)
        hu = torch.empty_like(ud)
        ctx.set_wait_test(wait_limit=2000, stop_after=2)
        ctx.hpsi(ud, hu)
        with pytest.raises(TdksError) as err:
            ctx.check()
        assert err.value.status == 4                        # TDKS_ETIMEOUT
        ctx.check()                                         # the error word was cleared
        ctx.set_wait_test()
        ctx.hpsi(ud, hu)
        ctx.check()
        tabs = O.projector_tables(S)
        V = O.local_potential(S) + O.hxc(S, O.density(S, psi))
        ref = O.hpsi(S, tabs, V, np.zeros(3), psi[0])
        assert _rel(hu.cpu().numpy()[0].astype(np.complex128), ref) < tol
