"""LDA with Perdew-Zunger correlation on the GPU (tdks_options.xc = 2) against the oracle.

The Hartree-exchange-correlation potential of a density on periodic and isolated grids (both
Hartree paths: the three-launch plane solve and the five line passes), the allocation-free entry
point with xc = 2, five predictor-corrector steps with correlation on, and the rejection of
xc values outside 0..3 (3 is TB-mBJ, tested on its own)."""
import ctypes as C

import numpy as np
import pytest

from oracle import tdks_oracle as O
from paper_1804_01404_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _systems():
    a = W.small_periodic()
    b = W.tiny(periodic=False, n=(7, 9, 11), natom=2, norb=2)
    c = W.isolated_cluster(n=22, natom=4, norb=3, radius=3.8, seed=2)
    return {"periodic-16": a, "isolated-ragged": b, "cluster-22": c}


SYSTEMS = _systems()


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_hxc_with_correlation(name):
    from paper_1804_01404_gb300.tdks import Context
    s = SYSTEMS[name]
    psi = W.initial_orbitals(s, 2)
    ctx = Context(s, precision="f64", xc=2)
    ctx.update_potential(torch.from_numpy(psi).cuda())
    got = ctx.grid_array(1).cpu().numpy()
    rho = O.density(s, psi)
    ref = O.hxc(s, rho, True, 2)
    assert np.max(np.abs(got - ref)) < 1e-11 * np.max(np.abs(ref))
    # the correlation part is really there: it differs from exchange only by more than the tolerance
    assert np.max(np.abs(ref - O.hxc(s, rho, True, 1))) > 1e-3 * np.max(np.abs(ref))
    ctx.close()


def test_noalloc_with_correlation():
    from paper_1804_01404_gb300 import tdks
    lib = tdks.load_library()
    f = lib.tdks_hxc_noalloc
    f.argtypes = [C.POINTER(tdks.Grid), C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p]
    f.restype = C.c_int
    s = SYSTEMS["periodic-16"]
    psi = W.initial_orbitals(s, 4)
    rho = torch.from_numpy(O.density(s, psi)).cuda()
    out = torch.full_like(rho, float("nan"))
    g = tdks.Grid((C.c_int * 3)(*s.n), (C.c_double * 3)(*s.h), 1)
    st = f(C.byref(g), C.c_void_p(rho.data_ptr()), C.c_void_p(out.data_ptr()), 1, 2, None)
    assert st == 0, lib.tdks_last_error().decode()
    torch.cuda.synchronize()
    ref = O.hxc(s, rho.cpu().numpy(), True, 2)
    assert np.max(np.abs(out.cpu().numpy() - ref)) < 1e-11 * np.max(np.abs(ref))
    st = f(C.byref(g), C.c_void_p(rho.data_ptr()), C.c_void_p(out.data_ptr()), 1, 3, None)
    assert st == 1                                  # TDKS_EINVAL


@pytest.mark.parametrize("name", ["periodic-16", "isolated-ragged"])
def test_pc_steps_with_correlation(name):
    from paper_1804_01404_gb300.tdks import Context
    s = SYSTEMS[name]
    psi0 = W.initial_orbitals(s, 3)
    if not s.periodic:
        psi0 = O.apply_kick(s, psi0, (0.0, 0.0, 0.05))
    n = 5
    ref, vref, hist = O.run(s, psi0, n, xc_on=2)
    ctx = Context(s, precision="f64", xc=2)
    u = torch.from_numpy(psi0).cuda()
    ctx.update_potential(u)
    d = []
    t = 0.0
    for _ in range(n):
        ctx.step(u, t, s.dt)
        t += s.dt
        d.append(ctx.read_step_observables()["dipole"])
    ctx.check()
    got = u.cpu().numpy()
    assert np.linalg.norm(got - ref) < 1e-10 * np.linalg.norm(ref)
    assert np.max(np.abs(ctx.grid_array(1).cpu().numpy() - vref)) < 1e-10 * np.max(np.abs(vref))
    assert np.max(np.abs(np.array(d) - hist["d"])) < 1e-10 * max(np.max(np.abs(hist["d"])), 1e-30)
    ctx.close()


def test_xc_option_range():
    from paper_1804_01404_gb300.tdks import Context, TdksError
    with pytest.raises(TdksError) as e:
        Context(SYSTEMS["periodic-16"], precision="f64", xc=4)
    assert "xc" in str(e.value)
