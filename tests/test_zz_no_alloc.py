"""tdks_hxc_noalloc, the entry point for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc: host programs whose device memory is handed out by a pool they
do not own, and latency-critical loops that must never allocate.  For them the
library computes the Hartree + exchange potential of a density in a fixed device work area that
is part of the library image (at most 64^3 FFT points).

The test compares its output with the potential the regular context computes from the same
density (tdks_update_potential, which uses context-owned buffers), on two calls in a row, for a
periodic and an isolated grid, and checks that grids beyond the limit are refused.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1804_01404_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _fn():
    from paper_1804_01404_gb300 import tdks
    lib = tdks.load_library()
    f = lib.tdks_hxc_noalloc
    f.argtypes = [C.POINTER(tdks.Grid), C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p]
    f.restype = C.c_int
    return f, lib, tdks


def _grid(tdks, s):
    return tdks.Grid((C.c_int * 3)(*s.n), (C.c_double * 3)(*s.h), 1 if s.periodic else 0)


def _systems():
    iso = W.isolated_cluster(n=22, natom=4, norb=3, radius=3.8, seed=2)
    return [W.small_periodic(), iso]


@pytest.mark.parametrize("sys_index", [0, 1])
def test_noalloc_matches_context_potential(sys_index):
    f, lib, tdks = _fn()
    s = _systems()[sys_index]
    stream = torch.cuda.current_stream()
    g = _grid(tdks, s)
    for call, seed in enumerate((3, 8)):          # two calls in a row, different densities
        ctx = tdks.Context(s, precision="f64")
        u = torch.from_numpy(W.initial_orbitals(s, seed)).to("cuda")
        ctx.update_potential(u)
        rho = ctx.grid_array(2)
        ref = ctx.grid_array(1)
        out = torch.full_like(ref, float("nan"))
        st = f(C.byref(g), C.c_void_p(rho.data_ptr()), C.c_void_p(out.data_ptr()), 1, 1,
               C.c_void_p(stream.cuda_stream))
        assert st == 0, lib.tdks_last_error().decode()
        torch.cuda.synchronize()
        err = (out - ref).abs().max().item() / ref.abs().max().item()
        assert err < 1e-12, (call, err)
        ctx.close()


def test_noalloc_rejects_oversize_grid():
    f, lib, tdks = _fn()
    s = W.tiny(periodic=False, n=(40, 8, 8))        # isolated: FFT length 80 > 64
    g = _grid(tdks, s)
    buf = torch.zeros(8 * 8 * 40, dtype=torch.float64, device="cuda")
    st = f(C.byref(g), C.c_void_p(buf.data_ptr()), C.c_void_p(buf.data_ptr()), 1, 1, None)
    assert st == 6, st                              # TDKS_EUNSUPPORTED
    assert "64" in lib.tdks_last_error().decode()


@pytest.mark.parametrize("sys_index", [0, 1])
def test_noalloc_public_wrapper_matches_the_oracle(sys_index):
    """The same entry point through the package's Python wrapper (tdks.hxc_noalloc), two calls in a
    row on one pair of buffers, against the oracle's Hartree + exchange potential of the density
    (periodic: G-space Poisson; isolated: zero-padded convolution with the cell-averaged self term)."""
    from oracle import tdks_oracle as O
    from paper_1804_01404_gb300 import tdks
    s = _systems()[sys_index]
    out = torch.empty((s.n[2], s.n[1], s.n[0]), dtype=torch.float64, device="cuda")
    for seed in (4, 9):
        rho_np = O.density(s, W.initial_orbitals(s, seed))
        rho = torch.from_numpy(rho_np).to("cuda")
        out.fill_(float("nan"))
        tdks.hxc_noalloc(s, rho, out, hartree=True, xc=1)
        torch.cuda.synchronize()
        ref = O.hxc(s, rho_np, True, 1)
        err = np.max(np.abs(out.cpu().numpy() - ref)) / np.max(np.abs(ref))
        assert err < 1e-12, (seed, err)
