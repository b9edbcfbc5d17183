"""C-ABI checks that need no GPU: the library builds, loads and exports every declared symbol,
and host-side argument validation rejects bad input before any CUDA call."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1804_01404_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1804_01404_gb300 import build, tdks
    if not os.path.exists(tdks.LIB_PATH):
        build.build()
    return tdks.load_library()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "tdks.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tdks_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert "tdks_init" in names and "tdks_step" in names and len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert lib.tdks_abi_version() == 4


def _init(lib, s, **kw):
    from paper_1804_01404_gb300 import tdks as T
    g = T.Grid((C.c_int * 3)(*kw.get("n", s.n)), (C.c_double * 3)(*s.h), int(s.periodic))
    L = kw.get("L", [s.n[a] * s.h[a] for a in range(3)])
    cell = T.Cell((C.c_double * 3)(*L))
    atoms = (T.AtomC * max(1, len(s.atoms)))()
    for i, at in enumerate(s.atoms):
        atoms[i] = T.AtomC((C.c_double * 3)(*at.R), at.Z, at.sigma, kw.get("proj", 0))
    pr = T.ProjectorC(s.proj.E_s, s.proj.E_p, kw.get("r_cut", s.proj.r_cut), s.proj.width)
    kp = np.ascontiguousarray(np.asarray(s.kpts, np.float64).ravel())
    kwt = np.ascontiguousarray(np.asarray(kw.get("kw", s.kw), np.float64))
    opts = T.Options(kw.get("precision", 0), 1, kw.get("xc", 1), 1, kw.get("ncell", 1), kw.get("obs_at_start", 0),
                     kw.get("norb_offset", 0), kw.get("norb_total", 0))
    ctx = C.c_void_p()
    st = lib.tdks_init(C.byref(g), C.byref(cell), atoms, len(s.atoms), C.byref(pr), 1,
                       kp.ctypes.data_as(C.POINTER(C.c_double)), kwt.ctypes.data_as(C.POINTER(C.c_double)),
                       len(kwt), kw.get("norb", s.norb), C.byref(opts), None, C.byref(ctx))
    return st, lib.tdks_last_error().decode()


@pytest.mark.parametrize("case,expect", [
    (dict(n=(3, 6, 6)), "grid points"),
    (dict(norb=0), "norb"),
    (dict(kw=[0.5]), "weights"),
    (dict(L=[1.0, 1.0, 1.0]), "cell length"),
    (dict(precision=7), "precision"),
    (dict(r_cut=2.0), "half the periodic cell"),
    (dict(proj=5), "projector index"),
    (dict(ncell=-2), "ncell"),
    (dict(obs_at_start=3), "obs_at_start"),
    (dict(xc=4), "xc must be"),
    (dict(norb_offset=1), "norb_offset needs norb_total"),
    (dict(norb_offset=3, norb_total=4), "exceeds norb_total"),
    (dict(norb_total=-1), "must be >= 0"),
])
def test_host_validation(lib, case, expect):
    s = W.tiny(periodic=True, n=(6, 6, 6), natom=1)
    st, msg = _init(lib, s, **case)
    assert st == 1, (st, msg)          # TDKS_EINVAL, returned before any device call
    assert expect in msg


def test_mbj_needs_one_cell(lib):
    """xc = 3 (TB-mBJ) with a batch of cells is refused before any device call (EUNSUPPORTED)."""
    s = W.tiny(periodic=True, n=(6, 6, 6), natom=1)
    st, msg = _init(lib, s, xc=3, ncell=2)
    assert st == 6 and "TB-mBJ" in msg, (st, msg)


def test_dos_argument_checks(lib):
    """tdks_dos rejects a non-positive width and empty arrays before any device call."""
    d = np.zeros(3)
    p = d.ctypes.data_as(C.POINTER(C.c_double))
    assert lib.tdks_dos(p, 1, 3, p, p, 3, 0.0, p, None) == 1
    assert lib.tdks_dos(p, 0, 3, p, p, 3, 0.1, p, None) == 1
    assert lib.tdks_dos(None, 1, 3, p, p, 3, 0.1, p, None) == 1


def test_binding_declares_every_symbol(lib):
    """The Python binding gives argument types to every function the header declares."""
    from paper_1804_01404_gb300 import tdks as T
    src = open(T.__file__).read()
    missing = [n for n in declared_symbols() if f'"{n}"' not in src and f"lib.{n}" not in src]
    assert not missing, missing
    assert lib.tdks_hxc_noalloc(None, None, None, 1, 1, None) == 1         # EINVAL before any device call


def test_null_context_rejected(lib):
    assert lib.tdks_hpsi(None, None, None, (C.c_double * 3)()) == 1
    assert lib.tdks_step(None, None, 0.0, 0.02) == 1


def _check_options(lib, s, norb, **kw):
    from paper_1804_01404_gb300 import tdks as T
    g = T.Grid((C.c_int * 3)(*s.n), (C.c_double * 3)(*s.h), int(s.periodic))
    o = T.Options(kw.get("precision", 1), 1, 1, 1, 1, 0, kw.get("norb_offset", 0), kw.get("norb_total", 0))
    return lib.tdks_check_options(C.byref(g), 1, norb, C.byref(o)), lib.tdks_last_error().decode()


def test_orbital_range_offset(lib):
    """The orbital range of a shard (orbital parallelism: the orbitals of each k-point split over
    contexts) is validated on the host: offset + norb must stay within norb_total, an offset needs
    a total, and the whole set (norb_total = 0 or = norb) is the default."""
    from paper_1804_01404_gb300 import tdks as T
    s = W.tiny(periodic=True, n=(6, 6, 6), natom=1)
    assert T.Options.norb_offset.offset == 6 * 4 and T.Options.norb_total.offset == 7 * 4
    assert C.sizeof(T.Options) == 8 * 4
    assert _check_options(lib, s, 4)[0] == 0
    assert _check_options(lib, s, 4, norb_total=4)[0] == 0
    assert _check_options(lib, s, 4, norb_offset=12, norb_total=16)[0] == 0
    assert _check_options(lib, s, 4, norb_offset=0, norb_total=16)[0] == 0
    st, msg = _check_options(lib, s, 4, norb_offset=13, norb_total=16)
    assert st == 1 and "exceeds norb_total" in msg
    st, msg = _check_options(lib, s, 4, norb_offset=2)
    assert st == 1 and "norb_offset needs norb_total" in msg
    st, msg = _check_options(lib, s, 4, precision=5)
    assert st == 1 and "precision" in msg


def test_noalloc_wrapper_refuses_wrong_sizes_before_any_call():
    """The Python wrapper of the allocation-free potential refuses arrays that do not hold the grid
    (a short array would be read or written past its end on the device) before it reaches the
    library; the size check comes first, so it runs without a GPU."""
    torch = pytest.importorskip("torch")
    from paper_1804_01404_gb300 import tdks as T
    s = W.tiny(periodic=True, n=(6, 6, 6), natom=1)
    good = torch.zeros((6, 6, 6), dtype=torch.float64)
    short = torch.zeros(6 * 6 * 6 - 1, dtype=torch.float64)
    with pytest.raises(ValueError, match="points"):
        T.hxc_noalloc(s, short, good)
    with pytest.raises(ValueError, match="points"):
        T.hxc_noalloc(s, good, short)
    with pytest.raises(ValueError, match="CUDA"):
        T.hxc_noalloc(s, good, good)                 # right size, but host tensors
