"""Thin ctypes binding of libtdks.so (argument marshalling only).

Every step of the propagation runs in the library's CUDA kernels; this module converts a
system description into the C structs of include/tdks.h and passes device pointers of torch
tensors.  There is no CPU fallback: if libtdks.so is missing or CUDA is unavailable the calls fail.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtdks.so")

TDKS_F64, TDKS_F32 = 0, 1
PRED_PC, PRED_EXTRAP, PRED_LEARNED = 0, 1, 2
STEP_OBS_DOUBLES = 11        # doubles of one step-observable block (tdks_copy_step_observables)
NN_NPARAMS = 9105
FIELD_NONE, FIELD_STEP, FIELD_PULSE, FIELD_TABLE = 0, 1, 2, 3
STATUS = {0: "TDKS_OK", 1: "TDKS_EINVAL", 2: "TDKS_ENOMEM", 3: "TDKS_ECUDA", 4: "TDKS_ETIMEOUT",
          5: "TDKS_ENONFINITE", 6: "TDKS_EUNSUPPORTED"}


class TdksError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Grid(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("h", C.c_double * 3), ("periodic", C.c_int)]


class Cell(C.Structure):
    _fields_ = [("L", C.c_double * 3)]


class AtomC(C.Structure):
    _fields_ = [("R", C.c_double * 3), ("Z", C.c_double), ("sigma", C.c_double), ("proj", C.c_int)]


class ProjectorC(C.Structure):
    _fields_ = [("E_s", C.c_double), ("E_p", C.c_double), ("r_cut", C.c_double), ("width", C.c_double)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("hartree", C.c_int), ("xc", C.c_int), ("pc", C.c_int),
                ("ncell", C.c_int), ("obs_at_start", C.c_int), ("norb_offset", C.c_int), ("norb_total", C.c_int)]


class Obs(C.Structure):
    _fields_ = [("J", C.c_double * 3), ("dipole", C.c_double * 3), ("norm_min", C.c_double),
                ("norm_max", C.c_double), ("e_band", C.c_double), ("n_elec", C.c_double),
                ("residual", C.c_double), ("fallbacks", C.c_double)]

    def as_dict(self):
        return dict(J=np.array(self.J[:]), dipole=np.array(self.dipole[:]), norm_min=self.norm_min,
                    norm_max=self.norm_max, e_band=self.e_band, n_elec=self.n_elec,
                    residual=self.residual, fallbacks=self.fallbacks)


NPHASE = 7
PHASES = ("taylor_predictor", "taylor_corrector", "hpsi", "hartree_xc", "observables", "other", "stencil_kernel")


class Stats(C.Structure):
    _fields_ = [("launches", C.c_longlong), ("calls", C.c_longlong * NPHASE), ("ms", C.c_double * NPHASE)]

    def as_dict(self):
        return dict(launches=int(self.launches),
                    calls={p: int(self.calls[i]) for i, p in enumerate(PHASES)},
                    ms={p: float(self.ms[i]) for i, p in enumerate(PHASES)})


_lib = None
_D3 = C.c_double * 3


def load_library(path: str = LIB_PATH):
    """Load libtdks.so and declare its signatures.  Raises if the library was not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} not found: build it with `python -m paper_1804_01404_gb300.build`")
    lib = C.CDLL(path)
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    sig = {
        "tdks_init": [C.POINTER(Grid), C.POINTER(Cell), C.POINTER(AtomC), i, C.POINTER(ProjectorC), i,
                      C.POINTER(C.c_double), C.POINTER(C.c_double), i, i, C.POINTER(Options), vp,
                      C.POINTER(vp)],
        "tdks_set_field": [vp, i, _D3, d, d, d],
        "tdks_add_pulse": [vp, _D3, d, d, d, d],
        "tdks_set_field_table": [vp, C.POINTER(C.c_double), i, d, d],
        "tdks_kick": [vp, vp, _D3],
        "tdks_update_potential": [vp, vp],
        "tdks_hpsi": [vp, vp, vp, _D3],
        "tdks_taylor_step": [vp, vp, d, _D3],
        "tdks_step": [vp, vp, d, d],
        "tdks_read_step_observables": [vp, C.POINTER(Obs)],
        "tdks_copy_step_observables": [vp, vp],
        "tdks_unpack_step_observables": [vp, vp, C.POINTER(Obs)],
        "tdks_observables": [vp, vp, _D3, vp, C.POINTER(Obs)],
        "tdks_check_options": [C.POINTER(Grid), i, i, C.POINTER(Options)],
        "tdks_get_grid_array": [vp, i, vp],
        "tdks_check": [vp],
        "tdks_profile": [vp, i],
        "tdks_set_predictor": [vp, i, d],
        "tdks_set_step_graph": [vp, i],
        "tdks_ms_init": [vp, i, i, d, C.POINTER(C.c_double), C.POINTER(C.c_double)],
        "tdks_ms_step": [vp, vp, d, d],
        "tdks_ms_read": [vp, C.POINTER(C.c_double), C.POINTER(C.c_double)],
        "tdks_nn_init": [vp, C.c_ulonglong],
        "tdks_nn_params": [vp, C.POINTER(C.c_float), i, i],
        "tdks_nn_train": [vp, vp, i, i, i, d, C.c_ulonglong, C.POINTER(C.c_double)],
        "tdks_nn_predict": [vp, vp, vp, i],
        "tdks_nn_gradient": [vp, vp, vp, C.POINTER(C.c_double), C.POINTER(C.c_float)],
        "tdks_stats_read": [vp, C.POINTER(Stats), i],
        "tdks_query": [vp, C.POINTER(i), C.POINTER(i), C.POINTER(i), C.POINTER(i), C.POINTER(i)],
        "tdks_tile_variant": [vp, i, C.POINTER(i), C.POINTER(C.c_float)],
        "tdks_cell_variant": [vp, i, C.POINTER(i), C.POINTER(C.c_float)],
        "tdks_project_variant": [vp, i, C.POINTER(i), C.POINTER(C.c_float)],
        "tdks_set_wait_test": [vp, C.c_longlong, i],
        "tdks_state_size": [vp, C.POINTER(C.c_size_t)],
        "tdks_ms_size": [vp, C.POINTER(i)],
        "tdks_probe_fp64": [C.POINTER(C.c_double)],
        "tdks_probe_fp32": [C.POINTER(C.c_double)],
        "tdks_oscillator_strength": [C.POINTER(C.c_double), i, d, d, C.POINTER(C.c_double), i,
                                     C.POINTER(C.c_double), vp],
        "tdks_conductivity": [C.POINTER(C.c_double), i, d, d, C.POINTER(C.c_double), i, i,
                              C.POINTER(C.c_double), C.POINTER(C.c_double), vp],
        "tdks_work": [C.POINTER(C.c_double), C.POINTER(C.c_double), i, d, C.POINTER(C.c_double), vp],
        "tdks_dos": [C.POINTER(C.c_double), i, i, C.POINTER(C.c_double), C.POINTER(C.c_double), i, d,
                     C.POINTER(C.c_double), vp],
        "tdks_field_at": [vp, d, C.POINTER(C.c_double), C.POINTER(C.c_double)],
        "tdks_hxc_noalloc": [C.POINTER(Grid), vp, vp, i, i, vp],
        "tdks_set_longitudinal": [vp, i, vp, d],
        "tdks_ground_state": [vp, vp, i, d, d, d, C.POINTER(C.c_double)],
        "tdks_excited_pairs": [vp, vp, vp, C.POINTER(C.c_double)],
        "tdks_longitudinal_read": [vp, C.POINTER(C.c_double)],
        "tdks_set_mbj": [vp, d],
        "tdks_orbital_energies": [vp, vp, C.POINTER(C.c_double), i, C.POINTER(C.c_double)],
        "tdks_mbj_c": [vp, C.POINTER(C.c_double)],
        "tdks_get_state": [vp, vp, C.c_size_t],
        "tdks_set_state": [vp, vp, C.c_size_t],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.tdks_last_error.restype = C.c_char_p
    lib.tdks_last_error.argtypes = []
    lib.tdks_abi_version.restype = C.c_int
    lib.tdks_destroy.argtypes = [vp]
    lib.tdks_destroy.restype = None
    _lib = lib
    return lib


def probe_fp64():
    """Measured FP64 FMA throughput of the current CUDA device, TFLOP/s (tdks_probe_fp64)."""
    lib = load_library()
    x = C.c_double()
    _check(lib.tdks_probe_fp64(C.byref(x)))
    return x.value


def probe_fp32():
    """Measured FP32 FMA throughput of the current CUDA device, TFLOP/s (tdks_probe_fp32)."""
    lib = load_library()
    x = C.c_double()
    _check(lib.tdks_probe_fp32(C.byref(x)))
    return x.value


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _stream_handle(stream):
    return C.c_void_p(stream.cuda_stream if stream is not None else 0)


def oscillator_strength(d, dt, kappa, E, stream=None):
    """df/dE of a dipole series d[i] = d(i dt) after the kick exp(i kappa r) (tdks_oscillator_strength)."""
    lib = load_library()
    d = np.ascontiguousarray(d, np.float64)
    E = np.ascontiguousarray(E, np.float64)
    out = np.zeros(len(E))
    _check(lib.tdks_oscillator_strength(_dptr(d), len(d), float(dt), float(kappa), _dptr(E), len(E), _dptr(out),
                                        _stream_handle(stream)))
    return out


def conductivity(I, dt, Ap0, w, subtract_mean=True, stream=None):
    """sigma(w) and eps(w) (complex arrays) of a current series I[i] = I(i dt) after the step
    A'(t) = Ap0 theta(t) (tdks_conductivity).  eps is None unless every w > 0."""
    lib = load_library()
    I = np.ascontiguousarray(I, np.float64)
    w = np.ascontiguousarray(w, np.float64)
    sig = np.zeros(2 * len(w))
    want_eps = bool(np.all(w > 0))
    eps = np.zeros(2 * len(w)) if want_eps else None
    _check(lib.tdks_conductivity(_dptr(I), len(I), float(dt), float(Ap0), _dptr(w), len(w), int(bool(subtract_mean)),
                                 _dptr(sig), _dptr(eps) if want_eps else None, _stream_handle(stream)))
    sigma = sig[0::2] + 1j * sig[1::2]
    return sigma, (eps[0::2] + 1j * eps[1::2]) if want_eps else None


def work(I, E, dt, stream=None):
    """W(t_i) = int_0^t_i I.E dt' of sampled I[i][3], E[i][3] at t_i = i dt (tdks_work)."""
    lib = load_library()
    I = np.ascontiguousarray(I, np.float64).reshape(-1, 3)
    E = np.ascontiguousarray(E, np.float64).reshape(-1, 3)
    if len(I) != len(E):
        raise ValueError("I and E need the same number of samples")
    out = np.zeros(len(I))
    _check(lib.tdks_work(_dptr(I), _dptr(E), len(I), float(dt), _dptr(out), _stream_handle(stream)))
    return out


def hxc_noalloc(system, rho, out, hartree=True, xc=1, stream=None):
    """V_H + V_xc of a density into out without allocating device memory (tdks_hxc_noalloc); rho and
    out are contiguous CUDA float64 tensors of the system's grid (n0 n1 n2 points) on the current
    device; asynchronous on `stream`.  Arrays of another size or on another device are refused here:
    the library cannot see their extent, and a short array would be accessed past its end."""
    import torch
    npts = int(system.n[0]) * int(system.n[1]) * int(system.n[2])
    for t in (rho, out):
        if t.numel() != npts:
            raise ValueError(f"rho and out must hold the grid's {npts} points, got {t.numel()}")
    for t in (rho, out):
        if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
            raise ValueError("rho and out must be contiguous CUDA float64 tensors")
        if t.device.index != torch.cuda.current_device():
            raise ValueError("rho and out must be on the current CUDA device")
    lib = load_library()
    g = Grid((C.c_int * 3)(*system.n), (C.c_double * 3)(*system.h), 1 if system.periodic else 0)
    _check(lib.tdks_hxc_noalloc(C.byref(g), C.c_void_p(rho.data_ptr()), C.c_void_p(out.data_ptr()), int(hartree),
                                int(xc), _stream_handle(stream)))


def dos(eps, kw, E, sigma, stream=None):
    """Gaussian-broadened, spin-saturated density of states of orbital energies eps[nk][norb] with
    k-weights kw at energies E (tdks_dos)."""
    lib = load_library()
    eps = np.ascontiguousarray(eps, np.float64)
    kw = np.ascontiguousarray(kw, np.float64)
    E = np.ascontiguousarray(E, np.float64)
    if eps.ndim != 2 or eps.shape[0] != len(kw):
        raise ValueError("eps must be [nk][norb] with nk = len(kw)")
    out = np.zeros(len(E))
    _check(lib.tdks_dos(_dptr(eps), eps.shape[0], eps.shape[1], _dptr(kw), _dptr(E), len(E), float(sigma), _dptr(out),
                        _stream_handle(stream)))
    return out


def _check(status):
    if status != 0:
        raise TdksError(status, _lib.tdks_last_error().decode())


def _vec3(v):
    return _D3(*[float(x) for x in (v if v is not None else (0.0, 0.0, 0.0))])


def _ptr(t, dtype=None):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected dtype {dtype}, got {t.dtype}")
    return C.c_void_p(t.data_ptr())


def _host_obs_ptr(t):
    import torch
    if not (isinstance(t, torch.Tensor) and t.device.type == "cpu" and t.is_contiguous()
            and t.dtype == torch.float64 and t.numel() >= STEP_OBS_DOUBLES):
        raise ValueError(f"expected a contiguous CPU float64 tensor of >= {STEP_OBS_DOUBLES} values")
    return C.c_void_p(t.data_ptr())


class Context:
    """One propagation context (libtdks tdks_ctx) for a system description.

    `system` needs: n, h, periodic, atoms (R, Z, sigma), proj (E_s, E_p, r_cut, width), kpts, kw,
    norb, field.  Orbitals are torch tensors [nk, norb, nz, ny, nx], complex128 (f64) or
    complex64 (f32), on the current CUDA device."""

    def __init__(self, system, precision="f64", hartree=True, xc=True, pc=True, stream=None, ncell=1,
                 obs_at_start=False, mbj_c=None, norb_offset=0, norb_total=0):
        import torch
        lib = load_library()
        self.lib = lib
        self.system = system
        self.precision = precision
        self.cdtype = torch.complex128 if precision == "f64" else torch.complex64
        g = Grid((C.c_int * 3)(*system.n), (C.c_double * 3)(*system.h), 1 if system.periodic else 0)
        cell = Cell((C.c_double * 3)(*[system.n[a] * system.h[a] for a in range(3)]))
        natom = len(system.atoms)
        atoms = (AtomC * max(natom, 1))()
        for i, at in enumerate(system.atoms):
            atoms[i] = AtomC(_D3(*at.R), at.Z, at.sigma, 0)
        pr = ProjectorC(system.proj.E_s, system.proj.E_p, system.proj.r_cut, system.proj.width)
        kp = np.ascontiguousarray(np.asarray(system.kpts, np.float64).reshape(-1))
        kw = np.ascontiguousarray(np.asarray(system.kw, np.float64))
        opts = Options(TDKS_F64 if precision == "f64" else TDKS_F32, int(hartree), int(xc), int(pc), int(ncell),
                       int(bool(obs_at_start)), int(norb_offset), int(norb_total))
        self.ncell = int(ncell)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        ctx = C.c_void_p()
        _check(lib.tdks_init(C.byref(g), C.byref(cell), atoms, natom, C.byref(pr), 1,
                             kp.ctypes.data_as(C.POINTER(C.c_double)),
                             kw.ctypes.data_as(C.POINTER(C.c_double)), len(kw), int(system.norb),
                             C.byref(opts), C.c_void_p(stream.cuda_stream), C.byref(ctx)))
        self.ctx = ctx
        if mbj_c is not None:
            self.set_mbj(mbj_c)
        f = getattr(system, "field", None)
        if f is not None and f.kind == "table":
            self.set_field_table(f.table, f.t0, f.dt_table)
        elif f is not None and f.kind != "none":
            kind = {"step": FIELD_STEP, "pulse": FIELD_PULSE}[f.kind]
            self.set_field(kind, f.A0, f.omega, f.T, f.cep)
            for (A0, omega, T, cep, delay) in getattr(f, "more", ()):
                self.add_pulse(A0, omega, T, cep, delay)

    def __del__(self):
        try:
            if getattr(self, "ctx", None) is not None and self.ctx.value:
                self.lib.tdks_destroy(self.ctx)
                self.ctx = None
        except Exception:
            pass

    def close(self):
        self.__del__()

    # ---- calls (asynchronous on the context stream unless stated)
    def set_field(self, kind, A0, omega=0.0, T=0.0, cep=0.0):
        _check(self.lib.tdks_set_field(self.ctx, int(kind), _vec3(A0), float(omega), float(T), float(cep)))

    def add_pulse(self, A0, omega, T, cep=0.0, delay=0.0):
        _check(self.lib.tdks_add_pulse(self.ctx, _vec3(A0), float(omega), float(T), float(cep), float(delay)))

    def set_field_table(self, table, t0, dt_table):
        tab = np.ascontiguousarray(table, np.float64).reshape(-1, 3)
        _check(self.lib.tdks_set_field_table(self.ctx, tab.ctypes.data_as(C.POINTER(C.c_double)), len(tab),
                                             float(t0), float(dt_table)))

    def ground_state(self, u, max_iter=500, tol=1e-8, degree=0, mix=0.3):
        """Self-consistent ground state into u (tdks_ground_state, Chebyshev-filtered subspace iteration
        of the given filter degree, 0: 10); returns (iterations, residual, band energy)."""
        out = (C.c_double * 3)()
        _check(self.lib.tdks_ground_state(self.ctx, _ptr(u, self.cdtype), int(max_iter), float(tol), float(degree),
                                          float(mix), out))
        return int(out[0]), float(out[1]), float(out[2])

    def excited_pairs(self, u, u_gs):
        """Number density of excited electron-hole pairs of u relative to the ground-state orbitals u_gs
        (tdks_excited_pairs)."""
        n = C.c_double()
        _check(self.lib.tdks_excited_pairs(self.ctx, _ptr(u, self.cdtype), _ptr(u_gs, self.cdtype), C.byref(n)))
        return n.value

    def set_longitudinal(self, enable, u=None, t0=0.0):
        """Longitudinal geometry on (A'_ind from d^2 A'_ind/dt^2 = 4 pi J, starting at rest with J of u
        at t0) or off (tdks_set_longitudinal)."""
        _check(self.lib.tdks_set_longitudinal(self.ctx, int(enable), _ptr(u, self.cdtype) if u is not None else None,
                                              float(t0)))

    def orbital_energies(self, u, Ap=None, rotate=False):
        """Ritz values of H_q in the span of each k's orbitals, ascending, numpy [nk, norb]; rotate=True
        also turns u into the Ritz vectors (tdks_orbital_energies)."""
        eps = np.zeros((len(self.system.kw), self.system.norb))
        ap = (C.c_double * 3)(*Ap) if Ap is not None else None
        _check(self.lib.tdks_orbital_energies(self.ctx, _ptr(u, self.cdtype), ap, int(bool(rotate)),
                                              eps.ctypes.data_as(C.POINTER(C.c_double))))
        return eps

    def set_mbj(self, c):
        """TB-mBJ (xc = 3): c > 0 fixes c, c <= 0 forms it from the density (tdks_set_mbj)."""
        _check(self.lib.tdks_set_mbj(self.ctx, float(c)))

    def mbj_c(self):
        """The c of the last TB-mBJ potential (tdks_mbj_c)."""
        v = C.c_double()
        _check(self.lib.tdks_mbj_c(self.ctx, C.byref(v)))
        return v.value

    def longitudinal_A(self):
        """A'_ind at the end of the last step (tdks_longitudinal_read)."""
        a = (C.c_double * 3)()
        _check(self.lib.tdks_longitudinal_read(self.ctx, a))
        return np.array(a[:])

    def field_at(self, t):
        """(A'(t), E(t) = -dA'/dt) of the context's field (tdks_field_at)."""
        ap = (C.c_double * 3)()
        e = (C.c_double * 3)()
        _check(self.lib.tdks_field_at(self.ctx, float(t), ap, e))
        return np.array(ap[:]), np.array(e[:])

    def kick(self, u, kappa):
        _check(self.lib.tdks_kick(self.ctx, _ptr(u, self.cdtype), _vec3(kappa)))

    def update_potential(self, u):
        _check(self.lib.tdks_update_potential(self.ctx, _ptr(u, self.cdtype)))

    def hpsi(self, u, hu, Aprime=None):
        _check(self.lib.tdks_hpsi(self.ctx, _ptr(u, self.cdtype), _ptr(hu, self.cdtype), _vec3(Aprime)))

    def taylor_step(self, u, dt, Aprime=None):
        _check(self.lib.tdks_taylor_step(self.ctx, _ptr(u, self.cdtype), float(dt), _vec3(Aprime)))

    def step(self, u, t, dt):
        _check(self.lib.tdks_step(self.ctx, _ptr(u, self.cdtype), float(t), float(dt)))

    def read_step_observables(self):
        o = Obs()
        _check(self.lib.tdks_read_step_observables(self.ctx, C.byref(o)))
        return o.as_dict()

    def copy_step_observables(self, host_buf):
        """Enqueue the copy of the last step's observable block (STEP_OBS_DOUBLES doubles) into
        host_buf, a page-locked CPU float64 tensor, without waiting (tdks_copy_step_observables)."""
        _check(self.lib.tdks_copy_step_observables(self.ctx, _host_obs_ptr(host_buf)))

    def unpack_step_observables(self, host_buf):
        """The observables of a block copied by copy_step_observables, once the stream has passed the
        copy (tdks_unpack_step_observables)."""
        o = Obs()
        _check(self.lib.tdks_unpack_step_observables(self.ctx, _host_obs_ptr(host_buf), C.byref(o)))
        return o.as_dict()

    def observables(self, u, Aprime=None, rho=None):
        """All observables of u (tdks_observables); rho: optional CUDA float64 tensor [nz, ny, nx] that
        receives the density of u."""
        o = Obs()
        _check(self.lib.tdks_observables(self.ctx, _ptr(u, self.cdtype), _vec3(Aprime),
                                         _ptr(rho) if rho is not None else None, C.byref(o)))
        return o.as_dict()

    def grid_array(self, which):
        """0: V_loc, 1: V_Hxc(t), 2: rho(t), 3: rho0 -> torch float64 [nz, ny, nx] on the device."""
        import torch
        n = self.system.n
        out = torch.empty((n[2], n[1], n[0]), dtype=torch.float64, device="cuda")
        _check(self.lib.tdks_get_grid_array(self.ctx, int(which), _ptr(out)))
        return out

    # ---- multiscale
    def ms_init(self, dX, m0, A_now, A_prev):
        a = np.ascontiguousarray(A_now, np.float64)
        b = np.ascontiguousarray(A_prev, np.float64)
        self.nX = len(a)
        _check(self.lib.tdks_ms_init(self.ctx, len(a), int(m0), float(dX), a.ctypes.data_as(C.POINTER(C.c_double)),
                                     b.ctypes.data_as(C.POINTER(C.c_double))))

    def ms_step(self, u, t, dt):
        _check(self.lib.tdks_ms_step(self.ctx, _ptr(u, self.cdtype), float(t), float(dt)))

    def ms_read(self):
        n = C.c_int()
        _check(self.lib.tdks_ms_size(self.ctx, C.byref(n)))
        self.nX = n.value
        A = np.zeros(self.nX)
        I = np.zeros(self.nX)
        _check(self.lib.tdks_ms_read(self.ctx, A.ctypes.data_as(C.POINTER(C.c_double)),
                                     I.ctypes.data_as(C.POINTER(C.c_double))))
        return A, I

    # ---- predictor and learned network
    def set_predictor(self, mode, threshold=1e-5):
        _check(self.lib.tdks_set_predictor(self.ctx, int(mode), float(threshold)))

    def set_step_graph(self, enable=True):
        """Predicted and multiscale steps as CUDA graphs (default; a predicted step decides on the device)
        or as stream launches (a predicted step decides on the host) (tdks_set_step_graph)."""
        _check(self.lib.tdks_set_step_graph(self.ctx, int(bool(enable))))

    def nn_init(self, seed=0):
        _check(self.lib.tdks_nn_init(self.ctx, int(seed)))

    def nn_params(self, values=None):
        """Get the FP32 parameters (values=None) or set them."""
        buf = np.zeros(NN_NPARAMS, np.float32) if values is None else np.ascontiguousarray(values, np.float32)
        _check(self.lib.tdks_nn_params(self.ctx, buf.ctypes.data_as(C.POINTER(C.c_float)), NN_NPARAMS,
                                       0 if values is None else 1))
        return buf

    def nn_train(self, vseq, epochs=1, batch=8, lr=1e-3, seed=0):
        """vseq: CUDA float64 tensor [nt, nz, ny, nx] of consecutive V_Hxc; returns per-epoch loss."""
        loss = np.zeros(epochs)
        _check(self.lib.tdks_nn_train(self.ctx, _ptr(vseq), int(vseq.shape[0]), int(epochs), int(batch),
                                      float(lr), int(seed), loss.ctypes.data_as(C.POINTER(C.c_double))))
        return loss

    def nn_predict(self, vhist, vpred, mode=2):
        """mode 0: linear extrapolation, 1: cubic extrapolation, 2: the network."""
        _check(self.lib.tdks_nn_predict(self.ctx, _ptr(vhist), _ptr(vpred), int(mode)))

    def nn_gradient(self, vhist, vnext):
        g = np.zeros(NN_NPARAMS, np.float32)
        loss = C.c_double()
        _check(self.lib.tdks_nn_gradient(self.ctx, _ptr(vhist), _ptr(vnext), C.byref(loss),
                                         g.ctypes.data_as(C.POINTER(C.c_float))))
        return loss.value, g

    def profile(self, enable=True):
        """Phase timing on (True or 1: every phase; 2: the orbital stencil kernel only) or off
        (tdks_profile)."""
        _check(self.lib.tdks_profile(self.ctx, int(enable)))

    def stats(self, reset=False):
        st = Stats()
        _check(self.lib.tdks_stats_read(self.ctx, C.byref(st), int(reset)))
        return st.as_dict()

    def check(self):
        _check(self.lib.tdks_check(self.ctx))

    def tile_variant(self, set=-1):
        """Stencil variants of the tiled path (tdks_tile_variant): returns ([H v, Horner] variants,
        tuning ms [[H v x 7], [Horner x 7]])."""
        v = (C.c_int * 2)()
        ms = (C.c_float * 14)()
        _check(self.lib.tdks_tile_variant(self.ctx, int(set), v, ms))
        return [v[0], v[1]], [[float(x) for x in ms[:7]], [float(x) for x in ms[7:]]]

    def project_variant(self, set=-1):
        """Schedule of the FP32 tensor-core projections of the tile path (tdks_project_variant): returns
        (schedule in use, tuning ms [2, 4, 8 warps per CTA])."""
        v = C.c_int()
        ms = (C.c_float * 3)()
        _check(self.lib.tdks_project_variant(self.ctx, int(set), C.byref(v), ms))
        return v.value, [float(x) for x in ms]

    def cell_variant(self, set=-1):
        """Buffer scheme of the cell kernels' Taylor launches (tdks_cell_variant): returns (scheme in
        use, tuning ms [two buffers, in-place sweep, two buffers with the grid size built in, in-place
        sweep with the grid size built in])."""
        v = C.c_int()
        ms = (C.c_float * 4)()
        _check(self.lib.tdks_cell_variant(self.ctx, int(set), C.byref(v), ms))
        return v.value, [float(x) for x in ms]

    def get_state(self):
        """Checkpoint of the time-stepping state (tdks_get_state) as a numpy uint8 array."""
        n = C.c_size_t()
        _check(self.lib.tdks_state_size(self.ctx, C.byref(n)))
        buf = np.zeros(n.value, np.uint8)
        _check(self.lib.tdks_get_state(self.ctx, buf.ctypes.data_as(C.c_void_p), n.value))
        return buf

    def set_state(self, buf):
        """Restore a checkpoint written by get_state (tdks_set_state)."""
        b = np.ascontiguousarray(buf, np.uint8)
        _check(self.lib.tdks_set_state(self.ctx, b.ctypes.data_as(C.c_void_p), b.size))

    def set_wait_test(self, wait_limit=0, stop_after=-1):
        """Timeout-path test hook (tdks_set_wait_test); defaults restore normal operation."""
        _check(self.lib.tdks_set_wait_test(self.ctx, int(wait_limit), int(stop_after)))

    def query(self):
        v = [C.c_int() for _ in range(5)]
        _check(self.lib.tdks_query(self.ctx, *[C.byref(x) for x in v]))
        return dict(zip(("npts", "nk", "norb", "precision", "nsphere_points"), [x.value for x in v]))
