"""Seeded synthetic workloads: system descriptions and initial orbitals.

This module is the one place that both the CUDA path and the FP64 CPU oracle take
their inputs from.  It holds geometry, k-point sets, field parameters and the
seeded random orbital generator, and none of the propagation arithmetic.

Shapes follow the paper's workloads: a periodic Si-like diamond cell driven by a
1.55 eV pulse (Sec. 4.2), an isolated nanocluster kicked by an impulse (Sec. 3.1,
3.3), and a chain of 256 unit cells coupled to a 1D Maxwell grid (Sec. 5).
No pseudopotential files or ground states exist here, so atoms are synthetic
erf/Gaussian pseudo-atoms and the initial orbitals are orthonormalised low-pass
random complex fields.

Units are Hartree atomic units (hbar = m = e = 1).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

HARTREE_EV = 27.211386245988
FS_AU = 41.341373335  # atomic units of time per femtosecond


@dataclass
class Atom:
    R: tuple          # position (bohr)
    Z: float          # local-potential charge, V = -Z erf(r/sigma)/r
    sigma: float = 0.8


@dataclass
class Projectors:
    """Kleinman-Bylander s + p channels shared by every atom (4 functions per atom)."""
    E_s: float = 1.0
    E_p: float = -1.0
    r_cut: float = 1.6
    width: float = 0.8


@dataclass
class Field:
    """Spatially uniform field, given as A'(t) = A(t)/c.

    kind = "none":  A' = 0.
    kind = "step":  A'(t) = A0 for t > 0 (impulsive kick in the velocity gauge, Eq. impulsive_A).
    kind = "pulse": A(t) = Im{A0 cos^2[pi(t-T/2)/T] exp[-i w (t-T/2) - 2 pi i cep]}, 0<t<T (Eq. pulse);
                    A0 here is already divided by c.  `more` adds delayed pulses of the same form,
                    each (A0, omega, T, cep, delay), and A' is the sum (pump-probe).
    kind = "table": A'(t) from samples table[i] = A'(t0 + i dt_table), linear in between, the end
                    samples outside the table.
    """
    kind: str = "none"
    A0: tuple = (0.0, 0.0, 0.0)
    omega: float = 0.0
    T: float = 0.0
    cep: float = 0.0
    more: tuple = ()
    table: object = None
    t0: float = 0.0
    dt_table: float = 0.0


@dataclass
class System:
    n: tuple                  # grid points (nx, ny, nz)
    h: tuple                  # spacing (hx, hy, hz), bohr
    periodic: bool
    atoms: list
    proj: Projectors
    kpts: np.ndarray          # [nk, 3]
    kw: np.ndarray            # [nk]
    norb: int
    dt: float = 0.02
    nsteps: int = 100
    field: Field = field(default_factory=Field)
    kick: tuple = (0.0, 0.0, 0.0)   # isolated systems: psi(0+) = exp(i kick . r) phi
    name: str = ""

    @property
    def npts(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])

    @property
    def nk(self) -> int:
        return int(len(self.kpts))

    @property
    def dV(self) -> float:
        return float(self.h[0] * self.h[1] * self.h[2])


def _gamma():
    return np.zeros((1, 3)), np.ones(1)


def mp_shifted(nkdiv: int, a: float):
    """Shifted Monkhorst-Pack grid: k_i in {(2j+1-n)/(2n)} * 2pi/a per axis, equal weights."""
    f = (2.0 * np.arange(nkdiv) + 1.0 - nkdiv) / (2.0 * nkdiv)
    kz, ky, kx = np.meshgrid(f, f, f, indexing="ij")
    k = np.stack([kx.ravel(), ky.ravel(), kz.ravel()], axis=1) * (2.0 * np.pi / a)
    return k, np.full(len(k), 1.0 / len(k))


DIAMOND_FRAC = np.array([
    [0.00, 0.00, 0.00], [0.00, 0.50, 0.50], [0.50, 0.00, 0.50], [0.50, 0.50, 0.00],
    [0.25, 0.25, 0.25], [0.25, 0.75, 0.75], [0.75, 0.25, 0.75], [0.75, 0.75, 0.25]])


def small_periodic(nsteps=100) -> System:
    """Periodic cubic cell L = 8 bohr, 16^3 grid, two Z=4 pseudo-atoms, 8 orbitals at Gamma,
    impulse kick kappa = 0.001 along z applied as an A'-step (velocity gauge)."""
    L, n = 8.0, 16
    kp, kw = _gamma()
    return System(n=(n, n, n), h=(L / n,) * 3, periodic=True,
                  atoms=[Atom((1.9, 2.1, 2.3), 4.0), Atom((5.8, 6.1, 5.6), 4.0)],
                  proj=Projectors(), kpts=kp, kw=kw, norb=8, dt=0.02, nsteps=nsteps,
                  field=Field("step", (0.0, 0.0, 0.001)), name="periodic-16^3-2atom-8orb")


def pulse_field(omega_ev=1.55, e0=1e-3, t_fs=10.0, axis=2) -> Field:
    w = omega_ev / HARTREE_EV
    a0 = [0.0, 0.0, 0.0]
    a0[axis] = e0 / w            # A0/c = E0/omega
    return Field("pulse", tuple(a0), omega=w, T=t_fs * FS_AU, cep=0.0)


def diamond_crystal(n=20, nkdiv=4, norb=16, a=10.26, nsteps=2000) -> System:
    """8-atom cubic diamond cell a = 10.26 bohr (Si-like), 20^3 grid, 16 orbitals x 4^3 shifted
    MP k-points, driven by a sin^2 pulse along z (1.55 eV, 1e-3 au peak field, 10 fs)."""
    kp, kw = mp_shifted(nkdiv, a)
    atoms = [Atom(tuple(f * a), 4.0) for f in DIAMOND_FRAC]
    return System(n=(n, n, n), h=(a / n,) * 3, periodic=True, atoms=atoms, proj=Projectors(),
                  kpts=kp, kw=kw, norb=norb, dt=0.02, nsteps=nsteps, field=pulse_field(),
                  name=f"diamond-{n}^3-{norb}orb-{len(kp)}k")


def random_cluster_atoms(natom=128, radius=14.0, dmin=3.0, seed=1):
    """Uniform random positions in a sphere (rejection-sampled to >= dmin apart), Z 50/50 of {1, 4}."""
    rng = np.random.default_rng(seed)
    pos = []
    for _ in range(1000 * natom + 1000):
        if len(pos) == natom:
            break
        p = rng.uniform(-radius, radius, 3)
        if np.dot(p, p) > radius * radius:
            continue
        if all(np.linalg.norm(p - q) >= dmin for q in pos):
            pos.append(p)
    if len(pos) < natom:
        raise ValueError(f"cannot place {natom} atoms {dmin} bohr apart in a sphere of radius {radius}")
    Z = rng.permutation(np.array([1.0] * (natom // 2) + [4.0] * (natom - natom // 2)))
    return [Atom(tuple(p), float(z)) for p, z in zip(pos, Z)]


def isolated_cluster(n=96, h=0.4, natom=128, norb=256, radius=14.0, seed=1, nsteps=4000) -> System:
    """Isolated cluster: n^3 grid, spacing 0.4 bohr, zero boundary, mixed Z=1/Z=4 pseudo-atoms,
    impulse kick exp(i 0.001 z)."""
    kp, kw = _gamma()
    return System(n=(n, n, n), h=(h,) * 3, periodic=False,
                  atoms=random_cluster_atoms(natom, radius, 3.0, seed), proj=Projectors(),
                  kpts=kp, kw=kw, norb=norb, dt=0.02, nsteps=nsteps,
                  kick=(0.0, 0.0, 0.001), name=f"cluster-{n}^3-{natom}atom-{norb}orb")


def multiscale_cell(n=16, nkdiv=2, norb=16, a=10.26) -> System:
    """One microscopic cell of the multiscale chain: 8-atom cubic cell, 16^3 grid, 16 x 8 k."""
    s = diamond_crystal(n=n, nkdiv=nkdiv, norb=norb, a=a, nsteps=1000)
    s.field = Field("none")
    s.name = f"ms-cell-{n}^3-{norb}orb-{len(s.kpts)}k"
    return s


def tiny(periodic=True, n=(6, 6, 6), norb=2, natom=1, nk=1, seed=0) -> System:
    """Tiny system for brute-force checks (dense matrices, explicit loops)."""
    rng = np.random.default_rng(1000 + seed)
    h = (0.55, 0.6, 0.65)
    box = np.array(n) * np.array(h)
    atoms = []
    for _ in range(natom):
        c = box / 2 if periodic else np.zeros(3)
        atoms.append(Atom(tuple(c + rng.uniform(-0.4, 0.4, 3)), 2.0, 0.7))
    if nk == 1:
        kp, kw = np.array([[0.13, -0.21, 0.17]]) if periodic else np.zeros((1, 3)), np.ones(1)
    else:
        kp = rng.uniform(-0.5, 0.5, (nk, 3)) if periodic else np.zeros((nk, 3))
        kw = np.full(nk, 1.0 / nk)
    return System(n=tuple(n), h=h, periodic=periodic, atoms=atoms,
                  proj=Projectors(E_s=0.7, E_p=-0.4, r_cut=1.3, width=0.65),
                  kpts=kp, kw=kw, norb=norb, dt=0.02, nsteps=4, name="tiny")


def _grid_freq(n, h):
    return [2.0 * np.pi * np.fft.fftfreq(n[a], d=h[a]) for a in range(3)]


def initial_orbitals(s: System, seed: int = 0, orthonormal: bool = True) -> np.ndarray:
    """Seeded orthonormalised low-pass random complex fields, complex128 [nk, norb, nz, ny, nx].

    Per (k, n) an independent PCG64 stream draws complex Gaussian coefficients on the grid's
    reciprocal lattice, damped by exp(-|G|^2/(2 Gc^2)) with Gc = 2 * (2 pi / L_max) and cut at
    3 Gc.  Isolated systems multiply by a sin^2 box window so the fields vanish at the faces.
    Each k-block is then Loewdin-orthonormalised in FP64 with sum |u|^2 dV = 1.
    The isolated kick exp(i kick . r) is NOT applied here.
    """
    nx, ny, nz = s.n
    gx, gy, gz = _grid_freq(s.n, s.h)
    G2 = gz[:, None, None] ** 2 + gy[None, :, None] ** 2 + gx[None, None, :] ** 2
    L = max(s.n[a] * s.h[a] for a in range(3))
    gc = 2.0 * (2.0 * np.pi / L)
    damp = np.exp(-G2 / (2.0 * gc * gc)) * (G2 <= 9.0 * gc * gc)
    if not s.periodic:
        wins = [np.sin(np.pi * (np.arange(m) + 1.0) / (m + 1.0)) ** 2 for m in (nz, ny, nx)]
        window = wins[0][:, None, None] * wins[1][None, :, None] * wins[2][None, None, :]
    out = np.empty((s.nk, s.norb, nz, ny, nx), np.complex128)
    for k in range(s.nk):
        for b in range(s.norb):
            rng = np.random.default_rng([seed, k, b, 7])
            c = (rng.standard_normal((nz, ny, nx)) + 1j * rng.standard_normal((nz, ny, nx))) * damp
            u = np.fft.ifftn(c)
            if not s.periodic:
                u = u * window
            out[k, b] = u
        U = out[k].reshape(s.norb, -1)
        if orthonormal:
            S = (U.conj() @ U.T) * s.dV
            w, V = np.linalg.eigh(S)
            X = (V * (1.0 / np.sqrt(w))) @ V.conj().T
            U = X.T @ U
        else:
            U = U / np.sqrt((np.abs(U) ** 2).sum(axis=1, keepdims=True) * s.dV)
        out[k] = U.reshape(s.norb, nz, ny, nx)
    return out
