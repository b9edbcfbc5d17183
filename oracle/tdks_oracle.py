"""FP64 CPU oracle of one real-time TDKS step (test infrastructure, not product code).

Only the tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import or run this module.  It shares no code with the CUDA path:
it reads plain system descriptions (grid, atoms, projectors, k-points, orbitals) and
recomputes everything from the paper's equations with numpy in float64/complex128.

What it computes (Hartree atomic units, hbar = m = e = 1, A' = A/c):

* Sec. 4.1, Eq. (TDKS_solid): Bloch orbitals w_nk evolve under
  H_q = 1/2 (-i grad + q)^2 + V_loc + V_NL^q + V_H + V_xc with q = k + A'(t).
  Isolated systems (Sec. 3.1, Eq. TDKS) are the case q = 0 with zero boundary.
  The gradient is discretised with 8th-order central differences (4 neighbours per side per
  axis, the 25-point Laplacian), so 1/2(-i grad+q)^2 -> -1/2 sum_a D2_a - i q.D1 + |q|^2/2.
* Sec. 3.1: V_ion is a local part plus Kleinman-Bylander separable projectors,
  V_NL = sum E |beta><beta|; Sec. 4.1 notes the nonlocal part follows the vector potential to
  keep gauge invariance, which in Bloch form gives projectors beta(r) exp(-i q.(r - R_a)).
* Program summary / Sec. 1: the evolution operator is a truncated Taylor expansion (4th
  order here) with a predictor-corrector step for the self-consistent potential.
* Eq. (rho): rho = 2 sum_p |psi_p|^2 (spin saturated), with k-weights for Bloch orbitals.
* Eq. (TDKS): Hartree potential e^2 int rho(r')/|r-r'|; periodic cells solve it in G-space,
  isolated boxes with a zero-padded (Hockney) convolution.
* Sec. 3.1 LDA: adiabatic local exchange (Slater) and, as an option, the Perdew-Zunger correlation.
* Sec. 4.1 names the Becke-Johnson potential and its Tran-Blaha variant as xc options: TB-mBJ
  exchange (published Becke-Roussel / Becke-Johnson / Tran-Blaha forms, restated) with the
  kinetic energy density of the time-dependent orbitals, its current's share removed.
* Sec. 3.1: dipole d = -int r (rho - rho0); Eq. (distribution): oscillator-strength spectrum.
* Sec. 4.1, Eq. (sigma_ft): conductivity and dielectric function from the current after an A step;
  the work of the field W(t) = int I.E dt (excitation energy per volume).
* Eq. (macro_current): macroscopic current including the nonlocal term.
* Eq. (pulse), Eq. (impulsive_A): fields.
* Eq. (Maxwell_ms): 1D wave equation driven by the cell currents.

Readings where the paper is silent (stencil order, Taylor order, predictor-corrector form,
projector shapes, Hockney self-term, kick on a periodic cell ...) are listed in the design
notes; each is restated at the function that uses it.

Parity status: every function here is pinned by the CPU tests against closed forms, brute
force or invariants (plane-wave dispersion, dense eigendecomposition, Hockney direct sum,
Gaussian/cosine charges, J = -dE/dA'/Omega, energy conservation, f-sum slope, the closed-form
masked Fourier integral and the free-electron plasma limit of eps; for TB-mBJ the hydrogen
Becke-Roussel hole, plane-wave kinetic densities and the uniform-gas correction term).  The full
predictor-corrector step has no closed form: it is pinned only through those invariants.
"""
from __future__ import annotations

import math
import numpy as np

C_LIGHT = 137.035999084

# 8th-order central differences (4 neighbours per side).  Second derivative:
# f'' ~ (1/h^2)[c0 f(0) + sum_m c_m (f(m) + f(-m))]; first derivative: f' ~ (1/h) sum_m d_m (f(m) - f(-m)).
FD2 = (-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0)
FD1 = (4.0 / 5.0, -1.0 / 5.0, 4.0 / 105.0, -1.0 / 280.0)

# numpy axis of each Cartesian direction for arrays laid out [..., z, y, x]
_AX = {0: -1, 1: -2, 2: -3}


# --------------------------------------------------------------------------------------------
# grid
# --------------------------------------------------------------------------------------------
def coords(s):
    """1D coordinate arrays (x, y, z).  Periodic: r_j = j h on [0, L).
    Isolated: centred, r_j = (j - (n-1)/2) h (Sec. 2.1 cuboid with vacuum outside)."""
    out = []
    for a in range(3):
        j = np.arange(s.n[a], dtype=np.float64)
        out.append(j * s.h[a] if s.periodic else (j - (s.n[a] - 1) / 2.0) * s.h[a])
    return out


def cell_volume(s):
    return float(np.prod([s.n[a] * s.h[a] for a in range(3)]))


def shifted(u, m, a, periodic):
    """Array whose value at grid index j along axis a is u at j + m (periodic wrap, or zero
    outside the box for isolated systems)."""
    ax = _AX[a]
    if periodic:
        return np.roll(u, -m, axis=ax)
    out = np.zeros_like(u)
    n = u.shape[ax]
    src = [slice(None)] * u.ndim
    dst = [slice(None)] * u.ndim
    if m >= 0:
        src[ax], dst[ax] = slice(m, n), slice(0, n - m)
    else:
        src[ax], dst[ax] = slice(0, n + m), slice(-m, n)
    out[tuple(dst)] = u[tuple(src)]
    return out


def d2(u, a, s):
    r = FD2[0] * u
    for m in range(1, 5):
        r = r + FD2[m] * (shifted(u, m, a, s.periodic) + shifted(u, -m, a, s.periodic))
    return r / (s.h[a] ** 2)


def d1(u, a, s):
    r = np.zeros_like(u)
    for m in range(1, 5):
        r = r + FD1[m - 1] * (shifted(u, m, a, s.periodic) - shifted(u, -m, a, s.periodic))
    return r / s.h[a]


# --------------------------------------------------------------------------------------------
# ionic potential (Sec. 3.1: local part + Kleinman-Bylander separable part)
# --------------------------------------------------------------------------------------------
def local_potential(s):
    """V_loc on the grid [nz, ny, nx] for pseudo-atoms V_a(r) = -Z erf(|r-R|/sigma)/|r-R|.

    Periodic: the lattice sum in G-space over the grid's reciprocal vectors, G != 0 only
    (uniform neutralising background; the G=0 constant only shifts orbital phases):
      V(G) = (1/Omega) sum_a (-4 pi Z_a / G^2) exp(-G^2 sigma_a^2 / 4) exp(-i G.R_a),
      V(r) = Re sum_G V(G) exp(i G.r).
    Isolated: the direct sum, with the r -> R limit -2Z/(sigma sqrt(pi))."""
    x, y, z = coords(s)
    if s.periodic:
        g = [2.0 * np.pi * np.fft.fftfreq(s.n[a], d=s.h[a]) for a in range(3)]
        GX, GY, GZ = g[0][None, None, :], g[1][None, :, None], g[2][:, None, None]
        G2 = GX ** 2 + GY ** 2 + GZ ** 2
        G2s = np.where(G2 == 0.0, 1.0, G2)
        Vg = np.zeros(G2.shape, np.complex128)
        for at in s.atoms:
            R = at.R
            Vg += (-4.0 * np.pi * at.Z / G2s) * np.exp(-G2 * at.sigma ** 2 / 4.0) * \
                np.exp(-1j * (GX * R[0] + GY * R[1] + GZ * R[2]))
        Vg[G2 == 0.0] = 0.0
        Vg /= cell_volume(s)
        return np.real(np.fft.ifftn(Vg) * G2.size)
    Z3, Y3, X3 = np.meshgrid(z, y, x, indexing="ij")
    V = np.zeros((s.n[2], s.n[1], s.n[0]))
    for at in s.atoms:
        d = np.sqrt((X3 - at.R[0]) ** 2 + (Y3 - at.R[1]) ** 2 + (Z3 - at.R[2]) ** 2)
        with np.errstate(divide="ignore", invalid="ignore"):
            v = -at.Z * _erf(d / at.sigma) / d
        v[d == 0.0] = -2.0 * at.Z / (at.sigma * math.sqrt(math.pi))
        V += v
    return V


def _erf(x):
    from scipy.special import erf
    return erf(x)


def projector_tables(s):
    """Kleinman-Bylander projector tables, one dict per atom.

    Channels s, px, py, pz with energies (E_s, E_p, E_p, E_p).  Shapes on the grid points
    within r_cut of the atom (minimum image for periodic cells; isolated: points in the box):
      g(d) = exp(-d^2 / (2 w^2)) (1 - d^2/r_cut^2)^2,  beta = N {1, dx, dy, dz} g(d),
    each normalised on the grid so that sum beta^2 dV = 1.  d is the displacement r - R_a of the
    nearest image, used for the gauge phase exp(i q.d)."""
    x, y, z = coords(s)
    L = [s.n[a] * s.h[a] for a in range(3)]
    if s.periodic and s.proj.r_cut >= 0.5 * min(L):
        raise ValueError("projector sphere larger than half the cell")
    tabs = []
    for at in s.atoms:
        comps = []
        for a, c in enumerate((x, y, z)):
            dd = c - at.R[a]
            if s.periodic:
                dd = dd - L[a] * np.round(dd / L[a])
            comps.append(dd)
        DX, DY, DZ = comps[0][None, None, :], comps[1][None, :, None], comps[2][:, None, None]
        D2 = DX ** 2 + DY ** 2 + DZ ** 2
        inside = D2 < s.proj.r_cut ** 2
        iz, iy, ix = np.nonzero(inside)
        idx = (iz * s.n[1] + iy) * s.n[0] + ix
        d = np.stack([comps[0][ix], comps[1][iy], comps[2][iz]], axis=1)
        r2 = (d ** 2).sum(axis=1)
        g = np.exp(-r2 / (2.0 * s.proj.width ** 2)) * (1.0 - r2 / s.proj.r_cut ** 2) ** 2
        beta = np.stack([g, d[:, 0] * g, d[:, 1] * g, d[:, 2] * g])
        beta /= np.sqrt((beta ** 2).sum(axis=1, keepdims=True) * s.dV)
        E = np.array([s.proj.E_s, s.proj.E_p, s.proj.E_p, s.proj.E_p])
        tabs.append(dict(idx=idx, d=d, beta=beta, E=E))
    return tabs


def projections(s, tabs, q, u, weight_by=None):
    """c[..., a, p] = sum_{r in S_a} beta_ap(r) exp(i q.d) u(r) dV for a batch u[..., nz, ny, nx].
    weight_by = axis index b multiplies the sum by d_b (the b_ap moments of the current)."""
    flat = u.reshape(u.shape[:-3] + (-1,))
    out = np.zeros(u.shape[:-3] + (len(tabs), 4), np.complex128)
    for ia, t in enumerate(tabs):
        ph = np.exp(1j * (t["d"] @ np.asarray(q, dtype=np.float64)))
        w = ph if weight_by is None else ph * t["d"][:, weight_by]
        out[..., ia, :] = (flat[..., t["idx"]] * w) @ t["beta"].T * s.dV
    return out


def apply_nonlocal(s, tabs, q, u):
    """V_NL^q u = sum_ap E_p beta_ap(r) exp(-i q.d) c_ap  (Sec. 3.1 KB form, Sec. 4.1 gauge)."""
    c = projections(s, tabs, q, u)
    out = np.zeros(u.shape[:-3] + (u.shape[-3] * u.shape[-2] * u.shape[-1],), np.complex128)
    for ia, t in enumerate(tabs):
        ph = np.exp(-1j * (t["d"] @ np.asarray(q, dtype=np.float64)))
        contrib = ((c[..., ia, :] * t["E"]) @ t["beta"]) * ph
        out[..., t["idx"]] += contrib        # indices are unique within one atom
    return out.reshape(u.shape)


# --------------------------------------------------------------------------------------------
# Hamiltonian (Eq. TDKS_solid in Bloch form; Eq. TDKS for isolated, q = 0)
# --------------------------------------------------------------------------------------------
def hpsi(s, tabs, V, q, u):
    """H_q u for a batch u[..., nz, ny, nx] sharing the same q = k + A'.
    H_q = -1/2 sum_a D2_a - i sum_a q_a D1_a + |q|^2/2 + V(r) + V_NL^q."""
    q = np.asarray(q, dtype=np.float64)
    out = np.zeros_like(u)
    for a in range(3):
        out += -0.5 * d2(u, a, s)
        if q[a] != 0.0:
            out += -1j * q[a] * d1(u, a, s)
    out += (0.5 * float(q @ q) + V) * u
    out += apply_nonlocal(s, tabs, q, u)
    return out


def taylor4(s, tabs, V, q, u, dt, order=4):
    """Truncated Taylor expansion of exp(-i H dt) applied to u: sum_{n<=order} (-i dt H)^n u / n!
    (Program summary: explicit integration by a truncated Taylor expansion; order 4 here)."""
    term = u.copy()
    acc = u.copy()
    for n in range(1, order + 1):
        term = (-1j * dt / n) * hpsi(s, tabs, V, q, term)
        acc = acc + term
    return acc


# --------------------------------------------------------------------------------------------
# density, Hartree, exchange (Eq. rho, Eq. TDKS, LDA)
# --------------------------------------------------------------------------------------------
def density(s, psi):
    """rho(r) = sum_k w_k sum_n 2 |u_nk(r)|^2 for psi[nk, norb, nz, ny, nx] (Eq. rho)."""
    return 2.0 * np.einsum("k,kn...->...", np.asarray(s.kw, np.float64), np.abs(psi) ** 2)


def box_self_integral(ax, ay, az):
    """Integral of 1/|r| over the box [0,ax]x[0,ay]x[0,az] (closed form of the Newton potential
    of a uniform box at its corner)."""
    a, b, c = ax, ay, az
    d = math.sqrt(a * a + b * b + c * c)
    return (a * b * math.log((c + d) / math.hypot(a, b)) + b * c * math.log((a + d) / math.hypot(b, c))
            + c * a * math.log((b + d) / math.hypot(c, a))
            - 0.5 * a * a * math.atan(b * c / (a * d)) - 0.5 * b * b * math.atan(c * a / (b * d))
            - 0.5 * c * c * math.atan(a * b / (c * d)))


def hockney_kernel(s):
    """Green's function 1/|r| on the (2n)^3 zero-padding grid.  Index m maps to the distance
    m h for m <= n and (2n - m) h above.  The r = 0 cell takes the mean of 1/|r| over one grid
    cell: g(0) = 8 * box_self_integral(h/2) / dV."""
    comps = []
    for a in range(3):
        m = np.arange(2 * s.n[a])
        comps.append(np.where(m <= s.n[a], m, 2 * s.n[a] - m) * s.h[a])
    X, Y, Z = comps[0][None, None, :], comps[1][None, :, None], comps[2][:, None, None]
    r = np.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    with np.errstate(divide="ignore"):
        g = 1.0 / r
    g[0, 0, 0] = 8.0 * box_self_integral(s.h[0] / 2, s.h[1] / 2, s.h[2] / 2) / s.dV
    return g


def hartree(s, rho):
    """V_H = int rho(r')/|r - r'| (Eq. TDKS, e = 1).
    Periodic: V_H(G) = 4 pi rho(G) / G^2, V_H(G=0) = 0.
    Isolated: V_H(r_i) = dV sum_j g(r_i - r_j) rho_j, evaluated by FFT on the zero-padded grid."""
    if s.periodic:
        g = [2.0 * np.pi * np.fft.fftfreq(s.n[a], d=s.h[a]) for a in range(3)]
        G2 = g[0][None, None, :] ** 2 + g[1][None, :, None] ** 2 + g[2][:, None, None] ** 2
        rg = np.fft.fftn(rho)
        with np.errstate(divide="ignore", invalid="ignore"):
            vg = np.where(G2 == 0.0, 0.0, 4.0 * np.pi * rg / np.where(G2 == 0.0, 1.0, G2))
        return np.real(np.fft.ifftn(vg))
    nz, ny, nx = rho.shape
    pad = np.zeros((2 * nz, 2 * ny, 2 * nx))
    pad[:nz, :ny, :nx] = rho
    conv = np.fft.ifftn(np.fft.fftn(pad) * np.fft.fftn(hockney_kernel(s)))
    return np.real(conv[:nz, :ny, :nx]) * s.dV


def lda_x(rho):
    """Slater exchange (spin-unpolarised LDA exchange):
    eps_x = -(3/4) (3 rho / pi)^(1/3),  V_x = d(rho eps_x)/d rho = -(3 rho / pi)^(1/3)."""
    r = np.maximum(rho, 0.0)
    vx = -np.cbrt(3.0 * r / np.pi)
    return vx, 0.75 * vx


# Perdew-Zunger parametrisation of the correlation energy per electron of the unpolarised gas
# (the LDA named in Sec. 3.1): eps_c(r_s) in two branches joined at r_s = 1.
PZ_G, PZ_B1, PZ_B2 = -0.1423, 1.0529, 0.3334
PZ_A, PZ_B, PZ_C, PZ_D = 0.0311, -0.048, 0.0020, -0.0116


def pz_eps_c(rs):
    """eps_c(r_s) = g / (1 + b1 sqrt(r_s) + b2 r_s) for r_s >= 1, A ln r_s + B + C r_s ln r_s + D r_s below."""
    rs = np.asarray(rs, np.float64)
    hi = PZ_G / (1.0 + PZ_B1 * np.sqrt(rs) + PZ_B2 * rs)
    lo = PZ_A * np.log(rs) + PZ_B + PZ_C * rs * np.log(rs) + PZ_D * rs
    return np.where(rs >= 1.0, hi, lo)


def lda_c(rho):
    """Correlation potential and energy density per electron: r_s = (3 / (4 pi rho))^(1/3),
    V_c = d(rho eps_c)/d rho = eps_c - (r_s / 3) d eps_c / d r_s, with the derivative of each branch
    written out; both are 0 where rho <= 0."""
    r = np.asarray(rho, np.float64)
    pos = r > 1e-30
    rs = np.cbrt(3.0 / (4.0 * np.pi * np.where(pos, r, 1.0)))
    eps = pz_eps_c(rs)
    sq = np.sqrt(rs)
    den = 1.0 + PZ_B1 * sq + PZ_B2 * rs
    deps_hi = -PZ_G * (0.5 * PZ_B1 / sq + PZ_B2) / den ** 2
    deps_lo = PZ_A / rs + PZ_C * (np.log(rs) + 1.0) + PZ_D
    deps = np.where(rs >= 1.0, deps_hi, deps_lo)
    vc = eps - rs / 3.0 * deps
    return np.where(pos, vc, 0.0), np.where(pos, eps, 0.0)


# Tran-Blaha modified Becke-Johnson exchange potential (TB-mBJ; Sec. 4.1 names the BJ potential and
# its Tran-Blaha variant as options besides the LDA, without formulas).  The published forms
# (Becke-Roussel 1989, Becke-Johnson 2006, Tran-Blaha 2009) are restated per spin; the system is
# spin-unpolarised, so every per-spin density is half the total.  Parameters: gamma of the
# Becke-Roussel hole curvature, alpha and beta (bohr^1/2) of c = alpha + beta sqrt(g).
BR_GAMMA = 0.8
MBJ_ALPHA, MBJ_BETA = -0.012, 1.023
MBJ_RHO_MIN = 1e-10          # below this density the potential is set to zero (reading)


def kinetic_density(s, psi, Ap=None):
    """Kinetic energy density and paramagnetic current density of Bloch orbitals with
    q = k + A' (Ap None: A' = 0), spin-saturated (factor 2) with k-weights:
    tau = sum_k w_k sum_n 2 * 1/2 |(D1 + i q) u|^2,  j_a = sum_k w_k sum_n 2 Im(conj(u) (D1_a + i q_a) u),
    rho = sum_k w_k sum_n 2 |u|^2.  Returns (rho, tau, j[3])."""
    shape = psi.shape[-3:]
    rho, tau = np.zeros(shape), np.zeros(shape)
    j = np.zeros((3,) + shape)
    for ik in range(s.nk):
        q = np.asarray(s.kpts[ik], np.float64) + (np.zeros(3) if Ap is None else np.asarray(Ap, np.float64))
        w = 2.0 * s.kw[ik]
        u = psi[ik]
        rho += w * np.sum(np.abs(u) ** 2, axis=0)
        for a in range(3):
            g = d1(u, a, s) + 1j * q[a] * u
            tau += 0.5 * w * np.sum(np.abs(g) ** 2, axis=0)
            j[a] += w * np.sum(np.imag(np.conj(u) * g), axis=0)
    return rho, tau, j


def tau_tilde(s, psi, Ap=None):
    """tau - |j|^2 / (2 rho): the kinetic energy density with the current's share removed, the
    time-dependent kinetic energy density the adiabatic TB-mBJ potential uses (reading).  A uniform
    shift of q (any A') leaves it unchanged; it is >= 0 (Cauchy-Schwarz), 0 where rho = 0."""
    rho, tau, j = kinetic_density(s, psi, Ap)
    pos = rho > 0
    jj = np.sum(j ** 2, axis=0)
    return np.where(pos, np.maximum(tau - jj / (2.0 * np.where(pos, rho, 1.0)), 0.0), 0.0)


def br_x(y):
    """Root x of the Becke-Roussel equation x exp(-2x/3) / (x - 2) = y, elementwise.  The left side
    falls monotonically on (0, 2) (from 0 to -inf) and on (2, inf) (from +inf to 0), so y < 0 has
    its root in (0, 2), y > 0 in (2, inf), and y = +-inf gives x = 2."""
    from scipy.optimize import brentq
    y = np.asarray(y, np.float64)
    out = np.empty(y.shape)
    f = lambda x, yy: x * math.exp(-2.0 * x / 3.0) / (x - 2.0) - yy
    for i, yy in np.ndenumerate(y):
        if not np.isfinite(yy):
            out[i] = 2.0
        elif yy < 0:                              # f(0) = -y > 0
            hi = 2.0 - 1e-15
            out[i] = 2.0 if f(hi, yy) >= 0 else brentq(f, 0.0, hi, args=(yy,), xtol=1e-15, rtol=1e-15, maxiter=500)
        else:                                     # f(2+) = +inf, f(inf) = -y < 0
            lo, hi = 2.0 + 1e-15, 4.0
            while f(hi, yy) > 0:
                hi *= 2.0
            out[i] = 2.0 if f(lo, yy) <= 0 else brentq(f, lo, hi, args=(yy,), xtol=1e-15, rtol=1e-15, maxiter=500)
    return out


def br_potential(rho_s, grad2_s, lap_s, D_s, gamma=BR_GAMMA):
    """Becke-Roussel exchange potential of one spin channel: the exchange hole modelled as an
    exponential exp(-a |r' - r - b|) normalised to -1, with the hole's curvature at r fixed by
    Q = (lap rho - 2 gamma D) / 6, D = sum_i |grad psi_i|^2 - |grad rho|^2 / (4 rho) (the Fermi-hole
    curvature, zero for one orbital).  x = a b solves x exp(-2x/3)/(x-2) = (2/3) pi^(2/3) rho^(5/3) / Q,
    b = (x^3 exp(-x) / (8 pi rho))^(1/3), and the potential of the hole at its reference point is
    v = -(1/b) (1 - exp(-x) - x exp(-x) / 2).  Inputs per spin: rho, |grad rho|^2, lap rho, D."""
    rho_s = np.asarray(rho_s, np.float64)
    Q = (np.asarray(lap_s, np.float64) - 2.0 * gamma * np.asarray(D_s, np.float64)) / 6.0
    K = (2.0 / 3.0) * np.pi ** (2.0 / 3.0) * rho_s ** (5.0 / 3.0)
    with np.errstate(divide="ignore"):
        y = np.where(Q != 0, K / np.where(Q != 0, Q, 1.0), np.inf)
    x = br_x(y)
    b = np.cbrt(x ** 3 * np.exp(-x) / (8.0 * np.pi * rho_s))
    return -(1.0 - np.exp(-x) - 0.5 * x * np.exp(-x)) / b


def density_derivatives(s, rho):
    """|grad rho|^2 and lap rho with the orbitals' 8th-order differences (periodic wrap or zero
    outside the box)."""
    g2 = sum(d1(rho, a, s) ** 2 for a in range(3))
    return g2, sum(d2(rho, a, s) for a in range(3))


def mbj_c(s, rho):
    """c = alpha + beta sqrt(g), g = (1/Omega) int |grad rho| / rho over the cell (points with
    rho <= MBJ_RHO_MIN add nothing; reading)."""
    g2, _ = density_derivatives(s, rho)
    pos = rho > MBJ_RHO_MIN
    g = np.sum(np.where(pos, np.sqrt(g2) / np.where(pos, rho, 1.0), 0.0)) / rho.size
    return MBJ_ALPHA + MBJ_BETA * math.sqrt(g)


def mbj_x(s, rho, tau_t, c=None):
    """TB-mBJ exchange potential, spin-unpolarised:
    v_x = c v_BR + (3c - 2) (1/pi) sqrt(5/12) sqrt(2 t_s / rho_s) with rho_s = rho/2, t_s = tau_t/2
    (tau_t in the (1/2) sum |grad psi|^2 convention) and v_BR of the spin channel, whose D is
    2 t_s - |grad rho_s|^2 / (4 rho_s).  c None or <= 0: c from the density (mbj_c).  Zero where
    rho <= MBJ_RHO_MIN.  Returns (v_x, c)."""
    if c is None or c <= 0:
        c = mbj_c(s, rho)
    g2, lap = density_derivatives(s, rho)
    pos = rho > MBJ_RHO_MIN
    rs = np.where(pos, 0.5 * rho, 1.0)
    ts = np.where(pos, 0.5 * np.asarray(tau_t, np.float64), 0.0)
    gs2 = 0.25 * g2                               # |grad rho_s|^2
    D = 2.0 * ts - gs2 / (4.0 * rs)
    vbr = br_potential(rs, gs2, 0.5 * lap, D)
    v = c * vbr + (3.0 * c - 2.0) / np.pi * math.sqrt(5.0 / 12.0) * np.sqrt(2.0 * ts / rs)
    return np.where(pos, v, 0.0), c


def hxc(s, rho, hartree_on=True, xc_on=True, psi=None, mbj_c=None):
    """V_H + V_xc; xc_on: 0/False none, 1/True Slater exchange, 2 exchange + PZ correlation,
    3 TB-mBJ exchange + PZ correlation (needs the orbitals psi that rho comes from; mbj_c fixes c)."""
    v = np.zeros_like(rho)
    if hartree_on:
        v = v + hartree(s, rho)
    if xc_on and xc_on != 3:
        v = v + lda_x(rho)[0]
    if xc_on in (2, 3):
        v = v + lda_c(rho)[0]
    if xc_on == 3:
        if psi is None:
            raise ValueError("xc 3 (TB-mBJ) needs the orbitals")
        v = v + mbj_x(s, rho, tau_tilde(s, psi), mbj_c)[0]
    return v


# --------------------------------------------------------------------------------------------
# fields (Eq. pulse, Eq. impulsive_A)
# --------------------------------------------------------------------------------------------
def _pulse(A0, omega, T, cep, t):
    """One pulse of Eq. (pulse): Im{A0 cos^2[pi(t-T/2)/T] e^{-i omega (t-T/2) - 2 pi i cep}}, 0 < t < T."""
    if not (0.0 < t < T):
        return np.zeros(3)
    env = math.cos(math.pi * (t - T / 2.0) / T) ** 2
    ph = -omega * (t - T / 2.0) - 2.0 * math.pi * cep
    return np.asarray(A0, np.float64) * env * math.sin(ph)      # Im{A0 env e^{i ph}} for real A0


def field_Aprime(f, t):
    """A'(t) = A(t)/c as a 3-vector.  Sec. 3.1 fields: the impulsive step (Eq. impulsive_A), the
    pulse of Eq. (pulse) and successive delayed pulses (pump-probe, their sum), and a numerical
    table (samples of A' at t0 + i dt, linear in between, the end samples outside)."""
    A0 = np.asarray(f.A0, np.float64)
    if f.kind == "none":
        return np.zeros(3)
    if f.kind == "step":
        return A0.copy() if t > 0.0 else np.zeros(3)
    if f.kind == "pulse":
        a = _pulse(A0, f.omega, f.T, f.cep, t)
        for (A1, w1, T1, c1, delay) in getattr(f, "more", ()):
            a = a + _pulse(A1, w1, T1, c1, t - delay)
        return a
    if f.kind == "table":
        tab = np.asarray(f.table, np.float64).reshape(-1, 3)
        x = (t - f.t0) / f.dt_table
        if len(tab) == 1 or x <= 0.0:
            return tab[0].copy()
        if x >= len(tab) - 1:
            return tab[-1].copy()
        i = int(math.floor(x))
        w = x - i
        return (1.0 - w) * tab[i] + w * tab[i + 1]
    raise ValueError(f.kind)


# --------------------------------------------------------------------------------------------
# observables (Eq. macro_current, dipole, energy)
# --------------------------------------------------------------------------------------------
def current(s, tabs, psi, Ap):
    """Macroscopic current density (Eq. macro_current, e = m = 1):
    J_a = -(1/Omega) sum_k w_k sum_n 2 [ Re sum_r u^* (-i D1_a + q_a) u dV
                                        + sum_{atom,p} 2 E_p Im(conj(b_ap^(a)) c_ap) ],
    q = k + A'; c_ap = <p^q|u>, b_ap^(a) the same moment weighted by d_a.  The second term is
    <u| dV_NL^q / dq_a |u>, the nonlocal current."""
    J = np.zeros(3)
    for ik in range(s.nk):
        q = np.asarray(s.kpts[ik], np.float64) + np.asarray(Ap, np.float64)
        u = psi[ik]
        c = projections(s, tabs, q, u)
        for a in range(3):
            loc = np.real(np.sum(np.conj(u) * (-1j * d1(u, a, s) + q[a] * u))) * s.dV
            nl = 0.0
            if tabs:                                  # no atoms: no nonlocal current
                b = projections(s, tabs, q, u, weight_by=a)
                nl = np.sum(2.0 * np.array([t["E"] for t in tabs])[None] * np.imag(np.conj(b) * c))
            J[a] += s.kw[ik] * 2.0 * (loc + nl)
    return -J / cell_volume(s)


def dipole(s, rho, rho0):
    """d_mu = -int r_mu (rho - rho0) dr (Sec. 3.1, e = 1)."""
    x, y, z = coords(s)
    dr = rho - rho0
    return -np.array([np.sum(dr * x[None, None, :]), np.sum(dr * y[None, :, None]),
                      np.sum(dr * z[:, None, None])]) * s.dV


def band_energy(s, tabs, Vloc, psi, Ap):
    """sum_k w_k sum_n 2 <u| T_q + V_loc + V_NL^q |u>."""
    e = 0.0
    for ik in range(s.nk):
        q = np.asarray(s.kpts[ik], np.float64) + np.asarray(Ap, np.float64)
        hu = hpsi(s, tabs, Vloc, q, psi[ik])
        e += s.kw[ik] * 2.0 * np.real(np.sum(np.conj(psi[ik]) * hu)) * s.dV
    return e


def total_energy(s, tabs, Vloc, psi, Ap, hartree_on=True, xc_on=True):
    """E = band energy + 1/2 int rho V_H + int rho eps_xc (eps_x, plus eps_c when xc_on == 2)."""
    rho = density(s, psi)
    e = band_energy(s, tabs, Vloc, psi, Ap)
    if hartree_on:
        e += 0.5 * np.sum(rho * hartree(s, rho)) * s.dV
    if xc_on:
        e += np.sum(rho * lda_x(rho)[1]) * s.dV
    if xc_on == 2:
        e += np.sum(rho * lda_c(rho)[1]) * s.dV
    return e


def norms(s, psi):
    return (np.abs(psi) ** 2).sum(axis=(-3, -2, -1)) * s.dV


# --------------------------------------------------------------------------------------------
# time step (Taylor + predictor-corrector)
# --------------------------------------------------------------------------------------------
def propagate_all(s, tabs, V, psi, Ap, dt):
    out = np.empty_like(psi)
    for ik in range(s.nk):
        q = np.asarray(s.kpts[ik], np.float64) + np.asarray(Ap, np.float64)
        out[ik] = taylor4(s, tabs, V, q, psi[ik], dt)
    return out


def pc_step(s, tabs, Vloc, psi, vhxc, t, dt, pc=True, hartree_on=True, xc_on=True, Ap=None, mbj_c=None):
    """One step t -> t + dt.

    Predictor: psi~ = T4[V_loc + V_Hxc(t)] psi(t); V~ = V_Hxc[rho(psi~)].
    Corrector: psi(t+dt) = T4[V_loc + (V_Hxc(t) + V~)/2] psi(t); V_Hxc(t+dt) = V_Hxc[rho(t+dt)].
    Both stages use A'(t + dt/2) (from s.field, or the given Ap).  With pc=False the step is
    T4[V_loc + V_Hxc(t)] alone.  V_Hxc of xc_on = 3 (TB-mBJ) takes the kinetic energy density of
    the same orbitals as the density.  Returns (psi(t+dt), V_Hxc(t+dt), rho(t+dt))."""
    if Ap is None:
        Ap = field_Aprime(s.field, t + 0.5 * dt) if s.periodic else np.zeros(3)
    vmid = vhxc
    if pc:
        pred = propagate_all(s, tabs, Vloc + vhxc, psi, Ap, dt)
        vpred = hxc(s, density(s, pred), hartree_on, xc_on, pred, mbj_c)
        vmid = 0.5 * (vhxc + vpred)
    new = propagate_all(s, tabs, Vloc + vmid, psi, Ap, dt)
    rho = density(s, new)
    return new, hxc(s, rho, hartree_on, xc_on, new, mbj_c), rho


def misfit(vnew, vpred):
    """Self-consistency misfit of a predicted potential: ||V_Hxc(t+dt) - V~||_2 / ||V_Hxc(t+dt)||_2
    (the reading of the "density residual" that decides whether a predicted step is kept)."""
    return float(np.linalg.norm(vnew - vpred) / np.linalg.norm(vnew))


def predicted_step(s, tabs, Vloc, psi, vhxc, vpred, t, dt, threshold, hartree_on=True, xc_on=True,
                   Ap=None, mbj_c=None):
    """One step with a predicted potential V~(t+dt) in place of the predictor half-step of the
    predictor-corrector scheme (Program summary):

        corrector  psi(t+dt) = T4[V_loc + (V_Hxc(t) + V~)/2] psi(t),  A'(t + dt/2),
                   V_Hxc(t+dt) = V_Hxc[rho(t+dt)],
        misfit     r = ||V_Hxc(t+dt) - V~|| / ||V_Hxc(t+dt)||.

    If r exceeds the threshold (or is not finite) the step is discarded and redone from psi(t) by
    the plain predictor-corrector step, which also supplies the returned misfit of its own
    predictor.  Returns (psi(t+dt), V_Hxc(t+dt), rho(t+dt), r of the predicted V~, accepted)."""
    if Ap is None:
        Ap = field_Aprime(s.field, t + 0.5 * dt) if s.periodic else np.zeros(3)
    new = propagate_all(s, tabs, Vloc + 0.5 * (vhxc + vpred), psi, Ap, dt)
    rho = density(s, new)
    vnew = hxc(s, rho, hartree_on, xc_on, new, mbj_c)
    r = misfit(vnew, vpred)
    if np.isfinite(r) and r <= threshold:
        return new, vnew, rho, r, True
    new, vnew, rho = pc_step(s, tabs, Vloc, psi, vhxc, t, dt, True, hartree_on, xc_on, Ap, mbj_c)
    return new, vnew, rho, r, False


def run_predicted(s, psi0, nsteps, predictor, threshold, hartree_on=True, xc_on=True, t0=0.0, mbj_c=None):
    """Propagate nsteps with predicted steps.  The history holds the last four V_Hxc (starting from
    V_Hxc[rho(psi0)]); while it has fewer than four the step is the plain predictor-corrector step.
    predictor(V0, V1, V2, V3) -> V~(t+dt) from V_Hxc(t), V_Hxc(t-dt), V_Hxc(t-2dt), V_Hxc(t-3dt).
    Returns the final psi, V_Hxc and per-step records: t, J(t+dt) (with A'(t+dt)), dipole of
    rho(t+dt), the misfit of the prediction (nan for plain steps) and the number of rejected
    predictions."""
    tabs = projector_tables(s)
    Vloc = local_potential(s)
    psi = psi0.copy()
    rho0 = density(s, psi)
    vhxc = hxc(s, rho0, hartree_on, xc_on, psi, mbj_c)
    hist = [vhxc]
    rec = dict(t=[], J=[], d=[], misfit=[])
    rejected = 0
    t = t0
    for _ in range(nsteps):
        if len(hist) >= 4:
            vpred = predictor(hist[-1], hist[-2], hist[-3], hist[-4])
            psi, vhxc, rho, r, ok = predicted_step(s, tabs, Vloc, psi, vhxc, vpred, t, s.dt, threshold,
                                                   hartree_on, xc_on, mbj_c=mbj_c)
            rejected += 0 if ok else 1
        else:
            psi, vhxc, rho = pc_step(s, tabs, Vloc, psi, vhxc, t, s.dt, True, hartree_on, xc_on, mbj_c=mbj_c)
            r = np.nan
        hist = (hist + [vhxc])[-4:]
        t += s.dt
        Ap = field_Aprime(s.field, t) if s.periodic else np.zeros(3)
        rec["t"].append(t)
        rec["J"].append(current(s, tabs, psi, Ap) if s.periodic else np.zeros(3))
        rec["d"].append(dipole(s, rho, rho0))
        rec["misfit"].append(r)
    out = {k: np.array(v) for k, v in rec.items()}
    out["rejected"] = rejected
    return psi, vhxc, out


def apply_kick(s, psi, kappa):
    """Isolated impulse (Sec. 3.1): psi(0+) = exp(i kappa . r) phi."""
    x, y, z = coords(s)
    ph = np.exp(1j * (kappa[0] * x[None, None, :] + kappa[1] * y[None, :, None]
                      + kappa[2] * z[:, None, None]))
    return psi * ph


def run(s, psi0, nsteps, pc=True, hartree_on=True, xc_on=True, record=True, mbj_c=None):
    """Propagate nsteps; returns final psi and per-step observables (t, J, dipole)."""
    tabs = projector_tables(s)
    Vloc = local_potential(s)
    psi = psi0.copy()
    rho0 = density(s, psi)
    vhxc = hxc(s, rho0, hartree_on, xc_on, psi, mbj_c)
    hist = dict(t=[], J=[], d=[])
    t = 0.0
    for _ in range(nsteps):
        psi, vhxc, rho = pc_step(s, tabs, Vloc, psi, vhxc, t, s.dt, pc, hartree_on, xc_on, mbj_c=mbj_c)
        t += s.dt
        if record:
            hist["t"].append(t)
            Ap = field_Aprime(s.field, t) if s.periodic else np.zeros(3)
            hist["J"].append(current(s, tabs, psi, Ap) if s.periodic else np.zeros(3))
            hist["d"].append(dipole(s, rho, rho0))
    return psi, vhxc, {k: np.array(v) for k, v in hist.items()}


# --------------------------------------------------------------------------------------------
# analysis: Eq. (distribution), Eq. (sigma_ft), Eq. (Maxwell_ms)
# --------------------------------------------------------------------------------------------
def oscillator_strength(t, d, kappa, energies):
    """df/dE = -(2E/(pi kappa)) Im int_0^T f(t/T) d(t) exp(iEt) dt, f(x) = 1 - 3x^2 + 2x^3.
    The kick exp(i kappa z) corresponds to F0 = -kappa in Eq. (distribution); the sign makes the
    spectrum positive and its integral the electron count (f-sum)."""
    t = np.asarray(t, np.float64)
    d = np.asarray(d, np.float64)
    T = t[-1]
    dt = t[1] - t[0]
    x = t / T
    f = 1.0 - 3.0 * x ** 2 + 2.0 * x ** 3
    E = np.asarray(energies, np.float64)
    integ = (f * d)[None, :] * np.exp(1j * E[:, None] * t[None, :])
    return -(2.0 * E / (np.pi * kappa)) * np.imag(integ.sum(axis=1) * dt)


def masked_transform(t, x, omegas, subtract_mean=False):
    """F(w) = dt sum_i f(t_i/T) (x_i - xbar) exp(i w t_i), f(s) = 1 - 3s^2 + 2s^3, T = t[-1]: the
    rectangle-rule form of the masked integrals of Eq. (distribution) and Eq. (sigma_ft).  With
    subtract_mean, xbar = sum f x / sum f (the mean whose removal makes F(0) = 0, as the Sec. 4.1
    example requires of sigma), else 0."""
    t = np.asarray(t, np.float64)
    x = np.asarray(x, np.float64)
    T = t[-1]
    dt = t[1] - t[0]
    s = t / T
    f = 1.0 - 3.0 * s ** 2 + 2.0 * s ** 3
    xbar = np.sum(f * x) / np.sum(f) if subtract_mean else 0.0
    w = np.asarray(omegas, np.float64)
    return ((f * (x - xbar))[None, :] * np.exp(1j * w[:, None] * t[None, :])).sum(axis=1) * dt


def conductivity(t, I, Ap0, omegas, subtract_mean=True):
    """Eq. (sigma_ft): sigma(w) = -(c / A0) int_0^T e^{iwt} f(t/T) I(t) dt for a vector-potential step
    A(t) = A0 theta(t); with A' = A/c the prefactor is -1/A'0.  Returns complex sigma."""
    return -masked_transform(t, I, omegas, subtract_mean) / Ap0


def dielectric(omegas, sigma):
    """Sec. 4.1: eps(w) = 1 + 4 pi i sigma(w) / w."""
    return 1.0 + 4.0 * np.pi * 1j * np.asarray(sigma) / np.asarray(omegas, np.float64)


def dense_hamiltonian(s, tabs, V, q):
    """H_q as a dense npts x npts matrix, column j = hpsi of the j-th unit vector (tiny grids only)."""
    N = s.npts
    H = np.zeros((N, N), np.complex128)
    for j in range(N):
        e = np.zeros(N, np.complex128)
        e[j] = 1.0
        H[:, j] = hpsi(s, tabs, V, q, e.reshape(s.n[2], s.n[1], s.n[0])).ravel()
    return H


def ground_state(s, hartree_on=True, xc_on=True, mix=0.3, tol=1e-10, max_iter=400, mbj_c=None):
    """Self-consistent ground state at A' = 0 (the static Kohn-Sham problem the paper's ground-state
    step solves before the time evolution): diagonalise H_k[V_loc + V_Hxc] densely for every k,
    occupy the lowest norb states (each normalised to sum |u|^2 dV = 1), form rho and V_Hxc[rho], and
    mix the potential linearly, V_in <- V_in + mix (V_out - V_in), until ||V_out - V_in|| / ||V_out||
    < tol.  Returns (psi [nk][norb][nz][ny][nx], eigenvalues [nk][norb], V_Hxc, iterations)."""
    tabs = projector_tables(s)
    Vloc = local_potential(s)
    shape = (s.n[2], s.n[1], s.n[0])
    zero = np.zeros(shape)
    # the potential enters H_k only on the diagonal: build the rest once per k
    H0 = [dense_hamiltonian(s, tabs, zero, np.asarray(s.kpts[k], np.float64)) for k in range(s.nk)]
    vin = np.zeros(shape)
    for it in range(1, max_iter + 1):
        psi = np.zeros((s.nk, s.norb) + shape, np.complex128)
        eig = np.zeros((s.nk, s.norb))
        for k in range(s.nk):
            E, U = np.linalg.eigh(H0[k] + np.diag((Vloc + vin).ravel()))
            eig[k] = E[:s.norb]
            psi[k] = (U[:, :s.norb].T / math.sqrt(s.dV)).reshape((s.norb,) + shape)
        vout = hxc(s, density(s, psi), hartree_on, xc_on, psi, mbj_c)
        err = np.linalg.norm(vout - vin) / max(np.linalg.norm(vout), 1e-300)
        if err < tol:
            return psi, eig, vout, it
        vin = vin + mix * (vout - vin)
    return psi, eig, vout, max_iter


def orbital_energies(s, tabs, V, psi, Ap=None):
    """Orbital energies of the ground-state outputs (Sec. 2.1: discrete orbital energies of isolated
    systems, energy bands of periodic ones): the Ritz values of H_q, q = k + A' (Ap None: A' = 0), in
    the span of each k's orbitals -- the eigenvalues of M z = e S z with M_ij = <u_i|H_q|u_j>,
    S_ij = <u_i|u_j> -- ascending, [nk][norb], and the Ritz vectors (the orbitals rotated into
    S-orthonormal eigenvectors of the projected problem).  For eigenvectors of H_q the Ritz values are
    their eigenvalues.  scipy.linalg.eigh solves the small generalised problem."""
    from scipy.linalg import eigh
    eps = np.zeros((s.nk, s.norb))
    rot = np.empty_like(psi)
    for ik in range(s.nk):
        q = np.asarray(s.kpts[ik], np.float64) + (np.zeros(3) if Ap is None else np.asarray(Ap, np.float64))
        U = psi[ik].reshape(s.norb, -1)
        HU = hpsi(s, tabs, V, q, psi[ik]).reshape(s.norb, -1)
        M = U.conj() @ HU.T * s.dV
        S = U.conj() @ U.T * s.dV
        e, Z = eigh(0.5 * (M + M.conj().T), 0.5 * (S + S.conj().T))
        eps[ik] = e
        rot[ik] = (Z.T @ U).reshape(psi[ik].shape)
    return eps, rot


def dos(eps, kw, E, sigma):
    """Density of states (Sec. 2.1 ground-state outputs), spin-saturated, with a Gaussian of width
    sigma for every level: D(E) = sum_k w_k sum_n 2 exp(-(E - e_nk)^2 / (2 sigma^2)) / (sigma sqrt(2 pi))."""
    E = np.asarray(E, np.float64)
    out = np.zeros_like(E)
    for ik in range(len(kw)):
        for e in np.asarray(eps[ik], np.float64):
            out += 2.0 * kw[ik] * np.exp(-0.5 * ((E - e) / sigma) ** 2) / (sigma * math.sqrt(2.0 * np.pi))
    return out


def excited_pairs(s, psi, psi_gs):
    """Number density of excited electron-hole pairs: (1/Omega) sum_k w_k 2 (norb - sum_{m,n}
    |<phi_km|psi_kn>|^2), the occupied weight outside the ground-state subspace."""
    n = 0.0
    for k in range(s.nk):
        O_ = psi_gs[k].reshape(s.norb, -1).conj() @ psi[k].reshape(s.norb, -1).T * s.dV
        n += 2.0 * s.kw[k] * (s.norb - np.sum(np.abs(O_) ** 2))
    return n / cell_volume(s)


def longitudinal_run(s, psi0, nsteps, t0=0.0, hartree_on=True, xc_on=True):
    """Longitudinal geometry (Sec. 4.1, thin film): A'(t) = A'_ext(t) + A'_ind(t) with
    d^2 A'_ind/dt^2 = 4 pi J(t) (E_ind = -4 pi P, dP/dt = J, E = -dA'/dt).  Per step:
    A^{n+1} = 2 A^n - A^{n-1} + 4 pi dt^2 J(t_n) (first step from rest, A^1 = 2 pi dt^2 J(t_0)), the
    predictor-corrector step with A'_ext(t + dt/2) + (A^n + A^{n+1})/2, and J(t + dt) with
    A'_ext(t + dt) + A^{n+1}.  Returns the orbitals and per-step records of J and A'_ind."""
    tabs = projector_tables(s)
    Vloc = local_potential(s)
    psi = psi0.copy()
    vhxc = hxc(s, density(s, psi), hartree_on, xc_on, psi)
    t = t0
    J = current(s, tabs, psi, field_Aprime(s.field, t))
    A_now, A_prev = np.zeros(3), None
    hist = dict(J=[], A_ind=[])
    for _ in range(nsteps):
        src = 4.0 * np.pi * s.dt ** 2 * J
        A_next = A_now + 0.5 * src if A_prev is None else 2.0 * A_now - A_prev + src
        Amid = field_Aprime(s.field, t + 0.5 * s.dt) + 0.5 * (A_now + A_next)
        psi, vhxc, _ = pc_step(s, tabs, Vloc, psi, vhxc, t, s.dt, True, hartree_on, xc_on, Ap=Amid)
        t += s.dt
        A_prev, A_now = A_now, A_next
        J = current(s, tabs, psi, field_Aprime(s.field, t) + A_now)
        hist["J"].append(J)
        hist["A_ind"].append(A_now.copy())
    return psi, {k: np.array(v) for k, v in hist.items()}


def field_E(f, t):
    """E(t) = -dA'/dt of field_Aprime: the pulse (and pulse trains) differentiated in closed form,
    tables by their piecewise slope (the mean of both sides at a sample), a step gives 0 for t != 0."""
    if f.kind in ("none", "step"):
        return np.zeros(3)
    if f.kind == "pulse":
        def dpulse(A0, omega, T, cep, tt):
            if not (0.0 < tt < T):
                return np.zeros(3)
            x = math.pi * (tt - T / 2.0) / T
            ph = -omega * (tt - T / 2.0) - 2.0 * math.pi * cep
            env = math.cos(x) ** 2
            denv = -2.0 * math.cos(x) * math.sin(x) * math.pi / T
            return np.asarray(A0, np.float64) * (denv * math.sin(ph) - env * omega * math.cos(ph))
        g = dpulse(f.A0, f.omega, f.T, f.cep, t)
        for (A1, w1, T1, c1, delay) in getattr(f, "more", ()):
            g = g + dpulse(A1, w1, T1, c1, t - delay)
        return -g
    if f.kind == "table":
        tab = np.asarray(f.table, np.float64).reshape(-1, 3)
        x = (t - f.t0) / f.dt_table
        if len(tab) == 1 or x < 0.0 or x > len(tab) - 1:
            return np.zeros(3)
        i = int(math.floor(x))
        if x == i:                                    # at a sample: mean of the two slopes
            lo = (tab[i] - tab[i - 1]) / f.dt_table if i > 0 else None
            hi = (tab[i + 1] - tab[i]) / f.dt_table if i + 1 < len(tab) else None
            sl = [v for v in (lo, hi) if v is not None]
            return -sum(sl) / len(sl)
        return -(tab[i + 1] - tab[i]) / f.dt_table
    raise ValueError(f.kind)


def work(t, J, E):
    """Sec. 4.1: W(t) = int_0^t I.E dt' per unit volume by the trapezoid rule on the samples; with I
    of Eq. (macro_current) and E = -dA'/dt this is (E_el(t) - E_el(0)) / Omega for an LDA energy
    functional (the sign that makes the field's work on the electrons positive)."""
    t = np.asarray(t, np.float64)
    g = np.sum(np.asarray(J, np.float64) * np.asarray(E, np.float64), axis=1)
    return np.concatenate([[0.0], np.cumsum(0.5 * (g[1:] + g[:-1]) * np.diff(t))])


def mur_boundary(A_next, A_now, c_dt_dX):
    """First-order Mur absorbing boundary at both ends of the 1D grid (waves leave the box):
    A_0^{n+1} = A_1^n + k (A_1^{n+1} - A_0^n), k = (c dt - dX)/(c dt + dX), mirrored at the right end."""
    k = (c_dt_dX - 1.0) / (c_dt_dX + 1.0)
    A_next[0] = A_now[1] + k * (A_next[1] - A_now[0])
    A_next[-1] = A_now[-2] + k * (A_next[-2] - A_now[-1])
    return A_next


def maxwell_step(A_now, A_prev, I, c_dt_dX, dt, c=C_LIGHT):
    """Leapfrog update of Eq. (Maxwell_ms), (1/c^2) A_tt - A_XX = (4 pi / c) I, interior points:
    A^{n+1}_X = 2A^n_X - A^{n-1}_X + (c dt/dX)^2 (A_{X+1} - 2A_X + A_{X-1}) + 4 pi c dt^2 I_X.
    End points are held (the caller supplies its own boundary)."""
    A_next = A_now.copy()
    lap = A_now[2:] - 2.0 * A_now[1:-1] + A_now[:-2]
    A_next[1:-1] = 2.0 * A_now[1:-1] - A_prev[1:-1] + c_dt_dX ** 2 * lap + 4.0 * np.pi * c * dt * dt * I[1:-1]
    return A_next


def multiscale_step(s, tabs, Vloc, cells, A_now, A_prev, I, m0, dX, t, dt, c=C_LIGHT):
    """One step of the coupled system (Sec. 5): Eq. (Maxwell_ms) by leapfrog with the cell currents
    I(X, t) and Mur boundaries gives A(X, t+dt); every microscopic cell X = m0 + j then takes one
    predictor-corrector step of Eq. (TDKS_ms) with A'(t+dt/2) = (A(X,t) + A(X,t+dt))/(2c) along z,
    and its current at t+dt (Eq. macro_current, with A'(t+dt)) becomes I(X, t+dt).
    cells: list of (psi, vhxc) per material point; returns (cells, A_next, A_now, I_next)."""
    c_dt_dX = c * dt / dX
    A_next = mur_boundary(maxwell_step(A_now, A_prev, I, c_dt_dX, dt, c), A_now, c_dt_dX)
    I_next = np.zeros_like(I)
    out = []
    for j, (psi, vhxc) in enumerate(cells):
        X = m0 + j
        Amid = np.array([0.0, 0.0, 0.5 * (A_now[X] + A_next[X]) / c])
        psi, vhxc, _ = pc_step(s, tabs, Vloc, psi, vhxc, t, dt, Ap=Amid)
        I_next[X] = current(s, tabs, psi, np.array([0.0, 0.0, A_next[X] / c]))[2]
        out.append((psi, vhxc))
    return out, A_next, A_now, I_next
