"""Pins of the oracle's TB-mBJ exchange potential (Sec. 4.1 names the Becke-Johnson potential and its
Tran-Blaha variant besides the LDA) against closed forms, brute force and invariants (CPU only).

Each test names the part it pins and the mistake it would catch."""
import math

import numpy as np

from oracle import tdks_oracle as O
from paper_1804_01404_gb300 import workloads as W


def _periodic(n, h):
    s = W.tiny(periodic=True, n=n, natom=0, nk=1, norb=1)
    s.h = h
    s.kpts = np.zeros((1, 3))
    s.kw = np.ones(1)
    return s


def test_becke_roussel_hydrogen():
    """The Becke-Roussel hole is exact for the hydrogen atom: for rho = exp(-2r)/pi (one spin, one
    orbital, D = 0) the hole is the whole density centred on the nucleus, and the potential equals
    minus its Hartree potential, -(1 - exp(-2r)(1 + r))/r.  A wrong constant in the root equation,
    in b or in the potential fails this."""
    r = np.linspace(0.05, 8.0, 80)
    rho = np.exp(-2 * r) / np.pi
    v = O.br_potential(rho, 4 * rho ** 2, rho * (4 - 4 / r), np.zeros_like(r))
    exact = -(1 - np.exp(-2 * r) * (1 + r)) / r
    assert np.max(np.abs(v - exact) / np.abs(exact)) < 1e-12


def test_becke_roussel_root_by_brute_force():
    """br_x against a sign change of x exp(-2x/3)/(x-2) - y located on a dense grid of x, on both
    branches (y < 0: x in (0, 2); y > 0: x in (2, inf)); y = inf gives 2."""
    xs = np.concatenate([np.linspace(1e-6, 2 - 1e-9, 400001), np.linspace(2 + 1e-9, 60, 400001)])
    G = xs * np.exp(-2 * xs / 3) / (xs - 2)
    for y in (-40.0, -1.3, -0.2, -1e-3, 1e-3, 0.2, 1.3, 40.0):
        f = G - y
        i = np.nonzero((f[:-1] > 0) & (f[1:] <= 0))[0]
        assert len(i) == 1, y                          # one root: the left side is monotonic per branch
        x = O.br_x(np.array([y]))[0]
        assert xs[i[0]] - 1e-4 <= x <= xs[i[0] + 1] + 1e-4, (y, x, xs[i[0]])
        assert (x < 2) == (y < 0)
    assert O.br_x(np.array([np.inf]))[0] == 2.0


def test_kinetic_density_of_a_plane_wave():
    """u = exp(iG.r)/sqrt(Omega): D1 u = i s(G) u with the stencil's symbol s_a = (2/h_a) sum_m d_m
    sin(m G_a h_a), so tau = (1/2)|s + q|^2 rho and j = (s + q) rho with rho = 2/Omega, and the
    current-free part tau - |j|^2/(2 rho) vanishes.  Pins the factor 1/2, the occupation 2, the sign
    of q in the derivative and the current's share."""
    n, h = (8, 9, 10), (0.5, 0.45, 0.4)
    s = _periodic(n, h)
    x, y, z = O.coords(s)
    L = [n[a] * h[a] for a in range(3)]
    G = [2 * np.pi * 2 / L[0], -2 * np.pi / L[1], 2 * np.pi * 3 / L[2]]
    Om = O.cell_volume(s)
    u = np.exp(1j * (G[0] * x[None, None, :] + G[1] * y[None, :, None] + G[2] * z[:, None, None])) / math.sqrt(Om)
    psi = u[None, None]
    Ap = np.array([0.11, -0.07, 0.05])
    sym = np.array([2.0 / h[a] * sum(O.FD1[m - 1] * math.sin(m * G[a] * h[a]) for m in range(1, 5)) for a in range(3)])
    qs = sym + Ap
    rho, tau, j = O.kinetic_density(s, psi, Ap)
    assert np.allclose(rho, 2 / Om, rtol=1e-13)
    assert np.allclose(tau, 0.5 * np.dot(qs, qs) * 2 / Om, rtol=1e-12)
    for a in range(3):
        assert np.allclose(j[a], qs[a] * 2 / Om, rtol=1e-12, atol=1e-15)
    assert np.max(np.abs(O.tau_tilde(s, psi, Ap))) < 1e-13 * np.max(tau)


def test_tau_tilde_single_orbital_is_the_weizsacker_form():
    """For one orbital u = A exp(i phi), tau - |j|^2/(2 rho) = w |grad A|^2 (= |grad rho|^2/(8 rho)):
    the phase drops out only if tau, j and rho carry consistent factors.  A and phi are smooth and
    periodic, the comparison is with their analytic gradients (the 8th-order differences of the
    oscillating phase leave ~3e-5 of the maximum)."""
    n, h = (32, 30, 28), (0.25, 0.27, 0.29)
    s = _periodic(n, h)
    x, y, z = O.coords(s)
    L = [n[a] * h[a] for a in range(3)]
    X, Y, Z = np.meshgrid(x, y, z, indexing="xy")
    X, Y, Z = (np.transpose(v, (2, 0, 1)) for v in (X, Y, Z))     # [z, y, x]
    kx, ky, kz = (2 * np.pi / L[a] for a in range(3))
    A = np.exp(0.4 * np.cos(kx * X) + 0.3 * np.sin(ky * Y) + 0.2 * np.cos(kz * Z))
    phi = 0.7 * np.sin(kx * X + ky * Y) + 0.5 * np.cos(kz * Z)
    gA = [A * (-0.4 * kx * np.sin(kx * X)), A * (0.3 * ky * np.cos(ky * Y)), A * (-0.2 * kz * np.sin(kz * Z))]
    psi = (A * np.exp(1j * phi))[None, None]
    tt = O.tau_tilde(s, psi, Ap=(0.2, -0.1, 0.3))
    exact = sum(g ** 2 for g in gA)                    # w = 1, one k
    assert np.max(np.abs(tt - exact)) < 1e-4 * np.max(exact)


def test_tau_tilde_gauge_invariance():
    """A uniform A' shifts every q: tau changes, tau - |j|^2/(2 rho) does not (several k-points and
    orbitals, random smooth orbitals)."""
    s = W.tiny(periodic=True, n=(6, 7, 8), natom=1, nk=3, norb=2)
    psi = W.initial_orbitals(s, 2)
    _, t0, _ = O.kinetic_density(s, psi)
    _, t1, _ = O.kinetic_density(s, psi, (0.3, -0.2, 0.5))
    assert np.max(np.abs(t1 - t0)) > 1e-3 * np.max(t0)
    a, b = O.tau_tilde(s, psi), O.tau_tilde(s, psi, (0.3, -0.2, 0.5))
    assert np.max(np.abs(a - b)) < 1e-12 * np.max(a)
    assert np.min(a) >= 0.0


def test_mbj_c_closed_form():
    """rho = rho0 exp(a cos(2 pi x / Lx)): |grad rho|/rho = a (2 pi/Lx) |sin(2 pi x/Lx)|, whose mean over
    the N grid points is a (2 pi/Lx) (2/N) cot(pi/N) (-> 4a/Lx as N grows; the kinks of |sin| make the
    grid mean differ from the integral by O(N^-2)), so c = alpha + beta sqrt(g) with alpha = -0.012,
    beta = 1.023."""
    n, h = (40, 6, 6), (0.2, 0.5, 0.5)
    s = _periodic(n, h)
    x, _, _ = O.coords(s)
    Lx = n[0] * h[0]
    a = 0.6
    rho = 0.05 * np.exp(a * np.cos(2 * np.pi * x / Lx))[None, None, :] * np.ones((n[2], n[1], 1))
    c = O.mbj_c(s, rho)
    g = a * (2 * np.pi / Lx) * (2.0 / n[0]) / math.tan(np.pi / n[0])
    assert abs(c - (-0.012 + 1.023 * math.sqrt(g))) < 1e-7           # the differences of rho: ~1e-8
    assert abs(g - 4 * a / Lx) < 3e-3 * g


def test_mbj_uniform_gas_correction_term():
    """Uniform gas (tau = (3/10)(3 pi^2)^(2/3) rho^(5/3), no gradients): v(c=1) - (3/2) v(c=2/3)
    leaves only the Becke-Johnson correction (1/pi) sqrt(5/12) sqrt(2 t_s/rho_s), which for the
    uniform gas is k_F,s/(2 pi), k_F,s = (6 pi^2 rho/2)^(1/3).  Pins the (3c - 2) factor, the spin
    halving of rho and tau and the constants of the correction."""
    s = _periodic((6, 6, 6), (0.5, 0.5, 0.5))
    for rho0 in (0.003, 0.08, 1.7):
        rho = np.full((6, 6, 6), rho0)
        tau = np.full((6, 6, 6), 0.3 * (3 * np.pi ** 2) ** (2 / 3) * rho0 ** (5 / 3))
        v1, _ = O.mbj_x(s, rho, tau, 1.0)
        v23, _ = O.mbj_x(s, rho, tau, 2.0 / 3.0)
        kfs = (6 * np.pi ** 2 * rho0 / 2) ** (1 / 3)
        assert np.allclose(v1 - 1.5 * v23, kfs / (2 * np.pi), rtol=1e-12)
        assert np.all(v23 < 0)


def test_mbj_two_electron_exponential_is_the_hydrogen_form():
    """Two electrons in one exponential orbital, phi^2 = Z^3 exp(-2 Z r)/pi per spin (rho = 2 phi^2,
    tau = |grad phi|^2): each spin channel is a one-orbital hydrogen-like density, D = 0, so with
    c = 2/3 (no correction term) mbj_x = (2/3) v_BR = -(2/3)(1 - exp(-2Zr)(1 + Zr))/r, with the
    derivatives of rho taken by the grid's differences (isolated box, compared away from the cusp).
    Pins the spin halving of rho, grad rho and lap rho and the D of mbj_x."""
    Z, nn, hh = 1.3, 41, 0.1
    s = W.tiny(periodic=False, n=(nn, nn, nn), natom=0, nk=1, norb=1)
    s.h = (hh, hh, hh)
    x, y, z = O.coords(s)
    r = np.sqrt(x[None, None, :] ** 2 + y[None, :, None] ** 2 + z[:, None, None] ** 2)
    phi2 = Z ** 3 * np.exp(-2 * Z * r) / np.pi
    rho = 2 * phi2
    tau = Z ** 2 * phi2                                   # |grad phi|^2 with phi = sqrt(phi2)
    v, _ = O.mbj_x(s, rho, tau, 2.0 / 3.0)
    exact = -(2.0 / 3.0) * (1 - np.exp(-2 * Z * r) * (1 + Z * r)) / np.where(r > 0, r, 1)
    sel = (r > 0.6) & (r < 1.4)
    assert sel.sum() > 1000
    assert np.max(np.abs(v[sel] - exact[sel]) / np.abs(exact[sel])) < 2e-4


def test_mbj_of_a_plane_wave_is_the_x2_closed_form():
    """One plane-wave orbital: rho is uniform (no gradient or Laplacian on the grid) and
    tau - |j|^2/(2 rho) = 0, so D = Q = 0, the Becke-Roussel root is x = 2 (the limit of the equation
    at Q -> 0), b = (8 e^-2 / (8 pi rho_s))^(1/3), the correction term vanishes and g = 0 gives
    c = alpha.  End to end through hxc: V_x = c v_BR = -alpha (1 - 2 e^-2) (pi e^2 rho_s)^(1/3).  The
    square roots of g and of t_s lift the rounding of the vanishing terms (~1e-16) to ~1e-8, which
    sets the tolerances."""
    n, h = (8, 9, 10), (0.5, 0.45, 0.4)
    s = _periodic(n, h)
    x, y, z = O.coords(s)
    L = [n[a] * h[a] for a in range(3)]
    G = [2 * np.pi / L[0], 2 * np.pi * 2 / L[1], 0.0]
    u = np.exp(1j * (G[0] * x[None, None, :] + G[1] * y[None, :, None] + G[2] * z[:, None, None]))
    u /= math.sqrt(O.cell_volume(s))
    psi = u[None, None]
    rho = O.density(s, psi)
    v = O.hxc(s, rho, False, 3, psi) - O.lda_c(rho)[0]
    rs = rho.mean() / 2
    vbr = -(1 - 2 * math.exp(-2.0)) * (math.pi * math.e ** 2 * rs) ** (1 / 3)
    assert abs(O.mbj_c(s, rho) - (-0.012)) < 1e-7
    assert np.allclose(v, -0.012 * vbr, rtol=1e-5, atol=0)
