"""Response analysis on the GPU (tdks_oscillator_strength, tdks_conductivity) against the oracle.

* The transforms themselves: the GPU results of Eq. (distribution) and Eq. (sigma_ft) on fixed
  series equal the oracle's to 1e-10 relative.
* The absorption-peak criterion: a kicked isolated system propagated with FP32 orbitals on the GPU
  (plain predictor-corrector and the extrapolated predictor) gives a dipole spectrum whose main
  peak lies within 0.01 eV of the peak of the FP64 oracle's own propagation.  The spectral
  resolution of the short run (2 pi / T) is much coarser; 0.01 eV is a precision criterion.
* The dielectric function of a periodic cell after the A' step (velocity-gauge kick): from the
  GPU's FP64 and FP32 current histories against the oracle's.
"""
import numpy as np
import pytest

from oracle import tdks_oracle as O
from paper_1804_01404_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

EV = 27.211386245988


def _rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / np.max(np.abs(np.asarray(b))))


def test_oscillator_strength_matches_oracle():
    from paper_1804_01404_gb300 import tdks as T
    dt, kappa = 0.02, 1e-3
    t = np.arange(0, 4001) * dt
    d = -(2 * kappa / 0.4) * np.sin(0.4 * t) + 3e-4 * np.sin(1.3 * t) * np.exp(-0.01 * t)
    E = np.linspace(0.0, 2.0, 1201)
    got = T.oscillator_strength(d, dt, kappa, E)
    ref = O.oscillator_strength(t, d, kappa, E)
    assert _rel(got, ref) < 1e-10


@pytest.mark.parametrize("subtract_mean", [False, True])
def test_conductivity_matches_oracle(subtract_mean):
    from paper_1804_01404_gb300 import tdks as T
    rng = np.random.default_rng(7)
    dt, Ap0 = 0.02, 1e-3
    t = np.arange(0, 2501) * dt
    I = 0.02 + 1e-3 * np.sin(0.55 * t) + 1e-4 * rng.standard_normal(len(t))
    w = np.linspace(0.05, 1.5, 301)
    sig, eps = T.conductivity(I, dt, Ap0, w, subtract_mean=subtract_mean)
    sref = O.conductivity(t, I, Ap0, w, subtract_mean=subtract_mean)
    assert _rel(sig, sref) < 1e-10
    assert _rel(eps, O.dielectric(w, sref)) < 1e-10
    sig0, eps0 = T.conductivity(I, dt, Ap0, np.array([0.0, 0.3]), subtract_mean=subtract_mean)
    assert eps0 is None
    if subtract_mean:                       # the mask-weighted mean removal enforces sigma(0) = 0
        assert abs(sig0[0]) < 1e-12 * np.max(np.abs(sig))


def test_response_argument_errors():
    from paper_1804_01404_gb300 import tdks as T
    with pytest.raises(T.TdksError):
        T.oscillator_strength(np.zeros(1), 0.02, 1e-3, np.array([0.1]))       # one sample
    with pytest.raises(T.TdksError):
        T.oscillator_strength(np.zeros(10), 0.02, 0.0, np.array([0.1]))       # kappa = 0
    with pytest.raises(T.TdksError):
        T.conductivity(np.zeros(10), -0.02, 1e-3, np.array([0.1]))             # dt <= 0


def _main_peak(spectrum_fn, lo=0.0, hi=2.0):
    """Energy (Ha) of the largest value of spectrum_fn(E): a 0.005 Ha scan, then a 0.001 eV grid
    around its maximum."""
    E = np.arange(lo, hi, 0.005)
    E0 = E[np.argmax(spectrum_fn(E))]
    Ef = np.arange(max(E0 - 0.01, 1e-6), E0 + 0.01, 0.001 / EV)
    return Ef[np.argmax(spectrum_fn(Ef))]


def test_absorption_peak_fp32_within_001_ev_of_oracle():
    from paper_1804_01404_gb300 import tdks as T
    s = W.tiny(periodic=False, n=(9, 10, 11), natom=2, norb=2)
    kappa = 1e-3
    nsteps = 600
    psi0 = O.apply_kick(s, W.initial_orbitals(s, 5), (0.0, 0.0, kappa))
    _, _, hist = O.run(s, psi0, nsteps)
    t = np.arange(0, nsteps + 1) * s.dt
    d_ref = np.concatenate([[0.0], hist["d"][:, 2]])
    E_ref = _main_peak(lambda E: O.oscillator_strength(t, d_ref, kappa, E))
    for mode in (T.PRED_PC, T.PRED_EXTRAP):
        ctx = T.Context(s, precision="f32")
        u = torch.from_numpy(psi0.astype(np.complex64)).cuda()
        ctx.update_potential(u)
        if mode != T.PRED_PC:
            ctx.nn_init(0)
            ctx.set_predictor(mode, 1e-5)
        d = [0.0]
        tt = 0.0
        for _ in range(nsteps):
            ctx.step(u, tt, s.dt)
            tt += s.dt
            d.append(ctx.read_step_observables()["dipole"][2])
        ctx.check()
        d = np.array(d)
        assert np.max(np.abs(d - d_ref)) < 1e-3 * np.max(np.abs(d_ref))
        E_gpu = _main_peak(lambda E: T.oscillator_strength(d, s.dt, kappa, E))
        assert abs(E_gpu - E_ref) * EV < 0.01, (mode, E_gpu * EV, E_ref * EV)
        ctx.close()


@pytest.mark.parametrize("precision,tol", [("f64", 1e-8), ("f32", 3e-4)])
def test_dielectric_function_of_a_kicked_cell(precision, tol):
    """Periodic cell with the A' step of Eq. (impulsive_A): eps(w) from the GPU's current history
    against eps from the oracle's, with the mean current removed as in the Sec. 4.1 example."""
    from paper_1804_01404_gb300 import tdks as T
    s = W.tiny(periodic=True, n=(6, 7, 8), natom=2, nk=2, norb=2)
    Ap0 = 1e-3
    s.field = W.Field("step", (0.0, 0.0, Ap0))
    nsteps = 300
    psi0 = W.initial_orbitals(s, 6)
    _, _, hist = O.run(s, psi0, nsteps)
    ctx = T.Context(s, precision=precision)
    u = torch.from_numpy(psi0.astype(np.complex128 if precision == "f64" else np.complex64)).cuda()
    ctx.update_potential(u)
    J = []
    tt = 0.0
    for _ in range(nsteps):
        ctx.step(u, tt, s.dt)
        tt += s.dt
        J.append(ctx.read_step_observables()["J"][2])
    ctx.check()
    ctx.close()
    J = np.array(J)
    Jref = hist["J"][:, 2]
    assert np.max(np.abs(J - Jref)) < tol * np.max(np.abs(Jref))
    w = np.linspace(0.1, 2.0, 200)
    t = np.arange(1, nsteps + 1) * s.dt - s.dt       # samples of J at t_1..t_n, re-based to 0
    _, eps = T.conductivity(J, s.dt, Ap0, w, subtract_mean=True)
    eps_ref = O.dielectric(w, O.conductivity(t, Jref, Ap0, w, subtract_mean=True))
    assert _rel(eps - 1.0, eps_ref - 1.0) < 10 * tol


def test_work_of_the_field():
    """Sec. 4.1 work W(t) = int I.E dt: the GPU's FP64 current history and the context's field
    (tdks_field_at) through tdks_work, against the oracle's current, closed-form E and work."""
    from paper_1804_01404_gb300 import tdks as T
    s = W.tiny(periodic=True, n=(6, 7, 8), natom=2, nk=2, norb=2)
    s.field = W.Field("pulse", (0.0, 0.0, 0.05), 0.5, 6.0, 0.0, more=(((0.02, 0.0, 0.0), 0.8, 2.0, 0.0, 2.5),))
    psi0 = W.initial_orbitals(s, 3)
    n = 300
    ctx = T.Context(s, precision="f64")
    u = torch.from_numpy(psi0).cuda()
    ctx.update_potential(u)
    o0 = ctx.observables(u, ctx.field_at(0.0)[0])
    J, E = [o0["J"]], [ctx.field_at(0.0)[1]]
    tt = 0.0
    for _ in range(n):
        ctx.step(u, tt, s.dt)
        tt += s.dt
        J.append(ctx.read_step_observables()["J"])
        Ap, Ef = ctx.field_at(tt)
        assert np.max(np.abs(Ap - O.field_Aprime(s.field, tt))) < 1e-15
        # central difference vs closed form; at a pulse onset (t = 2.5) the one-sided quadratic start
        # of the envelope costs O(h |A''|) ~ 1e-7
        assert np.max(np.abs(Ef - O.field_E(s.field, tt))) < 1e-6
        E.append(Ef)
    ctx.check()
    ctx.close()
    Wg = T.work(np.array(J), np.array(E), s.dt)
    _, _, hist = O.run(s, psi0, n)
    ts = np.arange(n + 1) * s.dt
    Jref = np.concatenate([[O.current(s, O.projector_tables(s), psi0, np.zeros(3))], hist["J"]])
    Wref = O.work(ts, Jref, np.array([O.field_E(s.field, t) for t in ts]))
    assert _rel(Wg, Wref) < 1e-6
    assert np.max(np.abs(Wref)) > 1e-6                       # the field does work
