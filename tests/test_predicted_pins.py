"""Pins of the oracle's predicted step (CPU): the scheme that replaces the predictor half-step of the
predictor-corrector (Program summary) by a predicted potential V~(t+dt), with the self-consistency
misfit deciding whether the step is kept, and of the BF16 storage format of the network.

What pins it, independent of the implementation:
  * fed the plain predictor's own potential, the predicted step IS the predictor-corrector step
    (a dropped 1/2, a wrong field time or a wrong base potential in the corrector breaks this);
  * with every prediction rejected the run equals the plain predictor-corrector run;
  * the scheme with the cubic extrapolation converges at second order in dt to a fine-step
    reference (a first-order slip, e.g. propagating with V(t) alone, gives a ratio near 2);
  * with no field the total energy drift falls at least as dt^2;
  * BF16 rounding: exact values of ties and non-ties, idempotence and the 2^-8 relative bound.
"""
import numpy as np

from oracle import nn_oracle as N
from oracle import tdks_oracle as O
from paper_1804_01404_gb300 import workloads as W


def _system(field="step"):
    s = W.tiny(periodic=True, n=(8, 8, 8), natom=1, norb=2)
    s.field = W.Field("step", (0.0, 0.01, 0.02)) if field == "step" else W.Field("none")
    return s


def test_predicted_step_with_the_pc_predictor_is_the_pc_step():
    s = _system()
    psi = W.initial_orbitals(s, 3)
    tabs, Vloc = O.projector_tables(s), O.local_potential(s)
    v = O.hxc(s, O.density(s, psi))
    t, dt = 0.3, 0.02
    Ap = O.field_Aprime(s.field, t + 0.5 * dt)
    pred = O.propagate_all(s, tabs, Vloc + v, psi, Ap, dt)        # the predictor half-step
    vpred = O.hxc(s, O.density(s, pred))
    a = O.predicted_step(s, tabs, Vloc, psi, v, vpred, t, dt, np.inf)
    b = O.pc_step(s, tabs, Vloc, psi, v, t, dt)
    assert a[4]
    assert np.max(np.abs(a[0] - b[0])) < 1e-14 * np.max(np.abs(b[0]))
    assert np.max(np.abs(a[1] - b[1])) < 1e-14 * np.max(np.abs(b[1]))
    # the misfit of that prediction is the PC's own, small but not zero
    assert 0 < a[3] == O.misfit(b[1], vpred) < 1e-3


def test_rejected_predictions_give_the_pc_run():
    s = _system()
    psi0 = W.initial_orbitals(s, 4)
    n = 8
    pa, va, ra = O.run_predicted(s, psi0, n, N.cubic_extrapolation, -1.0)
    pb, vb, rb = O.run(s, psi0, n)
    assert ra["rejected"] == n - 3
    assert np.max(np.abs(pa - pb)) < 1e-14 * np.max(np.abs(pb))
    assert np.max(np.abs(ra["J"] - rb["J"])) < 1e-14 * np.max(np.abs(rb["J"]))
    assert np.all(np.isnan(ra["misfit"][:3])) and np.all(ra["misfit"][3:] > 0)


def test_predicted_scheme_converges_at_second_order():
    s = _system(field="none")
    psi0 = W.initial_orbitals(s, 5)
    T = 0.48
    s.dt = T / 192
    ref, _, _ = O.run(s, psi0, 192, record=False)
    errs = []
    for nstep in (12, 24, 48):
        s.dt = T / nstep
        p, _, r = O.run_predicted(s, psi0, nstep, N.cubic_extrapolation, np.inf)
        assert r["rejected"] == 0
        errs.append(np.linalg.norm(p - ref) / np.linalg.norm(ref))
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs
    # the same test separates a first-order variant: propagating with V(t) alone
    tabs, Vloc = O.projector_tables(s), O.local_potential(s)

    def first_order(nstep):
        s.dt = T / nstep
        psi = psi0.copy()
        v = O.hxc(s, O.density(s, psi))
        hist = [v]
        for i in range(nstep):
            if len(hist) >= 4:
                psi = O.propagate_all(s, tabs, Vloc + v, psi, np.zeros(3), s.dt)   # V(t) only
                v = O.hxc(s, O.density(s, psi))
            else:
                psi, v, _ = O.pc_step(s, tabs, Vloc, psi, v, i * s.dt, s.dt)
            hist = (hist + [v])[-4:]
        return np.linalg.norm(psi - ref) / np.linalg.norm(ref)
    e1 = [first_order(n) for n in (24, 48)]
    assert e1[0] / e1[1] < 2.5, e1


def test_predicted_scheme_conserves_energy_at_second_order():
    s = _system(field="none")
    psi0 = W.initial_orbitals(s, 6)
    tabs, Vloc = O.projector_tables(s), O.local_potential(s)
    E0 = O.total_energy(s, tabs, Vloc, psi0, np.zeros(3))
    drift = []
    for dt, n in ((0.04, 12), (0.02, 24)):
        s.dt = dt
        p, _, r = O.run_predicted(s, psi0, n, N.cubic_extrapolation, np.inf)
        drift.append(abs(O.total_energy(s, tabs, Vloc, p, np.zeros(3)) - E0))
    assert drift[1] < drift[0] / 3.5, drift


def test_misfit_of_a_scaled_potential():
    rng = np.random.default_rng(2)
    v = rng.standard_normal((4, 5, 6))
    assert abs(O.misfit(v, 1.003 * v) - 0.003) < 1e-15


def test_bf16_rounding():
    one = 1.0
    ulp = 2.0 ** -7                                   # spacing of BF16 in [1, 2)
    vals = np.array([one + ulp / 2, one + 1.5 * ulp, one + ulp / 2 + 2.0 ** -20, -(one + 1.5 * ulp), 3.0, 0.0])
    exp = np.array([one, one + 2 * ulp, one + ulp, -(one + 2 * ulp), 3.0, 0.0])
    assert np.array_equal(N.bf16(vals), exp)          # ties to even, a non-tie rounds up, sign kept
    rng = np.random.default_rng(3)
    x = rng.standard_normal(10000) * 10.0 ** rng.uniform(-6, 6, 10000)
    b = N.bf16(x)
    assert np.array_equal(N.bf16(b), b)
    assert np.max(np.abs(b - x) / np.abs(x)) <= 2.0 ** -8 * (1 + 1e-7)
    # at most 8 significant bits survive
    m, _ = np.frexp(b)
    assert np.array_equal(m * 256, np.round(m * 256))


def test_bf16_forward_against_the_fp64_forward():
    """The stored-precision forward pass stays within a few BF16 ulps of the FP64 forward pass of the
    same rounded weights and inputs (only the two hidden activations are rounded in between), and a
    zero network predicts the cubic extrapolation exactly."""
    rng = np.random.default_rng(4)
    p = rng.standard_normal(N.NPARAMS) * 0.2
    x = rng.standard_normal((4, 4, 5, 6))
    out = N.forward_bf16(p, x, True)
    ref, _ = N.forward(N.bf16(p), N.bf16(x), True)
    assert 0 < np.max(np.abs(out - ref)) < 2.0 ** -6 * np.max(np.abs(ref))
    V = rng.standard_normal((4, 3, 4, 5))
    assert np.array_equal(N.predict_bf16(np.zeros(N.NPARAMS), *V, False), N.cubic_extrapolation(*V))
