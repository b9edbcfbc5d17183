"""Sec. 3.1 fields beyond the single pulse on the GPU: successive delayed pulses (pump-probe) and a
field given by a numerical table, against the oracle's steps with the same field; argument checks;
and the table surviving a checkpoint / restart."""
import numpy as np
import pytest

from oracle import tdks_oracle as O
from paper_1804_01404_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _system(field):
    s = W.tiny(periodic=True, n=(6, 7, 8), natom=2, nk=2, norb=2)
    s.field = field
    return s


def _pump_probe():
    return W.Field("pulse", (0.0, 0.0, 0.02), 0.3, 4.0, 0.1, more=(((0.01, 0.0, 0.015), 0.5, 3.0, 0.0, 1.2),))


def _run_gpu(s, psi0, t0, n, ctx=None):
    from paper_1804_01404_gb300.tdks import Context
    ctx = ctx or Context(s, precision="f64")
    u = torch.from_numpy(psi0).cuda()
    ctx.update_potential(u)
    J, t = [], t0
    for _ in range(n):
        ctx.step(u, t, s.dt)
        t += s.dt
        J.append(ctx.read_step_observables()["J"])
    ctx.check()
    return u.cpu().numpy(), np.array(J), ctx


def _run_oracle(s, psi0, t0, n):
    tabs = O.projector_tables(s)
    Vloc = O.local_potential(s)
    psi = psi0.copy()
    vhxc = O.hxc(s, O.density(s, psi))
    J, t = [], t0
    for _ in range(n):
        psi, vhxc, _ = O.pc_step(s, tabs, Vloc, psi, vhxc, t, s.dt)
        t += s.dt
        J.append(O.current(s, tabs, psi, O.field_Aprime(s.field, t)))
    return psi, np.array(J)


@pytest.mark.parametrize("kind", ["pump_probe", "table"])
def test_steps_with_field(kind):
    if kind == "pump_probe":
        f = _pump_probe()
    else:   # a coarse table of the pump-probe field: linear between samples 0.05 au apart
        pp = _pump_probe()
        ts = np.arange(0, 121) * 0.05
        f = W.Field("table", table=np.array([O.field_Aprime(pp, t) for t in ts]), t0=0.0, dt_table=0.05)
    s = _system(f)
    psi0 = W.initial_orbitals(s, 3)
    t0, n = 1.0, 12                   # both pulses act during these steps
    got, J, ctx = _run_gpu(s, psi0, t0, n)
    ref, Jref = _run_oracle(s, psi0, t0, n)
    assert np.linalg.norm(got - ref) < 1e-10 * np.linalg.norm(ref)
    assert np.max(np.abs(J - Jref)) < 1e-10 * np.max(np.abs(Jref))
    assert np.max(np.abs(Jref[-1] - Jref[0])) > 1e-4 * np.max(np.abs(Jref))     # the field drives the current
    ctx.close()


def test_field_argument_errors():
    from paper_1804_01404_gb300.tdks import Context, TdksError, FIELD_STEP
    s = _system(W.Field("step", (0.0, 0.0, 1e-3)))
    ctx = Context(s, precision="f64")
    with pytest.raises(TdksError):
        ctx.add_pulse((0, 0, 1e-3), 0.3, 4.0)                 # the field is a step, not a pulse
    with pytest.raises(TdksError):
        ctx.set_field_table(np.zeros((4, 3)), 0.0, 0.0)       # dt_table = 0
    ctx.set_field(FIELD_STEP, (0, 0, 1e-3))
    ctx.close()


def test_table_field_survives_checkpoint():
    """Three steps, checkpoint, three more: a fresh context restored from the state (field table
    included, the table not set again) continues like the original."""
    from paper_1804_01404_gb300.tdks import Context
    pp = _pump_probe()
    ts = np.arange(0, 121) * 0.05
    f = W.Field("table", table=np.array([O.field_Aprime(pp, t) for t in ts]), t0=0.0, dt_table=0.05)
    s = _system(f)
    psi0 = W.initial_orbitals(s, 4)
    a = Context(s, precision="f64")
    u = torch.from_numpy(psi0).cuda()
    a.update_potential(u)
    t = 1.0
    for _ in range(3):
        a.step(u, t, s.dt)
        t += s.dt
    state = a.get_state()
    mid = u.clone()
    for _ in range(3):
        a.step(u, t, s.dt)
        t += s.dt
    s_nofield = _system(W.Field("none"))
    b = Context(s_nofield, precision="f64")
    b.set_state(state)
    t = 1.0 + 3 * s.dt
    for _ in range(3):
        b.step(mid, t, s.dt)
        t += s.dt
    # the FP64 density sums may add in another order: agreement to rounding
    assert (mid - u).abs().max().item() < 1e-12 * u.abs().max().item()
    a.close()
    b.close()
