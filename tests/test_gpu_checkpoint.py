"""Checkpoint and restart (tdks_get_state / tdks_set_state): a fresh context restored from a state
and the saved orbitals continues exactly as the original context does."""
import numpy as np
import pytest

from paper_1804_01404_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


def _steps(ctx, u, s, t, n):
    J = []
    for _ in range(n):
        ctx.step(u, t, s.dt)
        t += s.dt
        J.append(ctx.read_step_observables()["J"])
    return np.array(J), t


@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("f32", 1e-6)])
@pytest.mark.parametrize("predictor", ["pc", "extrap"])
def test_restart_continues_like_the_original(precision, tol, predictor):
    from paper_1804_01404_gb300 import tdks as T
    s = W.small_periodic()
    dt_ = torch.complex128 if precision == "f64" else torch.complex64
    ctx = T.Context(s, precision=precision)
    u = torch.from_numpy(W.initial_orbitals(s, 2)).to("cuda", dt_)
    ctx.update_potential(u)
    if predictor == "extrap":
        ctx.set_predictor(T.PRED_EXTRAP, 1e-3)
    _, t = _steps(ctx, u, s, 0.0, 6)
    state = ctx.get_state()
    saved = u.clone()
    Ja, _ = _steps(ctx, u, s, t, 5)
    ua = u.cpu().numpy()
    ctx2 = T.Context(s, precision=precision)
    ctx2.set_state(state)
    u2 = saved.clone()
    Jb, _ = _steps(ctx2, u2, s, t, 5)
    ctx.check()
    ctx2.check()
    assert _rel(u2.cpu().numpy(), ua) < tol
    assert np.max(np.abs(Jb - Ja)) < tol * np.max(np.abs(Ja))
    assert ctx2.read_step_observables()["fallbacks"] == ctx.read_step_observables()["fallbacks"]


def test_restart_multiscale():
    from paper_1804_01404_gb300 import tdks as T
    s = W.tiny(periodic=True, n=(6, 7, 8), natom=1, nk=2, norb=2)
    s.field = W.Field("none")
    ncell, m0, dX = 3, 2, 40.0
    X = np.arange(8)
    A_now, A_prev = 0.3 * np.exp(-((X - 2.0) / 1.5) ** 2), 0.3 * np.exp(-((X - 1.9) / 1.5) ** 2)
    psis = np.stack([W.initial_orbitals(s, 30 + c) for c in range(ncell)])
    ctx = T.Context(s, precision="f64", ncell=ncell)
    u = torch.from_numpy(psis).cuda()
    ctx.update_potential(u)
    ctx.ms_init(dX, m0, A_now, A_prev)
    for _ in range(3):
        ctx.ms_step(u, 0.0, s.dt)
    state = ctx.get_state()
    saved = u.clone()
    for _ in range(2):
        ctx.ms_step(u, 0.0, s.dt)
    Aa, Ia = ctx.ms_read()
    ctx2 = T.Context(s, precision="f64", ncell=ncell)
    ctx2.set_state(state)
    u2 = saved.clone()
    for _ in range(2):
        ctx2.ms_step(u2, 0.0, s.dt)
    Ab, Ib = ctx2.ms_read()
    assert np.max(np.abs(Ab - Aa)) < 1e-13 * np.max(np.abs(Aa))
    assert np.max(np.abs(Ib - Ia)) < 1e-11 * np.max(np.abs(Ia))
    assert _rel(u2.cpu().numpy(), u.cpu().numpy()) < 1e-12


def test_foreign_or_truncated_state_is_rejected():
    from paper_1804_01404_gb300 import tdks as T
    s = W.small_periodic()
    ctx = T.Context(s, precision="f64")
    ctx.update_potential(torch.from_numpy(W.initial_orbitals(s, 1)).cuda())
    state = ctx.get_state()
    other = W.tiny(periodic=True, n=(8, 8, 8))
    with pytest.raises(T.TdksError) as e:
        T.Context(other, precision="f64").set_state(state)
    assert e.value.status == 1
    with pytest.raises(T.TdksError):
        T.Context(s, precision="f32").set_state(state)
    with pytest.raises(T.TdksError):
        T.Context(s, precision="f64").set_state(state[: len(state) // 2])
