"""The predicted step of tdks_step (TDKS_PRED_LEARNED, TDKS_PRED_EXTRAP) end to end against the
oracle's predicted step (oracle.tdks_oracle.run_predicted, pinned on the CPU in
tests/test_predicted_pins.py).

The network runs with fixed, seeded parameters; the oracle evaluates it at the network's storage
precision (nn_oracle.predict_bf16: BF16 weights, inputs and activations, FP64 sums), so the two sides
differ by the device's FP32 accumulation and, rarely, a BF16 rounding decision that it flips.  The
correction that the network adds is of the size of the cubic extrapolation's error, so those
differences reach the orbitals far below 1e-10.

System: the small periodic cell (16^3, two pseudo-atoms, 8 orbitals at Gamma, A'-step kick 0.001),
24 steps: three predictor-corrector steps fill the potential history, the other 21 are predicted.
Bounds: FP64 orbitals, V_Hxc, J and dipole within 1e-10 (relative); the FP32 orbitals' J and dipole
within 1e-4 of max |X| of the FP64 oracle (the error bound of FP32 orbitals).
"""
import numpy as np
import pytest

from oracle import nn_oracle as N
from oracle import tdks_oracle as O
from paper_1804_01404_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NSTEPS = 24


def _params():
    """Seeded weights with the output layer scaled so that the network's correction is of the size of
    a trained one (the size of the cubic extrapolation's own error; misfits 1.1e-5 against the
    cubic's 0.9e-5).  An untrained network of the same scale moves V~ by thirty times that, and the
    device's FP32 sums in it then reach the FP64 orbitals at a few 1e-10 after 21 steps."""
    p = np.random.default_rng(21).standard_normal(N.NPARAMS) * 0.15
    p[8672:] *= 0.03                       # W3 and b3
    return p


def _predictor(name, s):
    if name == "learned":
        p = _params()
        return lambda V0, V1, V2, V3: N.predict_bf16(p, V0, V1, V2, V3, s.periodic)
    return N.cubic_extrapolation


_ORACLE = {}


def _oracle(name, threshold):
    key = (name, threshold)
    if key not in _ORACLE:
        s = W.small_periodic(nsteps=NSTEPS)
        psi0 = W.initial_orbitals(s, 0)
        _ORACLE[key] = O.run_predicted(s, psi0, NSTEPS, _predictor(name, s), threshold)
    return _ORACLE[key]


def _gpu(name, threshold, precision, pipelined=False):
    """pipelined: read every step's observables as an application that keeps the stream busy does --
    tdks_copy_step_observables into one of two pinned host blocks, unpacked after the next step has
    been queued."""
    from paper_1804_01404_gb300 import tdks as T
    s = W.small_periodic(nsteps=NSTEPS)
    psi0 = W.initial_orbitals(s, 0)
    ctx = T.Context(s, precision=precision)
    u = torch.from_numpy(psi0).to("cuda", torch.complex128 if precision == "f64" else torch.complex64)
    ctx.update_potential(u)
    ctx.nn_init(0)
    ctx.nn_params(_params())
    ctx.set_predictor(T.PRED_LEARNED if name == "learned" else T.PRED_EXTRAP, threshold)
    J, d, r = [], [], []
    ring = [torch.zeros(T.STEP_OBS_DOUBLES, dtype=torch.float64).pin_memory() for _ in range(2)]
    evs = [torch.cuda.Event() for _ in range(2)]
    t = 0.0

    def take(o):
        J.append(o["J"])
        d.append(o["dipole"])
        r.append(o["residual"])

    for i in range(NSTEPS):
        ctx.step(u, t, s.dt)
        t += s.dt
        if not pipelined:
            o = ctx.read_step_observables()
            take(o)
            continue
        ctx.copy_step_observables(ring[i % 2])
        evs[i % 2].record(ctx.stream)
        if i > 0:
            evs[(i - 1) % 2].synchronize()
            take(ctx.unpack_step_observables(ring[(i - 1) % 2]))
    if pipelined:
        evs[(NSTEPS - 1) % 2].synchronize()
        o = ctx.unpack_step_observables(ring[(NSTEPS - 1) % 2])
        take(o)
        o2 = ctx.read_step_observables()
        assert np.array_equal(o2["J"], o["J"]) and o2["fallbacks"] == o["fallbacks"]
    ctx.check()
    out = dict(J=np.array(J), d=np.array(d), misfit=np.array(r), fallbacks=o["fallbacks"],
               psi=u.cpu().numpy().astype(np.complex128), v=ctx.grid_array(1).cpu().numpy())
    ctx.close()
    return out


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("name", ["learned", "cubic"])
def test_predicted_steps_fp64_match_the_oracle(name):
    psi, v, rec = _oracle(name, 1.0)
    g = _gpu(name, 1.0, "f64")
    assert rec["rejected"] == 0 and g["fallbacks"] == 0
    assert np.linalg.norm(g["psi"] - psi) < 1e-10 * np.linalg.norm(psi)
    assert _rel(g["v"], v) < 1e-10
    assert _rel(g["J"], rec["J"]) < 1e-10
    assert _rel(g["d"], rec["d"]) < 1e-10
    # misfits of the accepted predictions (the plain steps report the PC's own).  The misfit is a
    # difference of nearly equal potentials, so the network's FP32 sums show in it at ~1e-5 of its
    # value; the cubic extrapolation is FP64 on both sides.
    m = rec["misfit"][3:]
    assert np.max(np.abs(g["misfit"][3:] - m) / m) < (1e-4 if name == "learned" else 1e-6)


def test_learned_steps_fp32_within_the_current_and_dipole_bound():
    _, _, rec = _oracle("learned", 1.0)
    g = _gpu("learned", 1.0, "f32")
    assert g["fallbacks"] == 0
    assert _rel(g["J"], rec["J"]) < 1e-4
    assert _rel(g["d"], rec["d"]) < 1e-4


def test_learned_steps_with_rejections_match_the_oracle():
    """A threshold inside the range of the network's misfits: some predictions are kept, the others
    are redone with the plain predictor-corrector.  The threshold sits where no misfit of the oracle
    run lies within 0.2 % of it -- 20 times the bound on the misfit's discrepancy between the two
    sides -- so the device takes the same decisions."""
    _, _, free = _oracle("learned", 1.0)
    m = np.sort(free["misfit"][3:])
    gaps = np.log(m[1:] / m[:-1])
    j = int(np.argmax(gaps[len(m) // 4: 3 * len(m) // 4])) + len(m) // 4
    thr = float(np.sqrt(m[j] * m[j + 1]))
    psi, v, rec = _oracle("learned", thr)
    acc = rec["misfit"][3:]
    assert np.min(np.abs(np.log(acc / thr))) > 2e-3, "threshold too close to a misfit"
    assert 0 < rec["rejected"] < NSTEPS - 3
    g = _gpu("learned", thr, "f64")
    assert g["fallbacks"] == rec["rejected"]
    assert np.linalg.norm(g["psi"] - psi) < 1e-10 * np.linalg.norm(psi)
    assert _rel(g["J"], rec["J"]) < 1e-10
    assert _rel(g["d"], rec["d"]) < 1e-10


def test_pipelined_reads_of_learned_steps_with_rejections_match_the_oracle():
    """The same run with every step's observables copied without waiting and unpacked one step later
    (tdks_copy_step_observables / tdks_unpack_step_observables): the values and the fallback count of
    every step are those of the oracle run."""
    _, _, free = _oracle("learned", 1.0)
    m = np.sort(free["misfit"][3:])
    gaps = np.log(m[1:] / m[:-1])
    j = int(np.argmax(gaps[len(m) // 4: 3 * len(m) // 4])) + len(m) // 4
    thr = float(np.sqrt(m[j] * m[j + 1]))
    psi, v, rec = _oracle("learned", thr)
    g = _gpu("learned", thr, "f64", pipelined=True)
    assert 0 < rec["rejected"] and g["fallbacks"] == rec["rejected"]
    assert len(g["J"]) == NSTEPS
    assert _rel(g["J"], rec["J"]) < 1e-10
    assert _rel(g["d"], rec["d"]) < 1e-10
    assert np.linalg.norm(g["psi"] - psi) < 1e-10 * np.linalg.norm(psi)


def _tile_system():
    s = W.isolated_cluster(n=24, natom=5, norb=3, radius=3.5, seed=4)
    s.n = (40, 30, 28)                      # does not fit the shared-memory cell kernels: tile path
    s.h = (0.45, 0.5, 0.55)
    return s


@pytest.mark.parametrize("graph", [True, False])
@pytest.mark.parametrize("threshold", [1.0, 1e-300])
def test_predicted_steps_on_the_tile_path(graph, threshold):
    """Cubic-extrapolation steps on a large isolated grid (TMA tile kernels, projections on a side
    stream), every prediction kept (threshold 1) or every one rejected (the fallback body, which forks
    its own side stream inside the step graph), as a step graph and as stream launches, FP64, against
    the oracle's predicted run."""
    from paper_1804_01404_gb300 import tdks as T
    s = _tile_system()
    n = 7
    psi0 = O.apply_kick(s, W.initial_orbitals(s, 2), (0.0, 0.0, 0.01))
    psi, v, rec = O.run_predicted(s, psi0, n, N.cubic_extrapolation, threshold)
    assert rec["rejected"] == (0 if threshold == 1.0 else n - 3)
    ctx = T.Context(s, precision="f64")
    u = torch.from_numpy(psi0).to("cuda")
    ctx.update_potential(u)
    ctx.set_predictor(T.PRED_EXTRAP, threshold)
    ctx.set_step_graph(graph)
    d = []
    t = 0.0
    for _ in range(n):
        ctx.step(u, t, s.dt)
        t += s.dt
        d.append(ctx.read_step_observables()["dipole"])
    ctx.check()
    assert ctx.read_step_observables()["fallbacks"] == rec["rejected"]
    got = u.cpu().numpy()
    assert np.linalg.norm(got - psi) < 1e-10 * np.linalg.norm(psi)
    assert _rel(np.array(d), rec["d"]) < 1e-10
    ctx.close()
