"""Phase timing and launch counting of the C ABI (tdks_profile / tdks_stats_read) on the GPU.

The stencil-kernel phase is nested inside the Taylor phases: it must count one launch per Taylor
kernel call and never take longer than the phases around it."""
import numpy as np
import pytest

from paper_1804_01404_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_stencil_phase_nested_in_taylor_phases():
    from paper_1804_01404_gb300.tdks import Context
    s = W.small_periodic()
    ctx = Context(s, precision="f32")
    u = torch.from_numpy(W.initial_orbitals(s, 0).astype(np.complex64)).cuda()
    ctx.update_potential(u)
    ctx.stats(reset=True)
    ctx.profile(True)
    t = 0.0
    for _ in range(3):
        ctx.step(u, t, s.dt)
        t += s.dt
    st = ctx.stats(reset=True)
    ctx.profile(False)
    ctx.check()
    taylor_calls = st["calls"]["taylor_predictor"] + st["calls"]["taylor_corrector"]
    assert taylor_calls == 6 and st["calls"]["stencil_kernel"] == taylor_calls
    taylor_ms = st["ms"]["taylor_predictor"] + st["ms"]["taylor_corrector"]
    assert 0 < st["ms"]["stencil_kernel"] <= taylor_ms
    assert st["launches"] >= taylor_calls
    assert ctx.stats(reset=True)["launches"] == 0


def test_fp64_probe_is_plausible():
    """The FP64 FMA-rate probe behind the FP64 path's roofline returns a finite rate well below the
    FP32 rate of the device (FP64 runs at a small fraction of it here)."""
    from paper_1804_01404_gb300 import tdks as T
    r = T.probe_fp64()
    assert np.isfinite(r) and 0.05 < r < 100.0
