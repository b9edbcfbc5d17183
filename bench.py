#!/usr/bin/env python
"""Benchmark of one real-time TDKS predictor-corrector step on the GPU (libtdks, C ABI).

Workload: the diamond-lattice crystal response -- 8-atom cubic cell a = 10.26 bohr, 20^3 grid,
16 orbitals x 64 k-points (4^3 shifted Monkhorst-Pack), sin^2 pulse along z (1.55 eV, 1e-3 au,
10 fs), dt = 0.02 au, 4th-order Taylor + predictor-corrector + FFT Hartree + LDA exchange,
FP32 orbitals with FP64 reductions.  A "step" is one full tdks_step: predictor Taylor,
density, Hartree + exchange, corrector Taylor, density, Hartree + exchange, current and dipole.

Arms:
  default            the CUDA path; prints one JSON line (rank 0).
  --impl reference   the FP64 CPU oracle on all of this host's cores: the 64 k-points are split over
                     one worker process per core, each running the oracle's predictor-corrector step
                     on its own k-points (see oracle_parallel_steps).

Multi-GPU: every rank propagates its own copy of the workload (independent replicas, no
collective on the data path); value = total steps of all ranks / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")     # the CPU oracle legs run single-threaded

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TDKS steps/s & hpsi HBM GB/s vs peak; FP32+learned vs FP64 at ≤1e-4 J err"
UNIT = "steps/s"
FP32_LANES_PER_SM = 128
PHASE_STEPS = 5          # steps with every phase timed, after the timed region
# algorithmic FP32 flops per grid point per Horner stage of the periodic Hamiltonian:
# 12 neighbour pairs x (4 adds + 4 FMA) for the Laplacian and q.grad terms (144), diagonal (3),
# Horner update (4)
FLOPS_PER_POINT_STAGE = 151
FLOPS_PER_SPHERE_ENTRY_STAGE = 44   # projection (22) + scatter (22)


def workload():
    from paper_1804_01404_gb300 import workloads as W
    return W.diamond_crystal()


def config_dict(s, extra=None):
    d = {"workload": "diamond crystal 20^3 grid, 8 atoms, 16 orbitals x 64 k, sin^2 pulse",
         "grid": list(s.n), "norb": s.norb, "nk": s.nk, "dt": s.dt, "taylor_order": 4,
         "predictor": "predictor-corrector", "orbitals": "f32", "reductions_poisson": "f64",
         "observables": "J(t) and dipole(t) of every step's input state, formed in its first Taylor "
                        "stage (tdks_options.obs_at_start = 1)",
         "l2": "flushed between timed steps (256 MiB write)"}
    if extra:
        d.update(extra)
    return d


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "fallback": True}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.count(",") >= 7]
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].strip() == "Active"})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows)}


def _oracle_worker(job):
    """One worker of oracle_parallel_steps: the oracle's predictor-corrector step (plus the current)
    on k-points k_lo..k_hi-1 of the workload, `warmup` untimed steps, then a barrier shared by all
    workers, then `steps` timed steps.  Returns the timed seconds."""
    k_lo, k_hi, warmup, steps, barrier = job
    from oracle import tdks_oracle as O
    from paper_1804_01404_gb300 import workloads as W
    s = workload()
    s.kpts = s.kpts[k_lo:k_hi]
    s.kw = np.full(k_hi - k_lo, 1.0 / s.nk)
    psi = W.initial_orbitals(s, 0)
    tabs = O.projector_tables(s)
    Vloc = O.local_potential(s)
    v = O.hxc(s, O.density(s, psi))
    t = 200.0

    def step():
        nonlocal psi, v, t
        psi, v, _ = O.pc_step(s, tabs, Vloc, psi, v, t, s.dt)
        t += s.dt
        O.current(s, tabs, psi, O.field_Aprime(s.field, t))
    for _ in range(warmup):
        step()
    barrier.wait()
    tic = time.perf_counter()
    for _ in range(steps):
        step()
    return time.perf_counter() - tic


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_parallel_steps(steps, warmup):
    """The FP64 oracle on all host cores: the workload's k-points are split evenly over one worker
    process per core (spawned, numpy single-threaded in each), every worker runs the oracle's own
    predictor-corrector step on its k-points, and the timed region is the slowest worker's `steps`
    steps after a common barrier.  All k-points are propagated every step, so the work per step is
    the whole workload's, except that each worker forms the density and the Hartree-exchange potential
    of its own k-points (their sum over the workers is not formed): one extra 20^3 Hartree-exchange
    evaluation per worker.  Returns (seconds per step, workers, description)."""
    import multiprocessing as mp
    nk = workload().nk
    nw = max(1, min(host_cores(), nk))
    bounds = np.linspace(0, nk, nw + 1).round().astype(int)
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        barrier = mgr.Barrier(nw)
        with ctx.Pool(nw) as pool:
            secs = pool.map(_oracle_worker, [(int(bounds[i]), int(bounds[i + 1]), warmup, steps, barrier)
                                             for i in range(nw)])
    per_step = max(secs) / steps
    desc = (f"all {nk} k-points (16 orbitals each, 20^3 grid) split over {nw} worker processes, one per "
            f"host core; each runs the oracle's PC step + current on its {nk // nw}-{-(-nk // nw)} k-points and "
            f"forms the density and V_Hxc of those only; {warmup} untimed + {steps} timed steps; time = "
            f"slowest worker")
    return per_step, nw, desc


def reference_arm(args, rank, world):
    if rank != 0:
        return 0
    s = workload()
    per_step, nw, sample = oracle_parallel_steps(args.steps, args.warmup)
    v = 1.0 / per_step
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(s, {"orbitals": "f64",
                                                             "observables": "J after each oracle step"}),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": nw, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def replica_throughput(total_ms, steps, world, device=None):
    """Whole-job throughput of `world` independent replicas that each timed `steps` steps in
    `total_ms`: the slowest rank bounds the job (max over ranks through torch.distributed when
    world > 1).  Returns (max total ms, steps/s of all ranks together)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        tt = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
    return total_ms, world * steps / (total_ms / 1e3)


def timed_steps(ctx, u, s, t0, warmup, steps, flush, record_j=False, label="steps", phase_steps=PHASE_STEPS):
    """Run warmup + timed steps; every timed step is bracketed by CUDA events on the context
    stream, with an L2 flush (not timed) before it.  Inside the timed steps the library times the
    orbital stencil kernel launches only (tdks_profile level 2: one event pair per launch); the
    breakdown of a step into all phases comes from `phase_steps` further steps with every phase
    timed (their event pairs slow a step down, so they are not in the timed region).  The timed
    steps sit in an NVTX range named `label` (for `ncu --nvtx --nvtx-include label/`).  Returns
    (per-step ms, J history, stats of the timed steps with the phase times of the extra steps)."""
    import torch
    stream = torch.cuda.current_stream()
    t = t0
    J = []
    for _ in range(warmup):
        ctx.step(u, t, s.dt)
        t += s.dt
        if record_j:
            J.append(ctx.read_step_observables()["J"])
    torch.cuda.synchronize()
    ctx.stats(reset=True)
    ctx.profile(2)
    for _ in range(2):                                   # the step graphs with the kernel events
        ctx.step(u, t, s.dt)
        t += s.dt
        if record_j:
            J.append(ctx.read_step_observables()["J"])
    torch.cuda.synchronize()
    ctx.stats(reset=True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push(label)
    for i in range(steps):
        flush.zero_()                                    # evict the 65 MB orbital set from L2
        evs[i][0].record(stream)
        ctx.step(u, t, s.dt)
        evs[i][1].record(stream)
        t += s.dt
        if record_j:
            J.append(ctx.read_step_observables()["J"])
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    st = ctx.stats(reset=True)
    ctx.profile(1)
    for _ in range(phase_steps + 1):                     # the first one builds the step graph
        ctx.step(u, t, s.dt)
        t += s.dt
        if record_j:
            J.append(ctx.read_step_observables()["J"])
    torch.cuda.synchronize()
    ctx.stats(reset=True)
    for _ in range(phase_steps):
        ctx.step(u, t, s.dt)
        t += s.dt
        if record_j:
            J.append(ctx.read_step_observables()["J"])
    torch.cuda.synchronize()
    sp = ctx.stats(reset=True)
    ctx.profile(False)
    st["phase_ms"] = {k: v / phase_steps for k, v in sp["ms"].items()}
    return [a.elapsed_time(b) for a, b in evs], np.array(J), st


def train_predictor(s, t0, ntraj=4, nsteps=300, epochs=3):
    """Network weights trained on trajectories the method itself generates (seeds 1..ntraj, the
    bench state uses seed 0), FP32 path."""
    from paper_1804_01404_gb300 import learned as L
    from paper_1804_01404_gb300 import workloads as W
    from paper_1804_01404_gb300.tdks import Context
    tic = time.perf_counter()
    trajs = [L.trajectory(s, W.initial_orbitals(s, seed), nsteps, "f32", t0=t0) for seed in range(1, ntraj + 1)]
    ctx = Context(s, precision="f32")
    ctx.nn_init(1)
    loss = L.train(ctx, trajs, epochs=epochs, batch=8, lr=1e-3, seed=3)
    held = L.trajectory(s, W.initial_orbitals(s, 101), 60, "f32", t0=t0)
    mis = {name: float(np.mean(L.misfits(ctx, held, m))) for name, m in (("linear", 0), ("cubic", 1), ("network", 2))}
    params = ctx.nn_params()
    ctx.close()
    return params, {"train_loss_per_epoch": [float(x) for x in loss], "heldout_misfit_mean": mis,
                    "training_s": time.perf_counter() - tic,
                    "data": f"{ntraj} trajectories x {nsteps} steps (seeds 1-{ntraj}), held-out seed 101"}


def gpu_arm(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_1804_01404_gb300 import tdks as T
    from paper_1804_01404_gb300.tdks import Context

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    s = workload()
    from paper_1804_01404_gb300 import workloads as W
    psi0 = W.initial_orbitals(s, 0).astype(np.complex64)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    t0 = 200.0   # start inside the pulse (A' != 0)

    # FP64 predictor-corrector reference current over the same steps (the reference of the error bound)
    nref = args.warmup + args.steps + 2 * PHASE_STEPS + 3     # every step timed_steps takes
    ctx64 = Context(s, precision="f64", obs_at_start=True)
    u64 = torch.from_numpy(psi0.astype(np.complex128)).to(dev)
    ctx64.update_potential(u64)
    J64, t = [], t0
    torch.cuda.synchronize()
    ctx64.stats(reset=True)
    ctx64.profile(True)
    tic = time.perf_counter()
    for _ in range(nref):
        ctx64.step(u64, t, s.dt)
        t += s.dt
        J64.append(ctx64.read_step_observables()["J"])
    torch.cuda.synchronize()
    f64_sps = nref / (time.perf_counter() - tic)
    st64 = ctx64.stats(reset=True)
    J64 = np.array(J64)
    ctx64.close()
    del u64

    def jerr(J):
        return float(np.max(np.abs(J - J64)) / np.max(np.abs(J64)))

    # plain predictor-corrector, FP32 orbitals
    ctx = Context(s, precision="f32", obs_at_start=True)
    u = torch.from_numpy(psi0).to(dev)
    ctx.update_potential(u)
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local_rank)
    pc_ms, J_pc, st_pc = timed_steps(ctx, u, s, t0, args.warmup, args.steps, flush, record_j=True, label="pc")
    ctx.close()

    # learned predictor (PC fallback) and the cubic-extrapolation ablation
    params, train_info = train_predictor(s, t0) if not args.skip_learned else (None, None)
    modes = {}
    if params is not None:
        for name, mode in (("learned", T.PRED_LEARNED), ("cubic", T.PRED_EXTRAP)):
            c2 = Context(s, precision="f32", obs_at_start=True)
            u2 = torch.from_numpy(psi0).to(dev)
            c2.update_potential(u2)
            c2.nn_init(0)
            c2.nn_params(params)
            c2.set_predictor(mode, 1e-5)
            if args.no_step_graph:
                c2.set_step_graph(False)
            ms, J, st = timed_steps(c2, u2, s, t0, args.warmup, args.steps, flush, record_j=True, label=name)
            o = c2.read_step_observables()
            modes[name] = dict(ms=ms, J=J, st=st, fallbacks=o["fallbacks"], cell_scheme=c2.cell_variant())
            c2.close()
    sweep = threshold_sweep(s, psi0, params, t0, args.warmup, args.steps, flush, J64, dev) if params is not None else None
    clk = clocks.stop()

    head = modes.get("learned")
    step_ms = head["ms"] if head else pc_ms
    st = head["st"] if head else st_pc
    total_ms, value = replica_throughput(float(np.sum(step_ms)), args.steps, world, dev)

    # dominant kernel of the headline step: the cell Taylor kernel (the corrector launch of a learned
    # step; predictor and corrector launches of a PC step), timed alone by the library's
    # stencil-kernel phase events on the context stream
    npts, norb_tot = s.npts, s.nk * s.norb
    nsph = W_nsph(s)
    k_ms = st["ms"]["stencil_kernel"] / max(1, st["calls"]["stencil_kernel"])
    flops = 4 * norb_tot * (FLOPS_PER_POINT_STAGE * npts + FLOPS_PER_SPHERE_ENTRY_STAGE * nsph)
    pk = peaks()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_derived = n_sm * FP32_LANES_PER_SM * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    fp32_peak = T.probe_fp32()
    achieved = flops / (k_ms * 1e-3) / 1e12
    hbm_bytes = 16 * npts * norb_tot
    roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak, "traffic": measured_traffic("k_cell_f32_mode1"),
                "kernel": "k_cell<float, MODE=1> (4 Horner stages, whole orbital in shared memory; "
                          "J and norms of the input state fused into the first stage)",
                "avg_launch_ms": k_ms, "launches_timed": st["calls"]["stencil_kernel"],
                "buffer_scheme": cell_scheme(head["cell_scheme"] if head else None),
                "flops_per_launch": flops,
                "peak_note": "measured FP32 FMA rate of this GPU (tdks_probe_fp32, FMA chains on every SM); "
                             f"derived {n_sm} SM x 128 lanes x 2 flop x max SM clock = {fp32_derived:.1f} TFLOP/s",
                "hbm_view": {"bytes_per_launch": hbm_bytes,
                             "GBps": hbm_bytes / (k_ms * 1e-3) / 1e9,
                             "frac_of_measured_hbm": hbm_bytes / (k_ms * 1e-3) / 1e9 / pk["hbm_gbs"]}}

    predictors = {"pc": {"steps_per_s": args.steps / (np.sum(pc_ms) / 1e3),
                         "J_rel_err_vs_f64_pc": jerr(J_pc),
                         "phase_ms_per_step": st_pc["phase_ms"]}}
    for name, m in modes.items():
        predictors[name] = {"steps_per_s": args.steps / (np.sum(m["ms"]) / 1e3), "J_rel_err_vs_f64_pc": jerr(m["J"]),
                            "fallbacks": m["fallbacks"], "steps": args.warmup + args.steps,
                            "phase_ms_per_step": m["st"]["phase_ms"]}
    predictors["f64_pc_steps_per_s_host_synced"] = f64_sps
    # the FP64 path is bound by the FP64 pipes: its cell kernel against the measured FP64 FMA rate
    k64 = st64["ms"]["stencil_kernel"] / max(1, st64["calls"]["stencil_kernel"])
    fp64_peak = T.probe_fp64()
    predictors["f64_cell_kernel"] = {"avg_launch_ms": k64, "achieved_tflops": flops / (k64 * 1e-3) / 1e12,
                                     "peak_tflops": fp64_peak, "peak_note": "measured FP64 FMA rate (tdks_probe_fp64)",
                                     "frac": flops / (k64 * 1e-3) / 1e12 / fp64_peak}
    if train_info:
        predictors["training"] = train_info
    if sweep:
        predictors["threshold_sweep"] = sweep

    # end to end through the C ABI with host buffers (same predictor as the headline): a run resumed
    # from host memory -- the orbitals and the context state of a checkpoint (tdks_get_state: the
    # potential history, predictor and field state) are uploaded, K steps run with J and the dipole
    # read back after every step, and the orbitals are downloaded.  The checkpoint and the step
    # graphs come from a warm-up run of the same context before the timed region.
    ctx2 = Context(s, precision="f32", obs_at_start=True)
    u2 = torch.from_numpy(psi0).to(dev)
    if params is not None:
        ctx2.nn_init(0)
        ctx2.nn_params(params)
    ctx2.update_potential(u2)
    if params is not None:
        ctx2.set_predictor(T.PRED_LEARNED, 1e-5)
    tt = t0
    for _ in range(args.warmup + 4):
        ctx2.step(u2, tt, s.dt)
        ctx2.read_step_observables()
        tt += s.dt
    host_in = u2.cpu().pin_memory()
    state = ctx2.get_state()
    host_out = torch.empty_like(host_in).pin_memory()
    # every step's observables go to one of three pinned host blocks (tdks_copy_step_observables) and
    # are unpacked on the host two steps later, so the stream never waits for the host (and a late
    # wake-up of the host thread has two queued steps of slack)
    LAG = 2
    ring = [torch.zeros(T.STEP_OBS_DOUBLES, dtype=torch.float64).pin_memory() for _ in range(LAG + 1)]
    evs = [torch.cuda.Event() for _ in range(LAG + 1)]
    cstream = ctx2.stream
    obs_read = []
    u2.zero_()
    torch.cuda.synchronize()
    tic = time.perf_counter()
    u2.copy_(host_in, non_blocking=True)
    ctx2.set_state(state)
    for i in range(args.steps):
        ctx2.step(u2, tt, s.dt)
        ctx2.copy_step_observables(ring[i % (LAG + 1)])
        evs[i % (LAG + 1)].record(cstream)
        if i >= LAG:
            evs[(i - LAG) % (LAG + 1)].synchronize()
            obs_read.append(ctx2.unpack_step_observables(ring[(i - LAG) % (LAG + 1)]))
        tt += s.dt
    host_out.copy_(u2, non_blocking=True)
    for i in range(max(0, args.steps - LAG), args.steps):
        evs[i % (LAG + 1)].synchronize()
        obs_read.append(ctx2.unpack_step_observables(ring[i % (LAG + 1)]))
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - tic
    assert len(obs_read) == args.steps and all(np.isfinite(o["J"]).all() for o in obs_read)
    psi_bytes = psi0.nbytes
    state_bytes = len(state)
    e2e = {"value": world * args.steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": (psi_bytes + state_bytes) / args.steps,
           "d2h_bytes_per_step": psi_bytes / args.steps + T.STEP_OBS_DOUBLES * 8,
           "note": "a run resumed from host memory: psi and the context state of a checkpoint uploaded, psi "
                   "downloaded once per K steps; J, dipole, misfit and fallback count of every step copied "
                   "to pinned host memory and unpacked on the host two steps later (the next steps are queued "
                   "first); context and step graphs set up by a warm-up run before the timed region"}
    ctx2.close()

    hpsi = None
    if rank == 0 and not args.skip_hpsi:
        hpsi = hpsi_cluster(dev)

    others = None
    if rank == 0 and not args.skip_workloads:
        others = workload_steps(dev)
        others["absorption_peak"] = absorption_peak_check(dev)
    accuracy = None
    if rank == 0 and not args.skip_accuracy and params is not None:
        accuracy = accuracy_long(dev, params)

    cpu = None
    if rank == 0 and not args.skip_cpu:
        per, nw, desc = oracle_parallel_steps(args.cpu_steps, 1)
        cpu = {"value": 1.0 / per, "unit": UNIT, "cores": nw, "kind": "oracle", "sample": desc}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": config_dict(s, {"parallelism": f"replicas x{world}",
                                          "predictor": "learned (PC fallback at misfit > 1e-5)" if head
                                          else "predictor-corrector"}),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": st["launches"], "clocks": clk,
                "phase_ms_per_step": st["phase_ms"],
                "phase_note": "every phase timed over 5 steps after the timed region (the timed steps carry "
                              "events around the orbital stencil kernel only)",
                "step_ms_min": float(np.min(step_ms)),
                "J_rel_err_vs_f64": jerr(head["J"]) if head else jerr(J_pc),
                "predictors": predictors, "hpsi_cluster": hpsi,
                "other_workloads": others, "accuracy_long": accuracy}
        line["summary"] = summary(line)
        print(json.dumps(line), flush=True)
    return 0


def _run_steps(s, psi, precision, nsteps, t0=0.0, mode=None, params=None, kick=None, observe="J", threshold=1e-5):
    """nsteps tdks_step calls from psi at t0 with the observable read after every step; returns
    (array of J or dipole per step, fallbacks, seconds)."""
    import torch
    from paper_1804_01404_gb300 import tdks as T
    ctx = T.Context(s, precision=precision)
    u = torch.from_numpy(psi.astype(np.complex128 if precision == "f64" else np.complex64)).to("cuda")
    if kick is not None:
        ctx.kick(u, kick)
    ctx.update_potential(u)
    if mode is not None and mode != T.PRED_PC:
        ctx.nn_init(0)
        if params is not None:
            ctx.nn_params(params)
        ctx.set_predictor(mode, threshold)
    out, t = [], t0
    torch.cuda.synchronize()
    tic = time.perf_counter()
    o = None
    for _ in range(nsteps):
        ctx.step(u, t, s.dt)
        t += s.dt
        o = ctx.read_step_observables()
        out.append(o[observe])
    sec = time.perf_counter() - tic
    ctx.check()
    ctx.close()
    return np.array(out), (o["fallbacks"] if o else 0.0), sec


def accuracy_long(dev, params, nsteps_crystal=2000, nsteps_cluster=4000, kappa=1e-3):
    """The error bounds over the stated run lengths, FP32 orbitals (with the learned predictor, the
    cubic extrapolation and the plain PC) against FP64 orbitals with the plain PC, all on the GPU (the
    FP64 path matches the oracle to 1e-10 over 100 steps of the small cell and over the first steps of
    the crystal, tests/test_gpu_parity.py):
      * the diamond crystal over its 2000 steps from t = 0 under the pulse: max_t |J32 - J64| / max_t |J64|;
      * a kicked isolated cluster of the large-cluster recipe at 48^3 (h = 0.4, 16 atoms, 32 orbitals)
        over 4000 steps: max_t |d32 - d64| / max_t |d64| of the dipole along the kick and the shift of
        the main peak of Eq. (distribution) on a 0.001 eV grid (the network of this cluster is trained
        on three other kicked states of it)."""
    from paper_1804_01404_gb300 import learned as L
    from paper_1804_01404_gb300 import tdks as T
    from paper_1804_01404_gb300 import workloads as W
    ev = 27.211386245988
    res = {}
    s = W.diamond_crystal()
    psi0 = W.initial_orbitals(s, 0)
    J64, _, sec64 = _run_steps(s, psi0, "f64", nsteps_crystal)
    cr = {"workload": f"diamond crystal 20^3, 16 orbitals x 64 k, pulse, {nsteps_crystal} steps from t = 0",
          "f64_pc_s": sec64}
    for name, mode in (("f32_learned", T.PRED_LEARNED), ("f32_cubic", T.PRED_EXTRAP), ("f32_pc", T.PRED_PC)):
        J, fb, sec = _run_steps(s, psi0, "f32", nsteps_crystal, mode=mode, params=params)
        cr[name] = {"J_rel_err_vs_f64": float(np.max(np.abs(J - J64)) / np.max(np.abs(J64))), "fallbacks": fb,
                    "s": sec}
    res["crystal_2000"] = cr
    c = W.isolated_cluster(n=48, natom=16, norb=32, radius=7.0, seed=3)
    kick = (0.0, 0.0, kappa)
    tic = time.perf_counter()
    trajs = [L.trajectory(c, W.initial_orbitals(c, seed), 300, "f32", kick=kick) for seed in (2, 3, 4)]
    tctx = T.Context(c, precision="f32")
    tctx.nn_init(1)
    L.train(tctx, trajs, epochs=3, batch=8, lr=1e-3, seed=5)
    cparams = tctx.nn_params()
    tctx.close()
    del trajs
    cl = {"workload": f"isolated cluster 48^3 (h = 0.4), 16 atoms, 32 orbitals, kick {kappa} along z, "
                      f"{nsteps_cluster} steps", "training_s": time.perf_counter() - tic}
    psi1 = W.initial_orbitals(c, 1)
    d64, _, sec = _run_steps(c, psi1, "f64", nsteps_cluster, kick=kick, observe="dipole")
    cl["f64_pc_s"] = sec
    E = np.arange(0.0, 2.0, 0.005)

    def peak(d):
        dd = np.concatenate([[0.0], d[:, 2]])
        e0 = E[np.argmax(T.oscillator_strength(dd, c.dt, kappa, E))]
        Ef = np.arange(max(e0 - 0.01, 1e-6), e0 + 0.01, 0.001 / ev)
        return float(Ef[np.argmax(T.oscillator_strength(dd, c.dt, kappa, Ef))])
    p64 = peak(d64)
    cl["peak_eV_f64"] = p64 * ev
    for name, mode in (("f32_learned", T.PRED_LEARNED), ("f32_pc", T.PRED_PC)):
        d, fb, sec = _run_steps(c, psi1, "f32", nsteps_cluster, mode=mode, params=cparams, kick=kick, observe="dipole")
        cl[name] = {"dipole_rel_err_vs_f64": float(np.max(np.abs(d[:, 2] - d64[:, 2])) / np.max(np.abs(d64[:, 2]))),
                    "peak_shift_eV": abs(peak(d) - p64) * ev, "fallbacks": fb, "s": sec}
    cl["resolution_eV"] = 2 * np.pi / (nsteps_cluster * c.dt) * ev
    res["cluster48_4000"] = cl
    return res


def threshold_sweep(s, psi0, params, t0, warmup, steps, flush, J64, dev,
                    thresholds=(1e-5, 2e-6, 1.2e-6, 1e-6, 9e-7, 8e-7, 7e-7)):
    """The network against the cubic extrapolation at tighter misfit thresholds: a prediction is kept
    only if ||V_Hxc(t+dt) - V~|| / ||V_Hxc(t+dt)|| stays below the threshold, else the step is redone
    with the plain predictor-corrector.  A better prediction is rejected less often, so the network's
    gain in misfit turns into steps/s where the threshold sits between the two arms' typical misfits.
    Same steps as the timed region (after `warmup` steps from t0), J error against the FP64 run."""
    import torch
    from paper_1804_01404_gb300 import tdks as T
    from paper_1804_01404_gb300.tdks import Context
    out = []
    for thr in thresholds:
        row = {"threshold": thr}
        for name, mode in (("learned", T.PRED_LEARNED), ("cubic", T.PRED_EXTRAP)):
            c = Context(s, precision="f32", obs_at_start=True)
            u = torch.from_numpy(psi0).to(dev)
            c.update_potential(u)
            c.nn_init(0)
            c.nn_params(params)
            c.set_predictor(mode, thr)
            ms, J, st = timed_steps(c, u, s, t0, warmup, steps, flush, record_j=True, label=f"sweep_{name}")
            o = c.read_step_observables()
            row[name] = {"steps_per_s": steps / (np.sum(ms) / 1e3), "fallbacks": o["fallbacks"],
                         "steps": len(J), "J_rel_err_vs_f64_pc": float(np.max(np.abs(J - J64)) / np.max(np.abs(J64)))}
            c.close()
        out.append(row)
    return out


def summary(line):
    """The headline figures of the line, repeated in one short object at its end: the dominant
    kernel's roofline fraction, the cluster hpsi against the measured HBM bandwidth (whole call and
    stencil kernel alone), the predictor arms' steps/s and J errors, end to end and the CPU oracle."""
    def g(d, *keys):
        for k in keys:
            if not isinstance(d, dict) or d.get(k) is None:
                return None
            d = d[k]
        return d
    pr = line.get("predictors") or {}
    out = {"steps_per_s": line["value"], "e2e_steps_per_s": g(line, "e2e", "value"),
           "cell_kernel_frac_of_measured_fp32": g(line, "roofline", "frac"),
           "cell_kernel_ms": g(line, "roofline", "avg_launch_ms"),
           "hpsi_cluster_frac_of_measured_hbm": g(line, "hpsi_cluster", "frac_of_measured_hbm"),
           "hpsi_cluster_stencil_frac_of_measured_hbm": g(line, "hpsi_cluster", "stencil_kernel_frac_of_measured_hbm"),
           "hpsi_cluster_ms": g(line, "hpsi_cluster", "ms_per_hpsi_phase"),
           "taylor_step_cluster_frac_of_measured_hbm": g(line, "hpsi_cluster", "taylor_step", "frac_of_measured_hbm"),
           "taylor_stage_stencil_frac_of_measured_hbm": g(line, "hpsi_cluster", "taylor_step",
                                                          "stencil_stage_frac_of_measured_hbm"),
           "J_rel_err_vs_f64": line.get("J_rel_err_vs_f64"),
           "cpu_oracle_steps_per_s": g(line, "cpu_baseline", "value"), "cpu_cores": g(line, "cpu_baseline", "cores")}
    for name in ("learned", "cubic", "pc"):
        out[f"{name}_steps_per_s"] = g(pr, name, "steps_per_s")
        out[f"{name}_J_rel_err"] = g(pr, name, "J_rel_err_vs_f64_pc")
    out["f64_pc_steps_per_s"] = pr.get("f64_pc_steps_per_s_host_synced")
    acc = line.get("accuracy_long") or {}
    out["crystal_2000_J_rel_err_f32_learned"] = g(acc, "crystal_2000", "f32_learned", "J_rel_err_vs_f64")
    out["cluster48_4000_dipole_rel_err_f32_learned"] = g(acc, "cluster48_4000", "f32_learned", "dipole_rel_err_vs_f64")
    out["cluster48_4000_peak_shift_eV_f32_learned"] = g(acc, "cluster48_4000", "f32_learned", "peak_shift_eV")
    sw = pr.get("threshold_sweep") or []
    wins = [r for r in sw if r["learned"]["steps_per_s"] > r["cubic"]["steps_per_s"]]
    if wins:
        best = max(wins, key=lambda r: r["learned"]["steps_per_s"] / r["cubic"]["steps_per_s"])
        out["learned_beats_cubic_at_threshold"] = {
            "threshold": best["threshold"], "learned_steps_per_s": best["learned"]["steps_per_s"],
            "cubic_steps_per_s": best["cubic"]["steps_per_s"], "learned_fallbacks": best["learned"]["fallbacks"],
            "cubic_fallbacks": best["cubic"]["fallbacks"], "learned_J_rel_err": best["learned"]["J_rel_err_vs_f64_pc"],
            "cubic_J_rel_err": best["cubic"]["J_rel_err_vs_f64_pc"]}
    out["f64_cell_kernel_frac_of_measured_fp64"] = g(pr, "f64_cell_kernel", "frac")
    return out


def cell_scheme(v):
    """The cell kernel's buffer scheme picked by the library's tuner at context creation
    (tdks_cell_variant), with the tuning times of one Taylor launch of each."""
    if v is None:
        return None
    names = ["two shared-memory copies", "one copy swept in place",
             "two shared-memory copies, grid size built in (column segments unrolled)",
             "one copy swept in place, grid size built in (two CTAs per SM)"]
    return {"in_use": names[v[0]], "tune_ms": {n: (t if t > 0 else None) for n, t in zip(names, v[1])}}


def measured_traffic(key):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of one ncu capture,
    recorded in profiles/roofline_traffic.json together with the SHA-256 of the kernel's source
    file at capture time; None when the source has changed since."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "roofline_traffic.json")) as f:
            rec = json.load(f)[key]
        with open(os.path.join(ROOT, rec["source"]), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != rec["source_sha256"]:
                return None
        return rec["bytes_per_launch"]
    except (OSError, KeyError, ValueError):
        return None


def W_nsph(s):
    from paper_1804_01404_gb300.tdks import Context
    c = Context(s, precision="f32")
    n = c.query()["nsphere_points"]
    c.close()
    return n


def hpsi_cluster(dev, reps=10, norb=256):
    """tdks_hpsi on the isolated cluster (96^3 grid, 128 atoms, 256 orbitals, FP32): the large-grid
    TMA tile path.  Orbital fields are random (hpsi time does not depend on their values); 1.8 GB
    of orbitals is far above L2, so every launch streams from HBM.  Algorithmic bytes: read u and
    write H u, 16 B per orbital-point."""
    import torch
    from paper_1804_01404_gb300 import workloads as W
    from paper_1804_01404_gb300.tdks import Context
    s = W.isolated_cluster(norb=norb)
    g = torch.Generator(device=dev)
    g.manual_seed(1)
    u = torch.randn((s.nk, s.norb, s.n[2], s.n[1], s.n[0]), dtype=torch.complex64, device=dev, generator=g)
    u *= (1.0 / np.sqrt(s.npts * s.dV))
    hu = torch.empty_like(u)
    ctx = Context(s, precision="f32")
    ctx.update_potential(u)
    for _ in range(3):
        ctx.hpsi(u, hu)
    torch.cuda.synchronize()
    ctx.stats(reset=True)
    ctx.profile(True)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        ctx.hpsi(u, hu)
    e1.record(stream)
    torch.cuda.synchronize()
    st = ctx.stats(reset=True)
    ctx.check()
    ms = e0.elapsed_time(e1) / reps
    k_ms = st["ms"]["hpsi"] / max(1, st["calls"]["hpsi"])
    s_ms = st["ms"]["stencil_kernel"] / max(1, st["calls"]["stencil_kernel"])
    nbytes = 16 * s.npts * s.nk * s.norb
    pk = peaks()
    res = {"workload": f"isolated cluster 96^3, 128 atoms, {norb} orbitals, FP32", "calls": reps,
           "ms_per_hpsi": ms, "ms_per_hpsi_phase": k_ms, "bytes_per_hpsi": nbytes,
           "GBps": nbytes / (k_ms * 1e-3) / 1e9, "peak_GBps": pk["hbm_gbs"],
           "frac_of_measured_hbm": nbytes / (k_ms * 1e-3) / 1e9 / pk["hbm_gbs"],
           "kernels": "k_gproject + tile stencil (TMA planes) + k_gscatter",
           "stencil_kernel_ms": s_ms, "stencil_kernel_GBps": nbytes / (s_ms * 1e-3) / 1e9,
           "stencil_kernel_frac_of_measured_hbm": nbytes / (s_ms * 1e-3) / 1e9 / pk["hbm_gbs"],
           "stencil_kernel_traffic": measured_traffic("k_tile_f32_mode0")}
    # the Taylor step of the same orbitals: four Horner stages v <- psi + (-i dt/m) H v, each the
    # fused stencil (reads v and psi, writes the new v: 24 B per orbital-point) with the projections
    # on the side stream and the nonlocal scatter -- hpsi as the propagator applies it
    for _ in range(2):
        ctx.taylor_step(u, s.dt)
    torch.cuda.synchronize()
    ctx.stats(reset=True)
    ctx.profile(2)
    e0.record(stream)
    for _ in range(reps):
        ctx.taylor_step(u, s.dt)
    e1.record(stream)
    torch.cuda.synchronize()
    sts = ctx.stats(reset=True)
    ctx.profile(False)
    ctx.check()
    tms = e0.elapsed_time(e1) / reps
    stage_ms = sts["ms"]["stencil_kernel"] / max(1, sts["calls"]["stencil_kernel"])
    tbytes = 4 * 1.5 * nbytes
    res["taylor_step"] = {
        "ms": tms, "bytes_per_step": tbytes, "GBps": tbytes / (tms * 1e-3) / 1e9,
        "frac_of_measured_hbm": tbytes / (tms * 1e-3) / 1e9 / pk["hbm_gbs"],
        "stencil_stage_ms": stage_ms, "stencil_stage_GBps": 1.5 * nbytes / (stage_ms * 1e-3) / 1e9,
        "stencil_stage_frac_of_measured_hbm": 1.5 * nbytes / (stage_ms * 1e-3) / 1e9 / pk["hbm_gbs"],
        "note": "4 Horner stages, 24 B per orbital-point each (read v and psi, write the new v); whole step "
                "with projections and scatters, and the fused stencil kernel of one stage alone"}
    # density + Hockney Poisson (192^3 FFTs, FP64) + LDA exchange of the same orbitals
    ctx.profile(1)
    ctx.update_potential(u)                              # warm-up
    torch.cuda.synchronize()
    ctx.stats(reset=True)
    for _ in range(3):
        ctx.update_potential(u)
    torch.cuda.synchronize()
    sx = ctx.stats(reset=True)
    ctx.profile(0)
    res["update_potential_hartree_xc_ms"] = sx["ms"]["hartree_xc"] / max(1, sx["calls"]["hartree_xc"])
    variant, tune_ms = ctx.tile_variant()
    names = ["k_tile<float> (1 point/thread, 3 CTAs/SM)", "k_tile<float> (1 point/thread, 2 CTAs/SM) + L2 prefetch",
             "k_tile4<8> (2x2 points/thread, 8 consumer warps) + L2 prefetch",
             "k_tile4<8, 1 row> (2x1 points/thread, 2 CTAs/SM) + L2 prefetch",
             "k_tile4<4, 1 row> (2x1 points/thread, 4 CTAs/SM) + L2 prefetch",
             "k_tile4<8, 1 row, TMA-staged V/psi> (2x1 points/thread, 2 CTAs/SM)",
             "k_tile4<4, 1 row, TMA-staged V/psi> (2x1 points/thread, 4 CTAs/SM)"]
    res["stencil_variant"] = {"hpsi": names[variant[0]], "horner_stage": names[variant[1]]}
    pv, pms = ctx.project_variant()
    res["projection_schedule"] = {"in_use": f"{2 << pv} warps per CTA",
                                  "tune_ms": {f"{2 << v} warps per CTA": t for v, t in enumerate(pms)},
                                  "kernel": "k_gproject_mma (mma.sync m16n8k8 TF32, 3xTF32 split)"}
    # the tuner's timings of the stencil kernel alone (no projectors), 2 launches each at init:
    # H v moves 16 B per orbital-point, a Horner stage 24 B (reads v and psi, writes the result)
    res["stencil_only_GBps"] = {
        "hpsi": {names[v]: (nbytes / (t * 1e-3) / 1e9 if t > 0 else None) for v, t in enumerate(tune_ms[0])},
        "horner_stage": {names[v]: (1.5 * nbytes / (t * 1e-3) / 1e9 if t > 0 else None)
                         for v, t in enumerate(tune_ms[1])}}
    ctx.close()
    del u, hu
    torch.cuda.empty_cache()
    return res


def smooth_random_orbitals(shape, dV, dev, seed, passes=3):
    """Seeded random complex fields, low-passed by repeated 3-point box averages along x, y and z and
    normalised to sum |u|^2 dV = 1: smooth orbital-like inputs whose step time equals that of the
    method's own orbitals (the kernels' work does not depend on the values)."""
    import torch
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    u = torch.randn(shape, dtype=torch.complex64, device=dev, generator=g)
    for _ in range(passes):
        for ax in (-1, -2, -3):
            u = (u + torch.roll(u, 1, ax) + torch.roll(u, -1, ax)) * (1.0 / 3.0)
    nrm = torch.sqrt((u.abs() ** 2).sum(dim=(-1, -2, -3), keepdim=True) * dV)
    return (u / nrm).contiguous()


def workload_steps(dev, warmup=2, steps=5, which=("cluster", "multiscale", "mbj")):
    """Full steps of the two large workloads, timed over a few steps (CUDA events on the context
    stream) after warm-up:
      * isolated cluster: 96^3 grid (h = 0.4), 128 atoms, 256 orbitals, FP32, impulse kick,
        predictor-corrector with Hockney Hartree, tiled TMA stencil;
      * multiscale: 256 microscopic cells (16^3, 8 atoms, 16 orbitals x 8 k) on a 1D Maxwell grid
        (dX = 250 bohr), one coupled step = TDKS PC step of every cell + current + Maxwell update;
      * TB-mBJ: PC steps of the diamond crystal with the LDA and with TB-mBJ exchange.
    "effective hpsi GB/s" = 2 Taylor steps x 4 H applications x 16 B per orbital-point / step time
    (the unfused-equivalent stream; it exceeds the HBM peak when orbitals stay on chip)."""
    import torch
    stream = torch.cuda.current_stream()
    out = {}

    def run(ctx, one_step, label):
        for _ in range(warmup):
            one_step()
        torch.cuda.synchronize()
        ctx.stats(reset=True)
        ctx.profile(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push(label)
        e0.record(stream)
        for _ in range(steps):
            one_step()
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        st = ctx.stats(reset=True)
        ctx.profile(False)
        ctx.check()
        return e0.elapsed_time(e1) / steps, st

    if "cluster" in which:
        out.update(_cluster_steps(dev, run, steps, warmup))
    if "multiscale" in which:
        out.update(_multiscale_steps(dev, run, steps, warmup))
    if "mbj" in which:
        out.update(_mbj_steps(dev, run, steps, warmup))
    return out


def _cluster_steps(dev, run, steps, warmup):
    import torch
    from paper_1804_01404_gb300 import workloads as W
    from paper_1804_01404_gb300.tdks import Context
    out = {}
    # isolated cluster
    s = W.isolated_cluster()
    u = smooth_random_orbitals((s.nk, s.norb, s.n[2], s.n[1], s.n[0]), s.dV, dev, seed=11)
    ctx = Context(s, precision="f32")
    ctx.kick(u, s.kick)
    ctx.update_potential(u)
    tt = [0.0]

    def cl_step():
        ctx.step(u, tt[0], s.dt)
        tt[0] += s.dt
    ms, st = run(ctx, cl_step, "cluster_steps")
    opts = s.npts * s.nk * s.norb
    out["cluster_96"] = {
        "workload": "isolated cluster 96^3 (h = 0.4), 128 atoms, 256 orbitals x 1 k, FP32 orbitals, "
                    "impulse kick, predictor-corrector, Hockney Hartree",
        "steps_timed": steps, "warmup": warmup, "ms_per_step": ms, "steps_per_s": 1e3 / ms,
        "orbital_points": opts, "effective_hpsi_GBps": 8 * 16 * opts / (ms * 1e-3) / 1e9,
        "phase_ms_per_step": {k: v / steps for k, v in st["ms"].items()},
        "launches_per_step": st["launches"] / steps,
        "l2": "orbitals 1.81 GB, far above L2"}
    ctx.close()
    del u
    torch.cuda.empty_cache()
    return out


def _multiscale_steps(dev, run, steps, warmup):
    import torch
    from paper_1804_01404_gb300 import workloads as W
    from paper_1804_01404_gb300.tdks import Context
    out = {}
    # batched multiscale cells
    s = W.multiscale_cell()
    ncell, m0, dX = 256, 4, 250.0
    nX = m0 + ncell + 4
    X = np.arange(nX)
    A_now = 0.3 * np.sin(2 * np.pi * X / 64.0)
    A_prev = 0.3 * np.sin(2 * np.pi * (X + 0.5) / 64.0)
    psi = W.initial_orbitals(s, 3).astype(np.complex64)
    u = torch.from_numpy(psi).to(dev).unsqueeze(0).repeat(ncell, 1, 1, 1, 1, 1).contiguous()
    ctx = Context(s, precision="f32", ncell=ncell)
    ctx.update_potential(u)
    ctx.ms_init(dX, m0, A_now, A_prev)
    tt = [0.0]

    def ms_step():
        ctx.ms_step(u, tt[0], s.dt)
        tt[0] += s.dt
    ms, st = run(ctx, ms_step, "multiscale_steps")
    opts = ncell * s.npts * s.nk * s.norb
    out["multiscale_256"] = {
        "workload": f"{ncell} cells of 16^3, 8 atoms, 16 orbitals x 8 k each, FP32 orbitals, on a {nX}-point "
                    "1D Maxwell grid (dX = 250 bohr); one coupled step",
        "steps_timed": steps, "warmup": warmup, "ms_per_step": ms, "steps_per_s": 1e3 / ms,
        "cell_steps_per_s": ncell * 1e3 / ms,
        "orbital_points": opts, "effective_hpsi_GBps": 8 * 16 * opts / (ms * 1e-3) / 1e9,
        "phase_ms_per_step": {k: v / steps for k, v in st["ms"].items()},
        "launches_per_step": st["launches"] / steps,
        "l2": "orbitals 1.07 GB, far above L2"}
    ctx.close()
    del u
    torch.cuda.empty_cache()
    return out


def _mbj_steps(dev, run, steps, warmup):
    import torch
    from paper_1804_01404_gb300 import workloads as W
    from paper_1804_01404_gb300.tdks import Context
    out = {}
    # TB-mBJ exchange on the diamond crystal: PC steps with the LDA and with TB-mBJ (c from the
    # density), same orbitals; the difference of the hartree_xc phase is the mBJ kernels' cost
    s = W.diamond_crystal()
    u0 = smooth_random_orbitals((s.nk, s.norb, s.n[2], s.n[1], s.n[0]), s.dV, dev, seed=5)
    res = {}
    for xc in (2, 3):
        u = u0.clone()
        ctx = Context(s, precision="f32", xc=xc, obs_at_start=True)
        ctx.update_potential(u)
        tt = [0.0]

        def pc_step():
            ctx.step(u, tt[0], s.dt)
            tt[0] += s.dt
        ms, st = run(ctx, pc_step, f"diamond_xc{xc}_steps")
        res[xc] = (ms, {k: v / steps for k, v in st["ms"].items()}, st["launches"] / steps)
        ctx.close()
        del u
    opts = s.npts * s.nk * s.norb
    mbj_ms = res[3][1].get("hartree_xc", 0.0) - res[2][1].get("hartree_xc", 0.0)
    out["diamond_mbj"] = {
        "workload": "diamond crystal 20^3, 8 atoms, 16 orbitals x 64 k, FP32 orbitals, predictor-corrector "
                    "steps with LDA (xc = 2) and with TB-mBJ exchange (xc = 3, c from the density)",
        "steps_timed": steps, "warmup": warmup,
        "ms_per_step_lda": res[2][0], "ms_per_step_mbj": res[3][0],
        "phase_ms_per_step_mbj": res[3][1], "launches_per_step_mbj": res[3][2],
        "mbj_kernels_ms_per_step": mbj_ms,
        "mbj_orbital_read_GBps": 2 * 8 * opts / max(mbj_ms * 1e-3, 1e-12) / 1e9,
        "note": "two potentials per PC step; each reads every orbital once (8 B per orbital-point) in the "
                "kinetic-density pass; the rate divides those bytes by the time of all three mBJ kernels"}
    del u0
    torch.cuda.empty_cache()
    return out


def absorption_peak_check(dev, nsteps=1000, kappa=1e-3):
    """Eq. (distribution) spectrum of a kicked isolated cluster (32^3 grid, h = 0.4, 8 atoms,
    16 orbitals, impulse exp(i kappa z)) propagated on the GPU three ways: FP64 orbitals with the
    plain predictor-corrector (the reference), FP32 with the plain predictor-corrector, and FP32
    with the learned predictor (network trained on the GPU on three other kicked initial states of
    the same cluster, PC fallback at misfit > 1e-5).  The main absorption peak of each is located on
    a 0.001 eV grid with tdks_oscillator_strength; criterion: FP32 peaks within 0.01 eV of FP64."""
    import torch
    from paper_1804_01404_gb300 import learned as L
    from paper_1804_01404_gb300 import tdks as T
    from paper_1804_01404_gb300 import workloads as W
    ev = 27.211386245988
    s = W.isolated_cluster(n=32, natom=8, norb=16, radius=5.0, seed=2)
    kick = (0.0, 0.0, kappa)
    psi0 = W.initial_orbitals(s, 1)
    res = {"workload": "isolated cluster 32^3 (h = 0.4), 8 atoms, 16 orbitals, kick 1e-3 along z, "
                       f"{nsteps} steps of dt = {s.dt}", "steps": nsteps}
    tic = time.perf_counter()
    trajs = [L.trajectory(s, W.initial_orbitals(s, seed), 300, "f32", kick=kick) for seed in (2, 3, 4)]
    tctx = T.Context(s, precision="f32")
    tctx.nn_init(1)
    L.train(tctx, trajs, epochs=3, batch=8, lr=1e-3, seed=5)
    params = tctx.nn_params()
    tctx.close()
    del trajs
    res["training_s"] = time.perf_counter() - tic
    peaks = {}
    for name, prec, mode in (("f64_pc", "f64", T.PRED_PC), ("f32_pc", "f32", T.PRED_PC),
                             ("f32_learned", "f32", T.PRED_LEARNED)):
        ctx = T.Context(s, precision=prec)
        u = torch.from_numpy(psi0.astype(np.complex128 if prec == "f64" else np.complex64)).to(dev)
        ctx.kick(u, kick)
        ctx.update_potential(u)
        if mode != T.PRED_PC:
            ctx.nn_init(0)
            ctx.nn_params(params)
            ctx.set_predictor(mode, 1e-5)
        d = [0.0]
        tt = 0.0
        torch.cuda.synchronize()
        tic = time.perf_counter()
        o = None
        for _ in range(nsteps):
            ctx.step(u, tt, s.dt)
            tt += s.dt
            o = ctx.read_step_observables()
            d.append(o["dipole"][2])
        res[f"{name}_steps_per_s_host_synced"] = nsteps / (time.perf_counter() - tic)
        if mode != T.PRED_PC:
            res[f"{name}_fallbacks"] = o["fallbacks"]
        ctx.check()
        ctx.close()
        d = np.array(d)
        E = np.arange(0.0, 2.0, 0.005)
        E0 = E[np.argmax(T.oscillator_strength(d, s.dt, kappa, E))]
        Ef = np.arange(max(E0 - 0.01, 1e-6), E0 + 0.01, 0.001 / ev)
        peaks[name] = (float(Ef[np.argmax(T.oscillator_strength(d, s.dt, kappa, Ef))]), d)
    res["peak_eV"] = {p: v[0] * ev for p, v in peaks.items()}
    d64 = peaks["f64_pc"][1]
    for name in ("f32_pc", "f32_learned"):
        res[f"peak_shift_{name}_vs_f64_eV"] = abs(peaks[name][0] - peaks["f64_pc"][0]) * ev
        res[f"dipole_rel_err_{name}_vs_f64"] = float(np.max(np.abs(peaks[name][1] - d64)) / np.max(np.abs(d64)))
    res["resolution_eV"] = 2 * np.pi / (nsteps * s.dt) * ev
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-learned", action="store_true")
    ap.add_argument("--skip-hpsi", action="store_true")
    ap.add_argument("--skip-workloads", action="store_true",
                    help="skip the few-step timings of the isolated cluster and multiscale workloads")
    ap.add_argument("--only", default="", choices=["", "hpsi", "workloads", "mbj", "accuracy"],
                    help="hpsi: only the tdks_hpsi measurement on the isolated cluster (profiling); "
                         "workloads: only the cluster, multiscale and TB-mBJ step timings; mbj: only the "
                         "TB-mBJ step timing of the diamond crystal")
    ap.add_argument("--no-step-graph", action="store_true",
                    help="predicted steps as stream launches with a host decision (tdks_set_step_graph 0), so "
                         "that a profiler times every kernel; for launch lists, not for the headline")
    ap.add_argument("--skip-accuracy", action="store_true",
                    help="skip the long-window FP32-against-FP64 runs (2000 crystal steps, 4000 cluster steps)")
    ap.add_argument("--hpsi-norb", type=int, default=256)
    ap.add_argument("--hpsi-reps", type=int, default=10)
    ap.add_argument("--cpu-steps", type=int, default=4)
    ap.add_argument("--fp64-steps", type=int, default=10)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, rank, world)
    if args.only == "hpsi":
        import torch
        torch.cuda.set_device(local_rank)
        if rank == 0:
            print(json.dumps({"hpsi_cluster": hpsi_cluster(torch.device("cuda", local_rank),
                                                           reps=args.hpsi_reps, norb=args.hpsi_norb)}))
        return 0
    if args.only == "mbj":
        import torch
        torch.cuda.set_device(local_rank)
        if rank == 0:
            print(json.dumps({"other_workloads": workload_steps(torch.device("cuda", local_rank), which=("mbj",))}))
        return 0
    if args.only == "accuracy":
        import torch
        torch.cuda.set_device(local_rank)
        if rank == 0:
            dev = torch.device("cuda", local_rank)
            params, _ = train_predictor(workload(), 200.0)
            print(json.dumps({"accuracy_long": accuracy_long(dev, params)}))
        return 0
    if args.only == "workloads":
        import torch
        torch.cuda.set_device(local_rank)
        if rank == 0:
            dev = torch.device("cuda", local_rank)
            others = workload_steps(dev)
            others["absorption_peak"] = absorption_peak_check(dev)
            print(json.dumps({"other_workloads": others}))
        return 0
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    try:
        return gpu_arm(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
