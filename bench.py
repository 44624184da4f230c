#!/usr/bin/env python
"""Throughput of the driven coronal MHD step on GB300: MHD cell-updates/s per
RK3 step (cells x steps / time), FP32 path (FP32 state and stencils, FP64
potential-field FFT and reductions) on the 256^3 bipole workload, with the
FP64 path measured beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Under torchrun (N > 1) every rank runs an independent replica of the
workload (the single-GPU path is not split across GPUs); value = all cells
updated by all ranks / max-over-ranks time.  --impl reference times the FP64
CPU oracle (rank 0 only) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MHD cell-updates/s per RK step"
UNIT = "cell-updates/s"
WORDS_PER_CELL_STEP = 80  # algorithmic state words moved per cell per RK3 step
RUNS = 5                  # timed runs of K steps; the median is reported
# FP64 operations per cell and substep of rk_simple_kernel<double> (2 flops
# per DFMA, 1 per DADD / DMUL; each of the three one FP64-pipe instruction),
# from the ncu instruction counts summarised in
# profiles/rk_simple_fp64_flops_bipoles20_128x128x128.md
FP64_FLOPS_PER_CELL_SUBSTEP = 1459.4
FP64_PIPE_OPS_PER_CELL_SUBSTEP = 1022.3
# FP32 operations per cell and substep of rk_pair_kernel (f32x2 instructions
# one operation per cell, FFMA two flops; FFMA, FADD and FMUL one FMA-pipe
# lane operation each), from the ncu instruction counts in
# profiles/rk_pair_fp32_flops_bipoles20_128x128x128.md
FP32_FLOPS_PER_CELL_SUBSTEP = 1021.3
FP32_PIPE_OPS_PER_CELL_SUBSTEP = 621.3
RK_KERNEL = ("rk_pair_kernel (fused RHS + RK update, TMA z-march, two cells per thread in f32x2, "
             "z histories in TMEM)")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="bipoles40_256x256x256")
    ap.add_argument("--stats-every", type=int, default=10)
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--graph", action="store_true",
                    help="replay a CUDA graph of 10 steps in the timed region instead of launching the steps one "
                         "by one (measured no faster at 256^3: 2.455 against 2.431 ms per step)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-production", action="store_true")
    ap.add_argument("--adjoint-scale", action="store_true",
                    help="also run the checkpointed gradient of bipoles100_512x512x256 (minutes)")
    ap.add_argument("--scale-steps", type=int, default=0, help="0: the workload's step count (600)")
    ap.add_argument("--scale-iters", type=int, default=3)
    ap.add_argument("--drift", action="store_true",
                    help="also run ar_1024x1024x256 in FP32 and FP64 and compare energies, fluxes and fields")
    ap.add_argument("--drift-steps", type=int, default=100)
    ap.add_argument("--no-granulation", action="store_true",
                    help="skip timing the granulation driver on a 1024 x 1024 plane (Sect. 2.3)")
    ap.add_argument("--snapshot", action="store_true",
                    help="also time mhd_write_snapshot (var.h5 + grid.h5) of a 1024 x 1024 x 64 FP32 box")
    ap.add_argument("--cooling", action="store_true",
                    help="Newtonian cooling on (rate 0.5, height cut-off at 10 dz) in the throughput leg")
    return ap.parse_args()


def dist_setup():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(local)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi samples every 100 ms while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.idx)], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names[1:], parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def rk_traffic_bytes():
    """Per-launch DRAM traffic of the RK kernel from the committed ncu summary,
    valid only if the kernel source is unchanged since the capture."""
    path = os.path.join(ROOT, "profiles", "rk_traffic.txt")
    csrc = os.path.join(ROOT, "paper_1908_08557_gb300", "csrc")
    try:
        kv = {}
        for line in open(path):
            if line.strip() and not line.startswith("#"):
                k, v = line.split(None, 1)
                kv[k] = v.strip()
        blob = b"".join(open(os.path.join(csrc, f), "rb").read() for f in kv["sources"].split())
        sha = hashlib.sha256(blob).hexdigest()[:16]
        if kv.get("kernel_source_sha") != sha:
            return None
        return float(kv["bytes_per_launch_avg"])
    except Exception:
        return None


def cpu_oracle_sample(nx=256, ny=256, nz=32, steps=1):
    """One RK3 step of the FP64 oracle on a 256 x 256 x 32 slab of the same
    recipe (bipoles, solenoidal driver); returns (cell-updates/s, seconds)."""
    import inputs
    import oracle
    case = inputs.make_box(nx, ny, nz, seed=0, magnetogram="bipoles", n_mag=40, driver="solenoidal")
    axt, ayt = oracle.a_target(case.params, case.bz)
    u = oracle.to_padded(case.state)
    t0 = time.perf_counter()
    oracle.run(case.params, u, case.lnrho0, axt, ayt, case.v0, case.v1, case.t0, case.t1, 0.0, steps)
    dt = time.perf_counter() - t0
    return nx * ny * nz * steps / dt, dt


def cpu_oracle_runs():
    """The oracle on the smaller named workloads, once on one thread and once
    on every core (OMP_NUM_THREADS), each in a fresh interpreter: spots4 at
    32^3 for 50 steps, the 64^3 gradient workload for 5 steps.  The 256^3
    workload's 20 steps would take minutes on all cores and most of an hour
    on one, so its rate is the slab sample above."""
    import subprocess
    import sys
    code = ("import json, sys, time; sys.path.insert(0, %r); import inputs, oracle; "
            "c = inputs.make_case(sys.argv[1]); n = int(sys.argv[2]); t = time.perf_counter(); "
            "oracle.run_case(c, nsteps=n); el = time.perf_counter() - t; "
            "q = c.params; print(json.dumps({'seconds': el, 'value': q['nx'] * q['ny'] * q['nz'] * n / el}))"
            % ROOT)
    out = []
    for name, steps in (("spots4_32x32x32", 50), ("bipoles8_64x64x64", 5)):
        for threads in (1, os.cpu_count()):
            env = dict(os.environ, OMP_NUM_THREADS=str(threads))
            r = subprocess.run([sys.executable, "-c", code, name, str(steps)], capture_output=True, text=True,
                               env=env, timeout=600)
            if r.returncode != 0:
                out.append({"workload": name, "steps": steps, "threads": threads, "error": r.stderr[-300:]})
                continue
            d = json.loads(r.stdout.strip().splitlines()[-1])
            out.append({"workload": name, "steps": steps, "threads": threads, "value": d["value"], "unit": UNIT,
                        "seconds": d["seconds"]})
    return out


def _cuda_ms(stream, fn):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def adjoint_ratios(case, dev, ws):
    import torch

    import inputs
    from paper_1908_08557_gb300 import Simulation
    from paper_1908_08557_gb300.adjoint import Revolver, optimal_splits
    out = {}
    # per step at the bench size, frozen dt = 0.017 (about the CFL step)
    p = dict(case.params, dt_fixed=0.017)
    sim = Simulation(p, torch.tensor(case.state, dtype=torch.float32, device=dev), case.lnrho0, case.lnT0,
                     precision=32, adjoint=True, device=str(dev))
    sim.set_driver(torch.tensor(case.bz, dtype=torch.float32, device=dev),
                   torch.tensor(case.v0, dtype=torch.float32, device=dev),
                   torch.tensor(case.v1, dtype=torch.float32, device=dev), case.t0, case.t1)
    sim.step(2)
    ck = sim.new_checkpoint()
    t = sim.save(ck)
    fwd = _cuda_ms(sim.stream, lambda: sim.step(3)) / 3
    g = torch.Generator(device=dev).manual_seed(0)
    sim.adjoint_init(torch.randn((8, p["nz"], p["ny"], p["nx"]), dtype=torch.float32, device=dev, generator=g))
    sim.restore(ck, t)
    sim.adjoint_step()  # warm-up
    # each adjoint step starts from the checkpointed state; the restore (a
    # device copy) is timed apart from the step
    adj, rst = [], []
    for _ in range(3):
        rst.append(_cuda_ms(sim.stream, lambda: sim.restore(ck, t)))
        adj.append(_cuda_ms(sim.stream, sim.adjoint_step))
    adj = sum(adj) / len(adj)
    # the same reverse step from a tape of the step's substep states (kept by
    # the forward step when memory allows): no forward recomputation
    tape = sim.new_tape()
    sim.restore(ck, t)
    fwd_taped = _cuda_ms(sim.stream, lambda: sim.step_taped(tape))
    sim.adjoint_step_taped(tape)  # warm-up
    # (an NVTX range names these launches for a profiler's launch list)
    with torch.cuda.nvtx.range("adjoint_step_taped"):
        adj_taped = sum(_cuda_ms(sim.stream, lambda: sim.adjoint_step_taped(tape)) for _ in range(3)) / 3
    out["bench_workload"] = {"forward_ms_per_step": fwd, "adjoint_ms_per_step": adj,
                             "restore_ms": sum(rst) / len(rst), "ratio": adj / fwd,
                             "taped": {"forward_taped_ms_per_step": fwd_taped, "adjoint_ms_per_step": adj_taped,
                                       "ratio": adj_taped / fwd,
                                       "tape_gb": sim.tape_bytes() / 1e9}}
    del tape
    sim.close()
    del sim, ck
    torch.cuda.empty_cache()
    # full checkpointed sweep of the gradient workload
    c4 = inputs.make_case("bipoles8_64x64x64")
    p4 = dict(c4.params, dt_fixed=0.017)
    sim = Simulation(p4, torch.tensor(c4.state, dtype=torch.float32, device=dev), c4.lnrho0, c4.lnT0, precision=32,
                     adjoint=True, device=str(dev))
    sim.set_driver(torch.tensor(c4.bz, dtype=torch.float32, device=dev),
                   torch.tensor(c4.v0, dtype=torch.float32, device=dev),
                   torch.tensor(c4.v1, dtype=torch.float32, device=dev), c4.t0, c4.t1)
    # checkpoint slots from a state-history budget of 120 GB (the budget of
    # the 512 x 512 x 256 checkpointed workload): at 64^3 the whole history
    # fits as tapes (three substep states per step), so the reverse sweep
    # recomputes no forward substep at all
    budget = 120 * 2**30
    n = c4.nsteps
    slots = int(max(1, budget // sim.checkpoint_bytes() - 1))
    sim.set_time(0.0)
    ck0 = sim.new_checkpoint()
    t0 = sim.save(ck0)
    fwd = _cuda_ms(sim.stream, lambda: sim.step(n))
    sim.restore(ck0, t0)
    optimal_splits(n, slots)  # the schedule: planned once on the host, cached
    rv = Revolver(sim, slots)
    fwd_ck = _cuda_ms(sim.stream, lambda: rv.forward(n))
    sim.adjoint_init(torch.zeros((8, p4["nz"], p4["ny"], p4["nx"]), dtype=torch.float32, device=dev))
    rev_ms = _cuda_ms(sim.stream, rv.reverse)
    out["bipoles8_64x64x64"] = {"steps": n, "slots": slots, "budget_gb": budget / 2**30, "forward_ms": fwd,
                                 "forward_with_checkpoints_ms": fwd_ck,
                                 "reverse_ms": rev_ms, "ratio": rev_ms / fwd,
                                 "taped": bool(rv.tapes),
                                 "recompute_fraction": rv.recomputed_steps / n}
    sim.close()
    del sim
    torch.cuda.empty_cache()
    return out


def adjoint_scale_line(dev, steps, iters, slots=None, k=48, descend=True):
    """bipoles100_512x512x256, FP32, frozen dt: the B_z misfit on layer 48
    after `steps` steps against a target made by a forward run driven by a
    different seeded 100-bipole magnetogram and driver; its gradient with
    respect to (B_z, v0, v1) by the adjoint under binomial checkpointing with
    slots from a 120 GB state budget (or the given slot count); `iters`
    gradient evaluations, each followed (descend) by a gradient-descent step
    (step length a quarter of loss / |g|^2, halved once if the loss rises)."""
    import numpy as np
    import torch

    import inputs
    from paper_1908_08557_gb300 import Simulation
    from paper_1908_08557_gb300.adjoint import BzPlane, DrivenRun, optimal_splits
    c = inputs.make_case("bipoles100_512x512x256", dtype=np.float32)
    ct = inputs.make_case("bipoles100_512x512x256", seed=1, dtype=np.float32)
    steps = steps or c.nsteps
    p = dict(c.params, dt_fixed=0.017)
    T = lambda a: torch.tensor(a, dtype=torch.float32, device=dev)
    sim = Simulation(p, T(c.state), c.lnrho0, c.lnT0, precision=32, adjoint=True, device=str(dev))
    state0 = sim.read().clone()
    budget = 120 * 2**30
    if slots is None:
        slots = int(max(1, min(steps - 1, budget // sim.checkpoint_bytes() - 1)))
    else:
        budget = (slots + 1) * sim.checkpoint_bytes()

    def run(bz, v0, v1):
        sim.set_driver(bz, v0, v1, c.t0, c.t1)
        sim.write(state0)
        sim.set_time(0.0)
        sim.step(steps)
        return sim.bz_plane(sim.read(), k)

    target = run(T(ct.bz), T(ct.v0), T(ct.v1)).detach()
    params = [T(c.bz), T(c.v0), T(c.v1)]
    fwd_ms = _cuda_ms(sim.stream, lambda: run(*params))
    loss_of = lambda ps: float(0.5 * ((run(*ps) - target) ** 2).sum())
    optimal_splits(steps, slots)  # the schedule: planned once on the host, cached
    hist, out = [], {"steps": steps, "slots": slots, "budget_gb": budget / 2**30, "forward_ms": fwd_ms}
    loss = loss_of(params)
    for it in range(iters):
        leaves = [q.clone().requires_grad_(True) for q in params]
        box = {}

        def fwd():
            box["st"] = DrivenRun.apply(leaves[0], leaves[1], leaves[2], sim, state0, steps, slots, c.t0, c.t1)

        fwd_ck = _cuda_ms(sim.stream, fwd)
        lossv = 0.5 * ((BzPlane.apply(box["st"], sim, k) - target) ** 2).sum()
        rev = _cuda_ms(sim.stream, lambda: lossv.backward())
        g = [q.grad.detach() for q in leaves]
        if not descend:
            hist.append({"loss": float(lossv.detach()), "forward_with_checkpoints_ms": fwd_ck, "reverse_ms": rev,
                         "ratio": rev / fwd_ms})
            continue
        g2 = sum(float((x.double() ** 2).sum()) for x in g)
        eta = 0.25 * float(lossv.detach()) / max(g2, 1e-300)
        trial = [q - eta * x for q, x in zip(params, g)]
        new = loss_of(trial)
        if new > loss:
            eta *= 0.5
            trial = [q - eta * x for q, x in zip(params, g)]
            new = loss_of(trial)
        hist.append({"loss": float(lossv.detach()), "forward_with_checkpoints_ms": fwd_ck, "reverse_ms": rev,
                     "ratio": rev / fwd_ms, "loss_after_step": new})
        params, loss = trial, new
    out["iterations"] = hist
    out["layer"] = k
    if descend:
        out["loss_reduction"] = hist[0]["loss"] / loss if hist else None
    out["recompute_fraction"] = _revolve_recompute(steps, slots) / steps
    sim.close()
    del sim
    torch.cuda.empty_cache()
    return out


def _revolve_recompute(n, slots):
    """Forward steps the reverse sweep of Revolver recomputes: its schedule
    replayed on the host against a stand-in that only counts."""
    from paper_1908_08557_gb300.adjoint import Revolver

    class _Count:
        def new_checkpoint(self):
            return None

        def save(self, buf):
            return 0.0

        def restore(self, buf, t):
            pass

        def step(self, k):
            pass

        def adjoint_step(self):
            pass

    rv = Revolver(_Count(), slots)
    rv.forward(n)
    rv.reverse()
    return rv.recomputed_steps


def granulation_line(dev, n=1024, dt=10.0, t_end=600.0):
    """The granulation driver on an n x n plane of 0.23 Mm pixels (the
    driver figure's), Sect. 2.3's parameters: the first fill of the empty
    plane, then one update and one velocity every dt = 10 s of solar time
    (the snapshot cadence the paper names) up to t_end; the random draws of
    every update resident on the device before timing.  Steady-state means
    over the updates from one lifetime (300 s) on."""
    import numpy as np
    import torch

    import inputs
    from paper_1908_08557_gb300 import Granulation
    from paper_1908_08557_gb300.granulation import paper_params
    gen = Granulation(n, n, 1.0, 1.0, paper_params(mm_per_unit=0.23), device=str(dev))
    times = np.arange(0.0, t_end + dt / 2, dt)
    dr = []
    for u in range(len(times)):
        k, cl, ca = inputs.granulation_draws(n, n, seed=17, update=u)
        dr.append((torch.as_tensor(k.view(np.int32), device=dev), torch.as_tensor(cl, device=dev),
                   torch.as_tensor(ca, device=dev)))
    v = torch.empty((2, n, n), dtype=torch.float32, device=dev)
    gen.update(-1e6, *dr[0])  # warm-up: loads the kernels, places a population ...
    gen.velocity(-1e6, precision=32, out=v)
    gen.close()               # ... discarded: a fresh generator for the timed run
    gen = Granulation(n, n, 1.0, 1.0, paper_params(mm_per_unit=0.23), device=str(dev))
    l0 = gen.launch_count()
    rec = []
    for u, t in enumerate(times):
        box = {}
        tu = _cuda_ms(gen.stream, lambda: box.update(r=gen.update(float(t), *dr[u])))
        tv = _cuda_ms(gen.stream, lambda: gen.velocity(float(t), precision=32, out=v))
        occ, _ = gen.granules()
        rec.append((float(t), tu, box["r"], tv, int(occ.sum())))
    steady = [r for r in rec if r[0] >= 300.0]
    out = {"plane": f"{n}x{n}", "pixel_mm": 0.23, "update_every_s": dt, "updates": len(rec),
           "fill_ms": rec[0][1], "fill_rounds": rec[0][2], "granules_after_fill": rec[0][4],
           "update_ms": float(np.mean([r[1] for r in steady])),
           "update_rounds": float(np.mean([r[2] for r in steady])),
           "velocity_ms": float(np.mean([r[3] for r in steady])),
           "granules": float(np.mean([r[4] for r in steady])),
           "gpu_launches": gen.launch_count() - l0}
    gen.close()
    return out


def snapshot_line(dev):
    """mhd_write_snapshot of a 1024 x 1024 x 64 FP32 box of the production
    recipe after two steps: var.h5 (8 fields with the outer ghosts, grid,
    settings, time) and grid.h5 into a temporary directory of the host, the
    ghost fill and the device-to-host copies included (wall clock, the
    stream synchronised before; the files are not synced to disk, so the
    rate is that of the host's page cache)."""
    import torch

    import inputs
    from paper_1908_08557_gb300 import Simulation
    c = inputs.make_box(1024, 1024, 64, seed=0, dx=4.0, dy=4.0, magnetogram="bipoles", n_mag=400,
                        ar_pair=(5.0, 40.0, 200.0), driver="solenoidal")
    T = lambda a: torch.tensor(a, dtype=torch.float32, device=dev)
    sim = Simulation(c.params, T(c.state), c.lnrho0, c.lnT0, precision=32, device=str(dev))
    sim.set_driver(T(c.bz), T(c.v0), T(c.v1), c.t0, c.t1)
    sim.step(2)
    torch.cuda.synchronize()
    out = {}
    with tempfile.TemporaryDirectory() as d:
        var, grid = os.path.join(d, "var.h5"), os.path.join(d, "grid.h5")
        t0 = time.perf_counter()
        sim.write_snapshot(var, grid)
        sec = time.perf_counter() - t0
        size = os.path.getsize(var) + os.path.getsize(grid)
        out = {"box": "1024x1024x64 (padded 1030x1030x70), FP32", "seconds": sec, "bytes": size,
               "gb_per_s": size / sec / 1e9, "sync": "not synced to disk (page cache)"}
    sim.close()
    del sim
    torch.cuda.empty_cache()
    return out


def production_line(dev, ws):
    """Workload ar_1024x1024x256 in FP32, timed twice: with A stored about the
    FP64 initial potential field (a_background, the configuration that meets
    the FP32 tolerance at this size, where |A| reaches several hundred) and
    with A stored whole.  `value` is the former."""
    import numpy as np
    import torch

    import inputs
    from paper_1908_08557_gb300 import Simulation
    c = inputs.make_case("ar_1024x1024x256")
    p = c.params
    cells = p["nx"] * p["ny"] * p["nz"]
    out = {}
    for mode in ("a_background", "plain"):
        a0 = torch.tensor(c.state[0:3], dtype=torch.float64, device=dev) if mode == "a_background" else None
        sim = Simulation(p, c.state.astype(np.float32), c.lnrho0, c.lnT0, precision=32, stats_every=10,
                         device=str(dev), a_background=a0)
        del a0
        sim.set_driver(torch.tensor(c.bz, dtype=torch.float32, device=dev),
                       torch.tensor(c.v0, dtype=torch.float32, device=dev),
                       torch.tensor(c.v1, dtype=torch.float32, device=dev), c.t0, c.t1)
        sim.step(3)
        torch.cuda.synchronize()
        k = 10
        ms = _cuda_ms(sim.stream, lambda: sim.step(k))
        ms = max_over_ranks(ms, ws)
        # class times as the step runs (the substep-0 ghost rules and CFL
        # wait behind the FFT on the side stream and count its time too), and
        # with every kernel serialised on one stream (they add up to the step)
        sim.profile(True)
        sim.step(3)
        prof = sim.read_profile()
        sim.profile(False)
        sim.profile(2)
        sim.step(3)
        prof_serial = sim.read_profile()
        sim.profile(False)
        sim.close()
        del sim
        torch.cuda.empty_cache()
        rk_ms, rk_n = prof["rk"]
        achieved = WORDS_PER_CELL_STEP * cells * 4 / 3.0 / (rk_ms / rk_n / 1e3) / 1e9
        out[mode] = {"value": ws * cells * k / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / k, "steps": k,
                     "rk_achieved_gbs": achieved, "class_ms_per_step": {kk: v[0] / 3 for kk, v in prof.items()},
                     "class_ms_per_step_serialised": {kk: v[0] / 3 for kk, v in prof_serial.items()}}
    # the FP64 path at the same size (FP64-ALU bound; two timed steps)
    sim = Simulation(p, c.state, c.lnrho0, c.lnT0, precision=64, stats_every=10, device=str(dev))
    sim.set_driver(torch.tensor(c.bz, dtype=torch.float64, device=dev),
                   torch.tensor(c.v0, dtype=torch.float64, device=dev),
                   torch.tensor(c.v1, dtype=torch.float64, device=dev), c.t0, c.t1)
    sim.step(1)
    torch.cuda.synchronize()
    k64 = 2
    ms64 = max_over_ranks(_cuda_ms(sim.stream, lambda: sim.step(k64)), ws)
    sim.close()
    del sim
    torch.cuda.empty_cache()
    line = dict(out["a_background"])
    line["storage"] = "A about the FP64 initial field (a_background)"
    line["plain"] = out["plain"]
    line["fp64"] = {"value": ws * cells * k64 / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64 / k64,
                    "steps": k64, "dtype": "f64"}
    return line


def drift_line(dev, steps, reseed=50):
    """Production geometry ar_1024x1024x256: the FP32 path against an FP64 GPU
    run of the same steps from the same state.  The driver is re-seeded every
    `reseed` steps: the last snapshot becomes v0 and a new seeded solenoidal
    field v1, reached `reseed` steps of the current dt later.  Reports the
    diagnostics of both runs at the start and the end, their relative drift,
    the FP32/FP64 differences of the end values and the per-field relative L2
    difference of the end states."""
    import numpy as np
    import torch

    import inputs
    from paper_1908_08557_gb300 import Simulation
    c = inputs.make_case("ar_1024x1024x256")
    p = c.params
    km = min(32, p["nx"] // 2, p["ny"] // 2)
    drivers = [c.v0, c.v1]
    keys = ["e_kin", "e_mag", "e_th", "mass", "flux_net", "flux_abs", "divb_max"]
    res, ends = {}, {}
    for prec in (32, 64):
        tdt = torch.float32 if prec == 32 else torch.float64
        # FP32: A stored about the FP64 initial potential field
        a0 = torch.tensor(c.state[0:3], dtype=torch.float64, device=dev) if prec == 32 else None
        sim = Simulation(p, torch.tensor(c.state, dtype=tdt, device=dev), c.lnrho0, c.lnT0, precision=prec,
                         stats_every=0, device=str(dev), a_background=a0)
        del a0
        bz = torch.tensor(c.bz, dtype=tdt, device=dev)
        sim.set_driver(bz, torch.tensor(c.v0, dtype=tdt, device=dev), torch.tensor(c.v1, dtype=tdt, device=dev),
                       c.t0, c.t1)
        sim.fill_ghosts()  # the diagnostics read the ghost planes; the ghost rules are idempotent
        s0 = sim.compute_stats()
        t0 = time.perf_counter()
        for n in range(steps):
            if n > 0 and n % reseed == 0:
                k = n // reseed
                while len(drivers) < k + 2:
                    drivers.append(inputs.driver_solenoidal(p["nx"], p["ny"], km, 0.01, len(drivers)))
                t, dt = sim.time()
                sim.set_driver(bz, torch.tensor(drivers[k], dtype=tdt, device=dev),
                               torch.tensor(drivers[k + 1], dtype=tdt, device=dev), t, t + reseed * dt)
            sim.step(1)
        sim.fill_ghosts()
        s1 = sim.compute_stats()
        secs = time.perf_counter() - t0
        ends[prec] = sim.read().to(torch.float64)
        res[f"fp{prec}"] = {"start": {q: s0[q] for q in keys}, "end": {q: s1[q] for q in keys},
                            "drift": {q: (s1[q] - s0[q]) / abs(s0[q]) if s0[q] != 0 else None for q in keys[:4]},
                            "t_end": sim.time()[0], "seconds": secs}
        sim.close()
        del sim
        torch.cuda.empty_cache()
    e32, e64 = res["fp32"]["end"], res["fp64"]["end"]
    res["fp32_vs_fp64_end"] = {q: (e32[q] - e64[q]) / abs(e64[q]) if e64[q] != 0 else None for q in keys[:4]}
    res["fp32_vs_fp64_end"]["flux_net_over_flux_abs"] = (e32["flux_net"] - e64["flux_net"]) / e64["flux_abs"]
    res["fp32_vs_fp64_end"]["flux_abs"] = (e32["flux_abs"] - e64["flux_abs"]) / e64["flux_abs"]
    names = ["A_x", "A_y", "A_z", "u_x", "u_y", "u_z", "ln_rho", "ln_T"]
    res["field_rel_l2"] = {names[f]: float(torch.linalg.vector_norm(ends[32][f] - ends[64][f]) /
                                           torch.linalg.vector_norm(ends[64][f])) for f in range(8)}
    res["steps"] = steps
    res["reseed_every"] = reseed
    res["fp32_storage"] = "A about the FP64 initial field (a_background)"
    del ends
    torch.cuda.empty_cache()
    return res


def run_reference(args, ws, rank):
    if rank != 0:
        return
    import oracle
    oracle.build()
    nx, ny, nz = 128, 128, 16
    for _ in range(args.warmup):
        cpu_oracle_sample(nx, ny, nz, 1)
    times = []
    for _ in range(args.steps):
        _, dt = cpu_oracle_sample(nx, ny, nz, 1)
        times.append(dt)
    tot = sum(times)
    val = nx * ny * nz * args.steps / tot
    sample = f"one RK3 step of a {nx}x{ny}x{nz} box of the same recipe per step (FP64 oracle, OpenMP)"
    line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": args.workload},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_native(args, ws, rank, local):
    import numpy as np
    import torch

    import inputs
    from paper_1908_08557_gb300 import Simulation
    from paper_1908_08557_gb300.build import build
    if rank == 0:
        build()
    barrier(ws)
    build()  # no-op when up to date

    case = inputs.make_case(args.workload)
    if args.cooling:
        case.params = dict(case.params, nc_tau=0.5)
    p = case.params
    cells = p["nx"] * p["ny"] * p["nz"]
    dev = torch.device("cuda", local)

    # the handle on a stream of its own, so that its steps can be captured
    # into a CUDA graph (the library launches only on the handle's stream and
    # the side streams it forks from it)
    gstream = torch.cuda.Stream(device=dev)

    def make(precision, stats_every, stream=None):
        dt = torch.float32 if precision == 32 else torch.float64
        sim = Simulation(p, torch.tensor(case.state, dtype=dt, device=dev), case.lnrho0, case.lnT0,
                         precision=precision, stats_every=stats_every, device=str(dev), stream=stream)
        sim.set_driver(torch.tensor(case.bz, dtype=dt, device=dev), torch.tensor(case.v0, dtype=dt, device=dev),
                       torch.tensor(case.v1, dtype=dt, device=dev), case.t0, case.t1)
        return sim

    sim = make(32, args.stats_every, gstream)
    stream = sim.stream
    with torch.cuda.stream(gstream):
        sim.step(args.warmup)
    torch.cuda.synchronize()
    # a graph of G steps (G the diagnostics period, so every replay computes
    # the diagnostics at its first step as the eager schedule does), replayed
    # K / G times; eager launches if K is not a multiple of G
    G = args.stats_every if args.stats_every > 0 else 10
    use_graph = args.graph and args.steps % G == 0
    graph, glaunch = None, 0
    if use_graph:
        n0 = sim.launch_count()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=gstream):
            sim.step(G)
        glaunch = sim.launch_count() - n0
        with torch.cuda.stream(gstream):
            for _ in range(max(1, args.warmup // G)):
                graph.replay()
        torch.cuda.synchronize()

    def timed_steps():
        # graph replays launch on the current stream: the handle's
        with torch.cuda.stream(gstream):
            if use_graph:
                for _ in range(args.steps // G):
                    graph.replay()
            else:
                sim.step(args.steps)
    barrier(ws)
    torch.cuda.synchronize()
    # five timed runs of exactly K steps each, every one bracketed by a
    # barrier and a device synchronisation; the median run is the value
    clk = ClockSampler(local)
    clk.start()
    runs = []
    for r in range(RUNS):
        barrier(ws)
        torch.cuda.synchronize()
        n0 = sim.launch_count()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        timed_steps()
        e1.record(stream)
        torch.cuda.synchronize()
        launches = glaunch * (args.steps // G) if use_graph else sim.launch_count() - n0
        barrier(ws)
        runs.append(max_over_ranks(e0.elapsed_time(e1), ws))
    clocks = clk.stop()
    ms_max = sorted(runs)[RUNS // 2]
    value = ws * cells * args.steps / (ms_max / 1e3)

    # per-kernel-class timing on the library's stream (separate passes):
    # as the step runs (overlapped classes counted in full), and with every
    # kernel serialised on one stream, whose class times add up to the step
    nprof = min(args.steps, 20)
    sim.profile(True)
    sim.step(nprof)
    prof = sim.read_profile()
    sim.profile(False)
    sim.profile(2)
    sim.step(nprof)
    prof_serial = sim.read_profile()
    sim.profile(False)
    rk_ms, rk_n = prof["rk"]
    esz = 4
    alg_bytes_per_launch = WORDS_PER_CELL_STEP * cells * esz / 3.0
    achieved = alg_bytes_per_launch / (rk_ms / rk_n / 1e3) / 1e9
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks and "hbm_gbs" in peaks else 6800.0
    # the same launch against the FP32 FMA rate (the kernel's arithmetic
    # intensity is close to the ridge of the two peaks)
    roofline_alu = None
    try:
        from paper_1908_08557_gb300.binding import fma_peak
        peak32 = fma_peak(32, str(dev)) / 1e12
        ach32 = FP32_FLOPS_PER_CELL_SUBSTEP * cells / (rk_ms / rk_n / 1e3) / 1e12
        # pipe occupancy: lane operations against the FMA rate (peak / 2)
        ops32 = FP32_PIPE_OPS_PER_CELL_SUBSTEP * cells / (rk_ms / rk_n / 1e3) / 1e12
        roofline_alu = {"bound": "alu", "achieved": ach32, "peak": peak32, "unit": "TFLOP/s",
                        "frac": ach32 / peak32, "flops_per_cell_substep": FP32_FLOPS_PER_CELL_SUBSTEP,
                        "pipe_ops_per_cell_substep": FP32_PIPE_OPS_PER_CELL_SUBSTEP,
                        "pipe_frac": ops32 / (peak32 / 2),
                        "peak_source": "measured in this run (mhd_fma_peak, FP32 FMA chains)"}
    except Exception as exc:  # reported, not fatal
        roofline_alu = {"error": f"{type(exc).__name__}: {exc}"}
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": rk_traffic_bytes(), "kernel": RK_KERNEL,
                "peak_source": "measured" if peaks else "fallback",
                "alg_bytes_per_launch": alg_bytes_per_launch, "avg_launch_ms": rk_ms / rk_n,
                "class_ms_per_step": {k: v[0] / nprof for k, v in prof.items()},
                "class_ms_per_step_serialised": {k: v[0] / nprof for k, v in prof_serial.items()}}

    # end to end through the library's API with host buffers: each step
    # copies its driver snapshot (B_z, v0, v1) from pinned host memory to the
    # device on the handle's stream, hands it to mhd_set_driver (magnetogram
    # inversion included), steps, and copies one layer of the new state (u_z
    # at mid-height) back into pinned host memory -- all queued on the one
    # stream without a host synchronisation per step (the host waits once, at
    # the end, and then reads the time); wall clock over the whole loop
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.tensor(a, dtype=torch.float32).pin_memory()
        hb, hv0, hv1 = pin(case.bz), pin(case.v0), pin(case.v1)
        db, dv0, dv1 = (torch.empty_like(x, device=dev) for x in (hb, hv0, hv1))
        hplane = torch.empty((p["ny"], p["nx"]), dtype=torch.float32).pin_memory()
        dplane = torch.empty((p["ny"], p["nx"]), dtype=torch.float32, device=dev)
        kmid = p["nz"] // 2

        def e2e_step():
            with torch.cuda.stream(sim.stream):
                db.copy_(hb, non_blocking=True)
                dv0.copy_(hv0, non_blocking=True)
                dv1.copy_(hv1, non_blocking=True)
            sim.set_driver(db, dv0, dv1, case.t0, case.t1)
            sim.step(1)
            sim.read_plane(5, kmid, dplane)
            with torch.cuda.stream(sim.stream):
                hplane.copy_(dplane, non_blocking=True)

        for _ in range(2):
            e2e_step()
        sim.time()
        barrier(ws)
        t0 = time.perf_counter()
        ne2e = min(args.steps, 50)
        for _ in range(ne2e):
            e2e_step()
        sim.time()  # synchronises the stream
        el = time.perf_counter() - t0
        el = max_over_ranks(el, ws)
        e2e = {"value": ws * cells * ne2e / el, "unit": UNIT, "steps": ne2e,
               "h2d_bytes_per_step": int(hb.nbytes + hv0.nbytes + hv1.nbytes),
               "d2h_bytes_per_step": int(hplane.numel() * 4),
               "read_back": "u_z on layer nz/2 each step; t and dt once at the end",
               "sync": "one host synchronisation after the loop"}
    sim.close()
    del sim
    torch.cuda.empty_cache()

    fp64 = None
    if not args.no_fp64:
        s64 = make(64, args.stats_every)
        s64.step(1)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(s64.stream)
        s64.step(args.fp64_steps)
        f1.record(s64.stream)
        torch.cuda.synchronize()
        ms64 = max_over_ranks(f0.elapsed_time(f1), ws)
        s64.profile(True)
        s64.step(1)
        prof64 = s64.read_profile()
        s64.profile(False)
        fp64 = {"value": ws * cells * args.fp64_steps / (ms64 / 1e3), "unit": UNIT,
                "ms_per_step": ms64 / args.fp64_steps, "steps": args.fp64_steps,
                "dtype": "f64"}
        # the FP64 right-hand side is bound by the FP64 FMA pipe: its
        # roofline is the kernel's FP64 flops (per cell and substep, from an
        # ncu count of its DFMA / DADD / DMUL instructions) over its launch
        # time, against the FP64 FMA rate the library's probe measures here
        try:
            from paper_1908_08557_gb300.binding import fma_peak
            peak64 = fma_peak(64, str(dev)) / 1e12
            rk64_ms, rk64_n = prof64["rk"]
            ach64 = FP64_FLOPS_PER_CELL_SUBSTEP * cells / (rk64_ms / rk64_n / 1e3) / 1e12
            # pipe occupancy: DFMA, DADD and DMUL each take one FP64-pipe slot
            ops64 = FP64_PIPE_OPS_PER_CELL_SUBSTEP * cells / (rk64_ms / rk64_n / 1e3) / 1e12
            fp64["roofline"] = {"bound": "alu", "achieved": ach64, "peak": peak64, "unit": "TFLOP/s",
                                "frac": ach64 / peak64, "kernel": "rk_simple_kernel<double>",
                                "flops_per_cell_substep": FP64_FLOPS_PER_CELL_SUBSTEP,
                                "pipe_ops_per_cell_substep": FP64_PIPE_OPS_PER_CELL_SUBSTEP,
                                "pipe_frac": ops64 / (peak64 / 2),
                                "avg_launch_ms": rk64_ms / rk64_n,
                                "peak_source": "measured in this run (mhd_fma_peak, FP64 FMA chains)"}
        except Exception as exc:  # reported, not fatal
            fp64["roofline"] = {"error": f"{type(exc).__name__}: {exc}"}
        s64.close()
        del s64
        torch.cuda.empty_cache()

    # adjoint / forward time: one adjoint step (recompute of its substeps
    # included) against one forward step, at the bench size; and a full
    # checkpointed sweep of the gradient workload bipoles8_64x64x64
    # (100 steps, slots from a 120 GB budget) against its forward run
    adj = None
    if not args.no_adjoint:
        adj = adjoint_ratios(case, dev, ws)
        # the checkpointed regime at 512 x 512 x 256, bounded: 100 steps with
        # 12 slots recompute 0.87 of the steps, as 1000 steps do with the 56
        # slots of a 120 GB budget (0.94); one gradient-descent step
        try:
            sample = adjoint_scale_line(dev, 100, 1, slots=12, k=8, descend=False)
            sample["sample"] = ("one gradient of the B_z misfit on layer 8 after 100 of the workload's steps, 12 "
                                "checkpoint slots (recompute fraction close to that of 1000 steps under the 120 GB "
                                "budget); --adjoint-scale runs 600 steps with descent on layer 48")
            adj["bipoles100_512x512x256_sample"] = sample
        except Exception as exc:  # reported, not fatal
            adj["bipoles100_512x512x256_sample"] = {"error": f"{type(exc).__name__}: {exc}"}

    # production size 1024 x 1024 x 256 (FP32, horizontal spacing 4x vertical)
    prod = None
    if not args.no_production:
        prod = production_line(dev, ws)

    drift = None
    if args.drift:
        try:
            drift = drift_line(dev, args.drift_steps)
        except Exception as exc:  # reported, not fatal: the run is optional
            drift = {"error": f"{type(exc).__name__}: {exc}"}

    snap = None
    if args.snapshot:
        try:
            snap = snapshot_line(dev)
        except Exception as exc:  # reported, not fatal: the run is optional
            snap = {"error": f"{type(exc).__name__}: {exc}"}

    gran = None
    if not args.no_granulation:
        try:
            gran = granulation_line(dev)
        except Exception as exc:  # reported, not fatal: the run is optional
            gran = {"error": f"{type(exc).__name__}: {exc}"}

    scale = None
    if args.adjoint_scale:
        try:
            scale = adjoint_scale_line(dev, args.scale_steps, args.scale_iters)
        except Exception as exc:  # reported, not fatal: the run is optional
            scale = {"error": f"{type(exc).__name__}: {exc}"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        v, secs = cpu_oracle_sample()
        cpu = {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"one RK3 step of a 256x256x32 slab of the same recipe ({secs:.1f} s, FP64 oracle, OpenMP)",
               "runs": cpu_oracle_runs()}

    if rank == 0:
        state_gb = 3 * 8 * (p["nx"] + 16) * (p["ny"] + 6) * (p["nz"] + 6) * 4 / 1e9
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
                "runs_ms_per_step": [r / args.steps for r in runs], "timing": f"median of {RUNS} runs of K steps",
                "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": args.workload, "nx": p["nx"], "ny": p["ny"], "nz": p["nz"],
                           "precision": "fp32 state and stencils; fp64 FFT, CFL and diagnostics",
                           "stats_every": args.stats_every,
                           "newton_cooling": bool(args.cooling),
                           "l2": f"working set {state_gb:.2f} GB > 129 MB L2, no flush",
                           "launch": (f"CUDA graph of {G} steps replayed {args.steps // G} times" if use_graph
                                      else "steps launched one by one"),
                           "parallelism": f"replicas x{ws}"},
                "roofline": roofline, "roofline_alu": roofline_alu, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clocks, "fp64": fp64, "adjoint": adj, "production_1024x1024x256": prod}
        if scale is not None:
            line["adjoint_bipoles100_512x512x256"] = scale
        if drift is not None:
            line["drift_ar_1024x1024x256"] = drift
        if gran is not None:
            line["granulation_1024x1024"] = gran
        if snap is not None:
            line["snapshot"] = snap
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_native(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
