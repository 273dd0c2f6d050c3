#!/usr/bin/env python3
"""Throughput of the shrinking-domain PM step on GB300.

One "step" = one pass of the whole hot path (half drift + CIC deposit,
source + boundary values, multigrid Poisson solve to rtol, gradient + gather +
kick + drift, lightcone shrink) over the active particles of one simulation.
The workload is 256^3 particles on a 256^3 mesh, 2000 Mpc/h, Zel'dovich ICs
from P(k) ~ k^-1.5 exp(-k^2/2k_c^2) (seed 1), steps uniform in a from 0.01 to
1 in 200 steps.  --steps K times two windows of that schedule: K/2 steps from
a = 0.01 (periodic phase, every particle active) and K/2 steps from the first
open-phase step (a ~ 0.73: open boundaries, shrinking cube and particle set,
the lightcone compaction), the run's own state there (the steps in between
run untimed).

Tolerance: the metric compares the plain FP32 and the mixed (FP32 V-cycles
inside a double-float defect correction) solvers at equal residual.  The
FP32 potential stalls above 1e-7, so both run to max(1e-5, 10 x the plain
path's measured floor on the first step) unless --rtol is given; the mixed
path at 1e-7 is reported beside it.

value  = sum over timed steps of the active particle count / device time
         (mixed path at that tolerance; "arithmetic" says which form)
e2e    = the same through the C ABI with host buffers: each step copies the
         particles host->device, steps, and copies them back
Multi-GPU: independent replicas (one per rank, no collective on the data
path); value = all ranks' particle-steps / max rank time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "pm256"
METRIC = ("particle-steps/s, PM step at 256^3, mixed FP32/double-float multigrid, "
          "plain-vs-mixed equal residual")
UNIT = "particle-steps/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def aggregate_ranks(units, elapsed, device):
    """Whole-job figures over the ranks of the default process group (one
    replica per rank, no exchange on the data path): the sum of the units
    processed and the slowest rank's elapsed time."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(units), float(elapsed)
    s = torch.tensor([float(units)], device=device, dtype=torch.float64)
    m = torch.tensor([float(elapsed)], device=device, dtype=torch.float64)
    dist.all_reduce(s)
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    return s.item(), m.item()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _ics():
    from paper_1709_04703_gb300 import ics
    return ics.workload_ics(WORKLOAD), ics.WORKLOADS[WORKLOAD]


# particles reordered by cell at the start of every SORT_EVERY-th step
# (--sort-every; 0: the initial order, compacted stably)
SORT_EVERY = 32
# FP32 V-cycles that may share one defect in the mixed forms (--inner)
INNER = 4


def _inner(precision):
    return INNER if precision in ("mixed", "mixed64") else 1


def _new_sim(pos, mom, ids, cfg, rtol, precision, guess="warm"):
    from paper_1709_04703_gb300.sim import Sim
    return Sim(pos, mom, ids, cfg["n"], cfg["box"], cfg["a_init"], cfg["a_final"],
               cfg["steps"], rtol=rtol, precision=precision, max_vcycles=100, guess=guess,
               sort_every=SORT_EVERY, inner_vcycles=_inner(precision))


STRICT_RTOL = 1e-7

# the arithmetic each --precision computes in
DTYPE = {"mixed": "f32+df32", "fp32": "f32", "mixed64": "f32+f64"}
ARITHMETIC = {
    "mixed": "FP32 V-cycles inside a double-float (hi + lo FP32 pair, ~48-bit significand) "
             "defect correction; FP32 particles, int64 density",
    "fp32": "FP32 potential and V-cycles; FP32 particles, int64 density",
    "mixed64": "FP32 V-cycles inside an FP64 defect correction (FP64 potential); FP32 "
               "particles, int64 density",
}

# ncu dram__bytes_read.sum + dram__bytes_write.sum over the algorithmic bytes
# of the kernel class's launches at 256^3 on the current kernels
TRAFFIC_RATIO = {
    # the smoother's algorithmic bytes are 12 B per cell and sweep, 48 B per
    # pre + post pair of fused passes (the 256^3 level: 32 x 32 tiles)
    "smooth0": ((93332224 + 187955712) / (48.0 * 256**3), "k_rbgs2<32> pre + post at 256^3, "
                "profiles/rbgs2_pm256_level0.md"),
    "defect": ((327600640 + 515282176) / (335.5e6 + 536.9e6), "k_defect<0> + k_defect<1> at "
               "256^3, profiles/rbgs2_pm256_level0.md"),
    "deposit": (1127.8e6 / 1073.7e6, "k_drift_deposit at 256^3, "
                "profiles/defect_gather_deposit_pm256.md"),
    "gather": (1294.6e6 / 1342.2e6, "k_gather_kick_drift at 256^3, "
               "profiles/defect_gather_deposit_pm256.md"),
}


def _plain_floor(pos, mom, ids, cfg):
    """Relative residual at which the plain FP32 path stalls on the first
    step (100 V-cycles), 0 if it reaches the strict tolerance."""
    from paper_1709_04703_gb300 import _lib as L
    sim = _new_sim(pos, mom, ids, cfg, STRICT_RTOL, "fp32")
    try:
        sim.step(1)
        floor = 0.0
    except L.PmError:
        floor = float(sim.stats()["resid_last"])
    sim.close()
    return floor


def _first_open_step(sim, n, box):
    """Index of the schedule's first step whose keep cube lies inside the box
    (open boundaries and shrinking from there on): R = chi/cell + 1 cell
    <= n/2 - 1, the library's boundary rule."""
    chi = sim.schedule()["chi"]
    R = chi / (box / n) + 1.0
    return next(k for k in range(len(chi) - 1) if R[k] <= 0.5 * n - 1.0)


def _windows(K, k_open, steps):
    """The timed steps: K/2 from the start of the run (periodic phase, every
    particle active) and K/2 from the first open-phase step (shrinking
    cube, shrinking particle set).  Returns [(first step, count), ...]."""
    kb = min(K // 2, steps - k_open)
    return [(0, K - kb), (k_open, kb)]


def _run_windows(sim, windows, stream, per_window=None):
    """Step `sim` through the windows, timing each with CUDA events on the
    context's stream; untimed steps in between advance the run (its state
    at the second window is the run's own, not regenerated).  Returns
    (device ms, particle-steps, per-window records)."""
    import torch
    out, ms_tot, ps_tot = [], 0.0, 0
    for k0, cnt in windows:
        if cnt <= 0:
            continue
        gap = k0 - sim.stats()["step"]
        if gap > 0:
            sim.step(gap)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ps0 = sim.stats()["particle_steps"]
        vc0 = sim.stats()["vcycles_total"]
        if per_window is not None:
            per_window("start")
        torch.cuda.synchronize()
        ev0.record(stream)
        sim.step(cnt)
        ev1.record(stream)
        torch.cuda.synchronize()
        if per_window is not None:
            per_window("end")
        ms = ev0.elapsed_time(ev1)
        st = sim.stats()
        ps = st["particle_steps"] - ps0
        out.append({"first_step": k0, "steps": cnt, "ms_per_step": round(ms / cnt, 4),
                    "particle_steps": int(ps), "value": ps / (ms * 1e-3),
                    "vcycles": int(st["vcycles_total"] - vc0),
                    "n_active_end": int(st["n_active"]),
                    "phase": "periodic" if k0 == 0 else "open (shrinking)"})
        ms_tot += ms
        ps_tot += ps
    return ms_tot, ps_tot, out


def _variant(pos, mom, ids, cfg, windows, rtol, precision, guess="warm", net=None,
             gravity="poisson", bc="paper", shrink=True, assignment="cic"):
    """The same timed windows in another solver configuration."""
    from paper_1709_04703_gb300 import _lib as L
    from paper_1709_04703_gb300.sim import Sim
    sim = Sim(pos, mom, ids, cfg["n"], cfg["box"], cfg["a_init"], cfg["a_final"],
              cfg["steps"], rtol=rtol, precision=precision, max_vcycles=100, guess=guess,
              gravity=gravity, bc=bc, shrink=shrink, assignment=assignment,
              sort_every=SORT_EVERY,
              inner_vcycles=_inner(precision) if gravity == "poisson" and guess != "learned"
              else 1)
    if net is not None:
        sim.set_guess(net)
    out = {"precision": precision, "guess": guess, "rtol": rtol, "gravity": gravity,
           "assignment": assignment}
    if not shrink:
        out["box"] = "fixed periodic (no shrinking)"
    try:
        ms, ps, wins = _run_windows(sim, windows, sim.stream)
    except L.PmError as e:
        st = sim.stats()
        out.update(error=str(e), steps_done=st["step"], resid_last=st["resid_last"])
        sim.close()
        return out
    st = sim.stats()
    sim.close()
    K = sum(c for _, c in windows)
    out.update(value=ps / (ms * 1e-3), ms_per_step=ms / K,
               vcycles_total=sum(w["vcycles"] for w in wins),
               guess_used=st["guess_used_total"],
               windows=[{k: w[k] for k in ("first_step", "steps", "ms_per_step", "vcycles")}
                        for w in wins])
    return out


def _oracle_worker(task):
    """One host process: the FP64 oracle, as it stands, stepping an n^3
    replica of the workload from step k0 (ICs regenerated at that a) for up
    to `steps` steps or `budget_s` seconds.  Returns (particle-steps, s)."""
    import sys as _sys
    _sys.path.insert(0, ROOT)
    from oracle import cosmology as cz
    from oracle import pm as opm
    from paper_1709_04703_gb300 import ics
    n, k0, steps, budget_s = task
    cfg = ics.WORKLOADS[WORKLOAD]
    sched = cz.schedule(n, cfg["box"], 0.3, 0.7, cfg["a_init"], cfg["a_final"], cfg["steps"])
    pos, mom, _ = ics.zeldovich(n, cfg["alpha"], cfg["cutoff"], cfg["seed"], sched["a"][k0])
    x, p = pos.astype(np.float64), mom.astype(np.float64)
    ps = 0
    t0 = time.perf_counter()
    for k in range(k0, min(k0 + steps, cfg["steps"])):
        ps += len(x)
        x, p, info = opm.step(x, p, k, sched, n, 0.3, 1.0)
        if not info["periodic"]:
            keep = opm.keep_mask(x, sched["R"][k + 1], n)
            x, p = x[keep], p[keep]
        if time.perf_counter() - t0 >= budget_s:
            break
    return ps, time.perf_counter() - t0


def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_pool(n, starts, steps, budget_s):
    """The oracle on every host core at once: one process per core (spawned,
    so none inherits the parent's CUDA context), each a replica of the
    workload at n^3 starting at one of `starts` in turn.  Returns
    (particle-steps / wall s, cores, wall s, per-start particle-steps)."""
    import multiprocessing as mp
    cores = _host_cores()
    tasks = [(n, starts[w % len(starts)], steps, budget_s) for w in range(cores)]
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_worker, tasks)
    wall = time.perf_counter() - t0
    busy = max(r[1] for r in res)
    ps = sum(r[0] for r in res)
    return ps / busy, cores, busy, wall


def _k_open_oracle(n):
    from oracle import cosmology as cz
    from oracle import pm as opm
    from paper_1709_04703_gb300 import ics
    cfg = ics.WORKLOADS[WORKLOAD]
    sched = cz.schedule(n, cfg["box"], 0.3, 0.7, cfg["a_init"], cfg["a_final"], cfg["steps"])
    return next(k for k in range(cfg["steps"]) if not opm.active_cube(sched["R"][k], n)[2])


def cpu_baseline(budget_s=20.0, n_sample=128, window=5):
    """The FP64 oracle, as it stands, on all host cores: one process per
    core, each stepping a replica of the workload at n_sample^3 (same box,
    spectrum and seed) for `window` steps or budget_s seconds, half of them
    from a_init (periodic phase) and half from the first open-phase step
    (ICs regenerated at that a).  particle-steps/s = all processes' active
    particles over the steps run / the slowest process's time.  A 128^3
    replica: one oracle step at 256^3 takes ~1 min and ~3 GB per process."""
    k_open = _k_open_oracle(n_sample)
    val, cores, busy, wall = _oracle_pool(n_sample, [0, k_open], window, budget_s)
    return {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"oracle (numpy FP64, exact FFT / DST Poisson solves) in {cores} "
                      f"processes, one per host core, each a {n_sample}^3-particle replica of "
                      f"the 256^3 workload (same box, spectrum, seed) for up to {window} steps "
                      f"from step 0 (periodic; even processes) or step {k_open} (open phase, "
                      f"ICs at that a; odd processes), {busy:.1f} s"}


def run_reference(args):
    """--impl reference: the oracle as the reference arm, on all host cores
    (one process per core, spawned), on the same windows as the GPU arm:
    K/2 steps from a_init and K/2 from the first open-phase step, each
    process a replica of the 256^3 workload at 64^3 (ICs regenerated at the
    window's a), every process bounded to a minute."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    n = 64
    k_open = _k_open_oracle(n)
    half = max(1, args.steps // 2)
    val, cores, busy, wall = _oracle_pool(n, [0, k_open], half, 60.0)
    sample = (f"oracle (numpy FP64) in {cores} processes, one per host core, each a "
              f"{n}^3-particle replica of the 256^3 workload (same box, spectrum, seed) for up to "
              f"{half} steps from step 0 (even processes) or step {k_open} (open phase, ICs at "
              f"that a; odd processes), {busy:.1f} s")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * busy / half, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_mesh": 256, "n_particles": 256**3,
                       "box_mpch": 2000.0, "sample_mesh": n, "windows": "start + open phase"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _batch48(steps, warmup, sequential="all"):
    """The 48-realisation batched workload (mesh 32..128^3, boxes 200-1500
    Mpc/h, seeds 100-147, 50 steps from a = 0.02): the batched step over
    `steps` steps after `warmup` untimed ones on a separate batch, and the
    same realisations as separate contexts (sequential = "all": every one of
    them, one after another; "128": the 128^3 ones, for the per-particle rate
    of a single context at that size)."""
    import torch
    from paper_1709_04703_gb300 import _lib as L
    from paper_1709_04703_gb300 import ics
    from paper_1709_04703_gb300.sim import Batch, Sim
    cfgs = ics.batched_workload(range(100, 148))
    a0, a1, nsteps, rtol = cfgs[0]["a_init"], cfgs[0]["a_final"], cfgs[0]["steps"], cfgs[0]["rtol"]
    K = min(steps, nsteps)
    reals = []
    for c in cfgs:
        pos, mom, ids = ics.zeldovich(c["n"], c["alpha"], c["cutoff"], c["seed"], a0)
        reals.append(dict(pos=pos, mom=mom, ids=ids, n_mesh=c["n"], box=c["box"]))
    lib = L.load()
    K = min(K, nsteps - 1)
    W = min(warmup, nsteps - K)

    def timed(persistent):
        # the warm-up steps run on the timed batch itself, so the solve
        # graph's capture and the smoother's autotuning stay outside the
        # timed region; the timed steps are W .. W + K - 1
        batch = Batch(reals, a0, a1, nsteps, rtol=rtol)
        if persistent:
            batch.set_solve(persistent=True)
        batch.step(W)
        torch.cuda.synchronize()
        ps0 = sum(batch.stats(r)["particle_steps"] for r in range(len(reals)))
        vc0 = sum(batch.stats(r)["vcycles_total"] for r in range(len(reals)))
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = lib.pm_launch_count()
        torch.cuda.synchronize()
        with Clocks(0) as clk:
            ev0.record(batch.stream)
            batch.step(K)
            ev1.record(batch.stream)
            torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        launches = lib.pm_launch_count() - l0
        ps = sum(batch.stats(r)["particle_steps"] for r in range(len(reals))) - ps0
        vc = sum(batch.stats(r)["vcycles_total"] for r in range(len(reals))) - vc0
        batch.close()
        return ms, launches, ps, vc, clk
    ms, launches, ps, vc, clk = timed(False)
    p_ms, p_launches, p_ps, _, _ = timed(True)
    seq_ms, seq_ps = 0.0, 0
    pick = range(len(reals)) if sequential == "all" else \
        [r for r, c in enumerate(cfgs) if c["n"] == 128]
    for r in pick:
        re = reals[r]
        sim = Sim(re["pos"], re["mom"], re["ids"], re["n_mesh"], re["box"], a0, a1, nsteps,
                  rtol=rtol)
        sim.step(W)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        p0 = sim.stats()["particle_steps"]
        e0.record(sim.stream)
        sim.step(K)
        e1.record(sim.stream)
        torch.cuda.synchronize()
        seq_ms += e0.elapsed_time(e1)
        seq_ps += sim.stats()["particle_steps"] - p0
        sim.close()
    return {"value": ps / (ms * 1e-3), "unit": UNIT, "steps": K, "warmup": W,
            "timed_steps": f"{W}..{W + K - 1}",
            "ms_per_step": ms / K, "launches_per_step": launches / K,
            "solve": "graph: V-cycle loop as a conditional while node, decided on the device",
            "persistent_solve": {"value": p_ps / (p_ms * 1e-3), "ms_per_step": p_ms / K,
                                 "launches_per_step": p_launches / K,
                                 "solve": "one cooperative launch per solve, grid barriers"},
            "realisations": len(reals), "mesh_sizes": sorted({c["n"] for c in cfgs}),
            "particles": int(sum(len(r["pos"]) for r in reals)), "rtol": rtol,
            "vcycles": int(vc),
            ("sequential_contexts" if sequential == "all" else "single_context_128"):
                {"value": seq_ps / (seq_ms * 1e-3), "realisations": len(pick),
                 "ms_per_step": seq_ms / K},
            "clocks": clk.summary(), "gpu_launches": int(launches)}


def run_batch(args):
    """--workload batch48: the 48-realisation batched workload, compared with
    the same realisations run one context after another."""
    import torch
    torch.cuda.set_device(0)
    out = _batch48(args.steps, args.warmup, "all")
    line = {
        "metric": "particle-steps/s, batched PM step, 48 realisations",
        "value": out["value"], "unit": UNIT, "n_gpus": 1, "steps": out["steps"],
        "warmup": args.warmup, "ms_per_step": out["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+df32",
        "data": "synthetic (seeded Zel'dovich ICs)",
        "config": {"workload": "batch48", "realisations": out["realisations"],
                   "mesh_sizes": out["mesh_sizes"], "particles": out["particles"],
                   "rtol": out["rtol"], "vcycles": out["vcycles"],
                   "timed_steps": out["timed_steps"],
                   "solve": out["solve"]},
        "sequential_contexts": out["sequential_contexts"],
        "launches_per_step": out["launches_per_step"],
        "clocks": out["clocks"], "gpu_launches": out["gpu_launches"],
    }
    print(json.dumps(line), flush=True)
    return 0

def run_guess512(args):
    """--workload guess512: the learned initial guess on the 512^3 workload
    (512^3 particles and mesh, 3000 Mpc/h, 100 steps from a = 0.02, mixed
    precision to a relative residual of 1e-7): the same steps solved from
    the warm start alone (the method without the network) and from the
    network's correction of it; V-cycles saved, the network's time and the
    particle-steps/s of each."""
    import torch
    from paper_1709_04703_gb300 import train_guess
    torch.cuda.set_device(0)
    steps = args.steps if args.steps_given else None
    with Clocks(0) as clk:
        out = train_guess.compare("pm512", args.weights, ("warm", "learned"), steps)
    w, l = out["warm"], out["learned"]
    z = np.load(args.weights)
    meta = json.loads(str(z["meta"])) if "meta" in z.files else {}
    line = {"metric": "particle-steps/s, PM step at 512^3, learned initial guess against the "
                      "warm start, rtol 1e-7",
            "value": l["particle_steps_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": l["steps"], "higher_is_better": True, "dtype": "bf16 network, f32+df32 "
            "solve", "data": "synthetic (seeded Zel'dovich ICs)",
            "config": {"workload": "guess512", "n_mesh": 512, "n_particles": 512**3,
                       "box_mpch": 3000.0, "rtol": 1e-7,
                       "weights": os.path.relpath(args.weights, ROOT),
                       "trained_pairs": meta.get("pairs"), "trained_on": meta.get("workload")},
            "warm": w, "learned": l, "vcycles_saved": out["vcycles_saved"],
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


TABLE4 = {512.0: 1.08, 2048.0: 1.44, 8192.0: 3.02}   # Table 4, 512^3 particles


def _timed_run(pos, mom, ids, n, box, a0, steps, rtol, gravity, shrink, domain="cube"):
    """One whole run, each step device-timed on the context stream; per-step
    active particles and milliseconds, and the run's catalogue (lightcone
    records plus the particles never recorded) for P(k).  shrink=False is
    the fixed periodic box with the lightcone recorded (PM_SHRINK_RECORD)."""
    import torch
    from paper_1709_04703_gb300.sim import Sim
    # (the headline's solver: INNER FP32 V-cycles per defect, as --inner sets)
    inner = INNER if gravity == "poisson" and domain != "ball" else 1
    sim = Sim(pos, mom, ids, n, box, a0, 1.0, steps, rtol=rtol, precision="mixed",
              max_vcycles=100, gravity=gravity, bc="paper" if shrink else "periodic",
              shrink=True if shrink else "record", domain=domain, inner_vcycles=inner)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    n_act = []
    torch.cuda.synchronize()
    ev[0].record(sim.stream)
    for k in range(steps):
        n_act.append(sim.stats()["n_active"])
        sim.step(1)
        ev[k + 1].record(sim.stream)
    torch.cuda.synchronize()
    ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]
    st = sim.stats()
    ap, _, ai = sim.particles()
    lp, _, li, _ = sim.lightcone()
    sim.close()
    rest = ap if shrink else ap[~np.isin(ai, li)]
    return {"ms": sum(ms), "ms_step": ms, "n_active": n_act,
            "vcycles_total": int(st["vcycles_total"]),
            "catalogue": np.concatenate([lp, rest]).astype(np.float32)}


def _catalogue_pk(cat, box, n):
    """P(k) of a catalogue in the original box, alias-corrected (Jing 2005)."""
    import torch
    from paper_1709_04703_gb300.sim import pack, power_spectrum_jing
    p4, _ = pack(np.mod(cat, n).astype(np.float32), np.zeros_like(cat))
    k, p, _, _, _ = power_spectrum_jing(torch.from_numpy(p4).cuda(), box, n, n // 2)
    return k, p


def run_shrink_table(args):
    """--workload shrink_table: the whole-run time of the fixed periodic box
    (lightcone recorded, every particle integrated) over that of the
    shrinking box (Table 4's speed-up, Sec. 3.3), and the relative difference
    of the two lightcone catalogues' P(k) (Fig. 4), with the
    paper's run shape: n^3 particles on an n^3 mesh, a from 1/41 (z = 40) to
    1 in 1000 steps uniform in a, boxes 512, 2048 and 8192 Mpc/h.  Both
    gravities: the diffusion equation (the paper's pair of codes) and the
    static Poisson solve.  The same seeded ICs (in cell units) serve every
    box; the box sets the lightcone radius in cells and so the shrinking."""
    import torch
    from paper_1709_04703_gb300 import ics
    torch.cuda.set_device(0)
    n, steps, a0 = args.table_n, args.steps if args.steps_given else 1000, 1.0 / 41.0
    tol = args.rtol if args.rtol is not None else 1e-5
    pos, mom, ids = ics.zeldovich(n, -1.5, 0.5, 1, a0)
    # warm-up: a few steps of each kind
    for grav in args.gravities:
        for shrink in (True, False):
            _timed_run(pos, mom, ids, n, 8192.0, a0, max(3, args.warmup), tol, grav, shrink,
                       args.table_domain)
    rows = []
    for grav in args.gravities:
        for box in (512.0, 2048.0, 8192.0):
            sh = _timed_run(pos, mom, ids, n, box, a0, steps, tol, grav, True, args.table_domain)
            fx = _timed_run(pos, mom, ids, n, box, a0, steps, tol, grav, False,
                            args.table_domain)
            q = [steps // 4, steps // 2, (3 * steps) // 4]
            # Fig. 4: P(k) of the two catalogues in the original box, k <= k_Ny/2
            _, p_sh = _catalogue_pk(sh["catalogue"], box, n)
            _, p_fx = _catalogue_pk(fx["catalogue"], box, n)
            rel = np.abs(p_sh[: n // 4] / p_fx[: n // 4] - 1.0)
            rows.append({
                "gravity": grav, "box_mpch": box, "shrink_s": round(sh["ms"] * 1e-3, 3),
                "fixed_s": round(fx["ms"] * 1e-3, 3), "speedup": round(fx["ms"] / sh["ms"], 3),
                "paper_speedup": TABLE4[box],
                # Figs. 5 and 6 at a quarter, half and three quarters of the run
                "n_active_frac": [round(sh["n_active"][k] / n**3, 4) for k in q],
                "ms_step_ratio": [round(sh["ms_step"][k] / fx["ms_step"][k], 4) for k in q],
                "vcycles": [sh["vcycles_total"], fx["vcycles_total"]],
                "lightcone_pk_rel_diff": {"max": float(rel.max()),
                                          "rms": float(np.sqrt(np.mean(rel**2))),
                                          "k_range": "k_f .. k_Ny/2"}})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    line = {"metric": "whole-run speed-up, shrinking vs fixed periodic box", "unit": "x",
            "higher_is_better": True, "n_gpus": 1, "steps": steps,
            "data": "synthetic (seeded Zel'dovich ICs)",
            "config": {"workload": "shrink_table", "domain": args.table_domain,
                       "n_mesh": n, "n_particles": n**3,
                       "a": [a0, 1.0], "rtol": tol, "precision": "mixed"},
            "rows": rows}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    from paper_1709_04703_gb300 import _lib as L
    from paper_1709_04703_gb300.sim import pack
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    (pos, mom, ids), cfg = _ics()
    K = min(args.steps, cfg["steps"])
    lib = L.load()

    # warm-up: W steps on a throw-away context (same ICs)
    sim = _new_sim(pos, mom, ids, cfg, STRICT_RTOL, args.precision)
    sim.step(min(args.warmup, cfg["steps"]))
    k_open = _first_open_step(sim, cfg["n"], cfg["box"])
    sim.close()
    torch.cuda.synchronize()
    windows = _windows(K, k_open, cfg["steps"])

    # tolerance of the plain-vs-mixed comparison: the FP32 potential stalls
    # above 1e-7, so both paths run to max(1e-5, 10 x its measured floor)
    floor = _plain_floor(pos, mom, ids, cfg)
    rtol = args.rtol if args.rtol is not None else max(1e-5, 10.0 * floor)

    # timed: the two windows, device-resident inputs, no instrumentation;
    # the untimed steps between them advance the same run
    sim = _new_sim(pos, mom, ids, cfg, rtol, args.precision)
    stream = sim.stream   # the stream every kernel of the context is launched on
    tiles = {str(side): f"32x{ty} tiles, {zc} planes per CTA"
             for side, (ty, zc) in sorted(sim.smoother_tiles().items(), reverse=True)}
    launches, marks = [0], []

    def count(edge):
        c = lib.pm_launch_count()
        launches[0] += (-1 if edge == "start" else 1) * c
        if edge == "start":
            marks.append(c)
        else:
            # for a launch list of exactly this window's kernels:
            # ncu -k regex:^k -s <start> -c <count>
            print(f"timed window {len(marks) - 1}: library launches {marks[-1]} .. {c - 1}",
                  file=sys.stderr, flush=True)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        ms, psteps, wins = _run_windows(sim, windows, stream, count)
    if ws > 1:
        dist.barrier()
    st = sim.stats()
    import ctypes as C
    vstats = {"vcycles_total": sum(w["vcycles"] for w in wins), "n_active_end": st["n_active"],
              "n_lightcone": st["n_lightcone"], "escaped": st["escaped"]}
    sim.close()

    # the same windows again, one step at a time, with CUDA events around
    # every kernel class on the context's stream: per-class device time and
    # algorithmic bytes (the events cost a few % of the step, so the
    # headline comes from the uninstrumented run above), and per step the
    # active particles N, cells C and V-cycles k for the whole-step count
    sim = _new_sim(pos, mom, ids, cfg, rtol, args.precision)
    prof, per_step = None, []
    p0 = time.perf_counter()
    lib = L.load()
    for k0, cnt in windows:
        gap = k0 - sim.stats()["step"]
        if gap > 0:
            sim.step(gap)
        sim.profile(True)
        torch.cuda.synchronize()
        l_start = lib.pm_launch_count()
        for _ in range(cnt):
            n_act = sim.stats()["n_active"]
            sim.step(1)
            s1 = sim.stats()
            per_step.append((n_act, s1["cube_side"] ** 3, s1["vcycles_last"]))
        # the library's kernel launches of this window (for a launch list
        # of exactly these steps: ncu -k regex:^k_ -s <start> -c <count>)
        print(f"instrumented window from step {k0}: library launches {l_start} .. "
              f"{lib.pm_launch_count() - 1}", file=sys.stderr, flush=True)
        part = sim.profile_read()
        sim.profile(False)
        prof = part if prof is None else {
            c: {f: prof[c][f] + part[c][f] for f in ("ms", "groups", "bytes")} for c in prof}
    torch.cuda.synchronize()
    prof_wall_ms = (time.perf_counter() - p0) * 1e3
    if sum(v for _, _, v in per_step) != vstats["vcycles_total"]:
        raise RuntimeError("the instrumented repeat took a different number of V-cycles")
    sim.close()
    # whole-step algorithmic bytes (N active particles, C active cells, k
    # V-cycles, o = k outer defect-correction iterations in the mixed forms)
    o_of = (lambda v: v) if args.precision != "fp32" else (lambda v: 0)
    step_bytes = sum(64.0 * N + (24.0 + 74.0 * v + 40.0 * o_of(v)) * Cc for N, Cc, v in per_step)

    # the same windows with plain FP32 V-cycles at the same tolerance, the
    # mixed path at 1e-7 (below the plain floor), FP64 forms, the other
    # gravities and assignment, the fixed box and the learned guess
    compare = None
    if not args.no_compare:
        from paper_1709_04703_gb300 import train_guess
        first = [(0, 1)]
        compare = {"plain_fp32": _variant(pos, mom, ids, cfg, windows, rtol, "fp32"),
                   f"mixed_rtol_{STRICT_RTOL:g}": _variant(pos, mom, ids, cfg, windows,
                                                           STRICT_RTOL, "mixed"),
                   f"plain_fp32_rtol_{STRICT_RTOL:g}": _variant(pos, mom, ids, cfg, first,
                                                                STRICT_RTOL, "fp32")}
        # FP32 V-cycles inside an FP64-arithmetic defect correction (FP64
        # potential), at the same tolerance and at 1e-7
        compare["mixed_fp64_defect"] = _variant(pos, mom, ids, cfg, windows, rtol, "mixed64")
        compare[f"mixed_fp64_defect_rtol_{STRICT_RTOL:g}"] = _variant(
            pos, mom, ids, cfg, windows, STRICT_RTOL, "mixed64")
        # FP64 everywhere: potential, source and every multigrid level in
        # double, at the same tolerance and at 1e-7
        compare["plain_fp64"] = _variant(pos, mom, ids, cfg, windows, rtol, "fp64")
        compare[f"plain_fp64_rtol_{STRICT_RTOL:g}"] = _variant(pos, mom, ids, cfg, windows,
                                                               STRICT_RTOL, "fp64")
        # the paper's diffusion-equation gravity (two implicit half-substeps)
        compare["diffusion_gravity"] = _variant(pos, mom, ids, cfg, windows, rtol, "mixed",
                                                gravity="diffusion")
        # ... and with the paper's own explicit (ADE) sweeps instead of solves
        compare["diffusion_ade"] = _variant(pos, mom, ids, cfg, windows, rtol, "mixed",
                                            gravity="diffusion_ade")
        # TSC density assignment and force interpolation instead of CIC
        compare["tsc"] = _variant(pos, mom, ids, cfg, windows, rtol, "mixed", assignment="tsc")
        # the same steps in the fixed periodic box (every particle, every step)
        compare["no_shrink"] = _variant(pos, mom, ids, cfg, windows, rtol, "mixed",
                                        bc="periodic", shrink=False)
        net = train_guess.load(train_guess.DEFAULT_WEIGHTS)
        for tol in (rtol, STRICT_RTOL):
            key = "learned_guess" + ("" if tol == rtol else f"_rtol_{tol:g}")
            compare[key] = _variant(pos, mom, ids, cfg, windows, tol, args.precision, "learned",
                                    net)
            compare[key]["weights"] = os.path.relpath(train_guess.DEFAULT_WEIGHTS, ROOT)
        net.close()
        # the 48-realisation batched step (10 steps), with the 128^3 single
        # context's rate per particle beside it
        compare["batch48"] = _batch48(10, 3, "128")

    # end to end through the C ABI with host buffers (pinned): every timed
    # step copies the active particles host -> device, steps, and copies
    # them back; the untimed steps between the windows advance the run
    e2e = None
    if not args.no_e2e:
        sim = _new_sim(pos, mom, ids, cfg, rtol, args.precision)
        p4, m4 = pack(pos, mom, ids)
        hp = torch.from_numpy(p4).pin_memory()
        hm = torch.from_numpy(m4).pin_memory()
        h2d = d2h = 0
        dt, ps = 0.0, 0
        for k0, cnt in windows:
            gap = k0 - sim.stats()["step"]
            if gap > 0:
                sim.step(gap)
            n_act = sim.get_particles_host(hp, hm)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(cnt):
                L.check(lib.pm_set_particles(sim._ctx, C.c_void_p(hp.data_ptr()),
                                             C.c_void_p(hm.data_ptr()), n_act, 1), sim._ctx)
                h2d += 32 * n_act
                ps += n_act
                sim.step(1)
                n_act = sim.get_particles_host(hp, hm)
                d2h += 32 * n_act
            torch.cuda.synchronize()
            dt += time.perf_counter() - t0
        sim.close()
        e2e = {"value": ps / dt, "unit": UNIT, "h2d_bytes_per_step": h2d // K,
               "d2h_bytes_per_step": d2h // K}
        e2e_units, e2e_s = ps, dt

    # aggregate over ranks: sum of particle-steps, max of time
    tot_ps, max_ms = aggregate_ranks(psteps, ms, "cuda")
    if e2e is not None:
        e_ps, e_s = aggregate_ranks(e2e_units, e2e_s, "cuda")
        e2e["value"] = e_ps / e_s
    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return 0

    peak, peak_kind = _peaks()
    dom = max(prof, key=lambda k: prof[k]["ms"])
    d = prof[dom]
    achieved = d["bytes"] / (d["ms"] * 1e-3) / 1e9 if d["ms"] > 0 else 0.0
    # DRAM traffic per launch: the ncu ratio of DRAM to algorithmic bytes of
    # the class's 256^3 launches (profiles/), times this run's algorithmic
    # bytes per launch of the class
    traffic = None
    if dom in TRAFFIC_RATIO and d["groups"] > 0:
        traffic = TRAFFIC_RATIO[dom][0] * d["bytes"] / d["groups"]
    kernels = {k: {"ms": round(v["ms"], 3), "share": round(v["ms"] / max(1e-9, sum(
        x["ms"] for x in prof.values())), 4), "GB/s": round(v["bytes"] / (v["ms"] * 1e-3) / 1e9, 1)
        if v["ms"] > 0 else None} for k, v in prof.items()}
    line = {
        "metric": METRIC, "value": tot_ps / (max_ms * 1e-3), "unit": UNIT, "n_gpus": ws,
        "steps": K, "warmup": args.warmup, "ms_per_step": max_ms / K,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[args.precision],
        "arithmetic": ARITHMETIC[args.precision],
        "data": "synthetic (seeded Zel'dovich ICs)",
        "windows": wins,
        "config": {"workload": WORKLOAD, "n_mesh": 256, "n_particles": 256**3,
                   "box_mpch": 2000.0, "a": [cfg["a_init"], cfg["a_final"]],
                   "schedule_steps": cfg["steps"],
                   "timed_steps": [f"{k0}..{k0 + c - 1}" for k0, c in windows if c > 0],
                   "rtol": rtol,
                   "rtol_rule": "equal residual: max(1e-5, 10 x plain FP32 floor)"
                                if args.rtol is None else "given",
                   "plain_fp32_floor": floor,
                   "precision": args.precision, "sort_every": SORT_EVERY,
                   "inner_vcycles": _inner(args.precision),
                   "smoother": f"red-black SOR, factor {L.PM_MG_OMEGA}, V(2,2)",
                   "smoother_tiles": tiles,
                   "parallelism": f"replicas x{ws}",
                   "l2": "inputs larger than L2 (particles 537 MB, mesh 134 MB)"},
        "roofline": {"kernel": dom, "bound": "hbm", "achieved": round(achieved, 1),
                     "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": round(achieved / peak, 4),
                     "traffic": round(traffic) if traffic is not None else None,
                     "algorithmic_bytes_per_launch": round(d["bytes"] / max(1, d["groups"])),
                     "traffic_source": TRAFFIC_RATIO[dom][1] if dom in TRAFFIC_RATIO else None},
        "step_roofline": {"bound": "hbm", "bytes_per_step": round(step_bytes / K),
                          "achieved": round(step_bytes / (ms * 1e-3) / 1e9, 1),
                          "peak": peak, "unit": "GB/s",
                          "frac": round(step_bytes / (ms * 1e-3) / 1e9 / peak, 4),
                          "count": "sum over the timed steps of 64 N + (24 + 74 k + 40 o) C: N "
                                   "active particles, C active cells, k V-cycles, o = k outer "
                                   "iterations (0 in plain FP32)"},
        "kernels": kernels,
        "kernels_timing": "CUDA events around each kernel class on the context stream, in an "
                          f"instrumented repeat of the same {K} steps ({prof_wall_ms / K:.3f} "
                          "ms/step there, one step per call)",
        "solver": vstats,
        "clocks": clk.summary(),
        "gpu_launches": int(launches[0]),
    }
    if e2e is not None:
        line["e2e"] = e2e
    if compare is not None:
        line["compare"] = compare
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_budget)
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def main():
    global SORT_EVERY, INNER
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--rtol", type=float, default=None,
                    help="solver tolerance (default: equal-residual rule, see config)")
    ap.add_argument("--precision", choices=["mixed", "fp32", "mixed64"], default="mixed")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the plain-FP32 and learned-guess runs of the same steps")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sort-every", type=int, default=SORT_EVERY,
                    help="reorder the particles by cell every k-th step (0: never)")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--inner", type=int, default=INNER,
                    help="FP32 V-cycles per defect in the mixed forms (1: one)")
    ap.add_argument("--workload", choices=["pm256", "batch48", "shrink_table", "guess512"],
                    default="pm256")
    ap.add_argument("--weights", default=None,
                    help="guess512: network weights (default: the committed ones)")
    ap.add_argument("--table-n", type=int, default=512,
                    help="shrink_table: particles and mesh per side")
    ap.add_argument("--table-domain", choices=["cube", "sphere"], default="cube",
                    help="shrink_table: keep region")
    ap.add_argument("--gravities", nargs="+", default=["diffusion", "poisson"],
                    choices=["diffusion", "diffusion_ade", "poisson"],
                    help="shrink_table: gravity solvers")
    args = ap.parse_args()
    args.steps_given = "--steps" in sys.argv
    SORT_EVERY = max(0, args.sort_every)
    INNER = max(1, args.inner)
    if args.impl == "reference":
        return run_reference(args)
    from paper_1709_04703_gb300 import build
    build.build()
    if args.workload == "batch48":
        return run_batch(args)
    if args.workload == "shrink_table":
        return run_shrink_table(args)
    if args.workload == "guess512":
        if args.weights is None:
            from paper_1709_04703_gb300 import train_guess
            args.weights = train_guess.DEFAULT_WEIGHTS
        return run_guess512(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
