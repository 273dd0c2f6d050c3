"""Training of the learned initial guess (not in the paper) on pairs the
solver itself produces.

Each step of a shrinking-domain run (PM_MIXED, warm start) hands back, via
pm_capture, the residual r of its warm start and the correction e the
multigrid solve added to it (A e = r to the solve's tolerance).  The network
takes one Adam step on every pair whose cube side it can take, with the
residual-norm loss: with out_scale = 1 that loss is exactly
|r - A e_net|^2 / |r|^2, the square of the factor by which the network's
correction shrinks the residual of the start.

    python -m paper_1709_04703_gb300.train_guess --workload pm256 --seeds 1 2 \
        --out weights.npz
"""
import argparse
import json
import os
import sys
import time

import numpy as np
import torch

from . import ics
from .guess import GuessNet
from .sim import Sim

# trained by (9753 pairs: the 18-minute limit ended the run before 20000):
#   python -m paper_1709_04703_gb300.train_guess --workload pm256 \
#     --seeds 2 3 4 5 6 7 8 9 10 11 12 13 --pairs 20000 --max-seconds 1080 --out <this file>
DEFAULT_WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights",
                               "guess_l4_pm256_10k.npz")


_IC_CACHE = {}


def run_pairs(cfg, steps=None, on_pair=None, stop=None):
    """Run one realisation with capture armed; on_pair(k, r, e, side,
    periodic, stats) for every solve (r, e: CUDA views [1, s, s, s]); the
    run ends early once stop() is true."""
    key = (cfg["n"], cfg["alpha"], cfg["cutoff"], cfg["seed"], cfg["a_init"])
    if key not in _IC_CACHE:  # a pass over the seeds regenerates no initial conditions
        _IC_CACHE[key] = ics.workload_ics(cfg)
    pos, mom, ids = _IC_CACHE[key]
    n = cfg["n"]
    sim = Sim(pos, mom, ids, n, cfg["box"], cfg["a_init"], cfg["a_final"], cfg["steps"],
              rtol=cfg["rtol"])
    r = torch.zeros(n ** 3, device="cuda")
    e = torch.zeros(n ** 3, device="cuda")
    sim.capture(r, e)
    for k in range(cfg["steps"] if steps is None else steps):
        if stop is not None and stop():
            break
        sim.step(1)
        st = sim.stats()
        s = st["cube_side"]
        if on_pair is not None:
            on_pair(k, r[:s ** 3].view(1, s, s, s), e[:s ** 3].view(1, s, s, s), s,
                    bool(st["periodic"]), st)
    sim.capture(None, None)
    sim.close()


def train(net, cfgs, lr=1e-3, epochs=1, steps=None, log=None, pairs=None, max_seconds=None):
    """Online Adam on the pairs of every configuration in cfgs (epochs
    passes, or as many as it takes to reach `pairs` pairs when given; no
    further pair after max_seconds).  Returns the history [(epoch, seed,
    step, side, periodic, loss)]."""
    hist = []
    fits = lambda s: s >= 16 and s % (1 << (net.levels - 1)) == 0  # noqa: E731
    t_end = None if max_seconds is None else time.time() + max_seconds
    done = lambda: ((pairs is not None and len(hist) >= pairs) or  # noqa: E731
                    (t_end is not None and time.time() >= t_end))

    ep = 0
    while ep < epochs or (pairs is not None and not done()):
        for cfg in cfgs:
            if done():
                break

            def on_pair(k, r, e, s, per, st):
                if not fits(s) or done():
                    return
                loss = net.loss_grad(r, e, per, 1)
                net.adam(lr)
                hist.append((ep, cfg["seed"], k, s, int(per), loss))
                if log is not None and len(hist) % 100 == 0:
                    log(f"pair {len(hist)} epoch {ep} seed {cfg['seed']} step {k} side {s} "
                        f"periodic {int(per)} |r_after|/|r| {np.sqrt(loss):.4f}")
            run_pairs(cfg, steps, on_pair, done)
        ep += 1
        if (pairs is None and ep >= epochs) or (t_end is not None and time.time() >= t_end):
            break
    return hist


def evaluate(cfg, net=None, precision="mixed", guess="warm", steps=None, profile=False):
    """Run one realisation; V-cycles per solve, solves the network started,
    wall time (events on the context stream) and, with profile, the
    per-class times of pm_profile."""
    pos, mom, ids = ics.workload_ics(cfg)
    sim = Sim(pos, mom, ids, cfg["n"], cfg["box"], cfg["a_init"], cfg["a_final"], cfg["steps"],
              rtol=cfg["rtol"], precision=precision, guess=guess)
    if net is not None:
        sim.set_guess(net)
    if profile:
        sim.profile(True)
    k = cfg["steps"] if steps is None else steps
    vc, r0, rg, side = [], [], [], []
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(sim.stream)
    for _ in range(k):
        sim.step(1)
        st = sim.stats()
        vc.append(st["vcycles_last"])
        r0.append(st["resid_start"])
        rg.append(st["resid_guess"])
        side.append(st["cube_side"] * (1 if st["periodic"] else -1))
    t1.record(sim.stream)
    torch.cuda.synchronize()
    st = sim.stats()
    out = dict(steps=k, vcycles=vc, resid_start=r0, resid_guess=rg, side=side,
               vcycles_total=int(st["vcycles_total"]),
               guess_used=int(st["guess_used_total"]), ms=t0.elapsed_time(t1),
               particle_steps=int(st["particle_steps"]), resid_last=st["resid_last"])
    if profile:
        out["profile"] = sim.profile_read()
    sim.close()
    return out


def save(path, net, hist=None, meta=None):
    np.savez(path, params=net.params(), levels=net.levels, out_scale=net.out_scale,
             hist=np.array(hist if hist else [], dtype=np.float64),
             meta=json.dumps(meta or {}))


def load(path):
    z = np.load(path)
    return GuessNet(int(z["levels"]), params=z["params"], out_scale=float(z["out_scale"]))


def compare(workload, weights=DEFAULT_WEIGHTS, modes=("warm", "learned"), steps=None):
    """The same realisation solved from each start: V-cycles, time and the
    factor by which the network shrank the start residual."""
    cfg = dict(ics.WORKLOADS[workload])
    out = {"workload": workload, "weights": os.path.basename(weights)}
    for mode in modes:
        net = load(weights) if mode == "learned" else None
        r = evaluate(cfg, net, guess=mode, steps=steps, profile=True)
        if net is not None:
            net.close()
        prof = r.pop("profile")
        row = {k: r[k] for k in ("steps", "vcycles_total", "guess_used", "particle_steps")}
        row["ms"] = round(r["ms"], 2)
        row["particle_steps_per_s"] = r["particle_steps"] / (r["ms"] * 1e-3)
        row["guess_ms"] = round(prof["guess"]["ms"], 2)
        row["vcycle_ms"] = round(sum(prof[k]["ms"] for k in
                                     ("smooth0", "transfer0", "coarse", "defect")), 2)
        if mode == "learned":
            ratio = [g / s for g, s, u in zip(r["resid_guess"], r["resid_start"], r["vcycles"])
                     if s > 0]
            row["resid_ratio_median"] = float(np.median(ratio))
        out[mode] = row
    if "warm" in out and "learned" in out:
        out["vcycles_saved"] = out["warm"]["vcycles_total"] - out["learned"]["vcycles_total"]
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--workload", default="pm256")
    ap.add_argument("--seeds", type=int, nargs="+", default=[1])
    ap.add_argument("--epochs", type=int, default=1)
    ap.add_argument("--pairs", type=int, default=None,
                    help="train until this many pairs (passes over the seeds as needed)")
    ap.add_argument("--max-seconds", type=float, default=None,
                    help="take no further pair after this long")
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--levels", type=int, default=4)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--init", default=None, help="start from saved weights")
    ap.add_argument("--out", default=None)
    ap.add_argument("--eval", action="store_true",
                    help="compare warm and learned starts on --workload instead of training")
    ap.add_argument("--weights", default=DEFAULT_WEIGHTS)
    ap.add_argument("--modes", nargs="+", default=["warm", "learned"])
    a = ap.parse_args(argv)
    from . import build
    build.build()
    if a.eval:
        print(json.dumps(compare(a.workload, a.weights, a.modes, a.steps)))
        return 0
    if not a.out:
        ap.error("--out is required for training")
    net = load(a.init) if a.init else GuessNet(a.levels, out_scale=1.0)
    cfgs = []
    for s in a.seeds:
        c = dict(ics.WORKLOADS[a.workload])
        c["seed"] = s
        cfgs.append(c)
    t0 = time.time()
    hist = train(net, cfgs, a.lr, a.epochs, a.steps,
                 log=lambda m: print(m, file=sys.stderr, flush=True), pairs=a.pairs,
                 max_seconds=a.max_seconds)
    save(a.out, net, hist, dict(workload=a.workload, seeds=a.seeds, epochs=a.epochs,
                                pairs=len(hist), lr=a.lr, seconds=time.time() - t0))
    print(json.dumps(dict(pairs=len(hist), seconds=round(time.time() - t0, 1),
                          last_ratio=float(np.sqrt(hist[-1][-1])) if hist else None)))
    return 0


if __name__ == "__main__":
    sys.exit(main())
