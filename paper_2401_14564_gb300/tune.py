"""Autotuner for the launch shapes of the hot path.

Choices it sweeps, each timed with CUDA events through the C ABI on the
workload itself (inputs on the device, median of a few repetitions):
  - pp_make_ff_tuned: z-nodes per thread (4, 8, 16);
  - pp_relax_scan: force-field layout, linear or bricked (several brick shapes),
    timed on the scan alone, or on whole steps several in flight (afm.Pipeline)
    when the caller runs them that way: the two regimes can prefer different
    layouts (a lone scan is bound by its slowest columns' dependency chains,
    overlapped steps by issue slots and cache capacity);
  - pp_batch_run: the work-item shapes (force-field tile depth and width, relax tile width) and
    the persistent CTA count.
Every candidate computes the same values (the layout and the launch shape do
not change the arithmetic per node or per pixel), so the pick is a pure
speed decision.  Results are cached in a JSON file keyed by GPU name and
workload shape.
"""
from __future__ import annotations

import json
import os
import statistics

import torch

from . import afm, pp

BRICKS = [(0, None), (1, (4, 4, 4)), (1, (8, 8, 2)), (1, (8, 4, 4)), (1, (16, 4, 2)), (1, (4, 4, 8))]
ZPTS = (4, 8, 16)


def _key(case):
    g, s = case["grid"], case["scan"]
    return (f"{torch.cuda.get_device_name()}|grid{g['nx']}x{g['ny']}x{g['nz']}|atoms{len(case['atoms']['x'])}"
            f"|scan{s['nx']}x{s['ny']}x{s['nz']}|mi{case['probe']['min_image']}|rc{case['probe']['coul_rc']}"
            f"|qzz{case['probe'].get('Qzz', 0.0)}|interp{case['grid'].get('interp', 0)}")


def _time(fn, reps):
    stream = torch.cuda.current_stream()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def tune_case(case, reps=3, bricks=BRICKS, zpts=ZPTS, ff_energy=True, pipeline_slots=0):
    """Time every FF launch shape and every grid layout for the relaxation; return the fastest.
    ff_energy=False times the forces-only assembly (the one a Simulator with ff_energy=False runs).
    pipeline_slots > 0 times each layout on 4 x pipeline_slots whole steps through an
    afm.Pipeline of that many slots (the regime of Pipeline.run_many) instead of the scan alone."""
    atoms_t = afm.atoms_to_device(case["atoms"])
    atoms = pp.make_atoms(atoms_t)
    probe = pp.make_probe(case["probe"])
    ff_times = {}
    grid0 = pp.make_grid(case["grid"], 0)
    ff = torch.empty(pp.pp_ff_floats(grid0), dtype=torch.float32, device="cuda")
    for z in zpts:
        t = pp.Tuning(z, 0 if ff_energy or case["grid"].get("interp", 0) else 1)
        pp.pp_make_ff_tuned(atoms, probe, grid0, ff, t)
        ff_times[z] = _time(lambda: pp.pp_make_ff_tuned(atoms, probe, grid0, ff, t), reps)
    best_z = min(ff_times, key=ff_times.get)
    if case["grid"].get("interp", 0):
        bricks = [(0, None)]  # tricubic energy grids are linear
    relax_times = {}
    for layout, brick in bricks:
        if pipeline_slots > 0:
            tun = {"ff_zpt": best_z, "layout": layout, "brick": list(brick) if brick else None}
            pipe = afm.Pipeline(case, slots=pipeline_slots, tuning=tun,
                                ff_energy=ff_energy or bool(case["grid"].get("interp", 0)))
            items = [atoms_t] * (4 * pipeline_slots)
            pipe.run_many(items)
            relax_times[f"{layout}:{brick}"] = _time(lambda: pipe.run_many(items), reps) / len(items)
            del pipe
            torch.cuda.empty_cache()
            continue
        sim = afm.Simulator(case, layout=layout, brick=brick or (4, 4, 4), want_pos=False, want_iters=False)
        sim.make_ff(atoms_t)
        sim.relax()
        relax_times[f"{layout}:{brick}"] = _time(sim.relax, reps)
        del sim
    best = min(relax_times, key=relax_times.get)
    layout, brick = best.split(":", 1)
    brick = None if brick == "None" else tuple(int(v) for v in brick.strip("()").split(","))
    return {"ff_zpt": best_z, "layout": int(layout), "brick": list(brick) if brick else None,
            "ff_ms": ff_times, "relax_ms": relax_times,
            "layout_timing": "ms per step, whole steps %d in flight" % pipeline_slots if pipeline_slots > 0
            else "ms per scan alone"}


BATCH_SHAPES = (("ff_zpt", (8, 4)), ("ff_tile_w", (8, 4, 16)), ("relax_tile_w", (8, 4, 16)))


def tune_batch(batch_obj, reps=2, factors=(1, 2, 3, 4, 5, 6)):
    """Pick the batch's work-item shapes (force-field tile depth and width, relax tile width) and
    its persistent CTA count (0 = as many as fit, else multiples of the SM count) by coordinate
    descent from the defaults: each choice in turn is swept with the others held at their best so
    far, timing pp_batch_run itself (CUDA events, median of reps).  Every choice computes the
    same molecules bit for bit.  Leaves the pick in batch_obj.params and returns it with the
    timings."""
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    p = batch_obj.params
    tried = {}

    def run_with(cfg):
        key = ",".join(f"{k}={v}" for k, v in sorted(cfg.items()))
        if key not in tried:
            for k, v in cfg.items():
                setattr(p, k, v)
            batch_obj.run()
            tried[key] = _time(batch_obj.run, reps)
        return tried[key]

    best = {"ff_zpt": 8, "ff_tile_w": 8, "relax_tile_w": 8, "ctas": 0}
    t_default = best_t = run_with(best)
    for name, values in BATCH_SHAPES + (("ctas", (0,) + tuple(f * sms for f in factors)),):
        for v in values:
            cfg = dict(best, **{name: v})
            t = run_with(cfg)
            if t < best_t:
                best, best_t = cfg, t
    for k, v in best.items():
        setattr(p, k, v)
    return {"choice": best, "ms": best_t, "ms_default_shapes": t_default, "tried_ms": tried,
            "how": "coordinate descent over ff_zpt, ff_tile_w, relax_tile_w, then ctas; median of %d timed runs "
                   "each" % reps}


def cached(case, path=None, **kw):
    """tune_case() result from the cache at `path` (JSON), computing and storing it if absent."""
    path = path or os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")
    db = {}
    if os.path.exists(path):
        with open(path) as f:
            db = json.load(f)
    k = _key(case) + ("" if kw.get("ff_energy", True) else "|forces_only") + (
        f"|pipeline{kw['pipeline_slots']}" if kw.get("pipeline_slots", 0) else "")
    if k not in db:
        r = tune_case(case, **kw)
        db[k] = {"ff_zpt": r["ff_zpt"], "layout": r["layout"], "brick": r["brick"],
                 "ff_ms": {str(a): b for a, b in r["ff_ms"].items()}, "relax_ms": r["relax_ms"]}
        tmp = path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(db, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    return db[k]
