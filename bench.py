"""Benchmark of the probe-particle hot path on the 60-atom flake workload.

One step = FF grid assembly (K1: 256x256x200 nodes x 60 atoms) + relaxed scan
with the fused df epilogue (K2: 256x256 pixels x 40 heights, FIRE <= 200
iterations, ftol 1e-4 eV/A).  Inputs are seeded synthetic atoms resident in
HBM.  The L2 is flushed (a 256 MiB write, outside the timed events) before
every timed step.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the method as plain loops) on a
bounded sample of the same workload, on this machine's host cores.
N > 1 (torchrun): every rank runs an independent replica of the workload
(weak scaling; the method has no exchange between replicas).
"""
from __future__ import annotations

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

METRIC = "relaxed pixel·z-steps/sec + FF grid·atom evals/sec vs roofline; batched mol/s; bwd/fwd"
UNIT = "pixel·z-steps/s"
FLOPS_PER_PAIR = 30          # algorithmic FP32 flops per grid-node/atom pair (FMA = 2)
FLOPS_PER_PAIR_QUAD = 45     # the same with the tip-quadrupole term (+15)
FLOPS_PER_PAIR_FORCES = 26   # forces only: FLOPS_PER_PAIR without the 4 flops of the energy sum
QZZ_CO = -0.05               # CO tip quadrupole of the paper's point-charge simulations, e*A^2
BYTES_PER_FIRE_ITER = 96     # 8 corners x (Fx, Fy, Fz) FP32 per FIRE iteration
SM_COUNT_NOMINAL = 152       # GB300; the bench reads the count from the device it runs on

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from single-launch ncu
# captures summarised in profiles/, valid only for the kernel sources they were taken on: the
# bench reports them when the sources still hash the same, else traffic is null.
TRAFFIC = {
    "relax_scan": {"bytes": 66.21e6, "sha": "65e56d7ba4e85d47",
                   "files": ["relax_scan.cu", "relax_core.cuh", "interp.cuh"]},
    "relax_scan_tricubic": {"bytes": 24.60e6, "sha": "65e56d7ba4e85d47",
                            "files": ["relax_scan.cu", "relax_core.cuh", "interp.cuh"]},
    "ff_assemble": {"bytes": 148.45e6, "bytes_zpt16": 139.83e6, "sha": "82384c014f2b4572",
                    "files": ["ff_assemble.cu", "ff_core.cuh", "interp.cuh"]},
    "ff_assemble_quad": {"bytes": 148.68e6, "sha": "82384c014f2b4572",
                         "files": ["ff_assemble.cu", "ff_core.cuh", "interp.cuh"]},
    "ff_assemble_split": {"bytes": 357.10e6, "sha": "82384c014f2b4572",
                          "files": ["ff_assemble.cu", "ff_core.cuh", "interp.cuh"]},
    "ff_combine": {"bytes": 600.65e6, "sha": "82384c014f2b4572",
                   "files": ["ff_assemble.cu", "ff_core.cuh", "interp.cuh"]},
}


def measured_traffic(kernel, zpt=8):
    t = TRAFFIC[kernel]
    if _src_hash(t["files"]) != t["sha"]:
        return None
    return t.get("bytes_zpt16") if int(zpt) == 16 and kernel == "ff_assemble" else t["bytes"]
FP32_LANES_PER_SM = 128

# Figures from single-kernel ncu captures summarised in profiles/, valid for the sources they were
# taken on (same hash rule as TRAFFIC): the FP32 operations K1 executes per node-atom pair
# (sm__sass_thread_inst_executed_op_{fadd,fmul,ffma}_pred_on, FFMA counted twice, over the pairs of
# the launch) and the issue-active fraction of K2 (smsp__issue_active.avg.pct_of_peak_sustained_active).
EXECUTED = {  # per z-nodes-per-thread launch shape (16: a bulk launch of 12 x 16 layers and a tail of 8)
    "ff_forces": {"value": {8: 18.69, 16: 18.37}, "sha": "82384c014f2b4572",
                  "files": ["ff_assemble.cu", "ff_core.cuh", "interp.cuh"]},
    "ff_energy": {"value": None, "sha": None, "files": ["ff_assemble.cu", "ff_core.cuh", "interp.cuh"]},
}
ISSUE = {
    "relax_scan": {"value": 0.573, "sha": "65e56d7ba4e85d47", "files": ["relax_scan.cu", "relax_core.cuh", "interp.cuh"]},
}


def _src_hash(files):
    import hashlib

    h = hashlib.sha1()
    for f in files:
        with open(os.path.join(ROOT, "paper_2401_14564_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def executed_ff_flops(energy, zpt=8):
    t = EXECUTED["ff_energy" if energy else "ff_forces"]
    if t["value"] is None or t["sha"] != _src_hash(t["files"]):
        return None
    return t["value"].get(int(zpt))


def measured_issue(kernel):
    t = ISSUE[kernel]
    return t["value"] if t["sha"] == _src_hash(t["files"]) else None


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def sm_count():
    import torch

    return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)


def fp32_peak_tflops(sm_mhz, sms):
    return sms * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


def measure_l2_peak(reps=10, sizes_mib=(8, 16, 32, 48), bytes_per_launch=8 << 30):
    """L2 read bandwidth of this device: pp_read_probe (16-byte loads that bypass L1, every
    resident thread of a full-GPU grid) over buffers well inside the 129 MB L2, each launch
    reading about bytes_per_launch (several hundred microseconds, so that clocks and caches are in
    their steady state) once resident; best of reps CUDA-event timings per size, the best size
    kept."""
    import torch

    from paper_2401_14564_gb300 import pp

    sink = torch.zeros(1, device="cuda")
    stream = torch.cuda.current_stream()
    per_size = {}
    for mib in sizes_mib:
        buf = torch.rand(mib * (1 << 20) // 4, device="cuda")
        passes = max(1, bytes_per_launch // (mib << 20))
        for _ in range(3):
            pp.pp_read_probe(buf, passes, sink)
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pp.pp_read_probe(buf, passes, sink)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        per_size[mib] = passes * buf.numel() * 4 / (min(ts) * 1e-3) / 1e9
        del buf
    best = max(per_size, key=per_size.get)
    return {"peak_gbs": per_size[best], "read_gbs_by_mib": per_size, "buffer_mib": best,
            "how": "pp_read_probe (16-byte L1-bypassing loads from every resident thread) reading an L2-resident "
                   f"buffer of {best} MiB {max(1, bytes_per_launch // (best << 20))} times per launch; best of {reps} "
                   f"CUDA-event timings, best of {', '.join(str(m) for m in sizes_mib)} MiB"}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms.  The sampler is started (and its
    first sample awaited) before the timed region; only samples taken between begin() and end()
    are reported."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line))

    def start(self):
        import threading

        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={','.join(self.FIELDS)}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        threading.Thread(target=self._read, daemon=True).start()
        deadline = time.perf_counter() + 10.0
        while not self.lines and time.perf_counter() < deadline:
            time.sleep(0.01)

    def begin(self):
        self.t0 = time.perf_counter()

    def end(self):
        self.t1 = time.perf_counter()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.06)  # one more sample period
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        t0, t1 = self.t0 or 0.0, self.t1 or float("inf")
        inside = [ln for t, ln in self.lines if t0 <= t <= t1 + 0.05]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in inside:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < len(self.FIELDS):
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(case, target_s=12.0, chunk=8192, max_cols=None, full_ff=True):
    """FP64 oracle on a bounded sample of the flake workload, scaled to pixel.z-steps/s.

    Sample: the FF grid (all 256x256x200 nodes when full_ff, else the 71
    z-layers the probe visits, nodes 20..90, extrapolated by 200/71), then the
    relaxed scan (40 heights, with df) of seeded random pixel columns in chunks
    of `chunk` until the whole sample has taken about target_s seconds, all
    65536 columns are done, or max_cols is reached; the scan time is
    extrapolated by 65536 / (columns done).
    """
    import oracle

    g, s = case["grid"], case["scan"]
    npix = s["nx"] * s["ny"]
    k0, k1 = (0, g["nz"]) if full_ff else (20, 91)
    slab = dict(g, nz=k1 - k0, z0=g["z0"] + k0 * g["dz"])
    t0 = time.perf_counter()
    ff, _ = oracle.make_ff(case["atoms"], case["probe"], slab)
    t_ff = time.perf_counter() - t0
    order = np.random.default_rng(0).permutation(npix)
    limit = npix if max_cols is None else min(npix, max_cols)
    done, t_rx = 0, 0.0
    while done < limit and (done == 0 or t_ff + t_rx < target_s):
        cols = np.sort(order[done:min(limit, done + chunk)])
        t0 = time.perf_counter()
        r = oracle.relax_columns(ff, slab, None, None, s, case["tip"], case["fire"], cols, polish_tol=0.0)
        oracle.fz_to_df(r["fz"].T, s["dz"], case["df"])
        t_rx += time.perf_counter() - t0
        done += len(cols)
    t_full = t_ff * g["nz"] / (k1 - k0) + t_rx * npix / done
    reps = [t_full]
    # the whole workload fits in the budget: repeat it to a ~target_s sample and take the median
    while done == npix and max_cols is None and sum(reps) < target_s and len(reps) < 20:
        t0 = time.perf_counter()
        ff, _ = oracle.make_ff(case["atoms"], case["probe"], slab)
        r = oracle.relax_columns(ff, slab, None, None, s, case["tip"], case["fire"], np.arange(npix), polish_tol=0.0)
        oracle.fz_to_df(r["fz"].T, s["dz"], case["df"])
        reps.append(time.perf_counter() - t0)
    t_full = statistics.median(reps)
    units = npix * s["nz"]
    ff_desc = ("FF on all 256x256x200 nodes" if full_ff else "FF on nodes z 20..90 of 256x256x200, scaled by 200/71")
    scan_desc = (f"all {npix} pixel columns (the whole workload; median of {len(reps)} runs)" if done == npix
                 else f"{done} of {npix} seeded random pixel columns, scaled by {npix}/{done}")
    # the same on one core, on a small sample: 2 of the 200 grid planes and 256 seeded columns
    cores = oracle.max_threads()
    t0 = time.perf_counter()
    oracle.make_ff(case["atoms"], case["probe"], dict(g, nz=2), nthreads=1)
    t1_ff = (time.perf_counter() - t0) * g["nz"] / 2
    cols1 = np.sort(order[:256])
    t0 = time.perf_counter()
    r = oracle.relax_columns(ff, slab, None, None, s, case["tip"], case["fire"], cols1, polish_tol=0.0, nthreads=1)
    oracle.fz_to_df(r["fz"].T, s["dz"], case["df"])
    t1_rx = (time.perf_counter() - t0) * npix / len(cols1)
    oracle.make_ff(case["atoms"], case["probe"], dict(g, nz=2), nthreads=cores)  # restores the thread count
    return {"value": units / t_full, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"{ff_desc} ({(k1 - k0) * 256 * 256 * 60 / 1e6:.0f} M pairs, FP64, OpenMP) + FIRE scan "
                       f"(no Newton polish) x 40 heights + df of {scan_desc}"),
            "sample_seconds": sum(reps) if len(reps) > 1 else t_ff + t_rx, "ff_seconds": t_ff, "scan_columns": done,
            "repetitions": len(reps),
            "one_core": {"value": units / (t1_ff + t1_rx), "unit": UNIT, "cores": 1,
                         "sample": "FF on 2 of the 200 grid planes scaled by 100, FIRE scan + df of 256 seeded "
                                   "pixel columns scaled by 256"}}


def cpu_baseline_other():
    """FP64 oracle (all host cores) on stated samples of the batched and the slab workloads,
    reported per unit and projected to the whole workload.

    batch: the first 16 of the 1024 molecules, each FF grid + FIRE scan (no Newton polish) + df.
    slab: a 32 x 32 pixel tile at the centre of the 512 x 512 scan, all 60 heights, relaxed on an
    80 x 80 x 101 node window of the grid (2.4 A lateral margin, z 9 .. 19 A) built by direct
    minimum-image sums; FF pairs/s and pixel-heights/s projected to the 512 x 512 x 250 grid
    (1.65e11 pairs) and the 512 x 512 x 60 scan."""
    import oracle

    from paper_2401_14564_gb300 import synth

    out = {"cores": oracle.max_threads()}
    cases = synth.batch_cases(16)
    t0 = time.perf_counter()
    for c in cases:
        ff, _ = oracle.make_ff(c["atoms"], c["probe"], c["grid"])
        r = oracle.relax_scan(ff, c["grid"], c["atoms"], c["probe"], c["scan"], c["tip"], c["fire"], polish_tol=0.0)
        oracle.fz_to_df(r["fz"], c["scan"]["dz"], c["df"])
    t = time.perf_counter() - t0
    out["batch"] = {"mol_per_s": len(cases) / t, "seconds": t,
                    "sample": "molecules 1000..1015 of the 1024 (FF grid + FIRE scan + df each)"}
    c = synth.slab_case()
    g, s = c["grid"], c["scan"]
    i0, n, m = 240, 32, 24
    win = dict(g, nx=n + 2 * m, ny=n + 2 * m, nz=101, x0=g["x0"] + (i0 - m) * g["dx"],
               y0=g["y0"] + (i0 - m) * g["dy"], z0=g["z0"] + 90 * g["dz"], periodic_xy=0,
               Lx=g["nx"] * g["dx"], Ly=g["ny"] * g["dy"])
    t0 = time.perf_counter()
    ffw, _ = oracle.make_ff(c["atoms"], c["probe"], win)
    t_ff = time.perf_counter() - t0
    jj, ii = np.meshgrid(np.arange(i0, i0 + n), np.arange(i0, i0 + n), indexing="ij")
    cols = (jj * s["nx"] + ii).ravel()
    t0 = time.perf_counter()
    r = oracle.relax_columns(ffw, win, None, None, s, c["tip"], c["fire"], cols, polish_tol=0.0)
    oracle.fz_to_df(r["fz"].T, s["dz"], c["df"])
    t_rx = time.perf_counter() - t0
    natoms = len(c["atoms"]["x"])
    pairs_rate = win["nx"] * win["ny"] * win["nz"] * natoms / t_ff
    pz_rate = len(cols) * s["nz"] / t_rx
    full = g["nx"] * g["ny"] * g["nz"] * natoms / pairs_rate + s["nx"] * s["ny"] * s["nz"] / pz_rate
    out["slab"] = {"ff_pairs_per_s": pairs_rate, "pixel_z_per_s": pz_rate, "projected_forward_s": full,
                   "sample": f"FF on an {win['nx']}x{win['ny']}x{win['nz']} node window, scan of a {n}x{n} px "
                             "tile x 60 heights"}
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    from paper_2401_14564_gb300 import synth

    case = synth.flake_case()
    for _ in range(args.warmup):
        cpu_baseline(case, chunk=64, max_cols=64, full_ff=False)
    vals = []
    info = None
    for _ in range(args.steps):
        info = cpu_baseline(case, chunk=256, max_cols=256, full_ff=False)
        vals.append(info["value"])
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * case["scan"]["nx"] * case["scan"]["ny"]
            * case["scan"]["nz"] / value, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": workload_config(case, args.ff_energy),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": info["cores"], "kind": "oracle",
                             "sample": info["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


PLAN_FRAC, PLAN_LANES = 0.025, 4  # the scan plan's share of pixel columns and lanes per warp


def neighbour_case(case, seed=77, shift=0.05, dq=0.1):
    """The case with every atom moved by up to `shift` A per axis and every charge scaled by up to
    1 +- dq (seeded): the input the scan's pixel-to-warp plan is built from."""
    rng = np.random.default_rng(seed)
    atoms = dict(case["atoms"])
    for k in ("x", "y", "z"):
        v = np.asarray(atoms[k], dtype=np.float64)
        atoms[k] = v + rng.uniform(-shift, shift, size=v.shape)
    q = np.asarray(atoms["q"], dtype=np.float64)
    atoms["q"] = q * (1.0 + rng.uniform(-dq, dq, size=q.shape))
    return dict(case, atoms=atoms)


def workload_config(case, ff_energy=False):
    g, s = case["grid"], case["scan"]
    return {"workload": "flake60: 60-atom H-terminated aromatic flake (seed 42), FF grid 256x256x200 at 0.1 A, "
                        "scan 256x256 px x 40 heights, FIRE<=200 ftol 1e-4, df A=1 A k=1800 N/m f0=30.3 kHz",
            "atoms": len(case["atoms"]["x"]), "grid": [g["nx"], g["ny"], g["nz"]], "scan": [s["nx"], s["ny"], s["nz"]],
            "parallelism": "replicas",
            "ff": "forces and energies" if ff_energy else
                  "forces only: E slots written as 0 (the scan reads only the forces; --ff-energy adds E)",
            "l2": "headline steps: no flush, each step writes its own 210 MB FF grid (> the 129 MB L2) and reads "
                  "it back; per-kernel timings: 256 MiB write before every step"}


def measure_bwd_fwd(case, steps, warmup, flush, tag, ff_energy=False):
    """CUDA-event times of the forward (FF + relaxed scan + df) and of pp_backward on one workload
    (the adjoint reads the grid's forces only, so the forward assembles them as the main step does)."""
    import torch

    from paper_2401_14564_gb300 import afm, pp

    sim = afm.Simulator(case, ff_energy=ff_energy, plan_frac=0.0)
    atoms_t = afm.atoms_to_device(case["atoms"])
    n = len(case["atoms"]["x"])
    grads = {k: torch.empty(n, device="cuda") for k in ("x", "y", "z", "q", "R", "eps")}
    grads["tip"] = torch.empty(5, device="cuda")
    ws = torch.empty(pp.pp_backward_workspace(sim.grid) // 4 + 1, dtype=torch.float32, device="cuda")
    w = torch.randn(tuple(sim.df.shape), generator=torch.Generator().manual_seed(7)).to("cuda")
    atoms = pp.make_atoms(atoms_t)
    g = pp.make_grads(grads)

    def bwd():
        pp.pp_backward(atoms, sim.probe, sim.grid, sim.ff, sim.scan, sim.tip, sim.dfp, sim.pos, w, g, ws)

    for _ in range(max(warmup, 3)):
        sim.run(atoms_t)
        bwd()
    stream = torch.cuda.current_stream()
    tf, tb = [], []
    for _ in range(steps):
        flush.zero_()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        sim.run(atoms_t)
        e1.record(stream)
        flush.zero_()
        e2a = torch.cuda.Event(enable_timing=True)
        e2a.record(stream)
        bwd()
        e2.record(stream)
        torch.cuda.synchronize()
        tf.append(e0.elapsed_time(e1))
        tb.append(e2a.elapsed_time(e2))
    f, b = statistics.mean(tf), statistics.mean(tb)
    # the same forward with the force field in two parts beside the scan (Simulator.run_overlapped;
    # the first call learns the layers the scan reads, untimed)
    sim.run_overlapped(atoms_t, stream)
    torch.cuda.synchronize()
    sim.overlap_held()
    to, held = [], 0
    for _ in range(steps):
        flush.zero_()
        e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
        e0.record(stream)
        first = sim.run_overlapped(atoms_t, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        held += bool(sim.overlap_held())
        to.append(e0.elapsed_time(e1))
    return {"workload": tag, "fwd_ms": f, "bwd_ms": b, "ratio": b / f, "ff_energy": bool(ff_energy),
            "fwd_overlapped_ms": statistics.mean(to), "overlap": {"first_layers": list(first),
                                                                 "grid_layers": case["grid"]["nz"],
                                                                 "steps_held": held, "steps": steps},
            "note": "forward = FF + relaxed scan + fused df; backward = pp_backward (df adjoint, 3x3 implicit solves, "
                    "grid-adjoint scatter, per-atom pair-derivative sums); L2 flushed before each; "
                    "fwd_overlapped_ms: the force field of the layers the scan reads first, the rest beside "
                    "the scan (a step that left the first part would need its scan again: steps_held counts "
                    "those that did not)"}


def measure_slab(steps, warmup, flush, ff_energy=False):
    """2516-atom periodic slab: 512x512x250 grid with minimum image and an 8 A shifted-force
    Coulomb cut, 512x512 px x 60 heights; forward and adjoint times."""
    import torch

    from paper_2401_14564_gb300 import synth

    case = synth.slab_case()
    r = measure_bwd_fwd(case, steps, warmup, flush, "slab2016+mol500: 2516 atoms, grid 512x512x250, scan 512x512x60",
                        ff_energy)
    g, s = case["grid"], case["scan"]
    pairs = g["nx"] * g["ny"] * g["nz"] * len(case["atoms"]["x"])
    r["pixel_z_per_s_fwd"] = s["nx"] * s["ny"] * s["nz"] / (r["fwd_ms"] * 1e-3)
    r["pairs"] = pairs
    torch.cuda.empty_cache()
    return r


def measure_quadrupole(case, tuning, steps, warmup, flush, alu_peak):
    """The line's workload with the CO tip's quadrupole (Qzz = -0.05 e*A^2): K1's quadrupole
    variant and the whole step (FF + relaxed scan + fused df), CUDA events, L2 flushed."""
    import torch

    from paper_2401_14564_gb300 import afm

    qcase = dict(case, probe=dict(case["probe"], Qzz=QZZ_CO))
    sim = afm.Simulator(qcase, tuning=tuning, plan_frac=0.0)
    atoms = afm.atoms_to_device(qcase["atoms"])
    for _ in range(max(warmup, 3)):
        sim.run(atoms)
    stream = torch.cuda.current_stream()
    t_ff, t_rx = [], []
    for _ in range(steps):
        flush.zero_()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        sim.make_ff(atoms)
        e1.record(stream)
        sim.relax()
        e2.record(stream)
        torch.cuda.synchronize()
        t_ff.append(e0.elapsed_time(e1))
        t_rx.append(e1.elapsed_time(e2))
    g, s = qcase["grid"], qcase["scan"]
    pairs = g["nx"] * g["ny"] * g["nz"] * len(qcase["atoms"]["x"])
    ff_ms, rx_ms = statistics.mean(t_ff), statistics.mean(t_rx)
    tflops = pairs * FLOPS_PER_PAIR_QUAD / (ff_ms * 1e-3) / 1e12
    return {"workload": "flake60 with tip quadrupole Qzz = -0.05 e*A^2", "ff_ms": ff_ms, "relax_ms": rx_ms,
            "ms_per_step": ff_ms + rx_ms, "pixel_z_per_s": s["nx"] * s["ny"] * s["nz"] / ((ff_ms + rx_ms) * 1e-3),
            "ff_pair_evals_per_s": pairs / (ff_ms * 1e-3), "ff_flops_per_pair": FLOPS_PER_PAIR_QUAD,
            "ff_achieved_tflops": tflops, "ff_frac_of_alu_peak": tflops / alu_peak,
            "ff_traffic": measured_traffic("ff_assemble_quad")}


def measure_tricubic(case, steps, warmup, flush, spacings=(0.1, 0.2)):
    """The line's workload on tricubic energy grids (one float per node, F = -grad of the tricubic
    interpolant): at the same 0.1 A spacing and at 0.2 A (8x fewer nodes); FF, relaxed scan
    (fused df) and adjoint (pp_backward) times by CUDA events, L2 flushed, grid bytes."""
    import torch

    from paper_2401_14564_gb300 import afm, pp

    out = []
    g0 = case["grid"]
    for h in spacings:
        f = round(h / g0["dx"])
        g = dict(g0, nx=g0["nx"] // f, ny=g0["ny"] // f, nz=(g0["nz"] - 1) // f + 1, dx=h, dy=h, dz=h, interp=1)
        tcase = dict(case, grid=g)
        sim = afm.Simulator(tcase, plan_frac=0.0)
        atoms = afm.atoms_to_device(tcase["atoms"])
        n = len(tcase["atoms"]["x"])
        grads = {k: torch.empty(n, device="cuda") for k in ("x", "y", "z", "q", "R", "eps")}
        grads["tip"] = torch.empty(5, device="cuda")
        ws = torch.empty(pp.pp_backward_workspace(sim.grid) // 4 + 1, dtype=torch.float32, device="cuda")
        w = torch.randn(tuple(sim.df.shape), generator=torch.Generator().manual_seed(7)).to("cuda")
        pa, pg = pp.make_atoms(atoms), pp.make_grads(grads)

        def bwd():
            pp.pp_backward(pa, sim.probe, sim.grid, sim.ff, sim.scan, sim.tip, sim.dfp, sim.pos, w, pg, ws)

        for _ in range(max(warmup, 3)):
            sim.run(atoms)
            bwd()
        stream = torch.cuda.current_stream()
        t_ff, t_rx, t_bw = [], [], []
        for _ in range(steps):
            flush.zero_()
            e0, e1, e2, e3, e4 = (torch.cuda.Event(enable_timing=True) for _ in range(5))
            e0.record(stream)
            sim.make_ff(atoms)
            e1.record(stream)
            sim.relax()
            e2.record(stream)
            flush.zero_()
            e3.record(stream)
            bwd()
            e4.record(stream)
            torch.cuda.synchronize()
            t_ff.append(e0.elapsed_time(e1))
            t_rx.append(e1.elapsed_time(e2))
            t_bw.append(e3.elapsed_time(e4))
        s = tcase["scan"]
        ff_ms, rx_ms = statistics.mean(t_ff), statistics.mean(t_rx)
        pairs = g["nx"] * g["ny"] * g["nz"] * len(tcase["atoms"]["x"])
        # the same steps four in flight (afm.Pipeline, as the line's headline): other items' FF and
        # scans fill the issue slots of a scan whose slowest columns set its end
        pipe = afm.Pipeline(tcase, slots=4)
        pipe.run_many([atoms] * 8)
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        pipe.run_many([atoms] * (4 * steps))
        p1.record(stream)
        torch.cuda.synchronize()
        pipe_ms = p0.elapsed_time(p1) / (4 * steps)
        del pipe
        out.append({"spacing": h, "grid": [g["nx"], g["ny"], g["nz"]], "grid_bytes": g["nx"] * g["ny"] * g["nz"] * 4,
                    "ff_ms": ff_ms, "relax_ms": rx_ms, "ms_per_step": ff_ms + rx_ms, "bwd_ms": statistics.mean(t_bw),
                    "pixel_z_per_s": s["nx"] * s["ny"] * s["nz"] / ((ff_ms + rx_ms) * 1e-3),
                    "ms_per_step_pipelined": pipe_ms,
                    "pixel_z_per_s_pipelined": s["nx"] * s["ny"] * s["nz"] / (pipe_ms * 1e-3),
                    "ff_pair_evals_per_s": pairs / (ff_ms * 1e-3),
                    "fire_iters_mean": float(sim.iters.float().mean().item()),
                    "relax_traffic": measured_traffic("relax_scan_tricubic") if h == 0.1 else None})
        del sim, ws
    return out


def measure_df(case, steps, flush, hbm_gbs, shape=(60, 512, 512)):
    """K3 alone (pp_fz_to_df) on a seeded Fz volume of the slab scan's shape (60 heights x 512 x 512
    pixels) with the line's df parameters: algorithmic bytes = Fz read once + df written once;
    CUDA events, L2 flushed before each."""
    import torch

    from paper_2401_14564_gb300 import pp

    nz, ny, nx = shape
    dfp = pp.make_df(case["df"])
    dz = case["scan"]["dz"]
    m = pp.pp_df_margin(dfp.A_pp, dz)
    g = torch.Generator(device="cuda").manual_seed(11)
    fz = torch.randn((nz, ny, nx), generator=g, device="cuda")
    df = torch.empty((nz - 2 * m, ny, nx), device="cuda")
    for _ in range(3):
        pp.pp_fz_to_df(fz, nz, nx * ny, dz, dfp, df)
    stream = torch.cuda.current_stream()
    ts = []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pp.pp_fz_to_df(fz, nz, nx * ny, dz, dfp, df)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = statistics.median(ts)
    nbytes = 4 * (nz + (nz - 2 * m)) * nx * ny
    return {"workload": f"Fz {nz} heights x {nx}x{ny} px (seeded), {2 * m + 1}-tap stencil", "ms": ms,
            "bytes": nbytes, "gbs": nbytes / (ms * 1e-3) / 1e9, "frac_of_hbm": nbytes / (ms * 1e-3) / 1e9 / hbm_gbs}


def measure_split(case, steps, warmup, flush, hbm_gbs):
    """The line's workload with the electrostatics kept apart (pp_make_ff_split: LJ grid + point-charge
    grid per unit probe charge) and recombined for the probe charge (pp_ff_combine, 12 bytes moved per
    float); CUDA events, L2 flushed before each."""
    import torch

    from paper_2401_14564_gb300 import afm, pp

    grid = pp.make_grid(case["grid"], 0)
    n = pp.pp_ff_floats(grid)
    ff = torch.empty(n, dtype=torch.float32, device="cuda")
    el = torch.empty(n, dtype=torch.float32, device="cuda")
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    atoms = pp.make_atoms(afm.atoms_to_device(case["atoms"]))
    probe = pp.make_probe(case["probe"])
    Q = float(case["probe"]["Q"])
    for _ in range(max(warmup, 3)):
        pp.pp_make_ff_split(atoms, probe, grid, ff, el)
        pp.pp_ff_combine(ff, el, Q, grid, out)
    stream = torch.cuda.current_stream()
    t_split, t_comb = [], []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pp.pp_make_ff_split(atoms, probe, grid, ff, el)
        e1.record(stream)
        flush.zero_()
        e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        pp.pp_ff_combine(ff, el, Q, grid, out)
        e3.record(stream)
        torch.cuda.synchronize()
        t_split.append(e0.elapsed_time(e1))
        t_comb.append(e2.elapsed_time(e3))
    g = case["grid"]
    pairs = g["nx"] * g["ny"] * g["nz"] * len(case["atoms"]["x"])
    sm, cm = statistics.mean(t_split), statistics.mean(t_comb)
    gbs = 12 * n / (cm * 1e-3) / 1e9
    del ff, el, out
    return {"workload": "flake60, LJ and point-charge grids apart, recombined for Q = -0.1",
            "split_ff_ms": sm, "split_pair_evals_per_s": pairs / (sm * 1e-3), "combine_ms": cm,
            "combine_bytes": 12 * n, "combine_gbs": gbs, "combine_frac_of_hbm": gbs / hbm_gbs,
            "split_ff_traffic": measured_traffic("ff_assemble_split"), "combine_traffic": measured_traffic("ff_combine")}


IETS_BYTES_PER_POINT = 164  # position 12 + the cell's 8 corner float4 128 + eigenvalues and mode energies 24


def measure_iets(case, steps, warmup, flush, hbm_gbs):
    """IETS map (pp_iets) at the relaxed positions of the line's workload, on the trilinear force
    grid and on the 0.1 A tricubic energy grid; CUDA events, L2 flushed before each."""
    import torch

    from paper_2401_14564_gb300 import afm, pp

    out = []
    for interp in (0, 1):
        c = dict(case, grid=dict(case["grid"], interp=interp))
        sim = afm.Simulator(c, plan_frac=0.0)
        sim.run(afm.atoms_to_device(c["atoms"]))
        s = c["scan"]
        npts = s["nx"] * s["ny"] * s["nz"]
        eig = torch.empty(3 * npts, device="cuda")
        hw = torch.empty(3 * npts, device="cuda")

        def go():
            pp.pp_iets(sim.ff, sim.grid, sim.scan, sim.tip, sim.pos, 16.0, eig, hw)

        for _ in range(max(warmup, 3)):
            go()
        stream = torch.cuda.current_stream()
        ts = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            go()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = statistics.mean(ts)
        entry = {"grid": "trilinear force grid" if interp == 0 else "tricubic energy grid", "ms": ms,
                 "points_per_s": npts / (ms * 1e-3)}
        if interp == 0:
            gbs = IETS_BYTES_PER_POINT * npts / (ms * 1e-3) / 1e9
            entry.update({"bytes_per_point": IETS_BYTES_PER_POINT, "gbs": gbs, "frac_of_hbm": gbs / hbm_gbs})
        out.append(entry)
        del sim, eig, hw
    return {"workload": "flake60 relaxed positions, 2.62 M points, CO mass 16 amu", "points": out}


FFT_BYTES_PER_NODE = 224  # one correlation: pack 16 + 3 forward passes 48 + spectral 32 + 6 inverse passes 96 + output 32
FDBM_A, FDBM_BETA = 18.0, 1.0  # Pauli prefactor and exponent of the synthetic full-density workload


def measure_fdbm_sweep(reps, flush, sizes=((5, 3), (10, 6), (20, 12))):
    """Force-field step on periodic graphene sheets of growing size (grid points proportional to
    atoms, as in the paper's performance figure): Lennard-Jones + point charges by direct summation
    (K1, minimum image) against the full-density model's two FFT correlations (Hartree electrostatics
    of a quadrupolar tip charge + Pauli repulsion) on the same grid.  Synthetic densities."""
    import torch

    from paper_2401_14564_gb300 import afm, pp, synth

    out = []
    stream = torch.cuda.current_stream()

    def timed(fn):
        ts = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    for na, nb in sizes:
        case = synth.graphene_sweep_case(na, nb)
        g = case["grid"]
        dev = lambda a: torch.as_tensor(np.asarray(a, np.float32), device="cuda").contiguous()  # noqa: E731
        rho = dev(synth.valence_density(g, case["atoms"]))
        V = dev(synth.hartree_potential(g, case["atoms"]))
        pauli, quad = (dev(t) for t in synth.tip_densities(g))
        grid = pp.make_grid(g, 0)
        ff = torch.empty(pp.pp_ff_floats(grid), dtype=torch.float32, device="cuda")
        ws = torch.empty(pp.pp_fft_workspace(grid) // 4, dtype=torch.float32, device="cuda")
        atoms = pp.make_atoms(afm.atoms_to_device(case["atoms"]))
        probe = pp.make_probe(case["probe"])

        def lj():
            pp.pp_make_ff(atoms, probe, grid, ff)

        def fdbm():
            pp.pp_fft_correlate(V, quad, grid, 1.0, 1.0, ff, ws)
            pp.pp_fft_correlate(rho, pauli, grid, FDBM_A, FDBM_BETA, ff, ws, accumulate=True)

        for _ in range(2):
            lj()
            fdbm()
        t_lj, t_fd = timed(lj), timed(fdbm)
        nodes = g["nx"] * g["ny"] * g["nz"]
        n = len(case["atoms"]["x"])
        fft_bytes = nodes * (2 * FFT_BYTES_PER_NODE + 16)
        out.append({"sheet": f"{na}x{nb} cells", "atoms": n, "grid": [g["nx"], g["ny"], g["nz"]], "nodes": nodes,
                    "lj_pc_ms": t_lj, "fdbm_ms": t_fd, "lj_pc_pairs_per_s": nodes * n / (t_lj * 1e-3),
                    "fdbm_nodes_per_s": nodes / (t_fd * 1e-3), "fdbm_gbs": fft_bytes / (t_fd * 1e-3) / 1e9})
        del rho, V, pauli, quad, ff, ws
        torch.cuda.empty_cache()
    return {"workload": "periodic graphene sheets, grid ~0.1 A x 0.1 A x 0.125 A (powers of two), synthetic "
                        "Gaussian valence densities and Poisson Hartree potential; FDBM A = %g, beta = %g"
                        % (FDBM_A, FDBM_BETA),
            "fft_bytes_per_node": FFT_BYTES_PER_NODE, "points": out}


def measure_small(case, steps, warmup, flush, alu_peak, ff_energy=False, cpu=True):
    """A whole workload small enough for the oracle to run in full (benzene: 80x80x60 grid x 12
    atoms, 40x40 px x 20 heights): FF pairs/s and relaxed pixel-heights/s of K1 + K2 (fused df)
    by CUDA events with the L2 flushed before each step, beside the FP64 oracle timed on the
    whole workload on all host cores and on one core (FF + FIRE scan without the Newton polish
    + df, median of repeats)."""
    import torch

    from paper_2401_14564_gb300 import afm

    sim = afm.Simulator(case, ff_energy=ff_energy, plan_frac=0.0)
    atoms = afm.atoms_to_device(case["atoms"])
    for _ in range(max(warmup, 3)):
        sim.run(atoms)
    stream = torch.cuda.current_stream()
    t_ff, t_rx = [], []
    for _ in range(steps):
        flush.zero_()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        sim.make_ff(atoms)
        e1.record(stream)
        sim.relax()
        e2.record(stream)
        torch.cuda.synchronize()
        t_ff.append(e0.elapsed_time(e1))
        t_rx.append(e1.elapsed_time(e2))
    g, s = case["grid"], case["scan"]
    pairs = g["nx"] * g["ny"] * g["nz"] * len(case["atoms"]["x"])
    units = s["nx"] * s["ny"] * s["nz"]
    ff_ms, rx_ms = statistics.median(t_ff), statistics.median(t_rx)
    flops_pair = FLOPS_PER_PAIR if ff_energy else FLOPS_PER_PAIR_FORCES
    out = {"workload": f"{case['name']}: {len(case['atoms']['x'])} atoms, grid {g['nx']}x{g['ny']}x{g['nz']}, "
                       f"scan {s['nx']}x{s['ny']}x{s['nz']}",
           "ff_ms": ff_ms, "relax_ms": rx_ms, "ms_per_step": ff_ms + rx_ms,
           "ff_pair_evals_per_s": pairs / (ff_ms * 1e-3),
           "ff_frac_of_alu_peak": pairs * flops_pair / (ff_ms * 1e-3) / 1e12 / alu_peak,
           "relax_pixel_z_per_s": units / (rx_ms * 1e-3), "pixel_z_per_s": units / ((ff_ms + rx_ms) * 1e-3),
           "fire_iters_mean": float(sim.iters.float().mean().item())}
    if cpu:
        import oracle

        def oracle_step(nthreads):
            t0 = time.perf_counter()
            ff, _ = oracle.make_ff(case["atoms"], case["probe"], g, nthreads=nthreads)
            t1 = time.perf_counter()
            r = oracle.relax_scan(ff, g, None, None, s, case["tip"], case["fire"], polish_tol=0.0, nthreads=nthreads)
            oracle.fz_to_df(r["fz"], s["dz"], case["df"])
            return t1 - t0, time.perf_counter() - t1

        cores = oracle.max_threads()
        for nt, key in ((cores, "oracle_all_cores"), (1, "oracle_one_core")):
            reps = [oracle_step(nt) for _ in range(3 if nt > 1 else 1)]
            tf = statistics.median(r[0] for r in reps)
            tr = statistics.median(r[1] for r in reps)
            out[key] = {"cores": nt, "ff_pair_evals_per_s": pairs / tf, "relax_pixel_z_per_s": units / tr,
                        "pixel_z_per_s": units / (tf + tr)}
        oracle.make_ff(case["atoms"], case["probe"], dict(g, nz=2), nthreads=cores)  # restores the thread count
    del sim
    return out


def measure_batch(n_mol, steps, warmup, flush, seq_sample=64, ff_energy=False, autotune=True):
    """Batched molecules/s: pp_batch_run over n_mol seeded molecules replayed from a CUDA graph,
    beside the same molecules run one by one through pp_make_ff + pp_relax_scan (both with or
    both without the grids' energy sums)."""
    import torch

    from paper_2401_14564_gb300 import afm, batch, synth

    from paper_2401_14564_gb300 import tune

    cases = synth.batch_cases(n_mol)
    b = batch.Batch(cases, ff_energy=ff_energy)
    autotune = tune.tune_batch(b) if autotune else None
    b.capture()
    for _ in range(max(warmup, 1)):
        b.replay()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ts = []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    st, flags = b.status()
    t = statistics.median(ts)
    # end to end: the packed host atoms in, the batch's graph, every molecule's df image back to
    # pinned host memory, synchronised, wall clock (median of 5 calls)
    b.pack_atoms(cases)
    b.run_host()
    t_e2e = []
    for _ in range(5):
        t0 = time.perf_counter()
        b.run_host()
        t_e2e.append(time.perf_counter() - t0)
    e2e_ms = 1e3 * statistics.median(t_e2e)
    # the same molecules one at a time (first seq_sample of them), per-molecule buffers preallocated
    sims = [(afm.Simulator(c, ff_energy=ff_energy, plan_frac=0.0), afm.atoms_to_device(c["atoms"]))
            for c in cases[:seq_sample]]
    for sim, at in sims:
        sim.run(at)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.zero_()
    e0.record(stream)
    for sim, at in sims:
        sim.run(at)
    e1.record(stream)
    torch.cuda.synchronize()
    t_seq = e0.elapsed_time(e1) / len(sims)
    del sims
    out = {"workload": f"{n_mol} seeded molecules of 10-80 H/C/N/O/F atoms (seeds 1000+i), grids 128-256^2 x 60 "
                       f"at 0.1 A, scans 128x128x20; one persistent launch in a CUDA graph",
           "mol_per_s": n_mol / (t * 1e-3), "ms_per_batch": t, "pixel_z_per_s": b.pixel_heights / (t * 1e-3),
           "ff_pair_evals_per_s": b.pairs / (t * 1e-3), "status": st, "ff_energy": bool(ff_energy),
           "autotune": autotune,
           "e2e": {"mol_per_s": n_mol / (e2e_ms * 1e-3), "ms_per_batch": e2e_ms, "h2d_bytes": b.h2d_bytes(),
                   "d2h_bytes": b.d2h_bytes(),
                   "note": "Batch.run_host: packed host atoms in, the graph replayed, all df images out to pinned "
                           "host memory, synchronised; wall clock, median of 5"},
           "single_path_mol_per_s": 1e3 / t_seq,
           "single_path_note": f"pp_make_ff + pp_relax_scan per molecule, mean over the first {seq_sample}",
           "gpu_launches_per_batch": 2}
    del b
    torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--layout", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-slab", action="store_true")
    ap.add_argument("--no-bwdfwd", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-quad", action="store_true")
    ap.add_argument("--no-tricubic", action="store_true")
    ap.add_argument("--no-fdbm", action="store_true")
    ap.add_argument("--no-split", action="store_true")
    ap.add_argument("--no-iets", action="store_true")
    ap.add_argument("--ff-energy", action="store_true",
                    help="assemble the grid's energies too (the scan reads only the forces; default: E slots 0)")
    ap.add_argument("--zpt", type=int, default=0, help="FF z-nodes per thread (skips the autotuner)")
    ap.add_argument("--brick", default="", help="bricked layout bx,by,bz for the scan (skips the autotuner)")
    ap.add_argument("--batch-mol", type=int, default=1024)
    ap.add_argument("--tricubic-spacings", default="0.1,0.2", help="grid spacings (A) of the tricubic leg")
    ap.add_argument("--no-batch-tune", action="store_true", help="batched leg on the default work-item shapes")
    args = ap.parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch

    from paper_2401_14564_gb300 import afm, pp, synth
    from paper_2401_14564_gb300 import dist as ppd

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    case = synth.flake_case()
    tuning = None
    if args.zpt or args.brick:
        tuning = {"ff_zpt": args.zpt or 8, "layout": 1 if args.brick else args.layout,
                  "brick": [int(v) for v in args.brick.split(",")] if args.brick else None}
    elif not args.no_tune:
        from paper_2401_14564_gb300 import tune

        # layouts timed the way the headline runs them: whole steps, four in flight
        tuning = tune.tune_case(case, ff_energy=args.ff_energy, pipeline_slots=4)
    # four steps in flight, each slot with its own grid, outputs and stream: the next steps' force
    # fields and scans fill the issue slots a latency-bound scan leaves idle (measured on flake60
    # with the forces-only grid: 0.821 / 0.730 / 0.729 / 0.728 / 0.727 ms per step with
    # 3 / 4 / 5 / 6 / 8 slots, against about 1.3 ms one step at a time); slot 0 alone gives the
    # isolated per-kernel timings
    pipe = afm.Pipeline(case, slots=4, layout=args.layout, tuning=tuning, ff_energy=args.ff_energy)
    sim = pipe.sims[0]
    atoms = afm.atoms_to_device(case["atoms"])
    # iteration counts of a neighbouring input, for the scan's pixel-to-warp plan timed below (the
    # headline steps run without a plan: with several steps in flight the issue slots, not the
    # slowest tile, bound the step, and a plan's narrow warps cost more slots than they save)
    plan_src = neighbour_case(case)
    nsim = afm.Simulator(plan_src, layout=args.layout, tuning=tuning, ff_energy=args.ff_energy, plan_frac=0.0)
    nsim.run(afm.atoms_to_device(plan_src["atoms"]))
    neighbour_iters = nsim.iters
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MiB
    s = case["scan"]
    units = s["nx"] * s["ny"] * s["nz"]
    pairs = case["grid"]["nx"] * case["grid"]["ny"] * case["grid"]["nz"] * len(case["atoms"]["x"])

    for _ in range(max(args.warmup, 3)):
        pipe.run_many([atoms] * pipe.slots)
    torch.cuda.synchronize()

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    clocks.begin()
    # headline: K steps, each the whole path (FF grid -> relaxed scan -> df) for its input
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_wall0 = time.perf_counter()
    p0.record(stream)
    pipe.run_many([atoms] * args.steps)
    p1.record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    barrier()
    torch.cuda.synchronize()
    # per-kernel timings: the same K steps one at a time on slot 0, L2 flushed before each
    for k in range(args.steps):
        flush.zero_()
        e0, e1, e2 = evs[k]
        e0.record(stream)
        sim.make_ff(atoms)
        e1.record(stream)
        sim.relax()
        e2.record(stream)
    torch.cuda.synchronize()
    # single-image latency with the force field in two parts (Simulator.run_overlapped): the node
    # layers the scan reads first, then the scan while the other layers are assembled on a second
    # stream; a synchronisation after each step checks that the scan read only the first part (a
    # step where it did not also pays the scan again on the complete grid, as run_host does)
    sim.run_overlapped(atoms, stream)
    torch.cuda.synchronize()
    sim.overlap_held()  # the first call learns the layers the scan reads (untimed)
    ov_ms, ov_held = [], 0
    for k in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        first = sim.run_overlapped(atoms, stream)
        b.record(stream)
        torch.cuda.synchronize()
        t = a.elapsed_time(b)
        if sim.overlap_held():
            ov_held += 1
        else:
            a.record(stream)
            sim.relax(stream)
            b.record(stream)
            torch.cuda.synchronize()
            t += a.elapsed_time(b)
        ov_ms.append(t)
    ms_step_ov = ppd.max_over_ranks(statistics.mean(ov_ms))

    # K2 alone on the same grid under three schedules: 8x4 tiles only (the steps above), a plan
    # built from the neighbouring input's scan, and one from this very input's earlier scan
    def time_relax(reps=20):
        for _ in range(3):
            sim.relax(stream)
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sim.relax(stream)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    relax_sched = {"no_plan": time_relax()}
    sim.plan_frac, sim.plan_lanes, sim.auto_plan = PLAN_FRAC, PLAN_LANES, False
    sim.plan_from(neighbour_iters, stream)
    relax_sched["neighbour_plan"] = time_relax()
    sim.plan_from(sim.iters, stream)
    relax_sched["own_plan"] = time_relax()
    plan_cols = sim._plan_k
    sim.drop_plan()
    # a series of scans of one grid for five lateral tip stiffnesses (the force field is not rebuilt):
    # with auto_plan each scan runs on the plan of the previous stiffness's scan
    tip0 = sim.tip
    series = {}
    for planned in (False, True):
        sim.plan_frac, sim.auto_plan = (PLAN_FRAC if planned else 0.0), planned
        sim.drop_plan()
        ts = []
        for rep in range(2):
            for kxy in (0.20, 0.225, 0.25, 0.275, 0.30):
                sim.tip = pp.make_tip(dict(case["tip"], kx=kxy, ky=kxy))
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                sim.relax(stream)
                b.record(stream)
                torch.cuda.synchronize()
                if rep == 1:
                    ts.append(a.elapsed_time(b))
        series["planned" if planned else "no_plan"] = statistics.mean(ts)
    sim.tip = tip0
    sim.drop_plan()
    sim.plan_frac, sim.auto_plan = 0.0, True
    torch.cuda.synchronize()
    clocks.end()
    barrier()
    clk = clocks.stop()
    t_ff = [evs[k][0].elapsed_time(evs[k][1]) for k in range(args.steps)]
    t_rx = [evs[k][1].elapsed_time(evs[k][2]) for k in range(args.steps)]
    ms_step = ppd.max_over_ranks(p0.elapsed_time(p1) / args.steps)
    ms_step_seq = ppd.max_over_ranks(sum(a + b for a, b in zip(t_ff, t_rx)) / args.steps)
    iters = sim.iters.to(torch.int64)
    it_total = int(iters.sum().item())
    nonconv = float((sim.iters >= case["fire"]["max_iter"]).float().mean().item())
    # FIRE position updates per pixel-height, binned in powers of two up to max_iter
    edges = [0, 1, 2, 4, 8, 16, 32, 64, 128, case["fire"]["max_iter"], case["fire"]["max_iter"] + 1]
    it_hist = [int(((iters >= a) & (iters < b)).sum().item()) for a, b in zip(edges[:-1], edges[1:])]

    # end to end through the public API: pinned host atoms in, host df image out.  Per step with a
    # synchronisation after each (run_host), and as a stream of steps whose device-to-host copies
    # overlap the next step's compute (run_host_many: the serving path)
    for _ in range(2):
        sim.run_host(case["atoms"])
    e2e_t = []
    for _ in range(max(3, args.steps // 2)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.run_host(case["atoms"])
        e2e_t.append(time.perf_counter() - t0)
    e2e_sync_ms = ppd.max_over_ranks(1e3 * statistics.mean(e2e_t))
    n_stream = max(8, args.steps // 2)
    outs = pipe.host_outputs(n_stream)  # pinned result buffers, allocated before timing like run_host's
    pipe.run_host_many([case["atoms"]] * 4, outs)
    torch.cuda.synchronize()
    # three wall-clock runs of n_stream steps each, the median kept (one run is a single sample of
    # a host-timed region: a scheduling hiccup of the host shows in it)
    e2e_runs = []
    for _ in range(3):
        t0 = time.perf_counter()
        pipe.run_host_many([case["atoms"]] * n_stream, outs)
        e2e_runs.append(1e3 * (time.perf_counter() - t0) / n_stream)
    e2e_ms = ppd.max_over_ranks(statistics.median(e2e_runs))

    peaks, src = load_peaks()
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    sms = sm_count()
    l2 = measure_l2_peak()
    ff_ms, rx_ms = statistics.mean(t_ff), statistics.mean(t_rx)
    flops_pair = FLOPS_PER_PAIR if args.ff_energy else FLOPS_PER_PAIR_FORCES
    ff_tflops = pairs * flops_pair / (ff_ms * 1e-3) / 1e12
    alu_peak = fp32_peak_tflops(sm_max, sms)
    alu_src = f"{sms} SMs (read from the device) x 128 FP32 lanes x 2 x {sm_max:.0f} MHz ({src} max SM clock)"
    rx_gbs = it_total * BYTES_PER_FIRE_ITER / (rx_ms * 1e-3) / 1e9
    ff_zpt = int(tuning["ff_zpt"]) if tuning is not None else 8
    executed = executed_ff_flops(args.ff_energy, ff_zpt)
    kernels = {
        "ff_assemble": {"ms": ff_ms, "share": ff_ms / (ff_ms + rx_ms), "pair_evals_per_s": pairs / (ff_ms * 1e-3),
                        "flops_per_pair": flops_pair, "energy": bool(args.ff_energy),
                        "traffic": measured_traffic("ff_assemble", ff_zpt) if not args.ff_energy else None,
                        "achieved_tflops": ff_tflops, "peak_tflops": alu_peak, "frac": ff_tflops / alu_peak,
                        "executed_flops_per_pair": executed, "ff_zpt": ff_zpt,
                        "executed_frac": (pairs * executed / (ff_ms * 1e-3) / 1e12 / alu_peak) if executed else None,
                        "note": "frac counts the algorithmic flops per pair (the number the >= 50 % target is stated "
                                "in); executed_frac counts the FP32 operations the kernel executes, from ncu's "
                                "fadd/fmul/ffma counters (lateral terms are shared by a column's z-nodes, so fewer "
                                "are executed than the pair formula has)"},
        "relax_scan": {"ms": rx_ms, "share": rx_ms / (ff_ms + rx_ms), "pixel_z_per_s": units / (rx_ms * 1e-3),
                       "fire_iters_mean": it_total / units, "nonconverged_frac": nonconv,
                       "fire_iters_hist": {"bin_lower_edges": edges[:-1], "counts": it_hist},
                       "traffic": measured_traffic("relax_scan"), "gather_gbs": rx_gbs,
                       "l2_peak_gbs": l2["peak_gbs"], "frac_of_l2": rx_gbs / l2["peak_gbs"],
                       "hbm_peak_gbs": peaks["hbm_gbs"], "frac_of_hbm": rx_gbs / peaks["hbm_gbs"],
                       "issue_active": measured_issue("relax_scan"),
                       "schedules_ms": relax_sched,
                       "stiffness_series_ms": dict(series, note="mean scan time over kx = ky = 0.20 .. 0.30 N/m on "
                                                   "one grid (second pass); planned: each scan on the plan its "
                                                   "predecessor (another stiffness) built, plan time included"),
                       "plan": {"columns": plan_cols, "lanes": PLAN_LANES,
                                "neighbour": "the flake with its atoms moved by up to 0.05 A and its charges "
                                             "scaled by up to 1 +- 0.1 (seeded)",
                                "note": "ms and the roofline are the headline's schedule (no plan); a plan moves "
                                        "the costliest pixel columns of an earlier scan into 4-lane warps, which "
                                        "shortens a scan run alone but costs issue slots when steps overlap"}},
    }
    dom = "ff_assemble" if ff_ms >= rx_ms else "relax_scan"
    if dom == "ff_assemble":
        roof = {"kernel": "ff_assemble", "bound": "alu", "achieved": ff_tflops, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": ff_tflops / alu_peak, "traffic": measured_traffic("ff_assemble", ff_zpt), "peak_source": alu_src}
    else:
        roof = {"kernel": "relax_scan", "bound": "l2", "achieved": rx_gbs, "peak": l2["peak_gbs"], "unit": "GB/s",
                "frac": rx_gbs / l2["peak_gbs"], "traffic": measured_traffic("relax_scan"),
                "peak_source": "L2 bandwidth measured in this run (" + l2["how"] + "): the grid's z-slab the scan "
                               "visits is L2-resident and the 96 B of corner values per FIRE iteration are served "
                               "from registers, L1 and L2, not from HBM",
                "issue_active": measured_issue("relax_scan"),
                "note": "the scan is latency-bound (the FIRE update of a pixel is a dependent chain): issue_active "
                        "is the fraction of cycles the SM sub-partitions issued an instruction, from ncu"}

    line = {"metric": METRIC, "value": world * units / (ms_step * 1e-3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms_step,
            "ms_per_step_sequential": ms_step_seq,
            "ms_per_step_overlapped": ms_step_ov,
            "overlap": {"first_layers": list(first), "grid_layers": case["grid"]["nz"], "steps_held": ov_held,
                        "steps": args.steps,
                        "note": "one image at a time, L2 flushed: the FF of the node layers the scan reads (learnt "
                                "from the previous call, two layers of margin), then the scan beside the FF of the "
                                "other layers on a second stream (Simulator.run_overlapped); the scan reports the "
                                "layers it read and a step that left the first part is charged a second scan"},
            "pipeline": {"slots": pipe.slots,
                         "note": "the K timed steps run four at a time on four streams with their own grids and "
                                 "outputs (afm.Pipeline): later steps' FF and scans fill the issue slots left by "
                                 "a latency-bound scan; "
                                 "ms_per_step_sequential is the same step one at a time (K1 + K2 event times, L2 "
                                 "flushed), from which the per-kernel figures and the roofline are taken"},
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(case, args.ff_energy),
            "ff_pair_evals_per_s": world * pairs / (ff_ms * 1e-3),
            "roofline": roof, "kernels": kernels,
            "e2e": {"value": world * units / (e2e_ms * 1e-3), "unit": UNIT,
                    "h2d_bytes_per_step": sim.h2d_bytes(len(case["atoms"]["x"])), "d2h_bytes_per_step": sim.d2h_bytes(),
                    "ms_per_step_runs": e2e_runs,
                    "note": f"Pipeline.run_host_many over {n_stream} steps (median of 3 runs): every step's atoms copied in and df "
                            "image copied out on its slot's stream, four steps in flight; no L2 flush between these "
                            "steps (each rewrites the 210 MB grid, larger than L2)",
                    "per_step_synchronised": world * units / (e2e_sync_ms * 1e-3),
                    "per_step_synchronised_note": "Simulator.run_host, one image at a time, host-timed, on the "
                                                  "schedule its first calls picked (run_host_schedule)",
                    "run_host_schedule": sim._mode},
            "gpu_launches": (2 + (case["grid"]["nz"] % ff_zpt != 0)) * args.steps, "clocks": clk, "wall_s_timed": t_wall,
            "device": {"sm_count": sms, "l2": l2}}
    if tuning is not None:
        line["autotune"] = tuning
    g4 = synth.gradient_case()
    line["bwd_fwd"] = [] if args.no_bwdfwd else [
        measure_bwd_fwd(g4, max(3, args.steps // 2), args.warmup, flush,
                        "mol40 seed 4040: 40 atoms, grid %dx%dx%d, scan 128x128x20" % (
                            g4["grid"]["nx"], g4["grid"]["ny"], g4["grid"]["nz"]), args.ff_energy),
        measure_bwd_fwd(case, max(3, args.steps // 2), args.warmup, flush, "flake60 (this line's workload)",
                        args.ff_energy),
    ]
    if not args.no_fdbm:
        line["fdbm_sweep"] = measure_fdbm_sweep(5, flush)
    if not args.no_tricubic:
        line["tricubic"] = measure_tricubic(case, max(3, args.steps // 2), args.warmup, flush,
                                            tuple(float(v) for v in args.tricubic_spacings.split(",")))
    if not args.no_quad:
        line["quadrupole"] = measure_quadrupole(case, tuning, max(3, args.steps // 2), args.warmup, flush, alu_peak)
    if not args.no_split:
        line["split"] = measure_split(case, max(3, args.steps // 2), args.warmup, flush, peaks["hbm_gbs"])
    if not args.no_iets:
        line["iets"] = measure_iets(case, max(3, args.steps // 2), args.warmup, flush, peaks["hbm_gbs"])
    line["df_standalone"] = measure_df(case, 20, flush, peaks["hbm_gbs"])
    line["benzene"] = measure_small(synth.benzene_case(), max(3, args.steps // 2), args.warmup, flush, alu_peak,
                                    args.ff_energy, cpu=(rank == 0 and world == 1 and not args.no_cpu_baseline))
    if not args.no_slab:
        line["slab"] = measure_slab(3, 1, flush, args.ff_energy)
    if not args.no_batch:
        line["batched"] = measure_batch(args.batch_mol, max(3, args.steps // 4), args.warmup, flush,
                                        ff_energy=args.ff_energy, autotune=not args.no_batch_tune)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(case)
        line["cpu_baseline"]["other_configs"] = cpu_baseline_other()
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
