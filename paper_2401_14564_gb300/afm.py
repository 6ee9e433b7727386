"""User-level API: one molecule, force field -> relaxed scan -> df image.

`Simulator` owns the device buffers of one workload shape (grid and scan) and
runs the three C-ABI stages on the current torch stream; `run_host` is the
end-to-end call that starts from host atom arrays and returns the df image
in host memory.  `Pipeline` keeps several independent items in flight on
their own streams and buffers.  Nothing here computes: it allocates with torch and calls
libpp through `pp.py`.
"""
from __future__ import annotations

import numpy as np
import torch

from . import pp

ATOM_KEYS = ("x", "y", "z", "R", "eps", "q")


def atoms_to_device(atoms, device="cuda"):
    """Host atom dict (numpy) -> dict of float32 CUDA tensors."""
    return {k: torch.as_tensor(np.asarray(atoms[k], dtype=np.float32), device=device) for k in ATOM_KEYS}


class Simulator:
    """Preallocated FF grid, positions, Fz, iteration counts and df for one case shape."""

    def __init__(self, case, layout=0, brick=(4, 4, 4), fire=None, device="cuda", fused_df=True,
                 want_pos=True, want_iters=True, tuning=None, ff_energy=True, overlap_ff=True, plan_frac=None,
                 plan_lanes=4, auto_plan=True, plan_min_tiles=None):
        """tuning: an autotuner result ({"ff_zpt", "layout", "brick"}) overriding layout and brick.
        ff_energy=False: the grid's E slots are written as 0 and the energy sums skipped (the scan
        reads only the forces, which are unchanged); trilinear force grids only.
        overlap_ff: run_host may assemble the node layers the scan will read first and the others on
        a second stream while the scan runs (see run_overlapped): its first calls time that and the
        one-stage forward in turn and keep the faster; False: one stage after the other.
        plan_frac, plan_lanes: the pixel-to-warp plan of the scan (plan_from): that fraction of the
        pixel columns, the costliest in an earlier scan, runs plan_lanes to a warp; 0 = never; None =
        0.025 on a force grid and 0 on a tricubic energy grid, whose scan is bound by issue slots rather
        than by its slowest tile (flake60 at 0.2 A: 1.42 ms on its own plan against 1.31 without).
        auto_plan: every scan builds the plan for the next from its own iteration counts.
        plan_min_tiles: scans of fewer 8x4 pixel tiles get no plan (None: the GPU's SM count)."""
        self.case = case
        self.device = torch.device(device)
        if tuning is not None:
            layout = tuning["layout"]
            brick = tuple(tuning["brick"]) if tuning.get("brick") else brick
        if not ff_energy and case["grid"].get("interp", 0):
            raise ValueError("ff_energy=False needs a force grid (interp 0)")
        self.ff_energy = ff_energy
        self.zpt = None
        if tuning is not None or not ff_energy:
            self.zpt = pp.Tuning(int(tuning["ff_zpt"]) if tuning is not None else 0, 0 if ff_energy else 1)
        self.grid = pp.make_grid(case["grid"], layout=layout, brick=brick)
        self.probe = pp.make_probe(case["probe"])
        self.scan = pp.make_scan(case["scan"])
        self.tip = pp.make_tip(case["tip"])
        self.fire = pp.make_fire(fire or case["fire"])
        self.dfp = pp.make_df(case["df"])
        self.fused_df = fused_df
        s = case["scan"]
        self.m = pp.pp_df_margin(self.dfp.A_pp, self.scan.dz)
        if self.m < 0 or s["nz"] < 2 * self.m + 1:
            raise ValueError("scan has fewer heights than the df stencil needs")
        nz, ny, nx = s["nz"], s["ny"], s["nx"]
        # zeroed once: a bricked layout's padding nodes, which only the whole-grid call writes
        self.ff = torch.zeros(pp.pp_ff_floats(self.grid), dtype=torch.float32, device=self.device)
        self.pos = torch.empty((nz, ny, nx, 3), dtype=torch.float32, device=self.device) if want_pos else None
        self.fz = torch.empty((nz, ny, nx), dtype=torch.float32, device=self.device)
        self.iters = torch.empty((nz, ny, nx), dtype=torch.int32, device=self.device) if want_iters else None
        self.df = torch.empty((nz - 2 * self.m, ny, nx), dtype=torch.float32, device=self.device)
        self._host = None
        self.overlap_ff = overlap_ff
        self._mode = None      # run_host's schedule once its trial calls have picked one
        self._trial = {"overlap": [], "plain": []}
        self._trial_warm = False
        self.reruns = 0      # scans run again because they read a layer outside the first part
        self._span = None    # node layers the last overlapped scan read
        self._side = None    # second stream of the overlapped forward
        self._zspan_d = None
        self._zspan_h = None
        if plan_frac is None:
            plan_frac = 0.0 if case["grid"].get("interp", 0) else 0.025
        self.plan_frac = float(plan_frac)
        self.plan_lanes = int(plan_lanes)
        self.auto_plan = bool(auto_plan)
        self.plan_min_tiles = plan_min_tiles
        self._plan = None
        self._plan_k = 0       # k and lanes the held plan was built with
        self._plan_lanes = 0
        self._plan_ready = False

    def make_ff(self, atoms_dev, stream=None):
        if self.zpt is not None:
            pp.pp_make_ff_tuned(pp.make_atoms(atoms_dev), self.probe, self.grid, self.ff, self.zpt, stream)
        else:
            pp.pp_make_ff(pp.make_atoms(atoms_dev), self.probe, self.grid, self.ff, stream)

    def relax(self, stream=None, df=None, zspan=None):
        """Relaxed scan and df image (into `df`, default self.df), with the pixel-to-warp plan when one
        is held (see plan_from); with auto_plan, the plan for the next call is then built from this
        scan's iteration counts."""
        out = self.df if df is None else df
        plan = (self._plan, self._plan_k, self._plan_lanes) if self._plan_ready else None
        pp.pp_relax_scan(self.ff, self.grid, self.scan, self.tip, self.fire, self.pos, self.fz, self.iters,
                         self.dfp if self.fused_df else None, out if self.fused_df else None, stream,
                         zspan=zspan, plan=plan)
        if not self.fused_df:
            pp.pp_fz_to_df(self.fz, self.scan.nz, self.scan.nx * self.scan.ny, self.scan.dz, self.dfp, out, stream)
        if self.auto_plan and self.iters is not None:
            self.plan_from(self.iters, stream)

    # ---- pixel-to-warp plan of the scan
    def plan_from(self, iters, stream=None):
        """Builds the plan the next scans use from iteration counts of an earlier scan of this shape
        (this simulator's own, or another image's, e.g. a neighbouring geometry): the plan_frac
        costliest pixel columns run plan_lanes to a warp.  Outputs never depend on it."""
        if self.plan_frac <= 0:
            return
        tiles = ((self.scan.nx + 7) // 8) * ((self.scan.ny + 3) // 4)
        least = self.plan_min_tiles
        if least is None:
            least = torch.cuda.get_device_properties(self.device).multi_processor_count
        if tiles < least:
            # fewer 8x4 tiles than SMs: no tile shares an SM, and building the plan costs more than it
            # saves (benzene, 50 tiles: 0.163 against 0.149 ms per forward pass)
            return
        npix = self.scan.nx * self.scan.ny
        k = max(1, min(npix, int(round(self.plan_frac * npix))))
        if self._plan is None or (k, self.plan_lanes) != (self._plan_k, self._plan_lanes):
            # the plan's layout depends on k and the lanes: a new shape gets a new buffer
            n = pp.pp_relax_plan_size(self.scan, k, self.plan_lanes)
            self._plan = torch.empty((n + 3) // 4, dtype=torch.int32, device=self.device)
            self._plan_k, self._plan_lanes = k, self.plan_lanes
        pp.pp_relax_plan(iters, self.scan, self.fire.max_iter, self._plan_k, self._plan_lanes, self._plan, stream)
        self._plan_ready = True

    def drop_plan(self):
        """Scans go back to 8x4 pixel tiles alone (until the next plan_from)."""
        self._plan_ready = False

    def run(self, atoms_dev, stream=None, df=None):
        """Device-resident forward pass; returns the df tensor (device)."""
        self.make_ff(atoms_dev, stream)
        self.relax(stream, df)
        return self.df if df is None else df

    # ---- force field of the scan's layers first, the rest beside the scan
    def first_layers(self):
        """Node layers [k0, k1) assembled before the scan: those the last overlapped scan read, with
        two layers of margin on either side; before any, the layers within R0 + 1 A of the anchor
        heights (a PP hangs R0 from its anchor; the springs hold it near that sphere)."""
        g, s = self.case["grid"], self.case["scan"]
        nz = int(g["nz"])
        if self._span is not None:
            lo, hi = self._span[0] - 2, self._span[1] + 3
        else:
            reach = float(self.case["tip"]["R0"]) + 1.0
            zbot = s["z_top"] - (s["nz"] - 1) * s["dz"]
            lo = int(np.floor((zbot - reach - g["z0"]) / g["dz"]))
            hi = int(np.floor((s["z_top"] + reach - g["z0"]) / g["dz"])) + 2
        k0, k1 = min(max(lo, 0), nz - 1), min(max(hi, 1), nz)
        return (k0, k1) if k1 > k0 else (0, nz)

    def _ff_layers(self, atoms, k0, k1, stream):
        pp.pp_make_ff_layers(atoms, self.probe, self.grid, self.ff, k0, k1, self.zpt, stream)

    def run_overlapped(self, atoms_dev, stream=None):
        """Forward pass with the force field in two parts: layers [k0, k1) = first_layers() on
        `stream`, then the scan on `stream` (reporting the layers it read) while the other layers
        are assembled on a second stream; `stream` waits for both.  Returns (k0, k1).  The result
        stands only if the scan read nothing outside [k0, k1): check it with overlap_held() after
        synchronising (run_host does, and runs the scan again on the complete grid if not)."""
        st = stream or torch.cuda.current_stream()
        nz = int(self.case["grid"]["nz"])
        if self._side is None:
            self._side = torch.cuda.Stream(device=self.device)
            self._zspan_d = torch.empty(2, dtype=torch.int32, device=self.device)
            self._zspan_h = torch.empty(2, dtype=torch.int32, pin_memory=torch.cuda.is_available())
        k0, k1 = self.first_layers()
        atoms = pp.make_atoms(atoms_dev)
        self._ff_layers(atoms, k0, k1, st)
        first = torch.cuda.Event()
        first.record(st)
        self._side.wait_event(first)
        if k1 < nz:
            self._ff_layers(atoms, k1, nz, self._side)
        if k0 > 0:
            self._ff_layers(atoms, 0, k0, self._side)
        self.relax(st, zspan=self._zspan_d)
        with torch.cuda.stream(st):
            self._zspan_h.copy_(self._zspan_d, non_blocking=True)
        rest = torch.cuda.Event()
        rest.record(self._side)
        st.wait_event(rest)
        self._first = (k0, k1)
        return k0, k1

    def overlap_held(self):
        """After run_overlapped and a synchronise: True when the scan read only layers of the first
        part (its result is then that of run()); remembers the layers read for first_layers()."""
        lo, hi = int(self._zspan_h[0]), int(self._zspan_h[1])
        if lo > hi:  # nothing read (no pixel)
            return True
        self._span = (lo, hi)
        return self._first[0] <= lo and hi < self._first[1]

    # ---- end to end from host memory
    def _host_buffers(self, n_atoms):
        if self._host is None or self._host["n"] != n_atoms:
            pin = torch.cuda.is_available()
            self._host = {
                "n": n_atoms,
                "atoms_h": torch.empty((6, n_atoms), dtype=torch.float32, pin_memory=pin),
                "atoms_d": torch.empty((6, n_atoms), dtype=torch.float32, device=self.device),
                "df_h": torch.empty(tuple(self.df.shape), dtype=torch.float32, pin_memory=pin),
            }
        return self._host

    def run_host(self, atoms_host, out=None, stream=None):
        """Host atoms (numpy dict) -> host df image: H2D copy, FF, relax, df, D2H copy.

        Returns the host (pinned) df tensor after synchronising the stream.
        Bytes moved: 24 per atom host->device, 4 per df value device->host.
        """
        n = int(len(atoms_host["x"]))
        hb = self._host_buffers(n)
        for r, k in enumerate(ATOM_KEYS):
            hb["atoms_h"][r].copy_(torch.from_numpy(np.asarray(atoms_host[k], dtype=np.float32)))
        st = stream or torch.cuda.current_stream()
        overlap = self._forward_mode() == "overlap"
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(st):
            hb["atoms_d"].copy_(hb["atoms_h"], non_blocking=True)
            dev = {k: hb["atoms_d"][r] for r, k in enumerate(ATOM_KEYS)}
            e0.record(st)
            if overlap:
                self.run_overlapped(dev, st)
            else:
                self.run(dev, st)
            e1.record(st)
            hb["df_h"].copy_(self.df, non_blocking=True)
        st.synchronize()
        ms = e0.elapsed_time(e1)
        if overlap and not self.overlap_held():
            # the scan left the first part: run it again on the grid, complete by now
            self.reruns += 1
            with torch.cuda.stream(st):
                e0.record(st)
                self.relax(st)
                e1.record(st)
                hb["df_h"].copy_(self.df, non_blocking=True)
            st.synchronize()
            ms += e0.elapsed_time(e1)
        self._note_forward(overlap, ms)
        if out is not None:
            out.copy_(hb["df_h"])
            return out
        return hb["df_h"]

    # run_host's schedule: with overlap_ff, its first calls time the overlapped and the one-stage
    # forward in turn and keep the faster (the overlap pays on flake60, 0.99 against 1.16 ms, and
    # loses where the force field dominates the pass: the 2516-atom slab, 107.5 against 103.9 ms,
    # whose K1 gets too few CTAs per SM beside the scan's resident warps)
    _TRIALS = 3  # timed calls of each schedule

    def _forward_mode(self):
        if not self.overlap_ff:
            return "plain"
        if self._mode is not None:
            return self._mode
        n_ov, n_pl = len(self._trial["overlap"]), len(self._trial["plain"])
        # the first overlapped call (on the anchors' reach, not yet the band a scan read) is not counted
        if not self._trial_warm:
            return "overlap"
        return "overlap" if n_ov <= n_pl else "plain"

    def _note_forward(self, overlap, ms):
        if not self.overlap_ff or self._mode is not None:
            return
        if overlap and not self._trial_warm:
            self._trial_warm = True
            return
        self._trial["overlap" if overlap else "plain"].append(ms)
        if min(len(v) for v in self._trial.values()) >= self._TRIALS:
            med = {k: sorted(v)[len(v) // 2] for k, v in self._trial.items()}
            self._mode = "overlap" if med["overlap"] < med["plain"] else "plain"

    def host_outputs(self, n_items):
        """n_items pinned host tensors shaped like the df image, for run_host_many(outs=...)."""
        pin = torch.cuda.is_available()
        return [torch.empty(tuple(self.df.shape), dtype=torch.float32, pin_memory=pin) for _ in range(n_items)]

    def run_host_many(self, atoms_list, outs=None):
        """Host df images for a sequence of host atom sets, end to end: every item's atoms go host ->
        device and its df image device -> host, as in run_host.  The device-to-host copy of item k
        runs on a second stream while item k+1 computes (two device df buffers), so the copies
        overlap the neighbouring compute; the compute itself stays in order on the current stream.
        outs: pinned host tensors to write (see host_outputs), else allocated here."""
        n_items = len(atoms_list)
        if n_items == 0:
            return []
        n = int(len(atoms_list[0]["x"]))
        if any(int(len(a["x"])) != n for a in atoms_list):
            raise ValueError("run_host_many: every item needs the same number of atoms")
        cs = torch.cuda.current_stream()
        if getattr(self, "_copy_stream", None) is None:
            self._copy_stream = torch.cuda.Stream()
        xs = self._copy_stream
        pin = torch.cuda.is_available()
        if getattr(self, "_pipe", None) is None or self._pipe["n"] != n:
            self._pipe = {
                "n": n,
                "atoms_h": [torch.empty((6, n), dtype=torch.float32, pin_memory=pin) for _ in range(2)],
                "atoms_d": [torch.empty((6, n), dtype=torch.float32, device=self.device) for _ in range(2)],
                "df_d": [self.df, torch.empty_like(self.df)],
            }
        P = self._pipe
        if outs is None:
            outs = self.host_outputs(n_items)
        elif len(outs) < n_items:
            raise ValueError("run_host_many: fewer output buffers than items")
        h2d_done = [None, None]
        copy_done = [None, None]
        for k, atoms_host in enumerate(atoms_list):
            b = k & 1
            if h2d_done[b] is not None:
                h2d_done[b].synchronize()  # the staging buffer of item k-2 has been read
            for r, key in enumerate(ATOM_KEYS):
                P["atoms_h"][b][r].copy_(torch.from_numpy(np.asarray(atoms_host[key], dtype=np.float32)))
            with torch.cuda.stream(cs):
                P["atoms_d"][b].copy_(P["atoms_h"][b], non_blocking=True)
                h2d_done[b] = torch.cuda.Event()
                h2d_done[b].record(cs)
                if copy_done[b] is not None:
                    cs.wait_event(copy_done[b])  # item k-2's image has left this df buffer
                dev = {key: P["atoms_d"][b][r] for r, key in enumerate(ATOM_KEYS)}
                self.run(dev, cs, df=P["df_d"][b])
                computed = torch.cuda.Event()
                computed.record(cs)
            xs.wait_event(computed)
            with torch.cuda.stream(xs):
                outs[k].copy_(P["df_d"][b], non_blocking=True)
                copy_done[b] = torch.cuda.Event()
                copy_done[b].record(xs)
        xs.synchronize()
        cs.synchronize()
        return outs

    def h2d_bytes(self, n_atoms):
        return 6 * 4 * n_atoms

    def d2h_bytes(self):
        return self.df.numel() * 4

    def save(self, path, grid=True):
        """Write the last run's outputs (df, Fz, and the positions and iteration counts when kept;
        the force-field grid too unless grid=False) to a NumPy .npz file, with the case's grid and
        scan geometry.  The paper's CPU code keeps its grids on disk; here they are recomputed
        faster than read back, so this is for inspection, not for resuming."""
        torch.cuda.synchronize()
        out = {"df": self.df.cpu().numpy(), "fz": self.fz.cpu().numpy()}
        if self.pos is not None:
            out["pos"] = self.pos.cpu().numpy()
        if self.iters is not None:
            out["iters"] = self.iters.cpu().numpy()
        if grid:
            out["ff"] = self.ff.cpu().numpy()
        g, s = self.case["grid"], self.case["scan"]
        out["grid_geometry"] = np.array([g["nx"], g["ny"], g["nz"], g["x0"], g["y0"], g["z0"], g["dx"], g["dy"],
                                         g["dz"], g.get("interp", 0), self.grid.layout], dtype=np.float64)
        out["scan_geometry"] = np.array([s["nx"], s["ny"], s["nz"], s["x0"], s["y0"], s["px"], s["py"], s["z_top"],
                                         s["dz"]], dtype=np.float64)
        np.savez(path, **out)


class Pipeline:
    """Independent forward passes in flight `slots` at a time.

    Item k runs on slot k % slots, which owns a Simulator (grid, positions, Fz, df) and a stream,
    so the force fields and scans of later items overlap the relaxed scan of item k.  The scan is
    bound by the latency of its FIRE chains: one item's pixel columns give few warps per SM, and in
    its tail the slowest columns run alone; the other items' tiles fill those idle issue slots.
    Every item computes exactly what Simulator.run computes (same kernels, same inputs,
    bit-identical images).  Device memory: one Simulator's buffers per slot.
    """

    def __init__(self, case, slots=4, **sim_kwargs):
        if slots < 1:
            raise ValueError("Pipeline needs at least one slot")
        # no scan plan unless asked: with items in flight the issue slots bound a step, and a plan's
        # narrow warps cost more of them than the shorter slowest tile saves (flake60, 4 slots:
        # 0.739 ms per step without, 0.757-0.809 ms with plans of 1-5 % of the columns, 4-16 lanes)
        sim_kwargs.setdefault("plan_frac", 0.0)
        self.sims = [Simulator(case, **sim_kwargs) for _ in range(slots)]
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        self._host = None

    @property
    def slots(self):
        return len(self.sims)

    def _fork(self):
        cur = torch.cuda.current_stream()
        ev = torch.cuda.Event()
        ev.record(cur)
        for st in self.streams:
            st.wait_event(ev)
        return cur

    def _join(self, cur):
        for st in self.streams:
            ev = torch.cuda.Event()
            ev.record(st)
            cur.wait_event(ev)

    def run_many(self, atoms_devs, outs=None):
        """Device atoms of each item -> df images.  outs[k] (device tensors shaped like the df image)
        receive item k's image; with outs=None each image stays in its slot's df buffer until the
        slot's next item overwrites it.  Ordered after the current stream's work; the current
        stream waits for every item before its next launch."""
        if outs is not None and len(outs) < len(atoms_devs):
            raise ValueError("run_many: fewer output buffers than items")
        cur = self._fork()
        for k, dev in enumerate(atoms_devs):
            b = k % self.slots
            self.sims[b].run(dev, self.streams[b], df=None if outs is None else outs[k])
        self._join(cur)
        return outs

    def host_outputs(self, n_items):
        return self.sims[0].host_outputs(n_items)

    def run_host_many(self, atoms_list, outs=None):
        """Host atom sets -> host df images (pinned outs, see host_outputs), end to end: item k's
        atoms go host -> device, its force field, scan and df run, and its image comes back, all on
        its slot's stream, so the copies and the compute of neighbouring items overlap."""
        n_items = len(atoms_list)
        if n_items == 0:
            return []
        n = int(len(atoms_list[0]["x"]))
        if any(int(len(a["x"])) != n for a in atoms_list):
            raise ValueError("run_host_many: every item needs the same number of atoms")
        if outs is None:
            outs = self.host_outputs(n_items)
        elif len(outs) < n_items:
            raise ValueError("run_host_many: fewer output buffers than items")
        pin = torch.cuda.is_available()
        if self._host is None or self._host["n"] != n:
            self._host = {
                "n": n,
                "atoms_h": [torch.empty((6, n), dtype=torch.float32, pin_memory=pin) for _ in self.sims],
                "atoms_d": [torch.empty((6, n), dtype=torch.float32, device=sim.device) for sim in self.sims],
            }
        H = self._host
        staged = [None] * self.slots
        cur = self._fork()
        for k, atoms_host in enumerate(atoms_list):
            b = k % self.slots
            if staged[b] is not None:
                staged[b].synchronize()  # the slot's previous item has left the pinned staging buffer
            for r, key in enumerate(ATOM_KEYS):
                H["atoms_h"][b][r].copy_(torch.from_numpy(np.asarray(atoms_host[key], dtype=np.float32)))
            st = self.streams[b]
            with torch.cuda.stream(st):
                H["atoms_d"][b].copy_(H["atoms_h"][b], non_blocking=True)
                staged[b] = torch.cuda.Event()
                staged[b].record(st)
                dev = {key: H["atoms_d"][b][r] for r, key in enumerate(ATOM_KEYS)}
                self.sims[b].run(dev, st)
                outs[k].copy_(self.sims[b].df, non_blocking=True)
        self._join(cur)
        cur.synchronize()
        return outs

    def h2d_bytes(self, n_atoms):
        return self.sims[0].h2d_bytes(n_atoms)

    def d2h_bytes(self):
        return self.sims[0].d2h_bytes()


def afm(case, atoms=None, layout=0, fire=None, device="cuda"):
    """One-shot simulation of a case dict; returns host numpy arrays (df, fz, pos, iters, ff)."""
    sim = Simulator(case, layout=layout, fire=fire, device=device)
    dev = atoms_to_device(atoms if atoms is not None else case["atoms"], device)
    sim.run(dev)
    torch.cuda.synchronize()
    return {"df": sim.df.cpu().numpy(), "fz": sim.fz.cpu().numpy(), "pos": sim.pos.cpu().numpy(),
            "iters": sim.iters.cpu().numpy(), "ff": sim.ff, "sim": sim}
