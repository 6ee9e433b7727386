"""Many molecules in one persistent launch (pp_batch_run), optionally replayed from a CUDA graph.

`Batch` packs a list of workload dicts (same probe, tip, FIRE, df settings,
scan height step and periodic flag; any grid and scan sizes) into device
buffers: concatenated atoms, one descriptor per molecule with offsets into a
packed force-field buffer and packed fz / iters / df outputs.  `run()` issues
the C-ABI call on the current stream; `capture()` records it once in a CUDA
graph and `replay()` relaunches it.  Marshalling only: all work is in libpp.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import pp

ATOM_KEYS = ("x", "y", "z", "R", "eps", "q")


class Batch:
    def __init__(self, cases, device="cuda", want_pos=False, want_iters=True, ctas=0, fire=None,
                 spin_limit=0, wait_extra=0, ff_energy=True, ff_zpt=0, ff_tile_w=0, relax_tile_w=0):
        """ff_energy=False skips the energy sums of every molecule's grid (E slots 0; the scan
        outputs are unchanged).  ff_zpt, ff_tile_w, relax_tile_w and ctas set the work-item
        shapes and the persistent CTA count (0: defaults; tune.tune_batch picks them)."""
        if not cases:
            raise ValueError("empty batch")
        c0 = cases[0]
        dz = c0["scan"]["dz"]
        per = int(c0["grid"]["periodic_xy"])
        for c in cases:
            if (c["probe"] != c0["probe"] or c["tip"] != c0["tip"] or c["df"] != c0["df"]
                    or c["scan"]["dz"] != dz or int(c["grid"]["periodic_xy"]) != per
                    or (fire is None and c["fire"] != c0["fire"])):
                raise ValueError("all molecules of a batch share probe, tip, FIRE, df, scan dz and periodic_xy")
        self.device = torch.device(device)
        self.cases = cases
        self.nmol = len(cases)
        dfp = pp.make_df(c0["df"])
        self.m = pp.pp_df_margin(dfp.A_pp, dz)
        descs = (pp.MolDesc * self.nmol)()
        ff_off = out_off = df_off = atom_off = 0
        self.slices = []
        for n, c in enumerate(cases):
            g, s = c["grid"], c["scan"]
            na = len(c["atoms"]["x"])
            d = descs[n]
            d.ff_offset, d.out_offset, d.df_offset = ff_off, out_off, df_off
            d.atom_offset, d.n_atoms = atom_off, na
            d.nx, d.ny, d.nz = g["nx"], g["ny"], g["nz"]
            d.x0, d.y0, d.z0, d.dx, d.dy, d.dz = g["x0"], g["y0"], g["z0"], g["dx"], g["dy"], g["dz"]
            d.snx, d.sny, d.snz = s["nx"], s["ny"], s["nz"]
            d.sx0, d.sy0, d.spx, d.spy, d.z_top = s["x0"], s["y0"], s["px"], s["py"], s["z_top"]
            npts = s["nx"] * s["ny"] * s["nz"]
            ndf = s["nx"] * s["ny"] * (s["nz"] - 2 * self.m)
            self.slices.append({"ff": (ff_off, g["nx"] * g["ny"] * g["nz"]), "out": (out_off, npts),
                                "df": (df_off, ndf), "shape": (s["nz"], s["ny"], s["nx"]),
                                "grid_shape": (g["nz"], g["ny"], g["nx"])})
            ff_off += g["nx"] * g["ny"] * g["nz"]
            out_off += npts
            df_off += ndf
            atom_off += na
        raw = np.frombuffer(bytes(descs), dtype=np.uint8).copy()
        self.descs = torch.as_tensor(raw, device=self.device)
        packed = {k: np.concatenate([np.asarray(c["atoms"][k], dtype=np.float32) for c in cases]) for k in ATOM_KEYS}
        self.atoms_t = {k: torch.as_tensor(v, device=self.device) for k, v in packed.items()}
        self.atoms = pp.make_atoms(self.atoms_t)
        self.n_atoms = atom_off
        self.ff = torch.empty(4 * ff_off, dtype=torch.float32, device=self.device)
        self.fz = torch.empty(out_off, dtype=torch.float32, device=self.device)
        self.iters = torch.empty(out_off, dtype=torch.int32, device=self.device) if want_iters else None
        self.pos = torch.empty(3 * out_off, dtype=torch.float32, device=self.device) if want_pos else None
        self.df = torch.empty(df_off, dtype=torch.float32, device=self.device)
        self.ws = torch.empty(pp.pp_batch_workspace(self.nmol) // 4 + 4, dtype=torch.float32, device=self.device)
        bp = pp.BatchParams()
        bp.probe = pp.make_probe(c0["probe"])
        bp.tip = pp.make_tip(c0["tip"])
        bp.fire = pp.make_fire(fire or c0["fire"])
        bp.df = dfp
        bp.scan_dz = dz
        bp.periodic_xy = per
        bp.ff_capacity, bp.out_capacity, bp.df_capacity = ff_off, out_off, df_off
        bp.n_atoms_total = atom_off
        bp.ctas = ctas
        bp.spin_limit = spin_limit
        bp.wait_extra = wait_extra
        bp.ff_forces_only = 0 if ff_energy else 1
        bp.ff_zpt, bp.ff_tile_w, bp.relax_tile_w = ff_zpt, ff_tile_w, relax_tile_w
        self.params = bp
        self.graph = None
        self.pixel_heights = out_off
        self.pairs = sum(c["grid"]["nx"] * c["grid"]["ny"] * c["grid"]["nz"] * len(c["atoms"]["x"]) for c in cases)

    def run(self, stream=None):
        pp.pp_batch_run(self.descs, self.nmol, self.params, self.atoms, self.ff, self.pos, self.fz, self.iters,
                        self.df, self.ws, stream)

    def status(self):
        return pp.pp_batch_status(self.ws)

    def capture(self):
        """Record one run in a CUDA graph (warm the library on this device first)."""
        self.run()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run()
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def host_buffers(self):
        """Pinned host staging of run_host: packed atoms [6][n_atoms_total] (rows x, y, z, R, eps, q, the
        molecules in batch order) and the packed df images (the layout of self.df)."""
        if not hasattr(self, "_host"):
            pin = torch.cuda.is_available()
            self._host = {"atoms": torch.empty((6, self.n_atoms), dtype=torch.float32, pin_memory=pin),
                          "df": torch.empty(tuple(self.df.shape), dtype=torch.float32, pin_memory=pin)}
        return self._host

    def pack_atoms(self, cases):
        """Host atoms of len(cases) == nmol molecules (same atom counts as the batch's) packed into the
        pinned staging buffer of run_host."""
        h = self.host_buffers()["atoms"]
        for r, k in enumerate(ATOM_KEYS):
            h[r].copy_(torch.from_numpy(np.concatenate([np.asarray(c["atoms"][k], dtype=np.float32) for c in cases])))
        return h

    def run_host(self, atoms_host=None, stream=None):
        """End to end from host memory: the packed host atoms (default: the staging buffer as last packed)
        go to the device, the batch runs (its CUDA graph when captured), the packed df images come back to
        pinned host memory; returns that host tensor after synchronising.  The molecules' grids and scans
        stay those the batch was built with.  Bytes moved: 24 per atom in, 4 per df value out."""
        hb = self.host_buffers()
        src = hb["atoms"] if atoms_host is None else atoms_host
        st = stream or torch.cuda.current_stream()
        with torch.cuda.stream(st):
            for r, k in enumerate(ATOM_KEYS):
                self.atoms_t[k].copy_(src[r], non_blocking=True)
            if self.graph is not None:
                self.replay()
            else:
                self.run(st)
            hb["df"].copy_(self.df, non_blocking=True)
        st.synchronize()
        return hb["df"]

    def h2d_bytes(self):
        return 24 * self.n_atoms

    def d2h_bytes(self):
        return 4 * self.df.numel()

    def molecule(self, n):
        """Views of molecule n's outputs: fz, df, iters (and pos) in scan layout, ff as [nz][ny][nx][4]."""
        sl = self.slices[n]
        o, cnt = sl["out"]
        d0, dn = sl["df"]
        f0, fn = sl["ff"]
        nz, ny, nx = sl["shape"]
        out = {"fz": self.fz[o:o + cnt].view(nz, ny, nx),
               "df": self.df[d0:d0 + dn].view(nz - 2 * self.m, ny, nx),
               "ff": self.ff[4 * f0:4 * (f0 + fn)].view(*sl["grid_shape"], 4)}
        if self.iters is not None:
            out["iters"] = self.iters[o:o + cnt].view(nz, ny, nx)
        if self.pos is not None:
            out["pos"] = self.pos[3 * o:3 * (o + cnt)].view(nz, ny, nx, 3)
        return out
