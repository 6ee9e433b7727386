"""Bounds checks (the stand-in for a memory checker, which this pool does not offer): every
workload family runs on libpp_checked.so, whose kernels test each global gather and scatter
index against the size of its array and record a bit when one falls outside; none may fire.

Covered: the flake60 step (K1, K2 with fused df, K9, K3/K4/K5 adjoint, and the host-array call
with K1 on node-layer ranges beside the layer-reporting K2) on the force grid and on a 0.2 A
tricubic energy grid; a bricked-layout case with the layout converter and the
standalone df kernel; the quadrupole with minimum image and a Coulomb cutoff; the split force
field and its recombination; FFT correlations with a ragged shape and a 1024-long axis; a
batched launch of ragged molecules, also with other work-item shapes; the scan with the Newton
polish on a force grid and on an energy grid.  The library is loaded in a child process (PP_LIBRARY).
"""
import os
import subprocess
import sys

import pytest

from paper_2401_14564_gb300 import build

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import copy, sys
import numpy as np, torch
sys.path.insert(0, ROOT)
sys.path.insert(0, ROOT + "/tests")
from paper_2401_14564_gb300 import afm, batch, pp, synth
from helpers import case32

def backward(c, sim, at):
    n = len(c["atoms"]["x"])
    g = {k: torch.empty(n, device="cuda") for k in ("x", "y", "z", "q", "R", "eps")}
    g["tip"] = torch.empty(5, device="cuda")
    ws = torch.empty(pp.pp_backward_workspace(sim.grid) // 4 + 1, device="cuda")
    w = torch.randn(tuple(sim.df.shape), device="cuda")
    pp.pp_backward(pp.make_atoms(at), sim.probe, sim.grid, sim.ff, sim.scan, sim.tip, sim.dfp, sim.pos, w,
                   pp.make_grads(g), ws)

def iets(sim):
    n = sim.fz.numel()
    pp.pp_iets(sim.ff, sim.grid, sim.scan, sim.tip, sim.pos, 16.0, torch.empty(3 * n, device="cuda"),
               torch.empty(3 * n, device="cuda"))

def step(c, **kw):
    sim = afm.Simulator(c, **kw)
    at = afm.atoms_to_device(c["atoms"])
    sim.run(at)
    iets(sim)
    backward(c, sim, at)
    sim.run_host(c["atoms"])  # the force field in parts beside the layer-reporting scan
    return sim

flake = synth.flake_case()
step(flake)
g0 = flake["grid"]
step(dict(flake, grid=dict(g0, nx=128, ny=128, nz=100, dx=0.2, dy=0.2, dz=0.2, interp=1)))
small = case32(synth.small_case(seed=7, n_atoms=11, nxy=36, nz=33, scan_px=11, nz_scan=13))
sim = step(small, layout=1, brick=(4, 4, 4), fused_df=False)
lin = pp.make_grid(small["grid"], 0)
out = torch.empty(pp.pp_ff_floats(lin), device="cuda")
pp.pp_ff_convert(sim.ff, sim.grid, out, lin)
q = copy.deepcopy(small)
q["probe"] = synth.default_probe(coul_rc=3.0, min_image=1, Qzz=-0.1)
step(q)
grid = pp.make_grid(small["grid"], 0)
ff, el = (torch.empty(pp.pp_ff_floats(grid), device="cuda") for _ in range(2))
pp.pp_make_ff_split(pp.make_atoms(afm.atoms_to_device(small["atoms"])), pp.make_probe(small["probe"]), grid, ff, el)
pp.pp_ff_combine(ff, el, -0.1, grid, ff)
for shape in ((32, 16, 8), (2, 4, 8), (1024, 4, 8)):
    g = {"nx": shape[0], "ny": shape[1], "nz": shape[2], "x0": 0.0, "y0": 0.0, "z0": 0.0, "dx": 0.1, "dy": 0.1,
         "dz": 0.1, "periodic_xy": 1}
    gr = pp.make_grid(g, 0)
    f = torch.rand(shape[2] * shape[1] * shape[0], device="cuda")
    t = torch.rand(shape[2] * shape[1] * shape[0], device="cuda")
    ws = torch.empty(pp.pp_fft_workspace(gr) // 4, device="cuda")
    o = torch.empty(pp.pp_ff_floats(gr), device="cuda")
    pp.pp_fft_correlate(f, t, gr, 1.0, 1.0, o, ws)
    pp.pp_fft_correlate(f, t, gr, 2.0, 1.2, o, ws, accumulate=True)
cs = [case32(c) for c in synth.batch_cases(6, 1000)]
r = copy.deepcopy(cs[0])
r["scan"] = dict(r["scan"], nx=13, ny=7)
cs.append(r)
b = batch.Batch(cs)
b.run()
for zpt, fw, rw in ((4, 16, 4), (8, 4, 16)):
    batch.Batch(cs, ff_zpt=zpt, ff_tile_w=fw, relax_tile_w=rw).run()
# the Newton polish after FIRE, on the force and on the energy grid
step(small, fire=synth.parity_fire(polish=4))
step(dict(small, grid=dict(small["grid"], interp=1)), fire=synth.parity_fire(polish=4))
torch.cuda.synchronize()
print("FLAGS", pp.pp_check_flags())
"""


def test_no_bounds_check_fires():
    lib = build.build(checked=True)
    env = dict(os.environ, PP_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + CHILD], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    flags = int(r.stdout.strip().splitlines()[-1].split()[1])
    assert flags == 0, f"bounds checks fired: bits {flags:#x}"
