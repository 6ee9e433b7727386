"""GPU parity of the tricubic path (grid interp = 1: energy-only K1 variant,
K2 with F = -grad of the tricubic energy interpolant) against the FP64 oracle,
whose tricubic interpolant is pinned in tests/test_oracle_tricubic.py.

Bars as for the trilinear path: node energies to 1e-4 relative (1e-2 eV
floor) outside the core, relaxed positions to 1e-3 A and df to 1e-3 of the
image range on well-conditioned points in the same basin.
"""
import copy

import numpy as np
import pytest
import torch

from helpers import case32
from paper_2401_14564_gb300 import afm, pp, synth
from test_gpu_relax import check_parity, gpu_run

pytestmark = pytest.mark.gpu


def tc(c, **grid):
    c = copy.deepcopy(c)
    c["grid"] = dict(c["grid"], interp=1, **grid)
    return c


def gpu_grid(c, interp):
    g = dict(c["grid"], interp=interp)
    grid = pp.make_grid(g, 0)
    ff = torch.full((pp.pp_ff_floats(grid),), float("nan"), dtype=torch.float32, device="cuda")
    pp.pp_make_ff(pp.make_atoms(afm.atoms_to_device(c["atoms"])), pp.make_probe(c["probe"]), grid, ff)
    torch.cuda.synchronize()
    return ff.cpu().numpy()


def check_energy(orc, c):
    c = case32(c)
    g = c["grid"]
    E = gpu_grid(c, 1).reshape(g["nz"], g["ny"], g["nx"]).astype(np.float64)
    assert E.size == g["nx"] * g["ny"] * g["nz"]
    ref, core = orc.make_ff(c["atoms"], c["probe"], g)
    err = (np.abs(E - ref[..., 3]) / np.maximum(np.abs(ref[..., 3]), 1e-2))[~core]
    assert np.isfinite(E).all()
    assert err.max() <= 1e-4, err.max()
    # the energy-only launch forms the same sums; without the force terms the compiler may
    # round a step differently, so it agrees with the full grid's E to FP32 rounding only: a node
    # energy is a sum of cancelling pair terms of ~1 eV, each rounded at ~1e-7 eV
    full = gpu_grid(c, 0).reshape(g["nz"], g["ny"], g["nx"], 4)[..., 3].astype(np.float64)
    assert (np.abs(E - full) / np.maximum(np.abs(full), 1e-2)).max() <= 2e-5


def test_energy_grid_matches_oracle(orc):
    check_energy(orc, synth.small_case(seed=3, n_atoms=12, nxy=32, nz=37))


def test_energy_grid_min_image_cutoff_quadrupole(orc):
    c = synth.small_case(seed=5, n_atoms=20, nxy=24, nz=17)
    c["probe"] = synth.default_probe(coul_rc=3.0, min_image=1, Qzz=-0.1)
    check_energy(orc, c)


def test_tricubic_relax_parity_benzene(orc):
    check_parity(orc, tc(synth.benzene_case()))


def test_tricubic_relax_parity_ragged_scan(orc):
    # 12 x 15 pixels, 12 heights, periodic stencil wrap near the cell edges
    check_parity(orc, tc(synth.small_case(seed=3, n_atoms=12, nxy=32, nz=40, scan_px=12, nz_scan=12)))


def test_tricubic_relax_parity_clamped_grid(orc):
    # no lateral periodicity: stencil nodes clamp into the grid on every axis (the geometry of
    # the trilinear clamped-grid parity case)
    check_parity(orc, tc(synth.small_case(seed=8, n_atoms=10, nxy=36, nz=40, scan_px=11, nz_scan=13),
                         periodic_xy=0))


def test_tricubic_fused_df_equals_standalone_kernel():
    c = case32(tc(synth.benzene_case()))
    a = gpu_run(c, fused=True)
    b = gpu_run(c, fused=False)
    assert np.array_equal(a["fz"], b["fz"]) and np.array_equal(a["df"], b["df"])
