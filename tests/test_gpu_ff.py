"""GPU parity of K1 (FF grid assembly) against the FP64 oracle.

Bar: per-node relative force error |F_gpu - F_ref| / max(|F_ref|, 1e-3 eV/A)
<= 1e-4 outside the clamped core region.  Energies (stored for the user, not
used by the relaxation) to 1e-4 relative with a 1e-2 eV floor: far from the
sample the node energy is a small sum of cancelling pair terms, and the FP32
rounding of those terms (rsqrt to ~2 ulp, raised to the 6th/12th power) sits
near 1e-7 eV.  Layout changes must not change a single bit.
"""
import numpy as np
import pytest
import torch

from helpers import case32, ff_rel_err, linear_ff
from paper_2401_14564_gb300 import afm, pp, synth

pytestmark = pytest.mark.gpu

TOL = 1e-4


def gpu_ff(case, layout=0, brick=(4, 4, 4)):
    grid = pp.make_grid(case["grid"], layout, brick)
    ff = torch.full((pp.pp_ff_floats(grid),), float("nan"), dtype=torch.float32, device="cuda")
    pp.pp_make_ff(pp.make_atoms(afm.atoms_to_device(case["atoms"])), pp.make_probe(case["probe"]), grid, ff)
    return ff, grid


def as_linear(ff, grid, g):
    if grid.layout == 0:
        return linear_ff(ff.cpu().numpy(), g)
    lin = pp.make_grid(g, 0)
    out = torch.empty(pp.pp_ff_floats(lin), dtype=torch.float32, device="cuda")
    pp.pp_ff_convert(ff, grid, out, lin)
    return linear_ff(out.cpu().numpy(), g)


def check_full(orc, case):
    c = case32(case)
    ff, grid = gpu_ff(c)
    F = as_linear(ff, grid, c["grid"])
    ref, core = orc.make_ff(c["atoms"], c["probe"], c["grid"])
    assert np.isfinite(F).all()
    err = ff_rel_err(F, ref)[~core]
    eerr = (np.abs(F[..., 3] - ref[..., 3]) / np.maximum(np.abs(ref[..., 3]), 1e-2))[~core]
    assert err.max() <= TOL, err.max()
    assert eerr.max() <= TOL, eerr.max()
    # the core region is finite and has the reference's sign structure
    if core.any():
        assert np.isfinite(F[core]).all()
    return err


def test_small_ragged_case(orc):
    # 32 x 36 x 40 nodes: ragged against the 16 x 8 x 8 CTA tile in y and z
    check_full(orc, synth.small_case(seed=3, n_atoms=12, nxy=32, nz=37))


def test_benzene_grid(orc):
    check_full(orc, synth.benzene_case())


def test_many_atoms_min_image_cutoff(orc):
    # the 2016-atom bilayer plus a molecule: several shared-memory chunks, minimum image, shifted-force cut
    slab = synth.graphene_bilayer()
    mol = synth.shift_atoms(synth.random_molecule(77, 30), 25.6, 25.6, 6.65)
    atoms = synth.concat_atoms(slab, mol)
    atoms["q"] = atoms["q"] + np.linspace(-0.05, 0.05, len(atoms["q"]))
    # the minimum image uses the grid extent as the period: nx*dx = ny*dy = 51.2 A
    c = {"atoms": atoms, "probe": synth.default_probe(coul_rc=8.0, min_image=1),
         "grid": {"nx": 20, "ny": 22, "nz": 9, "x0": 0.013, "y0": 0.021, "z0": 8.0, "dx": 51.2 / 20,
                  "dy": 51.2 / 22, "dz": 0.41, "periodic_xy": 1}}
    check_full(orc, c)


def test_plain_coulomb_cutoff_only(orc):
    c = synth.small_case(seed=5, n_atoms=20, nxy=24, nz=17)
    c["probe"] = synth.default_probe(coul_rc=3.0)
    check_full(orc, c)


@pytest.mark.parametrize("brick", [(4, 4, 4), (8, 8, 4), (2, 4, 8), (1, 1, 1), (16, 16, 16), (8, 2, 1)])
def test_bricked_layout_is_bit_identical(brick):
    c = case32(synth.small_case(seed=4, n_atoms=9, nxy=26, nz=11))
    ff0, g0 = gpu_ff(c, 0)
    ff1, g1 = gpu_ff(c, 1, brick)
    lin = as_linear(ff1, g1, c["grid"])
    assert np.array_equal(lin, linear_ff(ff0.cpu().numpy(), c["grid"]))
    # padding slots are written (zeros), never left uninitialised
    assert torch.isfinite(ff1).all()
    # and converting back reproduces the bricked buffer exactly
    back = torch.empty_like(ff1)
    pp.pp_ff_convert(ff0, g0, back, g1)
    assert torch.equal(back, ff1)


def test_no_atoms_gives_zero_field():
    c = case32(synth.small_case(seed=4, n_atoms=9, nxy=20, nz=9))
    for k in ("x", "y", "z", "R", "eps", "q"):
        c["atoms"][k] = c["atoms"][k][:0]
    ff, grid = gpu_ff(c, 1, (4, 4, 4))
    assert torch.count_nonzero(ff).item() == 0


def test_flake_full_size_sampled_nodes(orc):
    # 256 x 256 x 200 grid and the 60-atom flake, as timed by the benchmark; 4000 sampled nodes
    c = case32(synth.flake_case())
    ff, grid = gpu_ff(c)
    g = c["grid"]
    F = ff.view(g["nz"], g["ny"], g["nx"], 4)
    rng = np.random.default_rng(0)
    idx = np.stack([rng.integers(0, g[n], 4000) for n in ("nz", "ny", "nx")], axis=1)
    got = F[idx[:, 0], idx[:, 1], idx[:, 2]].cpu().numpy().astype(np.float64)
    pts = np.stack([np.float32(g["x0"]) + idx[:, 2] * np.float32(g["dx"]),
                    np.float32(g["y0"]) + idx[:, 1] * np.float32(g["dy"]),
                    np.float32(g["z0"]) + idx[:, 0] * np.float32(g["dz"])], axis=1).astype(np.float64)
    ref, core = orc.ff_points(c["atoms"], c["probe"], g, pts)
    err = ff_rel_err(got, ref)[~core]
    assert err.max() <= TOL, err.max()
    assert torch.isfinite(F).all()


@pytest.mark.parametrize("zpt", [4, 8, 16])
@pytest.mark.parametrize("variant", ["plain", "min_image_cutoff", "quadrupole"])
def test_forces_only_grid_has_the_same_forces_and_zero_energies(orc, zpt, variant):
    # ff_forces_only drops the energy sums: every force component is bit for bit the full grid's,
    # every E slot is 0, and the forces still meet the oracle bar
    c = case32(synth.small_case(seed=6, n_atoms=14, nxy=34, nz=29))
    if variant == "min_image_cutoff":
        c["probe"] = dict(synth.default_probe(coul_rc=3.0, min_image=1), Q=c["probe"]["Q"])
    elif variant == "quadrupole":
        c["probe"] = dict(c["probe"], Qzz=-0.05)
    c = case32(c)
    grid = pp.make_grid(c["grid"], 0)
    atoms, probe = pp.make_atoms(afm.atoms_to_device(c["atoms"])), pp.make_probe(c["probe"])
    full = torch.full((pp.pp_ff_floats(grid),), float("nan"), dtype=torch.float32, device="cuda")
    forces = torch.full_like(full, float("nan"))
    pp.pp_make_ff_tuned(atoms, probe, grid, full, pp.Tuning(zpt, 0))
    pp.pp_make_ff_tuned(atoms, probe, grid, forces, pp.Tuning(zpt, 1))
    a, b = full.view(-1, 4), forces.view(-1, 4)
    assert torch.equal(a[:, :3], b[:, :3])
    assert torch.count_nonzero(b[:, 3]).item() == 0 and torch.count_nonzero(a[:, 3]).item() > 0
    ref, core = orc.make_ff(c["atoms"], c["probe"], c["grid"])
    F = linear_ff(forces.cpu().numpy(), c["grid"])
    assert ff_rel_err(F, ref)[~core].max() <= TOL


def test_forces_only_simulator_gives_the_same_images():
    c = case32(synth.small_case(seed=7, n_atoms=11, nxy=32, nz=36, scan_px=10, nz_scan=14))
    outs = []
    for energy in (True, False):
        sim = afm.Simulator(c, ff_energy=energy)
        sim.run(afm.atoms_to_device(c["atoms"]))
        outs.append((sim.df.clone(), sim.pos.clone(), sim.iters.clone()))
    for u, v in zip(*outs):
        assert torch.equal(u, v)


def test_forces_only_on_a_bricked_grid():
    # the forces-only flag is independent of the storage layout: bricked grid, padding written
    c = case32(synth.small_case(seed=8, n_atoms=10, nxy=26, nz=13))
    g1 = pp.make_grid(c["grid"], 1, (4, 4, 4))
    atoms, probe = pp.make_atoms(afm.atoms_to_device(c["atoms"])), pp.make_probe(c["probe"])
    full = torch.full((pp.pp_ff_floats(g1),), float("nan"), dtype=torch.float32, device="cuda")
    forces = torch.full_like(full, float("nan"))
    pp.pp_make_ff_tuned(atoms, probe, g1, full, pp.Tuning(8, 0))
    pp.pp_make_ff_tuned(atoms, probe, g1, forces, pp.Tuning(8, 1))
    a, b = full.view(-1, 4), forces.view(-1, 4)
    assert torch.isfinite(b).all()
    assert torch.equal(a[:, :3], b[:, :3]) and torch.count_nonzero(b[:, 3]).item() == 0


@pytest.mark.parametrize("variant", ["plain", "min_image_cutoff"])
def test_every_launch_shape_writes_the_same_grid(variant):
    # 4, 8 or 16 z-nodes per thread, the last z-block of a column ragged for all three (29 layers; at
    # 16 the last 13 go to a tail launch), the whole grid or a layer range: the same bits
    c = case32(synth.small_case(seed=16, n_atoms=13, nxy=34, nz=29))
    if variant == "min_image_cutoff":
        c["probe"] = dict(synth.default_probe(coul_rc=3.0, min_image=1), Q=c["probe"]["Q"])
        c = case32(c)
    grid = pp.make_grid(c["grid"], 0)
    atoms, probe = pp.make_atoms(afm.atoms_to_device(c["atoms"])), pp.make_probe(c["probe"])
    grids = {}
    for zpt in (4, 8, 16):
        g = torch.full((pp.pp_ff_floats(grid),), float("nan"), dtype=torch.float32, device="cuda")
        pp.pp_make_ff_tuned(atoms, probe, grid, g, pp.Tuning(zpt, 1))
        grids[zpt] = g
        part = torch.full_like(g, float("nan"))
        pp.pp_make_ff_layers(atoms, probe, grid, part, 3, 26, pp.Tuning(zpt, 1))
        torch.cuda.synchronize()
        n = c["grid"]["nx"] * c["grid"]["ny"] * 4
        assert torch.equal(part[3 * n:26 * n], g[3 * n:26 * n]), zpt
        assert torch.isnan(part[:3 * n]).all() and torch.isnan(part[26 * n:]).all()
    assert torch.isfinite(grids[8]).all()
    assert torch.equal(grids[4], grids[8]) and torch.equal(grids[16], grids[8])
