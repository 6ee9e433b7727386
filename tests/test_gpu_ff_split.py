"""The split force field (pp_make_ff_split, pp_ff_combine): Lennard-Jones (and
the tip quadrupole) in one grid, the point-charge field per unit probe charge
in another, recombined for any probe charge Q.

Oracle references: the LJ grid is the oracle's grid for the same probe with
Q = 0; the electrostatic grid is the oracle's grid with Q = 1, eps_PP = 0 (no
LJ) and Qzz = 0.  Bars as for pp_make_ff (K1): force 1e-4 relative with a
1e-3 eV/A floor outside the core, energy 1e-4 with a 1e-2 eV floor.  The
recombined grid is held to the same bars against the oracle's grid for Q, and
the combine kernel itself to one FP32 rounding of ff + Q ff_el.
"""
import copy

import numpy as np
import pytest
import torch

from helpers import case32, df_keep, ff_rel_err, ill_conditioned_within_bound, linear_ff, relax_compare
from paper_2401_14564_gb300 import afm, pp, synth

pytestmark = pytest.mark.gpu

TOL = 1e-4


def split(c, layout=0):
    grid = pp.make_grid(c["grid"], layout)
    n = pp.pp_ff_floats(grid)
    ff = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
    el = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
    pp.pp_make_ff_split(pp.make_atoms(afm.atoms_to_device(c["atoms"])), pp.make_probe(c["probe"]), grid, ff, el)
    return ff, el, grid


def host(t, g):
    if g.get("interp", 0) == 1:
        return t.cpu().numpy().astype(np.float64).reshape(g["nz"], g["ny"], g["nx"])
    return linear_ff(t.cpu().numpy(), g)


def check_grid(F, ref, core, energy_only=False):
    assert np.isfinite(F).all()
    if energy_only:
        eerr = (np.abs(F - ref[..., 3]) / np.maximum(np.abs(ref[..., 3]), 1e-2))[~core]
    else:
        assert ff_rel_err(F, ref)[~core].max() <= TOL
        eerr = (np.abs(F[..., 3] - ref[..., 3]) / np.maximum(np.abs(ref[..., 3]), 1e-2))[~core]
    assert eerr.max() <= TOL, eerr.max()


def refs(orc, c):
    lj_probe = dict(c["probe"], Q=0.0)
    el_probe = dict(c["probe"], Q=1.0, eps_pp=0.0, Qzz=0.0)
    lj, core = orc.make_ff(c["atoms"], lj_probe, c["grid"])
    el, core_el = orc.make_ff(c["atoms"], el_probe, c["grid"])
    return lj, el, core | core_el


CASES = {
    "plain": lambda: synth.small_case(seed=3, n_atoms=12, nxy=32, nz=37),
    "min_image_cutoff_quad": lambda: dict(synth.small_case(seed=5, n_atoms=20, nxy=24, nz=17),
                                          probe=synth.default_probe(coul_rc=3.0, min_image=1, Qzz=-0.1)),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("interp", [0, 1])
def test_split_grids_match_oracle(orc, name, interp):
    c = case32(CASES[name]())
    c["grid"] = dict(c["grid"], interp=interp)
    ff, el, grid = split(c)
    lj_ref, el_ref, core = refs(orc, c)
    check_grid(host(ff, c["grid"]), lj_ref, core, energy_only=interp == 1)
    check_grid(host(el, c["grid"]), el_ref, core, energy_only=interp == 1)


@pytest.mark.parametrize("layout", [0, 1])
def test_combined_grid_is_the_grid_for_each_charge(orc, layout):
    c = case32(CASES["plain"]())
    ff, el, grid = split(c, layout)
    out = torch.empty_like(ff)
    for Q in (-0.3, 0.0, 0.12):
        pp.pp_ff_combine(ff, el, Q, grid, out)
        torch.cuda.synchronize()
        # one FP32 rounding of ff + Q ff_el per float
        a, b, o = ff.cpu().numpy().astype(np.float64), el.cpu().numpy().astype(np.float64), out.cpu().numpy()
        exact = a + np.float32(Q) * b
        assert np.all(np.abs(o - exact) <= 2.0 ** -23 * (np.abs(a) + np.abs(np.float32(Q) * b)) + 1e-30)
        cq = copy.deepcopy(c)
        cq["probe"] = dict(c["probe"], Q=Q)
        ref, core = orc.make_ff(cq["atoms"], cq["probe"], cq["grid"])
        lin = out if layout == 0 else None
        if layout == 1:
            lg = pp.make_grid(c["grid"], 0)
            lin = torch.empty(pp.pp_ff_floats(lg), dtype=torch.float32, device="cuda")
            pp.pp_ff_convert(out, grid, lin, lg)
        check_grid(linear_ff(lin.cpu().numpy(), c["grid"]), ref, core)


def test_combine_in_place_and_odd_energy_grid():
    # an energy grid of 5 x 3 x 7 = 105 floats: 26 float4 plus a tail of one float
    c = case32(synth.small_case(seed=6, n_atoms=7, nxy=8, nz=10))
    c["grid"] = dict(c["grid"], nx=5, ny=3, nz=7, interp=1)
    ff, el, grid = split(c)
    assert ff.numel() == 105
    a, b = ff.cpu().numpy().astype(np.float64), el.cpu().numpy().astype(np.float64)
    pp.pp_ff_combine(ff, el, 0.7, grid, ff)  # in place
    torch.cuda.synchronize()
    qb = np.float64(np.float32(0.7)) * b
    # one FP32 rounding of a + Q b, the tail float included
    assert np.all(np.abs(ff.cpu().numpy() - (a + qb)) <= 2.0 ** -23 * (np.abs(a) + np.abs(qb)) + 1e-30)


def test_scan_on_a_recombined_grid_matches_the_oracle(orc):
    c = case32(CASES["plain"]())
    fire = synth.parity_fire()
    ff, el, grid = split(c)
    pp.pp_ff_combine(ff, el, c["probe"]["Q"], grid, ff)
    sim = afm.Simulator(c, fire=fire)
    sim.ff.copy_(ff)
    sim.relax()
    torch.cuda.synchronize()
    g = {"pos": sim.pos.cpu().numpy(), "fz": sim.fz.cpu().numpy(), "df": sim.df.cpu().numpy(),
         "iters": sim.iters.cpu().numpy()}
    o = orc.forward(c, fire=fire)
    dp, dfz, keep, n_ill, n_basin = relax_compare(g, o)
    assert n_ill + n_basin <= 0.02 * keep.size
    assert dp <= 1e-3, dp
    n_sel, n_ok = ill_conditioned_within_bound(g["pos"], o, fire["ftol"])
    assert n_ok == n_sel
    kd = df_keep(keep, (keep.shape[0] - g["df"].shape[0]) // 2)
    assert np.abs(g["df"] - o["df"])[kd].max() <= 1e-3 * (o["df"].max() - o["df"].min())
