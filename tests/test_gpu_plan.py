"""The scan's pixel-to-warp plan: pp_relax_plan lists the costliest pixel columns
of an earlier scan (exactly, up to its cost bins), and a scan run with any plan
-- its own, another image's, one column or all of them, one lane to a warp or
32 -- writes the bits of the scan without one."""
import copy

import numpy as np
import pytest
import torch

from helpers import case32
from paper_2401_14564_gb300 import afm, pp, synth

pytestmark = pytest.mark.gpu


def outputs(sim):
    return [t.clone() for t in (sim.df, sim.fz, sim.pos, sim.iters)]


def plan_parts(plan, npix, k, lanes):
    w = plan.cpu().numpy()
    off = 8 + 2048 + npix
    hb = (k + lanes - 1) // lanes
    lst = w[off:off + hb * lanes]
    mask = w[off + hb * lanes:off + hb * lanes + (npix + 31) // 32].view(np.uint32)
    bits = np.unpackbits(mask.view(np.uint8), bitorder="little")[:npix].astype(bool)
    return lst, bits


@pytest.mark.parametrize("k,lanes", [(1, 1), (37, 4), (100, 3), (200, 32)])
def test_plan_lists_the_costliest_columns(k, lanes):
    c = case32(synth.small_case(seed=21, n_atoms=12, nxy=36, nz=40, scan_px=13, nz_scan=15))
    sim = afm.Simulator(c, plan_frac=0.0)
    sim.run(afm.atoms_to_device(c["atoms"]))
    s = c["scan"]
    npix = s["nx"] * s["ny"]
    k = min(k, npix)
    plan = torch.zeros(pp.pp_relax_plan_size(sim.scan, k, lanes) // 4, dtype=torch.int32, device="cuda")
    pp.pp_relax_plan(sim.iters, sim.scan, sim.fire.max_iter, k, lanes, plan)
    torch.cuda.synchronize()
    lst, bits = plan_parts(plan, npix, k, lanes)
    chosen = lst[lst >= 0]
    assert len(chosen) == k and len(set(chosen.tolist())) == k and chosen.max() < npix
    assert np.array_equal(np.flatnonzero(bits), np.sort(chosen))
    assert (lst[k:] == -1).all()
    # costs binned as the plan bins them: every chosen column at or above the boundary bin,
    # every other one at or below it
    cost = sim.iters.cpu().numpy().astype(np.int64).sum(0).ravel()
    top, shift = s["nz"] * sim.fire.max_iter, 0
    while (top >> shift) >= 2048:
        shift += 1
    b = np.minimum(cost >> shift, 2047)
    t = np.sort(b)[::-1][k - 1]
    assert b[chosen].min() >= t
    assert b[np.setdiff1d(np.arange(npix), chosen)].max(initial=0) <= t


@pytest.mark.parametrize("variant", ["plain", "polish", "tricubic", "bricks", "unfused", "zspan"])
def test_planned_scan_writes_the_same_bits(variant):
    c = case32(synth.small_case(seed=22, n_atoms=11, nxy=40, nz=44, scan_px=17, nz_scan=14))
    kw = {}
    fire = None
    if variant == "polish":
        fire = synth.default_fire(polish=4)
    if variant == "tricubic":
        c["grid"] = dict(c["grid"], interp=1)
    if variant == "bricks":
        kw = dict(layout=1, brick=(4, 4, 4))
    if variant == "unfused":
        kw = dict(fused_df=False)
    atoms = afm.atoms_to_device(c["atoms"])
    ref = afm.Simulator(c, fire=fire, plan_frac=0.0, **kw)
    ref.run(atoms)
    want = outputs(ref)
    s = c["scan"]
    npix = s["nx"] * s["ny"]
    for frac, lanes in ((1.0 / npix, 1), (0.05, 4), (0.3, 8), (1.0, 32), (1.0, 1)):
        sim = afm.Simulator(c, fire=fire, plan_frac=frac, plan_lanes=lanes, auto_plan=False, plan_min_tiles=0,
                            **kw)
        sim.make_ff(atoms)
        sim.plan_from(ref.iters)
        zs = torch.empty(2, dtype=torch.int32, device="cuda") if variant == "zspan" else None
        sim.relax(zspan=zs)
        torch.cuda.synchronize()
        for a, b in zip(outputs(sim), want):
            assert torch.equal(a, b), (frac, lanes)


def test_another_images_plan_changes_nothing():
    # a plan is a schedule: one built from a moved molecule (or from no relation at all) still gives
    # this image's bits
    c = case32(synth.small_case(seed=23, n_atoms=12, nxy=40, nz=44, scan_px=16, nz_scan=14))
    other = copy.deepcopy(c)
    other["atoms"]["x"] = other["atoms"]["x"] + 0.6
    other["atoms"]["q"] = -other["atoms"]["q"]
    a_sim = afm.Simulator(other, plan_frac=0.0)
    a_sim.run(afm.atoms_to_device(other["atoms"]))
    atoms = afm.atoms_to_device(c["atoms"])
    ref = afm.Simulator(c, plan_frac=0.0)
    ref.run(atoms)
    want = outputs(ref)
    sim = afm.Simulator(c, plan_frac=0.1, auto_plan=False, plan_min_tiles=0)
    sim.plan_from(a_sim.iters)
    sim.run(atoms)
    torch.cuda.synchronize()
    for x, y in zip(outputs(sim), want):
        assert torch.equal(x, y)


def test_auto_plan_over_a_sequence_of_images():
    c = case32(synth.small_case(seed=24, n_atoms=10, nxy=36, nz=40, scan_px=15, nz_scan=13))
    auto = afm.Simulator(c, plan_min_tiles=0)  # each scan plans the next
    plain = afm.Simulator(c, plan_frac=0.0)
    for t in range(4):
        a = copy.deepcopy(c["atoms"])
        a["y"] = a["y"] - 0.04 * t
        at = afm.atoms_to_device(a)
        if t == 2:
            auto.plan_lanes = 8   # the plan held was built for 4 lanes: it is used as built, the next is for 8
        if t == 3:
            auto.plan_frac = 0.2
        auto.run(at)
        plain.run(at)
        torch.cuda.synchronize()
        assert auto._plan_ready
        for x, y in zip(outputs(auto), outputs(plain)):
            assert torch.equal(x, y), t


def test_small_scans_get_no_plan():
    # benzene's 40 x 40 pixels are 50 tiles, fewer than the SMs: no plan is built
    c = case32(synth.benzene_case())
    sim = afm.Simulator(c)
    sim.run(afm.atoms_to_device(c["atoms"]))
    sim.run(afm.atoms_to_device(c["atoms"]))
    assert not sim._plan_ready


def test_flake_scan_on_its_own_plan():
    # the full-size scan with the default plan (2.5 % of the columns, 4 lanes), built by the first call
    c = synth.flake_case()
    at = afm.atoms_to_device(c["atoms"])
    plain = afm.Simulator(c, ff_energy=False, plan_frac=0.0)
    plain.run(at)
    sim = afm.Simulator(c, ff_energy=False)
    sim.run(at)
    sim.run(at)
    torch.cuda.synchronize()
    assert sim._plan_ready and sim._plan_k == round(0.025 * 256 * 256)
    for x, y in zip(outputs(sim), outputs(plain)):
        assert torch.equal(x, y)
