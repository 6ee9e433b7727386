"""The force field in two parts beside the scan: pp_make_ff_layers writes exactly
the nodes of its layers, pp_relax_scan_ex reports every layer the scan read
(and its outputs are pp_relax_scan's), and Simulator.run_host with the
overlapped force field returns, call after call, the images of the one-stage
path, also when the scan leaves the first part and is run again."""
import copy

import numpy as np
import pytest
import torch

from helpers import case32
from paper_2401_14564_gb300 import afm, pp, synth

pytestmark = pytest.mark.gpu


def tall_case(seed=5):
    # a grid 12 A high of which the scan reads a band a few A thick
    c = synth.small_case(seed=seed, n_atoms=10, nxy=40, nz=120, scan_px=11, nz_scan=14, d=0.1)
    return case32(c)


def grid_and_atoms(c, layout=0, brick=(4, 4, 4)):
    g = pp.make_grid(c["grid"], layout=layout, brick=brick)
    atoms_t = afm.atoms_to_device(c["atoms"])
    return g, atoms_t, pp.make_atoms(atoms_t), pp.make_probe(c["probe"])


@pytest.mark.parametrize("layout,tuning", [(0, None), (0, (4, 1)), (0, (16, 0)), (1, (8, 1))])
def test_layers_write_exactly_their_nodes(layout, tuning):
    c = tall_case()
    g, _, A, probe = grid_and_atoms(c, layout=layout, brick=(4, 4, 8))
    n = pp.pp_ff_floats(g)
    tun = pp.Tuning(*tuning) if tuning is not None else None
    full = torch.empty(n, device="cuda")
    pp.pp_make_ff_tuned(A, probe, g, full, tun)
    nz = c["grid"]["nz"]
    # one band into a NaN-filled buffer: its nodes equal the whole-grid call's, nothing else is written
    band = torch.full((n,), float("nan"), device="cuda")
    pp.pp_make_ff_layers(A, probe, g, band, 37, 58, tun)
    # the three parts together give the whole grid (a zeroed buffer: bricked padding stays 0, as
    # the whole-grid call leaves it)
    parts = torch.zeros(n, device="cuda")
    for k0, k1 in ((37, 58), (58, nz), (0, 37)):
        pp.pp_make_ff_layers(A, probe, g, parts, k0, k1, tun)
    torch.cuda.synchronize()
    assert torch.equal(parts, full)
    if layout == 0:
        nx, ny = c["grid"]["nx"], c["grid"]["ny"]
        f = full.view(nz, ny, nx, 4)
        b = band.view(nz, ny, nx, 4)
        assert torch.equal(b[37:58], f[37:58])
        assert torch.isnan(b[:37]).all() and torch.isnan(b[58:]).all()


def test_layers_of_an_energy_grid():
    c = tall_case()
    c["grid"] = dict(c["grid"], interp=1)
    g, _, A, probe = grid_and_atoms(c)
    n = pp.pp_ff_floats(g)
    full = torch.empty(n, device="cuda")
    pp.pp_make_ff(A, probe, g, full)
    parts = torch.full((n,), float("nan"), device="cuda")
    nz = c["grid"]["nz"]
    for k0, k1 in ((0, 1), (1, 61), (61, nz)):  # a single layer is a valid part
        pp.pp_make_ff_layers(A, probe, g, parts, k0, k1)
    torch.cuda.synchronize()
    assert torch.equal(parts, full)


def scan_outputs(sim):
    return [t.clone() for t in (sim.df, sim.fz, sim.pos, sim.iters)]


def poison_outside(ff, c, lo, hi, interp):
    nz, ny, nx = c["grid"]["nz"], c["grid"]["ny"], c["grid"]["nx"]
    v = ff.view(nz, ny, nx, -1) if interp == 0 else ff.view(nz, ny, nx)
    v[:lo] = float("nan")
    v[hi + 1:] = float("nan")


@pytest.mark.parametrize("interp,polish", [(0, 0), (0, 4), (1, 0)])
def test_zspan_covers_every_layer_the_scan_reads(interp, polish):
    c = tall_case(seed=7)
    c["grid"] = dict(c["grid"], interp=interp)
    sim = afm.Simulator(c, fire=synth.default_fire(polish=polish), overlap_ff=False)
    atoms = afm.atoms_to_device(c["atoms"])
    sim.run(atoms)
    ref = scan_outputs(sim)
    zspan = torch.empty(2, dtype=torch.int32, device="cuda")
    pp.pp_relax_scan(sim.ff, sim.grid, sim.scan, sim.tip, sim.fire, sim.pos, sim.fz, sim.iters, sim.dfp, sim.df,
                     zspan=zspan)
    torch.cuda.synchronize()
    for a, b in zip(scan_outputs(sim), ref):
        assert torch.equal(a, b)  # the reporting scan computes what pp_relax_scan does
    lo, hi = int(zspan[0]), int(zspan[1])
    nz = c["grid"]["nz"]
    assert 0 <= lo <= hi <= nz - 1
    assert hi - lo < nz // 2  # a band, not the grid
    # every relaxed position lies in a cell of the band
    g = c["grid"]
    kz = np.floor((sim.pos[..., 2].cpu().numpy().astype(np.float64) - g["z0"]) / g["dz"])
    assert kz.min() >= lo - 1 and kz.max() <= hi
    # layers outside the band hold NaN now: the scan, run again, gives the same bits
    poison_outside(sim.ff, c, lo, hi, interp)
    sim.relax()
    torch.cuda.synchronize()
    for a, b in zip(scan_outputs(sim), ref):
        assert torch.equal(a, b)


@pytest.mark.parametrize("interp", [0, 1])
def test_run_host_overlapped_equals_one_stage_path(interp):
    c = tall_case(seed=9)
    c["grid"] = dict(c["grid"], interp=interp)
    items = []
    for t in range(4):
        a = copy.deepcopy(c["atoms"])
        a["x"] = a["x"] + 0.05 * t
        a["z"] = a["z"] - 0.03 * t
        items.append(a)
    plain = afm.Simulator(c, overlap_ff=False)
    ov = afm.Simulator(c)
    nz = c["grid"]["nz"]
    firsts = []
    for a in items:
        want = plain.run_host(a).clone()
        got = ov.run_host(a).clone()
        assert torch.equal(got, want)
        for x, y in zip(scan_outputs(ov)[1:], scan_outputs(plain)[1:]):
            assert torch.equal(x, y)
        assert torch.equal(ov.ff, plain.ff)  # the grid is complete after the call
        firsts.append(ov._first)
    assert ov.reruns == 0
    # the first call takes the anchors' reach, later ones the band the previous scan read
    assert firsts[1][1] - firsts[1][0] < firsts[0][1] - firsts[0][0] < nz


def test_scan_leaving_the_first_part_is_run_again():
    c = tall_case(seed=10)
    plain = afm.Simulator(c, overlap_ff=False)
    want = plain.run_host(c["atoms"]).clone()
    ov = afm.Simulator(c)
    nz = c["grid"]["nz"]
    for part in ((0, 2), (nz - 3, nz)):  # far from the band the scan reads
        ov.first_layers = lambda part=part: part
        got = ov.run_host(c["atoms"]).clone()
        assert torch.equal(got, want)
        assert torch.equal(ov.fz, plain.fz)
    assert ov.reruns == 2
