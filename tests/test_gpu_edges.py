"""Minimum-size and degenerate inputs of the GPU path against the FP64 oracle:
a single pixel with exactly 2m+1 heights (one df value), FIRE with no
iterations allowed, a grid two nodes high, and the smallest FFT grids; the
streamed and pipelined multi-item paths against one call per item.
"""
import copy

import numpy as np
import pytest
import torch

from helpers import case32
from paper_2401_14564_gb300 import afm, pp, synth
from test_gpu_fft import check as fft_check
from test_gpu_fft import run as fft_run
from test_gpu_relax import check_parity

pytestmark = pytest.mark.gpu


def test_single_pixel_with_the_minimum_number_of_heights(orc):
    c = copy.deepcopy(synth.benzene_case())
    m = pp.pp_df_margin(c["df"]["A_pp"], c["scan"]["dz"])
    c["scan"] = dict(c["scan"], nx=1, ny=1, nz=2 * m + 1, x0=0.71, y0=-0.33)
    c = case32(c)
    fire = synth.parity_fire()
    g = afm.afm(c, fire=fire)
    o = orc.forward(c, fire=fire)
    assert g["df"].shape == (1, 1, 1) and o["df"].shape == (1, 1, 1)
    assert np.abs(g["pos"] - o["pos"]).max() <= 1e-3
    # one df value: the image has no range, so the bar is 1e-3 of the value itself
    assert abs(g["df"].item() - o["df"].item()) <= 1e-3 * abs(o["df"].item())


def test_no_iterations_allowed_leaves_the_probe_at_rest(orc):
    c = case32(synth.small_case(seed=4, n_atoms=9, nxy=24, nz=30, scan_px=9, nz_scan=11))
    fire = synth.parity_fire(max_iter=0)
    g = afm.afm(c, fire=fire)
    assert (g["iters"] == 0).all()
    o = orc.relax_scan(orc.make_ff(c["atoms"], c["probe"], c["grid"])[0], c["grid"], None, None, c["scan"],
                       c["tip"], fire, polish_tol=0.0)
    # no update: every height starts (and stays) at anchor + d0
    s = c["scan"]
    k, j, i = np.meshgrid(np.arange(s["nz"]), np.arange(s["ny"]), np.arange(s["nx"]), indexing="ij")
    rest = np.stack([s["x0"] + i * s["px"], s["y0"] + j * s["py"], s["z_top"] - k * s["dz"] - c["tip"]["R0"]], -1)
    assert np.abs(g["pos"] - rest).max() < 1e-5
    assert np.abs(o["pos"] - rest).max() < 1e-12
    assert np.abs(g["fz"]).max() < 1e-6


def test_grid_two_nodes_high(orc):
    # nz = 2: one cell in z, every probe position clamps into it (fractions clamped to [0, 1])
    c = copy.deepcopy(synth.small_case(seed=5, n_atoms=8, nxy=24, nz=40, scan_px=8, nz_scan=11))
    g = c["grid"]
    c["grid"] = dict(g, nz=2, z0=g["z0"] + 1.5, dz=1.2)
    # a weak image (about 2 Hz of range): FIRE is stopped at 1e-6 eV/A so that its stopping
    # tolerance (positions within ftol / lambda) stays below the 1e-3-of-range df bar
    check_parity(orc, c, fire=synth.parity_fire(ftol=1e-6, max_iter=20000))


@pytest.mark.parametrize("shape", [(2, 2, 2), (2, 4, 8), (8, 2, 4)])
def test_smallest_fft_grids(orc, shape):
    g = {"nx": shape[0], "ny": shape[1], "nz": shape[2], "x0": 0.0, "y0": 0.0, "z0": 0.0, "dx": 0.4, "dy": 0.5,
         "dz": 0.3, "periodic_xy": 1}
    rng = np.random.default_rng(sum(shape))
    f = rng.standard_normal((shape[2], shape[1], shape[0]))
    t = rng.random((shape[2], shape[1], shape[0]))
    fft_check(fft_run(f, t, g, scale=1.3), orc.correlate(f, t, g, scale=1.3))


def test_streamed_host_path_equals_one_call_per_item():
    # run_host_many overlaps each item's copy-out with the next item's compute; the images must be
    # those of run_host, item by item
    c = case32(synth.small_case(seed=11, n_atoms=10, nxy=32, nz=36, scan_px=10, nz_scan=12))
    items = []
    for t in range(5):
        a = copy.deepcopy(c["atoms"])
        a["x"] = a["x"] + 0.07 * t
        a["q"] = a["q"] * (1.0 - 0.1 * t)
        items.append(a)
    sim = afm.Simulator(c)
    many = [o.clone() for o in sim.run_host_many(items)]
    one = [sim.run_host(a).clone() for a in items]
    for k in range(len(items)):
        assert torch.equal(many[k], one[k]), k
    assert not torch.equal(many[0], many[-1])


def test_pipeline_items_equal_one_run_per_item():
    # two items in flight on two streams with their own grids: every image is the single-item one
    c = case32(synth.small_case(seed=12, n_atoms=11, nxy=32, nz=36, scan_px=10, nz_scan=12))
    items = []
    for t in range(5):
        a = copy.deepcopy(c["atoms"])
        a["y"] = a["y"] - 0.05 * t
        a["eps"] = a["eps"] * (1.0 + 0.2 * t)
        items.append(a)
    sim = afm.Simulator(c)
    one = []
    for a in items:
        sim.run(afm.atoms_to_device(a))
        one.append(sim.df.clone())
    pipe = afm.Pipeline(c, slots=2)
    outs = [torch.empty_like(one[0]) for _ in items]
    pipe.run_many([afm.atoms_to_device(a) for a in items], outs)
    torch.cuda.synchronize()
    host = [o.clone() for o in pipe.run_host_many(items)]
    for k in range(len(items)):
        assert torch.equal(outs[k], one[k]), k
        assert torch.equal(host[k], one[k].cpu()), k
    assert not torch.equal(one[0], one[-1])


def test_saved_outputs_round_trip(tmp_path):
    c = case32(synth.small_case(seed=13, n_atoms=9, nxy=24, nz=30, scan_px=9, nz_scan=12))
    sim = afm.Simulator(c)
    sim.run(afm.atoms_to_device(c["atoms"]))
    path = tmp_path / "run.npz"
    sim.save(path)
    z = np.load(path)
    assert np.array_equal(z["df"], sim.df.cpu().numpy()) and np.array_equal(z["ff"], sim.ff.cpu().numpy())
    assert np.array_equal(z["pos"], sim.pos.cpu().numpy()) and np.array_equal(z["iters"], sim.iters.cpu().numpy())
    assert int(z["grid_geometry"][0]) == c["grid"]["nx"] and int(z["scan_geometry"][2]) == c["scan"]["nz"]


def test_read_probe_runs_and_writes_nothing():
    # the benchmark's L2 read-bandwidth probe: reads the buffer, leaves the sink alone
    buf = torch.rand(1 << 20, device="cuda")
    sink = torch.full((1,), 7.0, device="cuda")
    pp.pp_read_probe(buf, 3, sink)
    torch.cuda.synchronize()
    assert sink.item() == 7.0
