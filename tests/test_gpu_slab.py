"""The 2516-atom periodic slab at full size (512 x 512 x 250 grid, 512 x 512 px x 60 heights):
minimum-image lateral sums and the shifted-force Coulomb cut at 8 A, forward and adjoint.

The FP64 oracle cannot build the whole grid in test time (1.65e11 pair terms), so it checks
  - 3000 sampled grid nodes against direct sums;
  - an 8 x 8 pixel patch over the molecule, relaxed on an oracle window of the grid that the
    patch's probe particles stay inside (minimum image with the full 51.2 A period);
  - the adjoint with loss weights on that patch only: the CUDA adjoint evaluated at the oracle's
    relaxed positions of the patch against the oracle adjoint on the window.
"""
import numpy as np
import pytest
import torch

from helpers import case32, ff_rel_err
from paper_2401_14564_gb300 import afm, pp, synth

pytestmark = pytest.mark.gpu

KEYS = ("x", "y", "z", "q", "R", "eps")


@pytest.fixture(scope="module")
def slab():
    c = case32(synth.slab_case())
    fire = synth.parity_fire()
    sim = afm.Simulator(c, fire=fire)
    at = afm.atoms_to_device(c["atoms"])
    sim.run(at)
    torch.cuda.synchronize()
    return c, sim, at, fire


def window(c, i0, j0, k0, n, nzw):
    g = c["grid"]
    return dict(g, nx=n, ny=n, nz=nzw, x0=float(np.float32(g["x0"]) + i0 * np.float32(g["dx"])),
                y0=float(np.float32(g["y0"]) + j0 * np.float32(g["dy"])),
                z0=float(np.float32(g["z0"]) + k0 * np.float32(g["dz"])), periodic_xy=0,
                Lx=g["nx"] * g["dx"], Ly=g["ny"] * g["dy"])


def test_slab_grid_sampled_nodes(orc, slab):
    c, sim, at, fire = slab
    g = c["grid"]
    F = sim.ff.view(g["nz"], g["ny"], g["nx"], 4)
    rng = np.random.default_rng(5)
    # half the nodes anywhere (the grid starts inside the bilayer, so many are in the clamped
    # core), half in the heights the probe visits (z = 9 .. 19 A)
    idx = np.stack([rng.integers(0, g[n], 3000) for n in ("nz", "ny", "nx")], axis=1)
    idx[1500:, 0] = rng.integers(90, 191, 1500)
    got = F[idx[:, 0], idx[:, 1], idx[:, 2]].cpu().numpy().astype(np.float64)
    pts = np.stack([np.float32(g["x0"]) + idx[:, 2] * np.float32(g["dx"]),
                    np.float32(g["y0"]) + idx[:, 1] * np.float32(g["dy"]),
                    np.float32(g["z0"]) + idx[:, 0] * np.float32(g["dz"])], axis=1).astype(np.float64)
    ref, core = orc.ff_points(c["atoms"], c["probe"], g, pts)
    # the minimum-image field jumps where an atom sits half a period away; within 1e-4 A of that
    # plane (50x the FP32 rounding of a 25 A distance) the image is decided by rounding, so such
    # nodes are excluded like the clamped core (and must be rare)
    L = (g["nx"] * g["dx"], g["ny"] * g["dy"])
    half = np.zeros(len(pts), dtype=bool)
    for ax, key in ((0, "x"), (1, "y")):
        d = pts[:, None, ax] - np.asarray(c["atoms"][key])[None]
        d = np.abs(d - L[ax] * np.rint(d / L[ax]))
        half |= (np.abs(d - L[ax] / 2) < 1e-4).any(axis=1)
    assert half.mean() <= 0.05
    keep = ~core & ~half
    assert keep.sum() >= 1500
    assert ff_rel_err(got, ref)[keep].max() <= 1e-4


def patch(c):
    s = c["scan"]
    ii, jj = np.meshgrid(np.arange(252, 260), np.arange(252, 260))
    return (jj * s["nx"] + ii).ravel()


def test_slab_patch_relaxation_and_adjoint(orc, slab):
    c, sim, at, fire = slab
    s = c["scan"]
    cols = patch(c)
    # window: +-4.8 A around the patch laterally, z 9.0 .. 19.0 A
    win = window(c, 252 - 48, 252 - 48, 90, 104, 101)
    ffw, core = orc.make_ff(c["atoms"], c["probe"], win)
    o = orc.relax_columns(ffw, win, None, None, s, c["tip"], fire, cols)
    assert o["ok"].all()
    lo = np.array([win["x0"], win["y0"], win["z0"]]) + 1.0
    hi = np.array([win["x0"] + (win["nx"] - 1) * 0.1, win["y0"] + (win["ny"] - 1) * 0.1,
                   win["z0"] + (win["nz"] - 1) * 0.1]) - 1.0
    assert (o["pos"] > lo).all() and (o["pos"] < hi).all(), "the patch's probe left the oracle window"
    jj, ii = cols // s["nx"], cols % s["nx"]
    gp = np.moveaxis(sim.pos.cpu().numpy()[:, jj, ii], 0, 1)
    dp = np.linalg.norm(gp - o["pos"], axis=-1)
    keep = (o["lam"] >= 0.01) & (dp < 0.05)
    assert keep.mean() > 0.9
    assert dp[keep].max() <= 1e-3
    # adjoint with weights on the patch only, CUDA adjoint at the oracle's relaxed positions
    m = sim.m
    w = np.zeros((s["nz"] - 2 * m, s["ny"], s["nx"]))
    w[:, jj, ii] = np.random.default_rng(9).standard_normal((s["nz"] - 2 * m, len(cols)))
    pos = sim.pos.cpu().numpy().astype(np.float64)
    pos[:, jj, ii] = np.moveaxis(o["pos"], 0, 1)
    ref = orc.backward(ffw, win, c["atoms"], c["probe"], s, c["tip"], c["df"], pos, w)
    n = len(c["atoms"]["x"])
    g = {k: torch.empty(n, device="cuda") for k in KEYS}
    g["tip"] = torch.empty(5, device="cuda")
    ws = torch.empty(pp.pp_backward_workspace(sim.grid) // 4 + 1, device="cuda")
    pp.pp_backward(pp.make_atoms(at), sim.probe, sim.grid, sim.ff, sim.scan, sim.tip, sim.dfp,
                   torch.as_tensor(pos, dtype=torch.float32, device="cuda"),
                   torch.as_tensor(w, dtype=torch.float32, device="cuda"), pp.make_grads(g), ws)
    torch.cuda.synchronize()
    for k in KEYS:
        a, b = g[k].cpu().numpy().astype(np.float64), ref[k]
        assert np.linalg.norm(a - b) <= 1e-4 * max(np.linalg.norm(b), 1e-30), k
    t = g["tip"].cpu().numpy()
    for i, k in enumerate(("kx", "ky", "kR", "Q")):
        assert abs(t[i] - ref[k]) <= 1e-4 * max(abs(ref[k]), 1e-30), k
