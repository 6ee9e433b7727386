"""GPU parity of K2 (relaxed FIRE scan, trilinear lookup, fused df) against the FP64 oracle.

The GPU relaxes on its own FP32 grid from K1, the oracle on its FP64 grid.
Bars (parity FIRE settings, ftol = 1e-5 eV/A, 2000 iterations):
  relaxed PP positions <= 1e-3 A, df <= 1e-3 of the image's range,
on pixels whose oracle stiffness is well conditioned (smallest eigenvalue of
the symmetrised -J >= 0.01 eV/A^2) and that reached the same basin (|dp| <
0.05 A); the excluded counts are bounded.  With the timed settings (ftol =
1e-4) positions must stay inside the residual bound ftol/lambda_min.
"""
import copy

import numpy as np
import pytest
import torch

from helpers import case32, df_keep, ill_conditioned_within_bound, relax_compare
from paper_2401_14564_gb300 import afm, pp, synth

pytestmark = pytest.mark.gpu


def gpu_run(c, fire=None, layout=0, fused=True):
    out = afm.afm(c, fire=fire, layout=layout) if fused else None
    if not fused:
        sim = afm.Simulator(c, layout=layout, fire=fire, fused_df=False)
        sim.run(afm.atoms_to_device(c["atoms"]))
        torch.cuda.synchronize()
        out = {"df": sim.df.cpu().numpy(), "fz": sim.fz.cpu().numpy(), "pos": sim.pos.cpu().numpy(),
               "iters": sim.iters.cpu().numpy()}
    return out


def check_parity(orc, case, max_excluded_frac=0.02, fire=None):
    c = case32(case)
    fire = fire or synth.parity_fire()
    g = gpu_run(c, fire)
    o = orc.forward(c, fire=fire)
    assert o["ok"].all()
    assert np.isfinite(g["pos"]).all() and np.isfinite(g["df"]).all()
    assert (g["iters"] < fire["max_iter"]).mean() > 0.999
    dp, dfz, keep, n_ill, n_basin = relax_compare(g, o)
    assert (n_ill + n_basin) <= max_excluded_frac * keep.size, (n_ill, n_basin)
    assert dp <= 1e-3, dp
    n_sel, n_ok = ill_conditioned_within_bound(g["pos"], o, fire["ftol"])
    assert n_ok == n_sel, (n_ok, n_sel)
    m = (keep.shape[0] - g["df"].shape[0]) // 2
    kd = df_keep(keep, m)
    rng = o["df"].max() - o["df"].min()
    ddf = np.abs(g["df"] - o["df"])[kd].max()
    assert ddf <= 1e-3 * rng, (ddf, rng)
    return g, o, keep


def test_benzene_parity(orc):
    check_parity(orc, synth.benzene_case())


def test_small_ragged_scan_parity(orc):
    # 12 x 15 pixels: ragged against the 16 x 8 pixel CTA tile; 12 heights
    check_parity(orc, synth.small_case(seed=3, n_atoms=12, nxy=32, nz=40, scan_px=12, nz_scan=12))


def test_bricked_grid_same_images(orc):
    c = case32(synth.small_case(seed=6, n_atoms=14, nxy=40, nz=40, scan_px=16, nz_scan=14))
    a = gpu_run(c, synth.parity_fire(), layout=0)
    b = gpu_run(c, synth.parity_fire(), layout=1)
    # identical node values and identical arithmetic: bit-identical scans
    assert np.array_equal(a["pos"], b["pos"]) and np.array_equal(a["df"], b["df"])


@pytest.mark.parametrize("A", [1.0, 0.19, 0.79, 1.59, 1.79])
def test_fused_df_equals_standalone_kernel(A):
    # the standalone kernel (register window for half-widths 1..8, generic beyond) sums the taps in
    # the fused epilogue's order: bit-identical images for m = 5, 1, 4, 8, 9
    c = copy.deepcopy(synth.benzene_case())
    c["df"] = dict(c["df"], A_pp=A)
    c = case32(c)
    a = gpu_run(c, fused=True)
    b = gpu_run(c, fused=False)
    assert np.array_equal(a["fz"], b["fz"])
    assert np.array_equal(a["df"], b["df"])


def test_bench_settings_within_residual_bound(orc):
    c = case32(synth.benzene_case())
    g = gpu_run(c)  # ftol = 1e-4 eV/A, 200 iterations
    o = orc.forward(c)
    conv = g["iters"] < c["fire"]["max_iter"]
    dp = np.linalg.norm(g["pos"] - o["pos"], axis=-1)
    bound = c["fire"]["ftol"] / np.maximum(o["lam"], 1e-12) + 2e-4
    ok = (dp <= bound) | ~conv | (dp > 0.05)
    assert ok.mean() > 0.999
    assert conv.mean() > 0.99


def test_empty_sample_and_constant_field(orc):
    c = case32(synth.small_case(seed=2, n_atoms=5, nxy=16, nz=12, scan_px=7, nz_scan=11))
    g = c["grid"]
    grid = pp.make_grid(g, 0)
    for const, kR in (((0.0, 0.0, 0.0), 20.0), ((0.004, -0.003, -0.03), 20.0), ((-0.002, 0.001, -0.08), 20.0),
                      ((0.001, 0.002, -0.05), 1e4), ((0.0, 0.0, 0.04), 1e4)):
        # (a repulsive c_z above kx * R0 = 0.0624 eV/A would buckle the tip: s = c_z/d_z < -kx)
        c["tip"] = synth.default_tip(kR=kR)
        ff = torch.zeros(pp.pp_ff_floats(grid), dtype=torch.float32, device="cuda").view(-1, 4)
        ff[:, 0], ff[:, 1], ff[:, 2] = const
        s = c["scan"]
        nz, ny, nx = s["nz"], s["ny"], s["nx"]
        pos = torch.empty((nz, ny, nx, 3), device="cuda")
        fz = torch.empty((nz, ny, nx), device="cuda")
        it = torch.empty((nz, ny, nx), dtype=torch.int32, device="cuda")
        # a 1e4 N/m radial spring against 0.03 eV/A^2 of lateral stiffness needs many FIRE steps
        # (and a FIRE step that respects it: omega = sqrt(624 eV/A^2) = 25 -> dt = 0.04)
        fire = synth.parity_fire(max_iter=50000, dt0=0.04, dt_max=0.04) if kR > 100 else synth.parity_fire()
        pp.pp_relax_scan(ff.view(-1), grid, pp.make_scan(s), pp.make_tip(c["tip"]), pp.make_fire(fire), pos, fz, it)
        torch.cuda.synchronize()
        ref_ff = np.zeros((g["nz"], g["ny"], g["nx"], 4))
        ref_ff[..., 0], ref_ff[..., 1], ref_ff[..., 2] = [np.float32(v) for v in const]
        o = orc.relax_scan(ref_ff, g, None, None, s, c["tip"], fire)
        assert (it.cpu().numpy() < fire["max_iter"]).all()
        assert np.abs(pos.cpu().numpy() - o["pos"]).max() < 1e-3
        # Fz balances the constant sample force: FIRE leaves |G| < ftol = 1e-5
        assert np.abs(fz.cpu().numpy() - np.float32(const[2])).max() < 1.1e-5
        if const == (0.0, 0.0, 0.0):
            # at rest the deflection is exactly zero: no iteration, Fz exactly 0
            assert (it.cpu().numpy() == 0).all()
            assert np.abs(fz.cpu().numpy()).max() == 0.0


def test_stiff_springs_give_unrelaxed_lookup(orc):
    # kR = kx = ky = 1e4 N/m = 624 eV/A^2.  The kernel's FIRE state is the deflection from the
    # rest displacement, so the spring extension (~1e-4 A here) keeps full FP32 relative
    # precision and Fz is not quantised by ulp(R0).
    c = case32(synth.benzene_case())
    c["tip"] = synth.default_tip(kx=1e4, ky=1e4, kR=1e4)
    fire = synth.parity_fire(max_iter=20000, dt0=0.04, dt_max=0.04)  # dt ~ 1/omega of the stiff spring
    g = gpu_run(c, fire)
    o = orc.forward(c, fire=fire)
    rng = np.abs(o["fz"]).max()
    assert np.abs(g["fz"] - o["fz"]).max() <= 1e-3 * rng
    # and the oracle's relaxed image is the unrelaxed lookup within O(|F|/k)
    s = c["scan"]
    k = np.arange(s["nz"])[:, None, None]
    j = np.arange(s["ny"])[None, :, None]
    i = np.arange(s["nx"])[None, None, :]
    pts = np.stack(np.broadcast_arrays(s["x0"] + i * s["px"], s["y0"] + j * s["py"],
                                       s["z_top"] - k * s["dz"] - c["tip"]["R0"]), axis=-1)
    assert np.abs(g["pos"] - pts).max() < 1e-3


def test_flake_full_size_sampled_columns(orc):
    # the benchmark's 256 x 256 x 200 grid and 256 x 256 x 40 scan (same launch shapes), parity FIRE
    c = case32(synth.flake_case())
    fire = synth.parity_fire()
    g = gpu_run(c, fire)
    s, gr = c["scan"], c["grid"]
    rng = np.random.default_rng(1)
    cols = np.sort(rng.choice(s["nx"] * s["ny"], 48, replace=False))
    # PPs at the lowest heights can swing past the anchor (weak lateral springs deep in the
    # repulsive wall; the FP64 oracle does the same), so the oracle uses the whole grid
    slab = gr
    ff, core = orc.make_ff(c["atoms"], c["probe"], slab)
    o = orc.relax_columns(ff, slab, None, None, s, c["tip"], fire, cols)
    jj, ii = cols // s["nx"], cols % s["nx"]
    gp = np.moveaxis(g["pos"][:, jj, ii], 0, 1)
    gfz = g["fz"][:, jj, ii].T
    dp = np.linalg.norm(gp - o["pos"], axis=-1)
    keep = (o["lam"] >= 0.01) & (dp < 0.05)
    # about 5% of this workload's entries have lambda_min just under 0.01 eV/A^2 in the FP64
    # oracle itself (far-field pixels where the vdW curvature eats into the 0.0156 eV/A^2
    # lateral spring); those are held to their residual bound instead.  Well-conditioned entries
    # that settled in another basin are capped on their own
    assert keep.mean() > 0.9
    other_basin = (o["lam"] >= 0.01) & (dp >= 0.05)
    assert other_basin.mean() <= 0.005, other_basin.sum()
    assert dp[keep].max() <= 1e-3
    n_sel, n_ok = ill_conditioned_within_bound(gp, o, fire["ftol"])
    assert n_ok == n_sel, (n_ok, n_sel)
    fzr = np.abs(o["fz"]).max()
    assert np.abs(gfz - o["fz"])[keep].max() <= 1e-3 * fzr
    odf = orc.fz_to_df(o["fz"].T, s["dz"], c["df"])
    gdf = g["df"][:, jj, ii]
    kd = df_keep(keep.T, 5)
    assert np.abs(gdf - odf)[kd].max() <= 1e-3 * (g["df"].max() - g["df"].min())


def test_asymmetric_tip_on_a_clamped_grid_parity(orc):
    # a tilted rest displacement (d0x, d0y != 0), unequal lateral springs, and a grid that clamps
    # instead of wrapping laterally
    c = synth.small_case(seed=8, n_atoms=10, nxy=36, nz=40, scan_px=11, nz_scan=13)
    # (springs stiff enough that the lateral stiffness at rest, 0.022 / 0.017 eV/A^2, stays above
    # the 0.01 eV/A^2 conditioning cut of the comparison)
    c["tip"] = synth.default_tip(kx=0.35, ky=0.28, d0x=0.35, d0y=-0.25)
    c["grid"] = dict(c["grid"], periodic_xy=0)
    check_parity(orc, c)


def test_benzene_mirror_symmetry_on_the_gpu(orc):
    # benzene is symmetric under x -> -x and y -> -y; the periodic 80 x 80 grid from -8 A at 0.2 A
    # maps node i to node (80 - i) mod 80, and the 40 x 40 scan from -5.85 A at 0.3 A maps pixel i
    # to 39 - i.  The GPU's force field and image keep the symmetry to FP32 rounding (the oracle's
    # FP64 grid keeps it to 1e-12, tests/test_oracle_ff.py)
    c = case32(synth.benzene_case())
    g = gpu_run(c, synth.parity_fire())
    F = np.asarray(g["ff"].view(c["grid"]["nz"], c["grid"]["ny"], c["grid"]["nx"], 4).cpu().numpy(), np.float64)
    # node 0 (x = -8 A) would mirror onto x = +8 A, outside the grid (the field is summed over the
    # atoms alone, without periodic images), so the comparison runs over nodes 1..79; core nodes
    # (floored pairs, forces of hundreds of eV/A) are left out as in the parity tests
    _, core = orc.make_ff(c["atoms"], c["probe"], c["grid"])
    inner = ~core
    inner[:, 0, :] = False
    inner[:, :, 0] = False
    mx = np.roll(F[:, :, ::-1], 1, axis=2)[..., :3] * np.array([-1.0, 1.0, 1.0])  # node i -> 80 - i
    my = np.roll(F[:, ::-1, :], 1, axis=1)[..., :3] * np.array([1.0, -1.0, 1.0])  # node j -> 80 - j
    norm = np.maximum(np.linalg.norm(F[..., :3], axis=-1), 1e-3)
    assert (np.linalg.norm(mx - F[..., :3], axis=-1) / norm)[inner].max() <= 1e-4
    assert (np.linalg.norm(my - F[..., :3], axis=-1) / norm)[inner].max() <= 1e-4
    # the relaxed image: pixels mirrored into each other relax into mirrored basins (a bistable point
    # may fall either way under FP32 rounding: those are counted, not compared), and df agrees
    o = orc.forward(c, fire=synth.parity_fire())
    pos = g["pos"]
    px = pos[:, :, ::-1].copy()
    px[..., 0] = -px[..., 0]
    dpx = np.linalg.norm(px - pos, axis=-1)
    well = (o["lam"] >= 0.01) & (o["lam"][:, :, ::-1] >= 0.01)
    same = dpx < 0.05
    assert (well & ~same).mean() <= 0.01
    assert dpx[well & same].max() <= 2e-3
    keep = well & same
    kd = df_keep(keep, (keep.shape[0] - g["df"].shape[0]) // 2)
    rng = g["df"].max() - g["df"].min()
    assert np.abs(g["df"][:, :, ::-1] - g["df"])[kd].max() <= 1e-3 * rng
