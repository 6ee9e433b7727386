"""GPU parity of the tricubic path (grid interp = 1: energy-only K1 variant,
K2 with F = -grad of the tricubic energy interpolant) against the FP64 oracle,
whose tricubic interpolant is pinned in tests/test_oracle_tricubic.py.

Bars as for the trilinear path: node energies to 1e-4 relative (1e-2 eV
floor) outside the core, relaxed positions to 1e-3 A and df to 1e-3 of the
image range on well-conditioned points in the same basin; the adjoint on an
energy grid to relative L2 1e-4 per gradient vector at the oracle's relaxed
positions and 1e-3 end to end, as on force grids.
"""
import copy

import numpy as np
import pytest
import torch

from helpers import case32, df_keep, ill_conditioned_within_bound
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


# Bars of the energy-grid adjoint.  J holds minus the Hessian of the tricubic interpolant, formed
# in FP32 from node energies that are themselves FP32 sums of ~eV pair terms: a node error dE
# reaches J as dE * sum|w''| / dx^2 (about 400 dE per A^2 at dx = 0.15 A), and lambda = J^-T r
# carries it at 1 / lambda_min (lambda_min down to 0.013 eV/A^2 here).  The atom gradient vectors
# keep 1e-4.  The tip scalars sum lambda-weighted terms over every point and so pick up the least
# stable points in full: on the oracle's own grid (rounded to FP32, so only the adjoint kernels'
# arithmetic differs) they hold 5e-4 (measured <= 2.1e-4); on the GPU's grid, whose energies add
# K1's rounding, and end to end (each side's relaxed positions, the GPU's Newton-polished to the
# equilibrium the adjoint differentiates) the gradient bar of 1e-3 (measured <= 6.2e-4 on the
# GPU's grid).
TIP_ORACLE_GRID, TIP_OWN_GRID, TIP_E2E = 5e-4, 1e-3, 1e-3


@pytest.mark.parametrize("probe", [{}, dict(Qzz=-0.1), dict(coul_rc=3.0, min_image=1, Qzz=-0.1)])
def test_energy_grid_adjoint_kernels_on_the_oracle_grid(orc, probe):
    from test_gpu_backward import check, gpu_backward, rel, small, weights

    c = tc(small())
    c["probe"] = dict(c["probe"], **probe)
    c = case32(c)
    w = weights(c)
    o = orc.forward(c)
    ref = orc.backward(o["ff"], c["grid"], c["atoms"], c["probe"], c["scan"], c["tip"], c["df"], o["pos"], w,
                       want_grid_adj=True)
    got = gpu_backward(c, o["pos"], w, want_qzz=True, want_grid_adj=True, ff_host=o["ff"][..., 3])
    check(got, ref, 1e-4, tip_tol=TIP_ORACLE_GRID)
    if c["probe"]["Qzz"] != 0.0:
        assert got["Qzz"] == pytest.approx(ref["Qzz"], rel=TIP_ORACLE_GRID)
    # the node adjoint itself (K4's scatter over the 64-node stencils)
    assert rel(got["grid_adj"].ravel(), ref["grid_adj"].ravel()) <= 1e-4


@pytest.mark.parametrize("probe", [{}, dict(Qzz=-0.1), dict(coul_rc=3.0, min_image=1, Qzz=-0.1), dict(coul_rc=3.0)])
def test_isolated_energy_grid_adjoint_matches_oracle(orc, probe):
    from test_gpu_backward import check, gpu_backward, rel, small, weights

    c = tc(small())
    c["probe"] = dict(c["probe"], **probe)
    c = case32(c)
    w = weights(c, 3)
    o = orc.forward(c)
    ref = orc.backward(o["ff"], c["grid"], c["atoms"], c["probe"], c["scan"], c["tip"], c["df"], o["pos"], w,
                       want_grid_adj=True)
    got = gpu_backward(c, o["pos"], w, want_qzz=True, want_grid_adj=True)
    check(got, ref, 1e-4, tip_tol=TIP_OWN_GRID)
    if c["probe"]["Qzz"] != 0.0:
        assert got["Qzz"] == pytest.approx(ref["Qzz"], rel=TIP_OWN_GRID)
    assert rel(got["grid_adj"].ravel(), ref["grid_adj"].ravel()) <= 1e-4
    # the charge terms are linear in q_i Q and q_i Qzz
    lhs = float((c["atoms"]["q"] * got["q"]).sum())
    assert lhs == pytest.approx(c["probe"]["Q"] * got["Q"] + c["probe"]["Qzz"] * got["Qzz"], rel=1e-4)


def test_energy_grid_adjoint_end_to_end(orc):
    from test_gpu_backward import end_to_end, small, weights

    c = tc(small())
    end_to_end(orc, c, weights(c), 1e-3, tip_tol=TIP_E2E)


def test_energy_grid_autograd_matches_direct_call(orc):
    from paper_2401_14564_gb300 import autograd
    from test_gpu_backward import KEYS, gpu_backward, rel, small, weights

    c = tc(small())
    fire = synth.parity_fire()
    at = afm.atoms_to_device(c["atoms"])
    leaves = {k: at[k].clone().requires_grad_(True) for k in KEYS}
    t = {k: torch.tensor(float(c["tip"][k]), requires_grad=True) for k in ("kx", "ky", "kR")}
    Q = torch.tensor(float(c["probe"]["Q"]), requires_grad=True)
    df = autograd.afm_df(leaves, t["kx"], t["ky"], t["kR"], Q, c, fire=fire)
    w = weights(c)
    (df * torch.as_tensor(w, dtype=torch.float32, device="cuda")).sum().backward()
    direct = gpu_backward(c, afm.afm(c, fire=fire)["pos"], w)
    for k in KEYS:
        assert rel(leaves[k].grad.cpu().numpy(), direct[k]) < 1e-4, k


@pytest.mark.parametrize("h", [0.1, 0.2])
def test_flake_full_size_sampled_columns_on_energy_grids(orc, h):
    # the bench's tricubic leg: flake60 on energy grids at 0.1 A (256x256x200) and 0.2 A
    # (128x128x100), the 256 x 256 x 40 scan in its launch shape; 48 seeded columns against the
    # oracle relaxing on its own energy grid, 2000 sampled node energies against direct sums
    c = case32(synth.flake_case())
    g0 = c["grid"]
    f = round(h / g0["dx"])
    c["grid"] = dict(g0, nx=g0["nx"] // f, ny=g0["ny"] // f, nz=(g0["nz"] - 1) // f + 1, dx=h, dy=h, dz=h, interp=1)
    gr, s = c["grid"], c["scan"]
    fire = synth.parity_fire()
    g = gpu_run(c, fire)
    E = gpu_grid(c, 1).reshape(gr["nz"], gr["ny"], gr["nx"]).astype(np.float64)
    rng = np.random.default_rng(2)
    idx = np.stack([rng.integers(0, gr[n], 2000) for n in ("nz", "ny", "nx")], axis=1)
    pts = np.stack([np.float32(gr["x0"]) + idx[:, 2] * np.float32(gr["dx"]),
                    np.float32(gr["y0"]) + idx[:, 1] * np.float32(gr["dy"]),
                    np.float32(gr["z0"]) + idx[:, 0] * np.float32(gr["dz"])], axis=1).astype(np.float64)
    ref, core = orc.ff_points(c["atoms"], c["probe"], gr, pts)
    got = E[idx[:, 0], idx[:, 1], idx[:, 2]]
    assert (np.abs(got - ref[:, 3]) / np.maximum(np.abs(ref[:, 3]), 1e-2))[~core].max() <= 1e-4
    cols = np.sort(rng.choice(s["nx"] * s["ny"], 48, replace=False))
    ff, _ = orc.make_ff(c["atoms"], c["probe"], gr)
    o = orc.relax_columns(ff, gr, None, None, s, c["tip"], fire, cols)
    jj, ii = cols // s["nx"], cols % s["nx"]
    gp = np.moveaxis(g["pos"][:, jj, ii], 0, 1)
    gfz = g["fz"][:, jj, ii].T
    dp = np.linalg.norm(gp - o["pos"], axis=-1)
    keep = (o["lam"] >= 0.01) & (dp < 0.05)
    assert keep.mean() > 0.9
    assert dp[keep].max() <= 1e-3
    n_sel, n_ok = ill_conditioned_within_bound(gp, o, fire["ftol"])
    assert n_ok == n_sel, (n_ok, n_sel)
    assert np.abs(gfz - o["fz"])[keep].max() <= 1e-3 * np.abs(o["fz"]).max()
    odf = orc.fz_to_df(o["fz"].T, s["dz"], c["df"])
    kd = df_keep(keep.T, 5)
    assert np.abs(g["df"][:, jj, ii] - odf)[kd].max() <= 1e-3 * (g["df"].max() - g["df"].min())
