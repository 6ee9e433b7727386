"""GPU parity of the implicit adjoint (K3^T, K4, K5) against the FP64 oracle adjoint.

The oracle adjoint is pinned to central finite differences of the oracle's
forward pass (tests/test_oracle_adjoint.py).  Bars:
  - isolated: the CUDA adjoint evaluated at the oracle's relaxed positions
    agrees with the oracle to relative L2 <= 1e-4 per gradient vector;
  - end to end (each side relaxes on its own grid, ftol 1e-6 eV/A; 2e-7 on the
    40-atom workload): relative L2 <= 1e-3 per gradient vector (atom x, y, z,
    q, R, eps; tip kx, ky, kR, Q).
"""
import copy

import numpy as np
import pytest
import torch

from helpers import case32, df_keep
from paper_2401_14564_gb300 import afm, autograd, pp, synth

pytestmark = pytest.mark.gpu

KEYS = ("x", "y", "z", "q", "R", "eps")
TIP = ("kx", "ky", "kR", "Q")


def weights(c, seed=7):
    s = c["scan"]
    m = pp.pp_df_margin(c["df"]["A_pp"], s["dz"])
    return np.random.default_rng(seed).standard_normal((s["nz"] - 2 * m, s["ny"], s["nx"]))


def gpu_backward(c, pos, w, layout=0, want_qzz=False, want_grid_adj=False, ff_host=None):
    """CUDA adjoint at the given relaxed positions, on the CUDA FF grid, or on ff_host (a grid the
    oracle made, rounded to FP32) when given; dL/dQzz too if want_qzz; on an energy grid the node
    adjoint dL/dE_g [nz][ny][nx] from the workspace if want_grid_adj."""
    grid = pp.make_grid(c["grid"], layout)
    atoms_t = afm.atoms_to_device(c["atoms"])
    atoms = pp.make_atoms(atoms_t)
    if ff_host is None:
        ff = torch.empty(pp.pp_ff_floats(grid), dtype=torch.float32, device="cuda")
        pp.pp_make_ff(atoms, pp.make_probe(c["probe"]), grid, ff)
    else:
        assert layout == 0 and np.asarray(ff_host).size == pp.pp_ff_floats(grid)
        ff = torch.as_tensor(np.ascontiguousarray(ff_host, dtype=np.float32).ravel(), device="cuda")
    n = len(c["atoms"]["x"])
    g = {k: torch.full((n,), float("nan"), device="cuda") for k in KEYS}
    g["tip"] = torch.full((5,), float("nan"), device="cuda")
    ws = torch.empty(pp.pp_backward_workspace(grid) // 4 + 1, dtype=torch.float32, device="cuda")
    pos_t = torch.as_tensor(np.asarray(pos, dtype=np.float32), device="cuda").contiguous()
    w_t = torch.as_tensor(np.asarray(w, dtype=np.float32), device="cuda").contiguous()
    pp.pp_backward(atoms, pp.make_probe(c["probe"]), grid, ff, pp.make_scan(c["scan"]), pp.make_tip(c["tip"]),
                   pp.make_df(c["df"]), pos_t, w_t, pp.make_grads(g), ws)
    torch.cuda.synchronize()
    out = {k: g[k].cpu().numpy().astype(np.float64) for k in KEYS}
    t = g["tip"].cpu().numpy().astype(np.float64)
    out.update({k: t[i] for i, k in enumerate(TIP)})
    if want_qzz:
        out["Qzz"] = t[4]
    if want_grid_adj:
        assert c["grid"].get("interp", 0) == 1
        gg = c["grid"]
        nn = gg["nx"] * gg["ny"] * gg["nz"]
        out["grid_adj"] = ws[64:64 + nn].cpu().numpy().astype(np.float64).reshape(gg["nz"], gg["ny"], gg["nx"])
    return out


def rel(a, b):
    a, b = np.atleast_1d(a), np.atleast_1d(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def check(got, ref, tol, tip_tol=None):
    errs = {k: rel(got[k], ref[k]) for k in KEYS + TIP}
    lim = {k: (tip_tol if (tip_tol is not None and k in TIP) else tol) for k in errs}
    bad = {k: v for k, v in errs.items() if not v <= lim[k]}
    assert not bad, (bad, errs)
    return errs


def small():
    return case32(synth.small_case(seed=9, n_atoms=8, nxy=40, nz=36, scan_px=9, nz_scan=14, d=0.15))


@pytest.mark.parametrize("layout", [0, 1])
def test_isolated_adjoint_matches_oracle(orc, layout):
    c = small()
    w = weights(c)
    o = orc.forward(c)
    ref = orc.backward(o["ff"], c["grid"], c["atoms"], c["probe"], c["scan"], c["tip"], c["df"], o["pos"], w)
    got = gpu_backward(c, o["pos"], w, layout)
    check(got, ref, 1e-4)


def test_isolated_adjoint_min_image_cutoff(orc):
    c = small()
    c["probe"] = dict(c["probe"], coul_rc=3.0, min_image=1)
    w = weights(c, 3)
    o = orc.forward(c)
    ref = orc.backward(o["ff"], c["grid"], c["atoms"], c["probe"], c["scan"], c["tip"], c["df"], o["pos"], w)
    got = gpu_backward(c, o["pos"], w)
    check(got, ref, 1e-4)


def end_to_end(orc, c, w, tol, ftol=1e-6, tip_tol=None):
    """Each side relaxes on its own grid.  As in the relaxation parity, df outputs whose
    stencil touches an ill-conditioned point (lambda_min < 0.01 eV/A^2) or a point where the
    two sides settled in different basins get zero loss weight: near a bifurcation the
    gradient is dominated by 1/lambda and by which side of the saddle FP32 rounding lands on.
    The implicit adjoint differentiates the equilibrium G(p*) = 0 (the oracle polishes FIRE's
    answer by Newton to |G| < 1e-11 eV/A), so the GPU scan here polishes its own by up to four
    Newton steps: FIRE's stopping residual alone (|G| < ftol) moves the tip-parameter sums by
    about 6e-4 relative at ftol = 2e-7 and 5e-3 at 1e-6, in the FP64 oracle itself."""
    fire = synth.parity_fire(ftol=ftol, max_iter=20000, polish=4)
    g = afm.afm(c, fire=fire)
    assert (g["iters"] < fire["max_iter"]).mean() > 0.999
    o = orc.forward(c, fire=dict(fire, polish=0))
    keep = (o["lam"] >= 0.01) & (np.linalg.norm(g["pos"] - o["pos"], axis=-1) < 0.05)
    m = (keep.shape[0] - np.asarray(w).shape[0]) // 2
    w = np.where(df_keep(keep, m), w, 0.0)
    assert (w != 0).mean() > 0.8
    got = gpu_backward(c, g["pos"], w)
    ref = orc.backward(o["ff"], c["grid"], c["atoms"], c["probe"], c["scan"], c["tip"], c["df"], o["pos"], w)
    return check(got, ref, tol, tip_tol)


def test_end_to_end_small(orc):
    c = small()
    end_to_end(orc, c, weights(c), 1e-3)


def test_gradient_workload_end_to_end(orc):
    # 40-atom nonplanar molecule, 128 x 128 px x 20 heights, loss sum(w * df), w ~ N(0,1) seed 7;
    # every gradient vector, the tip scalars included, to relative L2 1e-3
    c = case32(synth.gradient_case())
    end_to_end(orc, c, c["w"], 1e-3, ftol=2e-7)


def test_charge_scaling_identity_on_gpu(orc):
    c = small()
    o = orc.forward(c)
    got = gpu_backward(c, o["pos"], weights(c))
    lhs = float((c["atoms"]["q"] * got["q"]).sum())
    assert lhs == pytest.approx(c["probe"]["Q"] * got["Q"], rel=1e-4)


def test_autograd_function_matches_direct_call(orc):
    c = small()
    fire = synth.parity_fire()
    at = afm.atoms_to_device(c["atoms"])
    leaves = {k: at[k].clone().requires_grad_(True) for k in KEYS}
    tips = {k: torch.tensor(float(c["tip"][k] if k != "Q" else c["probe"]["Q"]), requires_grad=True) for k in TIP}
    df = autograd.afm_df(leaves, tips["kx"], tips["ky"], tips["kR"], tips["Q"], c, fire=fire)
    w = weights(c)
    loss = (df * torch.as_tensor(w, dtype=torch.float32, device="cuda")).sum()
    loss.backward()
    g = afm.afm(c, fire=fire)
    direct = gpu_backward(c, g["pos"], w)
    # the two runs differ only in the order of FP32 atomic additions (and dL/dQ = sum q_i C_i
    # cancels across a neutral molecule), hence 1e-4 rather than bit equality
    for k in KEYS:
        assert rel(leaves[k].grad.cpu().numpy(), direct[k]) < 1e-4, k
    for k in TIP:
        assert rel(tips[k].grad.item(), direct[k]) < 1e-4, k


def test_autograd_positions_and_fz_are_not_differentiable():
    # only the df image carries the adjoint; a loss on the relaxed positions or on Fz must fail
    # loudly instead of receiving the df gradient's terms alone
    c = small()
    at = afm.atoms_to_device(c["atoms"])
    leaves = {k: at[k].clone().requires_grad_(True) for k in KEYS}
    tips = [torch.tensor(float(v), requires_grad=True) for v in
            (c["tip"]["kx"], c["tip"]["ky"], c["tip"]["kR"], c["probe"]["Q"], 0.0)]
    df, fz, pos = autograd.PPFunction.apply(*[leaves[k] for k in KEYS], *tips, c, 0, None)
    assert df.requires_grad and not fz.requires_grad and not pos.requires_grad
    with pytest.raises(RuntimeError):
        pos.sum().backward()
    df.sum().backward()
    assert all(torch.isfinite(leaves[k].grad).all() for k in KEYS)


def test_workspace_too_small_is_rejected():
    c = small()
    grid = pp.make_grid(c["grid"])
    need = pp.pp_backward_workspace(grid)
    ws = torch.empty(need // 4 - 4, dtype=torch.float32, device="cuda")
    n = len(c["atoms"]["x"])
    g = {k: torch.empty(n, device="cuda") for k in KEYS}
    g["tip"] = torch.empty(5, device="cuda")
    at = afm.atoms_to_device(c["atoms"])
    ff = torch.zeros(pp.pp_ff_floats(grid), device="cuda")
    s = c["scan"]
    pos = torch.zeros((s["nz"], s["ny"], s["nx"], 3), device="cuda")
    w = torch.zeros((s["nz"] - 10, s["ny"], s["nx"]), device="cuda")
    with pytest.raises(pp.PPError) as e:
        pp.pp_backward(pp.make_atoms(at), pp.make_probe(c["probe"]), grid, ff, pp.make_scan(s), pp.make_tip(c["tip"]),
                       pp.make_df(c["df"]), pos, w, pp.make_grads(g), ws)
    assert e.value.status == 4


def test_isolated_adjoint_asymmetric_tip_clamped_grid(orc):
    c = small()
    c["tip"] = synth.default_tip(kx=0.35, ky=0.28, d0x=0.35, d0y=-0.25)
    c["grid"] = dict(c["grid"], periodic_xy=0)
    c = case32(c)
    w = weights(c, 5)
    o = orc.forward(c)
    ref = orc.backward(o["ff"], c["grid"], c["atoms"], c["probe"], c["scan"], c["tip"], c["df"], o["pos"], w)
    got = gpu_backward(c, o["pos"], w)
    # dL/dkx = sum lambda_x e_x: with a tilted rest position e_x = d_x - d0x is a small difference of
    # ~0.35 A coordinates formed in FP32 (anchor included), and the sum over points cancels, so the
    # tip scalars are held to 1e-3 here; the atom gradients keep 1e-4
    check(got, ref, 1e-4, tip_tol=1e-3)
