"""GPU parity of the tip-quadrupole term (Secs. 2.2.3, 2.2.5: the CO tip's
quadrupolar charge distribution; -0.05 e*A^2 in the paper's point-charge
simulations) against the FP64 oracle, whose quadrupole is pinned to the
three-point-charge limit and closed forms (tests/test_oracle_quad.py).

Same bars as without it: FF nodes to 1e-4 relative outside the core, relaxed
positions to 1e-3 A and df to 1e-3 of the image range, the adjoint at the
oracle's positions to 1e-4 relative L2 per gradient vector (dL/dQzz
included), the batch bit-identical to the single-molecule path.
"""
import copy

import numpy as np
import pytest
import torch

from helpers import case32, ff_rel_err, linear_ff
from paper_2401_14564_gb300 import afm, autograd, batch, pp, synth
from test_gpu_backward import KEYS, gpu_backward, rel, weights
from test_gpu_relax import check_parity

pytestmark = pytest.mark.gpu

TIPQ = ("kx", "ky", "kR", "Q", "Qzz")


def with_quad(c, Qzz=-0.05, **probe):
    c = copy.deepcopy(c)
    c["probe"] = dict(c["probe"], Qzz=Qzz, **probe)
    return c


def gpu_ff(c):
    grid = pp.make_grid(c["grid"], 0)
    ff = torch.full((pp.pp_ff_floats(grid),), float("nan"), dtype=torch.float32, device="cuda")
    pp.pp_make_ff(pp.make_atoms(afm.atoms_to_device(c["atoms"])), pp.make_probe(c["probe"]), grid, ff)
    torch.cuda.synchronize()
    return linear_ff(ff.cpu().numpy(), c["grid"])


def check_ff(orc, c, zpt=None):
    c = case32(c)
    F = gpu_ff(c)
    ref, core = orc.make_ff(c["atoms"], c["probe"], c["grid"])
    err = ff_rel_err(F, ref)[~core]
    eerr = (np.abs(F[..., 3] - ref[..., 3]) / np.maximum(np.abs(ref[..., 3]), 1e-2))[~core]
    assert np.isfinite(F).all()
    assert err.max() <= 1e-4, err.max()
    assert eerr.max() <= 1e-4, eerr.max()
    # the term is not negligible on this grid (the comparison has teeth)
    ref0, _ = orc.make_ff(c["atoms"], dict(c["probe"], Qzz=0.0), c["grid"])
    assert ff_rel_err(ref0, ref)[~core].max() > 1e-2


def test_ff_parity_with_quadrupole(orc):
    check_ff(orc, with_quad(synth.small_case(seed=3, n_atoms=12, nxy=32, nz=37), Qzz=-0.1))


def test_ff_parity_with_quadrupole_min_image_cutoff(orc):
    c = synth.small_case(seed=5, n_atoms=20, nxy=24, nz=17)
    c["grid"]["periodic_xy"] = 1
    check_ff(orc, with_quad(c, Qzz=-0.15, coul_rc=3.0, min_image=1))


def test_ff_quadrupole_every_z_blocking(orc):
    c = case32(with_quad(synth.small_case(seed=4, n_atoms=10, nxy=24, nz=29)))
    grid = pp.make_grid(c["grid"], 0)
    atoms = pp.make_atoms(afm.atoms_to_device(c["atoms"]))
    outs = []
    for z in (4, 8, 16):
        ff = torch.full((pp.pp_ff_floats(grid),), float("nan"), dtype=torch.float32, device="cuda")
        pp.pp_make_ff_tuned(atoms, pp.make_probe(c["probe"]), grid, ff, pp.Tuning(z))
        outs.append(ff.cpu().numpy())
    # the z-blocking changes which thread computes a node, not its arithmetic
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[1], outs[2])


def test_relax_parity_with_quadrupole(orc):
    check_parity(orc, with_quad(synth.benzene_case(), Qzz=-0.1))


def test_batch_with_quadrupole_matches_single_path_bit_for_bit():
    cs = [case32(with_quad(c)) for c in synth.batch_cases(5, 3000)]
    b = batch.Batch(cs)
    b.run()
    st, flags = b.status()
    assert st == 0 and flags == 0
    for n, c in enumerate(cs):
        got = {k: v.cpu().numpy() for k, v in b.molecule(n).items()}
        sim = afm.Simulator(c)
        sim.run(afm.atoms_to_device(c["atoms"]))
        torch.cuda.synchronize()
        assert np.array_equal(got["df"], sim.df.cpu().numpy()), n
        assert np.array_equal(got["fz"], sim.fz.cpu().numpy()), n


def small_quad(**probe):
    c = synth.small_case(seed=9, n_atoms=8, nxy=40, nz=36, scan_px=9, nz_scan=14, d=0.15)
    return case32(with_quad(c, Qzz=-0.1, **probe))


def isolated(orc, c, w):
    o = orc.forward(c)
    ref = orc.backward(o["ff"], c["grid"], c["atoms"], c["probe"], c["scan"], c["tip"], c["df"], o["pos"], w)
    got = gpu_backward(c, o["pos"], w, want_qzz=True)
    errs = {k: rel(got[k], ref[k]) for k in KEYS + TIPQ}
    assert abs(ref["Qzz"]) > 0.0
    bad = {k: v for k, v in errs.items() if not v <= 1e-4}
    assert not bad, (bad, errs)
    return got, ref


def test_isolated_adjoint_with_quadrupole(orc):
    c = small_quad()
    isolated(orc, c, weights(c))


def test_isolated_adjoint_with_quadrupole_min_image_cutoff(orc):
    # the probe stays 3.7-5 A above the atoms: a 6 A cutoff keeps the term inside the scanned slab
    c = small_quad(coul_rc=6.0, min_image=1)
    isolated(orc, c, weights(c, 3))


def test_charge_identity_with_quadrupole_on_gpu(orc):
    c = small_quad()
    o = orc.forward(c)
    got = gpu_backward(c, o["pos"], weights(c), want_qzz=True)
    lhs = float((c["atoms"]["q"] * got["q"]).sum())
    rhs = c["probe"]["Q"] * got["Q"] + c["probe"]["Qzz"] * got["Qzz"]
    assert lhs == pytest.approx(rhs, rel=1e-4)


def test_autograd_quadrupole_gradient_matches_direct_call(orc):
    c = small_quad()
    fire = synth.parity_fire()
    at = afm.atoms_to_device(c["atoms"])
    leaves = {k: at[k].clone().requires_grad_(True) for k in KEYS}
    tips = {k: torch.tensor(float(c["tip"][k]), requires_grad=True) for k in ("kx", "ky", "kR")}
    Q = torch.tensor(float(c["probe"]["Q"]), requires_grad=True)
    Qzz = torch.tensor(float(c["probe"]["Qzz"]), requires_grad=True)
    df = autograd.afm_df(leaves, tips["kx"], tips["ky"], tips["kR"], Q, c, fire=fire, Qzz=Qzz)
    w = weights(c)
    (df * torch.as_tensor(w, dtype=torch.float32, device="cuda")).sum().backward()
    g = afm.afm(c, fire=fire)
    direct = gpu_backward(c, g["pos"], w, want_qzz=True)
    assert Qzz.grad is not None and Qzz.grad.item() != 0.0
    # the runs differ only in the order of FP32 atomic additions
    assert rel(Qzz.grad.item(), direct["Qzz"]) < 1e-4
    assert rel(Q.grad.item(), direct["Q"]) < 1e-4
    for k in KEYS:
        assert rel(leaves[k].grad.cpu().numpy(), direct[k]) < 1e-4, k
