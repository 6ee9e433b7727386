"""GPU parity of the IETS map (pp_iets) against the FP64 oracle.

Both evaluate the stiffness eigenvalues at the same (oracle) relaxed positions, each on its own
force-field grid.  Bar: |d lambda| <= 1e-4 eV/A^2 (the radial stiffness is 1.25 eV/A^2, the
lateral 0.0156) at all but 0.1 % of points -- a point lying within rounding of a cell face can
take the neighbouring cell's (piecewise constant) Jacobian on one side.
"""
import numpy as np
import pytest
import torch

from helpers import case32
from paper_2401_14564_gb300 import afm, pp, synth

pytestmark = pytest.mark.gpu


def gpu_iets(c, pos, mass=16.0):
    sim = afm.Simulator(c)
    sim.make_ff(afm.atoms_to_device(c["atoms"]))
    pos_t = torch.as_tensor(np.asarray(pos, dtype=np.float32), device="cuda").contiguous()
    eig = torch.empty(pos_t.shape, device="cuda")
    hw = torch.empty(pos_t.shape, device="cuda")
    pp.pp_iets(sim.ff, sim.grid, sim.scan, sim.tip, pos_t, mass, eig, hw)
    torch.cuda.synchronize()
    return eig.cpu().numpy().astype(np.float64), hw.cpu().numpy().astype(np.float64)


def test_benzene_iets_matches_oracle(orc):
    c = case32(synth.benzene_case())
    o = orc.forward(c)
    pos = o["pos"].astype(np.float32).astype(np.float64)
    ref, ref_hw = orc.iets(o["ff"], c["grid"], None, None, c["scan"], c["tip"], pos)
    got, got_hw = gpu_iets(c, pos)
    d = np.abs(got - ref).max(axis=-1)
    assert (d <= 1e-4).mean() >= 0.999, np.sort(d)[-10:]
    ok = d <= 1e-4
    # mode energies follow: relative 1e-3 where the mode is not soft
    stiff = ref > 1e-3
    rel = np.abs(got_hw - ref_hw) / np.maximum(ref_hw, 1e-12)
    assert rel[stiff & ok[..., None]].max() <= 1e-3


def test_at_rest_eigenvalues_are_the_springs(orc):
    c = case32(synth.small_case(seed=2, n_atoms=5, nxy=16, nz=12, scan_px=7, nz_scan=11))
    sim = afm.Simulator(c)
    sim.ff.zero_()
    s = c["scan"]
    k = np.arange(s["nz"])[:, None, None]
    j = np.arange(s["ny"])[None, :, None]
    i = np.arange(s["nx"])[None, None, :]
    pos = np.stack(np.broadcast_arrays(s["x0"] + i * s["px"], s["y0"] + j * s["py"],
                                       s["z_top"] - k * s["dz"] - c["tip"]["R0"]), axis=-1)
    pos_t = torch.as_tensor(pos, dtype=torch.float32, device="cuda").contiguous()
    eig = torch.empty(pos_t.shape, device="cuda")
    pp.pp_iets(sim.ff, sim.grid, sim.scan, sim.tip, pos_t, 16.0, eig)
    nm = 1.0 / 16.02176634
    want = np.sort(np.array([c["tip"]["kx"], c["tip"]["ky"], c["tip"]["kR"]]) * nm)
    np.testing.assert_allclose(eig.cpu().numpy().reshape(-1, 3), np.broadcast_to(want, (pos.size // 3, 3)),
                               rtol=2e-5)


def test_tricubic_grid_iets_matches_oracle(orc):
    # on an energy grid the sample part of the stiffness is the Hessian of the tricubic
    # interpolant: continuous across cell faces, so every point is compared
    c = case32(synth.benzene_case())
    c["grid"] = dict(c["grid"], interp=1)
    o = orc.forward(c)
    pos = o["pos"].astype(np.float32).astype(np.float64)
    ref, ref_hw = orc.iets(o["ff"], c["grid"], None, None, c["scan"], c["tip"], pos)
    got, got_hw = gpu_iets(c, pos)
    assert np.abs(got - ref).max() <= 1e-4, np.abs(got - ref).max()
    stiff = ref > 1e-3
    assert (np.abs(got_hw - ref_hw) / np.maximum(ref_hw, 1e-12))[stiff].max() <= 1e-3
