"""pp_backward_noalloc: the adjoint without a caller workspace.

Callers that cannot call cudaMalloc (a real-time acquisition or control loop,
a plugin whose host forbids device allocations after start-up, C or Fortran
code without a device allocator) use this entry point: it takes its scratch
from a fixed array inside the library.  The array is shared by every call and
keeps the previous call's contents, so the check runs two calls in a row with
different loss weights and compares each with pp_backward on a workspace the
test allocates, to the 1e-4 relative tolerance the other adjoint tests use for
run-to-run differences (FP32 atomics sum in a nondeterministic order).
"""
import numpy as np
import pytest
import torch

from helpers import case32
from paper_2401_14564_gb300 import afm, pp, synth

pytestmark = pytest.mark.gpu

KEYS = ("x", "y", "z", "q", "R", "eps")


def setup_case(interp=0):
    c = case32(synth.small_case(seed=9, n_atoms=8, nxy=40, nz=36, scan_px=9, nz_scan=14, d=0.15))
    c["grid"] = dict(c["grid"], interp=interp)
    sim = afm.Simulator(c, fire=synth.parity_fire())
    atoms_t = afm.atoms_to_device(c["atoms"])
    sim.run(atoms_t)
    return c, sim, atoms_t


def new_grads(n):
    g = {k: torch.full((n,), float("nan"), device="cuda") for k in KEYS}
    g["tip"] = torch.full((5,), float("nan"), device="cuda")
    return g


def flat(g):
    return np.concatenate([g[k].cpu().numpy() for k in KEYS + ("tip",)]).astype(np.float64)


@pytest.mark.parametrize("interp", [0, 1])
def test_noalloc_matches_workspace_entry_point_twice(interp):
    # on a force grid (a float4 grid adjoint per node) and on a tricubic energy grid (one float per
    # node) the scratch is laid out differently; both must match pp_backward
    c, sim, atoms_t = setup_case(interp)
    n = len(c["atoms"]["x"])
    atoms = pp.make_atoms(atoms_t)
    ws = torch.empty(pp.pp_backward_workspace(sim.grid) // 4 + 1, dtype=torch.float32, device="cuda")
    assert pp.pp_backward_workspace(sim.grid) <= pp.pp_backward_noalloc_capacity()
    rng = np.random.default_rng(21)
    for call in range(2):
        w = torch.as_tensor(rng.standard_normal(tuple(sim.df.shape)), dtype=torch.float32, device="cuda")
        ref, got = new_grads(n), new_grads(n)
        pp.pp_backward(atoms, sim.probe, sim.grid, sim.ff, sim.scan, sim.tip, sim.dfp, sim.pos, w,
                       pp.make_grads(ref), ws)
        pp.pp_backward_noalloc(atoms, sim.probe, sim.grid, sim.ff, sim.scan, sim.tip, sim.dfp, sim.pos, w,
                               pp.make_grads(got))
        torch.cuda.synchronize()
        a, b = flat(got), flat(ref)
        assert np.isfinite(a).all(), call
        for k in KEYS + ("tip",):
            ga, gb = got[k].cpu().numpy().astype(np.float64), ref[k].cpu().numpy().astype(np.float64)
            err = np.linalg.norm(ga - gb) / max(np.linalg.norm(gb), 1e-30)
            assert err <= 1e-4, (call, k, err)


def test_noalloc_rejects_a_grid_beyond_its_capacity():
    c, sim, atoms_t = setup_case()
    big = pp.make_grid(dict(c["grid"], nx=256, ny=256, nz=40))
    assert pp.pp_backward_workspace(big) > pp.pp_backward_noalloc_capacity()
    g = new_grads(len(c["atoms"]["x"]))
    ff = torch.zeros(pp.pp_ff_floats(big), device="cuda")
    w = torch.zeros(tuple(sim.df.shape), device="cuda")
    with pytest.raises(pp.PPError) as e:
        pp.pp_backward_noalloc(pp.make_atoms(atoms_t), sim.probe, big, ff, sim.scan, sim.tip, sim.dfp, sim.pos, w,
                               pp.make_grads(g))
    assert e.value.status == 4
    assert "static scratch" in str(e.value)
