"""Autotuner: every launch shape it can pick computes the same values.

The FF z-blocking (4, 8, 16 nodes per thread) and the grid layout (linear or
bricked) do not change the arithmetic per node or per pixel, so the images
must be bit-identical whichever candidate wins; the tuner must return one of
its candidates.
"""
import numpy as np
import pytest
import torch

from helpers import case32
from paper_2401_14564_gb300 import afm, pp, synth, tune

pytestmark = pytest.mark.gpu


def test_ff_launch_shapes_are_bit_identical():
    c = case32(synth.small_case(seed=12, n_atoms=17, nxy=40, nz=37))
    grid = pp.make_grid(c["grid"])
    atoms = pp.make_atoms(afm.atoms_to_device(c["atoms"]))
    probe = pp.make_probe(c["probe"])
    out = {}
    for z in (4, 8, 16):
        ff = torch.full((pp.pp_ff_floats(grid),), float("nan"), device="cuda")
        pp.pp_make_ff_tuned(atoms, probe, grid, ff, pp.Tuning(z))
        out[z] = ff.cpu().numpy()
    assert np.array_equal(out[4], out[8]) and np.array_equal(out[16], out[8])
    with pytest.raises(pp.PPError):
        pp.pp_make_ff_tuned(atoms, probe, grid, torch.empty(pp.pp_ff_floats(grid), device="cuda"), pp.Tuning(6))


def test_tuned_simulator_reproduces_default_images():
    c = case32(synth.benzene_case())
    r = tune.tune_case(c, reps=1)
    assert r["ff_zpt"] in (4, 8, 16)
    assert f"{r['layout']}:{tuple(r['brick']) if r['brick'] else None}" in r["relax_ms"]
    a = afm.Simulator(c)
    b = afm.Simulator(c, tuning=r)
    at = afm.atoms_to_device(c["atoms"])
    a.run(at)
    b.run(at)
    torch.cuda.synchronize()
    assert torch.equal(a.df, b.df) and torch.equal(a.fz, b.fz)


def test_forces_only_tuning_and_its_cache_entry(tmp_path):
    # the tuner times the forces-only assembly when asked, caches it under its own key, and the
    # tuned forces-only simulator reproduces the default images
    c = case32(synth.benzene_case())
    path = str(tmp_path / "tuning.json")
    full = tune.cached(c, path=path, reps=1)
    fo = tune.cached(c, path=path, reps=1, ff_energy=False)
    import json
    keys = sorted(json.load(open(path)))
    assert len(keys) == 2 and keys[1] == keys[0] + "|forces_only"
    assert fo["ff_zpt"] in (4, 8, 16) and full["ff_zpt"] in (4, 8, 16)
    a = afm.Simulator(c)
    b = afm.Simulator(c, tuning=fo, ff_energy=False)
    at = afm.atoms_to_device(c["atoms"])
    a.run(at)
    b.run(at)
    torch.cuda.synchronize()
    assert torch.equal(a.df, b.df) and torch.equal(a.fz, b.fz)
    assert torch.count_nonzero(b.ff.view(-1, 4)[:, 3]).item() == 0


def test_pipeline_regime_tuning_reproduces_the_images():
    # layouts timed on whole steps two in flight: the pick is one of the candidates and a pipeline
    # built with it gives the default images, item by item
    c = case32(synth.small_case(seed=13, n_atoms=9, nxy=32, nz=36, scan_px=10, nz_scan=12))
    r = tune.tune_case(c, reps=1, pipeline_slots=2, ff_energy=False)
    assert r["layout_timing"].startswith("ms per step")
    assert f"{r['layout']}:{tuple(r['brick']) if r['brick'] else None}" in r["relax_ms"]
    at = afm.atoms_to_device(c["atoms"])
    ref = afm.Simulator(c)
    ref.run(at)
    pipe = afm.Pipeline(c, slots=2, tuning=r, ff_energy=False)
    outs = [torch.empty_like(ref.df) for _ in range(3)]
    pipe.run_many([at] * 3, outs)
    torch.cuda.synchronize()
    for o in outs:
        assert torch.equal(o, ref.df)
