"""Fixtures under tests/golden/:

- paper_constants.json: numbers the paper prints (each with its place) that the
  defaults and readings take; checked against the code's defaults.
- oracle_benzene.json: FP64 oracle outputs on the benzene workload at sampled
  nodes and pixels, written by tests/golden/make_oracle_benzene.py (which calls
  only the oracle); any later change of the oracle's arithmetic shows here and
  must be justified by the passage it follows.
"""
import json
import os

import numpy as np

from paper_2401_14564_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_defaults_take_the_papers_numbers():
    pc = load("paper_constants.json")
    assert synth.default_tip()["R0"] == pc["R0_A"]["value"]
    import bench

    lo, hi = pc["co_quadrupole_range_eA2"]["value"]
    assert bench.QZZ_CO == pc["co_quadrupole_eA2"]["value"] and lo <= bench.QZZ_CO <= hi
    smin, smax = pc["grid_spacing_A"]["value"]
    for case in (synth.benzene_case(), synth.flake_case()):
        assert smin <= case["grid"]["dx"] <= smax


def test_oracle_reproduces_its_frozen_benzene_outputs(orc):
    g = load("oracle_benzene.json")
    c = synth.benzene_case()
    o = orc.forward(c, fire=synth.parity_fire())
    s = c["scan"]
    ff = o["ff"].reshape(-1, 4)[g["nodes"]]
    assert np.allclose(ff, g["ff"], rtol=1e-12, atol=1e-15)
    pos = o["pos"].reshape(s["nz"], -1, 3)
    assert np.allclose(pos[0, g["pixels"]], g["pos_k0"], rtol=0, atol=1e-10)
    assert np.allclose(pos[-1, g["pixels"]], g["pos_klast"], rtol=0, atol=1e-10)
    fz = o["fz"].reshape(s["nz"], -1)[:, g["pixels"]].T
    assert np.allclose(fz, g["fz"], rtol=0, atol=1e-10)
    df = o["df"].reshape(o["df"].shape[0], -1)[:, g["pixels"]].T
    assert np.allclose(df, g["df"], rtol=0, atol=1e-9)
