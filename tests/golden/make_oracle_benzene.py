"""Writes oracle_benzene.json: FP64 oracle outputs on the benzene workload at a few
sampled nodes and pixels, kept as a regression fixture of the oracle itself.

Calls only the oracle (and the seeded input generator).  Rerun only when the oracle's
arithmetic changes for a reason the commit names.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2401_14564_gb300 import synth  # noqa: E402


def main():
    c = synth.benzene_case()
    fire = synth.parity_fire()
    o = oracle.forward(c, fire=fire)
    rng = np.random.default_rng(2024)
    nodes = rng.choice(c["grid"]["nx"] * c["grid"]["ny"] * c["grid"]["nz"], 12, replace=False)
    ff = o["ff"].reshape(-1, 4)
    pix = rng.choice(c["scan"]["nx"] * c["scan"]["ny"], 6, replace=False)
    s = c["scan"]
    pos = o["pos"].reshape(s["nz"], -1, 3)
    fz = o["fz"].reshape(s["nz"], -1)
    df = o["df"].reshape(o["df"].shape[0], -1)
    out = {
        "_note": "FP64 oracle on the benzene workload (synth.benzene_case, parity FIRE settings); written by "
                 "make_oracle_benzene.py",
        "nodes": nodes.tolist(),
        "ff": ff[nodes].tolist(),
        "pixels": pix.tolist(),
        "pos_k0": pos[0, pix].tolist(),
        "pos_klast": pos[-1, pix].tolist(),
        "fz": fz[:, pix].T.tolist(),
        "df": df[:, pix].T.tolist(),
    }
    with open(os.path.join(HERE, "oracle_benzene.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
