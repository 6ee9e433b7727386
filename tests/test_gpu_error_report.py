"""FP32 (GPU) against FP64 (oracle) error of every output, measured and printed
(run with -s to see the table), each held to its parity bar:

  FF grid     relative force error (reading R8), max and 99.9th percentile outside the core;
  p*          max |p_gpu - p_oracle| (A) over well-conditioned points in the same basin;
  Fz          max |Fz_gpu - Fz_oracle| (eV/A) over the same points;
  df          max |df_gpu - df_oracle| / (df image range);
  gradients   relative L2 error per gradient vector at the oracle's relaxed positions.

Workloads: benzene (80x80x60 grid, 40x40x20 scan, the whole image), flake60 (the bench's
256x256x200 grid: 4000 seeded nodes; 48 seeded pixel columns of the 256x256x40 scan) and the
40-atom gradient workload (isolated adjoint).
"""
import numpy as np
import pytest

from helpers import case32, df_keep, ff_rel_err, relax_compare
from paper_2401_14564_gb300 import afm, synth
from test_gpu_backward import KEYS, TIP, gpu_backward, rel

pytestmark = pytest.mark.gpu

REPORT = []


def report(workload, output, value, bar):
    REPORT.append((workload, output, value, bar))
    print(f"  {workload:<10} {output:<28} {value:10.3e}   (bar {bar:.0e})")
    assert value <= bar, (workload, output, value, bar)


def test_benzene_every_output(orc):
    c = case32(synth.benzene_case())
    fire = synth.parity_fire()
    g = afm.afm(c, fire=fire)
    o = orc.forward(c, fire=fire)
    F = np.asarray(g["ff"].cpu().numpy(), dtype=np.float64).reshape(o["ff"].shape)
    err = ff_rel_err(F, o["ff"])[~o["core"]]
    print()
    report("benzene", "FF rel. error max", float(err.max()), 1e-4)
    report("benzene", "FF rel. error p99.9", float(np.percentile(err, 99.9)), 1e-4)
    dp, dfz, keep, _, _ = relax_compare(g, o)
    report("benzene", "p* max |dp| (A)", dp, 1e-3)
    report("benzene", "Fz max |dFz| (eV/A)", dfz, 1e-3 * np.abs(o["fz"]).max())
    kd = df_keep(keep, (keep.shape[0] - g["df"].shape[0]) // 2)
    rng = o["df"].max() - o["df"].min()
    report("benzene", "df max |ddf| / range", float(np.abs(g["df"] - o["df"])[kd].max() / rng), 1e-3)


def test_flake_sampled_outputs(orc):
    c = case32(synth.flake_case())
    fire = synth.parity_fire()
    g = afm.afm(c, fire=fire)
    gr, s = c["grid"], c["scan"]
    F = np.asarray(g["ff"].cpu().numpy(), dtype=np.float64).reshape(gr["nz"], gr["ny"], gr["nx"], 4)
    rng = np.random.default_rng(0)
    idx = np.stack([rng.integers(0, gr[n], 4000) for n in ("nz", "ny", "nx")], axis=1)
    pts = np.stack([np.float32(gr["x0"]) + idx[:, 2] * np.float32(gr["dx"]),
                    np.float32(gr["y0"]) + idx[:, 1] * np.float32(gr["dy"]),
                    np.float32(gr["z0"]) + idx[:, 0] * np.float32(gr["dz"])], axis=1).astype(np.float64)
    ref, core = orc.ff_points(c["atoms"], c["probe"], gr, pts)
    err = ff_rel_err(F[idx[:, 0], idx[:, 1], idx[:, 2]], ref)[~core]
    print()
    report("flake60", "FF rel. error max", float(err.max()), 1e-4)
    report("flake60", "FF rel. error p99.9", float(np.percentile(err, 99.9)), 1e-4)
    cols = np.sort(np.random.default_rng(1).choice(s["nx"] * s["ny"], 48, replace=False))
    ff, _ = orc.make_ff(c["atoms"], c["probe"], gr)
    o = orc.relax_columns(ff, gr, None, None, s, c["tip"], fire, cols)
    jj, ii = cols // s["nx"], cols % s["nx"]
    gp = np.moveaxis(g["pos"][:, jj, ii], 0, 1)
    dp = np.linalg.norm(gp - o["pos"], axis=-1)
    keep = (o["lam"] >= 0.01) & (dp < 0.05)
    report("flake60", "p* max |dp| (A)", float(dp[keep].max()), 1e-3)
    report("flake60", "Fz max |dFz| (eV/A)", float(np.abs(g["fz"][:, jj, ii].T - o["fz"])[keep].max()),
           1e-3 * np.abs(o["fz"]).max())
    odf = orc.fz_to_df(o["fz"].T, s["dz"], c["df"])
    kd = df_keep(keep.T, 5)
    report("flake60", "df max |ddf| / range",
           float(np.abs(g["df"][:, jj, ii] - odf)[kd].max() / (g["df"].max() - g["df"].min())), 1e-3)


def test_gradient_workload_adjoint(orc):
    c = case32(synth.gradient_case())
    fire = synth.parity_fire(ftol=2e-7, max_iter=20000)
    o = orc.forward(c, fire=fire)
    ref = orc.backward(o["ff"], c["grid"], c["atoms"], c["probe"], c["scan"], c["tip"], c["df"], o["pos"], c["w"])
    got = gpu_backward(c, o["pos"], c["w"])
    print()
    for k in KEYS:
        report("mol40", f"dL/d{k} rel. L2", rel(got[k], ref[k]), 1e-4)
    for k in TIP:
        report("mol40", f"dL/d{k} rel.", rel(got[k], ref[k]), 1e-3)
