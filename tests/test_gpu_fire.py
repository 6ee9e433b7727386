"""FIRE on the GPU (K2) step for step against the oracle's FIRE (Sec. 5.1.1 step 2; Bitzek et
al. 2006), and the optional Newton polish.

Both sides relax on the same force field: the oracle's FP64 grid rounded to FP32, which the GPU
scan reads as it is and the oracle reads back in FP64.  Only the precision of FIRE's own
arithmetic then differs, so FIRE's branch decisions (downhill mixing, uphill reset, step growth
after more than n_min downhill steps, alpha decay) must take the same turns: the number of
position updates per pixel and height equals the oracle's at >= 99 % of the points, under the
timed settings (dt0 = dt_max: no step growth, alpha decay on), with the step growth on, and at the
parity tolerance.  Where they differ, a residual landed within FP32 rounding of ftol (one update
more or less) or a downhill test F.v > 0 with F.v within rounding of zero went the other way and
the two trajectories part; either way both end at the same fixed point, within FIRE's stopping
residual ftol / lambda_min of it.
"""
import numpy as np
import pytest
import torch

from helpers import case32, relax_compare
from paper_2401_14564_gb300 import afm, batch, pp, synth

pytestmark = pytest.mark.gpu


def gpu_scan_on(ff32, c, fire):
    """K2 on a caller-made FP32 grid (linear layout) -> pos, fz, iters as numpy."""
    grid = pp.make_grid(c["grid"], 0)
    ff = torch.as_tensor(np.ascontiguousarray(ff32, dtype=np.float32).ravel(), device="cuda")
    s = c["scan"]
    nz, ny, nx = s["nz"], s["ny"], s["nx"]
    pos = torch.empty((nz, ny, nx, 3), device="cuda")
    fz = torch.empty((nz, ny, nx), device="cuda")
    it = torch.empty((nz, ny, nx), dtype=torch.int32, device="cuda")
    pp.pp_relax_scan(ff, grid, pp.make_scan(s), pp.make_tip(c["tip"]), pp.make_fire(fire), pos, fz, it)
    torch.cuda.synchronize()
    return {"pos": pos.cpu().numpy().astype(np.float64), "fz": fz.cpu().numpy().astype(np.float64),
            "iters": it.cpu().numpy()}


def oracle_grid32(orc, c):
    ff, core = orc.make_ff(c["atoms"], c["probe"], c["grid"])
    return ff.astype(np.float32)


FIRES = {
    "timed": {},
    "growth": dict(dt0=0.25, dt_max=1.0, n_min=2),
    "parity": dict(ftol=1e-5, max_iter=2000),
}


@pytest.mark.parametrize("which", sorted(FIRES))
@pytest.mark.parametrize("case", ["benzene", "small"])
def test_fire_update_counts_equal_the_oracle(orc, which, case):
    c = case32(synth.benzene_case() if case == "benzene" else
               synth.small_case(seed=3, n_atoms=12, nxy=32, nz=40, scan_px=12, nz_scan=12))
    fire = synth.default_fire(**FIRES[which])
    ff32 = oracle_grid32(orc, c)
    o = orc.relax_scan(ff32.astype(np.float64), c["grid"], None, None, c["scan"], c["tip"], fire, polish_tol=0.0)
    g = gpu_scan_on(ff32, c, fire)
    d = np.abs(g["iters"].astype(np.int64) - o["iters"])
    print(f"\n{case}/{which}: counts equal at {(d == 0).mean():.5f}, within one at {(d <= 1).mean():.5f}, "
          f"largest difference {d.max()}")
    assert (d == 0).mean() >= 0.99, ((d == 0).mean(), d.max())
    assert (d <= 1).mean() >= 0.997, ((d <= 1).mean(), d.max())
    # a wrong rule would also show as a different relaxed point: FIRE alone on both sides
    dp = np.linalg.norm(g["pos"] - o["pos"], axis=-1)
    assert np.median(dp) < 1e-4
    # points whose counts differ still reach the same fixed point (both stop below ftol)
    ref = orc.relax_scan(ff32.astype(np.float64), c["grid"], None, None, c["scan"], c["tip"], fire)
    lam = np.maximum(ref["lam"], 1e-3)
    diff = d > 0
    bound = 2.2 * fire["ftol"] / lam + 1e-4
    assert (dp[diff] <= bound[diff]).all(), (dp[diff] / bound[diff]).max()
    if which == "growth":
        # the settings reach the growth branch: more than n_min downhill steps in a row happen
        # whenever a point needs more than n_min + 2 updates
        assert (o["iters"] > fire["n_min"] + 2).mean() > 0.2


def test_newton_polish_reaches_the_oracle_fixed_point(orc):
    # timed FIRE settings (ftol 1e-4 eV/A) + up to 4 Newton steps: the relaxed points sit at the
    # equilibrium of the GPU's own grid, i.e. at the oracle's Newton-polished fixed point up to
    # K1's rounding over the stiffness (FIRE alone leaves ftol / lambda, up to 6e-3 A)
    c = case32(synth.benzene_case())
    fire = synth.default_fire()
    plain = afm.afm(c, fire=fire)
    pol = afm.afm(c, fire=dict(fire, polish=4))
    o = orc.forward(c, fire=fire)
    dp_plain, _, keep, _, _ = relax_compare(plain, o)
    dp_pol, dfz, keep2, n_ill, n_basin = relax_compare(pol, o)
    assert n_basin <= 0.01 * keep2.size
    assert dp_pol <= 5e-5, dp_pol
    assert dp_plain > 10 * dp_pol
    assert dfz <= 1e-5


def test_polish_is_refused_by_the_batch():
    cs = [case32(c) for c in synth.batch_cases(2, 1000)]
    b = batch.Batch(cs, fire=synth.default_fire(polish=2))
    with pytest.raises(pp.PPError) as e:
        b.run()
    assert e.value.status == 6
