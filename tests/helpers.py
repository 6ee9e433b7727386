"""Shared test utilities: float32-rounded inputs, error metrics, GPU runners."""
import copy

import numpy as np

F32_KEYS = ("x", "y", "z", "R", "eps", "q")


def f32(v):
    return float(np.float32(v))


def case32(case):
    """Round every input of a case to float32 so both sides see identical inputs."""
    c = copy.deepcopy(case)
    for k in F32_KEYS:
        c["atoms"][k] = np.asarray(c["atoms"][k], dtype=np.float32).astype(np.float64)
    for blk in ("probe", "grid", "scan", "tip", "fire", "df"):
        for k, v in c.get(blk, {}).items():
            if isinstance(v, float):
                c[blk][k] = f32(v)
    return c


def ff_rel_err(F_gpu, F_ref, floor=1e-3):
    """Per-node |F_gpu - F_ref| / max(|F_ref|, floor) (force components only)."""
    d = np.linalg.norm(F_gpu[..., :3] - F_ref[..., :3], axis=-1)
    return d / np.maximum(np.linalg.norm(F_ref[..., :3], axis=-1), floor)


def linear_ff(ff_flat, grid):
    """Flat linear-layout FF buffer -> [nz][ny][nx][4]."""
    return np.asarray(ff_flat, dtype=np.float64).reshape(grid["nz"], grid["ny"], grid["nx"], 4)


def relax_compare(r_gpu, r_orc, basin_tol=0.05, lam_min=0.01):
    """Position/Fz errors on pixels that are well conditioned and in the same basin.

    Returns (max |dp| over kept, max |dFz| over kept, keep mask [nz][ny][nx],
    number excluded for conditioning, number excluded as other basins).
    """
    dp = np.linalg.norm(r_gpu["pos"] - r_orc["pos"], axis=-1)
    well = r_orc["lam"] >= lam_min
    same = dp < basin_tol
    keep = well & same
    dfz = np.abs(r_gpu["fz"] - r_orc["fz"])
    return (float(dp[keep].max()) if keep.any() else 0.0, float(dfz[keep].max()) if keep.any() else 0.0, keep,
            int((~well).sum()), int((well & ~same).sum()))


def ill_conditioned_within_bound(pos_gpu, r_orc, ftol, lam_min=0.01, basin_tol=0.05, slack=1e-4):
    """Entries with 0 < lambda < lam_min in the same basin obey |dp| <= 1.1 ftol / lambda + slack.

    FIRE stops at |G| < ftol, so the GPU position can sit ftol/lambda from the fixed
    point (plus FP32 rounding of the grid, ~1e-6 relative); returns (checked, ok) counts.
    """
    dp = np.linalg.norm(pos_gpu - r_orc["pos"], axis=-1)
    lam = r_orc["lam"]
    sel = (lam > 0) & (lam < lam_min) & (dp < basin_tol)
    ok = dp[sel] <= 1.1 * ftol / lam[sel] + slack
    return int(sel.sum()), int(ok.sum())


def df_keep(keep, m):
    """A df output centred at c is compared when all heights c-m..c+m are kept."""
    nz = keep.shape[0]
    out = np.ones((nz - 2 * m,) + keep.shape[1:], dtype=bool)
    for s in range(2 * m + 1):
        out &= keep[s:s + nz - 2 * m]
    return out
