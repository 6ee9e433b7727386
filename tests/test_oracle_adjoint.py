"""Pins of the oracle's implicit adjoint.

The paper has no gradients; the oracle differentiates its own discrete model
at the relaxed equilibrium.  Central finite differences of the full oracle
forward pass (FF grid -> relaxed scan -> df) fix the result: to ~1e-6 in the
grid-free model (smooth), and to ~1e-3 in the grid model (the trilinear
interpolant has kinks on cell faces).  The charge scaling identity
sum_i q_i dL/dq_i = Q dL/dQ holds exactly in both.
"""
import copy

import numpy as np
import pytest

from paper_2401_14564_gb300 import synth


def tiny_case():
    c = synth.small_case(seed=9, n_atoms=6, nxy=40, nz=36, scan_px=5, nz_scan=12, d=0.15)
    c["fire"] = synth.default_fire(max_iter=5000, ftol=1e-6)
    rng = np.random.default_rng(7)
    m = 5
    c["w"] = rng.standard_normal((c["scan"]["nz"] - 2 * m, c["scan"]["ny"], c["scan"]["nx"]))
    return c


def loss(orc, c, grid_free):
    r = orc.forward(c, grid_free=grid_free, polish_tol=1e-13)
    assert r["ok"].all()
    return float((c["w"] * r["df"]).sum()), r


def perturbed(c, what, idx, h):
    c2 = copy.deepcopy(c)
    if what in ("x", "y", "z", "q", "R", "eps"):
        c2["atoms"][what] = c2["atoms"][what].copy()
        c2["atoms"][what][idx] += h
    elif what == "Q":
        c2["probe"]["Q"] += h
    else:
        c2["tip"][what] += h
    return c2


PARAMS = [("x", 0, 1e-4), ("y", 2, 1e-4), ("z", 1, 1e-4), ("z", 4, 1e-4), ("q", 3, 1e-4), ("R", 5, 1e-4),
          ("eps", 0, 1e-6), ("kx", None, 1e-4), ("ky", None, 1e-4), ("kR", None, 1e-3), ("Q", None, 1e-4)]


def grads_of(orc, c, r, grid_free):
    return orc.backward(None if grid_free else r["ff"], c["grid"], c["atoms"], c["probe"], c["scan"], c["tip"],
                        c["df"], r["pos"], c["w"])


def pick(g, what, idx):
    return g[what][idx] if idx is not None else g[what]


def test_grid_free_adjoint_matches_central_differences(orc):
    c = tiny_case()
    L0, r = loss(orc, c, True)
    g = grads_of(orc, c, r, True)
    for what, idx, h in PARAMS:
        fd = (loss(orc, perturbed(c, what, idx, h), True)[0] - loss(orc, perturbed(c, what, idx, -h), True)[0]) / (2 * h)
        an = pick(g, what, idx)
        assert an == pytest.approx(fd, rel=2e-5, abs=1e-6 * max(abs(fd), 1.0)), (what, idx, an, fd)


def test_grid_adjoint_matches_central_differences(orc):
    c = tiny_case()
    L0, r = loss(orc, c, False)
    g = grads_of(orc, c, r, False)
    an, fd = [], []
    for what, idx, h in PARAMS:
        fd.append((loss(orc, perturbed(c, what, idx, h), False)[0]
                   - loss(orc, perturbed(c, what, idx, -h), False)[0]) / (2 * h))
        an.append(pick(g, what, idx))
    an, fd = np.array(an), np.array(fd)
    # each component within 1e-3 of the gradient's scale
    assert np.abs(an - fd).max() < 1e-3 * np.abs(fd).max(), (an, fd)


@pytest.mark.parametrize("grid_free", [True, False])
def test_charge_scaling_identity(orc, grid_free):
    c = tiny_case()
    _, r = loss(orc, c, grid_free)
    g = grads_of(orc, c, r, grid_free)
    lhs = float((c["atoms"]["q"] * g["q"]).sum())
    assert lhs == pytest.approx(c["probe"]["Q"] * g["Q"], rel=1e-10)


def test_grid_adjoint_touches_only_the_scanned_slab(orc):
    c = tiny_case()
    _, r = loss(orc, c, False)
    g = orc.backward(r["ff"], c["grid"], c["atoms"], c["probe"], c["scan"], c["tip"], c["df"], r["pos"], c["w"],
                     want_grid_adj=True)
    adj = g["grid_adj"]
    nz_touched = np.nonzero(np.abs(adj).sum(axis=(1, 2, 3)))[0]
    zmin = r["pos"][..., 2].min()
    zmax = r["pos"][..., 2].max()
    gz = c["grid"]["z0"] + c["grid"]["dz"] * nz_touched
    assert gz.min() >= zmin - c["grid"]["dz"] - 1e-9 and gz.max() <= zmax + c["grid"]["dz"] + 1e-9


def test_gradient_workload_adjoint_matches_central_differences_on_20_coordinates(orc):
    """The 40-atom gradient workload (176x176x60 grid, 128x128x20 scan, loss sum(w df) with
    w ~ N(0,1) seed 7): the oracle's grid-model adjoint against FP64 central differences of its
    whole forward pass on 20 atom coordinates chosen with seed 11, h = 1e-4 A."""
    c = synth.gradient_case()
    fire = synth.parity_fire(ftol=1e-9, max_iter=20000)

    def L(cc):
        r = orc.forward(cc, fire=fire, polish_tol=1e-12)
        assert r["ok"].all()
        return float((c["w"] * r["df"]).sum()), r

    _, r = L(c)
    g = orc.backward(r["ff"], c["grid"], c["atoms"], c["probe"], c["scan"], c["tip"], c["df"], r["pos"], c["w"])
    rng = np.random.default_rng(c["fd_seed"])
    n = len(c["atoms"]["x"])
    picks = rng.choice(3 * n, 20, replace=False)
    h = 1e-4
    an, fd = [], []
    for p in picks:
        ia, ax = int(p // 3), "xyz"[int(p % 3)]
        fd.append((L(perturbed(c, ax, ia, h))[0] - L(perturbed(c, ax, ia, -h))[0]) / (2 * h))
        an.append(g[ax][ia])
    an, fd = np.array(an), np.array(fd)
    # grid model: relaxed points that cross a cell face within +-h see the trilinear kink
    assert np.abs(an - fd).max() < 1e-3 * np.abs(fd).max(), (an, fd)
