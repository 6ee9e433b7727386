"""Pins of the oracle's tip-quadrupole term (Secs. 2.2.3, 2.2.5: the CO tip's
quadrupolar charge distribution, moment -0.05 e*A^2 in the paper's
point-charge simulations).

The reading: an axial point quadrupole of second moment Qzz = sum_k q_k z_k^2
(no net charge, no dipole) rides on the PP without rotating; in the sample
potential V its energy is (Qzz/2) d^2V/dz^2.  What fixes it independently of
the oracle's own quadrupole formula:
  - the physical definition: three point charges +c, -2c, +c at z = +s, 0, -s
    around the PP (second moment 2 c s^2 = Qzz) tend to the quadrupole as
    s -> 0; the oracle's monopole path (pinned to Coulomb's law elsewhere)
    evaluates them;
  - closed forms on the axis and in the plane of a single charge;
  - F = -grad E by central differences;
  - the adjoint against central differences of the whole forward pass,
    including dL/dQzz, and the charge identity
    sum_i q_i dL/dq_i = Q dL/dQ + Qzz dL/dQzz (every electrostatic term is
    bilinear in a sample charge and a tip moment).
"""
import copy

import numpy as np
import pytest

from paper_2401_14564_gb300 import synth

KE = 14.3996454784
QZZ = -0.05


def probe(**kw):
    """Electrostatics only (eps_pp = 0 switches Lennard-Jones off)."""
    return synth.default_probe(**{"eps_pp": 0.0, "Q": 0.0, "Qzz": QZZ, **kw})


def grid_stub():
    return {"nx": 4, "ny": 4, "nz": 4, "x0": 0.0, "y0": 0.0, "z0": 0.0, "dx": 1.0, "dy": 1.0, "dz": 1.0,
            "periodic_xy": 0}


def far_points(atoms, n, seed, rmin=2.0):
    rng = np.random.default_rng(seed)
    xyz = np.stack([atoms["x"], atoms["y"], atoms["z"]], 1)
    pts = []
    while len(pts) < n:
        p = rng.uniform([-6, -6, 2.0], [6, 6, 7.0])
        if np.linalg.norm(xyz - p, axis=1).min() > rmin:
            pts.append(p)
    return np.array(pts)


def three_charges(orc, atoms, pts, s):
    c = QZZ / (2.0 * s * s)
    up, _ = orc.ff_points(atoms, probe(Q=c, Qzz=0.0), grid_stub(), pts + [0, 0, s])
    dn, _ = orc.ff_points(atoms, probe(Q=c, Qzz=0.0), grid_stub(), pts - [0, 0, s])
    mid, _ = orc.ff_points(atoms, probe(Q=-2.0 * c, Qzz=0.0), grid_stub(), pts)
    return up + dn + mid


def test_quadrupole_is_the_limit_of_three_point_charges(orc):
    atoms = synth.random_molecule(21, 14)
    pts = far_points(atoms, 40, 5)
    got, core = orc.ff_points(atoms, probe(), grid_stub(), pts)
    assert not core.any()
    s = 0.02
    # Richardson: the three-charge error is even in s, O(s^2)
    lim = (4.0 * three_charges(orc, atoms, pts, s / 2) - three_charges(orc, atoms, pts, s)) / 3.0
    scale = np.abs(got).max(axis=0)
    assert np.all(np.abs(got - lim) <= 1e-7 * scale), np.abs(got - lim).max(axis=0) / scale
    # and the unextrapolated construction is visibly O(s^2) away (the pin has teeth)
    raw = three_charges(orc, atoms, pts, s)
    assert np.abs(raw - got).max() > 1e3 * np.abs(lim - got).max()


def test_single_charge_closed_forms(orc):
    q = 0.3
    atoms = {"x": np.zeros(1), "y": np.zeros(1), "z": np.zeros(1), "R": np.ones(1), "eps": np.zeros(1),
             "q": np.array([q])}
    for h in (2.0, 3.5, 5.0):
        # on the axis: E = k_e q Qzz / h^3, F = 3 k_e q Qzz / h^4 z_hat
        out, _ = orc.ff_points(atoms, probe(), grid_stub(), np.array([[0.0, 0.0, h]]))
        assert out[0, 3] == pytest.approx(KE * q * QZZ / h**3, rel=1e-13)
        assert out[0, 2] == pytest.approx(3 * KE * q * QZZ / h**4, rel=1e-13)
        assert abs(out[0, 0]) < 1e-18 and abs(out[0, 1]) < 1e-18
        # in the plane of the charge: E = -k_e q Qzz / (2 x^3), F = -(3/2) k_e q Qzz / x^4 x_hat
        out, _ = orc.ff_points(atoms, probe(), grid_stub(), np.array([[h, 0.0, 0.0]]))
        assert out[0, 3] == pytest.approx(-0.5 * KE * q * QZZ / h**3, rel=1e-13)
        assert out[0, 0] == pytest.approx(-1.5 * KE * q * QZZ / h**4, rel=1e-13)
        assert abs(out[0, 2]) < 1e-18


def test_force_is_minus_gradient_of_energy(orc):
    atoms = synth.random_molecule(22, 10)
    pr = synth.default_probe(Qzz=QZZ)  # LJ + monopole + quadrupole together
    pts = far_points(atoms, 20, 6, rmin=2.5)
    F, _ = orc.ff_points(atoms, pr, grid_stub(), pts)
    h = 1e-4
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        Ep, _ = orc.ff_points(atoms, pr, grid_stub(), pts + e)
        Em, _ = orc.ff_points(atoms, pr, grid_stub(), pts - e)
        fd = -(Ep[:, 3] - Em[:, 3]) / (2 * h)
        assert np.allclose(F[:, a], fd, rtol=1e-6, atol=1e-8 * np.abs(F).max()), a


def test_cutoff_removes_the_term_beyond_rc(orc):
    q = 0.3
    atoms = {"x": np.zeros(1), "y": np.zeros(1), "z": np.zeros(1), "R": np.ones(1), "eps": np.zeros(1),
             "q": np.array([q])}
    pr = probe(coul_rc=4.0)
    inside, _ = orc.ff_points(atoms, pr, grid_stub(), np.array([[0.0, 0.0, 3.0]]))
    beyond, _ = orc.ff_points(atoms, pr, grid_stub(), np.array([[0.0, 0.0, 4.5]]))
    assert inside[0, 2] == pytest.approx(3 * KE * q * QZZ / 3.0**4, rel=1e-13)
    assert np.all(beyond == 0.0)


def tiny_case():
    c = synth.small_case(seed=9, n_atoms=6, nxy=40, nz=36, scan_px=5, nz_scan=12, d=0.15)
    c["fire"] = synth.default_fire(max_iter=5000, ftol=1e-6)
    c["probe"] = synth.default_probe(Qzz=-0.1)
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
    if what in ("x", "y", "z", "q", "R"):
        c2["atoms"][what] = c2["atoms"][what].copy()
        c2["atoms"][what][idx] += h
    else:
        c2["probe"][what] += h
    return c2


PARAMS = [("x", 1, 1e-4), ("z", 2, 1e-4), ("q", 3, 1e-4), ("q", 0, 1e-4), ("Qzz", None, 1e-4), ("Q", None, 1e-4)]


def test_grid_free_adjoint_with_quadrupole_matches_central_differences(orc):
    c = tiny_case()
    _, r = loss(orc, c, True)
    g = orc.backward(None, c["grid"], c["atoms"], c["probe"], c["scan"], c["tip"], c["df"], r["pos"], c["w"])
    assert abs(g["Qzz"]) > 0.0
    for what, idx, h in PARAMS:
        fd = (loss(orc, perturbed(c, what, idx, h), True)[0] - loss(orc, perturbed(c, what, idx, -h), True)[0]) / (2 * h)
        an = g[what][idx] if idx is not None else g[what]
        assert an == pytest.approx(fd, rel=2e-5, abs=1e-6 * max(abs(fd), 1.0)), (what, idx, an, fd)


def test_grid_adjoint_with_quadrupole_matches_central_differences(orc):
    c = tiny_case()
    _, r = loss(orc, c, False)
    g = orc.backward(r["ff"], c["grid"], c["atoms"], c["probe"], c["scan"], c["tip"], c["df"], r["pos"], c["w"])
    an, fd = [], []
    for what, idx, h in PARAMS:
        fd.append((loss(orc, perturbed(c, what, idx, h), False)[0]
                   - loss(orc, perturbed(c, what, idx, -h), False)[0]) / (2 * h))
        an.append(g[what][idx] if idx is not None else g[what])
    an, fd = np.array(an), np.array(fd)
    assert np.abs(an - fd).max() < 1e-3 * np.abs(fd).max(), (an, fd)


@pytest.mark.parametrize("grid_free", [True, False])
def test_charge_identity_with_quadrupole(orc, grid_free):
    c = tiny_case()
    _, r = loss(orc, c, grid_free)
    g = orc.backward(None if grid_free else r["ff"], c["grid"], c["atoms"], c["probe"], c["scan"], c["tip"],
                     c["df"], r["pos"], c["w"])
    lhs = float((c["atoms"]["q"] * g["q"]).sum())
    rhs = c["probe"]["Q"] * g["Q"] + c["probe"]["Qzz"] * g["Qzz"]
    assert lhs == pytest.approx(rhs, rel=1e-10)
    assert abs(c["probe"]["Qzz"] * g["Qzz"]) > 1e-3 * abs(rhs)
