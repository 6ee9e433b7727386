"""Pins of the oracle's force field and trilinear interpolation (CPU only).

Each check ties the oracle to a fact fixed outside its own code: closed-form
values of the LJ pair (Eq. LJ) at its minimum and zero crossing with the
mixing rules R_iPP = R_i + R_PP, e_iPP = sqrt(e_i e_PP); the Coulomb constant
rebuilt from SI constants (Eq. point charges); F = -grad E by finite
differences (Sec. 2.2); superposition; the mirror symmetry of benzene;
exactness of trilinear interpolation on trilinear fields (Sec. 5.1.1).
"""
import math

import numpy as np
import pytest

from paper_2401_14564_gb300 import synth


def one_atom(sym="C", q=0.0, xyz=(0.0, 0.0, 0.0)):
    return synth._atoms([sym], [xyz], [q])


def big_grid():
    return {"nx": 10, "ny": 10, "nz": 10, "x0": -50.0, "y0": -50.0, "z0": -50.0,
            "dx": 10.0, "dy": 10.0, "dz": 10.0, "periodic_xy": 0}


def test_lj_minimum_and_zero_follow_mixing_rules(orc):
    probe = synth.default_probe(Q=0.0)
    for sym in ("H", "C", "N", "O", "F"):
        a = one_atom(sym)
        R = synth.ELEMENTS[sym][0] + synth.ELEMENTS["O"][0]
        e = math.sqrt(synth.ELEMENTS[sym][1] * synth.ELEMENTS["O"][1])
        pts = np.array([[0.0, 0.0, R], [R, 0.0, 0.0], [0.0, R * 2 ** (-1 / 6), 0.0]])
        out, core = orc.ff_points(a, probe, big_grid(), pts)
        assert not core.any()
        # minimum of the well: E = -e_iPP, F = 0
        assert out[0, 3] == pytest.approx(-e, rel=1e-12)
        assert out[1, 3] == pytest.approx(-e, rel=1e-12)
        assert np.abs(out[0, :3]).max() < 1e-14
        # zero crossing of E at r = R / 2^(1/6)
        assert abs(out[2, 3]) < 1e-14
        # the force there is repulsive (points away from the atom)
        assert out[2, 1] > 0


def test_coulomb_constant_from_si():
    # k_e = e / (4 pi eps0) per Angstrom, in eV*A/e^2
    e, eps0 = 1.602176634e-19, 8.8541878128e-12
    ke = e / (4.0 * math.pi * eps0) / 1e-10
    assert ke == pytest.approx(14.3996454784, rel=1e-9)


def test_coulomb_point_charge(orc):
    e, eps0 = 1.602176634e-19, 8.8541878128e-12
    ke = e / (4.0 * math.pi * eps0) / 1e-10
    a = one_atom("C", q=0.3)
    a["eps"][:] = 0.0  # LJ off
    probe = synth.default_probe(Q=-0.1)
    pts = np.array([[3.0, 0.0, 0.0], [0.0, -2.0, 2.0], [1.0, 2.0, 3.0]])
    out, _ = orc.ff_points(a, probe, big_grid(), pts)
    r = np.linalg.norm(pts, axis=1)
    np.testing.assert_allclose(out[:, 3], ke * (-0.1) * 0.3 / r, rtol=1e-9)
    # opposite charges attract: the force points toward the atom
    np.testing.assert_allclose(out[:, :3], (ke * (-0.1) * 0.3 / r**3)[:, None] * pts, rtol=1e-9)
    assert np.all(np.sum(out[:, :3] * pts, axis=1) < 0)


def _grad_fd(orc, atoms, probe, grid, pts, h=1e-4):
    g = np.zeros((len(pts), 3))
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        Ep = orc.ff_points(atoms, probe, grid, pts + e)[0][:, 3]
        Em = orc.ff_points(atoms, probe, grid, pts - e)[0][:, 3]
        g[:, a] = (Ep - Em) / (2 * h)
    return g


@pytest.mark.parametrize("coul_rc,min_image", [(0.0, 0), (8.0, 0), (8.0, 1)])
def test_force_is_minus_grad_energy(orc, coul_rc, min_image):
    atoms = synth.random_molecule(17, 15)
    probe = synth.default_probe(coul_rc=coul_rc, min_image=min_image)
    grid = {"nx": 64, "ny": 64, "nz": 8, "x0": -6.4, "y0": -6.4, "z0": 0.0, "dx": 0.2, "dy": 0.2,
            "dz": 0.2, "periodic_xy": 1}
    rng = np.random.default_rng(5)
    pts = np.c_[rng.uniform(-6, 6, 60), rng.uniform(-6, 6, 60), rng.uniform(2.5, 6.0, 60)]
    out, core = orc.ff_points(atoms, probe, grid, pts)
    keep = ~core
    assert keep.sum() > 40
    g = _grad_fd(orc, atoms, probe, grid, pts)
    F = out[:, :3]
    err = np.linalg.norm(F[keep] + g[keep], axis=1) / np.maximum(np.linalg.norm(F[keep], axis=1), 1e-3)
    assert err.max() < 1e-6


def test_superposition(orc):
    A = synth.random_molecule(21, 10)
    B = synth.shift_atoms(synth.random_molecule(22, 7), 1.5, -0.5, 0.2)
    AB = synth.concat_atoms(A, B)
    probe = synth.default_probe()
    grid = {"nx": 12, "ny": 14, "nz": 6, "x0": -3.0, "y0": -3.0, "z0": 3.0, "dx": 0.5, "dy": 0.45,
            "dz": 0.3, "periodic_xy": 1}
    fa, _ = orc.make_ff(A, probe, grid)
    fb, _ = orc.make_ff(B, probe, grid)
    fab, _ = orc.make_ff(AB, probe, grid)
    np.testing.assert_allclose(fab, fa + fb, rtol=1e-12, atol=1e-14)


def test_core_floor_keeps_force_finite_and_linear(orc):
    a = one_atom("C", q=0.2)
    probe = synth.default_probe()
    R = synth.ELEMENTS["C"][0] + synth.ELEMENTS["O"][0]
    rmin = 0.5 * R
    d = np.array([0.3, -0.2, 0.5])
    d = d / np.linalg.norm(d)
    pts = np.array([0.4 * rmin * d, 0.8 * rmin * d, [0, 0, 0.0]])
    out, core = orc.ff_points(a, probe, big_grid(), pts)
    assert core.all()
    assert np.isfinite(out).all()
    # inside the floor the factor S is frozen, so F is linear in the displacement
    np.testing.assert_allclose(out[1, :3], 2.0 * out[0, :3], rtol=1e-12)
    np.testing.assert_allclose(out[2, :3], 0.0, atol=1e-300)
    np.testing.assert_allclose(out[0, 3], out[1, 3], rtol=1e-12)


def test_shifted_force_cutoff(orc):
    a = one_atom("C", q=0.3)
    a["eps"][:] = 0.0
    probe = synth.default_probe(coul_rc=8.0)
    pts = np.array([[0, 0, 7.999999], [0, 0, 8.000001], [0, 0, 9.0]])
    out, _ = orc.ff_points(a, probe, big_grid(), pts)
    # force and energy both go to zero continuously at rc
    assert abs(out[0, 2]) < 1e-7 and abs(out[0, 3]) < 1e-12
    assert out[1, 2] == 0.0 and out[2, 3] == 0.0


def test_minimum_image_equals_nearest_copy(orc):
    grid = {"nx": 40, "ny": 30, "nz": 4, "x0": 0.0, "y0": 0.0, "z0": 0.0, "dx": 0.5, "dy": 0.5,
            "dz": 0.5, "periodic_xy": 1}
    Lx, Ly = 20.0, 15.0
    a = one_atom("N", q=0.2, xyz=(19.0, 0.5, 0.0))
    probe_mi = synth.default_probe(min_image=1, coul_rc=6.0)
    probe = synth.default_probe(min_image=0, coul_rc=6.0)
    pts = np.array([[0.5, 14.5, 3.0], [1.0, 1.0, 2.5]])
    out_mi, _ = orc.ff_points(a, probe_mi, grid, pts)
    # the nearest images of the atom for the two points, placed explicitly
    img0 = one_atom("N", q=0.2, xyz=(19.0 - Lx, 0.5 + Ly, 0.0))
    img1 = one_atom("N", q=0.2, xyz=(19.0 - Lx, 0.5, 0.0))
    o0, _ = orc.ff_points(img0, probe, grid, pts[:1])
    o1, _ = orc.ff_points(img1, probe, grid, pts[1:])
    np.testing.assert_allclose(out_mi[0], o0[0], rtol=1e-12)
    np.testing.assert_allclose(out_mi[1], o1[0], rtol=1e-12)


def test_benzene_grid_mirror_symmetry(orc):
    c = synth.benzene_case()
    ff, core = orc.make_ff(c["atoms"], c["probe"], c["grid"])
    # nodes x_i = -8 + 0.2 i: x -> -x maps i -> 80 - i (i = 1..79)
    a = ff[:, :, 1:, :]
    b = ff[:, :, :0:-1, :]
    scale = np.abs(ff[..., :3]).max()
    np.testing.assert_allclose(a[..., 0], -b[..., 0], atol=1e-12 * scale)
    np.testing.assert_allclose(a[..., 1], b[..., 1], atol=1e-12 * scale)
    np.testing.assert_allclose(a[..., 2], b[..., 2], atol=1e-12 * scale)
    a = ff[:, 1:, :, :]
    b = ff[:, :0:-1, :, :]
    np.testing.assert_allclose(a[..., 1], -b[..., 1], atol=1e-12 * scale)
    np.testing.assert_allclose(a[..., 0], b[..., 0], atol=1e-12 * scale)
    # the ring plane z = 0 is a node plane: Fz vanishes there by symmetry outside the core
    assert np.abs(ff[0, ..., 2][~core[0]]).max() < 1e-12 * scale


def _trilinear_field(x, y, z, c):
    return (c[0] + c[1] * x + c[2] * y + c[3] * z + c[4] * x * y + c[5] * y * z + c[6] * x * z
            + c[7] * x * y * z)


def test_trilinear_exact_on_trilinear_fields(orc):
    grid = {"nx": 9, "ny": 7, "nz": 6, "x0": -1.0, "y0": 0.5, "z0": 2.0, "dx": 0.3, "dy": 0.25,
            "dz": 0.2, "periodic_xy": 0}
    rng = np.random.default_rng(1)
    coef = rng.standard_normal((3, 8))
    k, j, i = np.meshgrid(np.arange(6), np.arange(7), np.arange(9), indexing="ij")
    X, Y, Z = -1.0 + 0.3 * i, 0.5 + 0.25 * j, 2.0 + 0.2 * k
    ff = np.zeros((6, 7, 9, 4))
    for m in range(3):
        ff[..., m] = _trilinear_field(X, Y, Z, coef[m])
    # a trilinear field is trilinear inside every cell only if it is globally trilinear: it is
    pts = np.c_[rng.uniform(-1.0, 1.4, 200), rng.uniform(0.5, 2.0, 200), rng.uniform(2.0, 3.0, 200)]
    F, J = orc.interp_points(ff, grid, pts)
    for m in range(3):
        c = coef[m]
        x, y, z = pts.T
        np.testing.assert_allclose(F[:, m], _trilinear_field(x, y, z, c), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(J[:, m, 0], c[1] + c[4] * y + c[6] * z + c[7] * y * z, atol=1e-11)
        np.testing.assert_allclose(J[:, m, 1], c[2] + c[4] * x + c[5] * z + c[7] * x * z, atol=1e-11)
        np.testing.assert_allclose(J[:, m, 2], c[3] + c[5] * y + c[6] * x + c[7] * x * y, atol=1e-11)


def test_interp_z_clamp_and_periodic_wrap(orc):
    grid = {"nx": 8, "ny": 6, "nz": 5, "x0": 0.0, "y0": 0.0, "z0": 1.0, "dx": 0.5, "dy": 0.5,
            "dz": 0.5, "periodic_xy": 1}
    rng = np.random.default_rng(2)
    ff = rng.standard_normal((5, 6, 8, 4))
    p = np.array([[1.3, 0.7, 1.6]])
    F0, _ = orc.interp_points(ff, grid, p)
    F1, _ = orc.interp_points(ff, grid, p + np.array([[4.0, -3.0, 0.0]]))  # one period in x and y
    np.testing.assert_allclose(F0, F1, rtol=1e-12)
    # below the grid: the z0 plane; above it: the top plane (zero z-derivative)
    lo, Jlo = orc.interp_points(ff, grid, np.array([[1.0, 1.0, -3.0]]))
    np.testing.assert_allclose(lo[0], ff[0, 2, 2, :3], rtol=1e-12)
    assert np.all(Jlo[0, :, 2] == 0.0)
    hi, _ = orc.interp_points(ff, grid, np.array([[1.0, 1.0, 9.0]]))
    np.testing.assert_allclose(hi[0], ff[4, 2, 2, :3], rtol=1e-12)
    # across the periodic seam x in [3.5, 4.0): between node 7 and node 0
    seam, _ = orc.interp_points(ff, grid, np.array([[3.75, 1.0, 1.0]]))
    np.testing.assert_allclose(seam[0], 0.5 * (ff[0, 2, 7, :3] + ff[0, 2, 0, :3]), rtol=1e-12)


def test_window_with_full_period_equals_full_grid(orc):
    # a window of a laterally periodic grid, given the full grid's period for the minimum image,
    # reproduces the full grid's node values (used to check 512x512 slabs on a few patches)
    atoms = synth.concat_atoms(synth.random_molecule(31, 12), synth.shift_atoms(synth.random_molecule(32, 9), 7.0, 5.0))
    probe = synth.default_probe(min_image=1, coul_rc=6.0)
    full = {"nx": 40, "ny": 30, "nz": 5, "x0": -10.0, "y0": -7.5, "z0": 2.0, "dx": 0.5, "dy": 0.5, "dz": 0.4,
            "periodic_xy": 1}
    ff, _ = orc.make_ff(atoms, probe, full)
    win = dict(full, nx=10, ny=9, x0=-10.0 + 0.5 * 27, y0=-7.5 + 0.5 * 3, periodic_xy=0, Lx=20.0, Ly=15.0)
    fw, _ = orc.make_ff(atoms, probe, win)
    np.testing.assert_allclose(fw, ff[:, 3:12, 27:37], rtol=1e-12, atol=1e-15)
