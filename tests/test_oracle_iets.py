"""Pins of the oracle's IETS map (Sec. 3.3): stiffness eigenvalues of the probe particle.

K = -(J + J^T)/2 at the relaxed position.  Closed forms: at rest K = diag(kx, ky, kR); under a
constant sample force (0, 0, c) the springs alone give kx + s, ky + s, kR with
s = kR (1 - R0/|d|); a single atom straight below adds -f(h)/h laterally and -f'(h) axially for
its radial force f(h).  Mode energies hbar sqrt(lambda/m) from SI constants.
"""
import math

import numpy as np
import pytest

from paper_2401_14564_gb300 import synth

NM = 1.0 / (1.602176634e-19 * 1e20)  # 1 N/m in eV/A^2
HBAR, EV, AMU = 1.054571817e-34, 1.602176634e-19, 1.66053906660e-27


def bisect(f, lo, hi, n=200):
    flo = f(lo)
    for _ in range(n):
        mid = 0.5 * (lo + hi)
        fm = f(mid)
        if (fm > 0) == (flo > 0):
            lo, flo = mid, fm
        else:
            hi = mid
    return 0.5 * (lo + hi)


def flat(c=(0.0, 0.0, 0.0)):
    g = {"nx": 8, "ny": 8, "nz": 8, "x0": -4.0, "y0": -4.0, "z0": 0.0, "dx": 1.0, "dy": 1.0, "dz": 1.0,
         "periodic_xy": 1}
    ff = np.zeros((8, 8, 8, 4))
    ff[..., 0], ff[..., 1], ff[..., 2] = c
    return g, ff


def scan1(nz=3, z_top=6.0):
    return {"nx": 2, "ny": 1, "nz": nz, "x0": -0.5, "y0": 0.25, "px": 0.5, "py": 0.5, "z_top": z_top, "dz": 0.1}


def test_at_rest_the_stiffness_is_the_springs(orc):
    g, ff = flat()
    tip = synth.default_tip(kx=0.3, ky=0.2)
    s = scan1()
    r = orc.relax_scan(ff, g, None, None, s, tip, synth.default_fire())
    eig, hw = orc.iets(ff, g, None, None, s, tip, r["pos"], mass_amu=16.0)
    want = np.sort(np.array([0.3, 0.2, 20.0]) * NM)
    np.testing.assert_allclose(eig.reshape(-1, 3), np.broadcast_to(want, (eig.size // 3, 3)), rtol=1e-9)
    # hbar omega from k in N/m directly: sqrt(k / m) rad/s
    e_mev = [HBAR * math.sqrt(k / (16.0 * AMU)) / EV * 1e3 for k in (0.2, 0.3, 20.0)]
    np.testing.assert_allclose(hw.reshape(-1, 3), np.broadcast_to(e_mev, (hw.size // 3, 3)), rtol=1e-9)


def test_constant_force_deflected_springs(orc):
    c = -0.05
    g, ff = flat((0.0, 0.0, c))
    tip = synth.default_tip()
    kx, kR, R0 = 0.25 * NM, 20.0 * NM, 4.0
    rho = bisect(lambda r: kR * (r - R0) * 1.0 + c, R0, R0 + 1.0)  # on the axis: kR (rho - R0) = -c
    sR = kR * (1.0 - R0 / rho)
    r = orc.relax_scan(ff, g, None, None, scan1(), tip, synth.default_fire())
    eig, _ = orc.iets(ff, g, None, None, scan1(), tip, r["pos"])
    np.testing.assert_allclose(eig.reshape(-1, 3), np.broadcast_to([kx + sR, kx + sR, kR], (6, 3)), rtol=1e-8)


def test_single_atom_below_adds_its_curvature(orc):
    atoms = synth._atoms(["C"], [(0.0, 0.0, 0.0)], [0.1])
    probe = synth.default_probe(Q=-0.2)
    e = math.sqrt(synth.ELEMENTS["C"][1] * synth.ELEMENTS["O"][1])
    R = synth.ELEMENTS["C"][0] + synth.ELEMENTS["O"][0]
    ke = 1.602176634e-19 / (4.0 * math.pi * 8.8541878128e-12) / 1e-10
    kx, kR, R0 = 0.25 * NM, 20.0 * NM, 4.0

    def f(h):  # radial force on the PP at distance h from the atom
        return 12 * e * ((R / h) ** 12 - (R / h) ** 6) / h + ke * (-0.2) * 0.1 / h**2

    s = {"nx": 1, "ny": 1, "nz": 6, "x0": 0.0, "y0": 0.0, "px": 0.1, "py": 0.1, "z_top": 8.0, "dz": 0.2}
    grid = {"nx": 8, "ny": 8, "nz": 8, "x0": -40.0, "y0": -40.0, "z0": -40.0, "dx": 10.0, "dy": 10.0,
            "dz": 10.0, "periodic_xy": 0}
    r = orc.relax_scan(None, grid, atoms, probe, s, synth.default_tip(), synth.default_fire())
    eig, _ = orc.iets(None, grid, atoms, probe, s, synth.default_tip(), r["pos"])
    for k in range(s["nz"]):
        za = 8.0 - 0.2 * k
        rho = bisect(lambda rho: kR * (rho - R0) + f(za - rho), 3.0, 5.0)
        h = za - rho
        sR = kR * (1.0 - R0 / rho)
        fp = (f(h + 1e-5) - f(h - 1e-5)) / 2e-5
        lat, ax = kx + sR - f(h) / h, kR - fp
        np.testing.assert_allclose(sorted(eig[k, 0, 0]), sorted([lat, lat, ax]), rtol=1e-6, atol=1e-9)


def test_coupled_asymmetric_field_against_a_library_eigensolver(orc):
    # a linear sample field F = A (p - p_ref) with a non-symmetric, strongly coupled A is
    # interpolated exactly by the trilinear grid, so at the tip's rest offset (0, 0, -R0) the
    # stiffness is K = diag(kx, ky, kR) - (A + A^T)/2 (the springs' part is the at-rest pin
    # above); its eigenvalues come from numpy's symmetric eigensolver
    A = np.array([[0.010, 0.021, -0.015], [-0.004, 0.008, 0.030], [0.012, -0.020, 0.050]])
    g = {"nx": 8, "ny": 8, "nz": 8, "x0": -4.0, "y0": -4.0, "z0": 0.0, "dx": 1.0, "dy": 1.0, "dz": 1.0,
         "periodic_xy": 0}
    p_ref = np.array([0.3, -0.2, 2.5])
    zz, yy, xx = np.meshgrid(g["z0"] + np.arange(8.0), g["y0"] + np.arange(8.0), g["x0"] + np.arange(8.0),
                             indexing="ij")
    nodes = np.stack([xx, yy, zz], -1)
    ff = np.zeros((8, 8, 8, 4))
    ff[..., :3] = (nodes - p_ref) @ A.T
    tip = synth.default_tip()
    s = scan1(nz=2)
    pos = np.empty((s["nz"], s["ny"], s["nx"], 3))
    for k in range(s["nz"]):
        for i in range(s["nx"]):
            pos[k, 0, i] = [s["x0"] + i * s["px"], s["y0"], s["z_top"] - k * s["dz"] - 4.0]
    eig, _ = orc.iets(ff, g, None, None, s, tip, pos, mass_amu=16.0)
    K = np.diag([0.25 * NM, 0.25 * NM, 20.0 * NM]) - 0.5 * (A + A.T)
    want = np.linalg.eigvalsh(K)
    assert abs(want[0] - want[1]) > 1e-3  # a genuinely coupled lateral pair
    np.testing.assert_allclose(eig.reshape(-1, 3), np.broadcast_to(want, (eig.size // 3, 3)), rtol=1e-12,
                               atol=1e-14)
