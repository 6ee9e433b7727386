"""Pins of the oracle's relaxed scan (tip springs of Eq. F_tip, Eq. F_PP, FIRE
relaxation of Sec. 5.1.1 and the tip-force readout Fz = -F^T_{R,z} of Sec. 2.1).

The expected values come from problems with a known answer: an empty sample
(the PP rests at d0), a constant sample force (a 1D root in |d|, solved here by
bisection), a single atom straight below the tip (a 1D root along the axis),
the stiff-spring limit (the unrelaxed lookup), and the mirror symmetry of
benzene.  Grid -> grid-free convergence is checked to be second order.
"""
import math

import numpy as np
import pytest

from paper_2401_14564_gb300 import synth

NM = 1.0 / (1.602176634e-19 * 1e20)  # 1 N/m in eV/A^2, from SI


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


def flat_grid(c=(0.0, 0.0, 0.0)):
    grid = {"nx": 8, "ny": 8, "nz": 8, "x0": -4.0, "y0": -4.0, "z0": 0.0, "dx": 1.0, "dy": 1.0,
            "dz": 1.0, "periodic_xy": 1}
    ff = np.zeros((8, 8, 8, 4))
    ff[..., 0], ff[..., 1], ff[..., 2] = c
    return grid, ff


def scan3(nz=6):
    return {"nx": 3, "ny": 2, "nz": nz, "x0": -1.0, "y0": 0.5, "px": 0.7, "py": 0.4, "z_top": 6.0, "dz": 0.1}


def test_empty_sample_rests_at_d0(orc):
    grid, ff = flat_grid()
    tip = synth.default_tip(d0x=0.3, d0y=-0.2)
    s = scan3()
    r = orc.relax_scan(ff, grid, None, None, s, tip, synth.default_fire())
    assert (r["iters"] == 0).all()
    d0z = -math.sqrt(4.0**2 - 0.3**2 - 0.2**2)
    for k in range(s["nz"]):
        for j in range(2):
            for i in range(3):
                np.testing.assert_allclose(r["pos"][k, j, i], [s["x0"] + i * 0.7 + 0.3, 0.5 + j * 0.4 - 0.2,
                                                               6.0 - 0.1 * k + d0z], atol=1e-12)
    assert np.abs(r["fz"]).max() < 1e-12


@pytest.mark.parametrize("c", [(0.004, -0.003, -0.03), (-0.002, 0.0, -0.08), (0.0, 0.001, 0.01)])
def test_constant_sample_force(orc, c):
    grid, ff = flat_grid(c)
    tip = synth.default_tip()
    kx, ky, kR, R0 = 0.25 * NM, 0.25 * NM, 20.0 * NM, 4.0

    def d_of(rho):
        s = kR * (1.0 - R0 / rho)
        return np.array([c[0] / (s + kx), c[1] / (s + ky), c[2] / s])

    lo, hi = (R0 + 1e-9, R0 + 1.0) if c[2] < 0 else (R0 - 1.0, R0 - 1e-9)
    rho = bisect(lambda r: np.linalg.norm(d_of(r)) - r, lo, hi)
    d = d_of(rho)
    assert d[2] < 0
    r = orc.relax_scan(ff, grid, None, None, scan3(3), tip, synth.default_fire())
    assert r["ok"].all()
    s = scan3(3)
    for k in range(3):
        anchor = np.array([s["x0"] + 0.7, s["y0"] + 0.4, 6.0 - 0.1 * k])
        np.testing.assert_allclose(r["pos"][k, 1, 1] - anchor, d, atol=1e-9)
    # Fz = -F^T_{R,z} balances the sample force exactly
    np.testing.assert_allclose(r["fz"], c[2], rtol=1e-9)


def test_single_atom_on_axis(orc):
    atoms = synth._atoms(["C"], [(0.0, 0.0, 0.0)], [0.1])
    probe = synth.default_probe(Q=-0.2)
    e = math.sqrt(synth.ELEMENTS["C"][1] * synth.ELEMENTS["O"][1])
    R = synth.ELEMENTS["C"][0] + synth.ELEMENTS["O"][0]
    ke = 1.602176634e-19 / (4.0 * math.pi * 8.8541878128e-12) / 1e-10
    kR = 20.0 * NM

    def Fz_atom(h):  # force on the PP at height h straight above the atom
        return 12 * e * ((R / h) ** 12 - (R / h) ** 6) / h + ke * (-0.2) * 0.1 / h**2

    s = {"nx": 1, "ny": 1, "nz": 25, "x0": 0.0, "y0": 0.0, "px": 0.1, "py": 0.1, "z_top": 8.5, "dz": 0.1}
    grid = {"nx": 8, "ny": 8, "nz": 8, "x0": -40.0, "y0": -40.0, "z0": -40.0, "dx": 10.0, "dy": 10.0,
            "dz": 10.0, "periodic_xy": 0}
    r = orc.relax_scan(None, grid, atoms, probe, s, synth.default_tip(), synth.default_fire())
    for k in range(s["nz"]):
        za = 8.5 - 0.1 * k
        rho = bisect(lambda rho: kR * (rho - 4.0) + Fz_atom(za - rho), 3.0, 5.0)
        np.testing.assert_allclose(r["pos"][k, 0, 0], [0.0, 0.0, za - rho], atol=1e-9)
        np.testing.assert_allclose(r["fz"][k, 0, 0], Fz_atom(za - rho), rtol=1e-7, atol=1e-12)


def test_stiff_spring_limit_is_unrelaxed_lookup(orc):
    c = synth.benzene_case()
    ff, _ = orc.make_ff(c["atoms"], c["probe"], c["grid"])
    tip = synth.default_tip(kx=1e4, ky=1e4, kR=1e4)
    s = dict(c["scan"], nx=8, ny=8, x0=-2.0, y0=-1.5, px=0.5, py=0.45)
    # the FIRE step must respect the stiffest spring: omega = sqrt(624 eV/A^2) = 25, so dt = 0.04
    r = orc.relax_scan(ff, c["grid"], None, None, s, tip, synth.default_fire(ftol=1e-9, max_iter=5000, dt0=0.04,
                                                                             dt_max=0.04))
    k = np.arange(s["nz"])[:, None, None]
    j = np.arange(s["ny"])[None, :, None]
    i = np.arange(s["nx"])[None, None, :]
    pts = np.stack(np.broadcast_arrays(s["x0"] + i * s["px"], s["y0"] + j * s["py"],
                                       s["z_top"] - k * s["dz"] - 4.0), axis=-1).reshape(-1, 3)
    F, _ = orc.interp_points(ff, c["grid"], pts)
    Fmax = np.abs(F).max()
    kint = 1e4 * NM
    assert np.abs(r["pos"].reshape(-1, 3) - pts).max() < 2 * Fmax / kint
    np.testing.assert_allclose(r["fz"].reshape(-1), F[:, 2], atol=1e-3 * Fmax)


def test_benzene_newton_residual_and_image_symmetry(orc):
    c = synth.benzene_case()
    r = orc.forward(c)
    assert r["ok"].all()
    # Newton polish: |G| < 1e-11 eV/A at every pixel and height
    assert r["res"].shape == r["fz"].shape
    fz, df = r["fz"], r["df"]
    scale = np.abs(fz).max()
    stable = r["lam"] > 0.01
    mx = (np.abs(fz - fz[:, :, ::-1]) < 1e-8 * scale) | ~(stable & stable[:, :, ::-1])
    my = (np.abs(fz - fz[:, ::-1, :]) < 1e-8 * scale) | ~(stable & stable[:, ::-1, :])
    assert mx.mean() > 0.999 and my.mean() > 0.999
    assert np.abs(df - df[:, :, ::-1]).max() < 1e-6 * np.abs(df).max() or mx.all()
    # the attractive far field gives negative df, the repulsive close range positive
    assert df[0].mean() < 0 < df[-1].max()


def test_fire_converged_start_costs_no_iterations(orc):
    grid, ff = flat_grid((0.0, 0.0, -0.02))
    r = orc.relax_scan(ff, grid, None, None, scan3(4), synth.default_tip(), synth.default_fire())
    # after the first height the warm start (p* - dz z) is already the solution
    assert (r["iters"][0] > 0).all()
    assert (r["iters"][1:] == 0).all()


def test_grid_converges_to_grid_free_second_order(orc):
    c = synth.benzene_case()
    # z_top off the node planes: with PP heights on node planes the cell fraction is ~0 and the
    # interpolation error degenerates to O(h * offset), hiding the O(h^2) order
    s = dict(c["scan"], nx=6, ny=5, x0=-1.3, y0=-1.1, px=0.45, py=0.5, nz=12, z_top=9.037)
    free = orc.relax_scan(None, c["grid"], c["atoms"], c["probe"], s, c["tip"], c["fire"])
    errs = []
    hs = (0.2, 0.1, 0.05, 0.025)
    for h in hs:
        n = int(round(8.0 / h))
        g = {"nx": n, "ny": n, "nz": int(round(4.0 / h)), "x0": -4.0, "y0": -4.0, "z0": 2.5, "dx": h, "dy": h,
             "dz": h, "periodic_xy": 0}
        ff, core = orc.make_ff(c["atoms"], c["probe"], g)
        assert not core.any()
        r = orc.relax_scan(ff, g, None, None, s, c["tip"], c["fire"])
        errs.append(np.sqrt(np.mean((r["fz"] - free["fz"]) ** 2)))
    # least-squares order of convergence over an 8x range of spacings: 2 for trilinear, 1 if broken
    order = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    assert order > 1.7, (order, errs)


@pytest.mark.parametrize("alpha,dt", [(1.0, 0.4), (1.0, 1.0), (0.0, 0.4), (0.0, 1.0)])
def test_fire_special_cases_step_by_step(orc, alpha, dt):
    # FIRE's velocity mixing v <- (1 - alpha) v + alpha |v| F/|F| has two limits with a simpler
    # rule: alpha = 1 turns every downhill velocity onto the force direction at unchanged speed,
    # alpha = 0 leaves it alone (plain semi-implicit Euler); an uphill step (F.v <= 0) stops the
    # probe and scales the step by f_dec.  With f_alpha = 1 and the step growth held off, the
    # first positions from rest under a constant sample force follow from those rules and the tip
    # force law (Eq. F_tip) alone; dt = 1 overshoots, so the uphill reset is exercised too.
    c = np.array([0.004, -0.003, -0.03])
    grid, ff = flat_grid(tuple(c))
    tip = synth.default_tip(d0x=0.2, d0y=-0.1)
    kx, ky, kR, R0 = 0.25 * NM, 0.25 * NM, 20.0 * NM, 4.0
    d0 = np.array([0.2, -0.1, -math.sqrt(R0**2 - 0.2**2 - 0.1**2)])

    def force(d):
        dn = np.linalg.norm(d)
        return -kR * (dn - R0) / dn * d - np.array([kx, ky, 0.0]) * (d - d0) + c

    fire = synth.default_fire(alpha0=alpha, f_alpha=1.0, n_min=10**6, dt0=dt, dt_max=dt, ftol=1e-12, mass=1.3)
    s = scan3(1)
    resets = 0
    for n in range(1, 9):
        d, v, h = d0.copy(), np.zeros(3), dt
        for it in range(n):
            F = force(d)
            if it > 0:
                if F @ v > 0.0:
                    v = np.linalg.norm(v) * F / np.linalg.norm(F) if alpha == 1.0 else v
                else:
                    v = np.zeros(3)
                    h *= fire["f_dec"]
                    resets += n == 8
            v = v + h * F / fire["mass"]
            d = d + h * v
        r = orc.relax_scan(ff, grid, None, None, s, tip, dict(fire, max_iter=n), polish_tol=0.0)
        assert (r["iters"] == n).all()
        for j in range(s["ny"]):
            for i in range(s["nx"]):
                anchor = np.array([s["x0"] + i * s["px"], s["y0"] + j * s["py"], s["z_top"]])
                np.testing.assert_allclose(r["pos"][0, j, i] - anchor, d, atol=1e-12, rtol=0)
    if dt == 1.0:
        assert resets > 0  # the overshooting step size takes the uphill branch within 8 steps


def test_fire_step_growth_schedule_on_an_axial_force(orc):
    # A sample force along z under a tip hanging straight down (d0 = (0, 0, -R0)) keeps the probe
    # on the axis, where the tip force is linear in the deflection, F = c_z - kR e_z (Eq. F_tip with
    # |d| = R0 - e_z).  The velocity then stays parallel to the force, FIRE's mixing leaves it
    # unchanged, and while the probe has not yet passed the minimum every step is downhill.  The
    # positions are those of semi-implicit Euler under the step schedule of Bitzek et al.: dt0 for
    # the first n_min + 1 downhill steps after the first one, then growing by f_inc per step up to
    # dt_max (n_min = 2, f_inc = 1.25 from 0.2 reaches the 0.5 cap at the ninth update).
    cz = -0.03
    kR = 1.0 * NM  # soft radial spring: a quarter period of 6.3 time units, past the 12 steps' 4.2
    grid, ff = flat_grid((0.0, 0.0, cz))
    tip = synth.default_tip(kR=1.0)
    dt0, dt_max, f_inc, n_min, mass = 0.2, 0.5, 1.25, 2, 1.0
    fire = synth.default_fire(dt0=dt0, dt_max=dt_max, f_inc=f_inc, n_min=n_min, f_alpha=0.9, alpha0=0.3,
                              ftol=1e-12, mass=mass)
    s = scan3(1)
    for n in range(1, 13):
        e, v = 0.0, 0.0
        for it in range(n):
            h = min(dt0 * f_inc ** max(0, it - n_min - 1), dt_max)
            v += h * (cz - kR * e) / mass
            e += h * v
        assert e > cz / kR  # still above the minimum: every step was downhill
        r = orc.relax_scan(ff, grid, None, None, s, tip, dict(fire, max_iter=n), polish_tol=0.0)
        assert (r["iters"] == n).all()
        for j in range(s["ny"]):
            for i in range(s["nx"]):
                anchor = np.array([s["x0"] + i * s["px"], s["y0"] + j * s["py"], s["z_top"]])
                np.testing.assert_allclose(r["pos"][0, j, i] - anchor, [0.0, 0.0, -4.0 + e], atol=1e-12, rtol=0)
    assert min(dt0 * f_inc ** max(0, 11 - n_min - 1), dt_max) == dt_max  # the cap was reached


def fire_by_hand(force, d0, fire, n):
    """Bitzek et al.'s FIRE written out for n position updates from rest (the deflection-free
    start d0): returns the final d, the number of updates taken with a grown step, and the number
    of those that followed an uphill reset."""
    d, v = d0.copy(), np.zeros(3)
    dt, alpha, npos, grown, regrown, reset = fire["dt0"], fire["alpha0"], 0, 0, 0, False
    for it in range(n):
        F = force(d)
        if it > 0:
            if F @ v > 0.0:
                v = (1.0 - alpha) * v + alpha * np.linalg.norm(v) * F / np.linalg.norm(F)
                if npos > fire["n_min"]:
                    dt = min(dt * fire["f_inc"], fire["dt_max"])
                    alpha *= fire["f_alpha"]
                    grown += 1
                    regrown += reset
                npos += 1
            else:
                v = np.zeros(3)
                dt *= fire["f_dec"]
                alpha = fire["alpha0"]
                npos = 0
                reset = True
        v = v + dt * F / fire["mass"]
        d = d + dt * v
    return d, grown, regrown


@pytest.mark.parametrize("f_alpha,kR,dt0,n_min,steps", [(0.9, 1.0, 0.2, 2, 12), (0.99, 1.0, 0.2, 2, 12),
                                                         (0.9, 20.0, 0.5, 1, 24)])
def test_fire_growth_and_alpha_decay_step_by_step(orc, f_alpha, kR, dt0, n_min, steps):
    # A lateral + vertical constant sample force under a tilted tip: the probe moves off the axis,
    # so the velocity mixing acts on every downhill step, and after more than n_min downhill steps
    # the step grows and alpha decays.  Positions after each number of updates against FIRE
    # written out by hand (Bitzek et al. 2006) and Eq. F_tip, to 1e-12 A; the same run with alpha
    # held (f_alpha = 1) ends elsewhere, so the decay is seen.  With the 20 N/m radial spring and
    # dt0 = 0.5 the probe overshoots: the uphill reset is taken and the count of downhill steps
    # starts again before the step grows anew.
    c = np.array([0.012, -0.008, -0.03])
    grid, ff = flat_grid(tuple(c))
    tip = synth.default_tip(d0x=0.2, d0y=-0.1, kR=kR)
    kx, ky, kRe, R0 = 0.25 * NM, 0.25 * NM, kR * NM, 4.0
    d0 = np.array([0.2, -0.1, -math.sqrt(R0**2 - 0.2**2 - 0.1**2)])

    def force(d):
        dn = np.linalg.norm(d)
        return -kRe * (dn - R0) / dn * d - np.array([kx, ky, 0.0]) * (d - d0) + c

    fire = synth.default_fire(dt0=dt0, dt_max=2.5 * dt0, f_inc=1.25, n_min=n_min, f_alpha=f_alpha, alpha0=0.3,
                              ftol=1e-12, mass=1.0)
    s = scan3(1)
    for n in range(1, steps + 1):
        d, grown, regrown = fire_by_hand(force, d0, fire, n)
        r = orc.relax_scan(ff, grid, None, None, s, tip, dict(fire, max_iter=n), polish_tol=0.0)
        assert (r["iters"] == n).all()
        for j in range(s["ny"]):
            for i in range(s["nx"]):
                anchor = np.array([s["x0"] + i * s["px"], s["y0"] + j * s["py"], s["z_top"]])
                np.testing.assert_allclose(r["pos"][0, j, i] - anchor, d, atol=1e-12, rtol=0)
    assert grown >= 6  # the growth branch was taken on many of the updates
    if kR > 1.0:
        assert regrown >= 2  # ... also after an uphill reset
    held, _, _ = fire_by_hand(force, d0, dict(fire, f_alpha=1.0), steps)
    assert np.linalg.norm(held - d) > 1e-6
