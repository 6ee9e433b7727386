"""Pins of the oracle's tricubic interpolation of the grid potential (Sec.
5.1.1 step 2: tricubic interpolation of the potential, suggested by the paper
for larger spacings without stored forces).

Reading: tensor product of 1D cubic convolution (Catmull-Rom) through the
node energies; F = -grad of the interpolant.  Fixed independently of the
oracle's formula by:
  - interpolation: E equals the node value at every node, and F there is
    minus the central difference of the node energies;
  - reproduction: any field of degree <= 2 in each coordinate is reproduced
    exactly with its gradient and Hessian, while a cubic is not (so a wrong
    weight cannot hide);
  - C1: F is continuous across cell faces;
  - F = -grad E and J = dF/dp by central differences of the interpolant;
  - periodicity in x and y;
  - convergence to the grid-free model at second order in the spacing, and
    the relaxed scan converging to the grid-free relaxed scan;
  - the adjoint on an energy grid (atom, tip and charge gradients and the
    node-energy adjoint) against central differences of the whole forward
    pass, the charge scaling identity and a rigid shift of all atoms.
"""
import numpy as np
import pytest

from paper_2401_14564_gb300 import synth


def grid(nx=12, ny=10, nz=9, d=(0.3, 0.25, 0.2), periodic=0):
    return {"nx": nx, "ny": ny, "nz": nz, "x0": -1.0, "y0": 0.5, "z0": 2.0, "dx": d[0], "dy": d[1], "dz": d[2],
            "periodic_xy": periodic, "interp": 1}


def sample(g, fn):
    k, j, i = np.meshgrid(np.arange(g["nz"]), np.arange(g["ny"]), np.arange(g["nx"]), indexing="ij")
    x, y, z = g["x0"] + i * g["dx"], g["y0"] + j * g["dy"], g["z0"] + k * g["dz"]
    ff = np.zeros((g["nz"], g["ny"], g["nx"], 4))
    ff[..., 3] = fn(x, y, z)
    return ff


def interior_points(g, n, seed):
    """Points whose 4-node stencil lies inside the grid on every axis."""
    rng = np.random.default_rng(seed)
    lo = np.array([g["x0"] + 1.0 * g["dx"], g["y0"] + 1.0 * g["dy"], g["z0"] + 1.0 * g["dz"]])
    hi = np.array([g["x0"] + (g["nx"] - 2.0) * g["dx"], g["y0"] + (g["ny"] - 2.0) * g["dy"],
                   g["z0"] + (g["nz"] - 2.0) * g["dz"]])
    return rng.uniform(lo, hi - 1e-9, size=(n, 3))


def quad_field(x, y, z):
    return (0.3 + 1.2 * x - 0.7 * x**2) * (1.1 - 0.4 * y + 0.9 * y**2) * (0.5 + 0.8 * z - 0.3 * z**2)


def quad_grad_hess(p):
    x, y, z = p
    X, dX, ddX = 0.3 + 1.2 * x - 0.7 * x**2, 1.2 - 1.4 * x, -1.4
    Y, dY, ddY = 1.1 - 0.4 * y + 0.9 * y**2, -0.4 + 1.8 * y, 1.8
    Z, dZ, ddZ = 0.5 + 0.8 * z - 0.3 * z**2, 0.8 - 0.6 * z, -0.6
    g = np.array([dX * Y * Z, X * dY * Z, X * Y * dZ])
    H = np.array([[ddX * Y * Z, dX * dY * Z, dX * Y * dZ],
                  [dX * dY * Z, X * ddY * Z, X * dY * dZ],
                  [dX * Y * dZ, X * dY * dZ, X * Y * ddZ]])
    return X * Y * Z, g, H


def test_interpolates_node_values_with_central_difference_forces(orc):
    g = grid()
    rng = np.random.default_rng(3)
    ff = np.zeros((g["nz"], g["ny"], g["nx"], 4))
    ff[..., 3] = rng.standard_normal((g["nz"], g["ny"], g["nx"]))
    E = ff[..., 3]
    for (k, j, i) in [(3, 4, 5), (1, 1, 1), (6, 7, 9)]:
        p = np.array([[g["x0"] + i * g["dx"], g["y0"] + j * g["dy"], g["z0"] + k * g["dz"]]])
        e = orc.interp_energy_points(ff, g, p)[0]
        F, _ = orc.interp_points(ff, g, p)
        assert e == pytest.approx(E[k, j, i], abs=1e-12)
        want = -np.array([(E[k, j, i + 1] - E[k, j, i - 1]) / (2 * g["dx"]),
                          (E[k, j + 1, i] - E[k, j - 1, i]) / (2 * g["dy"]),
                          (E[k + 1, j, i] - E[k - 1, j, i]) / (2 * g["dz"])])
        assert np.allclose(F[0], want, rtol=1e-12, atol=1e-12)


def test_reproduces_degree_two_fields_exactly_but_not_cubics(orc):
    g = grid()
    ff = sample(g, quad_field)
    pts = interior_points(g, 50, 4)
    E = orc.interp_energy_points(ff, g, pts)
    F, J = orc.interp_points(ff, g, pts)
    for n, p in enumerate(pts):
        e, grad, H = quad_grad_hess(p)
        assert E[n] == pytest.approx(e, abs=1e-12)
        assert np.allclose(F[n], -grad, atol=1e-11)
        assert np.allclose(J[n], -H, atol=1e-10)
    cub = sample(g, lambda x, y, z: x**3)
    Ec = orc.interp_energy_points(cub, g, pts)
    assert np.abs(Ec - pts[:, 0] ** 3).max() > 1e-4


def test_forces_are_continuous_across_cell_faces(orc):
    g = grid()
    rng = np.random.default_rng(5)
    ff = np.zeros((g["nz"], g["ny"], g["nx"], 4))
    ff[..., 3] = rng.standard_normal((g["nz"], g["ny"], g["nx"]))
    eps = 1e-9
    for axis, key, d in ((0, "x0", "dx"), (1, "y0", "dy"), (2, "z0", "dz")):
        p = np.array([0.05, 1.23, 2.77])
        face = g[key] + 4 * g[d]
        a, b = p.copy(), p.copy()
        a[axis], b[axis] = face - eps, face + eps
        Fa, _ = orc.interp_points(ff, g, a[None])
        Fb, _ = orc.interp_points(ff, g, b[None])
        assert np.allclose(Fa, Fb, atol=1e-6), axis


def test_force_is_minus_gradient_and_jacobian_matches_differences(orc):
    g = grid()
    rng = np.random.default_rng(6)
    ff = np.zeros((g["nz"], g["ny"], g["nx"], 4))
    ff[..., 3] = rng.standard_normal((g["nz"], g["ny"], g["nx"]))
    pts = interior_points(g, 30, 7)
    F, J = orc.interp_points(ff, g, pts)
    h = 1e-6
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        dE = (orc.interp_energy_points(ff, g, pts + e) - orc.interp_energy_points(ff, g, pts - e)) / (2 * h)
        assert np.allclose(F[:, a], -dE, atol=1e-6)
        Fp, _ = orc.interp_points(ff, g, pts + e)
        Fm, _ = orc.interp_points(ff, g, pts - e)
        assert np.allclose(J[:, :, a], (Fp - Fm) / (2 * h), atol=1e-5)


def test_periodic_in_x_and_y(orc):
    g = grid(periodic=1)
    rng = np.random.default_rng(8)
    ff = np.zeros((g["nz"], g["ny"], g["nx"], 4))
    ff[..., 3] = rng.standard_normal((g["nz"], g["ny"], g["nx"]))
    p = np.array([[g["x0"] + 0.17, g["y0"] + 0.31, 2.9]])
    E0 = orc.interp_energy_points(ff, g, p)
    F0, _ = orc.interp_points(ff, g, p)
    for sh in ([g["nx"] * g["dx"], 0, 0], [0, -g["ny"] * g["dy"], 0], [2 * g["nx"] * g["dx"], g["ny"] * g["dy"], 0]):
        E1 = orc.interp_energy_points(ff, g, p + sh)
        F1, _ = orc.interp_points(ff, g, p + sh)
        assert E1[0] == pytest.approx(E0[0], abs=1e-12)
        assert np.allclose(F0, F1, atol=1e-12)
    # across the periodic seam the stencil wraps: a point half a cell left of x0 uses node nx-1
    q = np.array([[g["x0"] - 0.5 * g["dx"], 1.0, 2.9]])
    Eq = orc.interp_energy_points(ff, g, q)
    Es = orc.interp_energy_points(ff, g, q + [g["nx"] * g["dx"], 0, 0])
    assert Eq[0] == pytest.approx(Es[0], abs=1e-12)


def test_converges_to_the_grid_free_force_at_second_order(orc):
    atoms = synth.random_molecule(31, 12)
    probe = synth.default_probe()
    rng = np.random.default_rng(9)
    pts = np.column_stack([rng.uniform(-2, 2, 40), rng.uniform(-2, 2, 40), rng.uniform(3.3, 4.3, 40)])
    ref, _ = orc.ff_points(atoms, probe, {**grid(), "interp": 0}, pts)
    errs = []
    hs = (0.2, 0.1, 0.05)
    for h in hs:
        n = int(round(12.0 / h))
        nz = int(round(4.0 / h)) + 1
        g = {"nx": n, "ny": n, "nz": nz, "x0": -6.0, "y0": -6.0, "z0": 1.8, "dx": h, "dy": h, "dz": h,
             "periodic_xy": 0, "interp": 1}
        ff, _ = orc.make_ff(atoms, probe, g)
        F, _ = orc.interp_points(ff, g, pts)
        errs.append(np.abs(F - ref[:, :3]).max())
    order = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    assert order > 1.8, (errs, order)


def test_relaxed_scan_converges_to_the_grid_free_scan(orc):
    c = synth.small_case(seed=12, n_atoms=8, nxy=40, nz=40, scan_px=6, nz_scan=10, d=0.2)
    c["scan"]["z_top"] += 0.037  # heights off the node planes
    fire = synth.parity_fire()
    free = orc.relax_scan(None, c["grid"], c["atoms"], c["probe"], c["scan"], c["tip"], fire)
    errs = []
    hs = (0.2, 0.1, 0.05)
    g0 = c["grid"]
    lx, ly, lz = g0["nx"] * g0["dx"], g0["ny"] * g0["dy"], (g0["nz"] - 1) * g0["dz"]
    for h in hs:
        g = dict(g0, nx=int(round(lx / h)), ny=int(round(ly / h)), nz=int(round(lz / h)) + 1, dx=h, dy=h, dz=h,
                 interp=1)
        ff, _ = orc.make_ff(c["atoms"], c["probe"], g)
        r = orc.relax_scan(ff, g, c["atoms"], c["probe"], c["scan"], c["tip"], fire)
        errs.append(np.abs(r["pos"] - free["pos"]).max())
    order = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    assert errs[-1] < 1e-3 and order > 1.8, (errs, order)


def energy_grid_case(qzz=0.0):
    from test_oracle_adjoint import tiny_case

    c = tiny_case()
    c["grid"] = dict(c["grid"], interp=1)
    c["probe"] = dict(c["probe"], Qzz=qzz)
    return c


E_PARAMS = [("x", 0, 1e-4), ("y", 2, 1e-4), ("z", 1, 1e-4), ("z", 4, 1e-4), ("q", 3, 1e-4), ("R", 5, 1e-4),
            ("eps", 0, 1e-6), ("kx", None, 1e-4), ("ky", None, 1e-4), ("kR", None, 1e-3), ("Q", None, 1e-4),
            ("Qzz", None, 1e-4)]


def _perturbed(c, what, idx, h):
    import copy

    c2 = copy.deepcopy(c)
    if what in ("x", "y", "z", "q", "R", "eps"):
        c2["atoms"][what] = c2["atoms"][what].copy()
        c2["atoms"][what][idx] += h
    elif what in ("Q", "Qzz"):
        c2["probe"][what] += h
    else:
        c2["tip"][what] += h
    return c2


def _loss(orc, c):
    r = orc.forward(c, polish_tol=1e-13)
    assert r["ok"].all()
    return float((c["w"] * r["df"]).sum()), r


@pytest.mark.parametrize("qzz", [0.0, -0.05])
def test_energy_grid_adjoint_matches_central_differences(orc, qzz):
    # the interpolated force is C1 but its Jacobian jumps on cell faces, so a relaxed point that
    # crosses a face within +-h leaves an O(h) difference error: bar 1e-4 of the gradient's scale
    c = energy_grid_case(qzz)
    _, r = _loss(orc, c)
    g = orc.backward(r["ff"], c["grid"], c["atoms"], c["probe"], c["scan"], c["tip"], c["df"], r["pos"], c["w"])
    an, fd = [], []
    for what, idx, h in E_PARAMS:
        if what == "Qzz" and qzz == 0.0:
            continue
        fd.append((_loss(orc, _perturbed(c, what, idx, h))[0] - _loss(orc, _perturbed(c, what, idx, -h))[0]) / (2 * h))
        an.append(g[what][idx] if idx is not None else g[what])
    an, fd = np.array(an), np.array(fd)
    assert np.abs(an - fd).max() < 1e-4 * np.abs(fd).max(), (an, fd)


def test_energy_grid_adjoint_of_node_energies_matches_central_differences(orc):
    # dL/dE_g for nodes the relaxed scan reads: perturb one node energy, re-relax, re-image
    c = energy_grid_case()
    _, r = _loss(orc, c)
    g = orc.backward(r["ff"], c["grid"], c["atoms"], c["probe"], c["scan"], c["tip"], c["df"], r["pos"], c["w"],
                     want_grid_adj=True)
    adj = g["grid_adj"]
    assert adj.shape == (c["grid"]["nz"], c["grid"]["ny"], c["grid"]["nx"])
    flat = np.argsort(-np.abs(adj).ravel())[:6]

    def L(ff):
        rr = orc.relax_scan(ff, c["grid"], c["atoms"], c["probe"], c["scan"], c["tip"], c["fire"], 1e-13)
        return float((c["w"] * orc.fz_to_df(rr["fz"], c["scan"]["dz"], c["df"])).sum())

    # one node's energy moves the soft-spring probe by ~(h / dx) / k: the difference is taken at
    # h = 1e-6 eV, where its O(h^2) error is below 1e-5 of the value
    h = 1e-6
    for f in flat:
        k, j, i = np.unravel_index(f, adj.shape)
        fp, fm = r["ff"].copy(), r["ff"].copy()
        fp[k, j, i, 3] += h
        fm[k, j, i, 3] -= h
        fd = (L(fp) - L(fm)) / (2 * h)
        assert adj[k, j, i] == pytest.approx(fd, rel=5e-5), (k, j, i)


def test_energy_grid_charge_scaling_identity(orc):
    # the energy is linear in each product q_i Q and q_i Qzz, so sum_i q_i dL/dq_i = Q dL/dQ + Qzz dL/dQzz
    c = energy_grid_case(-0.05)
    _, r = _loss(orc, c)
    g = orc.backward(r["ff"], c["grid"], c["atoms"], c["probe"], c["scan"], c["tip"], c["df"], r["pos"], c["w"])
    lhs = float((c["atoms"]["q"] * g["q"]).sum())
    assert lhs == pytest.approx(c["probe"]["Q"] * g["Q"] + c["probe"]["Qzz"] * g["Qzz"], rel=1e-10)


def test_energy_grid_adjoint_along_a_rigid_shift_of_all_atoms(orc):
    # the directional derivative along moving every atom by the same dx is sum_i dL/dx_i
    c = energy_grid_case()
    _, r = _loss(orc, c)
    g = orc.backward(r["ff"], c["grid"], c["atoms"], c["probe"], c["scan"], c["tip"], c["df"], r["pos"], c["w"])
    h = 1e-4

    def shifted(s):
        import copy

        c2 = copy.deepcopy(c)
        c2["atoms"]["x"] = c2["atoms"]["x"] + s
        return c2

    fd = (_loss(orc, shifted(h))[0] - _loss(orc, shifted(-h))[0]) / (2 * h)
    assert g["x"].sum() == pytest.approx(fd, rel=1e-4, abs=1e-4 * np.abs(g["x"]).max())
