"""Seeded synthetic inputs shaped like the paper's workloads.

The paper images molecules (C60, pentacene, PTCDA, ...) and sweeps a periodic
graphene sheet (Sec. 5.3); none of those geometries, nor the OPLS table it uses
for Lennard-Jones parameters (Sec. 2.2.1), ship with it.  This module builds
stand-ins of the same shape from a seed: a benzene ring, a 60-atom
H-terminated aromatic flake, random H/C/N/O/F molecules of 10-80 atoms, and a
2016-atom AB graphene bilayer with a 500-atom molecule on it.

It holds input data and geometry only, none of the method's arithmetic: no
mixing rules, no unit conversion, no force law.  Spring constants stay in N/m,
lengths in Angstrom, energies in eV, charges in e.  Both the CUDA path and the
FP64 oracle take these dictionaries as their inputs.
"""
from __future__ import annotations

import math

import numpy as np

# Element-based LJ parameters (R in Angstrom, eps in eV).  Synthetic values of
# OPLS magnitude; the probe particle (an O of a CO tip) takes the O entry.
ELEMENTS = {
    "H": (1.49, 0.00068),
    "C": (1.91, 0.0037),
    "N": (1.78, 0.0074),
    "O": (1.66, 0.0091),
    "F": (1.75, 0.0026),
}


def _atoms(sym, xyz, q):
    xyz = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)
    R = np.array([ELEMENTS[s][0] for s in sym], dtype=np.float64)
    eps = np.array([ELEMENTS[s][1] for s in sym], dtype=np.float64)
    return {
        "sym": list(sym),
        "x": np.ascontiguousarray(xyz[:, 0]),
        "y": np.ascontiguousarray(xyz[:, 1]),
        "z": np.ascontiguousarray(xyz[:, 2]),
        "R": R,
        "eps": eps,
        "q": np.asarray(q, dtype=np.float64).copy(),
    }


def default_probe(**kw):
    """CO-like probe particle: O parameters, charge Q = -0.1 e, no tip quadrupole (Qzz in e*A^2)."""
    p = {"R_pp": ELEMENTS["O"][0], "eps_pp": ELEMENTS["O"][1], "Q": -0.1,
         "coul_rc": 0.0, "min_image": 0, "core_frac": 0.5, "Qzz": 0.0}
    p.update(kw)
    return p


def default_tip(**kw):
    """Lateral 0.25 N/m, radial 20 N/m, R0 = 4 Angstrom (springs in N/m)."""
    t = {"kx": 0.25, "ky": 0.25, "kR": 20.0, "R0": 4.0, "d0x": 0.0, "d0y": 0.0}
    t.update(kw)
    return t


def default_fire(**kw):
    """FIRE settings of the timed runs.

    N_min, f_inc, f_dec, alpha_start and f_alpha are the published defaults of
    Bitzek et al. (2006).  The paper gives no time step; dt0 = dt_max = 1.0
    (mass 1, time in sqrt(A^2/eV)) keeps semi-implicit Euler stable for
    stiffnesses up to 4 eV/A^2 (the radial spring is 1.25) and, from the
    warm start of the height above, converges in 35-50 % fewer iterations than
    growing the step from 0.2 to 0.8, with the same fixed points.
    """
    f = {"max_iter": 200, "ftol": 1e-4, "dt0": 1.0, "dt_max": 1.0, "f_inc": 1.1,
         "f_dec": 0.5, "alpha0": 0.1, "f_alpha": 0.99, "mass": 1.0, "n_min": 5}
    f.update(kw)
    return f


def parity_fire(**kw):
    """Tighter FIRE settings used when positions are compared to 1e-3 Angstrom."""
    return default_fire(**{"max_iter": 2000, "ftol": 1e-5, **kw})


def default_df(**kw):
    """qPlus-like cantilever: peak-to-peak amplitude 1 A, k = 1800 N/m, f0 = 30.3 kHz."""
    d = {"A_pp": 1.0, "k": 1800.0, "f0": 30300.0}
    d.update(kw)
    return d


# ---------------------------------------------------------------- molecules

def benzene():
    """Planar C6H6: C on a 1.39 A ring, H at 2.47 A, charges -/+0.115 e."""
    sym, xyz, q = [], [], []
    for k in range(6):
        a = math.radians(60.0 * k)
        sym.append("C"); xyz.append((1.39 * math.cos(a), 1.39 * math.sin(a), 0.0)); q.append(-0.115)
    for k in range(6):
        a = math.radians(60.0 * k)
        sym.append("H"); xyz.append((2.47 * math.cos(a), 2.47 * math.sin(a), 0.0)); q.append(0.115)
    return _atoms(sym, xyz, q)


def _hex_vertices(cq, cr, bond):
    # hexagon centres on a triangular lattice with spacing sqrt(3)*bond
    a = math.sqrt(3.0) * bond
    cx = a * (cq + 0.5 * cr)
    cy = a * (math.sqrt(3.0) / 2.0) * cr
    return [(cx + bond * math.cos(math.radians(30 + 60 * k)),
             cy + bond * math.sin(math.radians(30 + 60 * k))) for k in range(6)]


def _flake_atoms(hexes, bond=1.42, ch=1.09):
    verts = {}
    for (cq, cr) in hexes:
        for (x, y) in _hex_vertices(cq, cr, bond):
            verts[(round(x, 4), round(y, 4))] = (x, y)
    C = np.array(list(verts.values()))
    d = np.linalg.norm(C[:, None, :] - C[None, :, :], axis=-1)
    nb = (d > 0.1) & (d < bond * 1.05)
    H = []
    for i in range(len(C)):
        idx = np.nonzero(nb[i])[0]
        if len(idx) == 2:
            out = 2.0 * C[i] - C[idx[0]] - C[idx[1]]
            out /= np.linalg.norm(out)
            H.append(C[i] + ch * out)
    return C, np.array(H).reshape(-1, 2)


def aromatic_flake(n_target=60, seed=42):
    """H-terminated benzenoid flake grown hexagon by hexagon until C+H == n_target.

    Hexagons are added one at a time at a seeded random free neighbour site of
    the current flake (C-C 1.42 A, C-H 1.09 A along the outward bisector of a
    2-coordinated C).  A growth that overshoots n_target restarts from benzene
    with the same generator stream, so the result depends on the seed only.
    Charges ~ U(-0.2, 0.2), mean removed, rescaled so that max |q| <= 0.2.
    """
    rng = np.random.default_rng(seed)
    nbrs = [(1, 0), (-1, 0), (0, 1), (0, -1), (1, -1), (-1, 1)]
    for _attempt in range(10000):
        hexes = [(0, 0)]
        while True:
            C, H = _flake_atoms(hexes)
            n = len(C) + len(H)
            if n == n_target:
                break
            if n > n_target:
                hexes = None
                break
            cand = sorted({(q + a, r + b) for (q, r) in hexes for (a, b) in nbrs} - set(hexes))
            hexes.append(cand[rng.integers(len(cand))])
        if hexes is not None:
            break
    else:  # pragma: no cover
        raise RuntimeError("flake growth did not reach the target size")
    cen = np.concatenate([C, H]).mean(axis=0)
    C = C - cen
    H = H - cen
    xyz = np.concatenate([np.c_[C, np.zeros(len(C))], np.c_[H, np.zeros(len(H))]])
    sym = ["C"] * len(C) + ["H"] * len(H)
    q = rng.uniform(-0.2, 0.2, len(sym))
    q -= q.mean()
    m = np.abs(q).max()
    if m > 0.2:
        q *= 0.2 / m
    return _atoms(sym, xyz, q)


def random_molecule(seed, n_atoms=None, zmax=1.5, lateral_max=None, qmax=0.3):
    """Seeded tree-grown H/C/N/O/F molecule within |z| <= zmax of its mean plane.

    Atom 0 sits at the origin; each new atom bonds to a random existing atom at
    a length ~ U(1.0, 1.5) A along a random direction with |cos(tilt)| <= 0.5;
    a candidate closer than 1.0 A to any atom, or outside |z| <= zmax (and the
    optional lateral box), is rejected.  Charges ~ U(-qmax, qmax), neutralised
    and scaled into [-qmax, qmax].  The molecule is centred laterally.
    """
    rng = np.random.default_rng(seed)
    n = int(rng.integers(10, 81)) if n_atoms is None else int(n_atoms)
    pos = np.zeros((n, 3))
    k = 1
    tries = 0
    while k < n:
        tries += 1
        if tries > 2000 * n:  # pragma: no cover
            raise RuntimeError("molecule growth stalled")
        parent = pos[rng.integers(k)]
        b = rng.uniform(1.0, 1.5)
        phi = rng.uniform(0.0, 2.0 * math.pi)
        t = rng.uniform(-0.5, 0.5)
        s = math.sqrt(1.0 - t * t)
        cand = parent + b * np.array([s * math.cos(phi), s * math.sin(phi), t])
        if abs(cand[2]) > zmax:
            continue
        if lateral_max is not None and (abs(cand[0]) > lateral_max or abs(cand[1]) > lateral_max):
            continue
        if np.min(np.linalg.norm(pos[:k] - cand, axis=1)) < 1.0:
            continue
        pos[k] = cand
        k += 1
    pos[:, 0] -= 0.5 * (pos[:, 0].max() + pos[:, 0].min())
    pos[:, 1] -= 0.5 * (pos[:, 1].max() + pos[:, 1].min())
    pos[:, 2] -= pos[:, 2].mean()
    sym = list(rng.choice(["H", "C", "N", "O", "F"], size=n, p=[0.3, 0.4, 0.1, 0.1, 0.1]))
    q = rng.uniform(-qmax, qmax, n)
    q -= q.mean()
    m = np.abs(q).max()
    if m > qmax:
        q *= qmax / m
    return _atoms(sym, pos, q)


def graphene_bilayer(nx_cells=21, ny_cells=12, box=51.2, z_layers=(0.0, 3.35)):
    """AB-stacked bilayer: nx x ny rectangular 4-atom cells scaled to box x box A."""
    a = 2.46
    ax, ay = a, a * math.sqrt(3.0)
    basis = np.array([[0.0, 0.0], [a / 2, ay / 6], [a / 2, ay / 2], [0.0, 2 * ay / 3]])
    pts = []
    for i in range(nx_cells):
        for j in range(ny_cells):
            pts.append(basis + np.array([i * ax, j * ay]))
    P = np.concatenate(pts)
    P[:, 0] *= box / (nx_cells * ax)
    P[:, 1] *= box / (ny_cells * ay)
    shift = np.array([0.0, box / (ny_cells * ay) * ay / 3])  # B layer shifted by one C-C bond
    L0 = np.c_[P, np.full(len(P), z_layers[0])]
    L1 = np.c_[(P + shift) % box, np.full(len(P), z_layers[1])]
    xyz = np.concatenate([L0, L1])
    return _atoms(["C"] * len(xyz), xyz, np.zeros(len(xyz)))


def concat_atoms(a, b):
    out = {"sym": a["sym"] + b["sym"]}
    for k in ("x", "y", "z", "R", "eps", "q"):
        out[k] = np.concatenate([a[k], b[k]])
    return out


def shift_atoms(a, dx=0.0, dy=0.0, dz=0.0):
    out = dict(a)
    out["x"] = a["x"] + dx
    out["y"] = a["y"] + dy
    out["z"] = a["z"] + dz
    return out


# ---------------------------------------------------------------- workloads

def _grid(nx, ny, nz, x0, y0, z0, d, periodic_xy=1):
    return {"nx": nx, "ny": ny, "nz": nz, "x0": x0, "y0": y0, "z0": z0,
            "dx": d, "dy": d, "dz": d, "periodic_xy": periodic_xy}


def _scan(nx, ny, nz, x0, y0, px, py, z_top, dz=0.1):
    return {"nx": nx, "ny": ny, "nz": nz, "x0": x0, "y0": y0, "px": px, "py": py,
            "z_top": z_top, "dz": dz}


def _case(name, atoms, grid, scan, probe=None, tip=None, fire=None, df=None):
    return {"name": name, "atoms": atoms, "grid": grid, "scan": scan,
            "probe": probe or default_probe(), "tip": tip or default_tip(),
            "fire": fire or default_fire(), "df": df or default_df()}


def benzene_case():
    """Benzene on an 80x80x60 grid at 0.2 A; 40x40 px scan, 20 heights (PP 5.0 -> 3.1 A)."""
    grid = _grid(80, 80, 60, -8.0, -8.0, 0.0, 0.2)
    scan = _scan(40, 40, 20, -5.85, -5.85, 0.3, 0.3, 9.0)
    return _case("benzene_80x80x60_scan40x40x20", benzene(), grid, scan)


def flake_case():
    """60-atom flake on a 256x256x200 grid at 0.1 A; 256x256 px scan, 40 heights."""
    grid = _grid(256, 256, 200, -12.8, -12.8, 0.0, 0.1)
    scan = _scan(256, 256, 40, -12.75, -12.75, 0.1, 0.1, 11.0)
    return _case("flake60_256x256x200_scan256x256x40", aromatic_flake(60, 42), grid, scan)


def molecule_case(atoms, name, nz_grid=60, scan_px=128, nz_scan=20, R0=4.0):
    """Per-molecule grid and scan used by the batched and gradient workloads.

    Lateral nodes per side n = 16*ceil((extent + 8 A)/1.6 A) clamped to
    [128, 256] at 0.1 A; 60 z-nodes from 2 A above the topmost atom; a
    scan_px x scan_px scan over the full lateral extent with the PP
    (unrelaxed) going from 5.0 to 3.1 A above the topmost atom.
    """
    d = 0.1
    ext_x = atoms["x"].max() - atoms["x"].min()
    ext_y = atoms["y"].max() - atoms["y"].min()
    nx = int(min(256, max(128, 16 * math.ceil((ext_x + 8.0) / 1.6))))
    ny = int(min(256, max(128, 16 * math.ceil((ext_y + 8.0) / 1.6))))
    cx = 0.5 * (atoms["x"].max() + atoms["x"].min())
    cy = 0.5 * (atoms["y"].max() + atoms["y"].min())
    ztop = float(atoms["z"].max())
    x0 = float(round(cx - 0.5 * nx * d, 6))
    y0 = float(round(cy - 0.5 * ny * d, 6))
    grid = _grid(nx, ny, nz_grid, x0, y0, ztop + 2.0, d)
    px = nx * d / scan_px
    py = ny * d / scan_px
    scan = _scan(scan_px, scan_px, nz_scan, x0 + 0.5 * px, y0 + 0.5 * py, px, py,
                 ztop + 5.0 + R0, 0.1)
    return _case(name, atoms, grid, scan)


def batch_cases(n_mol=1024, first_seed=1000):
    """Molecule i uses seed first_seed+i and N ~ U{10..80}."""
    return [molecule_case(random_molecule(first_seed + i), f"mol{first_seed + i}")
            for i in range(n_mol)]


def gradient_case():
    """40-atom molecule (seed 4040); loss weights w ~ N(0,1) with seed 7."""
    c = molecule_case(random_molecule(4040, 40), "mol40_seed4040")
    m = int(math.ceil(0.5 * c["df"]["A_pp"] / c["scan"]["dz"] - 1e-9))
    nzo = c["scan"]["nz"] - 2 * m
    rng = np.random.default_rng(7)
    c["w"] = rng.standard_normal((nzo, c["scan"]["ny"], c["scan"]["nx"]))
    c["fd_seed"] = 11
    return c


def slab_case():
    """500-atom molecule on a 2016-atom AB bilayer, laterally periodic 512x512x250 grid.

    Minimum-image lateral sum and a shifted-force Coulomb cut at 8 A; the scan
    is 512x512 px and 60 heights, PP (unrelaxed) from 9.0 to 3.1 A above the
    topmost molecular atom.
    """
    # an incommensurate lateral offset keeps lattice rows off the grid's half-period planes,
    # where the minimum-image force is discontinuous
    slab = shift_atoms(graphene_bilayer(), 0.0123, 0.0321)
    mol = random_molecule(5000, 500, lateral_max=20.0)
    mol = shift_atoms(mol, 25.6, 25.6, 6.65)
    atoms = concat_atoms(slab, mol)
    grid = _grid(512, 512, 250, 0.0, 0.0, 0.0, 0.1)
    ztop = float(mol["z"].max())
    scan = _scan(512, 512, 60, 0.05, 0.05, 0.1, 0.1, ztop + 9.0 + 4.0)
    probe = default_probe(coul_rc=8.0, min_image=1)
    return _case("slab2016_mol500_512x512x250_scan512x512x60", atoms, grid, scan, probe=probe)


def small_case(seed=3, n_atoms=12, nxy=32, nz=40, scan_px=12, nz_scan=12, d=0.2):
    """A few-second case for oracle-vs-GPU parity on several tiles with ragged tails."""
    atoms = random_molecule(seed, n_atoms)
    grid = _grid(nxy, nxy + 4, nz, -0.5 * nxy * d, -0.5 * (nxy + 4) * d, atoms["z"].max() + 1.6, d)
    scan = _scan(scan_px, scan_px + 3, nz_scan, -0.35 * nxy * d, -0.35 * (nxy + 4) * d,
                 0.7 * nxy * d / scan_px, 0.7 * (nxy + 4) * d / (scan_px + 3),
                 atoms["z"].max() + 5.0 + 4.0, 0.1)
    return _case(f"small_seed{seed}", atoms, grid, scan)


# ------------------------------------------- densities for the FFT force fields
#
# Stand-ins for the DFT inputs of the Hartree and full-density models (the
# paper's densities and potentials come from DFT; none are available here):
# valence densities as sums of normalised Gaussians on a grid periodic in x, y
# and z, and the Hartree potential of a neutral Gaussian charge distribution
# from Poisson's equation, solved spectrally.  Input generation only.

VALENCE = {"H": (1.0, 0.45), "C": (4.0, 0.55), "N": (5.0, 0.52), "O": (6.0, 0.50), "F": (7.0, 0.48)}


def periodic_gaussians(grid, xyz, weights, sigmas, cut=6.0):
    """sum_i w_i * normalised Gaussian(sigma_i) at xyz_i on a grid periodic in x, y and z (period
    n * d), each Gaussian evaluated within cut * sigma of its nearest image (plus the next images
    when the window spans the whole axis); float64 [nz][ny][nx]."""
    n = (grid["nx"], grid["ny"], grid["nz"])
    d = (grid["dx"], grid["dy"], grid["dz"])
    o = (grid["x0"], grid["y0"], grid["z0"])
    L = [n[a] * d[a] for a in range(3)]
    out = np.zeros((n[2], n[1], n[0]))
    for p, w, sg in zip(np.asarray(xyz, dtype=float), weights, sigmas):
        idx, prof = [], []
        for a in range(3):
            half = int(math.ceil(cut * sg / d[a]))
            if 2 * half + 1 >= n[a]:
                i = np.arange(n[a])
                r = o[a] + i * d[a] - p[a]
                r = r - L[a] * np.round(r / L[a])
                g = sum(np.exp(-(r + m * L[a]) ** 2 / (2 * sg * sg)) for m in (-1, 0, 1))
            else:
                c = int(round((p[a] - o[a]) / d[a]))
                i = np.arange(c - half, c + half + 1)
                r = o[a] + i * d[a] - p[a]
                i = i % n[a]
                g = np.exp(-r * r / (2 * sg * sg))
            idx.append(i)
            prof.append(g)
        amp = w * (2 * np.pi * sg * sg) ** -1.5
        out[np.ix_(idx[2], idx[1], idx[0])] += amp * prof[2][:, None, None] * prof[1][None, :, None] * prof[0][None, None, :]
    return out


def valence_density(grid, atoms):
    """Synthetic valence density (e/A^3) of the atoms: one Gaussian per atom with the element's
    valence electron count and width."""
    xyz = np.c_[atoms["x"], atoms["y"], atoms["z"]]
    w = [VALENCE[s][0] for s in atoms["sym"]]
    sg = [VALENCE[s][1] for s in atoms["sym"]]
    return periodic_gaussians(grid, xyz, w, sg)


def hartree_potential(grid, atoms, sigma=0.35):
    """Hartree potential (V) of the atoms' partial charges smeared into Gaussians of width sigma,
    periodic in x, y and z: Poisson's equation del^2 V = -4 pi k_e rho solved in Fourier space
    (the k = 0 term, the mean, set to zero)."""
    k_e = 14.3996454784
    xyz = np.c_[atoms["x"], atoms["y"], atoms["z"]]
    q = np.asarray(atoms["q"], dtype=float)
    rho = periodic_gaussians(grid, xyz, q - q.mean(), [sigma] * len(q))
    kx = 2 * np.pi * np.fft.fftfreq(grid["nx"], grid["dx"])
    ky = 2 * np.pi * np.fft.fftfreq(grid["ny"], grid["dy"])
    kz = 2 * np.pi * np.fft.fftfreq(grid["nz"], grid["dz"])
    K2 = kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2
    R = np.fft.fftn(rho)
    V = np.zeros_like(R)
    nz = K2 > 0
    V[nz] = 4 * np.pi * k_e * R[nz] / K2[nz]
    return np.real(np.fft.ifftn(V))


def tip_densities(grid, sigma_pauli=0.55, n_pauli=6.0, qzz=-0.05, sigma_q=0.7, s_q=0.3):
    """Tip densities at offsets from the PP (centred on node 0, wrapped): the Pauli density of the
    CO tip (n_pauli electrons in one Gaussian) and an axial quadrupolar charge density (charges
    +c, -2c, +c at z = +s_q, 0, -s_q smeared by sigma_q, second moment 2 c s_q^2 = qzz)."""
    g0 = dict(grid, x0=0.0, y0=0.0, z0=0.0)
    pauli = periodic_gaussians(g0, [(0.0, 0.0, 0.0)], [n_pauli], [sigma_pauli])
    c = qzz / (2 * s_q * s_q)
    quad = periodic_gaussians(g0, [(0.0, 0.0, s_q), (0.0, 0.0, 0.0), (0.0, 0.0, -s_q)], [c, -2 * c, c],
                              [sigma_q] * 3)
    return pauli, quad


def graphene_sheet(na, nb, z=0.0):
    """Flat graphene: na x nb rectangular 4-atom cells (a = 2.46 A), small alternating charges."""
    a = 2.46
    ay = a * math.sqrt(3.0)
    basis = np.array([[0.0, 0.0], [a / 2, ay / 6], [a / 2, ay / 2], [0.0, 2 * ay / 3]])
    P = np.concatenate([basis + np.array([i * a, j * ay]) for i in range(na) for j in range(nb)])
    q = np.tile([0.02, -0.02, 0.02, -0.02], na * nb)
    return _atoms(["C"] * len(P), np.c_[P, np.full(len(P), z)], q)


def graphene_sweep_case(na, nb, nz=128, lz=16.0):
    """Periodic graphene sheet of na x nb cells for the size sweep of the force-field step (the
    paper's Fig. on performance): grid points proportional to atoms, about 0.1 A apart in x, y;
    sizes rounded to powers of two for the FFT path."""
    atoms = graphene_sheet(na, nb, z=4.0)
    a = 2.46
    lx, ly = na * a, nb * a * math.sqrt(3.0)

    def p2(v):
        return 1 << int(round(math.log2(v)))

    nx, ny = p2(lx / 0.1), p2(ly / 0.1)
    grid = {"nx": nx, "ny": ny, "nz": nz, "x0": 0.0, "y0": 0.0, "z0": 0.0, "dx": lx / nx, "dy": ly / ny,
            "dz": lz / nz, "periodic_xy": 1}
    return {"name": f"graphene{na}x{nb}", "atoms": atoms, "grid": grid, "probe": default_probe(min_image=1)}
