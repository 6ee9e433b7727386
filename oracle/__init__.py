"""FP64 CPU oracle of the Probe-Particle Model hot path -- TEST INFRASTRUCTURE.

Only the tests, the package smoke check and the CPU-baseline leg of the
benchmark may import this module.  It shares no code with the CUDA library:
`pp_oracle.c` is a plain double-precision restatement of the paper's model
(Sec. 2.1 tip springs and Eq. df; Sec. 2.2 Eqs. LJ and point charges;
Sec. 5.1.1 grid force field, trilinear interpolation and FIRE relaxation),
plus the implicit-function adjoint of that discrete model.

Parity pins for every function live in tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile pp_oracle.c with gcc (FP64, no fast-math, no FMA contraction, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Atoms(C.Structure):
    _fields_ = [("n", C.c_int)] + [(k, C.POINTER(C.c_double)) for k in ("x", "y", "z", "R", "eps", "q")]


class Probe(C.Structure):
    _fields_ = [("R_pp", C.c_double), ("eps_pp", C.c_double), ("Q", C.c_double),
                ("coul_rc", C.c_double), ("min_image", C.c_int), ("core_frac", C.c_double), ("Qzz", C.c_double)]


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int)] + \
               [(k, C.c_double) for k in ("x0", "y0", "z0", "dx", "dy", "dz")] + [("periodic_xy", C.c_int)] + \
               [("Lx", C.c_double), ("Ly", C.c_double), ("interp", C.c_int)]


class Tip(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("kx", "ky", "kR", "R0", "d0x", "d0y")]


class Scan(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int)] + \
               [(k, C.c_double) for k in ("x0", "y0", "px", "py", "z_top", "dz")]


class Fire(C.Structure):
    _fields_ = [("max_iter", C.c_int)] + \
               [(k, C.c_double) for k in ("ftol", "dt0", "dt_max", "f_inc", "f_dec", "alpha0", "f_alpha", "mass")] + \
               [("n_min", C.c_int)]


class DF(C.Structure):
    _fields_ = [("A_pp", C.c_double), ("k", C.c_double), ("f0", C.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            dp, ip, vp = C.POINTER(C.c_double), C.POINTER(C.c_int), C.c_void_p
            L.or_make_ff.argtypes = [C.POINTER(Atoms), C.POINTER(Probe), C.POINTER(Grid), dp, vp, C.c_int]
            L.or_ff_points.argtypes = [C.POINTER(Atoms), C.POINTER(Probe), C.POINTER(Grid), C.c_int, dp, dp, vp, C.c_int]
            L.or_interp_points.argtypes = [dp, C.POINTER(Grid), C.c_int, dp, dp, vp]
            L.or_relax_columns.argtypes = [vp, C.POINTER(Grid), C.POINTER(Atoms), C.POINTER(Probe), C.POINTER(Scan),
                                           C.POINTER(Tip), C.POINTER(Fire), C.c_int, ip, C.c_double,
                                           dp, dp, ip, dp, dp, ip, C.c_int]
            L.or_df_weights.argtypes = [C.c_double, C.c_double, vp]
            L.or_fz_to_df.argtypes = [dp, C.c_int, C.c_int, C.c_double, C.POINTER(DF), dp]
            L.or_backward.argtypes = [vp, C.POINTER(Grid), C.POINTER(Atoms), C.POINTER(Probe), C.POINTER(Scan),
                                      C.POINTER(Tip), C.POINTER(DF), dp, dp, dp, dp, vp, C.c_int]
            L.or_iets.argtypes = [vp, C.POINTER(Grid), C.POINTER(Atoms), C.POINTER(Probe), C.POINTER(Scan),
                                  C.POINTER(Tip), dp, C.c_double, dp, vp, C.c_int]
            L.or_correlate.argtypes = [dp, dp, C.POINTER(Grid), C.c_double, C.c_double, dp, C.c_int]
            L.or_correlate_nodes.argtypes = [dp, dp, C.POINTER(Grid), C.c_double, C.c_double, C.c_int,
                                             C.POINTER(C.c_long), dp, C.c_int]
            L.or_max_threads.restype = C.c_int
            _lib = L
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, t=C.c_double):
    return a.ctypes.data_as(C.POINTER(t))


class _Keep:
    """Holds the numpy buffers behind a ctypes struct alive."""

    def __init__(self):
        self.bufs = []

    def d(self, a):
        a = _d(a)
        self.bufs.append(a)
        return _ptr(a)


def _atoms(a, keep):
    return Atoms(len(a["x"]), *(keep.d(a[k]) for k in ("x", "y", "z", "R", "eps", "q")))


def _probe(p):
    return Probe(p["R_pp"], p["eps_pp"], p["Q"], p["coul_rc"], int(p["min_image"]), p["core_frac"],
                 float(p.get("Qzz", 0.0)))


def _grid(g):
    """Grid dict -> struct; optional "Lx", "Ly" set the minimum-image period of a window of a larger grid,
    optional "interp" = 1 selects tricubic interpolation of the node energies."""
    return Grid(g["nx"], g["ny"], g["nz"], g["x0"], g["y0"], g["z0"], g["dx"], g["dy"], g["dz"], int(g["periodic_xy"]),
                float(g.get("Lx", 0.0)), float(g.get("Ly", 0.0)), int(g.get("interp", 0)))


def _tip(t):
    return Tip(t["kx"], t["ky"], t["kR"], t["R0"], t["d0x"], t["d0y"])


def _scan(s):
    return Scan(s["nx"], s["ny"], s["nz"], s["x0"], s["y0"], s["px"], s["py"], s["z_top"], s["dz"])


def _fire(f):
    return Fire(int(f["max_iter"]), f["ftol"], f["dt0"], f["dt_max"], f["f_inc"], f["f_dec"],
                f["alpha0"], f["f_alpha"], f["mass"], int(f["n_min"]))


def _df(d):
    return DF(d["A_pp"], d["k"], d["f0"])


def max_threads() -> int:
    return int(lib().or_max_threads())


def make_ff(atoms, probe, grid, nthreads=0):
    """Force-field grid [nz][ny][nx][4] = (Fx, Fy, Fz, E) and the core mask [nz][ny][nx]."""
    keep = _Keep()
    g = _grid(grid)
    ff = np.empty((grid["nz"], grid["ny"], grid["nx"], 4))
    core = np.empty((grid["nz"], grid["ny"], grid["nx"]), dtype=np.uint8)
    rc = lib().or_make_ff(C.byref(_atoms(atoms, keep)), C.byref(_probe(probe)), C.byref(g), _ptr(ff),
                          core.ctypes.data_as(C.c_void_p), nthreads)
    if rc:
        raise ValueError("or_make_ff rejected its arguments")
    return ff, core.astype(bool)


def ff_points(atoms, probe, grid, pts, nthreads=0):
    """Direct-sum (Fx, Fy, Fz, E) at points pts[n][3] and a per-point core flag."""
    keep = _Keep()
    pts = _d(pts).reshape(-1, 3)
    out = np.empty((len(pts), 4))
    core = np.empty(len(pts), dtype=np.uint8)
    lib().or_ff_points(C.byref(_atoms(atoms, keep)), C.byref(_probe(probe)), C.byref(_grid(grid)), len(pts),
                       _ptr(pts), _ptr(out), core.ctypes.data_as(C.c_void_p), nthreads)
    return out, core.astype(bool)


def interp_energy_points(ff, grid, pts):
    """Tricubic interpolated energy at pts[n][3] (grid["interp"] must be 1)."""
    ff = _d(ff)
    pts = _d(pts).reshape(-1, 3)
    E = np.empty(len(pts))
    if lib().or_interp_energy_points(_ptr(ff), C.byref(_grid(grid)), len(pts), _ptr(pts), _ptr(E)):
        raise ValueError("energy interpolation needs a tricubic grid")
    return E


def interp_points(ff, grid, pts):
    """Interpolated force (trilinear, or -grad of the tricubic energy) and its Jacobian dF_a/dp_b at pts[n][3]."""
    ff = _d(ff)
    pts = _d(pts).reshape(-1, 3)
    F = np.empty((len(pts), 3))
    J = np.empty((len(pts), 3, 3))
    lib().or_interp_points(_ptr(ff), C.byref(_grid(grid)), len(pts), _ptr(pts), _ptr(F),
                           J.ctypes.data_as(C.c_void_p))
    return F, J


def relax_columns(ff, grid, atoms, probe, scan, tip, fire, cols, polish_tol=1e-11, nthreads=0):
    """Relax the pixel columns cols (j*nx+i) over all heights.  ff=None -> grid-free model."""
    keep = _Keep()
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    n, nz = len(cols), scan["nz"]
    pos = np.empty((n, nz, 3))
    fz = np.empty((n, nz))
    iters = np.empty((n, nz), dtype=np.int32)
    res = np.empty((n, nz))
    lam = np.empty((n, nz))
    ok = np.empty((n, nz), dtype=np.int32)
    ffp = None
    if ff is not None:
        ff = _d(ff)
        ffp = ff.ctypes.data_as(C.c_void_p)
    A = _atoms(atoms, keep) if atoms is not None else None
    Pr = _probe(probe) if probe is not None else None
    rc = lib().or_relax_columns(ffp, C.byref(_grid(grid)), C.byref(A) if A is not None else None,
                                C.byref(Pr) if Pr is not None else None, C.byref(_scan(scan)),
                                C.byref(_tip(tip)), C.byref(_fire(fire)), n,
                                cols.ctypes.data_as(C.POINTER(C.c_int)), float(polish_tol),
                                _ptr(pos), _ptr(fz), _ptr(iters, C.c_int), _ptr(res), _ptr(lam),
                                _ptr(ok, C.c_int), nthreads)
    if rc:
        raise ValueError("or_relax_columns rejected its arguments")
    return {"pos": pos, "fz": fz, "iters": iters, "res": res, "lam": lam, "ok": ok.astype(bool)}


def relax_scan(ff, grid, atoms, probe, scan, tip, fire, polish_tol=1e-11, nthreads=0):
    """Whole scan; outputs in scan layout: pos [nz][ny][nx][3], fz/iters/... [nz][ny][nx]."""
    nx, ny, nz = scan["nx"], scan["ny"], scan["nz"]
    r = relax_columns(ff, grid, atoms, probe, scan, tip, fire, np.arange(nx * ny), polish_tol, nthreads)
    out = {}
    for k, v in r.items():
        v = np.moveaxis(v, 1, 0)  # (nz, ncols, ...)
        out[k] = v.reshape((nz, ny, nx) + v.shape[2:])
    return out


def iets(ff, grid, atoms, probe, scan, tip, pos, mass_amu=16.0, nthreads=0):
    """Stiffness eigenvalues (eV/A^2, ascending) and mode energies (meV) at relaxed positions pos[nz][ny][nx][3]."""
    keep = _Keep()
    pos = _d(pos)
    shp = pos.shape[:-1]
    eig = np.empty(shp + (3,))
    hw = np.empty(shp + (3,))
    ffp = None
    if ff is not None:
        ff = _d(ff)
        ffp = ff.ctypes.data_as(C.c_void_p)
    A = _atoms(atoms, keep) if atoms is not None else None
    Pr = _probe(probe) if probe is not None else None
    rc = lib().or_iets(ffp, C.byref(_grid(grid)), C.byref(A) if A is not None else None,
                       C.byref(Pr) if Pr is not None else None, C.byref(_scan(scan)), C.byref(_tip(tip)), _ptr(pos),
                       float(mass_amu), _ptr(eig), hw.ctypes.data_as(C.c_void_p), nthreads)
    if rc:
        raise ValueError("or_iets rejected its arguments")
    return eig, hw


def df_weights(a, h):
    m = lib().or_df_weights(float(a), float(h), None)
    W = np.empty(2 * m + 1)
    lib().or_df_weights(float(a), float(h), W.ctypes.data_as(C.c_void_p))
    return W


def fz_to_df(fz, dz, df):
    """fz [nz][...] -> df [nz-2m][...] (Eq. df, centre labelling)."""
    fz = _d(fz)
    nz = fz.shape[0]
    npix = int(np.prod(fz.shape[1:])) if fz.ndim > 1 else 1
    m = lib().or_df_weights(0.5 * df["A_pp"], float(dz), None)
    out = np.empty((nz - 2 * m,) + fz.shape[1:])
    rc = lib().or_fz_to_df(_ptr(fz), nz, npix, float(dz), C.byref(_df(df)), _ptr(out))
    if rc:
        raise ValueError("or_fz_to_df: too few heights for the amplitude")
    return out


def backward(ff, grid, atoms, probe, scan, tip, df, pos, g_df, want_grid_adj=False, nthreads=0):
    """Gradient of sum(g_df * df) by the implicit adjoint.  ff=None -> grid-free model.
    grid_adj is dL/dF_g [nz][ny][nx][3] on a force grid and dL/dE_g [nz][ny][nx] on an energy grid."""
    keep = _Keep()
    pos = _d(pos)
    g_df = _d(g_df)
    n = len(atoms["x"])
    grads = np.zeros((n, 6))
    gtip = np.zeros(5)
    gadj = np.zeros((grid["nz"], grid["ny"], grid["nx"], 3)) if (want_grid_adj and ff is not None) else None
    ffp = None
    if ff is not None:
        ff = _d(ff)
        ffp = ff.ctypes.data_as(C.c_void_p)
    rc = lib().or_backward(ffp, C.byref(_grid(grid)), C.byref(_atoms(atoms, keep)), C.byref(_probe(probe)),
                           C.byref(_scan(scan)), C.byref(_tip(tip)), C.byref(_df(df)), _ptr(pos), _ptr(g_df),
                           _ptr(grads), _ptr(gtip), gadj.ctypes.data_as(C.c_void_p) if gadj is not None else None,
                           nthreads)
    if rc:
        raise ValueError("or_backward rejected its arguments")
    if gadj is not None and grid.get("interp", 0) == 1:
        gadj = gadj[..., 0].copy()
    return {"x": grads[:, 0], "y": grads[:, 1], "z": grads[:, 2], "R": grads[:, 3], "eps": grads[:, 4],
            "q": grads[:, 5], "kx": gtip[0], "ky": gtip[1], "kR": gtip[2], "Q": gtip[3], "Qzz": gtip[4], "grid_adj": gadj}


def forward(case, grid_free=False, fire=None, polish_tol=1e-11, nthreads=0):
    """Whole pipeline on a case dict: FF grid, relaxed scan, df image."""
    ff = None
    core = None
    if not grid_free:
        ff, core = make_ff(case["atoms"], case["probe"], case["grid"], nthreads)
    r = relax_scan(ff, case["grid"], case["atoms"], case["probe"], case["scan"], case["tip"],
                   fire or case["fire"], polish_tol, nthreads)
    r["df"] = fz_to_df(r["fz"], case["scan"]["dz"], case["df"])
    r["ff"] = ff
    r["core"] = core
    return r


def correlate(f, g, grid, scale=1.0, power=1.0, nthreads=0):
    """Cross-correlation force field [nz][ny][nx][4] = (Fx, Fy, Fz, E) of the periodic sample
    field f[nz][ny][nx] seen by the tip density g[nz][ny][nx] (offsets from the PP, wrapped)."""
    f, g = _d(f), _d(g)
    ff = np.empty((grid["nz"], grid["ny"], grid["nx"], 4))
    if lib().or_correlate(_ptr(f), _ptr(g), C.byref(_grid(grid)), scale, power, _ptr(ff), nthreads):
        raise ValueError("or_correlate rejected its arguments (sizes must be even)")
    return ff


def correlate_nodes(f, g, grid, nodes, scale=1.0, power=1.0, nthreads=0):
    """E of correlate() at the flat node indices `nodes` only."""
    f, g = _d(f), _d(g)
    nodes = np.ascontiguousarray(nodes, dtype=np.int64)
    E = np.empty(len(nodes))
    lib().or_correlate_nodes(_ptr(f), _ptr(g), C.byref(_grid(grid)), scale, power, len(nodes),
                             nodes.ctypes.data_as(C.POINTER(C.c_long)), _ptr(E), nthreads)
    return E
