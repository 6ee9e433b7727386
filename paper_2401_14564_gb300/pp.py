"""ctypes binding of libpp (include/pp.h): same entry points, argument marshalling only.

Every function takes torch CUDA tensors (device memory) and plain dicts of
parameters, turns them into the C structs of pp.h, and calls the library on
the current torch stream.  All arithmetic happens in the CUDA kernels; there is
no CPU path.  A missing or unloadable libpp.so raises at first use.
"""
from __future__ import annotations

import ctypes as C
import os
import re
import threading

import torch

PKG = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(os.path.dirname(PKG), "include", "pp.h")
# PP_LIBRARY selects another build of the library (the bounds-checked libpp_checked.so)
LIB_PATH = os.environ.get("PP_LIBRARY") or os.path.join(PKG, "libpp.so")

STATUS = {0: "PP_OK", 1: "PP_ERR_ARG", 2: "PP_ERR_SHAPE", 3: "PP_ERR_CUDA", 4: "PP_ERR_CAPACITY",
          5: "PP_ERR_TIMEOUT", 6: "PP_ERR_UNSUPPORTED"}


class PPError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


fp = C.POINTER(C.c_float)


class Atoms(C.Structure):
    _fields_ = [("n", C.c_int)] + [(k, C.c_void_p) for k in ("x", "y", "z", "R", "eps", "q")]


class Probe(C.Structure):
    _fields_ = [("R_pp", C.c_float), ("eps_pp", C.c_float), ("Q", C.c_float), ("coul_rc", C.c_float),
                ("min_image", C.c_int), ("core_frac", C.c_float), ("Qzz", C.c_float)]


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int)] + \
               [(k, C.c_float) for k in ("x0", "y0", "z0", "dx", "dy", "dz")] + \
               [(k, C.c_int) for k in ("periodic_xy", "layout", "bx", "by", "bz", "interp")]


class Tip(C.Structure):
    _fields_ = [(k, C.c_float) for k in ("kx", "ky", "kR", "R0", "d0x", "d0y")]


class Scan(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int)] + \
               [(k, C.c_float) for k in ("x0", "y0", "px", "py", "z_top", "dz")]


class Fire(C.Structure):
    _fields_ = [("max_iter", C.c_int)] + \
               [(k, C.c_float) for k in ("ftol", "dt0", "dt_max", "f_inc", "f_dec", "alpha0", "f_alpha", "mass")] + \
               [("n_min", C.c_int), ("polish", C.c_int)]


class DF(C.Structure):
    _fields_ = [("A_pp", C.c_float), ("k", C.c_float), ("f0", C.c_float)]


class MolDesc(C.Structure):
    _fields_ = [("ff_offset", C.c_longlong), ("out_offset", C.c_longlong), ("df_offset", C.c_longlong),
                ("atom_offset", C.c_int), ("n_atoms", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int)] + \
               [(k, C.c_float) for k in ("x0", "y0", "z0", "dx", "dy", "dz")] + \
               [("snx", C.c_int), ("sny", C.c_int), ("snz", C.c_int)] + \
               [(k, C.c_float) for k in ("sx0", "sy0", "spx", "spy", "z_top")]


class BatchParams(C.Structure):
    _fields_ = [("probe", Probe), ("tip", Tip), ("fire", Fire), ("df", DF), ("scan_dz", C.c_float),
                ("periodic_xy", C.c_int), ("ff_capacity", C.c_longlong), ("out_capacity", C.c_longlong),
                ("df_capacity", C.c_longlong), ("n_atoms_total", C.c_int), ("ctas", C.c_int),
                ("spin_limit", C.c_longlong), ("wait_extra", C.c_int), ("ff_forces_only", C.c_int),
                ("ff_tile_w", C.c_int), ("ff_zpt", C.c_int), ("relax_tile_w", C.c_int)]


class Tuning(C.Structure):
    _fields_ = [("ff_zpt", C.c_int), ("ff_forces_only", C.c_int)]


class ScanOpts(C.Structure):
    _fields_ = [("zspan", C.c_void_p), ("plan", C.c_void_p), ("plan_k", C.c_int), ("plan_lanes", C.c_int)]


class Grads(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("x", "y", "z", "q", "R", "eps", "tip")]


_lock = threading.Lock()
_lib = None


def declared_symbols(header=HEADER):
    """Names of the entry points declared in include/pp.h."""
    text = open(header).read()
    return re.findall(r"^PP_API\s+[\w\s\*]+?\b(pp_\w+)\s*\(", text, flags=re.M)


def lib():
    """Load libpp.so (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                                   "or python -m paper_2401_14564_gb300.build")
            L = C.CDLL(LIB_PATH)
            vp, st = C.c_void_p, C.c_int
            L.pp_ff_floats.argtypes = [C.POINTER(Grid)]
            L.pp_ff_floats.restype = C.c_size_t
            L.pp_df_margin.argtypes = [C.c_float, C.c_float]
            L.pp_df_margin.restype = C.c_int
            L.pp_make_ff.argtypes = [C.POINTER(Atoms), C.POINTER(Probe), C.POINTER(Grid), vp, vp]
            L.pp_make_ff.restype = st
            L.pp_make_ff_tuned.argtypes = [C.POINTER(Atoms), C.POINTER(Probe), C.POINTER(Grid), vp,
                                           C.POINTER(Tuning), vp]
            L.pp_make_ff_tuned.restype = st
            L.pp_make_ff_layers.argtypes = [C.POINTER(Atoms), C.POINTER(Probe), C.POINTER(Grid), vp,
                                            C.POINTER(Tuning), C.c_int, C.c_int, vp]
            L.pp_make_ff_layers.restype = st
            L.pp_make_ff_split.argtypes = [C.POINTER(Atoms), C.POINTER(Probe), C.POINTER(Grid), vp, vp, vp]
            L.pp_make_ff_split.restype = st
            L.pp_ff_combine.argtypes = [vp, vp, C.c_float, C.POINTER(Grid), vp, vp]
            L.pp_ff_combine.restype = st
            L.pp_relax_scan.argtypes = [vp, C.POINTER(Grid), C.POINTER(Scan), C.POINTER(Tip), C.POINTER(Fire),
                                        vp, vp, vp, C.POINTER(DF), vp, vp]
            L.pp_relax_scan.restype = st
            L.pp_relax_scan_ex.argtypes = [vp, C.POINTER(Grid), C.POINTER(Scan), C.POINTER(Tip), C.POINTER(Fire),
                                           vp, vp, vp, C.POINTER(DF), vp, C.POINTER(ScanOpts), vp]
            L.pp_relax_scan_ex.restype = st
            L.pp_relax_plan_size.argtypes = [C.POINTER(Scan), C.c_int, C.c_int]
            L.pp_relax_plan_size.restype = C.c_size_t
            L.pp_relax_plan.argtypes = [vp, C.POINTER(Scan), C.c_int, C.c_int, C.c_int, vp, vp]
            L.pp_relax_plan.restype = st
            L.pp_fz_to_df.argtypes = [vp, C.c_int, C.c_int, C.c_float, C.POINTER(DF), vp, vp]
            L.pp_fz_to_df.restype = st
            L.pp_ff_convert.argtypes = [vp, C.POINTER(Grid), vp, C.POINTER(Grid), vp]
            L.pp_ff_convert.restype = st
            L.pp_backward_workspace.argtypes = [C.POINTER(Grid)]
            L.pp_backward_workspace.restype = C.c_size_t
            L.pp_backward.argtypes = [C.POINTER(Atoms), C.POINTER(Probe), C.POINTER(Grid), vp, C.POINTER(Scan),
                                      C.POINTER(Tip), C.POINTER(DF), vp, vp, C.POINTER(Grads), vp, C.c_size_t, vp]
            L.pp_backward.restype = st
            L.pp_backward_noalloc.argtypes = [C.POINTER(Atoms), C.POINTER(Probe), C.POINTER(Grid), vp,
                                              C.POINTER(Scan), C.POINTER(Tip), C.POINTER(DF), vp, vp,
                                              C.POINTER(Grads), vp]
            L.pp_backward_noalloc.restype = st
            L.pp_backward_noalloc_capacity.argtypes = []
            L.pp_backward_noalloc_capacity.restype = C.c_size_t
            L.pp_batch_workspace.argtypes = [C.c_int]
            L.pp_batch_workspace.restype = C.c_size_t
            L.pp_batch_run.argtypes = [vp, C.c_int, C.POINTER(BatchParams), C.POINTER(Atoms), vp, vp, vp, vp, vp,
                                       vp, C.c_size_t, vp]
            L.pp_batch_run.restype = st
            L.pp_batch_status.argtypes = [vp, C.POINTER(C.c_int), vp]
            L.pp_batch_status.restype = st
            L.pp_iets.argtypes = [vp, C.POINTER(Grid), C.POINTER(Scan), C.POINTER(Tip), vp, C.c_float, vp, vp, vp]
            L.pp_iets.restype = st
            L.pp_fft_workspace.argtypes = [C.POINTER(Grid)]
            L.pp_fft_workspace.restype = C.c_size_t
            L.pp_fft_correlate.argtypes = [vp, vp, C.POINTER(Grid), C.c_float, C.c_float, C.c_int, vp, vp,
                                           C.c_size_t, vp]
            L.pp_fft_correlate.restype = st
            L.pp_check_flags.argtypes = [C.POINTER(C.c_uint)]
            L.pp_check_flags.restype = st
            L.pp_read_probe.argtypes = [vp, C.c_size_t, C.c_int, vp, vp]
            L.pp_read_probe.restype = st
            L.pp_last_error.argtypes = []
            L.pp_last_error.restype = C.c_char_p
            _lib = L
    return _lib


def _check(status):
    if status != 0:
        raise PPError(status, lib().pp_last_error().decode())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _dev(t, name, dtype=torch.float32, allow_none=False):
    if t is None:
        if allow_none:
            return None
        raise ValueError(f"{name} is required")
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


# ----------------------------------------------------------------- structs

def make_grid(g, layout=0, brick=(4, 4, 4)):
    """Grid dict -> pp_grid; g["interp"] = 1 (optional) selects a tricubic energy grid (linear layout)."""
    interp = int(g.get("interp", 0))
    return Grid(int(g["nx"]), int(g["ny"]), int(g["nz"]), g["x0"], g["y0"], g["z0"], g["dx"], g["dy"], g["dz"],
                int(g["periodic_xy"]), 0 if interp else int(g.get("layout", layout)),
                *[int(b) for b in g.get("brick", brick)], interp)


def make_probe(p):
    return Probe(p["R_pp"], p["eps_pp"], p["Q"], p["coul_rc"], int(p["min_image"]), p["core_frac"],
                 float(p.get("Qzz", 0.0)))


def make_tip(t):
    return Tip(t["kx"], t["ky"], t["kR"], t["R0"], t["d0x"], t["d0y"])


def make_scan(s):
    return Scan(int(s["nx"]), int(s["ny"]), int(s["nz"]), s["x0"], s["y0"], s["px"], s["py"], s["z_top"], s["dz"])


def make_fire(f):
    return Fire(int(f["max_iter"]), f["ftol"], f["dt0"], f["dt_max"], f["f_inc"], f["f_dec"], f["alpha0"],
                f["f_alpha"], f["mass"], int(f["n_min"]), int(f.get("polish", 0)))


def make_df(d):
    return DF(d["A_pp"], d["k"], d["f0"])


def make_atoms(t):
    """t: dict of six float32 CUDA tensors x, y, z, R, eps, q (length n).

    The returned struct holds references to the tensors, so their device memory
    stays allocated for as long as the struct is alive."""
    n = int(t["x"].numel())
    ptrs = [_dev(t[k], k) if n > 0 else 0 for k in ("x", "y", "z", "R", "eps", "q")]
    for k in ("x", "y", "z", "R", "eps", "q"):
        if t[k].numel() != n:
            raise ValueError("atom arrays differ in length")
    a = Atoms(n, *ptrs)
    a._tensors = dict(t)
    return a


# ----------------------------------------------------------------- entry points

def pp_ff_floats(grid: Grid) -> int:
    return int(lib().pp_ff_floats(C.byref(grid)))


def pp_df_margin(A_pp: float, dz: float) -> int:
    return int(lib().pp_df_margin(A_pp, dz))


def pp_make_ff(atoms: Atoms, probe: Probe, grid: Grid, ff: torch.Tensor, stream=None):
    if ff.numel() < pp_ff_floats(grid):
        raise ValueError("ff buffer smaller than pp_ff_floats(grid)")
    _check(lib().pp_make_ff(C.byref(atoms), C.byref(probe), C.byref(grid), _dev(ff, "ff"), _stream(stream)))


def pp_make_ff_tuned(atoms: Atoms, probe: Probe, grid: Grid, ff: torch.Tensor, tuning=None, stream=None):
    if ff.numel() < pp_ff_floats(grid):
        raise ValueError("ff buffer smaller than pp_ff_floats(grid)")
    _check(lib().pp_make_ff_tuned(C.byref(atoms), C.byref(probe), C.byref(grid), _dev(ff, "ff"),
                                  C.byref(tuning) if tuning is not None else None, _stream(stream)))


def pp_make_ff_layers(atoms: Atoms, probe: Probe, grid: Grid, ff: torch.Tensor, k_begin: int, k_end: int,
                      tuning=None, stream=None):
    """Node layers k_begin <= k < k_end of the grid (the values pp_make_ff_tuned writes there)."""
    if ff.numel() < pp_ff_floats(grid):
        raise ValueError("ff buffer smaller than pp_ff_floats(grid)")
    _check(lib().pp_make_ff_layers(C.byref(atoms), C.byref(probe), C.byref(grid), _dev(ff, "ff"),
                                   C.byref(tuning) if tuning is not None else None, int(k_begin), int(k_end),
                                   _stream(stream)))


def pp_make_ff_split(atoms: Atoms, probe: Probe, grid: Grid, ff: torch.Tensor, ff_el: torch.Tensor, stream=None):
    """LJ (+ quadrupole) into ff, point-charge electrostatics per unit probe charge into ff_el."""
    n = pp_ff_floats(grid)
    if ff.numel() < n or ff_el.numel() < n:
        raise ValueError("ff / ff_el buffer smaller than pp_ff_floats(grid)")
    _check(lib().pp_make_ff_split(C.byref(atoms), C.byref(probe), C.byref(grid), _dev(ff, "ff"), _dev(ff_el, "ff_el"),
                                  _stream(stream)))


def pp_ff_combine(ff: torch.Tensor, ff_el: torch.Tensor, Q: float, grid: Grid, out: torch.Tensor, stream=None):
    """out = ff + Q ff_el (the grid for probe charge Q); out may be ff."""
    n = pp_ff_floats(grid)
    if ff.numel() < n or ff_el.numel() < n or out.numel() < n:
        raise ValueError("buffer smaller than pp_ff_floats(grid)")
    _check(lib().pp_ff_combine(_dev(ff, "ff"), _dev(ff_el, "ff_el"), float(Q), C.byref(grid), _dev(out, "out"),
                               _stream(stream)))


def pp_relax_scan(ff, grid: Grid, scan: Scan, tip: Tip, fire: Fire, pos, fz, iters, fused_df=None, df=None,
                  stream=None, zspan=None, plan=None):
    """zspan: a device int32 tensor of 2 elements to receive the lowest and highest node layer the scan's
    interpolations read; plan: (buffer, k, lanes) from pp_relax_plan.  With either, pp_relax_scan_ex."""
    npx = scan.nx * scan.ny * scan.nz
    if fz.numel() < npx or (pos is not None and pos.numel() < 3 * npx) or (iters is not None and iters.numel() < npx):
        raise ValueError("output buffer too small for the scan")
    if ff.numel() < pp_ff_floats(grid):
        raise ValueError("ff buffer smaller than pp_ff_floats(grid)")
    if df is not None and fused_df is not None:
        m = pp_df_margin(fused_df.A_pp, scan.dz)
        if m >= 0 and df.numel() < (scan.nz - 2 * m) * scan.nx * scan.ny:
            raise ValueError("df buffer too small")
    args = (_dev(ff, "ff"), C.byref(grid), C.byref(scan), C.byref(tip), C.byref(fire),
            _dev(pos, "pos", allow_none=True), _dev(fz, "fz"), _dev(iters, "iters", torch.int32, allow_none=True),
            C.byref(fused_df) if fused_df is not None else None, _dev(df, "df", allow_none=True))
    if zspan is None and plan is None:
        _check(lib().pp_relax_scan(*args, _stream(stream)))
        return
    opts = ScanOpts(None, None, 0, 0)
    if zspan is not None:
        if zspan.numel() < 2:
            raise ValueError("zspan needs two ints")
        opts.zspan = _dev(zspan, "zspan", torch.int32)
    if plan is not None:
        buf, k, lanes = plan
        if buf.numel() * buf.element_size() < pp_relax_plan_size(scan, k, lanes):
            raise ValueError("plan buffer smaller than pp_relax_plan_size")
        opts.plan, opts.plan_k, opts.plan_lanes = _dev(buf, "plan", torch.int32), int(k), int(lanes)
    _check(lib().pp_relax_scan_ex(*args, C.byref(opts), _stream(stream)))


def pp_relax_plan_size(scan: Scan, k: int, lanes: int) -> int:
    return int(lib().pp_relax_plan_size(C.byref(scan), int(k), int(lanes)))


def pp_relax_plan(iters, scan: Scan, max_iter: int, k: int, lanes: int, plan, stream=None):
    """Pixel-to-warp plan (an int32 device tensor of pp_relax_plan_size bytes) from an earlier scan's iters."""
    n = pp_relax_plan_size(scan, k, lanes)
    if n and plan.numel() * plan.element_size() < n:
        raise ValueError("plan buffer smaller than pp_relax_plan_size")
    if iters.numel() < scan.nx * scan.ny * scan.nz:
        raise ValueError("iters smaller than the scan")
    _check(lib().pp_relax_plan(_dev(iters, "iters", torch.int32), C.byref(scan), int(max_iter), int(k), int(lanes),
                               _dev(plan, "plan", torch.int32), _stream(stream)))


def pp_fz_to_df(fz, nz: int, npix: int, dz: float, df_params: DF, df, stream=None):
    m = pp_df_margin(df_params.A_pp, dz)
    if fz.numel() < nz * npix or (m >= 0 and df.numel() < max(nz - 2 * m, 0) * npix):
        raise ValueError("buffer too small")
    _check(lib().pp_fz_to_df(_dev(fz, "fz"), int(nz), int(npix), float(dz), C.byref(df_params), _dev(df, "df"),
                             _stream(stream)))


def pp_ff_convert(src, src_grid: Grid, dst, dst_grid: Grid, stream=None):
    if src.numel() < pp_ff_floats(src_grid) or dst.numel() < pp_ff_floats(dst_grid):
        raise ValueError("buffer too small")
    _check(lib().pp_ff_convert(_dev(src, "src"), C.byref(src_grid), _dev(dst, "dst"), C.byref(dst_grid),
                               _stream(stream)))


def pp_backward_workspace(grid: Grid) -> int:
    return int(lib().pp_backward_workspace(C.byref(grid)))


def make_grads(g):
    """g: dict of float32 CUDA tensors x, y, z, q, R, eps (n each) and tip (5)."""
    n = int(g["x"].numel())
    if g["tip"].numel() < 5:
        raise ValueError("tip gradient needs 5 floats")
    gr = Grads(*[_dev(g[k], k) if n > 0 else 0 for k in ("x", "y", "z", "q", "R", "eps")], _dev(g["tip"], "tip"))
    gr._tensors = dict(g)
    return gr


def pp_backward(atoms: Atoms, probe: Probe, grid: Grid, ff, scan: Scan, tip: Tip, df_params: DF, pos, g_df,
                grads: Grads, ws, stream=None):
    npx = scan.nx * scan.ny * scan.nz
    m = pp_df_margin(df_params.A_pp, scan.dz)
    if pos.numel() < 3 * npx or (m >= 0 and g_df.numel() < max(scan.nz - 2 * m, 0) * scan.nx * scan.ny):
        raise ValueError("pos or g_df smaller than the scan")
    if ff.numel() < pp_ff_floats(grid):
        raise ValueError("ff buffer smaller than pp_ff_floats(grid)")
    _check(lib().pp_backward(C.byref(atoms), C.byref(probe), C.byref(grid), _dev(ff, "ff"), C.byref(scan),
                             C.byref(tip), C.byref(df_params), _dev(pos, "pos"), _dev(g_df, "g_df"), C.byref(grads),
                             _dev(ws, "ws", ws.dtype), ws.numel() * ws.element_size(), _stream(stream)))


def pp_backward_noalloc_capacity() -> int:
    return int(lib().pp_backward_noalloc_capacity())


def pp_backward_noalloc(atoms: Atoms, probe: Probe, grid: Grid, ff, scan: Scan, tip: Tip, df_params: DF, pos, g_df,
                        grads: Grads, stream=None):
    """pp_backward with the library's static scratch (no workspace argument, nothing allocated)."""
    npx = scan.nx * scan.ny * scan.nz
    m = pp_df_margin(df_params.A_pp, scan.dz)
    if pos.numel() < 3 * npx or (m >= 0 and g_df.numel() < max(scan.nz - 2 * m, 0) * scan.nx * scan.ny):
        raise ValueError("pos or g_df smaller than the scan")
    if ff.numel() < pp_ff_floats(grid):
        raise ValueError("ff buffer smaller than pp_ff_floats(grid)")
    _check(lib().pp_backward_noalloc(C.byref(atoms), C.byref(probe), C.byref(grid), _dev(ff, "ff"), C.byref(scan),
                                     C.byref(tip), C.byref(df_params), _dev(pos, "pos"), _dev(g_df, "g_df"),
                                     C.byref(grads), _stream(stream)))


def pp_batch_workspace(nmol: int) -> int:
    return int(lib().pp_batch_workspace(int(nmol)))


def pp_batch_run(descs, nmol: int, params: BatchParams, atoms: Atoms, ff, pos, fz, iters, df, ws, stream=None):
    """descs: uint8 CUDA tensor holding nmol pp_mol_desc records."""
    if descs.numel() < nmol * C.sizeof(MolDesc):
        raise ValueError("descriptor buffer too small")
    _check(lib().pp_batch_run(_dev(descs, "descs", torch.uint8), int(nmol), C.byref(params), C.byref(atoms),
                              _dev(ff, "ff"), _dev(pos, "pos", allow_none=True), _dev(fz, "fz"),
                              _dev(iters, "iters", torch.int32, allow_none=True), _dev(df, "df"),
                              _dev(ws, "ws", ws.dtype), ws.numel() * ws.element_size(), _stream(stream)))


def pp_batch_status(ws, stream=None):
    """(pp_status, flags) of the last batch run on ws; synchronises the stream."""
    flags = C.c_int(0)
    st = lib().pp_batch_status(_dev(ws, "ws", ws.dtype), C.byref(flags), _stream(stream))
    return int(st), int(flags.value)


def pp_iets(ff, grid: Grid, scan: Scan, tip: Tip, pos, mass_amu: float, eig, hw=None, stream=None):
    npx = scan.nx * scan.ny * scan.nz
    if pos.numel() < 3 * npx or eig.numel() < 3 * npx or (hw is not None and hw.numel() < 3 * npx):
        raise ValueError("buffer smaller than the scan")
    if ff.numel() < pp_ff_floats(grid):
        raise ValueError("ff buffer smaller than pp_ff_floats(grid)")
    _check(lib().pp_iets(_dev(ff, "ff"), C.byref(grid), C.byref(scan), C.byref(tip), _dev(pos, "pos"),
                         float(mass_amu), _dev(eig, "eig"), _dev(hw, "hw", allow_none=True), _stream(stream)))


def pp_fft_workspace(grid: Grid) -> int:
    return int(lib().pp_fft_workspace(C.byref(grid)))


def pp_fft_correlate(f, g, grid: Grid, scale: float, power: float, ff, ws, accumulate=False, stream=None):
    """Cross-correlation force field of the sample field f and the tip density g ([nz][ny][nx]
    float32 CUDA tensors) into ff (written, or added when accumulate)."""
    n = grid.nx * grid.ny * grid.nz
    if f.numel() < n or g.numel() < n:
        raise ValueError("f and g need nx*ny*nz floats")
    if ff.numel() < pp_ff_floats(grid):
        raise ValueError("ff buffer smaller than pp_ff_floats(grid)")
    nbytes = ws.numel() * ws.element_size()
    _check(lib().pp_fft_correlate(_dev(f, "f"), _dev(g, "g"), C.byref(grid), float(scale), float(power),
                                  int(bool(accumulate)), _dev(ff, "ff"), _dev(ws, "ws", ws.dtype), nbytes,
                                  _stream(stream)))


def pp_check_flags() -> int:
    """Bits of the bounds checks hit since the last call (bounds-checked library only; raises
    PPError with PP_ERR_UNSUPPORTED on a normal build)."""
    flags = C.c_uint(0)
    _check(lib().pp_check_flags(C.byref(flags)))
    return flags.value


def pp_read_probe(buf, passes, sink, stream=None):
    """Read the float32 CUDA tensor buf `passes` times (L2 read-bandwidth probe); sink: one float."""
    _check(lib().pp_read_probe(_dev(buf, "buf"), buf.numel(), int(passes), _dev(sink, "sink"), _stream(stream)))


def pp_last_error() -> str:
    return lib().pp_last_error().decode()
