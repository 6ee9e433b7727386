"""The C-ABI library loads without a GPU, exports every entry point that
include/pp.h declares, and rejects bad arguments on the host before any launch."""
import ctypes
import ctypes as C

import pytest

from paper_2401_14564_gb300 import build, pp


@pytest.fixture(scope="module")
def L():
    build.build()
    return pp.lib()


def test_exports_every_declared_symbol(L):
    names = pp.declared_symbols()
    assert {"pp_make_ff", "pp_relax_scan", "pp_fz_to_df", "pp_last_error"} <= set(names)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_ff_floats_and_layouts(L):
    g = pp.make_grid({"nx": 10, "ny": 6, "nz": 5, "x0": 0, "y0": 0, "z0": 0, "dx": 0.1, "dy": 0.1, "dz": 0.1,
                      "periodic_xy": 1})
    assert pp.pp_ff_floats(g) == 10 * 6 * 5 * 4
    g.layout = 1
    g.bx, g.by, g.bz = 4, 4, 2
    assert pp.pp_ff_floats(g) == (3 * 4) * (2 * 4) * (3 * 2) * 4
    g.bx = 3
    assert pp.pp_ff_floats(g) == 0
    g.layout = 0
    g.nz = 1
    assert pp.pp_ff_floats(g) == 0


def test_df_margin(L):
    assert pp.pp_df_margin(1.0, 0.1) == 5
    assert pp.pp_df_margin(1.0, 0.3) == 2
    assert pp.pp_df_margin(0.0, 0.1) == -1
    assert pp.pp_df_margin(1.0, -0.1) == -1


def test_null_arguments_rejected_on_host(L):
    assert L.pp_make_ff(None, None, None, None, None) == 1
    assert b"NULL" in L.pp_last_error()
    assert L.pp_relax_scan(None, None, None, None, None, None, None, None, None, None, None) == 1
    assert L.pp_fz_to_df(None, 10, 10, C.c_float(0.1), None, None, None) == 1


def test_bad_shapes_rejected_on_host(L):
    grid = pp.make_grid({"nx": 1, "ny": 6, "nz": 5, "x0": 0, "y0": 0, "z0": 0, "dx": 0.1, "dy": 0.1, "dz": 0.1,
                         "periodic_xy": 1})
    probe = pp.make_probe({"R_pp": 1.66, "eps_pp": 0.0091, "Q": -0.1, "coul_rc": 0.0, "min_image": 0,
                           "core_frac": 0.5})
    atoms = pp.Atoms(0, None, None, None, None, None, None)
    fake = C.c_void_p(16)  # never dereferenced: the shape check fails first
    assert L.pp_make_ff(C.byref(atoms), C.byref(probe), C.byref(grid), fake, None) == 2
    assert b"nz >= 2" in L.pp_last_error() or b"nx, ny, nz" in L.pp_last_error()
    probe.core_frac = 1.5
    grid.nx = 4
    assert L.pp_make_ff(C.byref(atoms), C.byref(probe), C.byref(grid), fake, None) == 1
    dfp = pp.DF(1.0, 1800.0, 30300.0)
    # 5 heights cannot hold an 11-tap stencil
    assert L.pp_fz_to_df(fake, 5, 7, C.c_float(0.1), C.byref(dfp), fake, None) == 2
    dfp.A_pp = 10.0  # 101 taps
    assert L.pp_fz_to_df(fake, 200, 7, C.c_float(0.1), C.byref(dfp), fake, None) == 6


def test_ctypes_structs_match_the_c_header(tmp_path):
    """Every struct the binding passes has the same size and field offsets as pp.h (gcc)."""
    import os
    import subprocess

    structs = {"pp_atoms": pp.Atoms, "pp_probe": pp.Probe, "pp_grid": pp.Grid, "pp_tip": pp.Tip, "pp_scan": pp.Scan,
               "pp_fire": pp.Fire, "pp_df": pp.DF, "pp_grads": pp.Grads, "pp_mol_desc": pp.MolDesc,
               "pp_batch_params": pp.BatchParams, "pp_tuning": pp.Tuning}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pp.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(pp.HEADER))
    subprocess.run(["gcc", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l}
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_tricubic_grids_are_validated_on_host(L):
    g = pp.make_grid({"nx": 10, "ny": 6, "nz": 5, "x0": 0, "y0": 0, "z0": 0, "dx": 0.1, "dy": 0.1, "dz": 0.1,
                      "periodic_xy": 1, "interp": 1})
    assert pp.pp_ff_floats(g) == 10 * 6 * 5
    g.layout = 1
    assert pp.pp_ff_floats(g) == 0  # energy grids are linear
    g.layout = 0
    g.interp = 2
    assert pp.pp_ff_floats(g) == 0
    g.interp = 1
    fake = C.c_void_p(16)  # never dereferenced: the grid check fails first
    atoms = pp.Atoms(0, None, None, None, None, None, None)
    probe = pp.make_probe({"R_pp": 1.66, "eps_pp": 0.0091, "Q": -0.1, "coul_rc": 0.0, "min_image": 0,
                           "core_frac": 0.5})
    scan = pp.make_scan({"nx": 4, "ny": 4, "nz": 12, "x0": 0.0, "y0": 0.0, "px": 0.1, "py": 0.1, "z_top": 0.3,
                         "dz": 0.1})
    tip = pp.make_tip({"kx": 0.25, "ky": 0.25, "kR": 20.0, "R0": 4.0, "d0x": 0.0, "d0y": 0.0})
    dfp = pp.DF(1.0, 1800.0, 30300.0)
    grads = pp.Grads(*([16] * 7))
    # the adjoint of an energy grid keeps one float per node; a smaller workspace is refused
    # before anything is read or launched
    assert L.pp_backward_workspace(C.byref(g)) == 256 + 4 * 10 * 6 * 5
    assert L.pp_backward(C.byref(atoms), C.byref(probe), C.byref(g), fake, C.byref(scan), C.byref(tip),
                         C.byref(dfp), fake, fake, C.byref(grads), fake, 256 + 4 * 10 * 6 * 5 - 4, None) == 4
    assert b"workspace too small" in L.pp_last_error()
    lin = pp.make_grid({"nx": 10, "ny": 6, "nz": 5, "x0": 0, "y0": 0, "z0": 0, "dx": 0.1, "dy": 0.1, "dz": 0.1,
                        "periodic_xy": 1})
    assert L.pp_ff_convert(fake, C.byref(g), fake, C.byref(lin), None) == 6


def test_fft_correlate_validated_on_host(L):
    def grid(nx, ny, nz, **kw):
        return pp.make_grid({"nx": nx, "ny": ny, "nz": nz, "x0": 0, "y0": 0, "z0": 0, "dx": 0.1, "dy": 0.1, "dz": 0.1,
                             "periodic_xy": 1, **kw})
    assert pp.pp_fft_workspace(grid(16, 8, 32)) == 3 * 32 * ((16 + 16) * 8 + 16) * 8  # padded rows and planes
    assert pp.pp_fft_workspace(grid(12, 8, 32)) == 0       # not a power of two
    assert pp.pp_fft_workspace(grid(16, 8, 2048)) == 0     # longer than 1024
    assert pp.pp_fft_workspace(grid(16, 8, 32, interp=1)) == 0
    fake = C.c_void_p(16)  # never dereferenced: the host checks fail first
    g = grid(12, 8, 32)
    assert L.pp_fft_correlate(fake, fake, C.byref(g), C.c_float(1), C.c_float(1), 0, fake, fake, 1 << 20, None) == 6
    g = grid(16, 8, 32)
    assert L.pp_fft_correlate(fake, fake, C.byref(g), C.c_float(1), C.c_float(1), 0, fake, fake, 100, None) == 4
    assert L.pp_fft_correlate(fake, fake, C.byref(g), C.c_float(1), C.c_float(0), 0, fake, fake, 1 << 20, None) == 1
    assert L.pp_fft_correlate(None, fake, C.byref(g), C.c_float(1), C.c_float(1), 0, fake, fake, 1 << 20, None) == 1
    # the sample field is read 16 bytes at a time
    assert L.pp_fft_correlate(C.c_void_p(20), fake, C.byref(g), C.c_float(1), C.c_float(1), 0, fake, fake, 1 << 20,
                              None) == 1
    assert b"aligned" in L.pp_last_error()


def test_split_and_combine_are_validated_on_host(L):
    g = pp.make_grid({"nx": 10, "ny": 6, "nz": 5, "x0": 0, "y0": 0, "z0": 0, "dx": 0.1, "dy": 0.1, "dz": 0.1,
                      "periodic_xy": 1})
    fake, other = C.c_void_p(16), C.c_void_p(32)  # never dereferenced: the host checks fail first
    atoms = pp.Atoms(0, None, None, None, None, None, None)
    probe = pp.make_probe({"R_pp": 1.66, "eps_pp": 0.0091, "Q": -0.1, "coul_rc": 0.0, "min_image": 0,
                           "core_frac": 0.5})
    assert L.pp_make_ff_split(C.byref(atoms), C.byref(probe), C.byref(g), fake, None, None) == 1
    assert b"ff_el" in L.pp_last_error()
    assert L.pp_make_ff_split(C.byref(atoms), C.byref(probe), C.byref(g), fake, fake, None) == 1
    assert b"different" in L.pp_last_error()
    assert L.pp_make_ff_split(C.byref(atoms), C.byref(probe), C.byref(g), fake, C.c_void_p(40), None) == 1
    assert b"aligned" in L.pp_last_error()
    assert L.pp_ff_combine(fake, other, C.c_float(float("nan")), C.byref(g), fake, None) == 1
    assert L.pp_ff_combine(fake, other, C.c_float(0.5), C.byref(g), C.c_void_p(8), None) == 1
    bad = pp.make_grid({"nx": 1, "ny": 6, "nz": 5, "x0": 0, "y0": 0, "z0": 0, "dx": 0.1, "dy": 0.1, "dz": 0.1,
                        "periodic_xy": 1})
    assert L.pp_ff_combine(fake, other, C.c_float(0.5), C.byref(bad), fake, None) == 2


def test_check_flags_unsupported_in_a_normal_build(L):
    flags = C.c_uint(7)
    assert L.pp_check_flags(C.byref(flags)) == 6 and flags.value == 0
    assert b"not a bounds-checked build" in L.pp_last_error()


def test_forces_only_option_is_validated_on_host(L):
    fake = C.c_void_p(16)  # never dereferenced: the host checks fail first
    atoms = pp.Atoms(0, None, None, None, None, None, None)
    probe = pp.make_probe({"R_pp": 1.66, "eps_pp": 0.0091, "Q": -0.1, "coul_rc": 0.0, "min_image": 0,
                           "core_frac": 0.5})
    g = pp.make_grid({"nx": 10, "ny": 6, "nz": 5, "x0": 0, "y0": 0, "z0": 0, "dx": 0.1, "dy": 0.1, "dz": 0.1,
                      "periodic_xy": 1})
    assert L.pp_make_ff_tuned(C.byref(atoms), C.byref(probe), C.byref(g), fake, C.byref(pp.Tuning(8, 2)), None) == 1
    assert b"ff_forces_only" in L.pp_last_error()
    # an energy-only grid has nothing but E to write
    g.interp = 1
    assert L.pp_make_ff_tuned(C.byref(atoms), C.byref(probe), C.byref(g), fake, C.byref(pp.Tuning(0, 1)), None) == 1
    assert b"interp = 1" in L.pp_last_error()


def test_noalloc_adjoint_validates_like_pp_backward(L):
    # pp_backward_noalloc makes pp_backward's checks in pp_backward's order (same status codes),
    # then its own capacity check; none of these calls reaches the GPU
    fake = C.c_void_p(256)  # never dereferenced: a check fails first
    atoms = pp.Atoms(0, None, None, None, None, None, None)
    probe = pp.make_probe({"R_pp": 1.66, "eps_pp": 0.0091, "Q": -0.1, "coul_rc": 0.0, "min_image": 0,
                           "core_frac": 0.5})
    scan = pp.make_scan({"nx": 4, "ny": 4, "nz": 12, "x0": 0.0, "y0": 0.0, "px": 0.1, "py": 0.1, "z_top": 0.3,
                         "dz": 0.1})
    tip = pp.make_tip({"kx": 0.25, "ky": 0.25, "kR": 20.0, "R0": 4.0, "d0x": 0.0, "d0y": 0.0})
    dfp = pp.DF(1.0, 1800.0, 30300.0)
    grads = pp.Grads(*([256] * 7))

    def grid(n):
        return pp.make_grid({"nx": n, "ny": n, "nz": 60, "x0": 0, "y0": 0, "z0": 0, "dx": 0.1, "dy": 0.1, "dz": 0.1,
                             "periodic_xy": 1})

    def both(g, pos=fake):
        gp = C.byref(g) if g is not None else None
        a = L.pp_backward(C.byref(atoms), C.byref(probe), gp, fake, C.byref(scan), C.byref(tip), C.byref(dfp), pos,
                          fake, C.byref(grads), fake, 1 << 40, None)
        b = L.pp_backward_noalloc(C.byref(atoms), C.byref(probe), gp, fake, C.byref(scan), C.byref(tip),
                                  C.byref(dfp), pos, fake, C.byref(grads), None)
        return a, b

    assert both(None) == (1, 1)                  # NULL grid: PP_ERR_ARG from both
    assert b"NULL" in L.pp_last_error()
    assert both(grid(1)) == (2, 2)               # invalid grid: PP_ERR_SHAPE from both
    big = grid(512)                              # 15.7 M nodes: beyond the static scratch
    assert L.pp_backward_workspace(C.byref(big)) > L.pp_backward_noalloc_capacity()
    assert both(big, pos=None) == (1, 1)         # a NULL argument wins over the capacity
    tip_bad = pp.make_tip({"kx": -1.0, "ky": 0.25, "kR": 20.0, "R0": 4.0, "d0x": 0.0, "d0y": 0.0})
    assert L.pp_backward_noalloc(C.byref(atoms), C.byref(probe), C.byref(big), fake, C.byref(scan),
                                 C.byref(tip_bad), C.byref(dfp), fake, fake, C.byref(grads), None) == 1
    assert L.pp_backward_noalloc(C.byref(atoms), C.byref(probe), C.byref(big), fake, C.byref(scan), C.byref(tip),
                                 C.byref(dfp), fake, fake, C.byref(grads), None) == 4
    assert b"static scratch" in L.pp_last_error()


def test_fire_polish_is_validated_on_host(L):
    fake = C.c_void_p(256)
    g = pp.make_grid({"nx": 8, "ny": 8, "nz": 8, "x0": 0, "y0": 0, "z0": 0, "dx": 0.1, "dy": 0.1, "dz": 0.1,
                      "periodic_xy": 1})
    scan = pp.make_scan({"nx": 4, "ny": 4, "nz": 12, "x0": 0.0, "y0": 0.0, "px": 0.1, "py": 0.1, "z_top": 0.3,
                         "dz": 0.1})
    tip = pp.make_tip({"kx": 0.25, "ky": 0.25, "kR": 20.0, "R0": 4.0, "d0x": 0.0, "d0y": 0.0})
    from paper_2401_14564_gb300 import synth

    for bad in (-1, 17):
        fire = pp.make_fire(synth.default_fire(polish=bad))
        assert L.pp_relax_scan(fake, C.byref(g), C.byref(scan), C.byref(tip), C.byref(fire), fake, fake, fake, None,
                               None, None) == 1
        assert b"FIRE" in L.pp_last_error()


def test_read_probe_validated_on_host(L):
    fake = C.c_void_p(256)
    assert L.pp_read_probe(None, 16, 1, fake, None) == 1
    assert L.pp_read_probe(C.c_void_p(8), 16, 1, fake, None) == 1      # not 16-byte aligned
    assert L.pp_read_probe(fake, 10, 1, fake, None) == 1               # not a multiple of 4 floats
    assert L.pp_read_probe(fake, 16, 0, fake, None) == 1               # no pass


def test_grid_axis_limit(L):
    # the cell lookup's add-based floor is exact below 2^22 nodes per axis: longer axes are refused
    ok = pp.make_grid({"nx": 1 << 22, "ny": 2, "nz": 2, "x0": 0, "y0": 0, "z0": 0, "dx": 0.1, "dy": 0.1, "dz": 0.1,
                       "periodic_xy": 1})
    assert pp.pp_ff_floats(ok) == 4 * (1 << 22) * 4
    bad = pp.make_grid({"nx": (1 << 22) + 1, "ny": 2, "nz": 2, "x0": 0, "y0": 0, "z0": 0, "dx": 0.1, "dy": 0.1,
                        "dz": 0.1, "periodic_xy": 1})
    assert pp.pp_ff_floats(bad) == 0


def test_ff_layers_and_zspan_validated_on_host(L):
    fake = C.c_void_p(256)  # never dereferenced: a host check fails first
    atoms = pp.Atoms(0, None, None, None, None, None, None)
    probe = pp.make_probe({"R_pp": 1.66, "eps_pp": 0.0091, "Q": -0.1, "coul_rc": 0.0, "min_image": 0,
                           "core_frac": 0.5})
    g = pp.make_grid({"nx": 10, "ny": 6, "nz": 5, "x0": 0, "y0": 0, "z0": 0, "dx": 0.1, "dy": 0.1, "dz": 0.1,
                      "periodic_xy": 1})
    for k0, k1 in ((-1, 3), (2, 2), (3, 2), (0, 6)):
        assert L.pp_make_ff_layers(C.byref(atoms), C.byref(probe), C.byref(g), fake, None, k0, k1, None) == 1
        assert b"k_begin" in L.pp_last_error()
    assert L.pp_make_ff_layers(None, C.byref(probe), C.byref(g), fake, None, 0, 2, None) == 1
    assert b"NULL" in L.pp_last_error()
    assert L.pp_make_ff_layers(C.byref(atoms), C.byref(probe), C.byref(g), fake, C.byref(pp.Tuning(5, 0)), 0, 2,
                               None) == 1
    bad = pp.make_grid({"nx": 1, "ny": 6, "nz": 5, "x0": 0, "y0": 0, "z0": 0, "dx": 0.1, "dy": 0.1, "dz": 0.1,
                        "periodic_xy": 1})
    assert L.pp_make_ff_layers(C.byref(atoms), C.byref(probe), C.byref(bad), fake, None, 0, 2, None) == 2

    scan = pp.make_scan({"nx": 4, "ny": 4, "nz": 12, "x0": 0.0, "y0": 0.0, "px": 0.1, "py": 0.1, "z_top": 0.3,
                         "dz": 0.1})
    tip = pp.make_tip({"kx": 0.25, "ky": 0.25, "kR": 20.0, "R0": 4.0, "d0x": 0.0, "d0y": 0.0})
    from paper_2401_14564_gb300 import synth

    fire = pp.make_fire(synth.default_fire())
    args = (fake, C.byref(g), C.byref(scan), C.byref(tip), C.byref(fire), fake, fake, fake, None, None)
    assert L.pp_relax_scan_ex(*args, None, None) == 1
    assert b"opts" in L.pp_last_error()
    opts = pp.ScanOpts(258, None, 0, 0)                                  # zspan not 4-byte aligned
    assert L.pp_relax_scan_ex(*args, C.byref(opts), None) == 1
    assert b"aligned" in L.pp_last_error()
    for k, lanes in ((0, 4), (4 * 4 + 1, 4), (8, 0), (8, 33)):          # the scan has 4 x 4 pixels
        opts = pp.ScanOpts(None, 256, k, lanes)
        assert L.pp_relax_scan_ex(*args, C.byref(opts), None) == 1
        assert b"plan_k" in L.pp_last_error()
    fire_bad = pp.make_fire(synth.default_fire(polish=-1))
    opts = pp.ScanOpts(256, None, 0, 0)
    assert L.pp_relax_scan_ex(fake, C.byref(g), C.byref(scan), C.byref(tip), C.byref(fire_bad), fake, fake, fake,
                              None, None, C.byref(opts), None) == 1     # pp_relax_scan's own checks follow
    assert b"pp_relax_scan_ex: invalid FIRE" in L.pp_last_error()


def test_relax_plan_validated_on_host(L):
    fake = C.c_void_p(256)
    scan = pp.make_scan({"nx": 10, "ny": 7, "nz": 12, "x0": 0.0, "y0": 0.0, "px": 0.1, "py": 0.1, "z_top": 0.3,
                         "dz": 0.1})
    n = L.pp_relax_plan_size(C.byref(scan), 5, 4)
    # header 8 + histogram 2048 + cost 70 + list ceil(5/4)*4 + mask ceil(70/32) int32 words
    assert n == 4 * (8 + 2048 + 70 + 8 + 3)
    for k, lanes in ((0, 4), (71, 4), (5, 0), (5, 33)):
        assert L.pp_relax_plan_size(C.byref(scan), k, lanes) == 0
        assert L.pp_relax_plan(fake, C.byref(scan), 200, k, lanes, fake, None) == 1
    assert L.pp_relax_plan(None, C.byref(scan), 200, 5, 4, fake, None) == 1
    assert L.pp_relax_plan(fake, C.byref(scan), 200, 5, 4, C.c_void_p(258), None) == 1
    assert L.pp_relax_plan(fake, C.byref(scan), -1, 5, 4, fake, None) == 1
    bad = pp.make_scan({"nx": 0, "ny": 7, "nz": 12, "x0": 0.0, "y0": 0.0, "px": 0.1, "py": 0.1, "z_top": 0.3,
                        "dz": 0.1})
    assert L.pp_relax_plan(fake, C.byref(bad), 200, 5, 4, fake, None) == 2
