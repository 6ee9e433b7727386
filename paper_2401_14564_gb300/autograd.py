"""Differentiable df image: torch.autograd.Function over pp_make_ff / pp_relax_scan / pp_backward.

Forward runs the three CUDA stages and saves the force-field grid and the
relaxed positions; backward runs the implicit adjoint (pp_backward) and
returns gradients for the atom arrays (x, y, z, q, R, eps) and the tip
scalars (kx, ky, kR, Q, Qzz).  Only the df image is differentiable: Fz and
the relaxed positions come back marked non-differentiable.  Only argument
marshalling happens here.
"""
from __future__ import annotations

import copy

import torch

from . import pp

ATOM_KEYS = ("x", "y", "z", "q", "R", "eps")


class PPFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, y, z, q, R, eps, kx, ky, kR, Q, Qzz, case, layout, fire):
        dev = x.device
        probe = dict(case["probe"], Q=float(Q), Qzz=float(Qzz))
        tip = dict(case["tip"], kx=float(kx), ky=float(ky), kR=float(kR))
        grid = pp.make_grid(case["grid"], layout)
        scan = pp.make_scan(case["scan"])
        s = case["scan"]
        dfp = pp.make_df(case["df"])
        m = pp.pp_df_margin(dfp.A_pp, scan.dz)
        atoms_t = {"x": x.contiguous(), "y": y.contiguous(), "z": z.contiguous(), "q": q.contiguous(),
                   "R": R.contiguous(), "eps": eps.contiguous()}
        atoms = pp.make_atoms(atoms_t)
        ff = torch.empty(pp.pp_ff_floats(grid), dtype=torch.float32, device=dev)
        pos = torch.empty((s["nz"], s["ny"], s["nx"], 3), dtype=torch.float32, device=dev)
        fz = torch.empty((s["nz"], s["ny"], s["nx"]), dtype=torch.float32, device=dev)
        df = torch.empty((s["nz"] - 2 * m, s["ny"], s["nx"]), dtype=torch.float32, device=dev)
        pp_probe, pp_tip = pp.make_probe(probe), pp.make_tip(tip)
        pp.pp_make_ff(atoms, pp_probe, grid, ff)
        pp.pp_relax_scan(ff, grid, scan, pp_tip, pp.make_fire(fire or case["fire"]), pos, fz, None, dfp, df)
        ctx.save_for_backward(*[atoms_t[k] for k in ATOM_KEYS], ff, pos)
        ctx.meta = (probe, tip, grid, scan, dfp, tuple(df.shape))
        # Fz and the relaxed positions are returned for inspection only: the adjoint propagates the
        # df image's gradient, so a loss on either must not pass through here silently
        ctx.mark_non_differentiable(fz, pos)
        return df, fz, pos

    @staticmethod
    def backward(ctx, g_df, g_fz, g_pos):
        *atoms_l, ff, pos = ctx.saved_tensors
        probe, tip, grid, scan, dfp, df_shape = ctx.meta
        atoms_t = dict(zip(ATOM_KEYS, atoms_l))
        dev = ff.device
        n = atoms_t["x"].numel()
        grads = {k: torch.empty(n, dtype=torch.float32, device=dev) for k in ATOM_KEYS}
        grads["tip"] = torch.empty(5, dtype=torch.float32, device=dev)
        ws = torch.empty(pp.pp_backward_workspace(grid) // 4 + 4, dtype=torch.float32, device=dev)
        if g_df is None:
            g_df = torch.zeros(df_shape, dtype=torch.float32, device=dev)
        pp.pp_backward(pp.make_atoms(atoms_t), pp.make_probe(probe), grid, ff, scan, pp.make_tip(tip), dfp, pos,
                       g_df.contiguous().to(torch.float32), pp.make_grads(grads), ws)
        gt = grads["tip"].cpu()
        return (grads["x"], grads["y"], grads["z"], grads["q"], grads["R"], grads["eps"],
                gt[0], gt[1], gt[2], gt[3], gt[4], None, None, None)


def afm_df(atoms_t, kx, ky, kR, Q, case, layout=0, fire=None, Qzz=None):
    """Differentiable df image.  atoms_t: dict of float32 CUDA tensors; kx, ky, kR, Q and the
    optional tip quadrupole Qzz (default: the case's): 0-dim CPU tensors."""
    if Qzz is None:
        Qzz = torch.tensor(float(case["probe"].get("Qzz", 0.0)))
    df, fz, pos = PPFunction.apply(atoms_t["x"], atoms_t["y"], atoms_t["z"], atoms_t["q"], atoms_t["R"],
                                   atoms_t["eps"], kx, ky, kR, Q, Qzz, case, layout, fire)
    return df
