"""GPU parity of pp_fft_correlate (cross-correlation force fields of Eqs.
El_conv and Pauli_FDBM through the convolution theorem) against the FP64
oracle's direct sum (tests/test_oracle_fft.py pins it).

Bar: every node's E and each force component within 2e-5 of the field's
maximum magnitude.  FP32 FFT rounding grows like log2(N) * 2^-24 of the
largest coefficient per transform (about 1e-6 for these sizes), and the
path takes three transforms and a spectral product.
"""
import numpy as np
import pytest
import torch

from paper_2401_14564_gb300 import pp, synth

pytestmark = pytest.mark.gpu

TOL = 2e-5


def run(f, g, grid, scale=1.0, power=1.0, ff=None, accumulate=False):
    gr = pp.make_grid(grid, 0)
    ft = torch.as_tensor(np.asarray(f, np.float32), device="cuda").contiguous()
    gt = torch.as_tensor(np.asarray(g, np.float32), device="cuda").contiguous()
    out = ff if ff is not None else torch.full((pp.pp_ff_floats(gr),), float("nan"), device="cuda")
    ws = torch.empty(pp.pp_fft_workspace(gr) // 4, dtype=torch.float32, device="cuda")
    pp.pp_fft_correlate(ft, gt, gr, scale, power, out, ws, accumulate=accumulate)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64).reshape(grid["nz"], grid["ny"], grid["nx"], 4)


def check(got, ref):
    # a component that vanishes identically (an axis of length 2 has only its Nyquist mode, whose
    # derivative is dropped) is measured against the field's largest component
    floor = 1e-6 * np.abs(ref).max()
    for c in range(4):
        scale = max(np.abs(ref[..., c]).max(), floor)
        err = np.abs(got[..., c] - ref[..., c]).max() / scale
        assert err <= TOL, (c, err)


def grid(nx, ny, nz, d=(0.2, 0.25, 0.3)):
    return {"nx": nx, "ny": ny, "nz": nz, "x0": 0.0, "y0": 0.0, "z0": 0.0, "dx": d[0], "dy": d[1], "dz": d[2],
            "periodic_xy": 1}


def fields(g, seed):
    rng = np.random.default_rng(seed)
    n = 12
    L = np.array([g["nx"] * g["dx"], g["ny"] * g["dy"], g["nz"] * g["dz"]])
    f = synth.periodic_gaussians(g, rng.random((n, 3)) * L, rng.uniform(0.5, 2.0, n), rng.uniform(0.4, 0.9, n))
    tip = synth.periodic_gaussians(g, [(0.0, 0.0, 0.0), (0.3, -0.2, 0.4)], [2.0, 0.7], [0.6, 0.5])
    return f, tip


@pytest.mark.parametrize("shape", [(16, 32, 8), (32, 16, 16), (8, 8, 64)])
def test_electrostatic_correlation_matches_oracle(orc, shape):
    g = grid(*shape)
    f, tip = fields(g, 1)
    f = f - f.mean()  # a potential: both signs
    check(run(f, tip, g), orc.correlate(f, tip, g))


def test_pauli_power_matches_oracle(orc):
    g = grid(32, 16, 16)
    f, tip = fields(g, 2)
    check(run(f, tip, g, scale=0.7, power=1.3), orc.correlate(f, tip, g, scale=0.7, power=1.3))


def test_accumulate_adds_to_the_grid(orc):
    g = grid(16, 16, 16)
    f, tip = fields(g, 3)
    base = torch.randn(16 * 16 * 16 * 4, device="cuda")
    before = base.cpu().numpy().astype(np.float64).reshape(16, 16, 16, 4)
    got = run(f, tip, g, ff=base, accumulate=True)
    check(got - before, orc.correlate(f, tip, g))


def test_gaussians_at_a_large_size_against_the_closed_form():
    # 128 x 128 x 64: too large for the direct sum, so the Gaussian closed form (summed variance)
    g = grid(128, 128, 64, d=(0.1, 0.1, 0.2))
    c = np.array([6.3, 7.1, 5.9])
    sf, sg = 0.6, 0.8
    f = synth.periodic_gaussians(g, [c], [1.0], [sf])
    tip = synth.periodic_gaussians(g, [(0.0, 0.0, 0.0)], [1.0], [sg])
    got = run(f, tip, g, scale=2.0)
    want = 2.0 * synth.periodic_gaussians(g, [c], [1.0], [np.hypot(sf, sg)])
    assert np.abs(got[..., 3] - want).max() <= TOL * want.max()
    # force: the analytic gradient of the Gaussian (nearest image suffices at this width)
    k, j, i = np.meshgrid(np.arange(g["nz"]), np.arange(g["ny"]), np.arange(g["nx"]), indexing="ij")
    r = [i * g["dx"] - c[0], j * g["dy"] - c[1], k * g["dz"] - c[2]]
    Ls = [g["nx"] * g["dx"], g["ny"] * g["dy"], g["nz"] * g["dz"]]
    r = [ra - La * np.round(ra / La) for ra, La in zip(r, Ls)]
    s2 = sf * sf + sg * sg
    for a in range(3):
        Fa = want * r[a] / s2  # F = -grad E = E r / s^2
        assert np.abs(got[..., a] - Fa).max() <= TOL * np.abs(Fa).max(), a


def test_spot_values_at_a_large_size(orc):
    g = grid(64, 64, 128, d=(0.1, 0.1, 0.125))
    f, tip = fields(g, 4)
    got = run(f, tip, g, scale=0.5, power=1.1)
    nodes = np.random.default_rng(5).choice(f.size, 16, replace=False)
    E = orc.correlate_nodes(f, tip, g, nodes, scale=0.5, power=1.1)
    assert np.abs(got[..., 3].reshape(-1)[nodes] - E).max() <= TOL * np.abs(got[..., 3]).max()


@pytest.mark.parametrize("shape", [(1024, 4, 8), (8, 1024, 4), (4, 8, 1024)])
def test_longest_axes(orc, shape):
    # the longest supported axis (1024: three radix-8 stages and a radix-2 one, 4 lines per tile)
    # along x, y and z; energies at seeded nodes against the direct sum
    g = grid(*shape, d=(0.05, 0.07, 0.06))
    f, tip = fields(g, sum(shape) + 1)
    got = run(f, tip, g, scale=1.7)
    nodes = np.random.default_rng(6).choice(f.size, 24, replace=False)
    E = orc.correlate_nodes(f, tip, g, nodes, scale=1.7)
    assert np.abs(got[..., 3].reshape(-1)[nodes] - E).max() <= TOL * np.abs(got[..., 3]).max()
    assert np.isfinite(got).all()


def test_fdbm_force_field_on_a_graphene_cell(orc):
    # the full-density model's two terms on a small periodic graphene cell: Hartree electrostatics
    # of the quadrupolar tip charge plus Pauli repulsion of the tip density, accumulated into one grid
    c = synth.graphene_sweep_case(3, 2, nz=32, lz=8.0)
    g = c["grid"]
    rho = synth.valence_density(g, c["atoms"])
    V = synth.hartree_potential(g, c["atoms"])
    pauli, quad = synth.tip_densities(g)
    got = run(V, quad, g)
    got = run(rho, pauli, g, scale=18.0, power=1.05, ff=torch.as_tensor(got.reshape(-1).astype(np.float32),
                                                                        device="cuda"), accumulate=True)
    ref = orc.correlate(V, quad, g) + orc.correlate(rho, pauli, g, scale=18.0, power=1.05)
    check(got, ref)
