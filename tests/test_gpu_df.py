"""GPU parity of K3 (Fz -> df, Eq. df) against the FP64 oracle, and its closed-form limits."""
import numpy as np
import pytest
import torch

from paper_2401_14564_gb300 import pp

pytestmark = pytest.mark.gpu

EVA2_NM = 16.02176634


def gpu_df(fz, dz, dfp):
    fz_t = torch.as_tensor(np.asarray(fz, dtype=np.float32), device="cuda").contiguous()
    nz = fz_t.shape[0]
    npix = fz_t[0].numel()
    m = pp.pp_df_margin(dfp["A_pp"], dz)
    out = torch.empty((nz - 2 * m,) + tuple(fz_t.shape[1:]), dtype=torch.float32, device="cuda")
    pp.pp_fz_to_df(fz_t, nz, npix, dz, pp.make_df(dfp), out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("A,dz,nz,npix", [(1.0, 0.1, 20, 1000), (0.37, 0.1, 9, 333), (1.0, 0.05, 41, 7),
                                          (0.2, 0.1, 3, 1), (2.0, 0.1, 21, 4097)])
def test_random_columns_match_oracle(orc, A, dz, nz, npix):
    rng = np.random.default_rng(int(A * 100) + nz)
    fz = rng.standard_normal((nz, npix)).astype(np.float32) * 0.05
    dfp = {"A_pp": A, "k": 1800.0, "f0": 30300.0}
    got = gpu_df(fz, dz, dfp)
    ref = orc.fz_to_df(fz.astype(np.float64), float(np.float32(dz)), {"A_pp": float(np.float32(A)), "k": 1800.0,
                                                                       "f0": 30300.0})
    assert got.shape == ref.shape
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()


def test_linear_force_law(orc):
    z = 9.0 - 0.1 * np.arange(30)
    Fp = 0.02
    fz = (-0.05 + Fp * z)[:, None] * np.ones((1, 64))
    got = gpu_df(fz, 0.1, {"A_pp": 1.0, "k": 1800.0, "f0": 30300.0})
    np.testing.assert_allclose(got, -30300.0 * Fp * EVA2_NM / 3600.0, rtol=2e-5)


def test_empty_pixel_axis():
    got = gpu_df(np.zeros((12, 0)), 0.1, {"A_pp": 1.0, "k": 1800.0, "f0": 30300.0})
    assert got.shape == (2, 0)


@pytest.mark.parametrize("m", list(range(1, 10)))
def test_every_half_width_matches_oracle(orc, m):
    # half-widths 1..8 take the register-window kernel, 9 the generic one; heights and pixels
    # ragged against the 8-height and 256-pixel blocks
    dz = 0.1
    A = 2 * m * dz - 0.01
    nz, npix = 2 * m + 1 + 13, 523
    rng = np.random.default_rng(100 + m)
    fz = rng.standard_normal((nz, npix)).astype(np.float32) * 0.05
    dfp = {"A_pp": A, "k": 1800.0, "f0": 30300.0}
    assert pp.pp_df_margin(A, dz) == m
    got = gpu_df(fz, dz, dfp)
    ref = orc.fz_to_df(fz.astype(np.float64), float(np.float32(dz)), {"A_pp": float(np.float32(A)), "k": 1800.0,
                                                                       "f0": 30300.0})
    assert got.shape == ref.shape == (nz - 2 * m, npix)
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()


def test_slab_scan_shape_sampled_columns(orc):
    # the standalone kernel at the 2516-atom slab's scan shape (60 heights x 512 x 512 px, the
    # bench's df_standalone volume): 256 sampled pixel columns against the oracle
    nz, ny, nx = 60, 512, 512
    g = torch.Generator(device="cuda").manual_seed(11)
    fz = torch.randn((nz, ny, nx), generator=g, device="cuda") * 0.05
    dfp = {"A_pp": 1.0, "k": 1800.0, "f0": 30300.0}
    m = pp.pp_df_margin(1.0, 0.1)
    out = torch.empty((nz - 2 * m, ny, nx), device="cuda")
    pp.pp_fz_to_df(fz, nz, nx * ny, 0.1, pp.make_df(dfp), out)
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    cols = rng.integers(0, nx * ny, 256)
    f = fz.view(nz, -1)[:, cols].cpu().numpy().astype(np.float64)
    got = out.view(nz - 2 * m, -1)[:, cols].cpu().numpy()
    ref = orc.fz_to_df(f, float(np.float32(0.1)), dfp)
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()
    assert torch.isfinite(out).all()
