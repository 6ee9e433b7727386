"""Pins of the oracle's cross-correlation force fields (Eq. El_conv: Hartree
electrostatics, Eq. Pauli_FDBM: full-density Pauli repulsion), computed by
direct summation on a periodic grid with the spectral derivative for F.

Fixed independently of the oracle's code by:
  - a delta tip density returns the sample field itself (E = f) and F is the
    exact derivative of band-limited fields; the Nyquist mode has none;
  - a shifted delta shifts the field by whole nodes;
  - normalised Gaussians correlate into the Gaussian with the summed
    variance (closed form; the periodic trapezoidal sum is spectrally
    accurate for widths above ~2 spacings), with its analytic gradient;
  - the Pauli power beta: Gaussian^beta is again a Gaussian, closed form;
  - spot values equal the full computation.
"""
import numpy as np
import pytest

GRID = {"nx": 16, "ny": 20, "nz": 24, "x0": 0.0, "y0": 0.0, "z0": 0.0, "dx": 0.5, "dy": 0.45, "dz": 0.4,
        "periodic_xy": 1}


def coords(g):
    k, j, i = np.meshgrid(np.arange(g["nz"]), np.arange(g["ny"]), np.arange(g["nx"]), indexing="ij")
    return i * g["dx"], j * g["dy"], k * g["dz"]


def lengths(g):
    return g["nx"] * g["dx"], g["ny"] * g["dy"], g["nz"] * g["dz"]


def delta(g, off=(0, 0, 0)):
    d = np.zeros((g["nz"], g["ny"], g["nx"]))
    d[off[2], off[1], off[0]] = 1.0 / (g["dx"] * g["dy"] * g["dz"])
    return d


def band_limited(g):
    x, y, z = coords(g)
    Lx, Ly, Lz = lengths(g)
    kx, ky, kz = 2 * np.pi * 3 / Lx, 2 * np.pi * 2 / Ly, 2 * np.pi / Lz
    f = np.sin(kx * x) * np.cos(ky * y) * (1 + 0.5 * np.sin(kz * z))
    grad = (kx * np.cos(kx * x) * np.cos(ky * y) * (1 + 0.5 * np.sin(kz * z)),
            -ky * np.sin(kx * x) * np.sin(ky * y) * (1 + 0.5 * np.sin(kz * z)),
            0.5 * kz * np.sin(kx * x) * np.cos(ky * y) * np.cos(kz * z))
    return f, grad


def periodic_gaussian(g, c, s2, amp=None):
    """Normalised Gaussian of variance s2 centred at c, summed over the neighbouring images;
    returns the field and its gradient."""
    x, y, z = coords(g)
    Lx, Ly, Lz = lengths(g)
    norm = (2 * np.pi * s2) ** -1.5 if amp is None else amp
    val = np.zeros_like(x)
    grad = [np.zeros_like(x) for _ in range(3)]
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            for cc in (-1, 0, 1):
                dx, dy, dz = x - c[0] - a * Lx, y - c[1] - b * Ly, z - c[2] - cc * Lz
                e = norm * np.exp(-(dx * dx + dy * dy + dz * dz) / (2 * s2))
                val += e
                grad[0] -= e * dx / s2
                grad[1] -= e * dy / s2
                grad[2] -= e * dz / s2
    return val, grad


def test_delta_tip_returns_the_field_with_its_exact_derivative(orc):
    f, grad = band_limited(GRID)
    ff = orc.correlate(f, delta(GRID), GRID)
    assert np.allclose(ff[..., 3], f, atol=1e-12)
    for a in range(3):
        assert np.allclose(ff[..., a], -grad[a], atol=1e-10), a


def test_nyquist_mode_has_no_derivative(orc):
    x, y, z = coords(GRID)
    f = np.cos(np.pi * x / GRID["dx"]) * (1.0 + 0.0 * y)  # (-1)^i
    ff = orc.correlate(f, delta(GRID), GRID)
    assert np.allclose(ff[..., 3], f, atol=1e-12)
    assert np.abs(ff[..., :3]).max() < 1e-9


def test_shifted_delta_shifts_by_whole_nodes(orc):
    rng = np.random.default_rng(1)
    f = rng.standard_normal((GRID["nz"], GRID["ny"], GRID["nx"]))
    off = (3, 5, 2)
    ff = orc.correlate(f, delta(GRID, off), GRID, scale=2.5)
    want = 2.5 * np.roll(f, shift=(-off[2], -off[1], -off[0]), axis=(0, 1, 2))
    assert np.allclose(ff[..., 3], want, atol=1e-12)


def test_gaussians_correlate_into_the_summed_variance(orc):
    sf, sg = 0.7 ** 2, 0.9 ** 2
    c = (3.1, 4.0, 5.3)
    f, _ = periodic_gaussian(GRID, c, sf)
    g, _ = periodic_gaussian(GRID, (0.0, 0.0, 0.0), sg)
    ff = orc.correlate(f, g, GRID, scale=1.7)
    want, wgrad = periodic_gaussian(GRID, c, sf + sg)
    scale = np.abs(want).max()
    assert np.abs(ff[..., 3] - 1.7 * want).max() < 1e-8 * scale
    gs = max(np.abs(w).max() for w in wgrad)
    for a in range(3):
        assert np.abs(ff[..., a] + 1.7 * wgrad[a]).max() < 1e-7 * gs, a


def test_pauli_power_of_gaussians(orc):
    beta, sf, sg = 1.3, 0.8 ** 2, 0.75 ** 2
    nf, ng = 0.9, 1.4
    c = (4.2, 2.2, 6.1)
    f, _ = periodic_gaussian(GRID, c, sf, amp=nf)
    g, _ = periodic_gaussian(GRID, (0.0, 0.0, 0.0), sg, amp=ng)
    ff = orc.correlate(f, g, GRID, scale=0.6, power=beta)
    # (n e^{-r^2/2s})^beta = n^beta (2 pi s/beta)^{3/2} * normalised Gaussian of variance s/beta
    mass = nf ** beta * (2 * np.pi * sf / beta) ** 1.5 * ng ** beta * (2 * np.pi * sg / beta) ** 1.5
    want, wgrad = periodic_gaussian(GRID, c, (sf + sg) / beta)
    assert np.abs(ff[..., 3] - 0.6 * mass * want).max() < 1e-7 * 0.6 * mass * want.max()
    # negative samples count as zero under a non-integer power
    f2 = f.copy()
    f2[f2 < 1e-3 * nf] = -1.0
    ff2 = orc.correlate(np.where(f2 < 0, 0.0, f2), g, GRID, scale=0.6, power=beta)
    assert np.array_equal(orc.correlate(f2, g, GRID, scale=0.6, power=beta), ff2)


def test_spot_values_equal_the_full_field(orc):
    rng = np.random.default_rng(2)
    f = rng.random((GRID["nz"], GRID["ny"], GRID["nx"]))
    g = rng.random((GRID["nz"], GRID["ny"], GRID["nx"])) * (rng.random((GRID["nz"], GRID["ny"], GRID["nx"])) < 0.1)
    full = orc.correlate(f, g, GRID, scale=0.3, power=1.2)
    nodes = rng.choice(f.size, 25, replace=False)
    E = orc.correlate_nodes(f, g, GRID, nodes, scale=0.3, power=1.2)
    assert np.allclose(E, full[..., 3].reshape(-1)[nodes], rtol=1e-13, atol=0)
