"""Pins of the oracle's frequency-shift conversion (Eq. df, Sec. 2.1).

Eq. df averages z * Fz(z) against 1/sqrt(A^2/4 - z^2) over one peak-to-peak
amplitude A.  Closed forms fix it: a force linear in z gives exactly
-f0 F'/(2k) for any amplitude; a constant force gives 0; an exponential force
F0 exp(-z/lambda) gives (f0/k) F0 exp(-z_c/lambda) I1(a/lambda)/a with a = A/2
(I1 from its power series here); small amplitudes tend to -f0 F'(z_c)/(2k).
"""
import math

import numpy as np
import pytest

EVA2_NM = 1.602176634e-19 / 1e-20  # 1 eV/A^2 in N/m, from SI


def bessel_i1(x, terms=40):
    return sum((x / 2) ** (2 * k + 1) / (math.factorial(k) * math.factorial(k + 1)) for k in range(terms))


@pytest.mark.parametrize("a,h", [(0.5, 0.1), (0.5, 0.05), (0.37, 0.1), (1.0, 0.3), (0.05, 0.1)])
def test_weights_moments(orc, a, h):
    W = orc.df_weights(a, h)
    m = (len(W) - 1) // 2
    u = h * np.arange(-m, m + 1)
    # odd kernel: zero on constants, antisymmetric weights
    assert abs(W.sum()) < 1e-14
    np.testing.assert_allclose(W, -W[::-1], atol=1e-15)
    # exact on linear functions: integral of u^2 / sqrt(a^2 - u^2) over [-a, a] = pi a^2 / 2
    assert (W * u).sum() == pytest.approx(math.pi * a * a / 2, rel=1e-13)


def _column(fz_of_z, z_top, dz, nz):
    z = z_top - dz * np.arange(nz)
    return z, fz_of_z(z)[:, None]


@pytest.mark.parametrize("A", [1.0, 0.6, 0.2])
def test_linear_force_exact(orc, A):
    f0, k = 30300.0, 1800.0
    F0, Fp = -0.05, 0.013  # eV/A and eV/A^2
    z, fz = _column(lambda z: F0 + Fp * z, 9.0, 0.1, 20)
    df = orc.fz_to_df(fz, 0.1, {"A_pp": A, "k": k, "f0": f0})
    np.testing.assert_allclose(df, -f0 * Fp * EVA2_NM / (2 * k), rtol=1e-12)


def test_constant_force_zero(orc):
    z, fz = _column(lambda z: np.full_like(z, 0.7), 9.0, 0.1, 20)
    df = orc.fz_to_df(fz, 0.1, {"A_pp": 1.0, "k": 1800.0, "f0": 30300.0})
    assert np.abs(df).max() < 1e-12


def test_exponential_force_closed_form(orc):
    f0, k, lam, F0, A = 30300.0, 1800.0, 0.6, -0.2, 1.0
    a = A / 2
    errs = []
    for dz in (0.1, 0.05, 0.025):
        nz = int(round(2.0 / dz)) + 1
        z, fz = _column(lambda z: F0 * np.exp(-z / lam), 6.0, dz, nz)
        df = orc.fz_to_df(fz, dz, {"A_pp": A, "k": k, "f0": f0})[:, 0]
        m = (nz - len(df)) // 2
        zc = z[m:nz - m]
        exact = (f0 / k) * F0 * np.exp(-zc / lam) * bessel_i1(a / lam) / a * EVA2_NM
        errs.append(np.abs(df / exact - 1).max())
    assert errs[0] < 2e-2
    # product integration of a piecewise-linear Fz: second order in dz
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5


def test_small_amplitude_limit(orc):
    f0, k, lam, F0 = 30300.0, 1800.0, 0.6, -0.2
    A, dz = 0.02, 0.002
    z, fz = _column(lambda z: F0 * np.exp(-z / lam), 5.0, dz, 41)
    df = orc.fz_to_df(fz, dz, {"A_pp": A, "k": k, "f0": f0})[:, 0]
    m = (41 - len(df)) // 2
    zc = z[m:41 - m]
    Fp = -F0 / lam * np.exp(-zc / lam)
    np.testing.assert_allclose(df, -f0 * Fp * EVA2_NM / (2 * k), rtol=1e-4)


def test_height_labels_and_direction(orc):
    # Fz is stored top-down (index k grows as the tip approaches); a force that grows toward
    # the sample (repulsive close range) must give a positive df
    z, fz = _column(lambda z: np.exp(-z), 4.0, 0.1, 15)
    df = orc.fz_to_df(fz, 0.1, {"A_pp": 1.0, "k": 1800.0, "f0": 30300.0})
    assert df.shape == (5, 1)
    assert (df > 0).all()
    assert np.all(np.diff(df[:, 0]) > 0)
