"""Pins of the spectral symbols and phi-functions."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import fft, model, spectral
from paper_2606_04347_gb300 import workloads as wl


def test_folded_wavenumbers_follow_sec32():
    # lambda_x(i) = (pi/X) i for i <= N/2 and (pi/X)(N - i) above (Sec. 3.2); X = pi, N = 8
    assert spectral.folded_wavenumbers(8, math.pi).tolist() == [0, 1, 2, 3, 4, 3, 2, 1]
    assert np.allclose(spectral.folded_wavenumbers(8, 1.0), math.pi * np.array([0, 1, 2, 3, 4, 3, 2, 1]))
    k = spectral.signed_wavenumbers(8, math.pi)
    assert k.tolist() == [0, 1, 2, 3, 0, -3, -2, -1]


def test_spectral_laplacian_and_gradient_of_eigenfunctions():
    p = wl.ModelParams(dim=3, n=(16, 8, 32), half_len=(math.pi, 2.0, 3.0))
    x, y, z = wl.grid(p.n, p.half_len, 3)
    kx, ky, kz = 3.0, 2 * math.pi / 4.0 * 1, 2 * math.pi / 6.0 * 5
    f = np.sin(kx * x) * np.cos(ky * y) * np.cos(kz * z) * np.ones(p.shape)
    lap = model.spectral_lap(f, p)
    assert np.max(np.abs(lap + (kx * kx + ky * ky + kz * kz) * f)) < 1e-10
    gx, gy, gz = model.spectral_grad(f, p)
    want = kx * np.cos(kx * x) * np.cos(ky * y) * np.cos(kz * z)
    assert np.max(np.abs(gx - want)) < 1e-11


def test_linear_symbols_at_zero_and_growth():
    p = wl.workload("c3", n=8)[0]
    lam = np.array([0.0, -1.0, -5.0])
    e2 = p.eps_phi ** 2
    # at lambda = 0 only the constant term of l^phi survives (Sec. 3.2)
    assert math.isclose(spectral.l_phi(p, lam)[0], (p.kappa * p.A1 * p.A2 + p.lambda_surf * p.A1 * e2) / (p.mu * e2 * e2))
    assert math.isclose(spectral.l_u(p, lam)[0], p.B2)
    assert np.all(np.diff(spectral.l_phi(p, lam)) > 0) and np.all(np.diff(spectral.l_u(p, lam)) > 0)


def _phi_quad(z, j):
    if j == 1:
        return integrate.quad(lambda s: math.exp(-z * (1 - s)), 0, 1, epsabs=0, epsrel=2e-14)[0]
    return integrate.quad(lambda s: s * math.exp(-z * (1 - s)), 0, 1, epsabs=0, epsrel=2e-14)[0]


def test_phi_functions_against_quadrature_and_limits():
    zs = np.array([0.0, 1e-12, 1e-6, 0.3, 0.999, 1.0, 1.001, 2.0, 10.0, 50.0])
    p0, p1, p2 = spectral.phi_functions(zs)
    for z, a1, a2 in zip(zs, p1, p2):
        assert math.isclose(a1, _phi_quad(z, 1), rel_tol=1e-12)
        assert math.isclose(a2, _phi_quad(z, 2), rel_tol=1e-12)
    assert p1[0] == 1.0 and p2[0] == 0.5
    assert np.all(p0 > 0) and np.all(p1 > 0) and np.all(p2 > 0)


def test_phi_functions_against_multiprecision():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    zs = np.concatenate([np.logspace(-10, 6, 60), [0.5, 0.9999999, 1.0000001]])
    p0, p1, p2 = spectral.phi_functions(zs)
    for z, a0, a1, a2 in zip(zs, p0, p1, p2):
        Z = mpmath.mpf(float(z))
        e = mpmath.exp(-Z)
        assert math.isclose(a0, float(e), rel_tol=4e-16, abs_tol=1e-300)
        assert math.isclose(a1, float((1 - e) / Z), rel_tol=2e-15)
        assert math.isclose(a2, float((e - 1 + Z) / Z ** 2), rel_tol=2e-15)
