"""Pins of the model terms: potential, indicator, splitting identities, recovery."""
import math

import numpy as np

from oracle import fd, model, spectral
from oracle import band as bm
from oracle.fft import fftn, ifftn_real
from paper_2606_04347_gb300 import workloads as wl


def test_potential_indicator_and_localisation_properties():
    s = np.linspace(0, 1, 100001)
    assert model.W(0.0) == 0 and model.W(1.0) == 0 and model.dW(0.0) == 0 and model.dW(1.0) == 0
    assert math.isclose(np.max(np.abs(model.d2W(s))), 36.0)            # L_W''
    f2 = np.gradient(model.df_ind(s), s)
    assert math.isclose(np.max(np.abs(f2[1:-1])), 6.0, rel_tol=1e-4)    # L_f''
    assert math.isclose(np.max(model.df_ind(s)), 1.5)                   # L_f'
    assert model.f_ind(0.0) == 0 and model.f_ind(1.0) == 1 and model.df_ind(0.0) == 0 and model.df_ind(1.0) == 0
    assert math.isclose(np.max(model.g_loc(s)), 1.125)                  # L_g
    # derivatives agree with finite differences of W and f
    assert np.allclose(np.gradient(model.W(s), s)[1:-1], model.dW(s)[1:-1], atol=1e-6)
    assert np.allclose(np.gradient(model.dW(s), s)[1:-1], model.d2W(s)[1:-1], atol=1e-5)
    assert np.allclose(np.gradient(model.f_ind(s), s)[1:-1], model.df_ind(s)[1:-1], atol=1e-8)


def test_tanh_profile_is_the_1d_equilibrium_of_W():
    # Phi = 0.5 + 0.5 tanh(3 x/eps) (Sec. 4.1) solves eps^2 Phi'' = W'(Phi)
    eps = 0.3
    x = np.linspace(-1, 1, 2001)
    t = np.tanh(3 * x / eps)
    phi = 0.5 + 0.5 * t
    phi_xx = 0.5 * (9 / eps ** 2) * (-2 * t * (1 - t * t))
    assert np.allclose(eps ** 2 * phi_xx, model.dW(phi), atol=1e-12)


def test_recovery_rule():
    G = np.array([0.5, 2e-3, 1e-3, 1e-6])
    GU = np.array([0.25, 1e-3, 7e-4, 3e-7])
    assert np.allclose(model.recover(GU, G, 1e-3), [0.5, 0.5, 7e-4, 3e-7])


def test_R1_minus_linear_part_is_force_balance_over_mu():
    p, phi, u, _ = wl.workload("c3", n=24)
    A0 = model.volume(phi, p) - 0.3
    r1 = model.R1(phi, u, p, A0)
    lphi = ifftn_real(spectral.l_phi(p, spectral.laplacian_symbol(p)) * fftn(phi))
    want = model.force_rhs(phi, u, p, A0)
    scale = np.max(np.abs(want))
    assert np.max(np.abs(r1 - lphi - want)) < 1e-10 * scale


def test_R2_plus_linear_part_is_OK_rhs_on_band():
    p, phi, u, _ = wl.workload("c3", n=24)
    h = p.h
    phi_old = phi + 1e-4 * np.random.default_rng(5).standard_normal(phi.shape)
    solver = model.BandSolver(p)
    r2 = model.R2_coupled(phi, phi_old, u, p, solver)
    g = model.g_loc(phi)
    band = bm.band_mask(phi)
    gu = g * u
    w = solver.w_prev
    rhs = (p.eps_u * fd.surface_laplacian(u, g, h) - g * model.dW(u) / p.eps_u
           - p.gamma * g * w - p.M * g * fd.inner(g, u - p.ubar, h)
           - model.advection_div(phi, phi_old, gu, p))
    lin = p.B2 * gu - p.eps_u * p.B1 * fd.laplacian(gu, h)     # L_u(gu) with the FD Laplacian
    assert np.max(np.abs((r2 - lin)[band] - rhs[band])) < 1e-10 * np.max(np.abs(rhs[band]))
    assert np.all(r2[~band] == 0)
    # the nonlocal solve: -Delta_S w = g (u - ubar) - mean on the band
    coeffs = bm.face_coeffs(g, band)
    lhs = bm.apply_neg_lap(w, coeffs, h)
    f = np.where(band, g * (u - p.ubar), 0.0)
    f = np.where(band, f - f[band].mean(), 0.0)
    assert np.max(np.abs(lhs - f)) < 1e-9 * np.max(np.abs(f))
