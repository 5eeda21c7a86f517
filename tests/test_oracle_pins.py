"""Pins of the oracle's model terms against independent mathematics (CPU only).

* The OK remainders R2 (fixed model and coupled model without advection) against the L2
  gradient of the discrete energy: Eq. (1.2) and the fixed-membrane equation of Sec. 1 are
  the L2-gradient flows of the membrane OK energy (Eq. (1.3); discrete form Eq. (2.16)), so
  R2 - L_u(g u) must equal -h^-d dE_h/dU, with E_h built from the dense matrices of the Sec. 2
  scheme and differentiated numerically.  Pins the sign and operand of the nonlocal term,
  the mass term, the well term and the surface Laplacian of both R2 functions.
* model.energy against section2.DenseScheme.energy on a grid whose band is the whole grid.
* The line-tension, area and alpha terms of R1 (Eq. (1.1), Sec. 3.1) on single-Fourier-mode
  membranes, where |grad phi|, Delta phi, <phi, 1>_h and the discrete surface Laplacian of a
  sine are known in closed form.
* The advection divergence (Sec. 1, v = -d_t phi grad phi / |grad phi|^2) for a rigidly
  translated profile, where v is a constant vector in closed form.
* One coupled ETD1/ETDRK2 step of the oracle's driver against the same step taken with dense
  matrix functions phi_j(tau L) of the two linear operators (scipy expm of augmented
  matrices), R1 and R2 from the functions pinned above.
"""
import math

import numpy as np
import pytest
from scipy.linalg import expm

from oracle import band as bm
from oracle import etd, fd, model, section2, spectral
from paper_2606_04347_gb300 import workloads as wl


# ---------------------------------------------------------------- full-band 2D grid
def _fullband_case(n=10):
    p = wl.workload("c1", n=n)[0].replace(eps_u=0.35, gamma=40.0, M=15.0, ubar=0.45, B1=1.0, B2=300.0,
                                          cg_rtol=1e-15)
    x, y = wl.grid(p.n, p.half_len, 2)
    phi = 0.5 + 0.3 * np.sin(x) * np.cos(y) + 0.05 * np.cos(2 * y)
    assert np.all(bm.band_mask(phi, p.band_mask_hi))        # the band is the whole grid
    U = wl.random_fields(p.shape, 31, 0.15, 0.85)
    return p, phi, U


def _grad(E, U, d=1e-3):
    """Fourth-order central differences of E at U, one component at a time."""
    out = np.zeros(U.size)
    base = U.ravel()
    for i in range(U.size):
        vals = []
        for s in (2, 1, -1, -2):
            V = base.copy()
            V[i] += s * d
            vals.append(E(V))
        out[i] = (-vals[0] + 8 * vals[1] - 8 * vals[2] + vals[3]) / (12 * d)
    return out.reshape(U.shape)


def test_model_energy_matches_dense_sec2_energy():
    p, phi, U = _fullband_case()
    h = p.h[:2]
    ds = section2.DenseScheme(phi, h, eps_u=p.eps_u, gamma=p.gamma, M=p.M, ubar=p.ubar, B=1.0)
    g = model.g_loc(phi)
    band = bm.band_mask(phi, p.band_mask_hi)
    e = model.energy(U, g, band, p, rtol=1e-15)
    assert math.isclose(e["total"], ds.energy(U.ravel()), rel_tol=1e-11)


def test_fixed_R2_is_minus_energy_gradient():
    p, phi, U = _fullband_case()
    h = p.h[:2]
    dx = float(np.prod(h))
    ds = section2.DenseScheme(phi, h, eps_u=p.eps_u, gamma=p.gamma, M=p.M, ubar=p.ubar, B=1.0)
    g = model.g_loc(phi)
    band = bm.band_mask(phi, p.band_mask_hi)
    r2 = model.R2_fixed(U, g, band, p, model.BandSolver(p))
    gu = g * U
    N = r2 - (p.B2 * gu - p.eps_u * p.B1 * fd.laplacian(gu, h))     # remove L_u(g u)
    want = -_grad(lambda V: ds.energy(V), U) / dx
    assert np.max(np.abs(N - want)) < 1e-7 * np.max(np.abs(want))


def test_coupled_R2_without_motion_is_minus_energy_gradient():
    """Eq. (1.2) with v = 0 (phi_old = phi): R2 - L_u(g u) = -h^-d dE/dU of the energy with the
    coupled operands g (u - ubar) in the nonlocal and mass terms."""
    p, phi, U = _fullband_case()
    h = p.h[:2]
    dx = float(np.prod(h))
    ds = section2.DenseScheme(phi, h, eps_u=p.eps_u, gamma=p.gamma, M=p.M, ubar=p.ubar, B=1.0)
    g = ds.g

    def E(V):
        q = g * (V - p.ubar)
        return (0.5 * p.eps_u * dx * float(V @ (-ds.DS @ V)) + dx * float(np.sum(g * model.W(V))) / p.eps_u
                + 0.5 * p.gamma * dx * float((ds.Kinv @ q) @ q) + 0.5 * p.M * (dx * float(np.sum(q))) ** 2)

    r2 = model.R2_coupled(phi, phi, U, p, model.BandSolver(p))
    gu = model.g_loc(phi) * U
    N = r2 - (p.B2 * gu - p.eps_u * p.B1 * fd.laplacian(gu, h))
    want = -_grad(E, U) / dx
    assert np.max(np.abs(N - want)) < 1e-7 * np.max(np.abs(want))


# ---------------------------------------------------------------- R1 on single modes
def _mode3d(n=16):
    p = wl.workload("c3", n=n)[0]
    x, y, z = wl.grid(p.n, p.half_len, 3)
    return p, x, y, z


def test_R1_alpha_term_on_a_single_mode():
    """u = 1 and u = 0 are wells of W, so the line term vanishes for both and the difference of
    R1 is the alpha term alone: (alpha/mu) |grad phi| (eps Delta phi - W'(phi)/eps)."""
    p, x, y, z = _mode3d()
    a, k, th = 0.3, np.array([1.0, 2.0, -1.0]), 0.3
    s = k[0] * x + k[1] * y + k[2] * z + th
    phi = 0.5 + a * np.sin(s) * np.ones(p.shape)
    one, zero = np.ones(p.shape), np.zeros(p.shape)
    diff = model.R1(phi, one, p, 0.0) - model.R1(phi, zero, p, 0.0)
    kk = float(k @ k)
    gradn = a * math.sqrt(kk) * np.abs(np.cos(s))
    lap = -a * kk * np.sin(s)
    e = p.eps_phi
    want = (p.alpha / p.mu) * gradn * (e * lap - model.dW(phi) / e)
    assert np.max(np.abs(diff - want)) < 1e-11 * np.max(np.abs(want))


def test_R1_area_term_on_a_single_mode():
    """<phi, 1>_h of 0.5 + a sin(k.x) is 0.5 |Omega|, and the area term is
    -(M_area/mu) (<phi,1>_h - A0) |grad phi| with |grad phi| = a |k| |cos(k.x)|."""
    p, x, y, z = _mode3d()
    a, k = 0.25, np.array([2.0, 0.0, 1.0])
    s = k[0] * x + k[1] * y + k[2] * z + 0.7
    phi = 0.5 + a * np.sin(s) * np.ones(p.shape)
    u = wl.random_fields(p.shape, 3, 0.2, 0.8)
    vol = 0.5 * (2 * math.pi) ** 3
    assert math.isclose(model.volume(phi, p), vol, rel_tol=1e-13)
    r_a = model.R1(phi, u, p, vol)              # area term off
    r_b = model.R1(phi, u, p, vol - 2.0)        # <phi,1> - A0 = 2
    gradn = a * math.sqrt(float(k @ k)) * np.abs(np.cos(s))
    want = -(p.M_area / p.mu) * 2.0 * gradn
    assert np.max(np.abs((r_b - r_a) - want)) < 1e-11 * np.max(np.abs(want))


def test_R1_line_term_on_a_planar_membrane():
    """phi depends on x only and u on y only: g is constant along y, so the discrete surface
    Laplacian of u = 0.5 + b sin(y) is g lambda_y (u - 0.5), lambda_y = -(4/h^2) sin^2(h/2), and
    the line term (lambda_line/mu)(eps_u Delta_S u - g W'(u)/eps_u)|grad phi| has a closed form
    (W'(0.5) = 0 for the reference field u = 0.5)."""
    p, x, y, z = _mode3d()
    p = p.replace(alpha=0.0)
    a, b = 0.3, 0.1
    phi = 0.5 + a * np.sin(x) * np.ones(p.shape)
    u = 0.5 + b * np.sin(y) * np.ones(p.shape)
    assert np.all(bm.band_mask(phi, p.band_mask_hi))
    diff = model.R1(phi, u, p, 1.0) - model.R1(phi, np.full(p.shape, 0.5), p, 1.0)
    hy = p.h[1]
    lam_y = -(4.0 / hy ** 2) * math.sin(hy / 2) ** 2
    g = model.g_loc(phi)
    lap_s = g * lam_y * (u - 0.5)
    gradn = a * np.abs(np.cos(x)) * np.ones(p.shape)
    want = (p.lambda_line / p.mu) * (p.eps_u * lap_s - g * model.dW(u) / p.eps_u) * gradn
    assert np.max(np.abs(diff - want)) < 1e-11 * np.max(np.abs(want))


# ---------------------------------------------------------------- advection
def test_advection_of_a_translated_profile():
    """phi_old = phi + tau c.D0 phi (a profile moved by c over one step, to first order) with
    phi = 0.5 + a sin(k.x + t0): the central gradient is D0 phi = a cos(k.x + t0) kt, kt_d =
    sin(k_d h_d)/h_d, so v = -d_t phi grad phi/|grad phi|^2 = (c.kt) kt/|kt|^2 is constant and
    div(g u v) = v . D0(g u), closed form for g u = 0.2 + b cos(m.x)."""
    p, x, y, z = _mode3d()
    h = np.array(p.h)
    a, b, t0 = 0.3, 0.1, 0.3
    k, m, c = np.array([1.0, 2.0, 0.0]), np.array([0.0, 1.0, 3.0]), np.array([0.7, -0.4, 1.3])
    s = k[0] * x + k[1] * y + k[2] * z + t0
    phi = 0.5 + a * np.sin(s) * np.ones(p.shape)
    kt = np.sin(k * h) / h
    d0phi = [a * np.cos(s) * kt[d] * np.ones(p.shape) for d in range(3)]
    phi_old = phi + p.tau * sum(c[d] * d0phi[d] for d in range(3))
    sm = m[0] * x + m[1] * y + m[2] * z
    gu = 0.2 + b * np.cos(sm) * np.ones(p.shape)
    v = float(c @ kt) * kt / float(kt @ kt)
    mt = np.sin(m * h) / h
    want = sum(v[d] * (-b * mt[d] * np.sin(sm)) for d in range(3)) * np.ones(p.shape)
    got = model.advection_div(phi, phi_old, gu, p)
    assert np.max(np.abs(got - want)) < 1e-6 * np.max(np.abs(want))


# ---------------------------------------------------------------- coupled step, dense route
def _dense_phi_mats(Lmat, tau):
    n = Lmat.shape[0]
    A = -tau * Lmat
    I, Z = np.eye(n), np.zeros((n, n))
    P0 = expm(A)
    P1 = expm(np.block([[A, I], [Z, Z]]))[:n, n:]
    P2 = expm(np.block([[A, I, Z], [Z, Z, I], [Z, Z, Z]]))[:n, 2 * n:]
    return P0, P1, P2


@pytest.mark.parametrize("scheme", [1, 2])
def test_coupled_step_matches_dense_matrix_functions(scheme):
    n = 8
    p = wl.workload("c3", n=n)[0].replace(scheme=scheme, tau=2e-5, cg_rtol=1e-15)
    x, y, z = wl.grid(p.n, p.half_len, 3)
    phi0 = 0.5 + 0.35 * np.sin(x + 0.2) * np.cos(y - 0.1) * np.ones(p.shape) + 0.05 * np.cos(z)
    u0 = wl.random_fields(p.shape, 13, 0.35, 0.65)
    A0 = model.volume(phi0, p) - 0.2
    cs = etd.CoupledStepper(p, A0=A0)
    got_phi, got_u = cs.step(phi0.copy(), u0.copy())
    # dense linear operators from the DFT matrix
    N = n ** 3
    k1 = np.arange(n)
    F1 = np.exp(-2j * np.pi * np.outer(k1, k1) / n)
    F3 = np.kron(np.kron(F1, F1), F1)
    lam = spectral.laplacian_symbol(p).ravel()
    to_real = lambda sym: (np.linalg.inv(F3) @ np.diag(sym) @ F3).real
    Pp = _dense_phi_mats(to_real(spectral.l_phi(p, lam)), p.tau)
    Pu = _dense_phi_mats(to_real(spectral.l_u(p, lam)), p.tau)
    sh = p.shape
    R1 = lambda f, u: model.R1(f.reshape(sh), u.reshape(sh), p, A0).ravel()
    f0, U = phi0.ravel(), u0.ravel()
    ft = Pp[0] @ f0 + p.tau * (Pp[1] @ R1(f0, U))
    fn = ft if scheme == 1 else ft + p.tau * (Pp[2] @ (R1(ft, U) - R1(f0, U)))
    G = model.g_loc(fn)
    band = bm.band_mask(fn.reshape(sh), p.band_mask_hi)
    comp = bm.components(band)
    solver = model.BandSolver(p)
    R2 = lambda u: model.R2_coupled(fn.reshape(sh), phi0, u.reshape(sh), p, solver, comp).ravel()
    rec = lambda GU: model.recover(GU, G, p.recover_delta)
    r2n = R2(U)
    GUt = Pu[0] @ (G * U) + p.tau * (Pu[1] @ r2n)
    if scheme == 2:
        GUt = GUt + p.tau * (Pu[2] @ (R2(rec(GUt)) - r2n))
    un = rec(GUt)
    assert np.max(np.abs(got_phi.ravel() - fn)) < 1e-12 * np.max(np.abs(fn))
    assert np.max(np.abs(got_u.ravel() - un)) < 1e-12 * np.max(np.abs(un))
    assert np.max(np.abs(un - U)) > 1e-6               # the step moved u (not a trivial match)
