"""Nonlinear terms, recovery, energy and mass of the membrane model (FP64 oracle).

Formulas follow the paper term by term:

* W(s) = 18 (s^2 - s)^2 (Sec. 1), W'(s) = 36 s (s - 1)(2 s - 1), W''(s) = 36 (6 s^2 - 6 s + 1).
* g(Phi) = 18 (Phi^2 - Phi)^2, the localisation used by Algorithm 1 and Sec. 3.3 (Sec. 1
  writes eps_phi^{-1} W(phi); the algorithm, which is what is run, drops the 1/eps).
* f(u) = 3 u^2 - 2 u^3, f'(u) = 6 u (1 - u)  (Sec. 1).
* R1(phi, u): the nonlinear remainder of the stabilised force balance (Sec. 3.1, the split
  of Eq. (1.1) with stabilisers A1, A2 into -L_phi phi + R1), evaluated by spectral
  collocation (Sec. 3.2) except the surface Laplacian of u, which is the finite-difference
  Delta_{S,h} of Eq. (2.3) and, like the whole line-tension term, lives on the band only.
* R2(phi, u): the nonlinear remainder of the stabilised OK equation (Sec. 3.1, the split of
  Eq. (1.2) into -L_u(gu) + R2), by second-order finite differences on the band (Sec. 3.2),
  zero off the band.  The nonlocal term gamma g Delta_S^{-1}(g (u - ubar)) is
  -gamma g w with w = (-Delta_{S,h})^{-1}(g (u - ubar)) solved on the band.
  The advection velocity v = -d_t phi grad(phi)/|grad(phi)|^2 (Sec. 1) uses
  d_t phi = (phi^{n+1} - phi^n)/tau, central differences and |grad phi|^2 + 1e-12.
* R2 of the fixed-membrane model: the Sec. 3 split applied to Eq. (2.1) with the discrete
  operands of Eq. (2.16): the nonlocal operand is g f(u), the mass operand g (f(u) - ubar).
* Discrete energy, Eq. (2.16).
"""
from __future__ import annotations

import numpy as np

from . import band as bandmod
from . import fd
from .fft import fftn, ifftn_real
from .spectral import derivative_symbols, laplacian_symbol


def W(s):
    return 18.0 * (s * s - s) ** 2


def dW(s):
    return 36.0 * s * (s - 1.0) * (2.0 * s - 1.0)


def d2W(s):
    return 36.0 * (6.0 * s * s - 6.0 * s + 1.0)


def g_loc(phi):
    return 18.0 * (phi * phi - phi) ** 2


def f_ind(u):
    return 3.0 * u * u - 2.0 * u ** 3


def df_ind(u):
    return 6.0 * u * (1.0 - u)


def recover(GU, G, delta):
    """U = GU/G where G > delta, U = GU elsewhere (Sec. 3.3, after Algorithm 1)."""
    safe = np.where(G > delta, G, 1.0)
    return np.where(G > delta, GU / safe, GU)


def spectral_lap(v, p):
    return ifftn_real(laplacian_symbol(p) * fftn(v))


def spectral_grad(v, p):
    V = fftn(v)
    return [ifftn_real(s * V) for s in derivative_symbols(p)]


def volume(phi, p):
    return float(np.prod(p.h[: p.dim]) * np.sum(phi))


def R1(phi, u, p, A0):
    """Nonlinear remainder of the force balance (Sec. 3.1)."""
    e = p.eps_phi
    h = p.h[: p.dim]
    lap = spectral_lap(phi, p)
    grads = spectral_grad(phi, p)
    gradn = np.sqrt(sum(gr * gr for gr in grads))
    Wp, Wpp = dW(phi), d2W(phi)
    Wm = Wp - p.A1 * phi
    g = g_loc(phi)
    band = bandmod.band_mask(phi, p.band_mask_hi)
    bend = (p.kappa / (p.mu * e * e) * (spectral_lap(Wm, p) + (Wpp - p.A2) * (lap - p.A1 * phi / (e * e)))
            - (p.kappa * Wpp / (p.mu * e ** 4) + p.lambda_surf / (p.mu * e * e)) * Wm)
    line = (p.lambda_line / p.mu) * (p.eps_u * fd.surface_laplacian(u, g, h) - g * dW(u) / p.eps_u) * gradn
    line = np.where(band, line, 0.0)
    area = -(p.M_area / p.mu) * (volume(phi, p) - A0) * gradn
    bio = (p.alpha / p.mu) * (u + p.u0) * gradn * (e * lap - Wp / e)
    return bend + line + area + bio


def force_rhs(phi, u, p, A0):
    """Right-hand side of Eq. (1.1) divided by mu, with the band-restricted line term.

    Used only to pin R1: R1 - L_phi phi must equal this.
    """
    e = p.eps_phi
    h = p.h[: p.dim]
    lap = spectral_lap(phi, p)
    grads = spectral_grad(phi, p)
    gradn = np.sqrt(sum(gr * gr for gr in grads))
    chem = lap - dW(phi) / (e * e)                      # Delta phi - W'(phi)/eps^2
    bending = spectral_lap(chem, p) - d2W(phi) / (e * e) * chem   # (Delta - W''/eps^2) chem
    g = g_loc(phi)
    band = bandmod.band_mask(phi, p.band_mask_hi)
    line = p.lambda_line * (p.eps_u * fd.surface_laplacian(u, g, h) - g * dW(u) / p.eps_u) * gradn
    line = np.where(band, line, 0.0)
    rhs = (p.lambda_surf * chem - p.kappa * bending + line
           - p.M_area * (volume(phi, p) - A0) * gradn
           + p.alpha * (u + p.u0) * (e * lap - dW(phi) / e) * gradn)
    return rhs / p.mu


class BandSolver:
    """Band (-Delta_{S,h})^{-1} with a warm start kept between calls."""

    def __init__(self, p):
        self.p = p
        self.w_prev = None
        self.last_iters = 0
        self.last_resid = 0.0

    def __call__(self, f, g, band, comp=None):
        h = self.p.h[: self.p.dim]
        x0 = self.w_prev if (self.w_prev is not None and self.w_prev.shape == f.shape) else None
        w, it, rel = bandmod.solve_neg_lap(f, g, band, h, self.p.cg_rtol, self.p.cg_maxit,
                                           x0=x0, comp=comp)
        self.w_prev = w
        self.last_iters, self.last_resid = it, rel
        return w


def advection_div(phi_new, phi_old, gu, p):
    """Central-difference divergence of g u v, v = -d_t phi grad phi / |grad phi|^2."""
    h = p.h[: p.dim]
    dtphi = (phi_new - phi_old) / p.tau
    gr = fd.central_grad(phi_new, h)
    n2 = sum(x * x for x in gr) + 1e-12
    F = [gu * (-dtphi * x / n2) for x in gr]
    return fd.central_div(F, h)


def R2_coupled(phi_new, phi_old, u, p, solver, comp=None):
    """Nonlinear remainder of the stabilised OK equation (Sec. 3.1), zero off the band."""
    h = p.h[: p.dim]
    g = g_loc(phi_new)
    band = bandmod.band_mask(phi_new, p.band_mask_hi)
    gu = g * u
    m = fd.inner(g, u - p.ubar, h)
    w = solver(g * (u - p.ubar), g, band, comp)
    r = (p.eps_u * (fd.surface_laplacian(u, g, h) - p.B1 * fd.laplacian(gu, h))
         + p.B2 * gu - g * dW(u) / p.eps_u - p.gamma * g * w - p.M * g * m
         - advection_div(phi_new, phi_old, gu, p))
    return np.where(band, r, 0.0)


def R2_fixed(u, g, band, p, solver, comp=None):
    """Fixed-membrane remainder: the Sec. 3 split of Eq. (2.1), operands as in Eq. (2.16)."""
    h = p.h[: p.dim]
    gu = g * u
    mf = fd.inner(g, f_ind(u) - p.ubar, h)
    w = solver(g * f_ind(u), g, band, comp)
    r = (p.eps_u * (fd.surface_laplacian(u, g, h) - p.B1 * fd.laplacian(gu, h))
         + p.B2 * gu - g * dW(u) / p.eps_u
         - p.gamma * g * df_ind(u) * w - p.M * g * df_ind(u) * mf)
    return np.where(band, r, 0.0)


def energy(U, g, band, p, comp=None, rtol=None):
    """Discrete energy of Eq. (2.16); the nonlocal inverse is the band solve.

    Returns a dict with the four terms, their sum and the mass <g (f(U) - ubar), 1>_h.
    """
    h = p.h[: p.dim]
    gf = g * f_ind(U)
    w, _, _ = bandmod.solve_neg_lap(gf, g, band, h, rtol or p.cg_rtol, p.cg_maxit, comp=comp)
    e_grad = 0.5 * p.eps_u * fd.grad_energy(U, g, h)
    e_well = fd.inner(g, W(U), h) / p.eps_u
    e_nonloc = 0.5 * p.gamma * fd.inner(w, gf, h)
    mass = fd.inner(g, f_ind(U) - p.ubar, h)
    e_mass = 0.5 * p.M * mass * mass
    return dict(grad=e_grad, well=e_well, nonlocal_=e_nonloc, mass_term=e_mass,
                total=e_grad + e_well + e_nonloc + e_mass, mass=mass)


def bound_stats(U, G, delta):
    """max |2U - 1|, min U and max U over the recovery set {G > delta}."""
    sel = G > delta
    if not np.any(sel):
        return 0.0, 0.0, 0.0
    Us = U[sel]
    return float(np.max(np.abs(2.0 * Us - 1.0))), float(Us.min()), float(Us.max())


def mass_coupled(U, G, p):
    return fd.inner(G, U - p.ubar, p.h[: p.dim])

