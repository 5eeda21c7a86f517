"""ETD1 / ETDRK2 drivers of the spectral scheme (FP64 oracle), Sec. 3.3 and Algorithm 1.

Per step, in the paper's order and notation (full complex spectra, the oracle's own FFT):

  phi-stage   R1^n   = FFT(R1(phi^n, u^n))
              phi~^  = phi0(tau l^phi) phi^n^ + tau phi1(tau l^phi) R1^n
              [RK2]  phi^{n+1}^ = phi~^ + tau phi2(tau l^phi) (FFT(R1(iFFT(phi~^), u^n)) - R1^n)
              phi^{n+1} = iFFT(phi^{n+1}^),  G = g(phi^{n+1})
  u-stage     GU^    = FFT(G u^n)               (new g times old u, Sec. 3.3)
              R2^n   = FFT(R2(phi^{n+1}, u^n))
              GU~^   = phi0(tau l^u) GU^ + tau phi1(tau l^u) R2^n
              [RK2]  U~ = recover(iFFT(GU~^), G)
                     GU^{n+1}^ = GU~^ + tau phi2(tau l^u) (FFT(R2(phi^{n+1}, U~)) - R2^n)
              u^{n+1} = recover(iFFT(GU^{n+1}^), G)

The fixed-membrane model freezes phi (the phi-stage is skipped, v = 0) and runs the same
u-stage with its own R2 (the Sec. 3 split of Eq. (2.1)).
"""
from __future__ import annotations

import numpy as np

from . import band as bandmod
from . import model
from .fft import fftn, ifftn_real
from .spectral import l_phi, l_u, laplacian_symbol, phi_functions


class Coefficients:
    """phi0, tau*phi1, tau*phi2 on the full spectrum for both linear symbols."""

    def __init__(self, p):
        lam = laplacian_symbol(p)
        a0, a1, a2 = phi_functions(p.tau * l_phi(p, lam))
        b0, b1, b2 = phi_functions(p.tau * l_u(p, lam))
        self.phi = (a0, p.tau * a1, p.tau * a2)
        self.u = (b0, p.tau * b1, p.tau * b2)


class FixedStepper:
    """Fixed membrane: G = g(Phi) and the band are set once from the frozen Phi."""

    def __init__(self, p, phi):
        self.p = p
        self.c = Coefficients(p)
        self.G = model.g_loc(phi)
        self.band = bandmod.band_mask(phi, p.band_mask_hi)
        self.comp = bandmod.components(self.band)
        self.solver = model.BandSolver(p)

    def R2(self, u):
        if self.p.linear_only:
            return np.zeros_like(u)
        return model.R2_fixed(u, self.G, self.band, self.p, self.solver, self.comp)

    def step(self, u):
        p, G = self.p, self.G
        b0, b1, b2 = self.c.u
        GU = fftn(G * u)
        Rn = fftn(self.R2(u))
        GUt = b0 * GU + b1 * Rn
        if p.scheme == 1:
            return model.recover(ifftn_real(GUt), G, p.recover_delta)
        Ut = model.recover(ifftn_real(GUt), G, p.recover_delta)
        GUn = GUt + b2 * (fftn(self.R2(Ut)) - Rn)
        return model.recover(ifftn_real(GUn), G, p.recover_delta)

    def run(self, u, nsteps, callback=None):
        for n in range(nsteps):
            u = self.step(u)
            if callback is not None:
                callback(n + 1, u)
        return u

    def energy(self, u):
        return model.energy(u, self.G, self.band, self.p, self.comp)


class CoupledStepper:
    """Coupled phi-u system, Algorithm 1."""

    def __init__(self, p, A0=None):
        self.p = p
        self.c = Coefficients(p)
        self.A0 = A0
        self.solver = model.BandSolver(p)

    def R1(self, phi, u):
        if self.p.linear_only:
            return np.zeros_like(phi)
        return model.R1(phi, u, self.p, self.A0)

    def R2(self, phi_new, phi_old, u, comp):
        if self.p.linear_only:
            return np.zeros_like(u)
        return model.R2_coupled(phi_new, phi_old, u, self.p, self.solver, comp)

    def step(self, phi, u):
        p = self.p
        if self.A0 is None or np.isnan(self.A0):
            self.A0 = model.volume(phi, p)
        a0, a1, a2 = self.c.phi
        b0, b1, b2 = self.c.u
        # phi-stage
        P = fftn(phi)
        R1n = fftn(self.R1(phi, u))
        Pt = a0 * P + a1 * R1n
        if p.scheme == 2:
            Pt = Pt + a2 * (fftn(self.R1(ifftn_real(Pt), u)) - R1n)
        phi_new = ifftn_real(Pt)
        G = model.g_loc(phi_new)
        # u-stage
        band = bandmod.band_mask(phi_new, p.band_mask_hi)
        comp = bandmod.components(band)
        GU = fftn(G * u)
        R2n = fftn(self.R2(phi_new, phi, u, comp))
        GUt = b0 * GU + b1 * R2n
        if p.scheme == 2:
            Ut = model.recover(ifftn_real(GUt), G, p.recover_delta)
            GUt = GUt + b2 * (fftn(self.R2(phi_new, phi, Ut, comp)) - R2n)
        u_new = model.recover(ifftn_real(GUt), G, p.recover_delta)
        return phi_new, u_new

    def run(self, phi, u, nsteps, callback=None):
        for n in range(nsteps):
            phi, u = self.step(phi, u)
            if callback is not None:
                callback(n + 1, phi, u)
        return phi, u

    def energy(self, phi, u):
        G = model.g_loc(phi)
        band = bandmod.band_mask(phi, self.p.band_mask_hi)
        return model.energy(u, G, band, self.p)
