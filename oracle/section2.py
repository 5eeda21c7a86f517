"""The theorem-backed fixed-membrane scheme of Sec. 2 on small dense grids (FP64 oracle).

Sec. 2.2 divides the fixed-membrane OK equation by g^{1/2} and integrates
    d(sqrt(g) u)/dt + L_phi (sqrt(g) u) = R_phi(u),
    L_phi = B I - eps_u G^{-1/2} Delta_{S,h} G^{-1/2},
    R_phi(u) = B sqrt(g) u - sqrt(g) W'(u)/eps_u - gamma sqrt(g) (-Delta_{S,h})^{-1}(g f(u)) f'(u)
               - M <g (f(u) - ubar), 1>_h sqrt(g) f'(u),
with ETD1 (Eq. (2.8)) and ETDRK2 (Eq. (2.9)-(2.10)).  L_phi is a symmetric variable-
coefficient matrix (not FFT-diagonal), so this module forms it densely (Remark in Sec. 2.2
identifies operators with matrices) and evaluates phi_j(tau L) through its eigen-
decomposition.  (-Delta_{S,h})^{-1} on the full periodic grid is the inverse on the range
(mean-free functions) applied after mean removal (Sec. 2.1).  Only for grids up to ~32^2: it exists to check the maximum-bound
and energy-stability theorems, which hold exactly for this scheme.
"""
from __future__ import annotations

import numpy as np

from . import band as bandmod
from . import fd, model
from .spectral import phi_functions

L_W2 = 36.0      # max over [0,1] of |W''|
L_F2 = 6.0       # max over [0,1] of |f''|
L_F1 = 1.5       # max over [0,1] of |f'|
L_G = 1.125      # max over [0,1] of g


def inverse_on_range(A):
    """The inverse of the symmetric positive semi-definite A on the orthogonal complement of
    its null space, zero on the null space: sum over eigenpairs with mu_k > 0 of
    q_k q_k^T / mu_k (eigenvalues below 1e-10 max|mu| count as the null space).  For
    A = -Delta_{S,h} the null space is the constants of each connected component, and this is
    the inverse on mean-free functions of Sec. 2.1."""
    mu, Q = np.linalg.eigh(0.5 * (A + A.T))
    keep = mu > 1e-10 * np.max(np.abs(mu))
    return (Q[:, keep] / mu[keep]) @ Q[:, keep].T


class DenseScheme:
    def __init__(self, phi, h, eps_u, gamma, M, ubar, B):
        self.shape = phi.shape
        self.h = h
        self.eps_u, self.gamma, self.M, self.ubar, self.B = eps_u, gamma, M, ubar, B
        self.g = model.g_loc(phi).ravel()
        n = self.g.size
        eye = np.eye(n)
        g2 = self.g.reshape(self.shape)
        self.DS = np.stack([fd.surface_laplacian(eye[k].reshape(self.shape), g2, h).ravel()
                            for k in range(n)], axis=1)
        proj = eye - np.full((n, n), 1.0 / n)
        self.Kinv = inverse_on_range(-self.DS) @ proj         # (-Delta_S)^{-1}(f - mean)
        sg = np.sqrt(self.g)
        self.sg = sg
        self.L = B * eye - eps_u * (self.DS / sg[:, None]) / sg[None, :]
        self.L = 0.5 * (self.L + self.L.T)
        self.area = float(np.prod(h)) * n

    def C_inf(self):
        """||(-Delta_{S,h})^{-1}||_{L^inf,h}: max row sum of |entries|."""
        return float(np.max(np.sum(np.abs(self.Kinv), axis=1)))

    def phi_mats(self, tau):
        mu, Q = np.linalg.eigh(self.L)
        out = []
        for f in phi_functions(tau * mu):
            out.append((Q * f) @ Q.T)
        return out

    def R(self, U):
        g, sg = self.g, self.sg
        gf = g * model.f_ind(U)
        w = self.Kinv @ gf
        mass = float(np.prod(self.h)) * np.sum(g * (model.f_ind(U) - self.ubar))
        return (self.B * sg * U - sg * model.dW(U) / self.eps_u
                - self.gamma * sg * w * model.df_ind(U) - self.M * mass * sg * model.df_ind(U))

    def step(self, U, tau, scheme, mats=None):
        P0, P1, P2 = mats if mats is not None else self.phi_mats(tau)
        V = self.sg * U
        Rn = self.R(U)
        Vt = P0 @ V + tau * (P1 @ Rn)
        if scheme == 1:
            return Vt / self.sg
        Ut = Vt / self.sg
        return (Vt + tau * (P2 @ (self.R(Ut) - Rn))) / self.sg

    def energy(self, U):
        """Eq. (2.16) with the full-grid inverse."""
        g = self.g
        dx = float(np.prod(self.h))
        gf = g * model.f_ind(U)
        e = (0.5 * self.eps_u * dx * float(U @ (-self.DS @ U))
             + dx * float(np.sum(g * model.W(U))) / self.eps_u
             + 0.5 * self.gamma * dx * float((self.Kinv @ gf) @ gf)
             + 0.5 * self.M * (dx * float(np.sum(g * (model.f_ind(U) - self.ubar)))) ** 2)
        return e


def B_mbp(eps_u, gamma, M, C, area):
    """Stabiliser of the maximum-bound condition, Eq. (2.15) (taken with equality)."""
    return L_W2 / eps_u + gamma * C * L_F2 * L_G + M * area * L_F2 * L_G


def B_energy(eps_u, gamma, M, C, area):
    """Stabiliser of the energy-stability theorem, Eq. (2.17)."""
    return L_W2 / eps_u + (0.5 * gamma * C + 0.5 * M * area) * (L_F2 + L_F1 ** 2) * L_G


class BandScheme:
    """The Sec. 2.2 scheme on the narrow band of a frozen membrane (FP64 oracle, dense).

    Sec. 2 assumes 0 < phi < 1 on the whole grid so that g > 0 everywhere.  For a membrane
    profile g underflows to 0 (or is ~1e-20) away from the interface, where g^{-1/2} is
    undefined, so the scheme is taken on the band {|2 phi - 1| < band_hi} of Sec. 3.2 with the
    readings of the band solve:

    * Delta_{S,h} restricted to the band with zero flux across the band edge (a face with an
      off-band end carries coefficient 0), so L = B I + eps_u S A S with A = -Delta_band,
      S = diag(g^{-1/2}) on band nodes: symmetric, with non-positive off-diagonal entries
      (the Metzler property of the exponential, Sec. 2.2) and L g^{1/2} = B g^{1/2};
    * (-Delta_{S,h})^{-1}(g f(u)) is the band solve with the mean removed on every
      connected band component (Sec. 2.1's mean removal, per component);
    * the mass <g (f(u) - ubar), 1>_h is the full-grid inner product (off-band terms are
      constant in time);
    * U off the band is not part of the system and keeps its value.

    With band_hi = 1 and 0 < phi < 1 everywhere the band is the whole grid and the scheme is
    DenseScheme's.  phi_j(tau L) by the eigen-decomposition of the band matrix (dense; band
    sizes up to a few thousand nodes).
    """

    def __init__(self, phi, h, eps_u, gamma, M, ubar, B, band_hi=0.99, cg_rtol=1e-14, linear_only=False):
        self.shape = phi.shape
        self.h = tuple(h)
        self.eps_u, self.gamma, self.M, self.ubar, self.B = eps_u, gamma, M, ubar, B
        self.linear_only = linear_only
        self.cg_rtol = cg_rtol
        self.g = model.g_loc(phi)
        self.band = bandmod.band_mask(phi, band_hi)
        self.comp = bandmod.components(self.band)
        self.idx = np.flatnonzero(self.band.ravel())
        self.A = self.band_neg_lap()
        gb = self.g.ravel()[self.idx]
        self.sg = np.sqrt(gb)
        isg = 1.0 / self.sg
        self.L = B * np.eye(self.idx.size) + eps_u * (isg[:, None] * self.A) * isg[None, :]
        self.L = 0.5 * (self.L + self.L.T)

    def band_neg_lap(self):
        """Dense -Delta_{S,h} on the band nodes (zero-flux band edge): the matrix whose action is
        band.apply_neg_lap restricted to band values, assembled face by face: a face between
        nodes p and q = p + e_d with coefficient c = g_{p+1/2 e_d} (both ends in the band)
        adds c/h_d^2 to (p,p) and (q,q) and -c/h_d^2 to (p,q) and (q,p)."""
        coeffs = bandmod.face_coeffs(self.g, self.band)
        pos = -np.ones(int(np.prod(self.shape)), dtype=np.int64)
        pos[self.idx] = np.arange(self.idx.size)
        pos = pos.reshape(self.shape)
        A = np.zeros((self.idx.size, self.idx.size))
        for d, c in enumerate(coeffs):
            q = fd.shift(pos, d, 1)                 # index of the node at p + e_d
            sel = (c != 0.0) & (pos >= 0) & (q >= 0)
            a, b, v = pos[sel], q[sel], c[sel] / self.h[d] ** 2
            np.add.at(A, (a, a), v)
            np.add.at(A, (b, b), v)
            np.add.at(A, (a, b), -v)
            np.add.at(A, (b, a), -v)
        return A

    def phi_mats(self, tau):
        mu, Q = np.linalg.eigh(self.L)
        return [(Q * f) @ Q.T for f in phi_functions(tau * mu)]

    def R(self, U):
        """R_phi(U) at the band nodes (U a full-grid field)."""
        if self.linear_only:
            return np.zeros(self.idx.size)
        g = self.g
        w, _, _ = bandmod.solve_neg_lap(g * model.f_ind(U), g, self.band, self.h, rtol=self.cg_rtol,
                                        comp=self.comp)
        mass = fd.inner(g, model.f_ind(U) - self.ubar, self.h)
        u = U.ravel()[self.idx]
        fp = model.df_ind(u)
        return self.sg * (self.B * u - model.dW(u) / self.eps_u - self.gamma * w.ravel()[self.idx] * fp
                          - self.M * mass * fp)

    def _with_band(self, U, Vb):
        out = U.copy()
        out.ravel()[self.idx] = Vb / self.sg
        return out

    def step(self, U, tau, scheme, mats=None):
        """ETD1 (Eq. (2.8)) or ETDRK2 (Eq. (2.9)-(2.10)) in the variable V = g^{1/2} U."""
        P0, P1, P2 = mats if mats is not None else self.phi_mats(tau)
        V = self.sg * U.ravel()[self.idx]
        Rn = self.R(U)
        Vt = P0 @ V + tau * (P1 @ Rn)
        if scheme == 1:
            return self._with_band(U, Vt)
        Ut = self._with_band(U, Vt)
        return self._with_band(U, Vt + tau * (P2 @ (self.R(Ut) - Rn)))

    def run(self, U, tau, scheme, nsteps):
        mats = self.phi_mats(tau)
        for _ in range(nsteps):
            U = self.step(U, tau, scheme, mats)
        return U

    def C_inf(self):
        """||(-Delta_band)^{-1}||_{L^inf,h} with per-component mean removal: max row sum of |K|,
        K = A^+ P, A^+ the inverse on the range, P the per-component mean projector."""
        comp, ncomp = self.comp
        c = comp.ravel()[self.idx]
        P = np.eye(self.idx.size)
        for k in range(ncomp):
            sel = np.flatnonzero(c == k)
            P[np.ix_(sel, sel)] -= 1.0 / sel.size
        K = inverse_on_range(self.A) @ P
        return float(np.max(np.sum(np.abs(K), axis=1)))

    def energy(self, U):
        """Eq. (2.16) for the band system: the gradient and well terms over band nodes and band
        faces, the nonlocal term with the band solve, the (full-grid) mass term."""
        g = self.g
        dx = float(np.prod(self.h))
        u = U.ravel()[self.idx]
        gb = g.ravel()[self.idx]
        gf = g * model.f_ind(U)
        w, _, _ = bandmod.solve_neg_lap(gf, g, self.band, self.h, rtol=self.cg_rtol, comp=self.comp)
        mass = fd.inner(g, model.f_ind(U) - self.ubar, self.h)
        return (0.5 * self.eps_u * dx * float(u @ (self.A @ u)) + dx * float(np.sum(gb * model.W(u))) / self.eps_u
                + 0.5 * self.gamma * dx * float(np.sum(w * gf)) + 0.5 * self.M * mass * mass)
