"""The theorem-backed fixed-membrane scheme of Sec. 2 on small dense grids (FP64 oracle).

Sec. 2.2 divides the fixed-membrane OK equation by g^{1/2} and integrates
    d(sqrt(g) u)/dt + L_phi (sqrt(g) u) = R_phi(u),
    L_phi = B I - eps_u G^{-1/2} Delta_{S,h} G^{-1/2},
    R_phi(u) = B sqrt(g) u - sqrt(g) W'(u)/eps_u - gamma sqrt(g) (-Delta_{S,h})^{-1}(g f(u)) f'(u)
               - M <g (f(u) - ubar), 1>_h sqrt(g) f'(u),
with ETD1 (Eq. (2.8)) and ETDRK2 (Eq. (2.9)-(2.10)).  L_phi is a symmetric variable-
coefficient matrix (not FFT-diagonal), so this module forms it densely (Remark in Sec. 2.2
identifies operators with matrices) and evaluates phi_j(tau L) through its eigen-
decomposition.  (-Delta_{S,h})^{-1} on the full periodic grid is the pseudo-inverse after
mean removal (Sec. 2.1).  Only for grids up to ~32^2: it exists to check the maximum-bound
and energy-stability theorems, which hold exactly for this scheme.
"""
from __future__ import annotations

import numpy as np

from . import fd, model
from .spectral import phi_functions

L_W2 = 36.0      # max over [0,1] of |W''|
L_F2 = 6.0       # max over [0,1] of |f''|
L_F1 = 1.5       # max over [0,1] of |f'|
L_G = 1.125      # max over [0,1] of g


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
        self.Kinv = np.linalg.pinv(-self.DS) @ proj            # (-Delta_S)^{-1}(f - mean)
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
