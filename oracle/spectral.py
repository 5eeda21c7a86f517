"""Spectral symbols and the phi-functions of the ETD schemes (FP64 oracle).

* Folded wavenumbers lambda_x(i) = (pi/X) i for 0 <= i <= N/2 and (pi/X)(N - i) above,
  the Laplacian symbol lambda_ijk = -(lambda_x^2 + lambda_y^2 + lambda_z^2)  (Sec. 3.2).
* Linear symbols (Sec. 3.2, from Eq. (3.1) and Eq. (3.2)):
      l^phi = kappa/mu lambda^2 - (kappa (A1 + A2) + lambda_surf eps^2)/(mu eps^2) lambda
              + (kappa A1 A2 + lambda_surf A1 eps^2)/(mu eps^4)
      l^u   = B2 - eps_u B1 lambda
* First derivative symbol i k with the signed wavenumber k = (pi/X) i for i < N/2,
  (pi/X)(i - N) for i > N/2 and 0 at the Nyquist index i = N/2 (the paper gives only the
  second-order symbol; a real field's odd derivative has no Nyquist component).
* phi_0(z) = exp(-z), phi_1(z) = (1 - exp(-z))/z, phi_2(z) = (exp(-z) - 1 + z)/z^2
  (Sec. 2.2, after Eq. (2.10)).  Below |z| = 1 the closed forms cancel, so the oracle
  sums the Taylor series phi_j(z) = sum_k (-z)^k / (k + j)! there.
"""
from __future__ import annotations

import math

import numpy as np


def folded_wavenumbers(n: int, half_len: float) -> np.ndarray:
    i = np.arange(n)
    return (math.pi / half_len) * np.where(i <= n // 2, i, n - i).astype(np.float64)


def signed_wavenumbers(n: int, half_len: float) -> np.ndarray:
    i = np.arange(n)
    k = np.where(i < n // 2, i, i - n).astype(np.float64)
    k[n // 2] = 0.0
    return (math.pi / half_len) * k


def _axes(p):
    """Per-axis (n, half_len) in array-axis order (z, y, x) or (y, x)."""
    nx, ny, nz = p.n
    X, Y, Z = p.half_len
    if p.dim == 2:
        return [(ny, Y), (nx, X)]
    return [(nz, Z), (ny, Y), (nx, X)]


def laplacian_symbol(p) -> np.ndarray:
    """lambda on the full spectrum (shape = field shape), lambda <= 0."""
    axes = _axes(p)
    lam = np.zeros([n for n, _ in axes])
    for ax, (n, L) in enumerate(axes):
        k = folded_wavenumbers(n, L)
        shape = [1] * len(axes)
        shape[ax] = n
        lam = lam - (k ** 2).reshape(shape)
    return lam


def derivative_symbols(p):
    """[i k_x, i k_y, (i k_z)] on the full spectrum, Nyquist set to zero."""
    axes = _axes(p)
    out = []
    for ax, (n, L) in enumerate(axes):
        k = signed_wavenumbers(n, L)
        shape = [1] * len(axes)
        shape[ax] = n
        out.append(np.broadcast_to(1j * k.reshape(shape), [m for m, _ in axes]))
    # return in (x, y, z) order
    return out[::-1]


def l_phi(p, lam):
    e2 = p.eps_phi ** 2
    return (p.kappa / p.mu * lam ** 2
            - (p.kappa * (p.A1 + p.A2) + p.lambda_surf * e2) / (p.mu * e2) * lam
            + (p.kappa * p.A1 * p.A2 + p.lambda_surf * p.A1 * e2) / (p.mu * e2 * e2))


def l_u(p, lam):
    return p.B2 - p.eps_u * p.B1 * lam


_TAYLOR_TERMS = 40


def phi_functions(z):
    """(phi0, phi1, phi2) evaluated elementwise at real z >= 0 (FP64)."""
    z = np.asarray(z, dtype=np.float64)
    phi0 = np.exp(-z)
    small = np.abs(z) < 1.0
    zs = np.where(small, z, 0.0)
    zl = np.where(small, 1.0, z)
    # Taylor branch: sum_k (-z)^k/(k+1)! and sum_k (-z)^k/(k+2)!, summed smallest term first
    s1 = np.zeros_like(zs)
    s2 = np.zeros_like(zs)
    for k in range(_TAYLOR_TERMS - 1, -1, -1):
        s1 = s1 + (-zs) ** k / math.factorial(k + 1)
        s2 = s2 + (-zs) ** k / math.factorial(k + 2)
    em1 = np.expm1(-zl)
    p1 = -em1 / zl
    p2 = (em1 + zl) / (zl * zl)
    return phi0, np.where(small, s1, p1), np.where(small, s2, p2)
