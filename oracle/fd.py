"""Second-order finite differences on the periodic grid (FP64 oracle), Sec. 2.1.

Arrays are (Nz, Ny, Nx) or (Ny, Nx), x fastest; `h` is (hx, hy[, hz]).  Array axis of a
direction d (0 = x, 1 = y, 2 = z) is ndim - 1 - d.

    D+_d u = (u_{i+1} - u_i)/h_d,  D-_d u = (u_i - u_{i-1})/h_d,
    g_{i+1/2} = (g_{i+1} + g_i)/2,
    Delta_{S,h} u = sum_d D-_d( g_{i+1/2} D+_d u )          (Eq. (2.3))
    Delta_h v     = sum_d (v_{i+1} - 2 v_i + v_{i-1})/h_d^2  (the constant-coefficient case)
    <f, g>_h      = h_x h_y (h_z) sum f g                    (Sec. 2.1)

Central differences (used for the membrane velocity of the advection term) are
(v_{i+1} - v_{i-1})/(2 h_d).
"""
from __future__ import annotations

import numpy as np


def _ax(u, d):
    return u.ndim - 1 - d


def shift(u, d, s):
    """u_{i+s} along direction d (periodic)."""
    return np.roll(u, -s, axis=_ax(u, d))


def dplus(u, d, h):
    return (shift(u, d, 1) - u) / h[d]


def dminus(u, d, h):
    return (u - shift(u, d, -1)) / h[d]


def face_avg(g, d):
    return 0.5 * (shift(g, d, 1) + g)


def surface_laplacian(u, g, h):
    """Delta_{S,h} u with face-averaged coefficient g (Eq. (2.3))."""
    out = np.zeros_like(u)
    for d in range(u.ndim):
        out += dminus(face_avg(g, d) * dplus(u, d, h), d, h)
    return out


def laplacian(v, h):
    out = np.zeros_like(v)
    for d in range(v.ndim):
        out += (shift(v, d, 1) - 2.0 * v + shift(v, d, -1)) / h[d] ** 2
    return out


def central_grad(v, h):
    return [(shift(v, d, 1) - shift(v, d, -1)) / (2.0 * h[d]) for d in range(v.ndim)]


def central_div(F, h):
    return sum((shift(F[d], d, 1) - shift(F[d], d, -1)) / (2.0 * h[d])
               for d in range(len(F)))


def inner(a, b, h):
    return float(np.prod(h) * np.sum(a * b))


def grad_energy(u, g, h):
    """<-Delta_{S,h} u, u>_h = sum over faces of g_{i+1/2} (D+ u)^2 times the cell volume."""
    return float(np.prod(h) * sum(np.sum(face_avg(g, d) * dplus(u, d, h) ** 2)
                                  for d in range(u.ndim)))
