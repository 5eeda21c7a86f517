"""Narrow band and the band-restricted inverse surface Laplacian (FP64 oracle).

Sec. 3.2 evaluates the nonlocal surface term only on a narrow band around the membrane and
leaves the band threshold, the band-edge treatment and the solver open.  Readings taken
here:

* band            = {|2 Phi - 1| < hi}, hi = 0.99 (equivalently g(Phi) > 4.46e-4);
* band edge       : a face with an off-band end carries coefficient 0 (zero flux);
* null space      : the band operator is singular on every connected band component, so
                    right-hand side and solution are projected to zero mean per component
                    (the whole-domain mean removal of Sec. 2.1, applied per component);
* solver          : Jacobi-preconditioned conjugate gradients to a relative residual rtol.

Connected components use 6-neighbour (4 in 2D) connectivity with periodic wrap.
"""
from __future__ import annotations

import numpy as np
from scipy import ndimage

from . import fd


def band_mask(phi, hi=0.99):
    return np.abs(2.0 * phi - 1.0) < hi


def components(band):
    """Integer labels 0..C-1 on band points (-1 elsewhere), periodic 6-connectivity."""
    struct = ndimage.generate_binary_structure(band.ndim, 1)
    lab, nlab = ndimage.label(band, structure=struct)
    parent = list(range(nlab + 1))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for ax in range(band.ndim):
        lo = np.take(lab, 0, axis=ax)
        hi = np.take(lab, -1, axis=ax)
        both = (lo > 0) & (hi > 0)
        for a, b in zip(lo[both].ravel(), hi[both].ravel()):
            ra, rb = find(int(a)), find(int(b))
            if ra != rb:
                parent[max(ra, rb)] = min(ra, rb)
    roots = np.array([find(i) for i in range(nlab + 1)])
    uniq = {r: i for i, r in enumerate(sorted(set(roots[1:].tolist())))}
    remap = np.array([-1] + [uniq[r] for r in roots[1:]], dtype=np.int64)
    return remap[lab], len(uniq)


def project_mean(v, comp, ncomp):
    """Subtract the per-component mean on the band; zero off the band."""
    out = np.where(comp >= 0, v, 0.0)
    for c in range(ncomp):
        sel = comp == c
        out[sel] -= out[sel].mean()
    return out


def face_coeffs(g, band):
    return [fd.face_avg(g, d) * band * fd.shift(band, d, 1) for d in range(g.ndim)]


def apply_neg_lap(w, coeffs, h):
    """(-Delta_{S,h} restricted to the band, zero-flux band edges) applied to w."""
    out = np.zeros_like(w)
    for d, c in enumerate(coeffs):
        flux = c * (fd.shift(w, d, 1) - w) / h[d]
        out -= (flux - fd.shift(flux, d, -1)) / h[d]
    return out


def jacobi_diag(coeffs, h):
    return sum((c + fd.shift(c, d, -1)) / h[d] ** 2 for d, c in enumerate(coeffs))


def solve_neg_lap(f, g, band, h, rtol=1e-13, maxit=20000, x0=None, comp=None):
    """w = (-Delta_{S,h})^{-1} (f - mean) on the band.  Returns (w, iters, rel_resid)."""
    if comp is None:
        comp, ncomp = components(band)
    else:
        comp, ncomp = comp
    coeffs = face_coeffs(g, band)
    diag = jacobi_diag(coeffs, h)
    diag = np.where(diag > 0, diag, 1.0)
    b = project_mean(f, comp, ncomp)
    bnorm = float(np.sqrt(np.sum(b * b)))
    x = np.zeros_like(b) if x0 is None else project_mean(x0, comp, ncomp)
    if bnorm == 0.0:
        return np.zeros_like(b), 0, 0.0
    r = b - apply_neg_lap(x, coeffs, h)
    z = np.where(comp >= 0, r / diag, 0.0)
    pvec = z.copy()
    rz = float(np.sum(r * z))
    it = 0
    rel = float(np.sqrt(np.sum(r * r))) / bnorm
    while rel > rtol and it < maxit:
        q = apply_neg_lap(pvec, coeffs, h)
        pq = float(np.sum(pvec * q))
        if pq <= 0.0:
            break
        a = rz / pq
        x += a * pvec
        r -= a * q
        z = np.where(comp >= 0, r / diag, 0.0)
        rz_new = float(np.sum(r * z))
        pvec = z + (rz_new / rz) * pvec
        rz = rz_new
        it += 1
        rel = float(np.sqrt(np.sum(r * r))) / bnorm
    return project_mean(x, comp, ncomp), it, rel
