"""Pins of the finite-difference operators and the band-restricted inverse."""
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import band as bm
from oracle import fd, model
from paper_2606_04347_gb300 import workloads as wl


def test_surface_laplacian_constant_g_is_discrete_laplacian():
    h = (0.1, 0.2, 0.3)
    u = np.random.default_rng(0).standard_normal((6, 5, 7))
    assert np.allclose(fd.surface_laplacian(u, np.full(u.shape, 2.5), h), 2.5 * fd.laplacian(u, h), atol=1e-12)


def test_discrete_laplacian_eigenvalue():
    n, L = 16, 2.0
    h = (L / n, L / n)
    x = np.arange(n) * h[0]
    k = 2 * math.pi * 3 / L
    u = np.sin(k * x)[None, :] * np.ones((n, n))
    lam = -(4.0 / h[0] ** 2) * math.sin(k * h[0] / 2) ** 2
    assert np.allclose(fd.laplacian(u, h), lam * u, atol=1e-10)


def test_surface_laplacian_symmetric_conservative_and_energy_identity():
    rng = np.random.default_rng(1)
    h = (0.3, 0.2)
    g = rng.uniform(0.1, 1.0, (9, 11))
    a, b = rng.standard_normal((2, 9, 11))
    La, Lb = fd.surface_laplacian(a, g, h), fd.surface_laplacian(b, g, h)
    assert math.isclose(fd.inner(La, b, h), fd.inner(a, Lb, h), rel_tol=1e-12)
    assert abs(np.sum(La)) < 1e-11 * np.sum(np.abs(La))
    assert math.isclose(fd.grad_energy(a, g, h), -fd.inner(La, a, h), rel_tol=1e-12)
    F = [rng.standard_normal((9, 11)) for _ in range(2)]
    assert abs(np.sum(fd.central_div(F, h))) < 1e-11


def _band_case():
    p = wl.ModelParams(dim=2, n=(48, 48, 1), half_len=(math.pi,) * 3)
    phi = wl.sphere_phi(p, 1.5, 0.15)
    g = model.g_loc(phi)
    band = bm.band_mask(phi)
    return p, g, band


def test_band_solve_matches_sparse_direct_solve():
    p, g, band = _band_case()
    h = p.h[:2]
    f = np.random.default_rng(2).standard_normal(g.shape)
    w, it, rel = bm.solve_neg_lap(f, g, band, h, rtol=1e-14)
    assert rel <= 1e-14
    idx = np.flatnonzero(band.ravel())
    n = idx.size
    pos = -np.ones(band.size, int)
    pos[idx] = np.arange(n)
    # assemble the band matrix column by column from unit vectors, then a bordered system
    cols = []
    coeffs = bm.face_coeffs(g, band)
    for j in idx:
        e = np.zeros(band.size)
        e[j] = 1.0
        cols.append(bm.apply_neg_lap(e.reshape(g.shape), coeffs, h).ravel()[idx])
    A = np.array(cols).T
    comp, nc = bm.components(band)
    assert nc == 1
    rhs = f.ravel()[idx] - f.ravel()[idx].mean()
    K = sp.bmat([[sp.csr_matrix(A), np.ones((n, 1))], [np.ones((1, n)), None]], format="csc")
    sol = spla.spsolve(K, np.concatenate([rhs, [0.0]]))[:n]
    assert np.max(np.abs(w.ravel()[idx] - sol)) < 1e-9 * np.max(np.abs(sol))
    assert np.allclose(w[~band], 0.0)


def test_components_periodic_and_per_component_mean():
    p = wl.ModelParams(dim=2, n=(40, 40, 1), half_len=(math.pi,) * 3)
    phi = np.maximum(wl.sphere_phi(p, 0.7, 0.08, (-1.6, 0, 0)), wl.sphere_phi(p, 0.7, 0.08, (1.6, 0, 0)))
    band = bm.band_mask(phi)
    comp, nc = bm.components(band)
    assert nc == 2
    # a band strip crossing the periodic boundary is one component
    strip = np.zeros((10, 10), bool)
    strip[:, 0] = True
    strip[:, 9] = True
    assert bm.components(strip)[1] == 1
    g = model.g_loc(phi)
    f = np.random.default_rng(4).standard_normal(g.shape)
    w, _, rel = bm.solve_neg_lap(f, g, band, p.h[:2], rtol=1e-13)
    assert rel <= 1e-13
    for c in range(nc):
        assert abs(w[comp == c].mean()) < 1e-12
