"""Pins of the band-restricted Sec. 2.2 scheme (oracle.section2.BandScheme), CPU only.

* The dense band matrix equals the band operator's action (band.apply_neg_lap) on band
  values, and L is symmetric with non-positive off-diagonal entries and L g^{1/2} = B g^{1/2}.
* With 0 < phi < 1 everywhere and band_hi = 1 the band is the whole grid and one ETD1 /
  ETDRK2 step and the energy equal DenseScheme's (pinned by the theorems in test_oracle_etd).
* phi_0, tau phi_1, tau^2 phi_2 of tau L from the eigen-decomposition equal expm(-tau L),
  L^{-1}(I - e^{-tau L}) and L^{-2}(e^{-tau L} - I + tau L) (a library exponential and solves).
* U = 1 and U = 0 on the band are steady states of the full model (W', f' vanish there and
  L g^{1/2} = B g^{1/2}); U = 1/2 is steady when gamma = M = 0.  A misplaced g^{+-1/2} breaks
  these.
* The maximum bound principle (B >= Eq. (2.15)'s stabiliser) and energy decay (B >= Eq. (2.17)'s)
  hold for the band system, with C the band inverse's L^inf norm.
* ETD1 and ETDRK2 converge at rates 1 and 2 in tau on the band.
"""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import band as bandmod
from oracle import section2
from paper_2606_04347_gb300 import workloads as wl


def _circle_case(n=24, eps_cells=2.0, r0=0.45):
    """2D [-1,1]^2 with a tanh circle of radius r0, eps_phi = eps_cells h (a thin annular band)."""
    p = wl.ModelParams(dim=2, n=(n, n, 1), half_len=(1.0, 1.0, 1.0))
    x, y = wl.grid(p.n, p.half_len, 2)
    eps = eps_cells * p.h[0]
    phi = 0.5 + 0.5 * np.tanh(3.0 * (r0 - np.sqrt(x ** 2 + y ** 2)) / eps) * np.ones(p.shape)
    return p, phi


ARGS = dict(eps_u=0.05, gamma=40.0, M=20.0, ubar=0.3)


def test_band_matrix_is_the_band_operator():
    p, phi = _circle_case()
    bs = section2.BandScheme(phi, p.h[:2], B=10.0, **ARGS)
    assert 50 < bs.idx.size < p.n[0] * p.n[1]
    rng = np.random.default_rng(3)
    w = np.zeros(phi.shape)
    w.ravel()[bs.idx] = rng.standard_normal(bs.idx.size)
    want = bandmod.apply_neg_lap(w, bandmod.face_coeffs(bs.g, bs.band), p.h[:2]).ravel()[bs.idx]
    assert np.max(np.abs(bs.A @ w.ravel()[bs.idx] - want)) < 1e-12 * np.max(np.abs(want))
    L = bs.L
    assert np.array_equal(L, L.T)
    off = L - np.diag(np.diag(L))
    assert off.max() <= 0.0
    assert np.max(np.abs(L @ bs.sg - 10.0 * bs.sg)) < 1e-10 * np.max(np.abs(np.diag(L)))


@pytest.mark.parametrize("scheme", [1, 2])
def test_full_band_equals_dense_scheme(scheme):
    p = wl.ModelParams(dim=2, n=(10, 10, 1), half_len=(math.pi,) * 3)
    x, y = wl.grid(p.n, p.half_len, 2)
    phi = 0.5 + 0.3 * np.sin(x) * np.cos(y)
    args = dict(eps_u=0.2, gamma=50.0, M=10.0, ubar=0.4, B=30.0)
    ds = section2.DenseScheme(phi, p.h[:2], **args)
    bs = section2.BandScheme(phi, p.h[:2], band_hi=1.0, **args)
    assert bs.idx.size == phi.size and bs.comp[1] == 1
    U = wl.random_fields(p.shape, 8)
    for tau in (1e-3, 0.5):
        want = ds.step(U.ravel(), tau, scheme).reshape(p.shape)
        got = bs.step(U, tau, scheme)
        assert np.max(np.abs(got - want)) < 1e-10
    assert abs(bs.energy(U) - ds.energy(U.ravel())) < 1e-10 * abs(ds.energy(U.ravel()))


@pytest.mark.parametrize("tau", [1e-3, 1.0, 10.0])
def test_phi_functions_of_band_matrix(tau):
    p, phi = _circle_case(16, r0=0.5)
    bs = section2.BandScheme(phi, p.h[:2], B=5.0, **ARGS)
    P0, P1, P2 = bs.phi_mats(tau)
    L, I = bs.L, np.eye(bs.L.shape[0])
    E = scipy.linalg.expm(-tau * L)
    assert np.max(np.abs(P0 - E)) < 1e-10
    assert np.max(np.abs(tau * P1 - np.linalg.solve(L, I - E))) < 1e-9 * max(1.0, tau)
    want2 = np.linalg.solve(L, np.linalg.solve(L, E - I + tau * L))
    assert np.max(np.abs(tau * tau * P2 - want2)) < 1e-9 * max(1.0, tau * tau)


@pytest.mark.parametrize("scheme", [1, 2])
def test_constant_states_are_steady(scheme):
    p, phi = _circle_case()
    bs = section2.BandScheme(phi, p.h[:2], B=50.0, **ARGS)
    off = wl.random_fields(p.shape, 4)
    for val in (1.0, 0.0):
        U = off.copy()
        U.ravel()[bs.idx] = val
        V = U
        for _ in range(3):
            V = bs.step(V, 0.05, scheme)
        assert np.max(np.abs(V - U)) < 1e-9     # rounding of the dense phi_j products, divided by g^{1/2}
    bs0 = section2.BandScheme(phi, p.h[:2], B=50.0, eps_u=0.05, gamma=0.0, M=0.0, ubar=0.3)
    U = off.copy()
    U.ravel()[bs0.idx] = 0.5
    assert np.max(np.abs(bs0.step(U, 0.05, scheme) - U)) < 1e-9
    # a perturbed state does move (the steady checks are not vacuous)
    U.ravel()[bs0.idx[::3]] = 0.7
    assert np.max(np.abs(bs0.step(U, 0.05, scheme) - U)) > 1e-3


@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("tau", [1e-3, 1.0, 100.0])
def test_band_maximum_bound_and_energy_decay(scheme, tau):
    p, phi = _circle_case(20, r0=0.5)
    probe = section2.BandScheme(phi, p.h[:2], B=1.0, **ARGS)
    C, area = probe.C_inf(), 4.0
    U0 = wl.random_fields(p.shape, 21)
    for B, check in ((section2.B_mbp(ARGS["eps_u"], ARGS["gamma"], ARGS["M"], C, area), "mbp"),
                     (section2.B_energy(ARGS["eps_u"], ARGS["gamma"], ARGS["M"], C, area), "energy")):
        bs = section2.BandScheme(phi, p.h[:2], B=B, **ARGS)
        mats = bs.phi_mats(tau)
        U, E = U0.copy(), bs.energy(U0)
        for _ in range(6):
            U = bs.step(U, tau, scheme, mats)
            if check == "mbp":
                assert U.min() >= -1e-12 and U.max() <= 1 + 1e-12
            else:
                En = bs.energy(U)
                assert En <= E + 1e-12 * abs(E)
                E = En


def test_band_scheme_temporal_orders():
    p, phi = _circle_case(20, r0=0.5)
    bs = section2.BandScheme(phi, p.h[:2], B=50.0, eps_u=0.05, gamma=20.0, M=5.0, ubar=0.4)
    U0 = wl.random_fields(p.shape, 5, 0.2, 0.8)
    T = 0.002
    ref = bs.run(U0.copy(), T / 512, 2, 512)
    for scheme, lo, hi in ((1, 0.9, 1.1), (2, 1.85, 2.15)):
        errs = [np.max(np.abs(bs.run(U0.copy(), T / nst, scheme, nst) - ref)) for nst in (8, 16, 32)]
        rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
        assert lo < rates[-1] < hi, (scheme, errs, rates)
