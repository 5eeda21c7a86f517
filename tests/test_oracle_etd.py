"""Pins of the ETD drivers: exact exponential of single modes, dense brute force,
the theorems of Sec. 2.2, and temporal orders."""
import math
import os

import numpy as np
import pytest
from scipy.linalg import expm

from oracle import etd, model, section2
from oracle import band as bm
from paper_2606_04347_gb300 import workloads as wl
from oracle import spectral

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_single_mode_coupled_linear_only_is_exact_exponential():
    p = wl.workload("c3", n=16)[0].replace(linear_only=1, tau=3e-4)
    x, y, z = wl.grid(p.n, p.half_len, 3)
    phi0 = 0.5 + 0.2 * np.cos(3 * x + 2 * y - z) * np.ones(p.shape)
    cs = etd.CoupledStepper(p, A0=0.0)
    phi, u = cs.run(phi0, np.full(p.shape, 0.5), 5)
    lam = np.array([0.0, -14.0])
    l = spectral.l_phi(p, lam)
    want = 0.5 * math.exp(-5 * p.tau * l[0]) + 0.2 * math.exp(-5 * p.tau * l[1]) * np.cos(3 * x + 2 * y - z)
    assert np.max(np.abs(phi - want)) < 1e-14


def test_single_mode_fixed_linear_only_constant_g():
    p = wl.workload("c2", n=16)[0].replace(linear_only=1, scheme=2, tau=1e-3)
    x, y, z = wl.grid(p.n, p.half_len, 3)
    st = etd.FixedStepper(p, np.full(p.shape, 0.5))      # g = 1.125 everywhere
    u0 = 0.5 + 0.1 * np.sin(2 * x - 5 * z) * np.ones(p.shape)
    u = st.run(u0, 4)
    l = spectral.l_u(p, np.array([0.0, -29.0]))
    want = 0.5 * math.exp(-4 * p.tau * l[0]) + 0.1 * math.exp(-4 * p.tau * l[1]) * np.sin(2 * x - 5 * z)
    assert np.max(np.abs(u - want)) < 1e-14


def _dense_phi_mats(Lmat, tau):
    n = Lmat.shape[0]
    A = -tau * Lmat
    I, Z = np.eye(n), np.zeros((n, n))
    P0 = expm(A)
    P1 = expm(np.block([[A, I], [Z, Z]]))[:n, n:]
    P2 = expm(np.block([[A, I, Z], [Z, Z, I], [Z, Z, Z]]))[:n, 2 * n:]
    return P0, P1, P2


@pytest.mark.parametrize("scheme", [1, 2])
def test_dense_8x8_brute_force_matches_fft_path(scheme):
    p = wl.workload("c1", n=8)[0].replace(scheme=scheme, tau=2e-3, cg_rtol=1e-15)
    phi = wl.sphere_phi(p, 1.6, 0.5)
    u0 = wl.random_fields(p.shape, 11, 0.3, 0.7)
    st = etd.FixedStepper(p, phi)
    got = st.step(u0)
    # dense route: spectral Laplacian from the DFT matrix, phi_j by expm of augmented matrices
    n = 8
    k = np.arange(n)
    F1 = np.exp(-2j * np.pi * np.outer(k, k) / n)
    F2 = np.kron(F1, F1)
    lam = spectral.laplacian_symbol(p).ravel()
    Lap = (np.linalg.inv(F2) @ np.diag(lam) @ F2).real
    Lu = p.B2 * np.eye(n * n) - p.eps_u * p.B1 * Lap
    P0, P1, P2 = _dense_phi_mats(Lu, p.tau)
    G = st.G.ravel()
    R = lambda U: st.R2(U.reshape(p.shape)).ravel()
    rec = lambda GU: model.recover(GU, G, p.recover_delta)
    U = u0.ravel()
    GUt = P0 @ (G * U) + p.tau * (P1 @ R(U))
    if scheme == 1:
        want = rec(GUt)
    else:
        Ut = rec(GUt)
        want = rec(GUt + p.tau * (P2 @ (R(Ut) - R(U))))
    assert np.max(np.abs(got.ravel() - want)) < 1e-11


def _sec2_case(n=10):
    p = wl.ModelParams(dim=2, n=(n, n, 1), half_len=(math.pi,) * 3)
    x, y = wl.grid(p.n, p.half_len, 2)
    phi = 0.5 + 0.3 * np.sin(x) * np.cos(y)
    return p, phi


@pytest.mark.parametrize("tau", [1e-3, 1.0, 100.0])
def test_sec2_exponential_is_nonnegative_and_weighted_contraction(tau):
    p, phi = _sec2_case()
    ds = section2.DenseScheme(phi, p.h[:2], eps_u=0.2, gamma=50.0, M=10.0, ubar=0.4, B=30.0)
    E = ds.phi_mats(tau)[0]
    assert E.min() >= -1e-14 * np.abs(E).max()                      # Metzler lemma
    w = ds.sg
    wnorm = np.max(np.sum(np.abs(E) * w[None, :], axis=1) / w)      # induced weighted norm
    assert wnorm <= math.exp(-30.0 * tau) * (1 + 1e-10)


@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("tau", [1e-3, 1.0, 100.0])
def test_sec2_maximum_bound_and_energy_decay(scheme, tau):
    p, phi = _sec2_case()
    args = dict(eps_u=0.2, gamma=50.0, M=10.0, ubar=0.4)
    probe = section2.DenseScheme(phi, p.h[:2], B=1.0, **args)
    C, area = probe.C_inf(), probe.area
    U0 = wl.random_fields(p.shape, 21).ravel()
    for B, check in ((section2.B_mbp(args["eps_u"], args["gamma"], args["M"], C, area), "mbp"),
                     (section2.B_energy(args["eps_u"], args["gamma"], args["M"], C, area), "energy")):
        ds = section2.DenseScheme(phi, p.h[:2], B=B, **args)
        mats = ds.phi_mats(tau)
        U, E = U0.copy(), ds.energy(U0)
        for _ in range(8):
            U = ds.step(U, tau, scheme, mats)
            if check == "mbp":
                assert U.min() >= -1e-12 and U.max() <= 1 + 1e-12
            else:
                En = ds.energy(U)
                assert En <= E + 1e-12 * abs(E)
                E = En


def _rates(errs):
    return [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


def test_sec2_temporal_orders_match_paper_tables():
    rows = {}
    for line in open(os.path.join(GOLDEN, "paper_table_rates.txt")):
        if line.strip() and not line.startswith("#"):
            name, *vals = line.split()
            rows[name] = [float(v) for v in vals]
    p, phi = _sec2_case(12)
    ds = section2.DenseScheme(phi, p.h[:2], eps_u=0.3, gamma=20.0, M=5.0, ubar=0.4, B=40.0)
    U0 = wl.random_fields(p.shape, 5, 0.2, 0.8).ravel()
    T = 0.064
    def run(tau, scheme):
        mats = ds.phi_mats(tau)
        U = U0.copy()
        for _ in range(int(round(T / tau))):
            U = ds.step(U, tau, scheme, mats)
        return U
    ref = {s: run(T / 2048, s) for s in (1, 2)}
    taus = [T / 16, T / 32, T / 64, T / 128]
    r1 = _rates([np.max(np.abs(run(t, 1) - ref[1])) for t in taus])
    r2 = _rates([np.max(np.abs(run(t, 2) - ref[2])) for t in taus])
    assert 0.9 <= r1[-1] <= 1.15 and all(0.9 <= v <= 1.15 for v in rows["ETD1"])
    assert 1.7 <= r2[-1] <= 2.15 and all(1.7 <= v <= 2.15 for v in rows["ETDRK2"])


def test_spectral_fixed_scheme_temporal_orders():
    p = wl.workload("c1", n=32)[0].replace(eps_u=0.4, gamma=20.0, M=20.0, B2=400.0, cg_rtol=1e-14)
    phi = wl.sphere_phi(p, 1.8, 0.3)
    u0 = wl.random_fields(p.shape, 9, 0.4, 0.6)
    T = 0.016
    def run(tau, scheme):
        st = etd.FixedStepper(p.replace(tau=tau, scheme=scheme), phi)
        return st.run(u0, int(round(T / tau)))
    G = model.g_loc(phi)
    sel = G > p.recover_delta
    out = {}
    for s in (1, 2):
        ref = run(T / 256, s)
        errs = [np.max(np.abs(run(T / m, s) - ref)[sel]) for m in (4, 8, 16)]
        out[s] = _rates(errs)
    assert 0.85 <= out[1][-1] <= 1.15
    assert 1.75 <= out[2][-1] <= 2.25
