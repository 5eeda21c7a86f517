"""The host half of the Sec. 2.2 scheme's Krylov evaluation (etd_krylov_coeffs), CPU only: the
library's phi_j(tau T) e_1 of a symmetric tridiagonal T, from its Jacobi eigen-decomposition
and its phi_j series / closed forms, against

* LAPACK's eigen-decomposition of T with phi_0 .. phi_3 at 40 digits (mpmath), and, where
  tau T is not small, scipy's matrix exponential and the identities tau T phi_1 = I - e^{-tau T},
  (tau T)^2 phi_2 = e^{-tau T} - I + tau T;
* tau = 0: phi_j(0) = 1/j!, so y = e_1 / j!;
* a Lanczos process (numpy, full reorthogonalisation) on an SPD matrix A: |b| V_m y converges
  to phi_j(tau A) b, and the library's estimate |b| beta_m tau tail follows the true error
  to within a factor 10 until the rounding floor.
"""
import math

import numpy as np
import pytest
import scipy.linalg

from paper_2606_04347_gb300 import abi


def _tridiag(m, seed, lo=50.0, hi=5000.0):
    rng = np.random.default_rng(seed)
    a = rng.uniform(lo, hi, m)
    b = rng.uniform(0.1, 0.45, m - 1) * np.minimum(a[:-1], a[1:])   # diagonally dominant: SPD
    return a, b


def _dense(a, b):
    return np.diag(a) + np.diag(b, 1) + np.diag(b, -1)


def _phi_mp(z, k):
    """phi_k(z) from the closed forms at 40 digits (no cancellation at these z)."""
    mpmath = pytest.importorskip("mpmath")
    with mpmath.workdps(40):
        z = mpmath.mpf(z)
        e = mpmath.exp(-z)
        if z == 0:
            return 1.0 / math.factorial(k)
        p = [e, (1 - e) / z]
        p.append((1 - p[1]) / z)
        p.append((mpmath.mpf(1) / 2 - p[2]) / z)
        return float(p[k])


@pytest.mark.parametrize("m", [1, 2, 5, 30, 128])
@pytest.mark.parametrize("tau", [1e-5, 1e-3, 2e-2])
def test_phi_of_tridiagonal_matches_eigen_reference(m, tau):
    a, b = _tridiag(m, m)
    lam, Q = np.linalg.eigh(_dense(a, b))
    for j in range(3):
        want = Q @ (np.array([_phi_mp(tau * l, j) for l in lam]) * Q[0])
        want_tail = abs(Q[m - 1] @ (np.array([_phi_mp(tau * l, j + 1) for l in lam]) * Q[0]))
        y, tail = abi.krylov_coeffs(a, b, tau, j)
        assert np.max(np.abs(y - want)) < 1e-12 * max(1.0, np.max(np.abs(want))), (m, tau, j)
        assert abs(tail - want_tail) < 1e-12 * max(1.0, want_tail) + 1e-15, (m, tau, j)


@pytest.mark.parametrize("tau", [1e-3, 2e-2])
def test_phi_of_tridiagonal_satisfies_exact_identities(tau):
    """Where tau T is not small the identities hold without cancellation: phi_0 = expm(-tau T),
    tau T phi_1 = I - e^{-tau T}, (tau T)^2 phi_2 = e^{-tau T} - I + tau T."""
    a, b = _tridiag(30, 4)
    Z = tau * _dense(a, b)
    I = np.eye(30)
    E = scipy.linalg.expm(-Z)
    ref = [E, np.linalg.solve(Z, I - E), np.linalg.solve(Z, np.linalg.solve(Z, E - I + Z))]
    for j in range(3):
        y, _ = abi.krylov_coeffs(a, b, tau, j)
        assert np.max(np.abs(y - ref[j][:, 0])) < 1e-10 * max(1.0, np.max(np.abs(ref[j][:, 0])))


@pytest.mark.parametrize("j", [0, 1, 2])
def test_tau_zero_gives_inverse_factorials(j):
    a, b = _tridiag(7, 3)
    y, tail = abi.krylov_coeffs(a, b, 0.0, j)
    want = np.zeros(7)
    want[0] = 1.0 / math.factorial(j)
    assert np.allclose(y, want, atol=1e-15, rtol=0)
    assert tail < 1e-15         # e_m^T phi_{j+1}(0) e_1 = 0 for m > 1 (up to the eigenvector rounding)


def _lanczos(A, v, m):
    n = A.shape[0]
    V = np.zeros((m + 1, n))
    al, be = np.zeros(m), np.zeros(m)
    V[0] = v / np.linalg.norm(v)
    for k in range(m):
        w = A @ V[k] - (be[k - 1] * V[k - 1] if k else 0.0)
        al[k] = w @ V[k]
        w -= al[k] * V[k]
        w -= V[:k + 1].T @ (V[:k + 1] @ w)
        be[k] = np.linalg.norm(w)
        V[k + 1] = w / be[k]
    return V, al, be


@pytest.mark.parametrize("j", [1, 2])
def test_krylov_estimate_follows_true_error(j):
    n, tau = 200, 1e-2
    rng = np.random.default_rng(11)
    c = 2000.0 * (1.0 + 0.5 * np.sin(0.1 * np.arange(n - 1)))
    A = 50.0 * np.eye(n)
    for i in range(n - 1):     # a 1D variable-coefficient Laplacian plus B: the shape of L
        A[i, i] += c[i]
        A[i + 1, i + 1] += c[i]
        A[i, i + 1] -= c[i]
        A[i + 1, i] -= c[i]
    bvec = rng.standard_normal(n)
    mu, Q = np.linalg.eigh(A)
    z = tau * mu
    phi = {1: -np.expm1(-z) / z, 2: (np.expm1(-z) + z) / z ** 2}[j]
    exact = Q @ (phi * (Q.T @ bvec))
    nb = np.linalg.norm(bvec)
    errs, ests = [], []
    for m in (8, 16, 24, 32, 40, 48, 56):
        V, al, be = _lanczos(A, bvec, m)
        y, tail = abi.krylov_coeffs(al, be[:-1], tau, j)
        got = nb * V[:m].T @ y
        errs.append(np.linalg.norm(got - exact) / np.linalg.norm(exact))
        ests.append(be[m - 1] * tau * tail / np.linalg.norm(y))
    assert errs[-1] < 1e-10 and errs[0] > 1e-3
    for e, s in zip(errs, ests):
        if e > 1e-12:
            assert s / 10 < e < 10 * s, (errs, ests)


@pytest.mark.parametrize("args", [dict(m=0), dict(m=129), dict(j=3), dict(tau=-1.0)])
def test_invalid_arguments(args):
    kw = dict(m=4, j=1, tau=1e-3)
    kw.update(args)
    m = kw["m"]
    a = np.ones(max(m, 1))
    b = np.zeros(max(m - 1, 1))
    y = np.zeros(max(m, 1))
    import ctypes as ct
    dp = ct.POINTER(ct.c_double)
    t = ct.c_double()
    code = abi.load_library().etd_krylov_coeffs(m, a.ctypes.data_as(dp), b.ctypes.data_as(dp), kw["tau"], kw["j"],
                                                y.ctypes.data_as(dp), ct.byref(t))
    assert code == 1
