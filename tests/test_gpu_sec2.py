"""GPU parity of the g^{1/2}-split scheme of Sec. 2.2 (model ETD_MODEL_FIXED_SQRTG = 2) with the
oracle's band scheme (oracle.section2.BandScheme: dense band matrix, phi_j by eigen-decomposition,
the paper's form phi_0 V + tau phi_1 R).  The GPU takes phi_j(tau L) through Lanczos Krylov
spaces to a relative error estimate of 1e-12 (FP64) and advances V + tau phi_1(tau L)(R - L V).

* 2D: the paper's rate-study membrane (circle, eps_phi = 10 h, eps_u = 10 h) at 64^2, random U0
  in [0.2, 0.8], ETD1 and ETDRK2, 8 steps of tau = 1e-4; FP64 to 1e-10 (relative L2 on the band),
  FP32-mixed to 2e-5.
* 3D: the c2 sphere at 32^3 (tau = 1e-2, tau L spans [20, 51]: Krylov spaces of 20-40), ETDRK2,
  4 steps, FP64 to 1e-10; the linear flow alone (R = 0, e^{-tau L} V) to 1e-10 at tau = 1e-4
  (at tau B = 20 the flow shrinks V by e^{-20}, and V + tau phi_1(tau L)(-L V) forms that by
  cancellation: an absolute error of rounding size, which only a near-zero result exposes).
* U off the band is never written (bit-exact).
* At the paper's full 256^2: U = 1 on the band is a steady state of the full model (W', f'
  vanish; L g^{1/2} = B g^{1/2}) to 1e-11, and the Krylov dimension is reported.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import section2  # noqa: E402
from paper_2606_04347_gb300 import Plan  # noqa: E402
from paper_2606_04347_gb300 import workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _oracle(p, phi):
    return section2.BandScheme(phi, p.h[:p.dim], eps_u=p.eps_u, gamma=p.gamma, M=p.M, ubar=p.ubar, B=p.B2,
                               band_hi=p.band_mask_hi, cg_rtol=1e-14, linear_only=bool(p.linear_only))


def _dev(x, prec):
    return torch.tensor(x, dtype=torch.float64 if prec == 0 else torch.float32, device=DEV)


def _band_rel(a, b, band):
    return float(np.linalg.norm((a - b)[band]) / np.linalg.norm(b[band]))


def _run_gpu(p, phi, U0, nsteps):
    plan = Plan(p)
    u = _dev(U0, p.precision)
    d = plan.step(_dev(phi, p.precision), u, nsteps, diag=True)
    plan.close()
    return u.cpu().numpy().astype(np.float64), d


def _paper2d_64(scheme, precision=0):
    p, phi, _ = wl.paper2d("circle", 10.0, scheme, precision, n=64)
    p = p.replace(model=2, cg_rtol=1e-13 if precision == 0 else 1e-6)
    U0 = wl.random_fields(p.shape, 31, 0.2, 0.8)
    return p, phi, U0


@pytest.mark.parametrize("scheme", [1, 2])
def test_sec2_2d_matches_oracle_fp64(scheme):
    p, phi, U0 = _paper2d_64(scheme)
    bs = _oracle(p, phi)
    want = bs.run(U0.copy(), p.tau, scheme, 8)
    got, d = _run_gpu(p, phi, U0, 8)
    print("2D scheme", scheme, "band", d["band_size"], "krylov dim", d["krylov_dim_last"])
    assert d["band_size"] == bs.idx.size
    assert 1 <= d["krylov_dim_last"] <= 128
    assert _band_rel(got, want, bs.band) < 1e-10
    assert np.array_equal(got[~bs.band], U0[~bs.band])


@pytest.mark.parametrize("scheme", [1, 2])
def test_sec2_2d_fp32_form(scheme):
    p, phi, U0 = _paper2d_64(scheme, precision=1)
    bs = _oracle(p.replace(precision=0), phi)
    want = bs.run(U0.copy(), p.tau, scheme, 8)
    got, _ = _run_gpu(p, phi, U0, 8)
    assert _band_rel(got, want, bs.band) < 2e-5


def test_sec2_3d_matches_oracle_fp64():
    p, phi, U0, _ = wl.workload("c2", n=32)
    p = p.replace(model=2, cg_rtol=1e-13)
    bs = _oracle(p, phi)
    want = bs.run(U0.copy(), p.tau, 2, 4)
    got, d = _run_gpu(p, phi, U0, 4)
    print("3D band", d["band_size"], "krylov dim", d["krylov_dim_last"])
    assert d["krylov_dim_last"] >= 8
    assert _band_rel(got, want, bs.band) < 1e-10
    assert np.array_equal(got[~bs.band], U0[~bs.band])


@pytest.mark.parametrize("scheme", [1, 2])
def test_sec2_3d_linear_flow(scheme):
    p, phi, U0, _ = wl.workload("c2", n=32)
    p = p.replace(model=2, linear_only=1, scheme=scheme, tau=1e-4, cg_rtol=1e-13)
    bs = _oracle(p, phi)
    want = bs.run(U0.copy(), p.tau, scheme, 5)
    got, _ = _run_gpu(p, phi, U0, 5)
    assert _band_rel(got, want, bs.band) < 1e-10


@pytest.mark.parametrize("scheme", [1, 2])
def test_sec2_full_size_steady_state(scheme):
    p, phi, _ = wl.paper2d("circle", 10.0, scheme, 0)
    p = p.replace(model=2, cg_rtol=1e-12)
    band = wl.band_of(phi, p.band_mask_hi)
    U0 = wl.random_fields(p.shape, 9)
    U0[band] = 1.0
    got, d = _run_gpu(p, phi, U0, 5)
    print("256^2 band", d["band_size"], "krylov dim", d["krylov_dim_last"])
    assert d["band_size"] == int(band.sum())
    assert np.max(np.abs(got - U0)) < 1e-11
