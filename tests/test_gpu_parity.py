"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, row by row.

Tolerances: FP64 paths must agree with the oracle to relative L2 1e-11 (full steps) or
tighter for single operators; FP32-mixed paths to relative L2 1e-5.
Integer work (the band index list) is compared bit for bit, the band decision taken in
the precision of the field on both sides.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import band as obm  # noqa: E402
from oracle import etd as oetd  # noqa: E402
from oracle import fft as offt  # noqa: E402
from oracle import model as omodel  # noqa: E402
from paper_2606_04347_gb300 import Plan  # noqa: E402
from paper_2606_04347_gb300 import workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def dev(x, prec):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64 if prec == 0 else torch.float32, device=DEV)


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


# ---------------------------------------------------------------- S1 / S6: the FFT
@pytest.mark.parametrize("prec,tol", [(0, 1e-13), (1, 2e-6)])
@pytest.mark.parametrize("shape", [(2, (32, 16, 1)), (2, (128, 128, 1)), (3, (16, 32, 8)), (3, (64, 64, 64)),
                                   (3, (32, 256, 16))])
def test_fft_forward_inverse_match_oracle(prec, tol, shape):
    dim, n = shape
    p = wl.workload("c3", n=8)[0].replace(dim=dim, n=n, model=0, precision=prec)
    f = wl.random_fields(p.shape, 17, -1.0, 1.0)
    plan = Plan(p)
    nxh = n[0] // 2 + 1
    spec_shape = p.shape[:-1] + (nxh,)
    out = torch.zeros(spec_shape, dtype=plan.cdtype, device=DEV)
    plan.fft_forward(dev(f, prec), out)
    want = offt.half_spectrum(offt.fftn(f))
    got = out.cpu().numpy()
    assert rel_l2(got.real, want.real) < tol and rel_l2(got.imag, want.imag) < tol * 10
    back = torch.zeros(p.shape, dtype=plan.dtype, device=DEV)
    plan.fft_inverse(out, back)
    assert rel_l2(host(back), f) < tol


@pytest.mark.parametrize("prec,tol", [(0, 1e-13), (1, 2e-6)])
@pytest.mark.parametrize("shape", [(3, (96, 96, 96)), (3, (64, 96, 32)), (3, (32, 64, 96)), (2, (96, 64, 1)),
                                   (2, (128, 96, 1))])
def test_fft_radix3_lengths_match_oracle(prec, tol, shape):
    """96-point axes (24 values on 4 lanes per team; 6-point column DFTs across y)."""
    dim, n = shape
    p = wl.workload("c3", n=8)[0].replace(dim=dim, n=n, model=0, precision=prec)
    f = wl.random_fields(p.shape, 23, -1.0, 1.0)
    plan = Plan(p)
    out = torch.zeros(p.shape[:-1] + (n[0] // 2 + 1,), dtype=plan.cdtype, device=DEV)
    plan.fft_forward(dev(f, prec), out)
    want = offt.half_spectrum(offt.fftn(f))
    got = out.cpu().numpy()
    assert rel_l2(got.real, want.real) < tol and rel_l2(got.imag, want.imag) < tol * 10
    back = torch.zeros(p.shape, dtype=plan.dtype, device=DEV)
    plan.fft_inverse(out, back)
    assert rel_l2(host(back), f) < tol


def test_fixed_96_matches_oracle():
    """Fixed-membrane ETDRK2 on a 96^3 grid (generic neighbour arithmetic, multigrid levels of
    96, 48, 24, 12 cells per axis), FP64 against the oracle to 1e-11; the FP32-mixed form within
    3e-5: here tau B2 = 4, so the u-stage's increment is nearly all of G U every step, and the
    FP32 transform noise of G U (eps32 rms(G U)) divided by G down to 1e-3 at the recovery edge
    sets the difference (1.2e-5 measured after 4 steps)."""
    p, phi, u, _ = wl.workload("c2", n=96)
    p = p.replace(tau=2e-3, cg_rtol=1e-13)
    # the same input for both precisions: phi and u as FP32 values
    phi, u = phi.astype(np.float32).astype(np.float64), u.astype(np.float32).astype(np.float64)
    want = oetd.FixedStepper(p, phi).run(u.copy(), 4)
    plan = Plan(p)
    ud = dev(u, 0)
    plan.step(dev(phi, 0), ud, 4)
    assert rel_l2(host(ud), want) < 1e-11
    plan32 = Plan(p.replace(precision=1, cg_rtol=1e-6))
    u32 = dev(u, 1)
    plan32.step(dev(phi, 1), u32, 4)
    assert rel_l2(host(u32), want) < 3e-5


# ---------------------------------------------------------------- S8: band compaction
@pytest.mark.parametrize("prec", [0, 1])
def test_band_index_list_is_bit_exact(prec):
    p, phi, u, _ = wl.workload("c3", n=64, precision=prec)
    plan = Plan(p)
    idx = torch.zeros(phi.size, dtype=torch.int32, device=DEV)
    cnt = plan.band(dev(phi, prec), idx)
    f = phi.astype(np.float64 if prec == 0 else np.float32)
    mask = np.abs(f.dtype.type(2) * f - f.dtype.type(1)) < f.dtype.type(p.band_mask_hi)
    want = np.flatnonzero(mask.ravel())
    assert cnt == want.size
    assert np.array_equal(idx[:cnt].cpu().numpy(), want)


# ---------------------------------------------------------------- S10: band solve
@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 2e-5)])
def test_nonlocal_band_solve_matches_oracle(prec, tol):
    p, phi, u, _ = wl.workload("c3", n=32, precision=prec)
    p = p.replace(cg_rtol=1e-13 if prec == 0 else 1e-6)
    g = omodel.g_loc(phi)
    band = obm.band_mask(phi)
    f = g * (u - p.ubar)
    want, _, _ = obm.solve_neg_lap(f, g, band, p.h, rtol=1e-14)
    plan = Plan(p)
    w = torch.zeros(p.shape, dtype=plan.dtype, device=DEV)
    it, res = plan.nonlocal_solve(dev(phi, prec), dev(f, prec), w)
    assert res <= p.cg_rtol and it > 0
    assert rel_l2(host(w), want) < tol


# ---------------------------------------------------------------- S7 / S9: remainders
@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-5)])
def test_R1_matches_oracle(prec, tol):
    p, phi, u, _ = wl.workload("c3", n=32, precision=prec)
    A0 = omodel.volume(phi, p) - 0.05
    p = p.replace(A0=A0)
    want = omodel.R1(phi, u, p, A0)
    plan = Plan(p)
    out = torch.zeros(p.shape, dtype=plan.dtype, device=DEV)
    plan.remainder(1, dev(phi, prec), None, dev(u, prec), out)
    assert rel_l2(host(out), want) < tol


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 5e-5)])
def test_R2_coupled_matches_oracle(prec, tol):
    p, phi, u, _ = wl.workload("c3", n=32, precision=prec)
    p = p.replace(cg_rtol=1e-13 if prec == 0 else 1e-6)
    phi_old = phi + 1e-3 * wl.random_fields(p.shape, 3, -1, 1) * obm.band_mask(phi)
    want = omodel.R2_coupled(phi, phi_old, u, p.replace(cg_rtol=1e-14), omodel.BandSolver(p.replace(cg_rtol=1e-14)))
    plan = Plan(p)
    out = torch.zeros(p.shape, dtype=plan.dtype, device=DEV)
    plan.remainder(2, dev(phi, prec), dev(phi_old, prec), dev(u, prec), out)
    assert rel_l2(host(out), want) < tol


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 5e-5)])
def test_R2_fixed_matches_oracle(prec, tol):
    p, phi, u, _ = wl.workload("c1", n=64, precision=prec)
    p = p.replace(cg_rtol=1e-13 if prec == 0 else 1e-6)
    g = omodel.g_loc(phi)
    band = obm.band_mask(phi)
    want = omodel.R2_fixed(u, g, band, p, omodel.BandSolver(p.replace(cg_rtol=1e-14)))
    plan = Plan(p)
    out = torch.zeros(p.shape, dtype=plan.dtype, device=DEV)
    plan.remainder(3, dev(phi, prec), None, dev(u, prec), out)
    assert rel_l2(host(out), want) < tol


# ---------------------------------------------------------------- S3-S5: exact exponential
@pytest.mark.parametrize("prec,tol", [(0, 1e-13), (1, 2e-6)])
def test_single_mode_coupled_linear_only(prec, tol):
    p = wl.workload("c3", n=32, precision=prec)[0].replace(linear_only=1, tau=3e-4, A0=0.0)
    x, y, z = wl.grid(p.n, p.half_len, 3)
    phi0 = 0.5 + 0.2 * np.cos(3 * x + 2 * y - z) * np.ones(p.shape)
    from oracle import spectral
    l = spectral.l_phi(p, np.array([0.0, -14.0]))
    want = 0.5 * math.exp(-5 * p.tau * l[0]) + 0.2 * math.exp(-5 * p.tau * l[1]) * np.cos(3 * x + 2 * y - z)
    plan = Plan(p)
    phi = dev(phi0, prec)
    u = dev(np.full(p.shape, 0.5), prec)
    plan.step(phi, u, 5)
    assert np.max(np.abs(host(phi) - want)) < tol


@pytest.mark.parametrize("scheme", [1, 2])
def test_single_mode_fixed_linear_only(scheme):
    p = wl.workload("c2", n=32)[0].replace(linear_only=1, scheme=scheme, tau=1e-3)
    x, y, z = wl.grid(p.n, p.half_len, 3)
    u0 = 0.5 + 0.1 * np.sin(2 * x - 5 * z) * np.ones(p.shape)
    from oracle import spectral
    l = spectral.l_u(p, np.array([0.0, -29.0]))
    want = 0.5 * math.exp(-4 * p.tau * l[0]) + 0.1 * math.exp(-4 * p.tau * l[1]) * np.sin(2 * x - 5 * z)
    plan = Plan(p)
    u = dev(u0, 0)
    plan.step(dev(np.full(p.shape, 0.5), 0), u, 4)
    assert np.max(np.abs(host(u) - want)) < 1e-13


# ---------------------------------------------------------------- full steps
def test_c1_fixed_etd1_100_steps_fp64_matches_oracle():
    p, phi, u, nsteps = wl.workload("c1")
    st = oetd.FixedStepper(p, phi)
    want = st.run(u.copy(), nsteps)
    plan = Plan(p)
    ud = dev(u, 0)
    d = plan.step(dev(phi, 0), ud, nsteps, diag=True)
    assert d["band_size"] == int(obm.band_mask(phi).sum())
    assert rel_l2(host(ud), want) < 1e-11
    e = plan.energy(dev(phi, 0), ud)
    ew = st.energy(want)
    assert abs(e["energy"] - ew["total"]) < 1e-10 * abs(ew["total"])
    assert abs(e["mass"] - ew["mass"]) < 1e-10 * max(1.0, abs(ew["mass"]))
    mb, mn, mx = omodel.bound_stats(want, st.G, p.recover_delta)
    assert abs(e["max_bound"] - mb) < 1e-10 and abs(e["umin"] - mn) < 1e-10 and abs(e["umax"] - mx) < 1e-10


@pytest.mark.parametrize("scheme", [1, 2])
def test_fixed_3d_matches_oracle(scheme):
    p, phi, u, _ = wl.workload("c2", n=32, scheme=scheme, tau=5e-3)
    st = oetd.FixedStepper(p, phi)
    want = st.run(u.copy(), 6)
    plan = Plan(p)
    ud = dev(u, 0)
    plan.step(dev(phi, 0), ud, 3)
    plan.step(None, ud, 3)          # later calls reuse the frozen membrane
    assert rel_l2(host(ud), want) < 1e-11


def _two_spheres(n):
    """c3 coupled parameters on a membrane of two separated spheres: a two-component band."""
    p = wl.workload("c3", n=n)[0]
    phi = wl.two_spheres_phi(p, (0.8, 0.6), ((-1.6, 0.0, 0.0), (1.6, 0.0, 0.0)), 0.12)
    band = obm.band_mask(phi, p.band_mask_hi)
    assert obm.components(band)[1] == 2
    u = np.where(band, wl.random_fields(p.shape, 7, 0.45, 0.55), 0.5)
    return p, phi, u, band


@pytest.mark.parametrize("n", [32, 64])
def test_nonlocal_two_component_band_matches_oracle(n):
    """Sec. 2.1 mean removal per connected band component: each component's solution has zero
    mean and the whole solution matches the oracle's per-component solve."""
    p, phi, u, band = _two_spheres(n)
    p = p.replace(cg_rtol=1e-13)
    g = omodel.g_loc(phi)
    f = np.where(band, wl.random_fields(p.shape, 8, -1.0, 1.0), 0.0)
    want, _, _ = obm.solve_neg_lap(f, g, band, p.h, rtol=1e-14)
    plan = Plan(p)
    w = torch.zeros(p.shape, dtype=torch.float64, device=DEV)
    it, rs = plan.nonlocal_solve(dev(phi, 0), dev(f, 0), w)
    got = host(w)
    comp, nc = obm.components(band)
    for c in range(nc):
        assert abs(got[comp == c].mean()) < 1e-12 * np.abs(got).max()
    assert rs <= 1e-13
    assert rel_l2(got, want) < 1e-10


def test_nonlocal_many_columns_band_matches_oracle():
    """A band of 128 disconnected z-columns (x + y even on a 16^3 grid): the cells of the
    multigrid hierarchy hold columns that touch only diagonally, so the labelling falls back to
    the union-find over the band, and the many components take the per-warp sums."""
    p = wl.workload("c3", n=16)[0].replace(cg_rtol=1e-13)
    z, y, x = np.meshgrid(np.arange(16), np.arange(16), np.arange(16), indexing="ij")
    phi = np.where((x + y) % 2 == 0, 0.5, 0.0)
    band = obm.band_mask(phi, p.band_mask_hi)
    assert obm.components(band)[1] == 128
    g = omodel.g_loc(phi)
    f = np.where(band, wl.random_fields(p.shape, 9, -1.0, 1.0), 0.0)
    want, _, _ = obm.solve_neg_lap(f, g, band, p.h, rtol=1e-14)
    plan = Plan(p)
    w = torch.zeros(p.shape, dtype=torch.float64, device=DEV)
    it, rs = plan.nonlocal_solve(dev(phi, 0), dev(f, 0), w)
    assert rs <= 1e-13
    assert rel_l2(host(w), want) < 1e-10


def test_coupled_two_component_band_matches_oracle_fp64():
    p, phi, u, _ = _two_spheres(32)
    cs = oetd.CoupledStepper(p)
    wphi, wu = cs.run(phi.copy(), u.copy(), 2)
    plan = Plan(p)
    phid, ud = dev(phi, 0), dev(u, 0)
    d = plan.step(phid, ud, 2, diag=True)
    assert rel_l2(host(phid), wphi) < 1e-11
    assert rel_l2(host(ud), wu) < 1e-11
    assert d["cg_resid_last"] <= p.cg_rtol


@pytest.mark.parametrize("scheme,n,steps", [(2, 32, 4), (1, 32, 4), (2, 64, 2)])
def test_coupled_matches_oracle_fp64(scheme, n, steps):
    p, phi, u, _ = wl.workload("c3", n=n, scheme=scheme)
    cs = oetd.CoupledStepper(p)
    wphi, wu = cs.run(phi.copy(), u.copy(), steps)
    plan = Plan(p)
    phid, ud = dev(phi, 0), dev(u, 0)
    plan.step(phid, ud, steps)
    assert rel_l2(host(phid), wphi) < 1e-11
    assert rel_l2(host(ud), wu) < 1e-11


def test_coupled_fp32_against_fp64_gpu():
    """FP32-mixed vs FP64 on the GPU after 20 coupled ETDRK2 steps from the same input:
    phi, u (plain relative L2 over the whole grid) and the energy within 1e-5."""
    p, phi, u, _ = wl.workload("c3", n=32)
    p = p.replace(cg_rtol=1e-12)
    ref = Plan(p)
    phi64, u64 = dev(phi, 0), dev(u, 0)
    ref.step(phi64, u64, 20)
    p32 = p.replace(precision=1, cg_rtol=1e-6)
    plan = Plan(p32)
    phi32, u32 = dev(phi, 1), dev(u, 1)
    d = plan.step(phi32, u32, 20, diag=True)
    U64, U32 = host(u64), host(u32)
    e64 = ref.energy(phi64, u64)
    e32 = plan.energy(phi32, u32)
    print("fp32 vs fp64: phi", rel_l2(host(phi32), host(phi64)), "u", rel_l2(U32, U64),
          "energy", abs(e32["energy"] - e64["energy"]) / abs(e64["energy"]),
          "max bound", e32["max_bound"], e64["max_bound"])
    assert rel_l2(host(phi32), host(phi64)) < 1e-5
    assert rel_l2(U32, U64) < 1e-5
    assert abs(e32["energy"] - e64["energy"]) < 1e-5 * abs(e64["energy"])
    # maximum bound: where the FP64 form keeps max|2U-1| <= 1, the FP32 form stays within 1e-6
    if e64["max_bound"] <= 1.0:
        assert e32["max_bound"] <= 1.0 + 1e-6
    assert d["cg_resid_last"] <= 1e-6


# ---------------------------------------------------------------- error paths
def test_nonfinite_state_is_reported():
    from paper_2606_04347_gb300.abi import EtdError
    p, phi, u, _ = wl.workload("c1", n=32)
    u = u.copy()
    u[3, 4] = np.nan
    plan = Plan(p)
    with pytest.raises(EtdError) as ei:
        plan.step(dev(phi, 0), dev(u, 0), 1, diag=True)
    assert ei.value.code in (4, 5)


def test_cg_iteration_cap_is_reported():
    from paper_2606_04347_gb300.abi import EtdError
    p, phi, u, _ = wl.workload("c1", n=32)
    plan = Plan(p.replace(cg_maxit=2))
    with pytest.raises(EtdError) as ei:
        plan.step(dev(phi, 0), dev(u, 0), 1, diag=True)
    assert ei.value.code == 5
