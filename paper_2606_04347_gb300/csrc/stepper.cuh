// stepper.cuh -- the plan: workspace, coefficient tables and the per-step kernel sequence
// of Algorithm 1 (coupled model) or its frozen-membrane form (fixed model).
#pragma once
#include <cudaTypedefs.h>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>
#include "kernels.cuh"
#include "krylov.cuh"
#include "ops.cuh"
#include "plan.h"

namespace etd {

static_assert(kCCMaxLev >= kMGMax, "component labelling covers every multigrid level");

// phi_0, phi_1, phi_2 of Sec. 2.2 in FP64: Taylor series below z = 1 (the closed forms
// cancel there), closed forms through expm1 above.
inline void phi_functions(double z, double& p0, double& p1, double& p2) {
  p0 = std::exp(-z);
  if (std::fabs(z) < 1.0) {
    double s1 = 0.0, s2 = 0.0, fac1 = 1.0, fac2 = 2.0;
    double zk = 1.0;
    double t1[32], t2[32];
    for (int k = 0; k < 30; ++k) {
      t1[k] = zk / fac1;
      t2[k] = zk / fac2;
      zk *= -z;
      fac1 *= (k + 2);
      fac2 *= (k + 3);
    }
    for (int k = 29; k >= 0; --k) {
      s1 += t1[k];
      s2 += t2[k];
    }
    p1 = s1;
    p2 = s2;
  } else {
    const double em1 = std::expm1(-z);
    p1 = -em1 / z;
    p2 = (em1 + z) / (z * z);
  }
}

template <typename T> class Stepper : public PlanBase {
 public:
  using C = typename Cplx<T>::type;

  Stepper(const etd_params& P, cudaStream_t s, const TileOpt& t = TileOpt{}) : P_(P), st_(s) {
    tune_zb_ = t.zb;
    tune_kb_ = t.kb;
    tune_direct_ = t.direct;
    try {
      init();
    } catch (...) {
      release();
      throw;
    }
  }
  ~Stepper() override {
    for (auto& e : ev_) cudaEventDestroy(e);
    release();
  }

  // ------------------------------------------------------------------ public operations
  void step(void* phi, void* u, int nsteps, etd_diag* last) override {
    if (nsteps < 0) throw Error(ETD_EINVAL, "nsteps < 0");
    if (!u) throw Error(ETD_EINVAL, "u is NULL");
    if (P_.model == ETD_MODEL_COUPLED) {
      if (!phi) throw Error(ETD_EINVAL, "coupled model needs phi");
      run_coupled(static_cast<T*>(phi), static_cast<T*>(u), nsteps);
    } else if (P_.model == ETD_MODEL_FIXED_SQRTG) {
      run_sqrtg(static_cast<const T*>(phi), static_cast<T*>(u), nsteps);
    } else {
      run_fixed(static_cast<const T*>(phi), static_cast<T*>(u), nsteps);
    }
    if (last) {
      std::memset(last, 0, sizeof(*last));
      ETD_CUDA(cudaMemsetAsync(flag_, 0, sizeof(int), st_));
      launch_check(static_cast<T*>(u));
      if (phi && P_.model == ETD_MODEL_COUPLED) launch_check(static_cast<T*>(phi));
      ETD_CUDA(cudaStreamSynchronize(st_));
      ETD_CUDA(cudaGetLastError());
      int h[3];
      ETD_CUDA(cudaMemcpy(h, status_, sizeof(int), cudaMemcpyDeviceToHost));
      ETD_CUDA(cudaMemcpy(h + 1, flag_, sizeof(int), cudaMemcpyDeviceToHost));
      ETD_CUDA(cudaMemcpy(h + 2, count_, sizeof(int), cudaMemcpyDeviceToHost));
      double sc[S_COUNT];
      ETD_CUDA(cudaMemcpy(sc, scal_, sizeof(sc), cudaMemcpyDeviceToHost));
      int it = 0;
      double rs = 0;
      ETD_CUDA(cudaMemcpy(&it, cg_iters_, sizeof(int), cudaMemcpyDeviceToHost));
      ETD_CUDA(cudaMemcpy(&rs, cg_resid_, sizeof(double), cudaMemcpyDeviceToHost));
      last->band_size = h[2];
      last->cg_iters_last = it;
      last->cg_resid_last = rs;
      last->volume = hvol_ * sc[S_VOL];
      last->mass = hvol_ * sc[S_MASS];
      last->krylov_dim_last = kry_dim_max_;
      if (h[1]) throw Error(ETD_ENONFINITE, "non-finite value in the state");
      check_status(h[0]);
    }
  }

  void energy(const void* phi, const void* u, etd_diag* out) override {
    if (!u || !out) throw Error(ETD_EINVAL, "u/out is NULL");
    const T* ph = static_cast<const T*>(phi);
    if (!ph) {
      if (!fixed_ready_) throw Error(ETD_EINVAL, "energy needs phi");
      ph = phiA_;
    }
    const T* U = static_cast<const T*>(u);
    T* Ge = gx_;
    T* xe = gy_;
    launch_grid(k_gloc<T>, g_.n, ph, Ge);
    compute_band(ph);
    band_dirty_ = true;
    cg_setup(Ge);
    ETD_CUDA(cudaMemsetAsync(xe, 0, sizeof(T) * g_.n, st_));
    cg_solve(RhsGF<T>{Ge, U}, xe);
    ETD_CUDA(cudaMemsetAsync(scal_ + S_GRAD, 0, sizeof(double) * 5, st_));
    double init[3] = {0.0, 1e300, -1e300};
    ETD_CUDA(cudaMemcpyAsync(scal_ + S_MAXB, init, sizeof(init), cudaMemcpyHostToDevice, st_));
    k_energy_terms<T><<<grid_for(g_.n), 256, 0, st_>>>(g_, mc_, Ge, U, ph, scal_);
    k_band_dot<T><<<nsm_ * 4, 256, 0, st_>>>(idx_, count_, xe, RhsGF<T>{Ge, U}, scal_ + S_NONLOC);
    ETD_CUDA(cudaGetLastError());
    ETD_CUDA(cudaStreamSynchronize(st_));
    double sc[S_COUNT];
    ETD_CUDA(cudaMemcpy(sc, scal_, sizeof(sc), cudaMemcpyDeviceToHost));
    int h[2];
    ETD_CUDA(cudaMemcpy(h, status_, sizeof(int), cudaMemcpyDeviceToHost));
    ETD_CUDA(cudaMemcpy(h + 1, count_, sizeof(int), cudaMemcpyDeviceToHost));
    std::memset(out, 0, sizeof(*out));
    const double mass = hvol_ * sc[S_MASSF];
    out->energy = 0.5 * P_.eps_u * hvol_ * sc[S_GRAD] + hvol_ * sc[S_WELL] / P_.eps_u +
                  0.5 * P_.gamma * hvol_ * sc[S_NONLOC] + 0.5 * P_.M * mass * mass;
    out->mass = mass;
    out->max_bound = sc[S_MAXB];
    out->umin = sc[S_UMIN];
    out->umax = sc[S_UMAX];
    out->volume = hvol_ * sc[S_VOLE];
    out->band_size = h[1];
    int it = 0;
    double rs = 0;
    ETD_CUDA(cudaMemcpy(&it, cg_iters_, sizeof(int), cudaMemcpyDeviceToHost));
    ETD_CUDA(cudaMemcpy(&rs, cg_resid_, sizeof(double), cudaMemcpyDeviceToHost));
    out->cg_iters_last = it;
    out->cg_resid_last = rs;
    check_status(h[0]);
  }

  void fft_forward(const void* field, void* half) override {
    fwd(ProLoad<T>{static_cast<const T*>(field)}, I_[0]);
    OpToStd<T> op{0, static_cast<C*>(half), g_.ny, g_.nxh};
    passb(op, I_[0], nullptr, outs({}));
    sync_check();
  }

  void fft_inverse(const void* half, void* field) override {
    OpFromStd<T> op{1, static_cast<const C*>(half), g_.ny, g_.nxh, sk_.inv_n};
    passb(op, nullptr, nullptr, outs({I_[0]}));
    inv(I_[0], EpiStore<T>{static_cast<T*>(field)});
    sync_check();
  }

  long band(const void* phi, int* idx) override {
    compute_band(static_cast<const T*>(phi));
    band_dirty_ = true;
    int cnt = 0;
    ETD_CUDA(cudaMemcpyAsync(&cnt, count_, sizeof(int), cudaMemcpyDeviceToHost, st_));
    ETD_CUDA(cudaStreamSynchronize(st_));
    if (cnt) ETD_CUDA(cudaMemcpyAsync(idx, idx_, sizeof(int) * cnt, cudaMemcpyDeviceToDevice, st_));
    sync_check();
    return cnt;
  }

  void nonlocal(const void* phi, const void* f, void* w, int* iters, double* resid) override {
    T* Ge = gx_;
    T* xe = static_cast<T*>(w);
    launch_grid(k_gloc<T>, g_.n, static_cast<const T*>(phi), Ge);
    compute_band(static_cast<const T*>(phi));
    band_dirty_ = true;
    cg_setup(Ge);
    // the solution is defined on the band only
    k_zero_off_band<<<grid_for(g_.n), 256, 0, st_>>>(g_.n, mask_, (void*)xe, (int)sizeof(T));
    cg_solve(RhsField<T>{static_cast<const T*>(f)}, xe);
    int it = 0;
    double rs = 0;
    ETD_CUDA(cudaMemcpyAsync(&it, cg_iters_, sizeof(int), cudaMemcpyDeviceToHost, st_));
    ETD_CUDA(cudaMemcpyAsync(&rs, cg_resid_, sizeof(double), cudaMemcpyDeviceToHost, st_));
    sync_check();
    if (iters) *iters = it;
    if (resid) *resid = rs;
  }

  void remainder(int which, const void* phi_, const void* phio_, const void* u_, void* out_) override {
    const T* phi = static_cast<const T*>(phi_);
    const T* U = static_cast<const T*>(u_);
    T* out = static_cast<T*>(out_);
    band_dirty_ = true;
    w_reset_ = true;
    if (which == 1) {
      ETD_CUDA(cudaMemsetAsync(scal_ + S_VOL, 0, sizeof(double), st_));
      launch_reduce(0, phi, nullptr, scal_ + S_VOL);
      set_a0_if_needed();
      forward_store(phi, sS_);
      derivs(sS_);
      phi_terms(phi, U);
      // Delta(W' - A1 phi) spectrally, then R1 = rest + kappa/(mu eps^2) Delta(W' - A1 phi)
      forward_store(wm_, sS_);
      OpDeriv<T> op{1, {1, 0, 0, 0, 0}, sS_, sk_};
      passb(op, nullptr, nullptr, outs({I_[0]}));
      inv(I_[0], EpiStore<T>{wm_});
      const T c = (T)(P_.kappa / (P_.mu * P_.eps_phi * P_.eps_phi));
      launch_grid(k_axpy<T>, g_.n, (const T*)rr_, c, (const T*)wm_, out);
    } else if (which == 2) {
      if (P_.model != ETD_MODEL_COUPLED) throw Error(ETD_EINVAL, "which = 2 needs a coupled plan");
      T* Ge = G_;
      launch_grid(k_gloc<T>, g_.n, phi, Ge);
      compute_band(phi);
      cg_setup(Ge);
      ETD_CUDA(cudaMemsetAsync(scal_ + S_MASS, 0, sizeof(double), st_));
      launch_reduce(1, U, Ge, scal_ + S_MASS);
      ETD_CUDA(cudaMemsetAsync(w_, 0, sizeof(T) * g_.n, st_));
      cg_solve(RhsGU<T>{Ge, U, P_.ubar}, w_);
      k_r2_coupled<T><<<grid_for(g_.n), 256, 0, st_>>>(g_, mc_, phi, static_cast<const T*>(phio_), U, w_, scal_,
                                                        hvol_, out);
    } else if (which == 3) {
      T* Ge = G_;
      launch_grid(k_gloc<T>, g_.n, phi, Ge);
      compute_band(phi);
      cg_setup(Ge);
      ETD_CUDA(cudaMemsetAsync(scal_ + S_MASS, 0, sizeof(double), st_));
      launch_reduce(2, U, Ge, scal_ + S_MASS);
      ETD_CUDA(cudaMemsetAsync(w_, 0, sizeof(T) * g_.n, st_));
      cg_solve(RhsGF<T>{Ge, U}, w_);
      k_r2_fixed<T><<<grid_for(g_.n), 256, 0, st_>>>(g_, mc_, Ge, mask_, U, w_, scal_, hvol_, out);
      fixed_ready_ = false;
    } else {
      throw Error(ETD_EINVAL, "which must be 1, 2 or 3");
    }
    sync_check();
  }

 private:
  // ------------------------------------------------------------------ set-up
  void init() {
    const int nx = P_.n[0], ny = P_.n[1], nz = P_.dim == 2 ? 1 : P_.n[2];
    int dev = 0;
    ETD_CUDA(cudaGetDevice(&dev));
    ETD_CUDA(cudaDeviceGetAttribute(&nsm_, cudaDevAttrMultiProcessorCount, dev));
    int optin = 0;
    ETD_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    g_.dim = P_.dim;
    g_.nx = nx;
    g_.ny = ny;
    g_.nz = nz;
    g_.nxh = nx / 2 + 1;
    g_.lx = 0;
    while ((1 << g_.lx) < nx) ++g_.lx;
    g_.ly = 0;
    while ((1 << g_.ly) < ny) ++g_.ly;
    auto is_pow2 = [](int v) { return (v & (v - 1)) == 0; };
    g_.pow2 = is_pow2(nx) && is_pow2(ny) && is_pow2(nz);
    g_.n = (long long)nx * ny * nz;
    g_.nhat = (long long)g_.nxh * ny * nz;
    g_.hx = 2.0 * P_.half_len[0] / nx;
    g_.hy = 2.0 * P_.half_len[1] / ny;
    g_.hz = P_.dim == 2 ? 1.0 : 2.0 * P_.half_len[2] / nz;
    hvol_ = g_.hx * g_.hy * (P_.dim == 2 ? 1.0 : g_.hz);
    if (!g_.pow2 && sizeof(T) == 4 && P_.model == ETD_MODEL_COUPLED)
      throw Error(ETD_EINVAL, "96-point axes are not supported by the FP32-mixed coupled form");
    if (!choose_tiles(g_, sizeof(C), smemA_, smemB1_, tune_zb_, tune_kb_))
      throw Error(ETD_EINVAL, "grid not supported by the two-pass FFT tiles");
    if ((size_t)optin < smemA_ || (size_t)optin < 2 * smemB1_) throw Error(ETD_EINVAL, "not enough shared memory");

    // model constants in the working precision
    mc_.eps_phi = (T)P_.eps_phi;
    mc_.eps_u = (T)P_.eps_u;
    mc_.mu = (T)P_.mu;
    mc_.lambda_surf = (T)P_.lambda_surf;
    mc_.kappa = (T)P_.kappa;
    mc_.lambda_line = (T)P_.lambda_line;
    mc_.M_area = (T)P_.M_area;
    mc_.alpha = (T)P_.alpha;
    mc_.u0 = (T)P_.u0;
    mc_.gamma = (T)P_.gamma;
    mc_.M = (T)P_.M;
    mc_.ubar = (T)P_.ubar;
    mc_.A1 = (T)P_.A1;
    mc_.A2 = (T)P_.A2;
    mc_.B1 = (T)P_.B1;
    mc_.B2 = (T)P_.B2;
    mc_.band_hi = (T)P_.band_mask_hi;
    mc_.delta = (T)P_.recover_delta;
    mc_.tau = (T)P_.tau;
    ub_ = split_ubar<T>(P_.ubar);
    const double h[3] = {g_.hx, g_.hy, g_.hz};
    for (int d = 0; d < 3; ++d) {
      mc_.ih2[d] = (T)(1.0 / (h[d] * h[d]));
      mc_.i2h[d] = (T)(0.5 / h[d]);
    }
    mc_.dim = P_.dim;
    mc_.linear_only = P_.linear_only;

    // limits of the bounded device waits; ETD_WAIT_BUDGET (clock cycles a grid barrier of the
    // band solve may wait) and ETD_WAIT_TRIES (polls of a pass-A tensor copy) lower them, so
    // that tests can make a wait run out and check the ETD_ETIMEOUT path
    if (const char* e = std::getenv("ETD_WAIT_BUDGET")) wait_budget_ = std::atoll(e);
    if (const char* e = std::getenv("ETD_WAIT_TRIES")) wait_tries_ = std::atoll(e);
    // shape of the band solve's multigrid cycle (tuning; every choice is a symmetric V-cycle,
    // so the preconditioned CG converges to the same tolerance): ETD_MG_LEVELS caps the levels,
    // ETD_MG_GRID_CELLS is the full-grid size from which a level runs grid-wide (else on one
    // block), ETD_MG_NU the smoothing sweeps per side (1 or 2), ETD_MG_CSWEEPS the Jacobi sweeps
    // on the coarsest level (even)
    if (const char* e = std::getenv("ETD_MG_LEVELS")) mg_maxlev_ = std::max(1, std::min(kMGMax, std::atoi(e)));
    if (const char* e = std::getenv("ETD_MG_GRID_CELLS")) mg_grid_cells_ = std::max(1LL, std::atoll(e));
    if (const char* e = std::getenv("ETD_MG_NU")) mg_nu_ = std::atoi(e) == 1 ? 1 : 2;
    if (const char* e = std::getenv("ETD_MG_CSWEEPS")) mg_csweeps_ = std::max(2, std::atoi(e) / 2 * 2);

    // side stream and fork/join events of the band set-up overlap
    ETD_CUDA(cudaStreamCreateWithFlags(&side_, cudaStreamNonBlocking));
    ETD_CUDA(cudaEventCreateWithFlags(&fork_ev_, cudaEventDisableTiming));
    ETD_CUDA(cudaEventCreateWithFlags(&join_ev_, cudaEventDisableTiming));

    // workspace
    for (int i = 0; i < 5; ++i) I_[i] = alloc<C>(g_.nhat);
    tma_setup();
    sphi_ = alloc<C>(g_.nhat);
    sS_ = alloc<C>(g_.nhat);
    sSu_ = alloc<C>(g_.nhat);
    T** reals[] = {&phiA_, &phiB_, &phit_, &lap_, &gx_, &gy_, &gz_, &rr_, &wm_, &r2_, &ut_, &G_, &w_,
                   &cg_.x, &cg_.r, &cg_.r1, &cg_.u, &cg_.p, &cg_.q, &cg_.idg};
    for (T** r : reals) *r = alloc<T>(g_.n);
    for (T** r : reals) ETD_CUDA(cudaMemset(*r, 0, sizeof(T) * g_.n));
    cg_.cap = (int)g_.n;
    cg_.c = alloc<T>(6 * (size_t)g_.n);
    cg_.nb = alloc<int>(6 * (size_t)g_.n);
    cg_.c16 = sizeof(T) == 4 ? alloc<__half>(6 * (size_t)g_.n) : nullptr;
    bmap_ = alloc<int>(g_.n);
    cc_parent_ = alloc<int>(g_.n);
    cc_cid_ = alloc<int>(g_.n);
    cc_comp_ = alloc<int>(g_.n);
    ncomp_ = alloc<int>(2);   // component count, fallback flag of the labelling
    ETD_CUDA(cudaMemset(ncomp_, 0, 2 * sizeof(int)));
    ccL_ = alloc<int>(kCCCoarse);
    csize_ = alloc<double>(kCompCap);
    csum_ = alloc<double>(2 * kCompCap);
    for (T*& h : hs_) {
      h = alloc<T>(g_.n);
      ETD_CUDA(cudaMemset(h, 0, sizeof(T) * g_.n));
    }
    init_multigrid();
    mask_ = alloc<unsigned char>(g_.n);
    idx_ = alloc<int>(g_.n);
    idx_old_ = alloc<int>(g_.n);
    nblk_ = (int)((g_.n + kCompactBlock - 1) / kCompactBlock);
    bcount_ = alloc<int>(nblk_);
    count_ = alloc<int>(1);
    count_old_ = alloc<int>(1);
    ETD_CUDA(cudaMemset(count_, 0, sizeof(int)));
    ETD_CUDA(cudaMemset(count_old_, 0, sizeof(int)));
    scal_ = alloc<double>(S_COUNT);
    ETD_CUDA(cudaMemset(scal_, 0, sizeof(double) * S_COUNT));
    acc_ = alloc<double>(16);
    bar_ = alloc<unsigned>(2);
    status_ = alloc<int>(1);
    flag_ = alloc<int>(1);
    cg_iters_ = alloc<int>(1);
    cg_resid_ = alloc<double>(1);
    cg_work_ = alloc<unsigned long long>(2);
    ETD_CUDA(cudaMemset(cg_work_, 0, 2 * sizeof(unsigned long long)));
    ETD_CUDA(cudaMemset(status_, 0, sizeof(int)));
    ETD_CUDA(cudaMemset(cg_iters_, 0, sizeof(int)));
    ETD_CUDA(cudaMemset(cg_resid_, 0, sizeof(double)));

    // twiddle tables w_N^e = exp(-2 pi i e / N) and the phi-function table, built in FP64
    twx_ = upload_twiddles(nx);
    twy_ = upload_twiddles(ny);
    twz_ = upload_twiddles(nz);
    if constexpr (sizeof(T) == 4) {
      if (P_.model == ETD_MODEL_COUPLED && g_.nz > 1) init_df(optin);
    }
    const double ks = M_PI / P_.half_len[0];
    const int mmax = (nx / 2) * (nx / 2) + (ny / 2) * (ny / 2) + (nz / 2) * (nz / 2);
    std::vector<T> tab(4 * (size_t)(mmax + 1), (T)0), tabu(4 * (size_t)(mmax + 1), (T)0);
    const double e2 = P_.eps_phi * P_.eps_phi;
    for (int m = 0; m <= mmax; ++m) {
      const double lam = -ks * ks * m;
      const double lphi = P_.kappa / P_.mu * lam * lam -
                          (P_.kappa * (P_.A1 + P_.A2) + P_.lambda_surf * e2) / (P_.mu * e2) * lam +
                          (P_.kappa * P_.A1 * P_.A2 + P_.lambda_surf * P_.A1 * e2) / (P_.mu * e2 * e2);
      const double lu = P_.B2 - P_.eps_u * P_.B1 * lam;
      double a0, a1, a2, b0, b1, b2;
      phi_functions(P_.tau * lphi, a0, a1, a2);
      phi_functions(P_.tau * lu, b0, b1, b2);
      T* t = tab.data() + 4 * (size_t)m;
      t[0] = (T)a0;
      t[1] = (T)(P_.tau * a1);
      t[2] = (T)(P_.tau * a2);
      t[3] = (T)std::expm1(-P_.tau * lphi);  // phi0 - 1 (the FP32 form's increments of phi^)
      T* tu = tabu.data() + 4 * (size_t)m;
      tu[0] = (T)std::expm1(-P_.tau * lu);  // phi0 - 1: the u-stage is advanced as an increment
      tu[1] = (T)(P_.tau * b1);
      tu[2] = (T)(P_.tau * b2);
    }
    tab_ = alloc<T>(tab.size());
    tabu_ = alloc<T>(tabu.size());
    ETD_CUDA(cudaMemcpy(tab_, tab.data(), sizeof(T) * tab.size(), cudaMemcpyHostToDevice));
    ETD_CUDA(cudaMemcpy(tabu_, tabu.data(), sizeof(T) * tabu.size(), cudaMemcpyHostToDevice));
    sk_.tab = tab_;
    sk_.tabu = tabu_;
    sk_.inv_n = (T)(1.0 / (double)g_.n);
    sk_.kscale = (T)ks;
    sk_.ksq = (T)(ks * ks);
    c_lap_ = (T)(P_.kappa / (P_.mu * e2));
    a0_set_ = !std::isnan(P_.A0);
    if (a0_set_) {
      double a0 = P_.A0;
      ETD_CUDA(cudaMemcpy(scal_ + S_A0, &a0, sizeof(double), cudaMemcpyHostToDevice));
    }
    ETD_CUDA(cudaDeviceSynchronize());
  }

  template <typename E = T> typename Cplx<E>::type* upload_twiddles(int n) {
    using CE = typename Cplx<E>::type;
    std::vector<CE> t(n);
    for (int e = 0; e < n; ++e) {
      const long double a = 2.0L * 3.14159265358979323846264338327950288L * e / n;
      t[e].x = E((double)cosl(a));
      t[e].y = E((double)(-sinl(a)));
    }
    CE* d = alloc<CE>(n);
    ETD_CUDA(cudaMemcpy(d, t.data(), sizeof(CE) * n, cudaMemcpyHostToDevice));
    return d;
  }

  // Double-float membrane state of the FP32-mixed coupled form: the carried phi spectrum
  // (dcomplex, plan layout), the low part of the real-space phi, the intermediate and
  // twiddles of the double-float forward transform, and the tile geometry of 16-byte complex
  // elements.
  void init_df(int optin) {
    gd_ = g_;
    if (!choose_tiles(gd_, sizeof(dcomplex), smemAd_, smemB1d_))
      throw Error(ETD_EINVAL, "grid not supported by the double-float FFT tiles");
    if ((size_t)optin < smemAd_ || (size_t)optin < 2 * smemB1d_) throw Error(ETD_EINVAL, "not enough shared memory");
    sphi_d_ = alloc<dcomplex>(g_.nhat);
    Id_ = alloc<dcomplex>(g_.nhat);
    philo_ = alloc<T>(g_.n);
    twx_d_ = upload_twiddles<dfloat>(g_.nx);
    twy_d_ = upload_twiddles<dfloat>(g_.ny);
    twz_d_ = upload_twiddles<dfloat>(g_.nz);
    dfphi_ = true;
  }

  template <typename U> U* alloc(size_t count) {
    void* p = nullptr;
    ETD_CUDA(cudaMalloc(&p, sizeof(U) * std::max<size_t>(count, 1)));
    allocs_.push_back(p);
    return static_cast<U*>(p);
  }

  void release() {
    for (void* p : allocs_) cudaFree(p);
    allocs_.clear();
    if (kry_mem_) cudaFree(kry_mem_);
    kry_mem_ = nullptr;
    kry_cap_ = 0;
    if (fork_ev_) cudaEventDestroy(fork_ev_);
    if (join_ev_) cudaEventDestroy(join_ev_);
    if (side_) cudaStreamDestroy(side_);
    fork_ev_ = join_ev_ = nullptr;
    side_ = nullptr;
  }

  // Work that depends only on phi^{n+1} and G (the band set-up) runs on a second stream
  // while the plan stream does the reductions and the forward transform of G u^n.
  template <typename F> void on_side_stream(F&& work) {
    ETD_CUDA(cudaEventRecord(fork_ev_, st_));
    ETD_CUDA(cudaStreamWaitEvent(side_, fork_ev_, 0));
    cudaStream_t main = st_;
    st_ = side_;
    try {
      work();
    } catch (...) {
      st_ = main;
      throw;
    }
    st_ = main;
    ETD_CUDA(cudaEventRecord(join_ev_, side_));
  }
  void join_side_stream() { ETD_CUDA(cudaStreamWaitEvent(st_, join_ev_, 0)); }

  // Two independent groups of launches, the first on the plan stream and the second on the
  // side stream: the last wave of one kernel overlaps the other's instead of idling SMs.
  template <typename A, typename B> void concurrently(A&& on_main, B&& on_side) {
    on_side_stream(on_side);
    on_main();
    join_side_stream();
  }

  // ------------------------------------------------------------------ launch helpers
  int grid_for(long long n) const {
    const long long b = (n + 255) / 256;
    return (int)std::max<long long>(1, std::min<long long>(b, (long long)nsm_ * 16));
  }

  template <typename K, typename... A> void launch_grid(K k, long long n, A... a) {
    k<<<grid_for(n), 256, 0, st_>>>(n, a...);
    ETD_CUDA(cudaGetLastError());
  }

  void launch_reduce(int mode, const T* a, const T* G, double* dst) {
    timed(ETD_K_REDUCE, (mode == 0 ? 1 : 2) * fld(), [&] {
      k_reduce<T><<<grid_for(g_.n), 256, 0, st_>>>(g_.n, mode, a, G, P_.ubar, dst);
    });
    ETD_CUDA(cudaGetLastError());
  }

  void launch_check(T* a) {
    k_check_finite<T><<<grid_for(g_.n), 256, 0, st_>>>(g_.n, a, flag_);
    ETD_CUDA(cudaGetLastError());
  }

  static int pro_reads(const ProLoad<T>&) { return 1; }
  static int pro_reads(const ProMul<T>&) { return 2; }
  static int epi_fields(const EpiStore<T>&) { return 1; }
  static int epi_fields(const EpiRecover<T>&) { return 3; }
  static int epi_fields(const EpiPhiG<T>& e) { return e.zero ? 3 : 2; }
  static int epi_fields(const EpiStoreVol<T>&) { return 1; }
  static int epi_fields(const EpiRecoverMass<T>&) { return 3; }
  static int epi_fields(const EpiPhiGVol<T>& e) { return e.zero ? 3 : 2; }
  static int epi_fields(const EpiPhiIncVol& e) { return e.zero ? 6 : 5; }  // phi^n hi, lo read; hi, lo, G (, R2) written

  // Kernel of the axis-length family (fft_family): 96-point axes have instantiations of their own.
  template <typename Pro> auto fwd_kernel() const {
    return fft_family(g_.nx) == 1 ? passA_fwd<T, Pro, 1> : passA_fwd<T, Pro, 0>;
  }
  template <typename Epi> auto inv_kernel() const {
    return fft_family(g_.nx) == 1 ? passA_inv<T, Epi, 1> : passA_inv<T, Epi, 0>;
  }
  template <typename Op> auto passb_kernel() const {
    return fft_family(g_.nz) == 1 ? passB<T, Op, 1> : passB<T, Op, 0>;
  }

  template <typename Pro> void fwd(Pro pro, C* out) {
    auto k = fwd_kernel<Pro>();
    // tile, then (staged store) the leftover-column buffer after the barrier slot
    const size_t smem = tma_bar_off_ + 16 + (size_t)ETD_PASSA_THREADS * sizeof(C);
    set_smem((const void*)k, smem);
    PassAIn pout{0, tma_box_, (int)tma_bar_off_, status_, wait_tries_};
    const CUtensorMap* map = tma_for(out, pout);
    timed(ETD_K_FFT_A_FWD, pro_reads(pro) * fld() + spc(), [&] {
      k<<<(g_.nz / g_.ZB) * g_.Y1, ETD_PASSA_THREADS, smem, st_>>>(g_, pro, out, twx_, twy_, *map, pout);
    });
    ETD_CUDA(cudaGetLastError());
  }

  // The tensor map of an intermediate buffer (and pin.tma = 1), or the unused empty map.
  const CUtensorMap* tma_for(const C* buf, PassAIn& pin) const {
    for (int i = 0; i < 5 && tma_ok_; ++i)
      if (buf == I_[i]) {
        pin.tma = 1;
        return &tma_map_[i];
      }
    return &tma_none_;
  }

  template <typename Epi> void inv(const C* in, Epi epi) {
    auto k = inv_kernel<Epi>();
    const size_t smem = tma_bar_off_ + 16;
    set_smem((const void*)k, smem);
    PassAIn pin{0, tma_box_, (int)tma_bar_off_, status_, wait_tries_};
    const CUtensorMap* map = tma_for(in, pin);
    timed(ETD_K_FFT_A_INV, spc() + epi_fields(epi) * fld(), [&] {
      k<<<(g_.nz / g_.ZB) * g_.Y1, ETD_PASSA_THREADS, smem, st_>>>(g_, in, epi, twx_, twy_, *map, pin);
    });
    ETD_CUDA(cudaGetLastError());
  }

  // Double-float transforms (direct pass-A loads and stores; geometry gd_).
  double dspc() const { return 2.0 * spc(); }
  template <typename Pro> void fwd_d(Pro pro, dcomplex* out) {
    auto k = passA_fwd<dfloat, Pro>;
    set_smem((const void*)k, smemAd_);
    PassAIn p{0, 0, 0, status_, wait_tries_};
    timed(ETD_K_FFT_A_FWD, fld() + dspc(), [&] {
      k<<<(gd_.nz / gd_.ZB) * gd_.Y1, ETD_PASSA_THREADS, smemAd_, st_>>>(gd_, pro, out, twx_d_, twy_d_, tma_none_, p);
    });
    ETD_CUDA(cudaGetLastError());
  }
  template <typename Op> void passb_d(const Op& op, const dcomplex* in0, dcomplex* out0, int nspec) {
    auto k = passB<dfloat, Op>;
    const size_t smemB = smemB1d_;
    set_smem((const void*)k, smemB);
    OutP<dcomplex> o;
    for (int i = 0; i < 5; ++i) o.p[i] = nullptr;
    o.p[0] = out0;
    const int nkb = (gd_.nxh + gd_.KB - 1) / gd_.KB;
    timed(ETD_K_FFT_B, nspec * dspc(), [&] {
      k<<<nkb * gd_.Y2, ETD_PASSB_THREADS, smemB, st_>>>(gd_, op, in0, nullptr, o, twy_d_, twz_d_);
    });
    ETD_CUDA(cudaGetLastError());
  }
  // phi^ = FFT(phi) in double-float into the carried spectrum.
  void forward_store_d(const T* field) {
    if constexpr (sizeof(T) == 4) {
      fwd_d(ProWiden{field}, Id_);
      OpStore<dfloat> op{0, sphi_d_};
      passb_d(op, Id_, nullptr, 3);  // intermediate read, spectrum written (both double-float) + its read
    }
  }
  // Tensor maps of the intermediates I_[0..4] for pass A's staged intermediate: 4-D
  // (2 Nz scalars, Y1, Nx/2+1, Y2), box (2 ZB, 1, Nx/2+1, Y2).  Used when the grid is 3D, the
  // box fits the pass-A tile, its rows are 16-byte multiples and every column of the box
  // can be read into registers in one round plus a short leftover (passA_cols_inv_staged);
  // otherwise, or if the driver does not provide the encoder, pass A loads directly.
  void tma_setup() {
    tma_bar_off_ = (smemA_ + 15) / 16 * 16;
    std::memset(&tma_none_, 0, sizeof(tma_none_));
    tma_ok_ = false;
    // ETD_PASSA_DIRECT=1 keeps the direct loads and stores (the two forms are compared in tests)
    const char* direct = std::getenv("ETD_PASSA_DIRECT");
    if ((direct && direct[0] == '1') || tune_direct_) return;
    const int nt = ETD_PASSA_THREADS, ncols = g_.ZB * g_.nxh;
    const size_t box = (size_t)2 * g_.ZB * g_.nxh * g_.Y2 * sizeof(T);
    const bool shape = g_.nz > 1 && g_.nxh <= 256 && g_.Y2 <= 256 && (2 * g_.ZB * sizeof(T)) % 16 == 0 &&
                       box <= smemA_ && (ncols <= nt || (ncols <= 2 * nt && (ncols - nt) * g_.Y2 <= nt));
    if (!shape) return;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return;
    }
    auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    const cuuint64_t dims[4] = {(cuuint64_t)2 * g_.nz, (cuuint64_t)g_.Y1, (cuuint64_t)g_.nxh, (cuuint64_t)g_.Y2};
    const cuuint64_t strides[3] = {(cuuint64_t)2 * g_.nz * sizeof(T), (cuuint64_t)2 * g_.nz * g_.Y1 * sizeof(T),
                                   (cuuint64_t)2 * g_.nz * g_.Y1 * g_.nxh * sizeof(T)};
    const cuuint32_t boxd[4] = {(cuuint32_t)(2 * g_.ZB), 1u, (cuuint32_t)g_.nxh, (cuuint32_t)g_.Y2};
    const cuuint32_t es[4] = {1u, 1u, 1u, 1u};
    for (int i = 0; i < 5; ++i) {
      const CUresult r = encode(&tma_map_[i], sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                                4, (void*)I_[i], dims, strides, boxd, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return;
    }
    tma_box_ = (uint32_t)box;
    tma_ok_ = true;
  }

  static OutP<C> outs(std::initializer_list<C*> l) {
    OutP<C> o;
    for (int i = 0; i < 5; ++i) o.p[i] = nullptr;
    int i = 0;
    for (C* c : l) o.p[i++] = c;
    return o;
  }

  // stored-spectrum traffic of each spectral operator (reads + writes of plan spectra)
  static int op_extra(const OpStore<T>&) { return 1; }
  static int op_extra(const OpDeriv<T>&) { return 1; }
  static int op_extra(const OpPhiPred<T>&) { return 2; }  // phi^ read; S (RK2) or phi~^ (ETD1) written
  static int op_extra(const OpPhiCorr<T>&) { return 2; }
  static int op_extra(const OpPhiPredInc& o) { return o.rk2 ? 3 : 4; }  // phi^ (double-float) read; S' or phi^ written
  static int op_extra(const OpPhiCorrInc&) { return 5; }  // S' read, phi^ read and written (double-float)
  static int op_extra(const OpDeriv<T, dcomplex>&) { return 2; }
  static int op_extra(const OpUPred<T>& o) { return o.rk2 ? 1 : 0; }
  static int op_extra(const OpUCorr<T>&) { return 1; }
  static int op_extra(const OpToStd<T>&) { return 1; }
  static int op_extra(const OpFromStd<T>&) { return 1; }

  template <typename Op> void passb(const Op& op, const C* in0, const C* in1, OutP<C> o) {
    auto k = passb_kernel<Op>();
    const size_t smemB = (Op::NI >= 2 || op.nout >= 2 ? 2 : 1) * smemB1_;  // two tiles: inputs, alternating outputs
    set_smem((const void*)k, smemB);
    const int nkb = (g_.nxh + g_.KB - 1) / g_.KB;
    timed(ETD_K_FFT_B, (Op::NI + op.nout + op_extra(op)) * spc(), [&] {
      k<<<nkb * g_.Y2, ETD_PASSB_THREADS, smemB, st_>>>(g_, op, in0, in1, o, twy_, twz_);
    });
    ETD_CUDA(cudaGetLastError());
  }

  void set_smem(const void* k, size_t bytes) {
    if (bytes > 48 * 1024) ETD_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  }

  void sync_check() {
    ETD_CUDA(cudaGetLastError());
    ETD_CUDA(cudaStreamSynchronize(st_));
    int s = 0;
    ETD_CUDA(cudaMemcpy(&s, status_, sizeof(int), cudaMemcpyDeviceToHost));
    check_status(s);
  }

  void check_status(int s) {
    if (s == 0) return;
    ETD_CUDA(cudaMemset(status_, 0, sizeof(int)));
    if (s == 5) throw Error(ETD_ENOTCONV, "band CG did not reach cg_rtol within cg_maxit iterations");
    if (s == 6) throw Error(ETD_ETIMEOUT, "a grid barrier of the band CG or the Lanczos process timed out");
    if (s == 7) throw Error(ETD_ETIMEOUT, "a tensor copy of the FFT pass A did not complete");
    if (s == 8) throw Error(ETD_EINVAL, "the band has more connected components than the band solve supports (4096)");
    throw Error(ETD_ECUDA, "device status word set");
  }

  // ------------------------------------------------------------------ building blocks
  // Narrow band of phi: mask, ascending index list, count (device).  The previous list
  // is kept in idx_old_ so the solution can be cleared on nodes that left the band.
  void compute_band(const T* phi) {
    cg_grid_ = 0;  // a new band: the solve's grid is the default until a frozen band sizes it
    std::swap(idx_, idx_old_);
    std::swap(count_, count_old_);
    if (g_.n % 4 == 0 && (reinterpret_cast<uintptr_t>(phi) & 15) == 0) {
      const int nb4 = (int)((g_.n + kCompactWide - 1) / kCompactWide);
      timed(ETD_K_BAND, fld() + (double)g_.n, [&] {
        k_band_count4<T><<<nb4, kCompactBlock, 0, st_>>>(g_.n, phi, mc_.band_hi, mask_, bcount_);
      });
      timed(ETD_K_BAND, 8.0 * nb4, [&] { k_band_scan<<<1, 1024, 0, st_>>>(nb4, bcount_, count_); });
      timed(ETD_K_BAND, (double)g_.n, [&] {
        k_band_scatter4<<<nb4, kCompactBlock, 0, st_>>>(g_.n, mask_, bcount_, idx_, bmap_);
      });
      ETD_CUDA(cudaGetLastError());
      return;
    }
    timed(ETD_K_BAND, fld() + (double)g_.n, [&] {
      k_band_count<T><<<nblk_, kCompactBlock, 0, st_>>>(g_.n, phi, mc_.band_hi, mask_, bcount_);
    });
    timed(ETD_K_BAND, 8.0 * nblk_, [&] { k_band_scan<<<1, 1024, 0, st_>>>(nblk_, bcount_, count_); });
    timed(ETD_K_BAND, (double)g_.n, [&] {
      k_band_scatter<<<nblk_, kCompactBlock, 0, st_>>>(g_.n, mask_, bcount_, idx_, bmap_);
    });
    ETD_CUDA(cudaGetLastError());
  }

  void cg_setup(const T* G) {
    CGVec<T> v = cg_;
    timed(ETD_K_BAND, 0.0, [&] { k_cg_setup<T><<<nsm_ * 8, 256, 0, st_>>>(g_, mc_, idx_, count_, mask_, bmap_, G, v); });
    mg_setup();
    label_components();
    ETD_CUDA(cudaGetLastError());
  }

  // Connected components of the band (their count, each node's component, their sizes): from
  // the multigrid hierarchy when every aggregate is connected inside its cell, else by the
  // union-find over the band (both enqueued; the one not needed returns at once).
  void label_components() {
    CGVec<T> v = cg_;
    CCLevels lv{};
    lv.nlev = mg_nlev_;
    lv.is3d = g_.nz > 1;
    for (int l = 0; l < mg_nlev_; ++l) {
      const HostLevel& H = lv_[l];
      CCLevel& C = lv.L[l];
      C.cap = H.cap;
      C.agg = H.agg;
      C.cnt = l == 0 ? count_ : H.cnt;
      C.nb = l == 0 ? cg_.nb : H.nb;
      C.child = l == 0 ? nullptr : H.child;
    }
    timed(ETD_K_BAND, 0.0, [&] {
      ETD_CUDA(cudaMemsetAsync(ncomp_, 0, 2 * sizeof(int), st_));   // count, fallback flag
      ETD_CUDA(cudaMemsetAsync(csize_, 0, sizeof(double) * kCompCap, st_));
      int* fb = ncomp_ + 1;
      if (mg_nlev_ > 1) k_cc_check<<<nsm_ * 2, 256, 0, st_>>>(lv, fb);
      k_cc_coarsest<<<1, kCCCoarse, 0, st_>>>(lv, ccL_, ncomp_, fb);
      k_cc_down<<<nsm_ * 4, 256, 0, st_>>>(lv, ccL_, ncomp_, cc_comp_, csize_, fb);
      k_cc_init<T><<<nsm_ * 4, 256, 0, st_>>>(count_, v, cc_parent_, fb);
      k_cc_link<T><<<nsm_ * 4, 256, 0, st_>>>(count_, v, cc_parent_, status_, fb);
      k_cc_roots<<<nsm_ * 4, 256, 0, st_>>>(count_, cc_parent_, cc_cid_, ncomp_, fb);
      k_cc_label<<<nsm_ * 4, 256, 0, st_>>>(count_, cc_parent_, cc_cid_, ncomp_, cc_comp_, csize_, status_, fb);
    });
  }

  // Initial guesses of the band solves of a step.  With P_n, C_n the predictor- and
  // corrector-stage solutions of step n, the guesses are
  //   predictor of step n+1:  C_n + (P_n - C_{n-1})     corrector:  P_{n+1} + (C_n - P_n)
  // (one stage per step: 2 P_n - P_{n-1}); each is off by O(tau^2) where the previous
  // solution alone is off by O(tau).  Three full-grid slots hold the history; the solve
  // writes its solution into the slot of the oldest entry.  Without history the guess is the
  // previous solution (the band values of w_).
  CGGuess<T> next_guess(bool corrector, bool rk2) {
    CGGuess<T> gs{w_, nullptr, nullptr, (T)0, (T)0, nullptr};
    int out = hO_;
    if (out < 0)
      for (int k = 0; k < 3; ++k)
        if (k != hP_ && k != hC_) {
          out = k;
          break;
        }
    if (!corrector) {
      if (rk2 && hC_ >= 0 && hP_ >= 0 && hO_ >= 0) {
        gs = {hs_[hC_], hs_[hP_], hs_[hO_], (T)1, (T)-1, nullptr};
      } else if (!rk2 && hP_ >= 0 && hO_ >= 0) {
        gs = {hs_[hP_], hs_[hP_], hs_[hO_], (T)1, (T)-1, nullptr};
      } else if (rk2 && hC_ >= 0) {
        gs.a = hs_[hC_];
      } else if (hP_ >= 0) {
        gs.a = hs_[hP_];
      }
      hO_ = hP_;
      hP_ = out;
    } else {
      if (hO_ >= 0 && hC_ >= 0) gs = {hs_[hP_], hs_[hC_], hs_[hO_], (T)1, (T)-1, nullptr};
      else if (hP_ >= 0) gs.a = hs_[hP_];
      hO_ = hC_;
      hC_ = out;
    }
    gs.hist = hs_[out];
    return gs;
  }

  template <typename Rhs> void cg_solve(Rhs rhs, T* x, CGGuess<T> gs = CGGuess<T>{}, double rtol = 0.0) {
    if (!gs.a) gs.a = x;
    CGVec<T> v = cg_;
    CGCtl c;
    c.acc = acc_;
    c.bar = bar_;
    c.status = status_;
    c.iters = cg_iters_;
    c.resid = cg_resid_;
    c.rtol = rtol > 0.0 ? rtol : P_.cg_rtol;
    c.maxit = P_.cg_maxit;
    c.budget = wait_budget_;
    c.work = cg_work_;
    c.ncomp = ncomp_;
    c.comp = cc_comp_;
    c.csize = csize_;
    c.csum = csum_;
    ETD_CUDA(cudaMemsetAsync(csum_, 0, sizeof(double) * 2 * kCompCap, st_));
    ETD_CUDA(cudaMemsetAsync(acc_, 0, sizeof(double) * 16, st_));
    ETD_CUDA(cudaMemsetAsync(bar_, 0, sizeof(unsigned) * 2, st_));
    auto k = k_cg<T, Rhs>;
    int per = 0;
    ETD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, 1024, 0));
    if (per < 1) throw Error(ETD_ECUDA, "band CG kernel cannot be resident");
    const int grid = cg_grid_ > 0 ? cg_grid_ : nsm_;
    const int* idx = idx_;
    const int* cnt = count_;
    T* wfull = x;
    MGP<T> mg = mgp();
    void* args[] = {&idx, &cnt, &v, &wfull, &rhs, &c, &mg, &gs};
    timed(ETD_K_CG, 0.0, [&] { ETD_CUDA(cudaLaunchCooperativeKernel((const void*)k, grid, 1024, args, 0, st_)); });
  }

  // Level l coarsens the grid 2x per axis l times (z only in 3D) while every coarsened
  // extent stays >= 4; levels whose full grid has >= 2^15 cells run on the whole GPU in the
  // V-cycle, smaller ones on one block.  The cycle is V(2,2) with a degree-2 Chebyshev pair of
  // Jacobi weights, the coarse-grid correction over-corrected by 1.9 (piecewise-constant
  // aggregation under-estimates it) and 2 sweeps on the coarsest level.
  void init_multigrid() {
    HostLevel& L0 = lv_[0];
    L0.ext = Ext{g_.nx, g_.ny, g_.nz};
    L0.cap = (int)g_.n;
    L0.agg = alloc<int>(g_.n);
    L0.e = alloc<T>(g_.n);
    L0.t = alloc<T>(g_.n);
    ETD_CUDA(cudaMemset(L0.e, 0, sizeof(T) * g_.n));
    ETD_CUDA(cudaMemset(L0.t, 0, sizeof(T) * g_.n));
    mg_nlev_ = 1;
    const bool is3d = g_.nz > 1;
    while (mg_nlev_ < mg_maxlev_) {
      const HostLevel& F = lv_[mg_nlev_ - 1];
      // coarsen while every extent is even and at least 8
      auto ok = [](int v) { return v >= 8 && v % 2 == 0; };
      if (!ok(F.ext.x) || !ok(F.ext.y) || (is3d && !ok(F.ext.z))) break;
      HostLevel& L = lv_[mg_nlev_];
      L.ext = Ext{F.ext.x / 2, F.ext.y / 2, is3d ? F.ext.z / 2 : 1};
      L.cap = L.ext.x * L.ext.y * L.ext.z;
      L.nblk = (L.cap + kCompactBlock - 1) / kCompactBlock;
      L.cnt = alloc<int>(1);
      L.list = alloc<int>(L.cap);
      L.map = alloc<int>(L.cap);
      L.bcount = alloc<int>(L.nblk);
      L.mark = alloc<unsigned char>(L.cap);
      L.c = alloc<T>(6 * (size_t)L.cap);
      L.nb = alloc<int>(6 * (size_t)L.cap);
      L.idg = alloc<T>(L.cap);
      L.agg = alloc<int>(L.cap);
      L.child = alloc<int>(8 * (size_t)L.cap);
      L.b = alloc<T>(L.cap);
      L.e = alloc<T>(L.cap);
      L.o = alloc<T>(L.cap);
      L.t = alloc<T>(L.cap);
      ETD_CUDA(cudaMemset(L.cnt, 0, sizeof(int)));
      ++mg_nlev_;
    }
    mg_gl_ = 1;
    while (mg_gl_ < mg_nlev_ && lv_[mg_gl_].cap >= mg_grid_cells_) ++mg_gl_;
  }

  // Coarse levels for the current band (level 0 = idx_, count_, mask_, bmap_, cg_).  Levels
  // whose full grid has more than 2^15 cells use grid-wide kernels; the rest are built by
  // one single-block launch (they are too small to fill the GPU, and launch gaps dominate).
  void mg_setup() {
    const int is3d = g_.nz > 1;
    int l = 1;
    for (; l < mg_nlev_ && lv_[l].cap > (1 << 15); ++l) {
      HostLevel& L = lv_[l];
      const HostLevel& F = lv_[l - 1];
      const int* flist = l == 1 ? idx_ : F.list;
      const int* fcnt = l == 1 ? count_ : F.cnt;
      const unsigned char* fmark = l == 1 ? mask_ : F.mark;
      const int* fmap = l == 1 ? bmap_ : F.map;
      const T* fc = l == 1 ? cg_.c : F.c;
      int* fagg = lv_[l - 1].agg;
      timed(ETD_K_BAND, 0.0, [&] {
        ETD_CUDA(cudaMemsetAsync(L.mark, 0, L.cap, st_));
        k_mg_mark<<<nsm_ * 4, 256, 0, st_>>>(flist, fcnt, F.ext, is3d, L.ext, L.mark);
        if (L.cap % 4 == 0) {  // levels here have at least 2^15 cells, x extent even
          const int nb4 = (int)(((long long)L.cap + kCompactWide - 1) / kCompactWide);
          k_mask_count4<<<nb4, kCompactBlock, 0, st_>>>(L.cap, L.mark, L.bcount);
          k_band_scan<<<1, 1024, 0, st_>>>(nb4, L.bcount, L.cnt);
          k_band_scatter4<<<nb4, kCompactBlock, 0, st_>>>(L.cap, L.mark, L.bcount, L.list, L.map);
        } else {
          k_mask_count<<<L.nblk, kCompactBlock, 0, st_>>>(L.cap, L.mark, L.bcount);
          k_band_scan<<<1, 1024, 0, st_>>>(L.nblk, L.bcount, L.cnt);
          k_band_scatter<<<L.nblk, kCompactBlock, 0, st_>>>(L.cap, L.mark, L.bcount, L.list, L.map);
        }
        k_mg_parent<<<nsm_ * 4, 256, 0, st_>>>(flist, fcnt, F.ext, is3d, L.ext, L.map, fagg);
        k_mg_coarse<T><<<nsm_ * 4, 256, 0, st_>>>(L.list, L.cnt, L.ext, is3d, fmark, fmap, F.ext, fc,
                                                  F.cap, L.map, L.c, L.nb, L.idg, L.child, L.cap);
      });
      ETD_CUDA(cudaGetLastError());
    }
    if (l < mg_nlev_) {
      MGSetTail<T> a{};
      a.first = l;
      a.nlev = mg_nlev_;
      a.is3d = is3d;
      for (int k = 0; k < mg_nlev_; ++k) {
        const HostLevel& H = lv_[k];
        MGSetLevel<T>& S = a.L[k];
        S.e = H.ext;
        S.cap = H.cap;
        S.agg = H.agg;
        if (k == 0) {
          S.cnt = count_;
          S.list = idx_;
          S.map = bmap_;
          S.mark = mask_;
          S.c = cg_.c;
          S.nb = cg_.nb;
          S.idg = cg_.idg;
          S.child = nullptr;
        } else {
          S.cnt = H.cnt;
          S.list = H.list;
          S.map = H.map;
          S.mark = H.mark;
          S.c = H.c;
          S.nb = H.nb;
          S.idg = H.idg;
          S.child = H.child;
        }
      }
      timed(ETD_K_BAND, 0.0, [&] { k_mg_setup_tail<T><<<1, 1024, 0, st_>>>(a); });
      ETD_CUDA(cudaGetLastError());
    }
  }

  MGP<T> mgp() const {
    MGP<T> m{};
    m.nlev = mg_nlev_;
    m.gl = mg_gl_;
    m.csweeps = mg_csweeps_;
    m.nu = mg_nu_;
    // degree-2 Chebyshev weights for D^-1 A on [lmax / 4, lmax], lmax = 2 (Gershgorin bound
    // for the Jacobi-scaled graph Laplacian): w_i = 1 / (c + r cos((2 i + 1) pi / 4))
    {
      const double lmax = 2.0, lmin = lmax / 4.0, cth = 0.5 * (lmax + lmin), rad = 0.5 * (lmax - lmin);
      const double cq = std::sqrt(0.5);
      m.w1 = (T)(1.0 / (cth + rad * cq));
      m.w2 = (T)(1.0 / (cth - rad * cq));
    }
    m.alpha = (T)1.9;
    m.c16 = cg_.c16;
    for (int l = 0; l < mg_nlev_; ++l) {
      const HostLevel& H = lv_[l];
      MGL<T>& L = m.L[l];
      L.cap = H.cap;
      L.agg = H.agg;
      L.e = H.e;
      L.t = H.t;
      if (l == 0) {
        L.cnt = count_;
        L.list = idx_;
        L.c = cg_.c;
        L.nb = cg_.nb;
        L.idg = cg_.idg;
        L.child = nullptr;
        L.b = cg_.r;
        L.o = cg_.u;
      } else {
        L.cnt = H.cnt;
        L.list = H.list;
        L.c = H.c;
        L.nb = H.nb;
        L.idg = H.idg;
        L.child = H.child;
        L.b = H.b;
        L.o = H.o;
      }
    }
    return m;
  }

  void set_a0_if_needed() {
    if (a0_set_) return;
    k_set_a0<<<1, 1, 0, st_>>>(scal_, hvol_);
    ETD_CUDA(cudaGetLastError());
    a0_set_ = true;
  }

  void forward_store(const T* field, C* spec) {
    fwd(ProLoad<T>{field}, I_[0]);
    OpStore<T> op{0, spec};
    passb(op, I_[0], nullptr, outs({}));
  }

  // Delta phi and grad phi of the stored spectrum into lap_, gx_, gy_, gz_.
  template <typename S> void derivs(const S* spec) {
    const int nd = g_.nz > 1 ? 4 : 3;
    OpDeriv<T, S> op{nd, {1, 2, 3, 4, 0}, spec, sk_};
    passb(op, nullptr, nullptr, outs({I_[0], I_[1], I_[2], I_[3]}));
    concurrently(
        [&] {
          inv(I_[0], EpiStore<T>{lap_});
          inv(I_[2], EpiStore<T>{gy_});
        },
        [&] {
          inv(I_[1], EpiStore<T>{gx_});
          if (nd == 4) inv(I_[3], EpiStore<T>{gz_});
        });
  }

  // R1 parts at (phi, u): rr_ = R1 without the Laplacian term, wm_ = W'(phi) - A1 phi.
  void phi_terms(const T* phi, const T* u) {
    timed(ETD_K_POINTWISE, (g_.nz > 1 ? 8 : 7) * fld(), [&] {
      k_r1<T><<<grid_for(g_.n), 256, 0, st_>>>(g_, mc_, phi, lap_, gx_, gy_, gz_, u, scal_, hvol_, rr_, wm_);
    });
    ETD_CUDA(cudaGetLastError());
  }

  void band_for_solve(const T* phi, const T* G) {
    compute_band(phi);
    if (w_reset_) {
      ETD_CUDA(cudaMemsetAsync(w_, 0, sizeof(T) * g_.n, st_));
      hP_ = hC_ = hO_ = -1;
      w_reset_ = false;
    } else {
      k_zero_left<<<nsm_ * 4, 256, 0, st_>>>(idx_old_, count_old_, mask_, (void*)w_, (int)sizeof(T));
    }
    cg_setup(G);
  }

  // ------------------------------------------------------------------ the coupled step
  void run_coupled(T* phi, T* u, int nsteps) {
    const bool rk2 = P_.scheme == ETD_ETDRK2;
    ETD_CUDA(cudaMemcpyAsync(phiA_, phi, sizeof(T) * g_.n, cudaMemcpyDeviceToDevice, st_));
    T* cur = phiA_;
    T* nxt = phiB_;
    if (dfphi_) {
      ETD_CUDA(cudaMemsetAsync(philo_, 0, sizeof(T) * g_.n, st_));
      forward_store_d(cur);
    } else {
      forward_store(cur, sphi_);
    }
    ETD_CUDA(cudaMemsetAsync(scal_ + S_VOL, 0, sizeof(double), st_));
    launch_reduce(0, cur, nullptr, scal_ + S_VOL);
    set_a0_if_needed();
    const int nd = g_.nz > 1 ? 4 : 3;
    for (int n = 0; n < nsteps; ++n) {
      // phi-stage predictor: R1(phi^n, u^n)
      if constexpr (sizeof(T) == 4) {
        if (dfphi_) derivs(sphi_d_);
        else derivs(sphi_);
      } else {
        derivs(sphi_);
      }
      phi_terms(cur, u);
      concurrently([&] { fwd(ProLoad<T>{rr_}, I_[0]); }, [&] { fwd(ProLoad<T>{wm_}, I_[1]); });
      if (rk2) {
        if constexpr (sizeof(T) == 4) {
          if (dfphi_) {
            OpPhiPredInc pred{1 + nd, {0, 1, 2, 3, 4}, sphi_d_, sS_, 1, c_lap_, sk_};
            passb(pred, I_[0], I_[1], outs({I_[0], I_[1], I_[2], I_[3], I_[4]}));
          }
        }
        if (!dfphi_) {
          OpPhiPred<T> pred{1 + nd, {0, 1, 2, 3, 4}, sphi_, sS_, 1, c_lap_, sk_};
          passb(pred, I_[0], I_[1], outs({I_[0], I_[1], I_[2], I_[3], I_[4]}));
        }
        concurrently(
            [&] {
              ETD_CUDA(cudaMemsetAsync(scal_ + S_VOL, 0, sizeof(double), st_));
              inv(I_[0], EpiStoreVol<T>{phit_, scal_ + S_VOL});
              inv(I_[2], EpiStore<T>{gx_});
            },
            [&] {
              inv(I_[1], EpiStore<T>{lap_});
              inv(I_[3], EpiStore<T>{gy_});
              if (nd == 4) inv(I_[4], EpiStore<T>{gz_});
            });
        phi_terms(phit_, u);  // R1(phi~, u^n): u frozen at u^n in the corrector (Sec. 3.3)
        concurrently([&] { fwd(ProLoad<T>{rr_}, I_[0]); }, [&] { fwd(ProLoad<T>{wm_}, I_[1]); });
        if constexpr (sizeof(T) == 4) {
          if (dfphi_) {
            OpPhiCorrInc corr{1, sphi_d_, sS_, c_lap_, sk_};
            passb(corr, I_[0], I_[1], outs({I_[0]}));
          }
        }
        if (!dfphi_) {
          OpPhiCorr<T> corr{1, sphi_, sS_, c_lap_, sk_};
          passb(corr, I_[0], I_[1], outs({I_[0]}));
        }
      } else if (dfphi_) {
        if constexpr (sizeof(T) == 4) {
          OpPhiPredInc pred{1, {0, 0, 0, 0, 0}, sphi_d_, sS_, 0, c_lap_, sk_};
          passb(pred, I_[0], I_[1], outs({I_[0]}));
        }
      } else {
        OpPhiPred<T> pred{1, {0, 0, 0, 0, 0}, sphi_, sS_, 0, c_lap_, sk_};
        passb(pred, I_[0], I_[1], outs({I_[0]}));
      }
      ETD_CUDA(cudaMemsetAsync(scal_ + S_VOL, 0, sizeof(double) * 2, st_));  // S_VOL, S_MASS
      if constexpr (sizeof(T) == 4) {
        if (dfphi_) inv(I_[0], EpiPhiIncVol{cur, philo_, nxt, G_, r2_, scal_ + S_VOL});
      }
      if (!dfphi_) inv(I_[0], EpiPhiGVol<T>{nxt, G_, r2_, scal_ + S_VOL});
      // u-stage: new g times old u (Sec. 3.3)
      on_side_stream([&] { band_for_solve(nxt, G_); });
      launch_reduce(1, u, G_, scal_ + S_MASS);
      fwd(ProMul<T>{G_, u}, I_[0]);
      join_side_stream();
      cg_solve(RhsGU<T>{G_, u, P_.ubar}, w_, next_guess(false, rk2), rk2 ? P_.cg_rtol_pred : 0.0);
      timed(ETD_K_POINTWISE, 0.0, [&] {  // bytes from the band-node counter
        k_r2_coupled_band<T><<<nsm_ * 8, 256, 0, st_>>>(g_, mc_, idx_, count_, nxt, cur, u, w_, scal_, hvol_, r2_,
                                                         cg_work_ + 1);
      });
      fwd(ProLoad<T>{r2_}, I_[1]);
      OpUPred<T> upred{1, sSu_, rk2 ? 1 : 0, sk_};
      passb(upred, I_[0], I_[1], outs({I_[0]}));
      if (rk2) {
        ETD_CUDA(cudaMemsetAsync(scal_ + S_MASS, 0, sizeof(double), st_));
        inv(I_[0], EpiRecoverMass<T>{ut_, G_, u, mc_.delta, ub_, scal_ + S_MASS});
        cg_solve(RhsGU<T>{G_, ut_, P_.ubar}, w_, next_guess(true, rk2));
        timed(ETD_K_POINTWISE, 0.0, [&] {
          k_r2_coupled_band<T><<<nsm_ * 8, 256, 0, st_>>>(g_, mc_, idx_, count_, nxt, cur, ut_, w_, scal_, hvol_, r2_,
                                                           cg_work_ + 1);
        });
        fwd(ProLoad<T>{r2_}, I_[0]);
        OpUCorr<T> ucorr{1, sSu_, sk_};
        passb(ucorr, I_[0], nullptr, outs({I_[0]}));
      }
      inv(I_[0], EpiRecover<T>{u, G_, u, mc_.delta});
      std::swap(cur, nxt);
    }
    ETD_CUDA(cudaMemcpyAsync(phi, cur, sizeof(T) * g_.n, cudaMemcpyDeviceToDevice, st_));
    ETD_CUDA(cudaGetLastError());
  }

  // ------------------------------------------------------------------ the fixed step
  // Fixed membrane: G = g(phi) and the band come from the phi of the first call (or of a
  // later call that passes one).  Returns true when they were (re)built.
  bool freeze_membrane(const T* phi) {
    if (phi) {
      ETD_CUDA(cudaMemcpyAsync(phiA_, phi, sizeof(T) * g_.n, cudaMemcpyDeviceToDevice, st_));
      fixed_ready_ = false;
    }
    if (fixed_ready_ && !band_dirty_) return false;
    if (!phi && !fixed_ready_) throw Error(ETD_EINVAL, "fixed model: the first call must pass phi");
    launch_grid(k_gloc<T>, g_.n, (const T*)phiA_, G_);
    band_for_solve(phiA_, G_);
    fixed_ready_ = true;
    // the frozen band's size sets the band solve's grid: about 2048 nodes per block of 1024
    // threads, so that small bands leave SMs to concurrent work (one read, once per membrane)
    int cnt = 0;
    ETD_CUDA(cudaMemcpyAsync(&cnt, count_, sizeof(int), cudaMemcpyDeviceToHost, st_));
    ETD_CUDA(cudaStreamSynchronize(st_));
    fixed_count_ = cnt;
    cg_grid_ = std::max(1, std::min(nsm_, (cnt + 2047) / 2048));
    band_dirty_ = false;
    return true;
  }

  void run_fixed(const T* phi, T* u, int nsteps) {
    const bool rk2 = P_.scheme == ETD_ETDRK2;
    freeze_membrane(phi);
    for (int n = 0; n < nsteps; ++n) {
      ETD_CUDA(cudaMemsetAsync(scal_ + S_MASS, 0, sizeof(double), st_));
      launch_reduce(2, u, G_, scal_ + S_MASS);
      cg_solve(RhsGF<T>{G_, u}, w_, next_guess(false, rk2), rk2 ? P_.cg_rtol_pred : 0.0);
      k_r2_fixed<T><<<grid_for(g_.n), 256, 0, st_>>>(g_, mc_, G_, mask_, u, w_, scal_, hvol_, r2_);
      fwd(ProMul<T>{G_, u}, I_[0]);
      fwd(ProLoad<T>{r2_}, I_[1]);
      OpUPred<T> upred{1, sSu_, rk2 ? 1 : 0, sk_};
      passb(upred, I_[0], I_[1], outs({I_[0]}));
      if (rk2) {
        inv(I_[0], EpiRecover<T>{ut_, G_, u, mc_.delta});
        ETD_CUDA(cudaMemsetAsync(scal_ + S_MASS, 0, sizeof(double), st_));
        launch_reduce(2, ut_, G_, scal_ + S_MASS);
        cg_solve(RhsGF<T>{G_, ut_}, w_, next_guess(true, rk2));
        k_r2_fixed<T><<<grid_for(g_.n), 256, 0, st_>>>(g_, mc_, G_, mask_, ut_, w_, scal_, hvol_, r2_);
        fwd(ProLoad<T>{r2_}, I_[0]);
        OpUCorr<T> ucorr{1, sSu_, sk_};
        passb(ucorr, I_[0], nullptr, outs({I_[0]}));
      }
      inv(I_[0], EpiRecover<T>{u, G_, u, mc_.delta});
    }
    ETD_CUDA(cudaGetLastError());
  }

  // ---- the g^{1/2}-split scheme of Sec. 2.2 (model ETD_MODEL_FIXED_SQRTG) -------------
  // Krylov workspace for the frozen band of fixed_count_ nodes: the Lanczos basis
  // (kKrylovMax + 1 vectors), w, R0, b, V~, g^{1/2}, g^{-1/2} (compact) and FP64 scalars.
  void krylov_setup() {
    const long long M = std::max(fixed_count_, 1);
    if (M > kry_cap_) {
      if (kry_mem_) ETD_CUDA(cudaFree(kry_mem_));
      kry_mem_ = nullptr;
      kry_cap_ = 0;
      const size_t ld = (size_t)((M + 31) / 32 * 32);
      const size_t vec = sizeof(T) * ld;
      const size_t bytes = vec * (kKrylovMax + 1 + 6) + sizeof(double) * (5 * kKrylovMax + 1);
      if (cudaMalloc(&kry_mem_, bytes) != cudaSuccess) {
        cudaGetLastError();
        kry_mem_ = nullptr;
        throw Error(ETD_ENOMEM, "Krylov workspace does not fit");
      }
      char* q = static_cast<char*>(kry_mem_);
      kV_ = reinterpret_cast<T*>(q);
      q += vec * (kKrylovMax + 1);
      T** v[] = {&kw_, &kR0_, &kb_, &kVt_, &ksg_, &kisg_};
      for (T** x : v) {
        *x = reinterpret_cast<T*>(q);
        q += vec;
      }
      double* d = reinterpret_cast<double*>(q);
      kal_ = d;
      kbe_ = d + kKrylovMax;
      kacc_ = d + 2 * kKrylovMax;
      ky_ = d + 4 * kKrylovMax;
      knrm_ = d + 5 * kKrylovMax;
      kld_ = (int)ld;
      kry_cap_ = M;
    }
    timed(ETD_K_BAND, 3.0 * sizeof(T) * fixed_count_, [&] {
      k_sec2_sqrtg<T><<<grid_for(fixed_count_), 256, 0, st_>>>(idx_, count_, G_, ksg_, kisg_);
    });
    ETD_CUDA(cudaGetLastError());
  }

  KrylovOp<T> kop() const { return KrylovOp<T>{cg_, kisg_, (T)P_.B2, (T)P_.eps_u}; }

  // Lanczos steps j0 .. j1-1 in one cooperative launch.
  void lanczos(int j0, int j1) {
    KrylovOp<T> op = kop();
    CGCtl c{};
    c.acc = kacc_;
    c.bar = bar_;
    c.status = status_;
    c.budget = wait_budget_;
    ETD_CUDA(cudaMemsetAsync(bar_, 0, sizeof(unsigned) * 2, st_));
    auto k = k_lanczos<T>;
    int per = 0;
    ETD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, 1024, 0));
    if (per < 1) throw Error(ETD_ECUDA, "Lanczos kernel cannot be resident");
    const int grid = cg_grid_ > 0 ? cg_grid_ : nsm_;
    const int* cnt = count_;
    T* V = kV_;
    int ld = kld_;
    T* w = kw_;
    double *al = kal_, *be = kbe_, *acc = kacc_;
    void* args[] = {&cnt, &op, &V, &ld, &w, &al, &be, &acc, &j0, &j1, &c};
    const double bytes = (double)fixed_count_ * (j1 - j0) * (15.0 * sizeof(T) + 24.0);
    timed(ETD_K_KRYLOV, bytes, [&] {
      ETD_CUDA(cudaLaunchCooperativeKernel((const void*)k, grid, 1024, args, 0, st_));
    });
  }

  // tau phi_j(tau L) x for the compact vector x: the Lanczos process from x / |x| grown in
  // chunks of kKrylovChunk steps until the estimated error of the omitted term,
  // |x| beta_m tau |e_m^T phi_{j+1}(tau T_m) e_1|, is below krylov_tol relative to the result
  // (or the process breaks down: an invariant subspace).  Leaves the combination weights
  // tau |x| phi_j(tau T_m) e_1 in ky_ and returns m (0 when x = 0).
  int krylov_phi(int j, const T* x) {
    const int nb = grid_for(fixed_count_);
    ETD_CUDA(cudaMemsetAsync(knrm_, 0, sizeof(double), st_));
    timed(ETD_K_KRYLOV, (double)sizeof(T) * fixed_count_,
          [&] { k_band_norm2<T><<<nb, 256, 0, st_>>>(count_, x, knrm_); });
    double n2 = 0.0;
    ETD_CUDA(cudaMemcpyAsync(&n2, knrm_, sizeof(double), cudaMemcpyDeviceToHost, st_));
    ETD_CUDA(cudaStreamSynchronize(st_));
    if (!std::isfinite(n2)) throw Error(ETD_ENONFINITE, "non-finite value in a Krylov start vector");
    if (n2 == 0.0) return 0;
    const double beta0 = std::sqrt(n2);
    timed(ETD_K_KRYLOV, 2.0 * sizeof(T) * fixed_count_,
          [&] { k_band_normalise<T><<<nb, 256, 0, st_>>>(count_, x, knrm_, kV_); });
    ETD_CUDA(cudaMemsetAsync(kacc_, 0, sizeof(double) * 2 * kKrylovMax, st_));
    const double tol = P_.krylov_tol > 0 ? P_.krylov_tol : (sizeof(T) == 8 ? 1e-12 : 1e-6);
    double ha[kKrylovMax], hb[kKrylovMax];
    std::vector<double> y;
    int m = 0, dim = 0;
    for (;;) {
      const int j1 = std::min(m + kKrylovChunk, kKrylovMax);
      lanczos(m, j1);
      ETD_CUDA(cudaMemcpyAsync(ha + m, kal_ + m, sizeof(double) * (j1 - m), cudaMemcpyDeviceToHost, st_));
      ETD_CUDA(cudaMemcpyAsync(hb + m, kbe_ + m, sizeof(double) * (j1 - m), cudaMemcpyDeviceToHost, st_));
      sync_check();
      dim = j1;
      bool invariant = false;
      for (int k = m; k < j1; ++k) {
        if (!std::isfinite(ha[k]) || !std::isfinite(hb[k]))
          throw Error(ETD_ENONFINITE, "non-finite Lanczos coefficient");
        if (!(hb[k] > 0.0)) {
          dim = k + 1;
          invariant = true;
          break;
        }
      }
      const double tail = krylov_coeffs(dim, ha, hb, P_.tau, j, y);
      double ny = 0.0;
      for (double v : y) ny += v * v;
      const double err = hb[dim - 1] * P_.tau * tail;
      if (invariant || err <= tol * std::sqrt(ny)) break;
      if (j1 == kKrylovMax)
        throw Error(ETD_ENOTCONV, "the Krylov space of phi_j(tau L) did not converge within 128 Lanczos steps");
      m = j1;
    }
    for (double& v : y) v *= P_.tau * beta0;
    ETD_CUDA(cudaMemcpyAsync(ky_, y.data(), sizeof(double) * dim, cudaMemcpyHostToDevice, st_));
    ETD_CUDA(cudaStreamSynchronize(st_));   // y is a host temporary
    kry_dim_max_ = std::max(kry_dim_max_, dim);
    return dim;
  }

  // One call of Sec. 2.2's scheme on the frozen band: per step the band solve of
  // (-Delta_S) w = g f(U) (and mass), R0 = R_phi(U), b = R0 - L V, V~ = V + tau phi_1(tau L) b;
  // ETDRK2 then the solve at U~, d = R_phi(U~) - R0 and V = V~ + tau phi_2(tau L) d.
  void run_sqrtg(const T* phi, T* u, int nsteps) {
    const bool rk2 = P_.scheme == ETD_ETDRK2;
    if (freeze_membrane(phi) || !kry_mem_) krylov_setup();
    if (rk2) ETD_CUDA(cudaMemcpyAsync(ut_, u, sizeof(T) * g_.n, cudaMemcpyDeviceToDevice, st_));
    const KrylovOp<T> op = kop();
    const int nb = grid_for(fixed_count_);
    const double M = (double)fixed_count_;
    kry_dim_max_ = 0;
    const bool nl = !P_.linear_only;   // the band solve and mass feed only the remainder
    for (int n = 0; n < nsteps; ++n) {
      if (nl) {
        ETD_CUDA(cudaMemsetAsync(scal_ + S_MASS, 0, sizeof(double), st_));
        launch_reduce(2, u, G_, scal_ + S_MASS);
        cg_solve(RhsGF<T>{G_, u}, w_, next_guess(false, rk2), rk2 ? P_.cg_rtol_pred : 0.0);
      }
      timed(ETD_K_POINTWISE, M * (11.0 * sizeof(T) + 32.0), [&] {
        k_sec2_first<T><<<nb, 256, 0, st_>>>(idx_, count_, mc_, op, ksg_, u, w_, scal_, hvol_, kR0_, kb_);
      });
      const int m1 = krylov_phi(1, kb_);
      timed(ETD_K_KRYLOV, M * ((m1 + 2.0 + (rk2 ? 1 : 0)) * sizeof(T) + 4.0), [&] {
        k_krylov_finish<T><<<nb, 256, 0, st_>>>(idx_, count_, kV_, kld_, ky_, m1, nullptr, ksg_, u,
                                                rk2 ? kVt_ : nullptr, rk2 ? ut_ : u);
      });
      if (!rk2) continue;
      if (nl) {
        ETD_CUDA(cudaMemsetAsync(scal_ + S_MASS, 0, sizeof(double), st_));
        launch_reduce(2, ut_, G_, scal_ + S_MASS);
        cg_solve(RhsGF<T>{G_, ut_}, w_, next_guess(true, rk2));
      }
      timed(ETD_K_POINTWISE, M * (5.0 * sizeof(T) + 4.0), [&] {
        k_sec2_second<T><<<nb, 256, 0, st_>>>(idx_, count_, mc_, ksg_, ut_, w_, scal_, hvol_, kR0_, kb_);
      });
      const int m2 = krylov_phi(2, kb_);
      timed(ETD_K_KRYLOV, M * ((m2 + 3.0) * sizeof(T) + 4.0), [&] {
        k_krylov_finish<T><<<nb, 256, 0, st_>>>(idx_, count_, kV_, kld_, ky_, m2, kVt_, ksg_, nullptr, nullptr, u);
      });
    }
    ETD_CUDA(cudaGetLastError());
  }

  // ------------------------------------------------------------------ timing
 public:
  double time_transforms(int reps) override {
    // forward: field -> spectrum (plan layout); inverse: spectrum -> field (identity multiplier)
    auto pair = [&] {
      forward_store(phiA_, sS_);
      OpDeriv<T> op{1, {0, 0, 0, 0, 0}, sS_, sk_};
      passb(op, nullptr, nullptr, outs({I_[0]}));
      inv(I_[0], EpiStore<T>{phiB_});
    };
    pair();
    cudaEvent_t a, b;
    ETD_CUDA(cudaEventCreate(&a));
    ETD_CUDA(cudaEventCreate(&b));
    ETD_CUDA(cudaEventRecord(a, st_));
    for (int r = 0; r < reps; ++r) pair();
    ETD_CUDA(cudaEventRecord(b, st_));
    ETD_CUDA(cudaEventSynchronize(b));
    float ms = 0;
    ETD_CUDA(cudaEventElapsedTime(&ms, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    sync_check();
    return ms / std::max(reps, 1);
  }

  void tiles(int* zb, int* kb, int* tma) const override {
    *zb = g_.ZB;
    *kb = g_.KB;
    *tma = tma_ok_ ? 1 : 0;
  }

  void timing(int enable) override {
    if (enable) {
      if (ev_.empty()) {
        ev_.resize(2 * kTimedMax);
        for (auto& e : ev_) ETD_CUDA(cudaEventCreate(&e));
      }
      ETD_CUDA(cudaStreamSynchronize(st_));
      recs_.clear();
      for (int k = 0; k < ETD_K_NKINDS; ++k) {
        t_ms_[k] = 0;
        t_bytes_[k] = 0;
        t_n_[k] = 0;
        t_timed_[k] = 0;
      }
      ETD_CUDA(cudaMemset(cg_work_, 0, 2 * sizeof(unsigned long long)));
    }
    timing_ = enable != 0;
  }

  void timing_read(int kind, double* ms, long* launches, double* bytes) override {
    ETD_CUDA(cudaStreamSynchronize(st_));
    for (const Rec& r : recs_) {
      float t = 0;
      ETD_CUDA(cudaEventElapsedTime(&t, ev_[2 * r.slot], ev_[2 * r.slot + 1]));
      t_ms_[r.kind] += t;
      ++t_timed_[r.kind];
    }
    recs_.clear();
    unsigned long long work = 0;
    unsigned long long works[2] = {0, 0};
    ETD_CUDA(cudaMemcpy(works, cg_work_, sizeof(works), cudaMemcpyDeviceToHost));
    work = works[0];
    *ms = t_ms_[kind];
    *launches = t_n_[kind];
    // band CG: 18 element accesses per band node and CG iteration (x, r, p, A p, three face
    // coefficients and six neighbour indices, read or written: 72 B in FP32) times the
    // measured iteration count, from the device work counter.  The multigrid V-cycle behind
    // each iteration moves several times that; the count is the plain-CG figure on purpose.
    *bytes = kind == ETD_K_CG ? 18.0 * sizeof(T) * (double)work : t_bytes_[kind];
    // band-list R2: phi^n, phi^old, u, w read and R2 written once per band node
    if (kind == ETD_K_POINTWISE) *bytes += 5.0 * sizeof(T) * (double)works[1];
  }

 private:
  static constexpr int kTimedMax = 16384;
  struct Rec {
    int slot, kind;
  };
  template <typename F> void timed(int kind, double bytes, F&& launch) {
    if (!timing_) {
      launch();
      return;
    }
    ++t_n_[kind];
    t_bytes_[kind] += bytes;
    const int slot = (int)(slot_next_ % kTimedMax);
    const bool rec = (int)recs_.size() < kTimedMax;
    if (rec) ETD_CUDA(cudaEventRecord(ev_[2 * slot], st_));
    launch();
    if (rec) {
      ETD_CUDA(cudaEventRecord(ev_[2 * slot + 1], st_));
      recs_.push_back(Rec{slot, kind});
      ++slot_next_;
    }
  }
  double fld() const { return (double)g_.n * sizeof(T); }        // one real field
  double spc() const { return (double)g_.nhat * sizeof(C); }     // one half spectrum
  bool timing_ = false;
  std::vector<cudaEvent_t> ev_;
  std::vector<Rec> recs_;
  size_t slot_next_ = 0;
  double t_ms_[ETD_K_NKINDS] = {}, t_bytes_[ETD_K_NKINDS] = {};
  long t_n_[ETD_K_NKINDS] = {}, t_timed_[ETD_K_NKINDS] = {};
  unsigned long long* cg_work_ = nullptr;

  // ------------------------------------------------------------------ state
  etd_params P_;
  cudaStream_t st_;
  cudaStream_t side_ = nullptr;
  cudaEvent_t fork_ev_ = nullptr, join_ev_ = nullptr;
  Geo g_{};
  ModelC<T> mc_{};
  Ubar<T> ub_{};
  SpecConst<T> sk_{};
  T c_lap_{};
  double hvol_ = 1.0;
  int nsm_ = 1;
  int tune_zb_ = 0, tune_kb_ = 0;           // requested pass-A z-planes / pass-B pencil blocks (0: default)
  int tune_direct_ = 0;                      // 1: direct pass-A loads/stores (no tensor-copy staging)
  int cg_grid_ = 0;                          // blocks of the band solve (0: one per SM)
  long long wait_budget_ = 4000000000LL;   // grid barrier: clock cycles before ETD_ETIMEOUT
  long long wait_tries_ = 1LL << 22;       // pass-A tensor copy: mbarrier polls before ETD_ETIMEOUT
  size_t smemA_ = 0, smemB1_ = 0;
  std::vector<void*> allocs_;
  C* I_[5] = {};
  CUtensorMap tma_map_[5];
  CUtensorMap tma_none_;
  bool tma_ok_ = false;
  uint32_t tma_box_ = 0;
  size_t tma_bar_off_ = 0;
  C *sphi_ = nullptr, *sS_ = nullptr, *sSu_ = nullptr;
  T *phiA_ = nullptr, *phiB_ = nullptr, *phit_ = nullptr, *lap_ = nullptr, *gx_ = nullptr, *gy_ = nullptr,
    *gz_ = nullptr, *rr_ = nullptr, *wm_ = nullptr, *r2_ = nullptr, *ut_ = nullptr, *G_ = nullptr,
    *w_ = nullptr;
  CGVec<T> cg_{};
  unsigned char* mask_ = nullptr;
  int* bmap_ = nullptr;
  // connected components of the band: union-find parents, root ids, node components, sizes
  int *cc_parent_ = nullptr, *cc_cid_ = nullptr, *cc_comp_ = nullptr, *ncomp_ = nullptr, *ccL_ = nullptr;
  double *csize_ = nullptr, *csum_ = nullptr;
  // multigrid hierarchy of the band solve (level 0 = the band itself)
  struct HostLevel {
    Ext ext{1, 1, 1};   // grid extents of the level
    int cap = 0, nblk = 0;
    int *cnt = nullptr, *list = nullptr, *map = nullptr, *bcount = nullptr;
    unsigned char* mark = nullptr;
    T *c = nullptr, *idg = nullptr, *b = nullptr, *e = nullptr, *o = nullptr, *t = nullptr;
    int *nb = nullptr, *agg = nullptr, *child = nullptr;
  };
  HostLevel lv_[kMGMax];
  int mg_nlev_ = 1, mg_gl_ = 1;
  int mg_maxlev_ = kMGMax, mg_nu_ = 2, mg_csweeps_ = 2;
  long long mg_grid_cells_ = 1LL << 15;
  int *idx_ = nullptr, *idx_old_ = nullptr, *bcount_ = nullptr, *count_ = nullptr, *count_old_ = nullptr;
  int nblk_ = 0;
  T* tab_ = nullptr;
  T* tabu_ = nullptr;
  C *twx_ = nullptr, *twy_ = nullptr, *twz_ = nullptr;
  double *scal_ = nullptr, *acc_ = nullptr, *cg_resid_ = nullptr;
  unsigned* bar_ = nullptr;
  int *status_ = nullptr, *flag_ = nullptr, *cg_iters_ = nullptr;
  bool a0_set_ = false, fixed_ready_ = false, band_dirty_ = false, w_reset_ = true;
  T* hs_[3] = {};                 // solution history of the band solves (full grid)
  // double-float membrane state (FP32-mixed coupled form)
  bool dfphi_ = false;
  Geo gd_{};
  size_t smemAd_ = 0, smemB1d_ = 0;
  dcomplex *sphi_d_ = nullptr, *Id_ = nullptr;
  dcomplex *twx_d_ = nullptr, *twy_d_ = nullptr, *twz_d_ = nullptr;
  T* philo_ = nullptr;
  int hP_ = -1, hC_ = -1, hO_ = -1;  // slots: last predictor, last corrector, the older entry
  // frozen band size and the Krylov workspace of the g^{1/2}-split scheme
  int fixed_count_ = 0;
  void* kry_mem_ = nullptr;
  long long kry_cap_ = 0;
  int kld_ = 0, kry_dim_max_ = 0;
  T *kV_ = nullptr, *kw_ = nullptr, *kR0_ = nullptr, *kb_ = nullptr, *kVt_ = nullptr, *ksg_ = nullptr, *kisg_ = nullptr;
  double *kal_ = nullptr, *kbe_ = nullptr, *kacc_ = nullptr, *ky_ = nullptr, *knrm_ = nullptr;
};

}  // namespace etd
