// etd_api.cu -- the extern "C" boundary declared in include/etd.h.  Validates arguments,
// dispatches to the precision-specific plan and turns exceptions into status codes.
#include <cmath>
#include <cstdio>
#include <string>
#include "plan.h"

struct etd_plan_s {
  etd::PlanBase* impl;
  etd_params params;
};

namespace {
thread_local std::string g_last_error;

etd_status fail(etd_status s, const std::string& m) {
  g_last_error = m;
  return s;
}

bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

etd_status validate(const etd_params& p) {
  if (p.dim != 2 && p.dim != 3) return fail(ETD_EINVAL, "dim must be 2 or 3");
  const int nz = p.dim == 2 ? 1 : p.n[2];
  if (p.dim == 2 && p.n[2] != 1) return fail(ETD_EINVAL, "2D plans need n[2] = 1");
  for (int d = 0; d < 2; ++d)
    if (!pow2(p.n[d]) || p.n[d] < 8 || p.n[d] > 256) return fail(ETD_EINVAL, "Nx, Ny must be powers of two in [8, 256]");
  if (p.dim == 3 && (!pow2(nz) || nz < 8 || nz > 256)) return fail(ETD_EINVAL, "Nz must be a power of two in [8, 256]");
  for (int d = 0; d < p.dim; ++d)
    if (!(p.half_len[d] > 0)) return fail(ETD_EINVAL, "half lengths must be positive");
  for (int d = 1; d < p.dim; ++d)
    if (std::fabs(p.half_len[d] - p.half_len[0]) > 1e-12 * p.half_len[0])
      return fail(ETD_EINVAL, "only cubic boxes (X = Y = Z) are supported");
  if (p.scheme != ETD_ETD1 && p.scheme != ETD_ETDRK2) return fail(ETD_EINVAL, "scheme must be ETD1 or ETDRK2");
  if (p.model != ETD_MODEL_FIXED && p.model != ETD_MODEL_COUPLED) return fail(ETD_EINVAL, "unknown model");
  if (p.model == ETD_MODEL_COUPLED && p.dim != 3) return fail(ETD_EINVAL, "the coupled model is 3D");
  if (p.precision != ETD_FP64 && p.precision != ETD_FP32_MIXED) return fail(ETD_EINVAL, "unknown precision");
  if (!(p.tau > 0) || !(p.eps_u > 0) || !(p.eps_phi > 0)) return fail(ETD_EINVAL, "tau and eps must be positive");
  if (p.model == ETD_MODEL_COUPLED && !(p.mu > 0)) return fail(ETD_EINVAL, "mu must be positive");
  if (!(p.band_mask_hi > 0) || !(p.band_mask_hi <= 1)) return fail(ETD_EINVAL, "band_mask_hi must be in (0, 1]");
  if (!(p.cg_rtol > 0) || p.cg_maxit < 1) return fail(ETD_EINVAL, "cg_rtol > 0 and cg_maxit >= 1 required");
  if (!(p.cg_rtol_pred >= 0)) return fail(ETD_EINVAL, "cg_rtol_pred >= 0 required");
  return ETD_OK;
}

template <typename F> etd_status guard(F&& f) {
  try {
    f();
    g_last_error.clear();
    return ETD_OK;
  } catch (const etd::Error& e) {
    return fail(e.code, e.what());
  } catch (const std::bad_alloc&) {
    return fail(ETD_ENOMEM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(ETD_ECUDA, e.what());
  } catch (...) {
    return fail(ETD_ECUDA, "unknown error");
  }
}
}  // namespace

namespace etd {
// Lets other translation units of the library report through etd_last_error().
void set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace etd

extern "C" {

etd_status etd_plan(const etd_params* params, void* cuda_stream, etd_plan_t* out) {
  if (!out) return fail(ETD_EINVAL, "out is NULL");
  *out = nullptr;
  if (!params) return fail(ETD_EINVAL, "params is NULL");
  etd_status s = validate(*params);
  if (s != ETD_OK) return s;
  etd_plan_s* h = nullptr;
  s = guard([&] {
    h = new etd_plan_s;
    h->params = *params;
    h->impl = nullptr;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    h->impl = params->precision == ETD_FP64 ? etd::make_plan_f64(*params, st) : etd::make_plan_f32(*params, st);
  });
  if (s != ETD_OK) {
    if (h) delete h;
    return s;
  }
  *out = h;
  return ETD_OK;
}

etd_status etd_step(etd_plan_t plan, void* phi, void* u, int nsteps, etd_diag* last) {
  if (!plan) return fail(ETD_EINVAL, "plan is NULL");
  return guard([&] { plan->impl->step(phi, u, nsteps, last); });
}

etd_status etd_energy(etd_plan_t plan, const void* phi, const void* u, etd_diag* out) {
  if (!plan) return fail(ETD_EINVAL, "plan is NULL");
  return guard([&] { plan->impl->energy(phi, u, out); });
}

etd_status etd_free(etd_plan_t plan) {
  if (!plan) return ETD_OK;
  delete plan->impl;
  delete plan;
  return ETD_OK;
}

const char* etd_last_error(void) { return g_last_error.c_str(); }

etd_status etd_fft_forward(etd_plan_t plan, const void* field, void* half) {
  if (!plan || !field || !half) return fail(ETD_EINVAL, "NULL argument");
  return guard([&] { plan->impl->fft_forward(field, half); });
}

etd_status etd_fft_inverse(etd_plan_t plan, const void* half, void* field) {
  if (!plan || !field || !half) return fail(ETD_EINVAL, "NULL argument");
  return guard([&] { plan->impl->fft_inverse(half, field); });
}

etd_status etd_band(etd_plan_t plan, const void* phi, int* idx, long* count) {
  if (!plan || !phi || !idx || !count) return fail(ETD_EINVAL, "NULL argument");
  return guard([&] { *count = plan->impl->band(phi, idx); });
}

etd_status etd_nonlocal(etd_plan_t plan, const void* phi, const void* f, void* w, int* iters, double* resid) {
  if (!plan || !phi || !f || !w) return fail(ETD_EINVAL, "NULL argument");
  return guard([&] { plan->impl->nonlocal(phi, f, w, iters, resid); });
}

etd_status etd_remainder(etd_plan_t plan, int which, const void* phi, const void* phi_old, const void* u,
                         void* out) {
  if (!plan || !phi || !u || !out) return fail(ETD_EINVAL, "NULL argument");
  if (which == 2 && !phi_old) return fail(ETD_EINVAL, "which = 2 needs phi_old");
  return guard([&] { plan->impl->remainder(which, phi, phi_old, u, out); });
}

etd_status etd_timing(etd_plan_t plan, int enable) {
  if (!plan) return fail(ETD_EINVAL, "plan is NULL");
  return guard([&] { plan->impl->timing(enable); });
}

etd_status etd_timing_read(etd_plan_t plan, int kind, double* total_ms, long* launches, double* algo_bytes) {
  if (!plan || !total_ms || !launches || !algo_bytes) return fail(ETD_EINVAL, "NULL argument");
  if (kind < 0 || kind >= ETD_K_NKINDS) return fail(ETD_EINVAL, "unknown kernel kind");
  return guard([&] { plan->impl->timing_read(kind, total_ms, launches, algo_bytes); });
}

}  // extern "C"
