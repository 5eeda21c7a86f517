// etd_api.cu -- the extern "C" boundary declared in include/etd.h.  Validates arguments,
// dispatches to the precision-specific plan and turns exceptions into status codes.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <map>
#include <string>
#include <tuple>
#include <vector>
#include "fft.cuh"
#include "krylov.cuh"
#include "plan.h"

struct etd_plan_s {
  etd::PlanBase* impl;
  etd_params params;
};

// A batch of independent runs: one plan and one stream per run.  Steps are taken run by run
// on the runs' streams, forked from and joined back into the batch stream; after two eager
// steps (the band solves' initial-guess history is then full and repeats every 6 steps), 6
// steps of every run are captured into one CUDA graph and replayed.
struct etd_batch_s {
  struct Run {
    etd::PlanBase* plan = nullptr;
    etd_params params{};
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    etd::TileOpt tile{};
    void* phi = nullptr;   // pointers the captured graph was recorded with
    void* u = nullptr;
  };
  std::vector<Run> runs;
  cudaStream_t user = nullptr;    // the caller's stream: every call is ordered after its prior work
  cudaStream_t origin = nullptr;  // the batch's own stream (graphs are recorded and replayed on it)
  cudaEvent_t fork = nullptr, enter = nullptr, leave = nullptr;
  cudaGraphExec_t exec = nullptr;
  int block = 6;      // steps per graph replay
  long steps = 0;     // steps every run has taken
  int graph = -1;     // 1: replaying a graph; 0: capture unavailable, eager steps; -1: not tried
  double tune_ms = 0; // time spent by the autotuner
  std::string graph_error;  // why the graph could not be recorded (graph = 0)
};

namespace {
thread_local std::string g_last_error;

etd_status fail(etd_status s, const std::string& m) {
  g_last_error = m;
  return s;
}

// Axis lengths of the two-pass FFT (fft_length_ok): powers of two from 8 to 256, and 96.
bool length_ok(int n) { return etd::fft_length_ok(n); }

etd_status validate(const etd_params& p) {
  if (p.dim != 2 && p.dim != 3) return fail(ETD_EINVAL, "dim must be 2 or 3");
  const int nz = p.dim == 2 ? 1 : p.n[2];
  if (p.dim == 2 && p.n[2] != 1) return fail(ETD_EINVAL, "2D plans need n[2] = 1");
  for (int d = 0; d < 2; ++d)
    if (!length_ok(p.n[d])) return fail(ETD_EINVAL, "Nx, Ny must be powers of two in [8, 256] or 96");
  if (p.dim == 3 && !length_ok(nz)) return fail(ETD_EINVAL, "Nz must be a power of two in [8, 256] or 96");
  for (int d = 0; d < p.dim; ++d)
    if (!(p.half_len[d] > 0)) return fail(ETD_EINVAL, "half lengths must be positive");
  for (int d = 1; d < p.dim; ++d)
    if (std::fabs(p.half_len[d] - p.half_len[0]) > 1e-12 * p.half_len[0])
      return fail(ETD_EINVAL, "only cubic boxes (X = Y = Z) are supported");
  if (p.scheme != ETD_ETD1 && p.scheme != ETD_ETDRK2) return fail(ETD_EINVAL, "scheme must be ETD1 or ETDRK2");
  if (p.model != ETD_MODEL_FIXED && p.model != ETD_MODEL_COUPLED && p.model != ETD_MODEL_FIXED_SQRTG)
    return fail(ETD_EINVAL, "unknown model");
  if (p.model == ETD_MODEL_FIXED_SQRTG && !(p.B2 > 0)) return fail(ETD_EINVAL, "the Sec. 2.2 scheme needs B = B2 > 0");
  if (!(p.krylov_tol >= 0) || !(p.krylov_tol < 1)) return fail(ETD_EINVAL, "krylov_tol must be in [0, 1)");
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

etd_status etd_krylov_coeffs(int m, const double* alpha, const double* beta, double tau, int j, double* y,
                             double* tail) {
  if (m < 1 || m > etd::kKrylovMax) return fail(ETD_EINVAL, "m must be in [1, 128]");
  if (j < 0 || j > 2) return fail(ETD_EINVAL, "j must be 0, 1 or 2");
  if (!alpha || (m > 1 && !beta) || !y || !tail) return fail(ETD_EINVAL, "NULL argument");
  if (!(tau >= 0)) return fail(ETD_EINVAL, "tau must be >= 0");
  return guard([&] {
    std::vector<double> v;
    *tail = etd::krylov_coeffs(m, alpha, beta, tau, j, v);
    for (int k = 0; k < m; ++k) y[k] = v[k];
  });
}

}  // extern "C"

// ---- batched runs --------------------------------------------------------------------

namespace {

etd::PlanBase* make_plan(const etd_params& p, cudaStream_t st, const etd::TileOpt& t) {
  return p.precision == ETD_FP64 ? etd::make_plan_f64(p, st, t) : etd::make_plan_f32(p, st, t);
}

// Tile candidates of one grid: pass-A z-planes (divisors of Nz), pass-B pencil blocks (powers
// of two up to what a CTA's teams hold), tensor-copy staging on or off (3D only).
std::vector<etd::TileOpt> tile_candidates(const etd_params& p) {
  std::vector<etd::TileOpt> out;
  const int nz = p.dim == 2 ? 1 : p.n[2];
  const size_t csize = p.precision == ETD_FP64 ? 16 : 8;
  const int zbs[4] = {1, 2, 4, 8};
  for (int zb : zbs) {
    if (nz == 1 && zb != 1) continue;
    if (nz > 1 && (zb == 1 || nz % zb)) continue;
    for (int kb = 1; kb <= 64; kb *= 2) {
      etd::Geo g{};
      g.dim = p.dim;
      g.nx = p.n[0];
      g.ny = p.n[1];
      g.nz = nz;
      g.nxh = g.nx / 2 + 1;
      size_t sa = 0, sb = 0;
      if (!etd::choose_tiles(g, csize, sa, sb, zb, nz > 1 ? kb : 0)) continue;
      for (int direct = 0; direct <= (nz > 1 ? 1 : 0); ++direct) out.push_back(etd::TileOpt{zb, nz > 1 ? kb : 0, direct});
      if (nz == 1) break;
    }
  }
  return out;
}

// Fastest forward + inverse transform pair over the candidates, one grid and precision at a
// time (temporary fixed-membrane plans on the batch stream; the pair is what every stage of
// the step runs).
etd::TileOpt autotune(const etd_params& p, cudaStream_t st) {
  etd_params q = p;
  q.model = ETD_MODEL_FIXED;
  etd::TileOpt best{};
  double best_ms = 1e300;
  for (const etd::TileOpt& t : tile_candidates(q)) {
    etd::PlanBase* plan = nullptr;
    try {
      plan = make_plan(q, st, t);
      const double ms = plan->time_transforms(5);
      if (ms < best_ms) {
        best_ms = ms;
        best = t;
      }
    } catch (const etd::Error&) {
      cudaGetLastError();
    }
    delete plan;
  }
  return best;
}

void batch_release(etd_batch_s* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (auto& r : b->runs) {
    delete r.plan;
    if (r.done) cudaEventDestroy(r.done);
    if (r.stream) cudaStreamDestroy(r.stream);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->enter) cudaEventDestroy(b->enter);
  if (b->leave) cudaEventDestroy(b->leave);
  if (b->origin) cudaStreamDestroy(b->origin);
  delete b;
}

// Steps of every run, each on its own stream between a fork and a join on the batch stream.
void batch_eager(etd_batch_s* b, void* const* phi, void* const* u, int nsteps, bool first) {
  ETD_CUDA(cudaEventRecord(b->fork, b->origin));
  for (size_t i = 0; i < b->runs.size(); ++i) {
    auto& r = b->runs[i];
    ETD_CUDA(cudaStreamWaitEvent(r.stream, b->fork, 0));
    const bool pass_phi = phi && (first || r.params.model == ETD_MODEL_COUPLED);
    r.plan->step(pass_phi ? phi[i] : nullptr, u[i], nsteps, nullptr);
    ETD_CUDA(cudaEventRecord(r.done, r.stream));
    ETD_CUDA(cudaStreamWaitEvent(b->origin, r.done, 0));
  }
}

// Capture `block` steps of every run into one graph.  Returns false (and leaves the batch on
// eager steps) if the capture or the instantiation fails; the plans' host-side state is the
// same after a whole number of 6-step blocks, so a failed capture leaves them consistent.
bool batch_capture(etd_batch_s* b, void* const* phi, void* const* u) {
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  bool ok = true;
  try {
    batch_eager(b, phi, u, b->block, false);
  } catch (const etd::Error& ex) {
    ok = false;
    b->graph_error = ex.what();
  }
  const cudaError_t e = cudaStreamEndCapture(b->origin, &graph);
  if (!ok || e != cudaSuccess || !graph) {
    if (ok) b->graph_error = std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e);
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return false;
  }
  const cudaError_t ei = cudaGraphInstantiate(&b->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {
    b->graph_error = std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ei);
    b->exec = nullptr;
    cudaGetLastError();
    return false;
  }
  for (size_t i = 0; i < b->runs.size(); ++i) {
    b->runs[i].phi = phi ? phi[i] : nullptr;
    b->runs[i].u = u[i];
  }
  return true;
}

}  // namespace

extern "C" {

etd_status etd_plan_batch(const etd_params* params, int nruns, void* cuda_stream, int autotune_tiles,
                          etd_batch_t* out) {
  if (!out) return fail(ETD_EINVAL, "out is NULL");
  *out = nullptr;
  if (!params || nruns < 1) return fail(ETD_EINVAL, "params is NULL or nruns < 1");
  for (int i = 0; i < nruns; ++i) {
    const etd_status v = validate(params[i]);
    if (v != ETD_OK) return fail(v, "run " + std::to_string(i) + ": " + g_last_error);
    if (params[i].model == ETD_MODEL_FIXED_SQRTG)
      return fail(ETD_EINVAL, "run " + std::to_string(i) +
                                  ": the Sec. 2.2 scheme sizes its Krylov spaces on the host between launches and "
                                  "cannot run inside a batch graph; use etd_plan");
  }
  etd_batch_s* b = new etd_batch_s;
  b->user = static_cast<cudaStream_t>(cuda_stream);
  const etd_status s = guard([&] {
    ETD_CUDA(cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking));
    ETD_CUDA(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
    ETD_CUDA(cudaEventCreateWithFlags(&b->enter, cudaEventDisableTiming));
    ETD_CUDA(cudaEventCreateWithFlags(&b->leave, cudaEventDisableTiming));
    const auto t0 = std::chrono::steady_clock::now();
    std::map<std::tuple<int, int, int, int, int>, etd::TileOpt> tuned;
    b->runs.resize(nruns);
    for (int i = 0; i < nruns; ++i) {
      auto& r = b->runs[i];
      r.params = params[i];
      const auto key = std::make_tuple(params[i].dim, params[i].n[0], params[i].n[1], params[i].n[2],
                                       params[i].precision);
      if (autotune_tiles) {
        auto it = tuned.find(key);
        if (it == tuned.end()) it = tuned.emplace(key, autotune(params[i], b->origin)).first;
        r.tile = it->second;
      }
      ETD_CUDA(cudaStreamCreateWithFlags(&r.stream, cudaStreamNonBlocking));
      ETD_CUDA(cudaEventCreateWithFlags(&r.done, cudaEventDisableTiming));
      r.plan = make_plan(r.params, r.stream, r.tile);
    }
    b->tune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  });
  if (s != ETD_OK) {
    batch_release(b);
    return s;
  }
  *out = b;
  return ETD_OK;
}

etd_status etd_batch_step(etd_batch_t b, void* const* phi, void* const* u, int nsteps) {
  if (!b || !u) return fail(ETD_EINVAL, "batch or u is NULL");
  if (nsteps < 0) return fail(ETD_EINVAL, "nsteps < 0");
  const int nr = (int)b->runs.size();
  for (int i = 0; i < nr; ++i) {
    if (!u[i]) return fail(ETD_EINVAL, "u[" + std::to_string(i) + "] is NULL");
    const bool need_phi = b->steps == 0 || b->runs[i].params.model == ETD_MODEL_COUPLED;
    if (need_phi && (!phi || !phi[i])) return fail(ETD_EINVAL, "phi[" + std::to_string(i) + "] is needed");
  }
  return guard([&] {
    ETD_CUDA(cudaEventRecord(b->enter, b->user));
    ETD_CUDA(cudaStreamWaitEvent(b->origin, b->enter, 0));
    // a graph is tied to the field pointers it was recorded with
    if (b->exec) {
      bool same = true;
      for (int i = 0; i < nr; ++i) {
        const auto& r = b->runs[i];
        const void* p = (phi && r.params.model == ETD_MODEL_COUPLED) ? phi[i] : nullptr;
        if (r.u != u[i] || (r.params.model == ETD_MODEL_COUPLED && r.phi != p)) same = false;
      }
      if (!same) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
      }
    }
    while (nsteps > 0 && b->steps < 2) {
      batch_eager(b, phi, u, 1, b->steps == 0);
      ++b->steps;
      --nsteps;
    }
    if (nsteps >= b->block && b->graph != 0 && !b->exec) {
      // capture records (does not run) one block of steps; the plans' host state then stands
      // 6 steps on, which is the state it started from
      b->graph = batch_capture(b, phi, u) ? 1 : 0;
    }
    while (b->exec && nsteps >= b->block) {
      ETD_CUDA(cudaGraphLaunch(b->exec, b->origin));
      b->steps += b->block;
      nsteps -= b->block;
    }
    if (nsteps > 0) {
      batch_eager(b, phi, u, nsteps, false);
      b->steps += nsteps;
    }
    ETD_CUDA(cudaEventRecord(b->leave, b->origin));
    ETD_CUDA(cudaStreamWaitEvent(b->user, b->leave, 0));
  });
}

etd_status etd_batch_info(etd_batch_t b, int run, int* zb, int* kb, int* tma, int* graph) {
  if (!b || run < 0 || run >= (int)b->runs.size()) return fail(ETD_EINVAL, "no such run");
  // the reason a graph could not be recorded, if any, is left in etd_last_error()
  const etd_status st = guard([&] {
    int z = 0, k = 0, t = 0;
    b->runs[run].plan->tiles(&z, &k, &t);
    if (zb) *zb = z;
    if (kb) *kb = k;
    if (tma) *tma = t;
    if (graph) *graph = b->graph;
  });
  if (st == ETD_OK && b->graph == 0) g_last_error = b->graph_error;
  return st;
}

etd_status etd_batch_check(etd_batch_t b, void* const* phi, void* const* u, etd_diag* diag) {
  if (!b || !u) return fail(ETD_EINVAL, "batch or u is NULL");
  return guard([&] {
    ETD_CUDA(cudaStreamSynchronize(b->origin));
    ETD_CUDA(cudaStreamSynchronize(b->user));
    for (size_t i = 0; i < b->runs.size(); ++i) {
      auto& r = b->runs[i];
      etd_diag d;
      void* p = (phi && r.params.model == ETD_MODEL_COUPLED) ? phi[i] : nullptr;
      try {
        r.plan->step(p, u[i], 0, &d);
      } catch (const etd::Error& e) {
        throw etd::Error(e.code, "run " + std::to_string(i) + ": " + e.what());
      }
      if (diag) diag[i] = d;
    }
  });
}

etd_status etd_batch_free(etd_batch_t b) {
  if (!b) return ETD_OK;
  cudaStreamSynchronize(b->origin);
  cudaStreamSynchronize(b->user);
  batch_release(b);
  return ETD_OK;
}

}  // extern "C"
