// plan.h -- precision-independent plan interface behind the C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdexcept>
#include <string>
#include "etd.h"

namespace etd {

struct Error : public std::runtime_error {
  etd_status code;
  Error(etd_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define ETD_CUDA(call)                                                                       \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      throw ::etd::Error(e_ == cudaErrorMemoryAllocation ? ETD_ENOMEM : ETD_ECUDA,           \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                \
  } while (0)

// Tile options of a plan (0 = the default choice): pass-A z-planes per CTA, pass-B pencil
// blocks per CTA, and direct pass-A loads/stores instead of tensor-copy staging.
struct TileOpt {
  int zb = 0, kb = 0, direct = 0;
};

class PlanBase {
 public:
  virtual ~PlanBase() {}
  virtual void step(void* phi, void* u, int nsteps, etd_diag* last) = 0;
  virtual void energy(const void* phi, const void* u, etd_diag* out) = 0;
  virtual void fft_forward(const void* field, void* half) = 0;
  virtual void fft_inverse(const void* half, void* field) = 0;
  virtual long band(const void* phi, int* idx) = 0;
  virtual void nonlocal(const void* phi, const void* f, void* w, int* iters, double* resid) = 0;
  virtual void remainder(int which, const void* phi, const void* phi_old, const void* u, void* out) = 0;
  virtual void timing(int enable) = 0;
  virtual void timing_read(int kind, double* ms, long* launches, double* bytes) = 0;
  // Milliseconds per forward + inverse transform pair of the plan's grid (mean of reps, after
  // one untimed pair), with its tiles.
  virtual double time_transforms(int reps) = 0;
  // The tiles in use: pass-A z-planes, pass-B pencil blocks, tensor-copy staging (1/0).
  virtual void tiles(int* zb, int* kb, int* tma) const = 0;
};

PlanBase* make_plan_f32(const etd_params& p, cudaStream_t s, const TileOpt& t = TileOpt{});
PlanBase* make_plan_f64(const etd_params& p, cudaStream_t s, const TileOpt& t = TileOpt{});

}  // namespace etd
