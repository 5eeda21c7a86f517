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
};

PlanBase* make_plan_f32(const etd_params& p, cudaStream_t s);
PlanBase* make_plan_f64(const etd_params& p, cudaStream_t s);

}  // namespace etd
