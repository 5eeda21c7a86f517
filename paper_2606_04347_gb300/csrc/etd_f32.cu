// Single-precision (FP32 storage and FFT, FP64 tables and reductions) instantiation.
#include "stepper.cuh"
namespace etd {
PlanBase* make_plan_f32(const etd_params& p, cudaStream_t s, const TileOpt& t) { return new Stepper<float>(p, s, t); }
}  // namespace etd
