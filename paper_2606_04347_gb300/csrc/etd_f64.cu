// Double-precision instantiation.
#include "stepper.cuh"
namespace etd {
PlanBase* make_plan_f64(const etd_params& p, cudaStream_t s, const TileOpt& t) { return new Stepper<double>(p, s, t); }
}  // namespace etd
