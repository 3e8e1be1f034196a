// FP64 plan (every kernel in double precision).
#include "plan.cuh"

namespace dynot {
PlanBase* new_plan_f64() { return new Plan<double>(); }
}  // namespace dynot
