// FP32 plan (the MIXED and FP32 precision modes).
#include "plan.cuh"

namespace dynot {
PlanBase* new_plan_f32() { return new Plan<float>(); }
}  // namespace dynot
