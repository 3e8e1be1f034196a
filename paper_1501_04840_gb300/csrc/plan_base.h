// Plan interface shared by the C ABI (api.cu) and the FP32 / FP64 plan
// implementations (plan_f32.cu, plan_f64.cu).
#pragma once
#include "../../include/dynot.h"

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "common.cuh"
#include "misc_kernels.cuh"

namespace dynot {

// Record a thread-local error message (read by ot_last_error) and return s.
ot_status seterr(ot_status s, const char* fmt, ...);

#define CUDA_OK(x)                                                                                       \
  do {                                                                                                   \
    cudaError_t e_ = (x);                                                                                \
    if (e_ != cudaSuccess)                                                                               \
      return seterr(e_ == cudaErrorMemoryAllocation ? OT_ENOMEM : OT_ECUDA, "%s: %s (%s:%d)", #x,        \
                    cudaGetErrorString(e_), __FILE__, __LINE__);                                         \
  } while (0)

#define OT_TRY(x)                  \
  do {                             \
    ot_status s_ = (x);            \
    if (s_ != OT_OK) return s_;    \
  } while (0)

// --------------------------------------------------------------------------
// device memory owner
// --------------------------------------------------------------------------
struct DevMem {
  void* p = nullptr;
  ~DevMem() {
    if (p) cudaFree(p);
  }
};

// --------------------------------------------------------------------------
// plans
// --------------------------------------------------------------------------
// residual, energy (caller units) and mass drift of one problem at a check
struct ProblemCheck {
  double residual = 0, energy = 0, drift = 0, dual = 0, gap = 0;
};

struct PlanBase {
  ot_grid grid{};
  int B = 1, d = 3;
  int n1 = 1, n2 = 1, C = 1, P = 2, S = 1;
  long long N = 0;
  bool hue = false;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  int device = 0;
  Compact cp{};
  std::vector<double> out_scale;  // per problem: solver units -> caller units
  virtual ~PlanBase() {
    if (own_stream && st) cudaStreamDestroy(st);
  }
  virtual ot_status init() = 0;
  // init: packed path (caller units) or NULL; dual_init: b = bbar = grad J(K x0 + (0, f_b^+)) / sigma
  // where the density is >= dual_support (solver units), zero elsewhere;
  // fallback > 0: restart cold when the residual of the first check exceeds it (*used_cold = 1).
  // init_dual (packed dual, or NULL) replaces the formula.
  virtual ot_status solve(const float* f0, const float* f1, int iters, double tol, const float* init,
                          const float* init_dual, int dual_init, double dual_support, double fallback,
                          ot_solve_stats* stats, int* used_cold) = 0;
  virtual ot_status path(float* f, float* m0, float* m1, float* m2) = 0;
  virtual ot_status state_set(const float* f0, const float* f1, const float* x, const float* b,
                              const float* bb) = 0;
  virtual ot_status state_get(float* x, float* b, float* bb) = 0;
  virtual ot_status iterate(int iters, ot_solve_stats* stats) = 0;
  virtual ot_status project(const float* f0, const float* f1, const float* a, float* x, float* phi) = 0;
  virtual ot_status profile(int iters, double ms[5]) = 0;
  // mixed-size batches: staging, one plain pair / single iteration, asynchronous checks
  virtual ot_status stage_problem(int bi, const float* f0, const float* f1) = 0;
  virtual ot_status prepare_staged() = 0;
  virtual ot_status enqueue_pair() = 0;
  virtual ot_status enqueue_single() = 0;
  virtual ot_status enqueue_check_async() = 0;
  virtual ot_status collect(std::vector<ProblemCheck>& per) = 0;
  virtual int parity() const = 0;
  // per-problem retirement (mixed-size batches): enable_retirement() before any graph is captured makes
  // every kernel skip the problems whose flag is 0; set_active uploads the flags on stream s, and collect
  // leaves the entries of retired problems as they were
  virtual ot_status enable_retirement() = 0;
  virtual ot_status set_active(const std::vector<int>& act, cudaStream_t s) = 0;
  virtual ot_status path_one(int bi, float* f, float* m0, float* m1, float* m2) = 0;
};

PlanBase* new_plan_f32();
PlanBase* new_plan_f64();

}  // namespace dynot
