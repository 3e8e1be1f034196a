// Host side of the C ABI declared in include/dynot.h: plans, workspace,
// transform tables, kernel selection, the iteration driver with CUDA graphs,
// residual checks and the checkpoint / single-step entry points.
#include "../../include/dynot.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "abi_guard.h"
#include "plan_base.h"

using namespace dynot;

namespace dynot {

namespace {
thread_local std::string t_err;
}

ot_status seterr(ot_status s, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  t_err = buf;
  return s;
}

}  // namespace dynot

namespace {

ot_status make_compact(PlanBase& P) {
  Compact& c = P.cp;
  c.n[0] = P.n1; c.n[1] = P.n2; c.n[2] = P.C;
  c.per[0] = P.grid.bc[0] == OT_BC_PERIODIC;
  c.per[1] = P.d >= 2 && P.grid.bc[1] == OT_BC_PERIODIC;
  c.per[2] = P.d >= 3 && P.grid.bc[2] == OT_BC_PERIODIC;
  c.P = P.P;
  c.d = P.d;
  long long off = 0;
  for (int k = 0; k < 3; ++k) {
    c.off[k] = off;
    if (k < P.d) {
      long long dims = 1;
      for (int j = 0; j < 3; ++j) dims *= (j == k) ? (c.per[k] ? c.n[j] : c.n[j] - 1) : c.n[j];
      c.len[k] = dims * P.P;
    } else {
      c.len[k] = 0;
    }
    off += c.len[k];
  }
  c.off[3] = off;
  c.len[3] = (long long)(P.P - 1) * P.S;
  c.total = off + c.len[3];
  return OT_OK;
}

ot_status validate(const ot_grid* gi, int batch, ot_grid& g) {
  if (!gi) return seterr(OT_EINVAL, "grid is NULL");
  g = *gi;
  if (g.ndim < 1 || g.ndim > 3) return seterr(OT_EINVAL, "ndim must be 1, 2 or 3");
  if (batch < 1) return seterr(OT_EINVAL, "batch must be >= 1");
  for (int k = 0; k < g.ndim; ++k) {
    if (g.n[k] < 1) return seterr(OT_EINVAL, "n[%d] must be >= 1", k);
    if (g.bc[k] != OT_BC_PERIODIC && g.bc[k] != OT_BC_NEUMANN) return seterr(OT_EINVAL, "bc[%d] invalid", k);
    if (g.axis_scale[k] == 0) g.axis_scale[k] = g.n[k];
    if (!(g.axis_scale[k] > 0)) return seterr(OT_EINVAL, "axis_scale[%d] must be > 0", k);
  }
  for (int k = g.ndim; k < 3; ++k) {
    g.n[k] = 1;
    g.bc[k] = OT_BC_NEUMANN;
    g.axis_scale[k] = 1;
  }
  if (g.P < 2 || g.P > 64) return seterr(OT_EUNSUPPORTED, "P must be in [2, 64]");
  if (g.sigma == 0) g.sigma = 0.3;
  if (g.tau == 0) g.tau = 0.99 / g.sigma;
  if (!(g.sigma > 0) || !(g.tau > 0) || !(g.tau * g.sigma < 1))
    return seterr(OT_EINVAL, "need sigma > 0, tau > 0, tau*sigma < 1 (Algorithm 1)");
  if (g.check_every <= 0) g.check_every = 10;
  if (g.lam_fp64 <= 0) g.lam_fp64 = 64.0;
  if (g.precision < 0 || g.precision > 2) return seterr(OT_EINVAL, "precision invalid");
  const bool hue = g.ndim == 1 && g.bc[0] == OT_BC_PERIODIC;
  // the kernels address the cells of one problem with 32-bit offsets
  if ((long long)g.P * g.n[0] * g.n[1] * g.n[2] >= (1LL << 31))
    return seterr(OT_EUNSUPPORTED, "a problem must have fewer than 2^31 cells (P n1 n2 C)");
  if (!hue) {
    if (g.n[2] > dynot::kMaxC) return seterr(OT_EUNSUPPORTED, "colour axis longer than %d", kMaxC);
    if (g.n[0] < 2) return seterr(OT_EUNSUPPORTED, "n[0] must be >= 2");
    if (g.n[0] > 4096 || g.n[1] > 4096) return seterr(OT_EUNSUPPORTED, "axes longer than 4096");
  } else {
    if (g.n[0] < 2 || g.n[0] > 8192) return seterr(OT_EUNSUPPORTED, "hue bins must be in [2, 8192]");
  }
  return OT_OK;
}

}  // namespace

struct ot_plan_s {
  std::unique_ptr<PlanBase> impl;
};

// A mixed-size batch: problems of equal shape share one batched plan (a group),
// each group runs on its own stream, and whole iterations of every group are
// captured into one CUDA graph (fork/join across the group streams).
struct ot_batch_s {
  std::vector<std::unique_ptr<PlanBase>> groups;
  std::vector<int> grp, idx;           // problem -> (group, index inside the group)
  cudaStream_t main = nullptr;
  bool own_main = false;
  cudaEvent_t fork = nullptr, t0 = nullptr, t1 = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  ~ot_batch_s() {
    if (main) cudaStreamSynchronize(main);
    for (auto& g : groups)
      if (g && g->st) cudaStreamSynchronize(g->st);
    for (auto& e : gexec)
      if (e) cudaGraphExecDestroy(e);
    for (cudaEvent_t e : {fork, t0, t1})
      if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : join)
      if (e) cudaEventDestroy(e);
    groups.clear();
    if (own_main && main) cudaStreamDestroy(main);
  }
};

namespace {

bool same_shape(const ot_grid& a, const ot_grid& b) {
  if (a.ndim != b.ndim || a.P != b.P || a.precision != b.precision) return false;
  if (a.sigma != b.sigma || a.tau != b.tau || a.lam_fp64 != b.lam_fp64) return false;
  for (int k = 0; k < 3; ++k)
    if (a.n[k] != b.n[k] || a.bc[k] != b.bc[k] || a.axis_scale[k] != b.axis_scale[k]) return false;
  return true;
}

ot_status make_plan(const ot_grid& g, int batch, void* stream, std::unique_ptr<PlanBase>& out);

// fork from the main stream to every group stream and join back
ot_status batch_capture(ot_batch_s& b, int parity) {
  if (b.gexec[parity]) return OT_OK;
  cudaGraph_t gr = nullptr;
  CUDA_OK(cudaStreamBeginCapture(b.main, cudaStreamCaptureModeThreadLocal));
  CUDA_OK(cudaEventRecord(b.fork, b.main));
  for (size_t i = 0; i < b.groups.size(); ++i) {
    PlanBase& P = *b.groups[i];
    CUDA_OK(cudaStreamWaitEvent(P.st, b.fork, 0));
    OT_TRY(P.enqueue_pair());
    CUDA_OK(cudaEventRecord(b.join[i], P.st));
    CUDA_OK(cudaStreamWaitEvent(b.main, b.join[i], 0));
  }
  cudaError_t e = cudaStreamEndCapture(b.main, &gr);
  if (e != cudaSuccess) return seterr(OT_ECUDA, "batch graph capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&b.gexec[parity], gr, 0);
  cudaGraphDestroy(gr);
  if (e != cudaSuccess) return seterr(OT_ECUDA, "batch graph instantiate: %s", cudaGetErrorString(e));
  return OT_OK;
}

}  // namespace

extern "C" {

void ot_grid_rgb(ot_grid* g, int n1, int n2, int P) {
  if (!g) return;
  std::memset(g, 0, sizeof *g);
  g->ndim = 3;
  g->n[0] = n1; g->n[1] = n2; g->n[2] = 3;
  g->bc[0] = OT_BC_NEUMANN; g->bc[1] = OT_BC_NEUMANN; g->bc[2] = OT_BC_PERIODIC;
  g->P = P;
  g->sigma = 0.3;
  g->tau = 0.99 / 0.3;
  g->precision = OT_PREC_MIXED;
  g->check_every = 10;
  g->lam_fp64 = 64.0;
}

void ot_grid_hue(ot_grid* g, int bins, int P) {
  if (!g) return;
  ot_grid_rgb(g, bins, 1, P);
  g->ndim = 1;
  g->n[1] = g->n[2] = 1;
  g->bc[0] = OT_BC_PERIODIC;
}

ot_status ot_plan(const ot_grid* gi, int batch, void* cuda_stream, ot_plan_t* out) {
  return ot_guard([&]() -> ot_status {
    if (!out) return seterr(OT_EINVAL, "out is NULL");
    *out = nullptr;
    ot_grid g;
    OT_TRY(validate(gi, batch, g));
    std::unique_ptr<PlanBase> impl;
    OT_TRY(make_plan(g, batch, cuda_stream, impl));
    ot_plan_s* h = new ot_plan_s;
    h->impl = std::move(impl);
    *out = h;
    return OT_OK;
  });
}

}  // extern "C"

namespace {
ot_status make_plan(const ot_grid& g, int batch, void* cuda_stream, std::unique_ptr<PlanBase>& impl) {
  // problems x time steps index the third grid dimension of the per-step kernels (at most 65535)
  if ((long long)batch * g.P > 65535) return seterr(OT_EUNSUPPORTED, "batch * P must be at most 65535");
  if (g.precision == OT_PREC_FP64) impl.reset(new_plan_f64());
  else impl.reset(new_plan_f32());
  PlanBase& P = *impl;
  P.grid = g;
  P.B = batch;
  P.d = g.ndim;
  P.n1 = g.n[0]; P.n2 = g.n[1]; P.C = g.n[2];
  P.P = g.P;
  P.S = P.n1 * P.n2 * P.C;
  P.N = (long long)P.P * P.S;
  P.hue = g.ndim == 1 && g.bc[0] == OT_BC_PERIODIC;
  if (cuda_stream) {
    P.st = (cudaStream_t)cuda_stream;
  } else {
    CUDA_OK(cudaStreamCreateWithFlags(&P.st, cudaStreamNonBlocking));
    P.own_stream = true;
  }
  OT_TRY(make_compact(P));
  OT_TRY(P.init());
  CUDA_OK(cudaStreamSynchronize(P.st));
  return OT_OK;
}
}  // namespace

extern "C" {

ot_status ot_batch_create(const ot_grid* grids, int count, void* cuda_stream, ot_batch_t* out) {
  return ot_guard([&]() -> ot_status {
    if (!out || !grids || count < 1) return seterr(OT_EINVAL, "bad batch arguments");
    *out = nullptr;
    std::unique_ptr<ot_batch_s> b(new ot_batch_s);
    std::vector<ot_grid> keys;
    std::vector<int> counts;
    b->grp.resize(count);
    b->idx.resize(count);
    for (int i = 0; i < count; ++i) {
      ot_grid g;
      OT_TRY(validate(&grids[i], 1, g));
      int k = -1;
      for (size_t j = 0; j < keys.size(); ++j)
        if (same_shape(keys[j], g)) { k = (int)j; break; }
      if (k < 0) {
        k = (int)keys.size();
        keys.push_back(g);
        counts.push_back(0);
      }
      b->grp[i] = k;
      b->idx[i] = counts[k]++;
    }
    for (size_t j = 0; j < keys.size(); ++j) {
      std::unique_ptr<PlanBase> p;
      OT_TRY(make_plan(keys[j], counts[j], nullptr, p));   // each group on a stream of its own
      OT_TRY(p->enable_retirement());                      // converged problems stop iterating
      b->groups.push_back(std::move(p));
    }
    if (cuda_stream) {
      b->main = (cudaStream_t)cuda_stream;
    } else {
      CUDA_OK(cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking));
      b->own_main = true;
    }
    CUDA_OK(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
    CUDA_OK(cudaEventCreate(&b->t0));
    CUDA_OK(cudaEventCreate(&b->t1));
    b->join.resize(b->groups.size());
    for (auto& e : b->join) CUDA_OK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    *out = b.release();
    return OT_OK;
  });
}

int ot_batch_groups(ot_batch_t b) { return b ? (int)b->groups.size() : 0; }

void ot_batch_destroy(ot_batch_t b) { delete b; }

ot_status ot_batch_solve(ot_batch_t b, const float* const* f0, const float* const* f1, int iters, double tol,
                         int check_every, ot_solve_stats* stats) {
  return ot_guard([&]() -> ot_status {
    if (!b || !f0 || !f1 || iters < 1) return seterr(OT_EINVAL, "bad batch solve arguments");
    const int count = (int)b->grp.size();
    for (int i = 0; i < count; ++i) OT_TRY(b->groups[b->grp[i]]->stage_problem(b->idx[i], f0[i], f1[i]));
    for (auto& g : b->groups) OT_TRY(g->prepare_staged());   // validation, rescaling, cold start
    for (size_t i = 0; i < b->groups.size(); ++i) {
      CUDA_OK(cudaEventRecord(b->join[i], b->groups[i]->st));
      CUDA_OK(cudaStreamWaitEvent(b->main, b->join[i], 0));
    }
    // every problem starts active; one that meets tol at a check is retired: its kernels return at once
    // from then on, so its state and path stay those of that check
    std::vector<std::vector<int>> act(b->groups.size());
    for (size_t i = 0; i < b->groups.size(); ++i) {
      act[i].assign(b->groups[i]->B, 1);
      OT_TRY(b->groups[i]->set_active(act[i], b->main));
    }
    std::vector<int> its(count, 0);
    int live = count;
    CUDA_OK(cudaEventRecord(b->t0, b->main));
    const int K = check_every > 0 ? check_every : iters;
    int done = 0;
    std::vector<std::vector<ProblemCheck>> per(b->groups.size());
    while (done < iters && live > 0) {
      const int chunk = std::min(K, iters - done);
      const int plain = chunk - 1;
      const int par = b->groups[0]->parity();
      if (plain >= 2) OT_TRY(batch_capture(*b, par));
      for (int r = 0; r < plain / 2; ++r) CUDA_OK(cudaGraphLaunch(b->gexec[par], b->main));
      // the remaining single iteration and the checked one, per group after the graph
      CUDA_OK(cudaEventRecord(b->fork, b->main));
      for (size_t i = 0; i < b->groups.size(); ++i) {
        PlanBase& P = *b->groups[i];
        CUDA_OK(cudaStreamWaitEvent(P.st, b->fork, 0));
        if (plain % 2) OT_TRY(P.enqueue_single());
        OT_TRY(P.enqueue_check_async());
        CUDA_OK(cudaEventRecord(b->join[i], P.st));
        CUDA_OK(cudaStreamWaitEvent(b->main, b->join[i], 0));
      }
      CUDA_OK(cudaStreamSynchronize(b->main));
      done += chunk;
      for (size_t i = 0; i < b->groups.size(); ++i) OT_TRY(b->groups[i]->collect(per[i]));
      std::vector<char> changed(b->groups.size(), 0);
      for (int i = 0; i < count; ++i) {
        const int gi = b->grp[i], k = b->idx[i];
        if (!act[gi][k]) continue;
        its[i] = done;
        if (tol > 0 && per[gi][k].residual <= tol) {
          act[gi][k] = 0;
          changed[gi] = 1;
          --live;
        }
      }
      for (size_t i = 0; i < b->groups.size(); ++i)
        if (changed[i]) OT_TRY(b->groups[i]->set_active(act[i], b->main));
    }
    const bool converged = live == 0;
    CUDA_OK(cudaEventRecord(b->t1, b->main));
    CUDA_OK(cudaEventSynchronize(b->t1));
    float ms = 0;
    CUDA_OK(cudaEventElapsedTime(&ms, b->t0, b->t1));
    if (stats) {
      for (int i = 0; i < count; ++i) {
        const ProblemCheck& c = per[b->grp[i]][b->idx[i]];
        stats[i].iterations = its[i];
        stats[i].residual = c.residual;
        stats[i].energy = c.energy;
        stats[i].mass_drift = c.drift;
        stats[i].dual_value = c.dual;
        stats[i].gap = c.gap;
        stats[i].elapsed_ms = ms;
      }
    }
    if (tol > 0 && !converged)
      return seterr(OT_ENOTCONV, "batch: %d problems above the tolerance after %d iterations", live, done);
    return OT_OK;
  });
}

ot_status ot_batch_path(ot_batch_t b, int i, float* f, float* m0, float* m1, float* m2) {
  return ot_guard([&]() -> ot_status {
    if (!b || i < 0 || i >= (int)b->grp.size()) return seterr(OT_EINVAL, "bad batch problem index");
    return b->groups[b->grp[i]]->path_one(b->idx[i], f, m0, m1, m2);
  });
}

void ot_destroy(ot_plan_t p) {
  if (!p) return;
  if (p->impl && p->impl->st) cudaStreamSynchronize(p->impl->st);
  delete p;
}

// the per-call grid of ot_solve / ot_solve_warm: sizes must match the plan; check_every applies
static ot_status call_grid(PlanBase& P, const ot_grid* g) {
  if (!g) return OT_OK;
  if (g->ndim != P.grid.ndim || g->P != P.grid.P) return seterr(OT_EINVAL, "grid does not match the plan");
  for (int k = 0; k < g->ndim; ++k)
    if (g->n[k] != P.grid.n[k] || g->bc[k] != P.grid.bc[k]) return seterr(OT_EINVAL, "grid does not match the plan");
  const double sg = g->sigma > 0 ? g->sigma : P.grid.sigma;
  const double ta = g->tau > 0 ? g->tau : 0.99 / sg;
  if (!(sg * ta < 1)) return seterr(OT_EINVAL, "need tau*sigma < 1");
  if (sg != P.grid.sigma || ta != P.grid.tau)
    return seterr(OT_EINVAL, "sigma/tau differ from the plan's; create a plan with them");
  if (g->check_every > 0) P.grid.check_every = g->check_every;
  return OT_OK;
}

ot_status ot_solve(ot_plan_t p, const float* f0, const float* f1, const ot_grid* g, int iters, double tol,
                   const float* init_path, ot_solve_stats* stats) {
  return ot_guard([&]() -> ot_status {
    if (!p) return seterr(OT_EINVAL, "plan is NULL");
    PlanBase& P = *p->impl;
    OT_TRY(call_grid(P, g));
    return P.solve(f0, f1, iters, tol, init_path, nullptr, 0, 0.0, 0.0, stats, nullptr);
  });
}

ot_status ot_solve_warm(ot_plan_t p, const float* f0, const float* f1, const ot_grid* g, int iters, double tol,
                        const float* init_path, const float* init_dual, int dual_init, double dual_support,
                        double fallback_residual, ot_solve_stats* stats, int* used_cold) {
  return ot_guard([&]() -> ot_status {
    if (!p) return seterr(OT_EINVAL, "plan is NULL");
    if (!init_path) return seterr(OT_EINVAL, "init_path is required");
    if (!(fallback_residual >= 0) || !(dual_support >= 0))
      return seterr(OT_EINVAL, "fallback_residual and dual_support must be >= 0");
    PlanBase& P = *p->impl;
    OT_TRY(call_grid(P, g));
    return P.solve(f0, f1, iters, tol, init_path, init_dual, dual_init, dual_support, fallback_residual, stats,
                   used_cold);
  });
}

ot_status ot_path(ot_plan_t p, float* f, float* m0, float* m1, float* m2) {
  return ot_guard([&]() -> ot_status {
    if (!p) return seterr(OT_EINVAL, "plan is NULL");
    return p->impl->path(f, m0, m1, m2);
  });
}

size_t ot_path_size(ot_plan_t p) { return p ? (size_t)p->impl->B * p->impl->cp.total : 0; }
size_t ot_dual_size(ot_plan_t p) {
  return p ? (size_t)p->impl->B * (p->impl->d + 1) * (size_t)p->impl->N : 0;
}

ot_status ot_state_set(ot_plan_t p, const float* f0, const float* f1, const float* x, const float* b,
                       const float* bb) {
  return ot_guard([&]() -> ot_status {
    if (!p) return seterr(OT_EINVAL, "plan is NULL");
    return p->impl->state_set(f0, f1, x, b, bb);
  });
}

ot_status ot_state_get(ot_plan_t p, float* x, float* b, float* bb) {
  return ot_guard([&]() -> ot_status {
    if (!p) return seterr(OT_EINVAL, "plan is NULL");
    return p->impl->state_get(x, b, bb);
  });
}

ot_status ot_iterate(ot_plan_t p, int iters, ot_solve_stats* stats) {
  return ot_guard([&]() -> ot_status {
    if (!p) return seterr(OT_EINVAL, "plan is NULL");
    return p->impl->iterate(iters, stats);
  });
}

ot_status ot_project(ot_plan_t p, const float* f0, const float* f1, const float* a, float* x, float* phi) {
  return ot_guard([&]() -> ot_status {
    if (!p) return seterr(OT_EINVAL, "plan is NULL");
    return p->impl->project(f0, f1, a, x, phi);
  });
}

static ot_status prox_impl(bool cardano, int count, int ncomp, double sigma, const float* am, const float* af,
                           float* u, float* v) {
  if (count < 0 || ncomp < 1 || ncomp > 3 || !(sigma > 0)) return seterr(OT_EINVAL, "bad prox arguments");
  if (count == 0) return OT_OK;
  if (!am || !af || !u || !v) return seterr(OT_EINVAL, "NULL prox buffer");
  const size_t n = (size_t)count;
  DevMem m;
  CUDA_OK(cudaMalloc(&m.p, sizeof(float) * n * (2 * ncomp + 2)));
  float* dam = (float*)m.p;
  float* daf = dam + n * ncomp;
  float* du = daf + n;
  float* dv = du + n * ncomp;
  CUDA_OK(cudaMemcpy(dam, am, sizeof(float) * n * ncomp, cudaMemcpyDefault));
  CUDA_OK(cudaMemcpy(daf, af, sizeof(float) * n, cudaMemcpyDefault));
  const int blocks = (int)std::min<size_t>((n + 255) / 256, 4096);
  if (cardano) k_prox_cells<true><<<blocks, 256>>>(count, ncomp, (float)sigma, dam, daf, du, dv);
  else k_prox_cells<false><<<blocks, 256>>>(count, ncomp, (float)sigma, dam, daf, du, dv);
  CUDA_OK(cudaGetLastError());
  CUDA_OK(cudaMemcpy(u, du, sizeof(float) * n * ncomp, cudaMemcpyDefault));
  CUDA_OK(cudaMemcpy(v, dv, sizeof(float) * n, cudaMemcpyDefault));
  return OT_OK;
}

ot_status ot_prox(int count, int ncomp, double sigma, const float* am, const float* af, float* u, float* v) {
  return ot_guard([&]() -> ot_status {
    return prox_impl(false, count, ncomp, sigma, am, af, u, v);
  });
}

ot_status ot_prox_cardano(int count, int ncomp, double sigma, const float* am, const float* af, float* u, float* v) {
  return ot_guard([&]() -> ot_status {
    return prox_impl(true, count, ncomp, sigma, am, af, u, v);
  });
}

ot_status ot_profile(ot_plan_t p, int iters, double ms[5], const char** names) {
  return ot_guard([&]() -> ot_status {
    if (!p || !ms) return seterr(OT_EINVAL, "plan or ms is NULL");
    if (names)
      *names = p->impl->hue ? "hue_fwd,hue_t,hue_inv,update,iteration"
                            : "rhs_fwd_xt,solve_yc,inv_xt,update,iteration";
    return p->impl->profile(iters, ms);
  });
}

const char* ot_last_error(void) { return t_err.c_str(); }

int ot_abi_version(void) { return OT_ABI_VERSION; }

}  // extern "C"
