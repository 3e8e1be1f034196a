// Kernels of one PDHG iteration (Algorithm 1) on the grid with three spatial
// axes x (n1), y (n2), colour (C) and P time intervals.
//
//   K_A  rhs_fwd_xt : r = A a - f_b^-  (section 3, step 1), then the forward
//                     DCT-II along x and along t, per (y, c) row of a problem.
//   K_B  solve_yc   : forward DCT-II along y, the colour eigen-solve with the
//                     division by the eigenvalues of A A^T (zero mode -> 0),
//                     inverse DCT along y, per strip of W x-frequencies and one
//                     t-frequency.
//   K_C  inv_xt     : inverse DCT along t and x -> phi = (A A^T)^+ r.
//   K_D  update     : x^{r+1} = a - A^T phi, u = S_M m, v = S_F f + f_b^+,
//                     per-cell prox of J, b^{r+1}, bbar^{r+1} = 2 b^{r+1} - b^r,
//                     and the next a = x^{r+1} - tau sigma K^T bbar^{r+1}
//                     (steps 1-4 of Algorithm 1).  bbar at the neighbour cell of
//                     each face is recomputed in place, so the iteration state
//                     is just (a, b).
#pragma once
#include "common.cuh"
#include "fft.cuh"

namespace dynot {

// ---------------------------------------------------------------------------
// shared helpers
// ---------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ size_t cidx(const Geo<T>& g, int b, int t, int ix, int iy, int ic) {
  return ((size_t)(b * g.P + t) * g.S) + (size_t)ix + (size_t)g.n1 * ((size_t)iy + (size_t)g.n2 * ic);
}

// FP32 quotients, roots and the cube root of Newton's starting point from the hardware's approximate
// instructions (PTX rcp.approx, sqrt.approx, lg2.approx, ex2.approx; about one unit in the last place, with
// subnormal operands flushed to zero).  Newton's method corrects its own rounding, and the quotients of
// the results are a few units off at most.  FP64 uses the correctly rounded operations.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float fdiv_fast(float a, float b) { return a * rcp_approx(b); }
__device__ __forceinline__ double fdiv_fast(double a, double b) { return a / b; }
__device__ __forceinline__ float sqrt_fast(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double sqrt_fast(double x) { return sqrt(x); }
// d^(1/3) = 2^(log2(d) / 3) for d > 0 (0 otherwise)
__device__ __forceinline__ float cbrt_start(float d) {
  float l, r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(d));
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(l * (1.f / 3.f)));
  return d > 0.f ? r : 0.f;
}
__device__ __forceinline__ double cbrt_start(double d) { return cbrt(d); }

// Per-cell proximal map of J (section 3, step 2):
//   argmin_{u,v} |u|^2/(2v) + sigma/2 |u - a_m|^2 + sigma/2 (v - a_f)^2.
// With z = sigma v, e = sigma a_f and d = sigma^2 |a_m|^2 / 2 the cubic of the
// paper, 2 (1 + sigma v)^2 (v - a_f) = sigma |a_m|^2, reads
//   q(z) = (1 + z)^2 (z - e) - d = 0,   u = z a_m / (1 + z),  v = z / sigma.
// A root z > 0 exists iff e + d > 0; otherwise (u, v) = (0, 0).  With w = 1 + z
// and c = 1 + e the root satisfies w^2 (w - c) = d, which gives the upper
// bounds w <= c + min(d^(1/3), d/c^2) for c > 0 and w <= min(d^(1/3), sqrt(d/|c|))
// for c <= 0.  q is increasing and convex for z >= max(e, 0), so Newton's
// method from that bound decreases monotonically to the root.
template <typename T>
__device__ __forceinline__ void prox_J(T am0, T am1, T am2, T af, T sigma, T inv_sigma, T& u0, T& u1, T& u2, T& v) {
  const T s2 = am0 * am0 + am1 * am1 + am2 * am2;
  const T e = sigma * af;
  const T d = T(0.5) * sigma * sigma * s2;
  const bool live = e + d > T(0);
  const T c = T(1) + e;
  const T cbd = cbrt_start(d);
  // both starts are computed and one is selected, so that the three channels of a cell interleave
  const T zpos = e + min(cbd, fdiv_fast(d, c * c));                  // c > 0
  const T zneg = min(cbd, sqrt_fast(fdiv_fast(d, fabs(c)))) - T(1);   // c <= 0
  T z = live ? max(c > T(0) ? zpos : zneg, T(0)) : T(0);
  // Stop when the step is below a few units in the last place of the data
  // scale |e| + d + z: near e + d = 0 the root cannot be resolved more finely
  // in this precision, and a purely relative test would never be met there.
  const T tol = (sizeof(T) == 4 ? T(4.0 / 16777216.0) : T(4.0 / 9007199254740992.0)) * (fabs(e) + d);
  const T eps = sizeof(T) == 4 ? T(4.0 / 16777216.0) : T(4.0 / 9007199254740992.0);
  // Newton's method corrects its own rounding, so its steps use the fast
  // division; the result below uses the correctly rounded one.  Three steps
  // are taken unconditionally (the stop rule is met within three on typical
  // cells, and a step from a converged z leaves it in place); the loop runs
  // only while a cell has not met it.
  auto newton = [&]() {
    const T w = T(1) + z;
    const T zme = z - e;
    const T q = w * w * zme - d;
    const T dq = w * (T(2) * zme + w);
    const T step = fdiv_fast(q, dq);
    z -= step;
    return step;
  };
  newton();
  newton();
  T step = newton();
#pragma unroll 1
  for (int it = 3; it < 40 && live && fabs(step) > eps * z + tol; ++it) step = newton();
  z = live ? max(z, T(0)) : T(0);
  const T r = fdiv_fast(z, T(1) + z);
  u0 = r * am0;
  u1 = r * am1;
  u2 = r * am2;
  v = z * inv_sigma;
}

// The same prox with the cubic's root in closed form (Cardano, section 3 "Step 2"; no iteration).
// In w = 1 + z with c = 1 + e the cubic reads w^3 - c w^2 - d = 0; w = t + c/3 gives the depressed
// cubic t^3 + p t + q = 0 with p = -c^2/3 and -q/2 = A = c^3/27 + d/2, and its discriminant
// D = A^2 - c^6/729 = d (c^3/27 + d/4).
// - D >= 0 (always when c > 0): one real root t = r + c^2/(9 r), r = cbrt(A + sqrt D).  The second
//   term is cbrt(A - sqrt D) rewritten through (A + sqrt D)(A - sqrt D) = (c^2/9)^3, which avoids
//   the cancellation of the textbook form.
// - D < 0 (c < 0, small d): three real roots; the largest is t = 2 m cos(acos(A / m^3) / 3), m = |c|/3.
template <typename T>
__device__ __forceinline__ void prox_J_cardano(T am0, T am1, T am2, T af, T sigma, T inv_sigma, T& u0, T& u1, T& u2,
                                               T& v) {
  const T s2 = am0 * am0 + am1 * am1 + am2 * am2;
  const T e = sigma * af;
  const T d = T(0.5) * sigma * sigma * s2;
  if (!(e + d > T(0))) {
    u0 = u1 = u2 = v = T(0);
    return;
  }
  const T c = T(1) + e;
  const T c3_27 = c * c * c * T(1.0 / 27.0);
  const T A = c3_27 + T(0.5) * d;
  const T D = d * (c3_27 + T(0.25) * d);
  T w;
  if (D >= T(0)) {
    const T r = cbrt(A + sqrt(D));
    w = r + fdiv_fast(c * c * T(1.0 / 9.0), r) + c * T(1.0 / 3.0);
  } else {
    const T m = fabs(c) * T(1.0 / 3.0);
    const T arg = fdiv_fast(A, m * m * m);
    w = T(2) * m * cos(acos(min(max(arg, T(-1)), T(1))) * T(1.0 / 3.0)) + c * T(1.0 / 3.0);
  }
  const T z = max(w - T(1), T(0));
  const T rr = fdiv_fast(z, T(1) + z);
  u0 = rr * am0;
  u1 = rr * am1;
  u2 = rr * am2;
  v = z * inv_sigma;
}

#ifndef DYNOT_PROX_CARDANO
#define DYNOT_PROX_CARDANO 0   // 1: the update kernels use the closed form instead of Newton
#endif
template <typename T>
__device__ __forceinline__ void prox_cell(T am0, T am1, T am2, T af, T sigma, T inv_sigma, T& u0, T& u1, T& u2, T& v) {
  if (DYNOT_PROX_CARDANO) prox_J_cardano<T>(am0, am1, am2, af, sigma, inv_sigma, u0, u1, u2, v);
  else prox_J<T>(am0, am1, am2, af, sigma, inv_sigma, u0, u1, u2, v);
}

// ---------------------------------------------------------------------------
// K_D: fused projection correction + prox + dual update + next a
// ---------------------------------------------------------------------------

template <typename T>
struct CellCtx {
  const Geo<T>& g;
  const Arrays<T>& A;
  int b;

  __device__ __forceinline__ T phi(int t, int x, int y, int c) const { return A.phi[cidx(g, b, t, x, y, c)]; }

  // x^{r+1} at the right face of (t, x, y, c) along axis k (3 = time); zero at Neumann boundaries.
  __device__ __forceinline__ T xr(int k, int t, int x, int y, int c) const {
    const size_t i0 = cidx(g, b, t, x, y, c);
    if (k == 0) {
      int x1 = x + 1;
      if (x1 == g.n1) { if (!g.per1) return T(0); x1 = 0; }
      return comp<T>(A.a, i0, 0) + g.s1 * (A.phi[cidx(g, b, t, x1, y, c)] - A.phi[i0]);
    } else if (k == 1) {
      int y1 = y + 1;
      if (y1 == g.n2) { if (!g.per2) return T(0); y1 = 0; }
      return comp<T>(A.a, i0, 1) + g.s2 * (A.phi[cidx(g, b, t, x, y1, c)] - A.phi[i0]);
    } else if (k == 2) {
      int c1 = c + 1;
      if (c1 == g.C) { if (!g.perc) return T(0); c1 = 0; }
      return comp<T>(A.a, i0, 2) + g.sc * (A.phi[cidx(g, b, t, x, y, c1)] - A.phi[i0]);
    } else {
      if (t == g.P - 1) return T(0);
      return comp<T>(A.a, i0, 3) + g.sp * (A.phi[cidx(g, b, t + 1, x, y, c)] - A.phi[i0]);
    }
  }
  // x^{r+1} at the left face = right face of the previous cell (wrapping), or the boundary value
  __device__ __forceinline__ T xl(int k, int t, int x, int y, int c) const {
    if (k == 0) {
      if (x == 0) { if (!g.per1) return T(0); return xr(0, t, g.n1 - 1, y, c); }
      return xr(0, t, x - 1, y, c);
    } else if (k == 1) {
      if (y == 0) { if (!g.per2) return T(0); return xr(1, t, x, g.n2 - 1, c); }
      return xr(1, t, x, y - 1, c);
    } else if (k == 2) {
      if (c == 0) { if (!g.perc) return T(0); return xr(2, t, x, y, g.C - 1); }
      return xr(2, t, x, y, c - 1);
    } else {
      if (t == 0) return A.f0[(size_t)b * g.S + x + (size_t)g.n1 * (y + (size_t)g.n2 * c)];
      return xr(3, t - 1, x, y, c);
    }
  }
  __device__ __forceinline__ T xr_t_or_f1(int t, int x, int y, int c) const {
    if (t == g.P - 1) return A.f1[(size_t)b * g.S + x + (size_t)g.n1 * (y + (size_t)g.n2 * c)];
    return xr(3, t, x, y, c);
  }

  // Steps 2-4 at one cell.  Outputs bbar (4), b^{r+1} (4), the right faces of x^{r+1},
  // K x^{r+1} + (0, f_b^+) and the prox result.
  __device__ __forceinline__ void cell(int t, int x, int y, int c, T bb[4], T bn[4], T xrr[4], T kx[4],
                                       T& U0, T& U1, T& U2, T& V) const {
#pragma unroll
    for (int k = 0; k < 3; ++k) xrr[k] = xr(k, t, x, y, c);
    xrr[3] = xr_t_or_f1(t, x, y, c);
    kx[0] = T(0.5) * (xl(0, t, x, y, c) + xrr[0]);
    kx[1] = T(0.5) * (xl(1, t, x, y, c) + xrr[1]);
    kx[2] = T(0.5) * (xl(2, t, x, y, c) + xrr[2]);
    kx[3] = T(0.5) * (xl(3, t, x, y, c) + xrr[3]);
    const size_t i0 = cidx(g, b, t, x, y, c);
    const v4<T> bv = A.b[i0];
    const T bo[4] = {bv.x, bv.y, bv.z, bv.w};
    const T am0 = kx[0] + bo[0], am1 = kx[1] + bo[1], am2 = kx[2] + bo[2], af = kx[3] + bo[3];
    prox_cell<T>(am0, am1, am2, af, g.sigma, T(1) / g.sigma, U0, U1, U2, V);
    bn[0] = am0 - U0;
    bn[1] = am1 - U1;
    bn[2] = am2 - U2;
    bn[3] = af - V;
#pragma unroll
    for (int k = 0; k < 4; ++k) bb[k] = T(2) * bn[k] - bo[k];
    if (t == g.P - 1) xrr[3] = T(0);  // the f1 value is not a face of x
  }

  __device__ __forceinline__ T bbar_only(int k, int t, int x, int y, int c) const {
    T bb[4], bn[4], xrr[4], kx[4], U0, U1, U2, V;
    cell(t, x, y, c, bb, bn, xrr, kx, U0, U1, U2, V);
    return bb[k];
  }
};

// Residual accumulators (FP64, one set per problem):
//   0: sum |b^{r+1} - b^r|^2   1: sum |K x + (0, f_b^+)|^2   2: sum J(u, v)
//   3: sum <b^{r+1}, w> (the dual value over sigma; w = K x0 + (0, f_b^+))
//   mass[b*P + t]: sum over space of f at time (t+1)/P
constexpr int kAcc = 4;

template <typename T>
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T, bool CHECK, bool WRITE_X>
__global__ void __launch_bounds__(128) k_update(Geo<T> g, Arrays<T> A, double* __restrict__ acc,
                                                double* __restrict__ mass) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  int z = blockIdx.z;
  const int c = z % g.C;
  z /= g.C;
  const int t = z % g.P;
  const int b = z / g.P;
  if (retired(g, b)) return;
  const bool live = x < g.n1;
  double r_db = 0, r_kx = 0, r_J = 0, r_m = 0, r_w = 0;
  if (live) {
    CellCtx<T> cc{g, A, b};
    T bb[4], bn[4], xrr[4], kx[4], U0, U1, U2, V;
    cc.cell(t, x, y, c, bb, bn, xrr, kx, U0, U1, U2, V);
    const size_t i0 = cidx(g, b, t, x, y, c);
    T an[4];
    // a^{r+1} at the right faces: x^{r+1} - tau sigma (bbar_here + bbar_next) / 2
    if (x + 1 < g.n1 || g.per1) {
      const T o = cc.bbar_only(0, t, x + 1 < g.n1 ? x + 1 : 0, y, c);
      an[0] = xrr[0] - g.ts * T(0.5) * (bb[0] + o);
    } else {
      an[0] = T(0);
    }
    if (y + 1 < g.n2 || g.per2) {
      const T o = cc.bbar_only(1, t, x, y + 1 < g.n2 ? y + 1 : 0, c);
      an[1] = xrr[1] - g.ts * T(0.5) * (bb[1] + o);
    } else {
      an[1] = T(0);
    }
    if (c + 1 < g.C || g.perc) {
      const T o = cc.bbar_only(2, t, x, y, c + 1 < g.C ? c + 1 : 0);
      an[2] = xrr[2] - g.ts * T(0.5) * (bb[2] + o);
    } else {
      an[2] = T(0);
    }
    if (t + 1 < g.P) {
      const T o = cc.bbar_only(3, t + 1, x, y, c);
      an[3] = xrr[3] - g.ts * T(0.5) * (bb[3] + o);
    } else {
      an[3] = T(0);
    }
    A.an[i0] = mk4<T>(an[0], an[1], an[2], an[3]);
    A.bn[i0] = mk4<T>(bn[0], bn[1], bn[2], bn[3]);
    if (WRITE_X) A.x[i0] = mk4<T>(xrr[0], xrr[1], xrr[2], xrr[3]);
    if (CHECK) {
      const v4<T> bo4 = A.b[i0];
      const T bo[4] = {bo4.x, bo4.y, bo4.z, bo4.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const double db = (double)bn[k] - (double)bo[k];
        r_db += db * db;
        r_kx += (double)kx[k] * (double)kx[k];
      }
      const double uu = (double)U0 * U0 + (double)U1 * U1 + (double)U2 * U2;
      if (V > T(0)) r_J = uu / (2.0 * (double)V);
      r_m = (double)xrr[3];
      const v4<T> wv = A.w[i0];
      r_w = (double)bn[0] * wv.x + (double)bn[1] * wv.y + (double)bn[2] * wv.z + (double)bn[3] * wv.w;
    }
  }
  if (CHECK) {
    __shared__ double red[4][5];
    r_db = warp_sum<T>(r_db);
    r_kx = warp_sum<T>(r_kx);
    r_J = warp_sum<T>(r_J);
    r_m = warp_sum<T>(r_m);
    r_w = warp_sum<T>(r_w);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
      red[w][0] = r_db;
      red[w][1] = r_kx;
      red[w][2] = r_J;
      red[w][3] = r_m;
      red[w][4] = r_w;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
      double s = 0;
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i][threadIdx.x];
      if (threadIdx.x < 3) atomicAdd(&acc[(size_t)b * kAcc + threadIdx.x], s);
      else if (threadIdx.x == 4) atomicAdd(&acc[(size_t)b * kAcc + 3], s);
      else if (t < g.P - 1) atomicAdd(&mass[(size_t)b * g.P + t], s);
    }
  }
}

// ---------------------------------------------------------------------------
// K_A: r = A a - f_b^- and forward DCT along x and t, per (y, c) row
// ---------------------------------------------------------------------------

// Shared-memory carve-up of the x/t kernels.
template <typename T>
struct XtSmem {
  T* tile;      // [P][ld]
  c2<T>* scr;   // FFT scratch
  c2<T>* tw;    // [n1]
  c2<T>* hw;    // [n1]
  T* Mt;        // [P][PMAX]
  T* cos4;      // dense fallback table [4 n1]
};

struct XtTables {
  const void* tw;    // c2<T>[n1]
  const void* hw;    // c2<T>[n1]
  const void* Mt_f;  // forward t-DCT, [P][PMAX]
  const void* Mt_i;  // inverse t-DCT
  const void* cos4;  // [4 n1]; for a periodic x axis the (cos, sin)(2 pi m / n1) pairs instead
  const void* twt;   // c2<T>[P]: exp(-2 pi i j / P)   (register t-DCT when P == PMAX <= 32)
  const void* hwt;   // c2<T>[P]: exp(-i pi k / (2P))
};

// The time transform runs in registers by FFT when P fills the template width
// (16 or 32) and DYNOT_TFFT is set; otherwise it is the dense matrix product.
#ifndef DYNOT_TFFT
#define DYNOT_TFFT 1
#endif
#ifndef DYNOT_XT_MINB
#define DYNOT_XT_MINB 2   // blocks per SM the forward x/t kernel is compiled for
#endif
#ifndef DYNOT_RHS_UNROLL
#define DYNOT_RHS_UNROLL 8   // time planes of right-hand-side loads in flight per thread
#endif
constexpr int kRhsUnroll = DYNOT_RHS_UNROLL;
#ifndef DYNOT_XTC_MINB
#define DYNOT_XTC_MINB 3  // blocks per SM the inverse x/t kernel is compiled for (measured faster at 3)
#endif
template <int PMAX, int N1>
__device__ __forceinline__ bool t_by_fft(int P) { return DYNOT_TFFT && N1 > 0 && PMAX <= 32 && P == PMAX; }

// Shared-memory layout of the x/t kernels; the same function sizes it on the host.
// The FFT path needs the twiddle tables, the dense path the cosine table.
template <typename T>
__host__ __device__ __forceinline__ size_t xt_layout(XtSmem<T>* s, char* sm, int P, int n1, int PMAX, int scr_elems,
                                                     bool dense) {
  size_t off = 0;
  auto take = [&](size_t bytes) { char* p = sm + off; off += (bytes + 15) & ~size_t(15); return p; };
  T* tile = (T*)take(sizeof(T) * (size_t)(P + 1) * n1);
  c2<T>* scr = (c2<T>*)take(sizeof(c2<T>) * (size_t)scr_elems);
  c2<T>* tw = dense ? nullptr : (c2<T>*)take(sizeof(c2<T>) * n1);
  c2<T>* hw = dense ? nullptr : (c2<T>*)take(sizeof(c2<T>) * n1);
  T* Mt = (T*)take(sizeof(T) * (size_t)P * PMAX);
  T* cos4 = dense ? (T*)take(sizeof(T) * 4 * n1) : nullptr;
  if (s) {
    s->tile = tile; s->scr = scr; s->tw = tw; s->hw = hw; s->Mt = Mt; s->cos4 = cos4;
  }
  return off;
}

// Writes the (t, x) tile [P][n1] of one (y, c) row to dst (cell layout: planes S apart).  FP32 rows whose
// length is a multiple of 4 go out as 16-byte vectors (a plane's n1 / 4 vectors per pass of the block, 256 / (n1 / 4)
// planes at once), which takes a quarter of the store instructions of one cell per thread.
template <typename T>
__device__ __forceinline__ void store_tile_rows(const T* tile, T* __restrict__ dst, size_t S, int P, int n1) {
  if constexpr (std::is_same<T, float>::value) {
    const int nv = n1 >> 2;
    if ((n1 & 3) == 0 && nv <= (int)blockDim.x && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
      const int per = blockDim.x / nv, xv = threadIdx.x % nv, tq = threadIdx.x / nv;
      if (tq < per) {
#pragma unroll 8
        for (int t = tq; t < P; t += per)
          *reinterpret_cast<float4*>(dst + (size_t)t * S + 4 * xv) =
              *reinterpret_cast<const float4*>(tile + t * n1 + 4 * xv);
      }
      return;
    }
  }
  for (int t = 0; t < P; ++t)
    for (int x = threadIdx.x; x < n1; x += blockDim.x) dst[(size_t)t * S + x] = tile[t * n1 + x];
}

// N1 == 0 selects the dense x transform.
template <typename T, int N1, int N2, int PMAX>
__global__ void __launch_bounds__(256, DYNOT_XT_MINB) k_rhs_fwd_xt(Geo<T> g, const v4<T>* __restrict__ ap,
                                                    const T* __restrict__ f0, const T* __restrict__ f1,
                                                    T* __restrict__ rhat, XtTables tb, int scr_elems) {
  extern __shared__ __align__(16) char smraw[];
  const int y = blockIdx.x, c = blockIdx.y, b = blockIdx.z;
  if (retired(g, b)) return;
  const int n1 = g.n1, P = g.P;
  XtSmem<T> s;
  xt_layout<T>(&s, smraw, P, n1, PMAX, scr_elems, N1 == 0);
  const T* as = reinterpret_cast<const T*>(ap);   // component k of cell i at as[4 i + k]
  // tables
  if (N1) load_tables<T>(s.tw, s.hw, (const c2<T>*)tb.tw, (const c2<T>*)tb.hw, n1);
  else for (int j = threadIdx.x; j < 4 * n1; j += blockDim.x) s.cos4[j] = ((const T*)tb.cos4)[j];
  const bool tfft = t_by_fft<PMAX, N1>(P);
  if (tfft) {
    c2<T>* tt = (c2<T>*)s.Mt;
    for (int j = threadIdx.x; j < P; j += blockDim.x) {
      tt[j] = ((const c2<T>*)tb.twt)[j];
      tt[P + j] = ((const c2<T>*)tb.hwt)[j];
    }
  } else {
    for (int j = threadIdx.x; j < P * PMAX; j += blockDim.x) s.Mt[j] = ((const T*)tb.Mt_f)[j];
  }
  pdl_wait();   // a (previous update) is read from here on
  // divergence of a and the time difference with the boundary densities
  const int ym = y > 0 ? y - 1 : (g.per2 ? g.n2 - 1 : -1);
  const int cm = c > 0 ? c - 1 : (g.perc ? g.C - 1 : -1);
  const size_t S = g.S;
  const size_t rowbase = (size_t)b * P * S + (size_t)n1 * (y + (size_t)g.n2 * c);
  const long long dy = ym >= 0 ? (long long)n1 * (ym - y) : 0;                 // offset to the y-1 row
  const long long dc = cm >= 0 ? (long long)n1 * g.n2 * (cm - c) : 0;          // offset to channel c-1
  for (int x = threadIdx.x; x < n1; x += blockDim.x) {
    const int xm = x > 0 ? x - 1 : (g.per1 ? n1 - 1 : -1);
    const size_t sb = (size_t)b * S + x + (size_t)n1 * (y + (size_t)g.n2 * c);
    const T f0v = f0[sb], f1v = f1[sb];
    const size_t c0 = rowbase + x;                 // this cell at t = 0
    const long long dx = xm - x;                   // offset to the x-1 cell (used only when it exists)
    T fprev = f0v;                                 // f face below plane t (f0 at t = 0)
#pragma unroll kRhsUnroll
    for (int t = 0; t < P; ++t) {
      const size_t o = c0 + (size_t)t * S;
      const v4<T> av = ap[o];
      T r = g.s1 * (av.x - (xm >= 0 ? as[4 * (o + dx)] : T(0)));
      r += g.s2 * (av.y - (ym >= 0 ? as[4 * (o + dy) + 1] : T(0)));
      r += g.sc * (av.z - (cm >= 0 ? as[4 * (o + dc) + 2] : T(0)));
      const T fnext = (t == P - 1) ? f1v : av.w;
      r += g.sp * (fnext - fprev);
      fprev = av.w;
      s.tile[t * n1 + x] = r;
    }
  }
  const int Pr = P + (P & 1);  // the pair packing needs an even row count
  if (Pr != P)
    for (int x = threadIdx.x; x < n1; x += blockDim.x) s.tile[P * n1 + x] = T(0);
  __syncthreads();
  Rows<T, 1, 1> rows{s.tile, n1, 0};
  if constexpr (N1 > 0) {
    if (g.per1) DctPow2<T, N1, N2, false, 256, true>::forward(rows, Pr, s.scr, s.tw, s.hw);
    else DctPow2<T, N1, N2, false, 256>::forward(rows, Pr, s.scr, s.tw, s.hw);
  } else {
    if (g.per1) rdft_dense_rows<T, false>(rows, P, n1, false, (T*)s.scr, 2 * scr_elems, (const c2<T>*)s.cos4);
    else dct_dense_rows<T, false>(rows, P, n1, false, (T*)s.scr, 2 * scr_elems, s.cos4);
  }
  // (the FFT path leaves a trailing barrier; the dense path too)
  if constexpr (PMAX <= 32 && N1 > 0) {
    if (tfft) dct_cols_fft<T, PMAX, false, N1 * N2>(s.tile, n1, (const c2<T>*)s.Mt, (const c2<T>*)s.Mt + P);
    else dct_cols<T, PMAX>(s.tile, n1, n1, P, s.Mt);
  } else {
    dct_cols<T, PMAX>(s.tile, n1, n1, P, s.Mt);
  }
  __syncthreads();
  pdl_trigger();
  store_tile_rows<T>(s.tile, rhat + cidx(g, b, 0, 0, y, c), (size_t)g.S, P, n1);
}

// ---------------------------------------------------------------------------
// Split x/t passes, for grids whose whole (t, x) plane of one (y, c) does not fit shared memory (the FP64
// plan at n1 = 512, P = 64).  The same transforms as K_A and K_C in separate launches:
//   k_rhs_cells : r = A a - f_b^- into hat, one cell per thread;
//   k_rows_x    : the DCT-II along x (or its inverse) of kRowsX rows [t][x] of one (y, c) per block, from
//                 src into dst (in place when they are the same array);
//   k_cols_t    : the DCT-II along t (or its inverse) of kColsT columns of one (y, c) per block, in place,
//                 as the dense product with the transform matrix.
// ---------------------------------------------------------------------------
constexpr int kRowsX = 16, kColsT = 128;

template <typename T>
__global__ void __launch_bounds__(256) k_rhs_cells(Geo<T> g, const v4<T>* __restrict__ ap, const T* __restrict__ f0,
                                                   const T* __restrict__ f1, T* __restrict__ r) {
  const long long tot = (long long)g.B * g.N;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < tot; id += (long long)gridDim.x * blockDim.x) {
    long long q = id;
    const int x = q % g.n1; q /= g.n1;
    const int y = q % g.n2; q /= g.n2;
    const int c = q % g.C; q /= g.C;
    const int t = q % g.P;
    const int b = (int)(q / g.P);
    if (retired(g, b)) continue;
    const v4<T> av = ap[id];
    const int xm = x > 0 ? x - 1 : (g.per1 ? g.n1 - 1 : -1);
    const int ym = y > 0 ? y - 1 : (g.per2 ? g.n2 - 1 : -1);
    const int cm = c > 0 ? c - 1 : (g.perc ? g.C - 1 : -1);
    const size_t sb = (size_t)b * g.S + x + (size_t)g.n1 * (y + (size_t)g.n2 * c);
    T v = g.s1 * (av.x - (xm >= 0 ? comp<T>(ap, cidx(g, b, t, xm, y, c), 0) : T(0)));
    v += g.s2 * (av.y - (ym >= 0 ? comp<T>(ap, cidx(g, b, t, x, ym, c), 1) : T(0)));
    v += g.sc * (av.z - (cm >= 0 ? comp<T>(ap, cidx(g, b, t, x, y, cm), 2) : T(0)));
    const T fnext = (t == g.P - 1) ? f1[sb] : av.w;
    const T fprev = (t == 0) ? f0[sb] : comp<T>(ap, id - g.S, 3);
    v += g.sp * (fnext - fprev);
    r[id] = v;
  }
}

// Shared memory of k_rows_x: the row tile, the FFT scratch (or the dense scratch) and the tables.
template <typename T>
__host__ __device__ __forceinline__ size_t rows_x_layout(char* sm, int n1, int scr_elems, bool dense, T** tile,
                                                         c2<T>** scr, c2<T>** tw, c2<T>** hw, T** cos4) {
  size_t off = 0;
  auto take = [&](size_t bytes) { char* p = sm + off; off += (bytes + 15) & ~size_t(15); return p; };
  *tile = (T*)take(sizeof(T) * (size_t)kRowsX * n1);
  *scr = (c2<T>*)take(sizeof(c2<T>) * (size_t)scr_elems);
  *tw = dense ? nullptr : (c2<T>*)take(sizeof(c2<T>) * n1);
  *hw = dense ? nullptr : (c2<T>*)take(sizeof(c2<T>) * n1);
  *cos4 = dense ? (T*)take(sizeof(T) * 4 * n1) : nullptr;
  return off;
}

template <typename T, int N1, int N2, bool INV>
__global__ void __launch_bounds__(256) k_rows_x(Geo<T> g, const T* __restrict__ src, T* __restrict__ dst,
                                                XtTables tb, int scr_elems) {
  extern __shared__ __align__(16) char smraw[];
  const int t0 = blockIdx.x * kRowsX, yc = blockIdx.y, b = blockIdx.z;
  if (retired(g, b)) return;
  const int n1 = g.n1, P = g.P;
  const int nr = min(kRowsX, P - t0), nre = nr + (nr & 1);   // rows of this block, even for the pairs
  T *tile, *cos4;
  c2<T> *scr, *tw, *hw;
  rows_x_layout<T>(smraw, n1, scr_elems, N1 == 0, &tile, &scr, &tw, &hw, &cos4);
  if (N1) load_tables<T>(tw, hw, (const c2<T>*)tb.tw, (const c2<T>*)tb.hw, n1);
  else for (int j = threadIdx.x; j < 4 * n1; j += blockDim.x) cos4[j] = ((const T*)tb.cos4)[j];
  pdl_wait();
  const size_t base = ((size_t)b * P + t0) * g.S + (size_t)yc * n1;   // row t0 of (y, c) = yc
  for (int i = threadIdx.x; i < nre * n1; i += blockDim.x) {
    const int r = i / n1, x = i - r * n1;
    tile[i] = r < nr ? src[base + (size_t)r * g.S + x] : T(0);
  }
  __syncthreads();
  Rows<T, 1, 1> rows{tile, n1, 0};
  if constexpr (N1 > 0) {
    if (g.per1) {
      if (INV) DctPow2<T, N1, N2, false, 256, true>::inverse(rows, nre, scr, tw, hw);
      else DctPow2<T, N1, N2, false, 256, true>::forward(rows, nre, scr, tw, hw);
    } else {
      if (INV) DctPow2<T, N1, N2, false, 256>::inverse(rows, nre, scr, tw, hw);
      else DctPow2<T, N1, N2, false, 256>::forward(rows, nre, scr, tw, hw);
    }
  } else {
    if (g.per1) rdft_dense_rows<T, false>(rows, nr, n1, INV, (T*)scr, 2 * scr_elems, (const c2<T>*)cos4);
    else dct_dense_rows<T, false>(rows, nr, n1, INV, (T*)scr, 2 * scr_elems, cos4);
  }
  __syncthreads();
  pdl_trigger();
  for (int i = threadIdx.x; i < nr * n1; i += blockDim.x) {
    const int r = i / n1, x = i - r * n1;
    dst[base + (size_t)r * g.S + x] = tile[i];
  }
}

template <typename T, int PMAX>
__global__ void __launch_bounds__(kColsT) k_cols_t(Geo<T> g, T* __restrict__ hat, const T* __restrict__ Mt_g) {
  extern __shared__ __align__(16) char smraw[];
  const int x0 = blockIdx.x * kColsT, yc = blockIdx.y, b = blockIdx.z;
  if (retired(g, b)) return;
  const int n1 = g.n1, P = g.P;
  const int w = min(kColsT, n1 - x0);
  T* Mt = (T*)smraw;                  // [P][PMAX]
  T* tile = Mt + (size_t)P * PMAX;    // [P][kColsT]
  for (int j = threadIdx.x; j < P * PMAX; j += blockDim.x) Mt[j] = Mt_g[j];
  pdl_wait();
  const size_t base = (size_t)b * P * g.S + (size_t)yc * n1 + x0;
  for (int i = threadIdx.x; i < P * kColsT; i += blockDim.x) {
    const int t = i / kColsT, x = i - t * kColsT;
    tile[i] = x < w ? hat[base + (size_t)t * g.S + x] : T(0);
  }
  __syncthreads();
  dct_cols<T, PMAX>(tile, kColsT, w, P, Mt);
  __syncthreads();
  pdl_trigger();
  for (int i = threadIdx.x; i < P * kColsT; i += blockDim.x) {
    const int t = i / kColsT, x = i - t * kColsT;
    if (x < w) hat[base + (size_t)t * g.S + x] = tile[i];
  }
}

// K_C: inverse DCT along t and x -> phi
template <typename T, int N1, int N2, int PMAX>
__global__ void __launch_bounds__(256, DYNOT_XTC_MINB) k_inv_xt(Geo<T> g, const T* __restrict__ phihat, T* __restrict__ phi,
                                                XtTables tb, int scr_elems) {
  extern __shared__ __align__(16) char smraw[];
  const int y = blockIdx.x, c = blockIdx.y, b = blockIdx.z;
  if (retired(g, b)) return;
  const int n1 = g.n1, P = g.P;
  XtSmem<T> s;
  xt_layout<T>(&s, smraw, P, n1, PMAX, scr_elems, N1 == 0);
  if (N1) load_tables<T>(s.tw, s.hw, (const c2<T>*)tb.tw, (const c2<T>*)tb.hw, n1);
  else for (int j = threadIdx.x; j < 4 * n1; j += blockDim.x) s.cos4[j] = ((const T*)tb.cos4)[j];
  const bool tfft = t_by_fft<PMAX, N1>(P);
  if (tfft) {
    c2<T>* tt = (c2<T>*)s.Mt;
    for (int j = threadIdx.x; j < P; j += blockDim.x) {
      tt[j] = ((const c2<T>*)tb.twt)[j];
      tt[P + j] = ((const c2<T>*)tb.hwt)[j];
    }
  } else {
    for (int j = threadIdx.x; j < P * PMAX; j += blockDim.x) s.Mt[j] = ((const T*)tb.Mt_i)[j];
  }
  pdl_wait();   // the spectral array (y/colour pass) is read from here on
  // the (t, x) plane of this (y, c), all rows in flight at once
  async_rows<T>(s.tile, n1, phihat + cidx(g, b, 0, 0, y, c), (long long)g.S, P, n1);
  cp_async_wait_all();
  __syncthreads();
  if constexpr (PMAX <= 32 && N1 > 0) {
    if (tfft) dct_cols_fft<T, PMAX, true, N1 * N2>(s.tile, n1, (const c2<T>*)s.Mt, (const c2<T>*)s.Mt + P);
    else dct_cols<T, PMAX>(s.tile, n1, n1, P, s.Mt);
  } else {
    dct_cols<T, PMAX>(s.tile, n1, n1, P, s.Mt);
  }
  __syncthreads();
  const int Pr = P + (P & 1);
  if (Pr != P)
    for (int x = threadIdx.x; x < n1; x += blockDim.x) s.tile[P * n1 + x] = T(0);
  __syncthreads();
  Rows<T, 1, 1> rows{s.tile, n1, 0};
  if constexpr (N1 > 0) {
    if (g.per1) DctPow2<T, N1, N2, false, 256, true>::inverse(rows, Pr, s.scr, s.tw, s.hw);
    else DctPow2<T, N1, N2, false, 256>::inverse(rows, Pr, s.scr, s.tw, s.hw);
  } else {
    if (g.per1) rdft_dense_rows<T, false>(rows, P, n1, true, (T*)s.scr, 2 * scr_elems, (const c2<T>*)s.cos4);
    else dct_dense_rows<T, false>(rows, P, n1, true, (T*)s.scr, 2 * scr_elems, s.cos4);
  }
  pdl_trigger();
  store_tile_rows<T>(s.tile, phi + cidx(g, b, 0, 0, y, c), (size_t)g.S, P, n1);
}

// ---------------------------------------------------------------------------
// K_B: y transform, colour eigen-solve and eigenvalue divide, inverse y
// ---------------------------------------------------------------------------



constexpr int kMaxC = 4;

// Shared-memory layout of the y/colour kernel; the same function sizes it on the host.
// The tile is [c][y][w] with a channel stride padded to 8 (mod 32) words so that
// the interleaved row pairs of the y transform fall into distinct banks.
__host__ __device__ __forceinline__ int yc_cstride(int n2, int W) {
  const int base = n2 * W;
  return base + ((8 - base % 32) + 32) % 32;
}

template <typename T>
__host__ __device__ __forceinline__ size_t yc_layout(char* sm, int C, int n2, int W, int scr_elems, bool dense,
                                                     T** tile, c2<T>** scr, c2<T>** tw, c2<T>** hw, T** cos4,
                                                     T** l2, T** tabs) {
  size_t off = 0;
  auto take = [&](size_t bytes) { char* p = sm + off; off += (bytes + 15) & ~size_t(15); return p; };
  *tile = (T*)take(sizeof(T) * (size_t)C * yc_cstride(n2, W));
  *scr = (c2<T>*)take(sizeof(c2<T>) * (size_t)scr_elems);
  *tw = dense ? nullptr : (c2<T>*)take(sizeof(c2<T>) * n2);
  *hw = dense ? nullptr : (c2<T>*)take(sizeof(c2<T>) * n2);
  *cos4 = dense ? (T*)take(sizeof(T) * 4 * n2) : nullptr;
  *l2 = (T*)take(sizeof(T) * n2);
  *tabs = (T*)take(sizeof(T) * (kMaxC * kMaxC + kMaxC + W));   // Q (padded 4x4), lambda_c, lambda_x of the strip
  return off;
}

struct YcTables {
  const void* tw;      // c2<T>[n2]
  const void* hw;      // c2<T>[n2]
  const void* cos4;    // [4 n2]; for a periodic y axis the (cos, sin)(2 pi m / n2) pairs instead
  const void* lam1;    // T[n1]   eigenvalues along x
  const void* lam2;    // T[n2]
  const void* lamt;    // T[P]
  const double* lam1d; // the same in double
  const double* lam2d;
  const double* lamtd;
  const void* Qc;      // colour eigenbasis, T[C*C], Qc[c*C + j]
  const void* lamc;    // T[C]
  const double* lamcd;
  double lam_fp64;     // eigenvalues below this are divided in FP64
};

// NT threads per block: 12 row pairs of length M1 * M2 per FFT chunk (NT = 12 M1) fill every
// thread for the 3 x 8 = 24 rows of an RGB strip; the dense path uses 256.
template <typename T, int M1, int M2, int W, int NT>
__global__ void __launch_bounds__(NT, 768 / NT) k_solve_yc(Geo<T> g, T* __restrict__ hat, YcTables tb, int scr_elems) {
  extern __shared__ __align__(16) char smraw[];
  const int x0 = blockIdx.x * W, kt = blockIdx.y, b = blockIdx.z;
  if (retired(g, b)) return;
  const int n1 = g.n1, n2 = g.n2, C = g.C;
  const int w_act = min(W, n1 - x0);
  const int cst = yc_cstride(n2, W);
  T *tile, *cos4, *l2, *tabs;
  c2<T> *scr, *tw, *hw;
  yc_layout<T>(smraw, C, n2, W, scr_elems, M1 == 0, &tile, &scr, &tw, &hw, &cos4, &l2, &tabs);
  T* Qs = tabs;                      // [4][4], zero outside C x C
  T* lcs = tabs + kMaxC * kMaxC;     // [4]
  T* l1s = lcs + kMaxC;              // [W]
  if (M1) load_tables<T>(tw, hw, (const c2<T>*)tb.tw, (const c2<T>*)tb.hw, n2);
  else for (int j = threadIdx.x; j < 4 * n2; j += blockDim.x) cos4[j] = ((const T*)tb.cos4)[j];
  for (int j = threadIdx.x; j < n2; j += blockDim.x) l2[j] = ((const T*)tb.lam2)[j];
  if (threadIdx.x < kMaxC * kMaxC) {
    const int c = threadIdx.x / kMaxC, j = threadIdx.x % kMaxC;
    Qs[threadIdx.x] = (c < C && j < C) ? ((const T*)tb.Qc)[c * C + j] : T(0);
  }
  if (threadIdx.x < kMaxC) lcs[threadIdx.x] = threadIdx.x < C ? ((const T*)tb.lamc)[threadIdx.x] : T(0);
  if (threadIdx.x < W) l1s[threadIdx.x] = threadIdx.x < w_act ? ((const T*)tb.lam1)[x0 + threadIdx.x] : T(0);
  pdl_wait();   // the spectral array (forward x/t pass) is read from here on
  // load [c][y][w] (zero beyond the last column so pairs stay well defined); the rows (c, y) of the
  // strip are n1 apart in hat, W wide in the tile: whole-strip asynchronous copies when aligned
  const size_t plane = ((size_t)b * g.P + kt) * g.S + x0;
  constexpr int V = 16 / (int)sizeof(T);
  if (w_act == W && W % V == 0 && n1 % V == 0 && x0 % V == 0 && cst % V == 0 && ((uintptr_t)hat & 15) == 0) {
    constexpr int PER = W / V;
    for (int i = threadIdx.x; i < C * n2 * PER; i += blockDim.x) {
      const int r = i / PER, k = i - r * PER;   // r = c * n2 + y
      const int c = r / n2, yy = r - c * n2;
      cp_async16(tile + c * cst + yy * W + k * V, hat + plane + (size_t)r * n1 + k * V);
    }
  } else {
    for (int c = 0; c < C; ++c) {
      const T* src = hat + plane + (size_t)c * n1 * n2;
      T* dst = tile + c * cst;
      for (int j = threadIdx.x; j < n2 * W; j += blockDim.x) {
        const int w = j % W, y = j / W;
        dst[j] = (w < w_act) ? src[(size_t)y * n1 + w] : T(0);
      }
    }
  }
  cp_async_wait_all();
  __syncthreads();
  Rows<T, W, W> rows{tile, cst, 1};
  const int nrows = C * W;
  if constexpr (M1 > 0) {
    if (g.per2) DctPow2<T, M1, M2, true, NT, true>::forward(rows, nrows, scr, tw, hw);
    else DctPow2<T, M1, M2, true, NT>::forward(rows, nrows, scr, tw, hw);
  } else {
    if (g.per2) rdft_dense_rows<T, true>(rows, nrows, n2, false, (T*)scr, 2 * scr_elems, (const c2<T>*)cos4);
    else dct_dense_rows<T, true>(rows, nrows, n2, false, (T*)scr, 2 * scr_elems, cos4);
  }
  // colour eigen-solve: phi_c = sum_j Q[c][j] (sum_c' Q[c'][j] r_c') / lambda(kx, ky, j, kt)
  {
    const T lt = ((const T*)tb.lamt)[kt];
    const float thr = (float)tb.lam_fp64;
    T Q[kMaxC][kMaxC], lc[kMaxC];
#pragma unroll
    for (int c = 0; c < kMaxC; ++c) {
      lc[c] = lcs[c];
#pragma unroll
      for (int j = 0; j < kMaxC; ++j) Q[c][j] = Qs[c * kMaxC + j];
    }
    for (int i = threadIdx.x; i < n2 * W; i += blockDim.x) {
      const int w = i % W, ky = i / W;
      if (w >= w_act) continue;
      T r[kMaxC], co[kMaxC];
#pragma unroll
      for (int cc = 0; cc < kMaxC; ++cc) r[cc] = cc < C ? tile[cc * cst + i] : T(0);
      const T lxyt = l1s[w] + l2[ky] + lt;
#pragma unroll
      for (int j = 0; j < kMaxC; ++j) {
        T s = 0;
#pragma unroll
        for (int cc = 0; cc < kMaxC; ++cc) s = fma(Q[cc][j], r[cc], s);
        const T lam = lxyt + lc[j];
        if (j >= C || !(lam > T(0))) {
          co[j] = T(0);     // padding, or the zero eigenvalue of the pseudo-inverse
        } else if ((float)lam < thr) {
          // low modes: eigenvalue and quotient in double precision
          const double ld = tb.lam1d[x0 + w] + tb.lam2d[ky] + tb.lamtd[kt] + tb.lamcd[j];
          co[j] = ld > 0.0 ? (T)((double)s / ld) : T(0);
        } else {
          co[j] = fdiv_fast(s, lam);   // a few ulp; the low modes above take the exact FP64 path
        }
      }
#pragma unroll
      for (int cc = 0; cc < kMaxC; ++cc) {
        if (cc >= C) continue;
        T s = 0;
#pragma unroll
        for (int j = 0; j < kMaxC; ++j) s = fma(Q[cc][j], co[j], s);
        tile[cc * cst + i] = s;
      }
    }
  }
  __syncthreads();
  if constexpr (M1 > 0) {
    if (g.per2) DctPow2<T, M1, M2, true, NT, true>::inverse(rows, nrows, scr, tw, hw);
    else DctPow2<T, M1, M2, true, NT>::inverse(rows, nrows, scr, tw, hw);
  } else {
    if (g.per2) rdft_dense_rows<T, true>(rows, nrows, n2, true, (T*)scr, 2 * scr_elems, (const c2<T>*)cos4);
    else dct_dense_rows<T, true>(rows, nrows, n2, true, (T*)scr, 2 * scr_elems, cos4);
  }
  pdl_trigger();
  for (int c = 0; c < C; ++c) {
    T* dst = hat + plane + (size_t)c * n1 * n2;
    const T* src = tile + c * cst;
    for (int j = threadIdx.x; j < n2 * W; j += blockDim.x) {
      const int w = j % W, y = j / W;
      if (w < w_act) dst[(size_t)y * n1 + w] = src[j];
    }
  }
}

}  // namespace dynot

namespace dynot {

// ---------------------------------------------------------------------------
// K_D, tiled: the same steps as k_update for grids whose x and y axes are
// Neumann, with every neighbour's prox result shared instead of recomputed.
//
// A block of 32 x 8 threads covers 32 x-columns and 8 y-rows; each thread owns
// one (x, y) column with all C colour cells and streams over a chunk of time
// planes, carrying the time neighbour in registers.  bbar at x+1 comes from
// the next lane (warp shuffle), bbar at y+1 from the next row (shared memory),
// bbar at c+1 from the same thread.  Blocks overlap by one column and one row:
// the last lane and the last row only compute the prox their neighbours need
// and write nothing, unless they sit on the last column / row of the grid.
// A time chunk [t0, t0 + TC) also computes plane t0 + TC for bbar_f of its last face.
// ---------------------------------------------------------------------------
constexpr int kTX = 32, kTY = 8;
#ifndef DYNOT_UPD_MINB
#define DYNOT_UPD_MINB 3   // blocks per SM the tiled update is compiled for
#endif

// Per-block partial sums of the residual check: [problem][block][kPart] with
// 0: |b+ - b|^2, 1: |K x + (0, f_b^+)|^2, 2: J(u, v), 3 + t: mass of the time slice t (t < 64),
// kPartW = 67: <b+, w> (the dual value over sigma).
constexpr int kPart = 68;
constexpr int kPartW = 67;

// Strides of the tiled update's arrays: a time plane, a row, a colour channel and a problem of the cell arrays,
// and a row and a problem of the boundary densities.  Grids with rows along y: S, n1, n1 n2, P S; n1, S.  A
// batch of hue problems runs with its problems as the rows (cell arrays [problem][t][bin], densities
// [problem][bin]): n1, P n1, -, 0; n1, 0 -- with the y difference factor set to zero the rows do not couple.
struct TileLayout {
  int plane, row, chan;
  long long prob;
  int frow;
  long long fprob;
};

// Per-block partial sums of a check (called by every thread of a 32 x 8 block after its plane loop):
// FP64 sums of the threads' compensated partials, written to part[problem][block][...].
template <typename T>
__device__ __forceinline__ void block_check_partials(const KSum<T>& r_db, const KSum<T>& r_kx, const KSum<T>& r_J,
                                                     const KSum<T>& r_w, int lane, int row, int nch, int b, int t0,
                                                     int tend, int P, double* __restrict__ part,
                                                     const double (&smass)[64]) {
  __shared__ double red[kTY][4];
  double d[4] = {(double)r_db.s - (double)r_db.c, (double)r_kx.s - (double)r_kx.c, (double)r_J.s - (double)r_J.c,
                 (double)r_w.s - (double)r_w.c};
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int q = 0; q < 4; ++q) d[q] += __shfl_xor_sync(0xffffffffu, d[q], o);
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < 4; ++q) red[row][q] = d[q];
  __syncthreads();
  const int tid = lane + kTX * row;
  const int nblk = gridDim.x * gridDim.y * nch;    // blocks of one problem
  const int jb = ((blockIdx.z % nch) * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  double* pp = part + ((size_t)b * nblk + jb) * kPart;
  if (tid < 4) {
    double sum = 0;
    for (int i = 0; i < kTY; ++i) sum += red[i][tid];
    pp[tid < 3 ? tid : kPartW] = sum;
  }
  for (int t = tid; t < 64; t += kTX * kTY) pp[3 + t] = (t >= t0 && t < tend && t < P - 1) ? smass[t] : 0.0;
}

// The body of the tiled update.  INTERIOR: every thread of the block has both x and y neighbours
// inside the grid, so the boundary tests fold away (about three quarters of the blocks at 256^2).
template <typename T, int C, bool CHECK, bool WRITE_X, bool INTERIOR, bool PXY>
__device__ __forceinline__ void update_tiled_body(const Geo<T>& g, const Arrays<T>& A, int TC, const TileLayout& Lt,
                                                  double* __restrict__ part, T (&sbb)[2][kTY][kTX][C],
                                                  double (&smass)[64]) {
  const int lane = threadIdx.x, row = threadIdx.y;
  const int x = blockIdx.x * (kTX - 1) + lane;
  const int y = blockIdx.y * (kTY - 1) + row;
  const int nch = (g.P + TC - 1) / TC;
  const int b = blockIdx.z / nch;
  if (retired(g, b)) return;
  const int t0 = (blockIdx.z % nch) * TC;
  const int tend = min(t0 + TC, g.P);           // planes [t0, tend) are written
  const int tlast = min(tend, g.P - 1);          // planes [t0, tlast] are computed
  // periodic x / y (edge blocks only): threads past the last cell stand for cells 0, 1, ... so that the
  // shuffles and the shared-memory exchange see the wrapped neighbours; every cell is written by a lane
  // that is not the block's halo lane or row (the grid has ceil(n / (kT - 1)) blocks on a periodic axis)
  const bool px = PXY && !INTERIOR && g.per1, py = PXY && !INTERIOR && g.per2;
  const bool vx = INTERIOR || x < g.n1, vy = INTERIOR || y < g.n2;
  const bool live = vx && vy;
  const int xs = vx ? x : (px ? x % g.n1 : g.n1 - 1);   // clamped (Neumann) or wrapped (periodic)
  const int ys = vy ? y : (py ? y % g.n2 : g.n2 - 1);
  const bool out = live && (lane < kTX - 1 || (!INTERIOR && !px && x == g.n1 - 1)) &&
                   (row < kTY - 1 || (!INTERIOR && !py && y == g.n2 - 1));
  const bool hasR = INTERIOR || px || xs < g.n1 - 1, hasL = INTERIOR || px || xs > 0;
  const bool hasU = INTERIOR || py || ys < g.n2 - 1, hasD = INTERIOR || py || ys > 0;
  // offsets to the four neighbours in the plane (wrapped on a periodic axis)
  // 32-bit offsets from per-thread column bases (problem sizes stay below 2^31 cells)
  const int S = Lt.plane, sy = Lt.row, sc = Lt.chan;
  const int dxr = (px && xs == g.n1 - 1) ? 1 - g.n1 : 1;
  const int dxl = (px && xs == 0) ? g.n1 - 1 : -1;
  const int dyu = (py && ys == g.n2 - 1) ? (1 - g.n2) * sy : sy;
  const int dyd = (py && ys == 0) ? (g.n2 - 1) * sy : -sy;
  const size_t col = (size_t)b * Lt.prob + xs + (size_t)sy * ys;
  const size_t col2 = (size_t)b * Lt.fprob + xs + (size_t)Lt.frow * ys;
  const v4<T>* __restrict__ pa = A.a + col;
  const v4<T>* __restrict__ pb = A.b + col;
  const T* __restrict__ pas = reinterpret_cast<const T*>(pa);   // scalar component loads: pas[4 o + k]
  const T* __restrict__ pph = A.phi + col;
  const T* __restrict__ pf0 = A.f0 + col2;
  const T* __restrict__ pf1 = A.f1 + col2;
  v4<T>* __restrict__ qa = A.an + col;
  v4<T>* __restrict__ qb = A.bn + col;
  const T s1 = g.s1, s2 = g.s2, scl = g.sc, sp = g.sp, ts = g.ts, half = T(0.5);
  const T isg = T(1) / g.sigma;
  const bool perc = g.perc;
  if (CHECK) {
    for (int i = threadIdx.x + kTX * threadIdx.y; i < 64; i += kTX * kTY) smass[i] = 0.0;
  }
  // residual, energy and dual terms: per-thread compensated partial sums in the working precision,
  // every sum across threads in FP64
  KSum<T> r_db, r_kx, r_J, r_w;
  pdl_wait();   // phi (inverse x/t pass) and the state are read from here on

  T phic[C], xfp[C], bbfp[C];
  // the next a of the previous plane's faces along x, y, colour: stored together with its f face,
  // which is known one plane later
  T cax[C], cay[C], cac[C];
  // state entering plane t0: phi(t0), x_f at the face t0 - 1 (or f0)
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const int o = t0 * S + c * sc;
    phic[c] = pph[o];
    xfp[c] = (t0 == 0) ? pf0[c * sc] : pas[4 * (o - S) + 3] + sp * (phic[c] - pph[o - S]);
    bbfp[c] = T(0);
    cax[c] = cay[c] = cac[c] = T(0);
  }

#pragma unroll 1
  for (int t = t0; t <= tlast; ++t) {
    const int pt = t * S;
    const bool write_plane = t < tend;
    const bool tnext = t + 1 < g.P;
    T bb[C][4], bn[C][4], xr[C][4], phn[C];
    // loads of this plane (all channels first, so that they overlap)
    v4<T> la[C], lb4[C];
    T phy[C], phd[C], la1d[C], la0l[C], phl[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const int o = pt + c * sc;
      la[c] = pa[o];
      lb4[c] = pb[o];
      phn[c] = tnext ? pph[o + S] : T(0);
      phy[c] = hasU ? pph[o + dyu] : T(0);
      phd[c] = hasD ? pph[o + dyd] : T(0);
      la1d[c] = hasD ? pas[4 * (o + dyd) + 1] : T(0);
      la0l[c] = (lane == 0 && hasL) ? pas[4 * (o + dxl)] : T(0);
      phl[c] = (lane == 0 && hasL) ? pph[o + dxl] : T(0);
    }
    T lb[C][4];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      lb[c][0] = lb4[c].x;
      lb[c][1] = lb4[c].y;
      lb[c][2] = lb4[c].z;
      lb[c][3] = lb4[c].w;
    }
    // right faces of x^{r+1}
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const T ph = phic[c];
      T phx = __shfl_down_sync(0xffffffffu, ph, 1);
      if (lane == kTX - 1 && hasR) phx = pph[pt + c * sc + dxr];
      xr[c][0] = hasR ? la[c].x + s1 * (phx - ph) : T(0);
      xr[c][1] = hasU ? la[c].y + s2 * (phy[c] - ph) : T(0);
      xr[c][3] = tnext ? la[c].w + sp * (phn[c] - ph) : pf1[c * sc];
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const int c1 = (c + 1 == C) ? 0 : c + 1;
      const bool hasC = perc || (c + 1 < C);
      xr[c][2] = hasC ? la[c].z + scl * (phic[c1] - phic[c]) : T(0);
    }
    // left faces, interpolation to the cell, prox, dual update
#pragma unroll
    for (int c = 0; c < C; ++c) {
      T xlx = __shfl_up_sync(0xffffffffu, xr[c][0], 1);
      if (lane == 0) xlx = la0l[c] + s1 * (phic[c] - phl[c]);
      if (!hasL) xlx = T(0);
      const T xly = hasD ? la1d[c] + s2 * (phic[c] - phd[c]) : T(0);
      const int cm = (c == 0) ? C - 1 : c - 1;
      const T xlc = (perc || c > 0) ? xr[cm][2] : T(0);
      const T k0 = half * (xlx + xr[c][0]);
      const T k1 = half * (xly + xr[c][1]);
      const T k2 = half * (xlc + xr[c][2]);
      const T k3 = half * (xfp[c] + xr[c][3]);
      const T am0 = k0 + lb[c][0], am1 = k1 + lb[c][1], am2 = k2 + lb[c][2], af = k3 + lb[c][3];
      T U0, U1, U2, V;
      prox_cell<T>(am0, am1, am2, af, g.sigma, isg, U0, U1, U2, V);
      bn[c][0] = am0 - U0;
      bn[c][1] = am1 - U1;
      bn[c][2] = am2 - U2;
      bn[c][3] = af - V;
#pragma unroll
      for (int k = 0; k < 4; ++k) bb[c][k] = T(2) * bn[c][k] - lb[c][k];
      if (CHECK && out && write_plane) {
        // per-cell terms in the working precision, sums compensated, then in FP64
        T db2 = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const T db = bn[c][k] - lb[c][k];
          db2 = fma(db, db, db2);
        }
        r_db.add(db2);
        r_kx.add(k0 * k0 + k1 * k1 + k2 * k2 + k3 * k3);
        if (V > T(0)) r_J.add(fdiv_fast(U0 * U0 + U1 * U1 + U2 * U2, T(2) * V));
        const v4<T> wv = A.w[col + pt + c * sc];
        r_w.add(bn[c][0] * wv.x + bn[c][1] * wv.y + bn[c][2] * wv.z + bn[c][3] * wv.w);
      }
    }
    // neighbours' bbar: x+1 by shuffle, y+1 through shared memory
    const int par = t & 1;
#pragma unroll
    for (int c = 0; c < C; ++c) sbb[par][row][lane][c] = bb[c][1];
    __syncthreads();
    if (out && t > t0) {
      // plane t-1 is complete with its f face t-1 (between planes t-1 and t), owned by this chunk when t > t0
#pragma unroll
      for (int c = 0; c < C; ++c)
        qa[pt - S + c * sc] = mk4<T>(cax[c], cay[c], cac[c], xfp[c] - ts * half * (bbfp[c] + bb[c][3]));
    }
    if (write_plane) {
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const T bxn = __shfl_down_sync(0xffffffffu, bb[c][0], 1);
        const T byn = (row + 1 < kTY) ? sbb[par][row + 1][lane][c] : T(0);
        const int c1 = (c + 1 == C) ? 0 : c + 1;
        const bool hasC = perc || (c + 1 < C);
        cax[c] = hasR ? xr[c][0] - ts * half * (bb[c][0] + bxn) : T(0);
        cay[c] = hasU ? xr[c][1] - ts * half * (bb[c][1] + byn) : T(0);
        cac[c] = hasC ? xr[c][2] - ts * half * (bb[c][2] + bb[c1][2]) : T(0);
        if (out) {
          const int o = pt + c * sc;
          qb[o] = mk4<T>(bn[c][0], bn[c][1], bn[c][2], bn[c][3]);
          if (WRITE_X) A.x[col + o] = mk4<T>(xr[c][0], xr[c][1], xr[c][2], tnext ? xr[c][3] : T(0));
        }
      }
      if (CHECK && tnext) {
        T mt = 0;
        if (out) {
#pragma unroll
          for (int c = 0; c < C; ++c) mt += xr[c][3];
        }
        double m = (double)mt;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
        if (lane == 0) atomicAdd(&smass[t], m);
      }
    }
    // carry to the next plane
#pragma unroll
    for (int c = 0; c < C; ++c) {
      xfp[c] = xr[c][3];
      bbfp[c] = bb[c][3];
      phic[c] = phn[c];
    }
  }
  // the last plane of the problem has no f face (f1 is a boundary value): store it with zero there
  if (out && tlast == tend - 1) {
#pragma unroll
    for (int c = 0; c < C; ++c) qa[tlast * S + c * sc] = mk4<T>(cax[c], cay[c], cac[c], T(0));
  }
  pdl_trigger();
  if (CHECK) block_check_partials<T>(r_db, r_kx, r_J, r_w, lane, row, nch, b, t0, tend, g.P, part, smass);
}

// PXY: the edge blocks handle periodic x / y (a separate instance, so that the Neumann kernel keeps its
// register allocation)
template <typename T, int C, bool CHECK, bool WRITE_X, bool PXY>
__global__ void __launch_bounds__(kTX * kTY, DYNOT_UPD_MINB) k_update_tiled(Geo<T> g, Arrays<T> A, int TC,
                                                                TileLayout Lt, double* __restrict__ part) {
  __shared__ T sbb[2][kTY][kTX][C];   // bbar_y exchange, double-buffered by plane parity
  __shared__ double smass[64];
  const int x0 = blockIdx.x * (kTX - 1), y0 = blockIdx.y * (kTY - 1);
  const bool interior = x0 >= 1 && x0 + kTX < g.n1 && y0 >= 1 && y0 + kTY < g.n2;
  if (interior) update_tiled_body<T, C, CHECK, WRITE_X, true, PXY>(g, A, TC, Lt, part, sbb, smass);
  else update_tiled_body<T, C, CHECK, WRITE_X, false, PXY>(g, A, TC, Lt, part, sbb, smass);
}


// Sum the per-block partials of each problem (one block per problem) into acc and mass: one warp per quantity
// (the 3 residual and energy terms, the P mass sums, the dual term), lanes striding over the blocks in a fixed order.
static __global__ void k_reduce_check(const double* __restrict__ part, int nblk, int P, double* __restrict__ acc,
                               double* __restrict__ mass, const int* __restrict__ active) {
  const int b = blockIdx.x;
  if (active != nullptr && active[b] == 0) return;
  const double* pb = part + (size_t)b * nblk * kPart;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int qi = warp; qi < 4 + P; qi += nw) {
    const int q = qi < 3 + P ? qi : kPartW;
    double s = 0;
    for (int j = lane; j < nblk; j += 32) s += pb[(size_t)j * kPart + q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      if (q < 3) acc[(size_t)b * kAcc + q] = s;
      else if (q == kPartW) acc[(size_t)b * kAcc + 3] = s;
      else if (q - 3 < P) mass[(size_t)b * P + (q - 3)] = s;
    }
  }
}

}  // namespace dynot
