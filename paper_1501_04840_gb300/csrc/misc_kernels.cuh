// Data-movement kernels around the iteration: input validation, mass
// rescaling (section 4), conversion between the paper's compact face layout
// (section 2) and the cell-aligned internal layout, the step-1 operand
// a = x - tau sigma K^T bbar, the projection correction x = a - A^T phi, and
// the per-cell prox entry point.
#pragma once
#include "common.cuh"
#include "rgb_kernels.cuh"

namespace dynot {

// Per pair: [0] sum f0, [1] sum f1, [2] min f0, [3] min f1, [4] non-finite count (doubles).
constexpr int kChk = 5;

static __global__ void k_check_inputs(const float* __restrict__ f0, const float* __restrict__ f1, int S,
                               double* __restrict__ out) {
  const int b = blockIdx.y;
  double s0 = 0, s1 = 0, bad = 0;
  float m0 = INFINITY, m1 = INFINITY;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S; i += gridDim.x * blockDim.x) {
    const float a = f0[(size_t)b * S + i], c = f1[(size_t)b * S + i];
    if (!isfinite(a) || !isfinite(c)) bad += 1;
    s0 += a;
    s1 += c;
    m0 = fminf(m0, a);
    m1 = fminf(m1, c);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    bad += __shfl_xor_sync(0xffffffffu, bad, o);
    m0 = fminf(m0, __shfl_xor_sync(0xffffffffu, m0, o));
    m1 = fminf(m1, __shfl_xor_sync(0xffffffffu, m1, o));
  }
  __shared__ double sh[32][5];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    sh[w][0] = s0; sh[w][1] = s1; sh[w][2] = m0; sh[w][3] = m1; sh[w][4] = bad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a0 = 0, a1 = 0, mm0 = INFINITY, mm1 = INFINITY, bb = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      a0 += sh[i][0]; a1 += sh[i][1]; bb += sh[i][4];
      mm0 = fmin(mm0, sh[i][2]); mm1 = fmin(mm1, sh[i][3]);
    }
    double* o = out + (size_t)b * kChk;
    atomicAdd(&o[0], a0);
    atomicAdd(&o[1], a1);
    atomicAdd(&o[4], bb);
    // min via compare-and-swap on the bit pattern of non-negative doubles is not
    // order preserving for negatives; use a loop on the double value instead
    for (int q = 2; q <= 3; ++q) {
      const double v = q == 2 ? mm0 : mm1;
      unsigned long long* addr = (unsigned long long*)&o[q];
      unsigned long long old = *addr, assumed;
      do {
        assumed = old;
        if (__longlong_as_double(assumed) <= v) break;
        old = atomicCAS(addr, assumed, __double_as_longlong(v));
      } while (assumed != old);
    }
  }
}

template <typename T>
__global__ void k_scale_boundary(const float* __restrict__ f0, const float* __restrict__ f1, int S,
                                 const double* __restrict__ sc, T* __restrict__ g0, T* __restrict__ g1) {
  const int b = blockIdx.y;
  const double s0 = sc[2 * b], s1 = sc[2 * b + 1];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S; i += gridDim.x * blockDim.x) {
    g0[(size_t)b * S + i] = (T)((double)f0[(size_t)b * S + i] * s0);
    g1[(size_t)b * S + i] = (T)((double)f1[(size_t)b * S + i] * s1);
  }
}

// Compact layout of component k (0..2 faces, 3 = f) of one problem; returns the
// compact index of the internal slot (t, x, y, c) or -1 if the slot is not a
// variable of the model (Neumann boundary face, f at slot P-1).
struct Compact {
  int n[3], per[3], P, d;
  long long off[4];   // offsets of m_0, m_1, m_2, f inside one problem's packed path
  long long len[4];
  long long total;    // packed floats per problem

  __host__ __device__ long long index(int k, int t, int x, int y, int c) const {
    int i[3] = {x, y, c};
    int dim[3] = {n[0], n[1], n[2]};
    if (k == 3) {
      if (t >= P - 1) return -1;
    } else {
      if (k >= d) return -1;
      if (per[k]) {
        i[k] = (i[k] + 1) % n[k];   // internal face right of cell i = paper face i + 1
      } else {
        if (i[k] == n[k] - 1) return -1;
        dim[k] = n[k] - 1;
      }
    }
    return off[k] + i[0] + (long long)dim[0] * (i[1] + (long long)dim[1] * (i[2] + (long long)dim[2] * t));
  }
};

// internal (T, four components per cell, scaled by `scale`) <- packed (float)
template <typename T>
__global__ void k_unpack_path(Geo<T> g, Compact cp, const float* __restrict__ packed, double scale, v4<T>* xo) {
  const long long tot = (long long)g.B * g.N;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < tot; id += (long long)gridDim.x * blockDim.x) {
    long long r = id;
    const int x = r % g.n1; r /= g.n1;
    const int y = r % g.n2; r /= g.n2;
    const int c = r % g.C; r /= g.C;
    const int t = r % g.P;
    const int b = (int)(r / g.P);
    T v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const long long ci = cp.index(k, t, x, y, c);
      v[k] = ci < 0 ? T(0) : (T)((double)packed[(long long)b * cp.total + ci] * scale);
    }
    xo[id] = mk4<T>(v[0], v[1], v[2], v[3]);
  }
}

// packed (float, times scale) <- internal; dst[k] may be separate arrays (stride per problem lenk)
template <typename T>
__global__ void k_pack_path(Geo<T> g, Compact cp, const v4<T>* xi, double scale,
                            float* __restrict__ packed, float* d0, float* d1, float* d2, float* d3) {
  const long long tot = (long long)g.B * g.N;
  float* ds[4] = {d0, d1, d2, d3};
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < tot; id += (long long)gridDim.x * blockDim.x) {
    long long r = id;
    const int x = r % g.n1; r /= g.n1;
    const int y = r % g.n2; r /= g.n2;
    const int c = r % g.C; r /= g.C;
    const int t = r % g.P;
    const int b = (int)(r / g.P);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const long long ci = cp.index(k, t, x, y, c);
      if (ci < 0) continue;
      const float v = (float)((double)comp<T>(xi, id, k) * scale);
      if (packed) packed[(long long)b * cp.total + ci] = v;
      if (ds[k]) ds[k][(long long)b * cp.len[k] + ci - cp.off[k]] = v;
    }
  }
}

// a = x - tau sigma K^T bbar at the right faces (step 1 of Algorithm 1).
template <typename T>
__global__ void k_make_a(Geo<T> g, const v4<T>* __restrict__ x, const v4<T>* __restrict__ bb, v4<T>* __restrict__ a) {
  const long long tot = (long long)g.B * g.N;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < tot; id += (long long)gridDim.x * blockDim.x) {
    long long r = id;
    const int ix = r % g.n1; r /= g.n1;
    const int iy = r % g.n2; r /= g.n2;
    const int ic = r % g.C; r /= g.C;
    const int t = r % g.P;
    const int b = (int)(r / g.P);
    T out[4];
    // x axis
    {
      int j = ix + 1;
      bool ok = true;
      if (j == g.n1) { ok = g.per1; j = 0; }
      out[0] = ok ? comp<T>(x, id, 0) - g.ts * T(0.5) * (comp<T>(bb, id, 0) + comp<T>(bb, cidx(g, b, t, j, iy, ic), 0)) : T(0);
    }
    {
      int j = iy + 1;
      bool ok = true;
      if (j == g.n2) { ok = g.per2; j = 0; }
      out[1] = ok ? comp<T>(x, id, 1) - g.ts * T(0.5) * (comp<T>(bb, id, 1) + comp<T>(bb, cidx(g, b, t, ix, j, ic), 1)) : T(0);
    }
    {
      int j = ic + 1;
      bool ok = true;
      if (j == g.C) { ok = g.perc; j = 0; }
      out[2] = ok ? comp<T>(x, id, 2) - g.ts * T(0.5) * (comp<T>(bb, id, 2) + comp<T>(bb, cidx(g, b, t, ix, iy, j), 2)) : T(0);
    }
    out[3] = (t + 1 < g.P) ? comp<T>(x, id, 3) - g.ts * T(0.5) * (comp<T>(bb, id, 3) + comp<T>(bb, cidx(g, b, t + 1, ix, iy, ic), 3)) : T(0);
    a[id] = mk4<T>(out[0], out[1], out[2], out[3]);
  }
}

// Dual of a fixed point of step 2 of Algorithm 1 for a given path x: there
// y = K x + (0, f_b^+) and 0 = grad J(y) + sigma (y - K x - (0, f_b^+) - b), so
// b = grad J(y) / sigma.  For J(u, v) = |u|^2 / (2 v) (section 2) the gradient
// depends on the velocity w = u / v alone: grad J = (w, -|w|^2 / 2).  v is
// clamped below by vmin and |w| above by wmax (an optimal path on the domain
// moves no mass faster than the domain's diameter per unit time).  Cells with
// v < vsup start from b = 0 (where the density vanishes the dual of an optimal
// path lies anywhere in the subdifferential of J at 0, which this formula does
// not predict).
template <typename T>
__global__ void k_dual_init(Geo<T> g, const v4<T>* __restrict__ x, const T* __restrict__ f0, const T* __restrict__ f1,
                            T inv_sigma, T vmin, T wmax, T vsup, v4<T>* __restrict__ bo) {
  const long long tot = (long long)g.B * g.N;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < tot; id += (long long)gridDim.x * blockDim.x) {
    long long r = id;
    const int ix = r % g.n1; r /= g.n1;
    const int iy = r % g.n2; r /= g.n2;
    const int ic = r % g.C; r /= g.C;
    const int t = r % g.P;
    const int b = (int)(r / g.P);
    // left faces: the right face of the previous cell (wrapping on periodic axes, zero on Neumann ones)
    T left[3];
    left[0] = ix > 0 ? comp<T>(x, cidx(g, b, t, ix - 1, iy, ic), 0) : (g.per1 ? comp<T>(x, cidx(g, b, t, g.n1 - 1, iy, ic), 0) : T(0));
    left[1] = iy > 0 ? comp<T>(x, cidx(g, b, t, ix, iy - 1, ic), 1) : (g.per2 ? comp<T>(x, cidx(g, b, t, ix, g.n2 - 1, ic), 1) : T(0));
    left[2] = ic > 0 ? comp<T>(x, cidx(g, b, t, ix, iy, ic - 1), 2) : (g.perc ? comp<T>(x, cidx(g, b, t, ix, iy, g.C - 1), 2) : T(0));
    T u[3];
    for (int k = 0; k < 3; ++k) u[k] = T(0.5) * (left[k] + comp<T>(x, id, k));   // right faces are zero where absent
    const size_t s = (size_t)b * g.S + ix + (size_t)g.n1 * (iy + (size_t)g.n2 * ic);
    const T fl = t == 0 ? f0[s] : comp<T>(x, cidx(g, b, t - 1, ix, iy, ic), 3);
    const T fr = t == g.P - 1 ? f1[s] : comp<T>(x, id, 3);
    const T vraw = T(0.5) * (fl + fr);
    const T v = max(vraw, vmin);
    const T on = vraw >= vsup ? T(1) : T(0);
    T w[3] = {on * u[0] / v, on * u[1] / v, on * u[2] / v};
    const T w2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    const T lim = w2 > wmax * wmax ? wmax / sqrt(w2) : T(1);
    for (int k = 0; k < 3; ++k) w[k] *= lim;
    bo[id] = mk4<T>(w[0] * inv_sigma, w[1] * inv_sigma, w[2] * inv_sigma,
                    -T(0.5) * (w[0] * w[0] + w[1] * w[1] + w[2] * w[2]) * inv_sigma);
  }
}

// w = K x0 + (0, f_b^+) at the cells (S_M m0 and S_F f0 + f_b^+ of section 2) for the least-norm feasible
// path x0 = (m0, f0): the dual value of a check is sigma <b, w> (the dual function of the problem at
// p = sigma b, with the infimum over C_d taken at x0).
template <typename T>
__global__ void k_dual_weights(Geo<T> g, const v4<T>* __restrict__ x, const T* __restrict__ f0,
                               const T* __restrict__ f1, v4<T>* __restrict__ w) {
  const long long tot = (long long)g.B * g.N;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < tot; id += (long long)gridDim.x * blockDim.x) {
    long long r = id;
    const int ix = r % g.n1; r /= g.n1;
    const int iy = r % g.n2; r /= g.n2;
    const int ic = r % g.C; r /= g.C;
    const int t = r % g.P;
    const int b = (int)(r / g.P);
    T left[3];
    left[0] = ix > 0 ? comp<T>(x, cidx(g, b, t, ix - 1, iy, ic), 0) : (g.per1 ? comp<T>(x, cidx(g, b, t, g.n1 - 1, iy, ic), 0) : T(0));
    left[1] = iy > 0 ? comp<T>(x, cidx(g, b, t, ix, iy - 1, ic), 1) : (g.per2 ? comp<T>(x, cidx(g, b, t, ix, g.n2 - 1, ic), 1) : T(0));
    left[2] = ic > 0 ? comp<T>(x, cidx(g, b, t, ix, iy, ic - 1), 2) : (g.perc ? comp<T>(x, cidx(g, b, t, ix, iy, g.C - 1), 2) : T(0));
    const size_t s = (size_t)b * g.S + ix + (size_t)g.n1 * (iy + (size_t)g.n2 * ic);
    const T fl = t == 0 ? f0[s] : comp<T>(x, cidx(g, b, t - 1, ix, iy, ic), 3);
    const T fr = t == g.P - 1 ? f1[s] : comp<T>(x, id, 3);
    w[id] = mk4<T>(T(0.5) * (left[0] + comp<T>(x, id, 0)), T(0.5) * (left[1] + comp<T>(x, id, 1)),
                   T(0.5) * (left[2] + comp<T>(x, id, 2)), T(0.5) * (fl + fr));
  }
}

// x = a - A^T phi at the right faces (the correction of the projection).
template <typename T>
__global__ void k_correct(Geo<T> g, Arrays<T> A) {
  const long long tot = (long long)g.B * g.N;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < tot; id += (long long)gridDim.x * blockDim.x) {
    long long r = id;
    const int ix = r % g.n1; r /= g.n1;
    const int iy = r % g.n2; r /= g.n2;
    const int ic = r % g.C; r /= g.C;
    const int t = r % g.P;
    const int b = (int)(r / g.P);
    CellCtx<T> cc{g, A, b};
    A.x[id] = mk4<T>(cc.xr(0, t, ix, iy, ic), cc.xr(1, t, ix, iy, ic), cc.xr(2, t, ix, iy, ic), cc.xr(3, t, ix, iy, ic));
  }
}

// bbar = 2 b - bprev and type conversion helpers
template <typename T>
__global__ void k_axpby(long long n, T alpha, const T* __restrict__ x, T beta, const T* __restrict__ y,
                        T* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = alpha * x[i] + (y ? beta * y[i] : T(0));
}

template <typename T>
__global__ void k_fill(long long n, T v, T* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = v;
}

template <typename To, typename Ti>
__global__ void k_convert(long long n, const Ti* __restrict__ in, To* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (To)in[i];
}

// component k of an interleaved array <-> a plain float array of n cells
template <typename T>
__global__ void k_comp_in(long long n, const float* __restrict__ in, v4<T>* __restrict__ out, int k) {
  T* o = reinterpret_cast<T*>(out);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    o[4 * i + k] = (T)in[i];
}
template <typename T>
__global__ void k_comp_out(long long n, const v4<T>* __restrict__ in, int k, float* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (float)comp<T>(in, i, k);
}
// component k of bbar = 2 b - bprev, formed in T
template <typename T>
__global__ void k_bbar_out(long long n, const v4<T>* __restrict__ b, const v4<T>* __restrict__ bprev, int k,
                           float* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (float)(T(2) * comp<T>(b, i, k) - comp<T>(bprev, i, k));
}

template <bool CARDANO>
static __global__ void k_prox_cells(int count, int ncomp, float sigma, const float* __restrict__ am,
                                    const float* __restrict__ af, float* __restrict__ u, float* __restrict__ v) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const float a0 = am[i];
    const float a1 = ncomp > 1 ? am[(size_t)count + i] : 0.f;
    const float a2 = ncomp > 2 ? am[2 * (size_t)count + i] : 0.f;
    float u0, u1, u2, vv;
    if (CARDANO) prox_J_cardano<float>(a0, a1, a2, af[i], sigma, 1.f / sigma, u0, u1, u2, vv);
    else prox_J<float>(a0, a1, a2, af[i], sigma, 1.f / sigma, u0, u1, u2, vv);
    u[i] = u0;
    if (ncomp > 1) u[(size_t)count + i] = u1;
    if (ncomp > 2) u[2 * (size_t)count + i] = u2;
    v[i] = vv;
  }
}

}  // namespace dynot
