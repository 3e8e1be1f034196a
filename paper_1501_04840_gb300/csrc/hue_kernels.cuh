// Poisson solve of the hue variant (section 5): one periodic axis of n bins and
// P time intervals, A A^T = n^2 Delta_{n,per} (x) I + p^2 Delta_p (x) I
// (section 3, the derivation case of the paper).
//
// Along the periodic axis the DFT diagonalises Delta_{n,per} with eigenvalues
// 4 sin^2(pi j / n), equal for j and n - j.  The pseudo-inverse therefore only
// needs the real Fourier basis (cos and sin pairs), which keeps everything real:
//   slot 0 = sum r_i, slots 2j-1, 2j = sum r_i cos, sum r_i sin (2 pi i j / n),
//   slot n-1 = sum r_i (-1)^i for even n.
// The time axis uses the DCT-II as on the RGB path.
//
//   H_A  hue_fwd  : r = A a - f_b^- and the forward real DFT, per time row.
//   H_B  hue_t    : forward DCT along t, divide, inverse DCT, per slot column.
//   H_C  hue_inv  : inverse real DFT -> phi, per time row.
// The cell update is the shared kernel K_D with n2 = C = 1.
#pragma once
#include "common.cuh"
#include "rgb_kernels.cuh"

namespace dynot {

struct HueTables {
  const void* cs;      // c2<T>[n]: (cos, sin)(2 pi m / n)
  const void* lam;     // T[n] eigenvalue of each slot
  const double* lamd;
  const void* lamt;    // T[P]
  const double* lamtd;
  const void* Mt_f;    // [P][PMAX]
  const void* Mt_i;
  double lam_fp64;
};

template <typename T>
__device__ __forceinline__ T hue_basis(const c2<T>* cs, int n, int slot, int i) {
  if (slot == 0) return T(1);
  if ((n & 1) == 0 && slot == n - 1) return (i & 1) ? T(-1) : T(1);
  const int j = (slot + 1) >> 1;
  const c2<T> w = cs[(int)(((long long)i * j) % n)];
  return (slot & 1) ? w.x : w.y;
}

template <typename T>
__global__ void __launch_bounds__(256) k_hue_fwd(Geo<T> g, CPtr4<T> ap, const T* __restrict__ f0,
                                                 const T* __restrict__ f1, T* __restrict__ hat, HueTables tb) {
  extern __shared__ __align__(16) char smraw[];
  const int t = blockIdx.x, b = blockIdx.y;
  const int n = g.n1, P = g.P;
  T* row = (T*)smraw;
  c2<T>* cs = (c2<T>*)(smraw + ((sizeof(T) * n + 15) & ~size_t(15)));
  for (int m = threadIdx.x; m < n; m += blockDim.x) cs[m] = ((const c2<T>*)tb.cs)[m];
  const T* ax = ap.p[0];
  const T* af = ap.p[3];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int im = i > 0 ? i - 1 : n - 1;  // periodic
    const size_t i0 = (size_t)(b * P + t) * n + i;
    T r = g.s1 * (ax[i0] - ax[(size_t)(b * P + t) * n + im]);
    const T fnext = (t == P - 1) ? f1[(size_t)b * n + i] : af[i0];
    const T fprev = (t == 0) ? f0[(size_t)b * n + i] : af[i0 - n];
    r += g.sp * (fnext - fprev);
    row[i] = r;
  }
  __syncthreads();
  for (int slot = threadIdx.x; slot < n; slot += blockDim.x) {
    // four interleaved partial sums: shorter rounding chains and independent FMAs
    T acc[4] = {0, 0, 0, 0};
    int i = 0;
    for (; i + 3 < n; i += 4) {
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fma(row[i + q], hue_basis<T>(cs, n, slot, i + q), acc[q]);
    }
    for (; i < n; ++i) acc[0] = fma(row[i], hue_basis<T>(cs, n, slot, i), acc[0]);
    hat[(size_t)(b * P + t) * n + slot] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
  }
}

template <typename T, int PMAX>
__global__ void __launch_bounds__(128) k_hue_t(Geo<T> g, T* __restrict__ hat, HueTables tb) {
  extern __shared__ __align__(16) char smraw[];
  const int P = g.P, n = g.n1, b = blockIdx.y;
  T* Mf = (T*)smraw;
  T* Mi = Mf + PMAX * PMAX;
  for (int j = threadIdx.x; j < P * PMAX; j += blockDim.x) {
    Mf[j] = ((const T*)tb.Mt_f)[j];
    Mi[j] = ((const T*)tb.Mt_i)[j];
  }
  __syncthreads();
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= n) return;
  T v[PMAX], w[PMAX];
#pragma unroll
  for (int t = 0; t < PMAX; ++t) v[t] = t < P ? hat[(size_t)(b * P + t) * n + slot] : T(0);
  const T ls = ((const T*)tb.lam)[slot];
#pragma unroll
  for (int k = 0; k < PMAX; ++k) {
    if (k >= P) { w[k] = T(0); continue; }
    T acc = 0;
#pragma unroll
    for (int t = 0; t < PMAX; ++t) acc = fma(Mf[k * PMAX + t], v[t], acc);
    const T lam = ls + ((const T*)tb.lamt)[k];
    if (!(lam > T(0))) {
      acc = T(0);
    } else if ((double)lam < tb.lam_fp64) {
      acc = (T)((double)acc / (tb.lamd[slot] + tb.lamtd[k]));
    } else {
      acc = acc / lam;
    }
    w[k] = acc;
  }
  for (int t = 0; t < P; ++t) {
    T acc = 0;
#pragma unroll
    for (int k = 0; k < PMAX; ++k) acc = fma(Mi[t * PMAX + k], w[k], acc);
    hat[(size_t)(b * P + t) * n + slot] = acc;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_hue_inv(Geo<T> g, const T* __restrict__ hat, T* __restrict__ phi,
                                                 HueTables tb) {
  extern __shared__ __align__(16) char smraw[];
  const int t = blockIdx.x, b = blockIdx.y;
  const int n = g.n1, P = g.P;
  T* row = (T*)smraw;
  c2<T>* cs = (c2<T>*)(smraw + ((sizeof(T) * n + 15) & ~size_t(15)));
  for (int m = threadIdx.x; m < n; m += blockDim.x) cs[m] = ((const c2<T>*)tb.cs)[m];
  for (int i = threadIdx.x; i < n; i += blockDim.x) row[i] = hat[(size_t)(b * P + t) * n + i];
  __syncthreads();
  const T invn = T(1) / T(n);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    // slots 1..n-1 carry weight 2 except the Nyquist slot of even n (weight 1)
    T acc[4] = {0, 0, 0, 0};
    const int last = (n & 1) ? n : n - 1;
    int slot = 1;
    for (; slot + 3 < last; slot += 4) {
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fma(row[slot + q], hue_basis<T>(cs, n, slot + q, i), acc[q]);
    }
    for (; slot < last; ++slot) acc[0] = fma(row[slot], hue_basis<T>(cs, n, slot, i), acc[0]);
    T sum = T(2) * ((acc[0] + acc[1]) + (acc[2] + acc[3])) + row[0];
    if (!(n & 1)) sum += row[n - 1] * hue_basis<T>(cs, n, n - 1, i);
    phi[(size_t)(b * P + t) * n + i] = sum * invn;
  }
}

}  // namespace dynot
