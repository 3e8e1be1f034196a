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
__global__ void __launch_bounds__(256) k_hue_fwd(Geo<T> g, const v4<T>* __restrict__ ap, const T* __restrict__ f0,
                                                 const T* __restrict__ f1, T* __restrict__ hat, HueTables tb) {
  extern __shared__ __align__(16) char smraw[];
  const int t = blockIdx.x, b = blockIdx.y;
  if (retired(g, b)) return;
  const int n = g.n1, P = g.P;
  T* row = (T*)smraw;
  c2<T>* cs = (c2<T>*)(smraw + ((sizeof(T) * n + 15) & ~size_t(15)));
  for (int m = threadIdx.x; m < n; m += blockDim.x) cs[m] = ((const c2<T>*)tb.cs)[m];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int im = i > 0 ? i - 1 : n - 1;  // periodic
    const size_t i0 = (size_t)(b * P + t) * n + i;
    const v4<T> av = ap[i0];
    T r = g.s1 * (av.x - comp<T>(ap, (size_t)(b * P + t) * n + im, 0));
    const T fnext = (t == P - 1) ? f1[(size_t)b * n + i] : av.w;
    const T fprev = (t == 0) ? f0[(size_t)b * n + i] : comp<T>(ap, i0 - n, 3);
    r += g.sp * (fnext - fprev);
    row[i] = r;
  }
  __syncthreads();
  for (int slot = threadIdx.x; slot < n; slot += blockDim.x) {
    // four interleaved partial sums: shorter rounding chains and independent FMAs.  The basis
    // index (i j) mod n of the cos / sin slots advances by 4 j per step instead of a modulo per term.
    T acc[4] = {0, 0, 0, 0};
    int i = 0;
    if (slot == 0 || ((n & 1) == 0 && slot == n - 1)) {
      // the constant slot and, for even n, the alternating Nyquist slot
      const bool alt = slot != 0;
      for (; i + 3 < n; i += 4) {
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = fma(row[i + q], (alt && ((i + q) & 1)) ? T(-1) : T(1), acc[q]);
      }
    } else {
      const bool use_cos = slot & 1;
      const int j = (slot + 1) >> 1;
      int idx[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) idx[q] = (int)(((long long)q * j) % n);
      const int step = (int)((4LL * j) % n);
      for (; i + 3 < n; i += 4) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const c2<T> w = cs[idx[q]];
          acc[q] = fma(row[i + q], use_cos ? w.x : w.y, acc[q]);
          idx[q] += step;
          if (idx[q] >= n) idx[q] -= n;
        }
      }
    }
    for (; i < n; ++i) acc[0] = fma(row[i], hue_basis<T>(cs, n, slot, i), acc[0]);
    hat[(size_t)(b * P + t) * n + slot] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
  }
}

// Shared memory of k_hue_t: the two DCT matrices with padded rows, and one column per slot of the
// input and of the divided spectrum.
template <typename T, int PMAX>
__host__ __device__ constexpr size_t hue_t_smem() {
  return sizeof(T) * (2 * (size_t)PMAX * (PMAX + 1) + 2 * (size_t)(256 / PMAX) * PMAX);
}
template <typename T>
__host__ __device__ inline size_t hue_t_smem_for(int pmax) {
  return pmax == 16 ? hue_t_smem<T, 16>() : (pmax == 32 ? hue_t_smem<T, 32>() : hue_t_smem<T, 64>());
}

// 256 threads = 256 / PMAX slot columns x PMAX time indices: thread (slot, k) forms the k-th DCT
// coefficient of its column and divides it, then (after a barrier) the k-th time sample of the inverse.
template <typename T, int PMAX>
__global__ void __launch_bounds__(256) k_hue_t(Geo<T> g, T* __restrict__ hat, HueTables tb) {
  extern __shared__ __align__(16) char smraw[];
  constexpr int SL = 256 / PMAX, LD = PMAX + 1;
  const int P = g.P, n = g.n1, b = blockIdx.y;
  if (retired(g, b)) return;
  T* Mf = (T*)smraw;            // [k][t], row stride LD
  T* Mi = Mf + PMAX * LD;       // [t][k]
  T* v = Mi + PMAX * LD;        // [SL][PMAX] input columns
  T* w = v + SL * PMAX;         // [SL][PMAX] divided spectra
  for (int j = threadIdx.x; j < P * PMAX; j += blockDim.x) {
    const int r = j / PMAX, c = j - r * PMAX;
    Mf[r * LD + c] = ((const T*)tb.Mt_f)[j];
    Mi[r * LD + c] = ((const T*)tb.Mt_i)[j];
  }
  const int sl = threadIdx.x / PMAX, k = threadIdx.x - sl * PMAX;
  const int slot = blockIdx.x * SL + sl;
  const bool act = slot < n && k < P;
  v[sl * PMAX + k] = act ? hat[(size_t)(b * P + k) * n + slot] : T(0);
  __syncthreads();
  T acc = 0;
  if (act) {
#pragma unroll 16
    for (int t = 0; t < PMAX; ++t) acc = fma(Mf[k * LD + t], v[sl * PMAX + t], acc);
    const T lam = ((const T*)tb.lam)[slot] + ((const T*)tb.lamt)[k];
    if (!(lam > T(0))) {
      acc = T(0);
    } else if ((double)lam < tb.lam_fp64) {
      acc = (T)((double)acc / (tb.lamd[slot] + tb.lamtd[k]));
    } else {
      acc = acc / lam;
    }
  }
  w[sl * PMAX + k] = act ? acc : T(0);
  __syncthreads();
  if (act) {
    T y = 0;
#pragma unroll 16
    for (int kk = 0; kk < PMAX; ++kk) y = fma(Mi[k * LD + kk], w[sl * PMAX + kk], y);
    hat[(size_t)(b * P + k) * n + slot] = y;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_hue_inv(Geo<T> g, const T* __restrict__ hat, T* __restrict__ phi,
                                                 HueTables tb) {
  extern __shared__ __align__(16) char smraw[];
  const int t = blockIdx.x, b = blockIdx.y;
  if (retired(g, b)) return;
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
    // slots s, s+1 (cos, sin of frequency j) and s+2, s+3 (frequency j+1) for odd s: the basis
    // indices i j and i (j+1) mod n advance by 2 i per step of 4 slots
    int ia = i % n, ib = (int)((2LL * i) % n);
    const int step = (int)((2LL * i) % n);
    for (; slot + 3 < last; slot += 4) {
      const c2<T> wa = cs[ia], wb = cs[ib];
      acc[0] = fma(row[slot], wa.x, acc[0]);
      acc[1] = fma(row[slot + 1], wa.y, acc[1]);
      acc[2] = fma(row[slot + 2], wb.x, acc[2]);
      acc[3] = fma(row[slot + 3], wb.y, acc[3]);
      ia += step;
      if (ia >= n) ia -= n;
      ib += step;
      if (ib >= n) ib -= n;
    }
    for (; slot < last; ++slot) acc[0] = fma(row[slot], hue_basis<T>(cs, n, slot, i), acc[0]);
    T sum = T(2) * ((acc[0] + acc[1]) + (acc[2] + acc[3])) + row[0];
    if (!(n & 1)) sum += row[n - 1] * hue_basis<T>(cs, n, n - 1, i);
    phi[(size_t)(b * P + t) * n + i] = sum * invn;
  }
}

}  // namespace dynot
