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

// ---------------------------------------------------------------------------
// The real DFT along the bins as a dense matrix product (FP32 plans with at most kHueGemmMax bins and at
// least kHueGemmRows rows, where the product fills the GPU; single pairs keep the per-row kernels): the
// transform of all B P rows at once is C = R W^T with W[slot][i] the basis of the real Fourier slots
// (forward) or its inverse with the weights 1, 2, ..., 2, (1) / n (inverse, stored transposed).
//   H_R  hue_rhs  : r = A a - f_b^- per cell (one thread per cell) into a row array;
//   H_G  gemm_nt  : C[M][N] = sum_k A[m][k] B[n][k], 64 x 64 tiles of 4 x 4 outputs per thread, K in steps
//                   of 16 through shared memory.
// ---------------------------------------------------------------------------
constexpr int kHueGemmMax = 1024, kHueGemmRows = 512;

template <typename T>
__global__ void __launch_bounds__(256) k_hue_rhs(Geo<T> g, const v4<T>* __restrict__ ap, const T* __restrict__ f0,
                                                 const T* __restrict__ f1, T* __restrict__ r) {
  const int n = g.n1, P = g.P;
  const long long tot = (long long)g.B * P * n;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < tot; id += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(id % n);
    const long long row = id / n;
    const int t = (int)(row % P), b = (int)(row / P);
    if (retired(g, b)) continue;
    const int im = i > 0 ? i - 1 : n - 1;   // periodic
    const v4<T> av = ap[id];
    T v = g.s1 * (av.x - comp<T>(ap, id - i + im, 0));
    const T fnext = (t == P - 1) ? f1[(size_t)b * n + i] : av.w;
    const T fprev = (t == 0) ? f0[(size_t)b * n + i] : comp<T>(ap, id - n, 3);
    v += g.sp * (fnext - fprev);
    r[id] = v;
  }
}

static __global__ void __launch_bounds__(128) k_gemm_nt(int M, int N, int K, const float* __restrict__ A,
                                                 const float* __restrict__ Bm, float* __restrict__ C) {
  // 128 threads, 8 x 4 outputs each; K in steps of 32 through two shared-memory buffers: the global loads of
  // the next step are in flight (in registers) while the products of this one run, one barrier per step
  constexpr int BK = 32, LD = 68;
  __shared__ __align__(16) float As[2][BK][LD];
  __shared__ __align__(16) float Bs[2][BK][LD];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // columns 4 tx .. 4 tx + 3, rows 8 ty .. 8 ty + 7
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  // loads: element q of this thread is row (tid >> 3) + 16 (q >> 2), k (tid & 7) + 8 (q & 3) of the step; a
  // warp reads 32-byte runs of four rows, and its transposed stores hit 32 different banks
  const int lk = threadIdx.x & 7, lr = threadIdx.x >> 3;
  float ra[16], rb[16];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int r = lr + 16 * (q >> 2), k = k0 + lk + 8 * (q & 3);
      ra[q] = (k < K && m0 + r < M) ? A[(size_t)(m0 + r) * K + k] : 0.f;
      rb[q] = (k < K && n0 + r < N) ? Bm[(size_t)(n0 + r) * K + k] : 0.f;
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      As[buf][lk + 8 * (q & 3)][lr + 16 * (q >> 2)] = ra[q];
      Bs[buf][lk + 8 * (q & 3)][lr + 16 * (q >> 2)] = rb[q];
    }
  };
  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  fetch(0);
  stash(0);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < K; k0 += BK) {
    const bool more = k0 + BK < K;
    if (more) fetch(k0 + BK);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      // each run of 16 terms is summed on its own and then added to the total, which keeps the rounding
      // error of a sum over K terms near that of 16 + K / 16 additions
      float part[8][4];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) part[i][j] = 0.f;
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) {
        const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][16 * h + kk][8 * ty]);
        const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][16 * h + kk][8 * ty + 4]);
        const float4 b = *reinterpret_cast<const float4*>(&Bs[buf][16 * h + kk][4 * tx]);
        const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) part[i][j] = fmaf(av[i], bv[j], part[i][j]);
      }
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += part[i][j];
    }
    if (more) stash(buf ^ 1);   // buffer buf ^ 1 was last read before the previous barrier
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int m = m0 + 8 * ty + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int nn = n0 + 4 * tx + j;
      if (nn < N) C[(size_t)m * N + nn] = acc[i][j];
    }
  }
}

// C[z][m][n] = sum_k A[m][k] B[z][k][n] for every batch z (A row-major [M][K]; B, C row-major [K][N], [M][N]
// per batch, batch stride `bs`), the time transforms of all slot columns of the hue rows at once, with the
// per-step partial sums of k_gemm_nt.  DIV divides every output by its eigenvalue lamt[m] + lam[n] (zero
// mode -> 0; below lam_fp64 in double), as k_hue_t does between its two products.
template <bool DIV>
__global__ void __launch_bounds__(256) k_gemm_tn(int M, int N, int K, const float* __restrict__ A,
                                                 const float* __restrict__ Bm, float* __restrict__ C, long long bs,
                                                 HueTables tb) {
  __shared__ __align__(16) float As[16][68];
  __shared__ __align__(16) float Bs[16][68];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  const float* Bz = Bm + (size_t)blockIdx.z * bs;
  float* Cz = C + (size_t)blockIdx.z * bs;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = 0; k0 < K; k0 += 16) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = threadIdx.x + 256 * q;
      const int r = idx >> 4, kk = idx & 15;         // A: row r of the tile, k kk
      As[kk][r] = (m0 + r < M && k0 + kk < K) ? A[(size_t)(m0 + r) * K + k0 + kk] : 0.f;
      const int kb = idx >> 6, c = idx & 63;         // B: k kb of the tile, column c
      Bs[kb][c] = (k0 + kb < K && n0 + c < N) ? Bz[(size_t)(k0 + kb) * N + n0 + c] : 0.f;
    }
    __syncthreads();
    float part[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) part[i][j] = 0.f;
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      const float4 a = *reinterpret_cast<const float4*>(&As[kk][4 * ty]);
      const float4 b = *reinterpret_cast<const float4*>(&Bs[kk][4 * tx]);
      const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) part[i][j] = fmaf(av[i], bv[j], part[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] += part[i][j];
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + 4 * ty + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int nn = n0 + 4 * tx + j;
      if (nn >= N) continue;
      float v = acc[i][j];
      if (DIV) {
        const float lam = ((const float*)tb.lam)[nn] + ((const float*)tb.lamt)[m];
        if (!(lam > 0.f)) v = 0.f;
        else if ((double)lam < tb.lam_fp64) v = (float)((double)v / (tb.lamd[nn] + tb.lamtd[m]));
        else v = v / lam;
      }
      Cz[(size_t)m * N + nn] = v;
    }
  }
}

// The time transforms of the hue rows with the divide between them, in one launch for P <= 64: block
// (column block, problem z) takes X = hat[z][0:P][n0:n0+64] into shared memory, forms Y = (Mf X) / lambda
// there (the forward DCT along t and the eigen-divide of k_gemm_tn<true>) and writes Mi Y back to the same
// place (k_gemm_tn<false>).  Mf [k][t] and Mi [t][k] are held transposed, so that the four rows of a thread
// are one 16-byte read; the sums run in the same groups of 16 terms as k_gemm_tn's.
constexpr int kHueTdivMaxP = 64, kHueTdivLD = 68;
constexpr size_t kHueTdivSmem = sizeof(float) * 3 * 64 * kHueTdivLD;

static __global__ void __launch_bounds__(256) k_hue_tdiv(int P, int N, const float* __restrict__ Mf,
                                                  const float* __restrict__ Mi, float* __restrict__ hat,
                                                  long long bs, HueTables tb) {
  extern __shared__ __align__(16) float tsm[];
  constexpr int LD = kHueTdivLD;
  float* MfT = tsm;              // [t][k]
  float* MiT = tsm + 64 * LD;    // [k][t]
  float* X = tsm + 128 * LD;     // [t][n], then Y [k][n]
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int n0 = blockIdx.x * 64;
  float* hz = hat + (size_t)blockIdx.y * bs;
  {
    // all 48 loads of this thread in flight at once, then the shared-memory stores
    float vm[16], vi[16], vx[16];
    const int c = threadIdx.x & 63;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int r = (threadIdx.x >> 6) + 4 * q;   // row r, column c of the P x P matrices (zero outside)
      const bool in = r < P && c < P;
      vm[q] = in ? Mf[(size_t)r * P + c] : 0.f;
      vi[q] = in ? Mi[(size_t)r * P + c] : 0.f;
      vx[q] = (r < P && n0 + c < N) ? hz[(size_t)r * N + n0 + c] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int r = (threadIdx.x >> 6) + 4 * q;
      MfT[c * LD + r] = vm[q];
      MiT[c * LD + r] = vi[q];
      X[r * LD + c] = vx[q];
    }
  }
  __syncthreads();
  // products of the 4 x 4 outputs of this thread, in runs of 16 terms over the padded 64
  auto product = [&](const float* AT, float (&acc)[4][4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k0 = 0; k0 < P; k0 += 16) {
      float part[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) part[i][j] = 0.f;
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) {
        const float4 a = *reinterpret_cast<const float4*>(&AT[(k0 + kk) * LD + 4 * ty]);
        const float4 b = *reinterpret_cast<const float4*>(&X[(k0 + kk) * LD + 4 * tx]);
        const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) part[i][j] = fmaf(av[i], bv[j], part[i][j]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += part[i][j];
    }
  };
  float acc[4][4];
  product(MfT, acc);
  __syncthreads();   // every thread is done with X: it now takes Y
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = 4 * ty + i;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int nn = n0 + 4 * tx + j;
      float v = 0.f;
      if (m < P && nn < N) {
        v = acc[i][j];
        const float lam = ((const float*)tb.lam)[nn] + ((const float*)tb.lamt)[m];
        if (!(lam > 0.f)) v = 0.f;
        else if ((double)lam < tb.lam_fp64) v = (float)((double)v / (tb.lamd[nn] + tb.lamtd[m]));
        else v = v / lam;
      }
      X[m * LD + 4 * tx + j] = v;
    }
  }
  __syncthreads();
  product(MiT, acc);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int t = 4 * ty + i;
    if (t >= P) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int nn = n0 + 4 * tx + j;
      if (nn < N) hz[(size_t)t * N + nn] = acc[i][j];
    }
  }
}

}  // namespace dynot
