// Shared-memory DCT-II engine for the Poisson solve of section 3 (step 1).
//
// Forward:  X[k] = sum_{n<N} x[n] cos(pi k (2n+1) / (2N))   (unnormalised DCT-II)
// Inverse:  the exact inverse of the forward map (DCT-III with weights 1/N, 2/N).
// Forward followed by inverse is the identity, so the eigenvalue divide of the
// Poisson solve needs no normalisation factors: the paper's orthonormal C_p
// differs from this map only by a diagonal scaling, which commutes with the
// diagonal of eigenvalues.
//
// Power-of-two lengths use Makhoul's reduction of the DCT-II of a real sequence
// to a DFT of the same length (J. Makhoul, "A fast cosine transform in one and
// two dimensions", IEEE Trans. ASSP 28(1), 1980):
//     v[n] = x[2n], v[N-1-n] = x[2n+1];  X[k] = Re(exp(-i pi k/(2N)) V[k]),
// with two real rows packed into one complex sequence (z = v_a + i v_b,
// V_a = (Z_k + conj Z_{N-k})/2, V_b = (Z_k - conj Z_{N-k})/(2i)).  The DFT of
// length N = N1*N2 is Bailey's four-step split: N1-point DFTs in registers,
// twiddles, a transpose through shared memory, N2-point DFTs in registers.
// Each register DFT is an unrolled radix-2 Cooley-Tukey decimation in time.
// Other lengths use the dense cosine sum (O(N) per output).
#pragma once
#include "common.cuh"

namespace dynot {

template <int R> struct Log2 { static constexpr int v = 1 + Log2<R / 2>::v; };
template <> struct Log2<1> { static constexpr int v = 0; };

__host__ __device__ constexpr int bitrev_c(int i, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r = (r << 1) | ((i >> b) & 1);
  return r;
}

// In-register DFT of length R (power of two):
//   Z[k] = sum_n z[n] W^{nk},  W = exp(-2 pi i / R) (forward) or its conjugate (INV).
// twN[j] = exp(-2 pi i j / NT) with R | NT supplies W_R^e = twN[e * NT / R].
template <typename T, int R, int NT, bool INV>
__device__ __forceinline__ void dft_reg(c2<T> (&z)[R], const c2<T>* __restrict__ twN) {
  constexpr int L = Log2<R>::v;
  c2<T> a[R];
#pragma unroll
  for (int i = 0; i < R; ++i) a[bitrev_c(i, L)] = z[i];
#pragma unroll
  for (int stage = 0; stage < L; ++stage) {
    const int m = 2 << stage;
#pragma unroll
    for (int k = 0; k < R; k += m) {
#pragma unroll
      for (int j = 0; j < m / 2; ++j) {
        c2<T> t = a[k + j + m / 2];
        if (j != 0) {
          if (4 * j == m) {          // W_m^{m/4} = -i (forward), +i (inverse)
            t = INV ? mk2<T>(-t.y, t.x) : mk2<T>(t.y, -t.x);
          } else {
            const c2<T> w = twN[j * (NT / m)];
            t = INV ? cmulc<T>(t, w) : cmul<T>(t, w);
          }
        }
        const c2<T> u = a[k + j];
        a[k + j] = cadd<T>(u, t);
        a[k + j + m / 2] = csub<T>(u, t);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < R; ++i) z[i] = a[i];
}

// Fill twiddle tables in shared memory: tw[j] = exp(-2 pi i j/N), hw[k] = exp(-i pi k/(2N)).
// gtw / ghw are the same tables precomputed in double on the host.
template <typename T>
__device__ __forceinline__ void load_tables(c2<T>* tw, c2<T>* hw, const c2<T>* gtw, const c2<T>* ghw, int N) {
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    tw[j] = gtw[j];
    hw[j] = ghw[j];
  }
}

// Rows of a shared-memory tile.  Row r starts at base + (r / W) * rs_hi + (r % W) * rs_lo,
// element n of a row is at + n * es.  (W, rs_hi, rs_lo, es) describe both the
// row-major x tile ([t][x]: W huge, rs_lo = ld, es = 1) and the column layout
// of the y pass ([c][y][w]: rows are (c, w), es = W).
template <typename T>
struct Rows {
  T* base;
  int W, rs_hi, rs_lo, es;
  __device__ __forceinline__ T* row(int r) const { return base + (r / W) * rs_hi + (r % W) * rs_lo; }
};

// Power-of-two DCT via the four-step DFT.  PFAST selects the work-item order:
// false = element index fastest (rows contiguous in memory), true = row-pair
// index fastest (rows interleaved, as in the y pass).  The scratch holds
// npairs_per_chunk * N complex values.
template <typename T, int N1, int N2, bool PFAST>
struct DctPow2 {
  static constexpr int N = N1 * N2;
  static_assert((N1 & (N1 - 1)) == 0 && (N2 & (N2 - 1)) == 0, "power-of-two factors");

  __device__ static __forceinline__ int perm(int n) { return n < N / 2 ? 2 * n : 2 * N - 1 - 2 * n; }

  // scratch address of (pair p, slot j in [0, N)) for a chunk of cp pairs
  __device__ static __forceinline__ int sidx(int p, int j, int cp) { return PFAST ? j * cp + p : p * N + j; }
  // transpose slot of (k1, n2) with an XOR swizzle against bank conflicts (element-fast order)
  __device__ static __forceinline__ int tslot(int k1, int n2) {
    return PFAST ? k1 * N2 + n2 : k1 * N2 + (n2 ^ (k1 & (N2 - 1)));
  }

  // largest chunk of pairs such that pass 2 has one work item per thread
  __device__ static __forceinline__ int chunk_pairs() { return blockDim.x / N1; }

  __device__ static void forward(const Rows<T>& rows, int nrows, c2<T>* __restrict__ scr,
                                 const c2<T>* __restrict__ tw, const c2<T>* __restrict__ hw) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int npairs = nrows / 2;
    const int CP = chunk_pairs();
    for (int p0 = 0; p0 < npairs; p0 += CP) {
      const int cp = min(CP, npairs - p0);
      // pass 1: N1-point DFTs over n1 (stride N2), twiddle W_N^{n2 k1}
      for (int it = tid; it < cp * N2; it += nt) {
        int p, n2;
        if (PFAST) { n2 = it / cp; p = it - n2 * cp; } else { p = it / N2; n2 = it - p * N2; }
        const T* ra = rows.row(2 * (p0 + p));
        const T* rb = rows.row(2 * (p0 + p) + 1);
        c2<T> z[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) {
          const int q = perm(N2 * n1 + n2) * rows.es;
          z[n1] = mk2<T>(ra[q], rb[q]);
        }
        dft_reg<T, N1, N, false>(z, tw);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) {
          c2<T> v = z[k1];
          if (k1 != 0) v = cmul<T>(v, tw[(n2 * k1) & (N - 1)]);
          scr[sidx(p, tslot(k1, n2), cp)] = v;
        }
      }
      __syncthreads();
      // pass 2: N2-point DFTs over n2 -> Z[k1 + N1 k2], in place (one item per thread)
      {
        const int it = tid;
        const bool act = it < cp * N1;
        int p = 0, k1 = 0;
        c2<T> y[N2];
        if (act) {
          if (PFAST) { k1 = it / cp; p = it - k1 * cp; } else { p = it / N1; k1 = it - p * N1; }
#pragma unroll
          for (int n2 = 0; n2 < N2; ++n2) y[n2] = scr[sidx(p, tslot(k1, n2), cp)];
          dft_reg<T, N2, N, false>(y, tw);
        }
        __syncthreads();
        if (act) {
#pragma unroll
          for (int k2 = 0; k2 < N2; ++k2) scr[sidx(p, k1 + N1 * k2, cp)] = y[k2];
        }
      }
      __syncthreads();
      // post: split the packed spectra and rotate by exp(-i pi k / (2N))
      for (int it = tid; it < cp * N; it += nt) {
        int p, k;
        if (PFAST) { k = it / cp; p = it - k * cp; } else { p = it / N; k = it - p * N; }
        const c2<T> zk = scr[sidx(p, k, cp)];
        const c2<T> zm = scr[sidx(p, (N - k) & (N - 1), cp)];
        // V_a = (Z_k + conj Z_m)/2 ; V_b = (Z_k - conj Z_m)/(2i)
        const T vax = T(0.5) * (zk.x + zm.x), vay = T(0.5) * (zk.y - zm.y);
        const T vbx = T(0.5) * (zk.y + zm.y), vby = T(0.5) * (zm.x - zk.x);
        const c2<T> h = hw[k];  // (cos, -sin) of pi k/(2N)
        T* ra = rows.row(2 * (p0 + p));
        T* rb = rows.row(2 * (p0 + p) + 1);
        ra[k * rows.es] = h.x * vax - h.y * vay;
        rb[k * rows.es] = h.x * vbx - h.y * vby;
      }
      __syncthreads();
    }
  }

  __device__ static void inverse(const Rows<T>& rows, int nrows, c2<T>* __restrict__ scr,
                                 const c2<T>* __restrict__ tw, const c2<T>* __restrict__ hw) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int npairs = nrows / 2;
    const int CP = chunk_pairs();
    const T invN = T(1) / T(N);
    for (int p0 = 0; p0 < npairs; p0 += CP) {
      const int cp = min(CP, npairs - p0);
      // pre + pass 1: V[k] = exp(i pi k/(2N)) (X[k] - i X[N-k]), Z = V_a + i V_b; inverse DFT over n1
      for (int it = tid; it < cp * N2; it += nt) {
        int p, n2;
        if (PFAST) { n2 = it / cp; p = it - n2 * cp; } else { p = it / N2; n2 = it - p * N2; }
        const T* ra = rows.row(2 * (p0 + p));
        const T* rb = rows.row(2 * (p0 + p) + 1);
        c2<T> z[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) {
          const int k = N2 * n1 + n2;
          const T xa = ra[k * rows.es], xb = rb[k * rows.es];
          const T xam = k ? ra[(N - k) * rows.es] : T(0);
          const T xbm = k ? rb[(N - k) * rows.es] : T(0);
          const c2<T> h = hw[k];                 // conj(h) = (cos, +sin)
          // V_a = (h.x - i h.y) (xa - i xam)
          const T vax = h.x * xa - h.y * xam, vay = -h.x * xam - h.y * xa;
          const T vbx = h.x * xb - h.y * xbm, vby = -h.x * xbm - h.y * xb;
          z[n1] = mk2<T>(vax - vby, vay + vbx);  // V_a + i V_b
        }
        dft_reg<T, N1, N, true>(z, tw);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) {
          c2<T> v = z[k1];
          if (k1 != 0) v = cmulc<T>(v, tw[(n2 * k1) & (N - 1)]);
          scr[sidx(p, tslot(k1, n2), cp)] = v;
        }
      }
      __syncthreads();
      // pass 2: inverse N2-point DFTs; v = IDFT(Z)/N; x[perm(m)] = v[m]
      for (int it = tid; it < cp * N1; it += nt) {
        int p, k1;
        if (PFAST) { k1 = it / cp; p = it - k1 * cp; } else { p = it / N1; k1 = it - p * N1; }
        c2<T> y[N2];
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) y[n2] = scr[sidx(p, tslot(k1, n2), cp)];
        dft_reg<T, N2, N, true>(y, tw);
        T* ra = rows.row(2 * (p0 + p));
        T* rb = rows.row(2 * (p0 + p) + 1);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
          const int q = perm(k1 + N1 * k2) * rows.es;
          ra[q] = y[k2].x * invN;
          rb[q] = y[k2].y * invN;
        }
      }
      __syncthreads();
    }
  }
};

// Dense DCT of arbitrary length along rows: cos4[m] = cos(pi m / (2N)), m < 4N.
// scr holds one chunk of rows * N values.  Forward X[k] = sum_n x[n] cos4[k(2n+1) mod 4N];
// inverse x[n] = (1/N) (X[0] + 2 sum_{k>=1} X[k] cos4[k(2n+1) mod 4N]).
template <typename T, bool PFAST>
__device__ void dct_dense_rows(const Rows<T>& rows, int nrows, int N, bool inverse, T* __restrict__ scr,
                               int scr_cap, const T* __restrict__ cos4) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int M4 = 4 * N;
  const int CR = max(1, scr_cap / N);
  for (int r0 = 0; r0 < nrows; r0 += CR) {
    const int cr = min(CR, nrows - r0);
    for (int it = tid; it < cr * N; it += nt) {
      int r, k;
      if (PFAST) { k = it / cr; r = it - k * cr; } else { r = it / N; k = it - r * N; }
      const T* x = rows.row(r0 + r);
      T acc = 0;
      if (!inverse) {
        int m = k;  // k (2n+1) mod 4N, stepping n
        const int step = (2 * k) % M4;
        for (int n = 0; n < N; ++n) {
          acc += x[n * rows.es] * cos4[m];
          m += step;
          if (m >= M4) m -= M4;
        }
      } else {
        // output index is n = k here; sum over frequencies j
        const int n = k;
        const int step = 2 * n + 1;
        int m = 0;
        acc = x[0] * T(0.5);
        for (int j = 1; j < N; ++j) {
          m += step;
          if (m >= M4) m -= M4;
          acc += x[j * rows.es] * cos4[m];
        }
        acc *= T(2) / T(N);
      }
      scr[PFAST ? k * cr + r : r * N + k] = acc;
    }
    __syncthreads();
    for (int it = tid; it < cr * N; it += nt) {
      int r, k;
      if (PFAST) { k = it / cr; r = it - k * cr; } else { r = it / N; k = it - r * N; }
      rows.row(r0 + r)[k * rows.es] = scr[PFAST ? k * cr + r : r * N + k];
    }
    __syncthreads();
  }
}

// Dense transform along columns of a [P][ld] tile (the time axis): every
// thread owns whole columns in registers.  Mt is P x PMAX row-major with zero
// padding: out[k] = sum_t Mt[k*PMAX + t] in[t].
template <typename T, int PMAX>
__device__ void dct_cols(T* __restrict__ buf, int ld, int ncols, int P, const T* __restrict__ Mt) {
  for (int col = threadIdx.x; col < ncols; col += blockDim.x) {
    T v[PMAX];
#pragma unroll
    for (int t = 0; t < PMAX; ++t) v[t] = (t < P) ? buf[t * ld + col] : T(0);
    for (int k = 0; k < P; ++k) {
      const T* row = Mt + k * PMAX;
      T acc = 0;
#pragma unroll
      for (int t = 0; t < PMAX; ++t) acc = fma(row[t], v[t], acc);
      buf[k * ld + col] = acc;
    }
  }
}

}  // namespace dynot
