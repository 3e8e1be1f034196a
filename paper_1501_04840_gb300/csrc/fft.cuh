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
// Each register DFT is an unrolled radix-2 Cooley-Tukey decimation in time; an
// N2 of 3 * 2^k (lengths 96 = 16 * 6 and 192 = 16 * 12) adds one radix-3 step.
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

// The same DFT for input already stored in bit-reversed order (z[bitrev(i)] = input i),
// computed in place without a second register array.
template <typename T, int R, int NT, bool INV>
__device__ __forceinline__ void dft_reg_br(c2<T> (&a)[R], const c2<T>* __restrict__ twN) {
  constexpr int L = Log2<R>::v;
#pragma unroll
  for (int stage = 0; stage < L; ++stage) {
    const int m = 2 << stage;
#pragma unroll
    for (int k = 0; k < R; k += m) {
#pragma unroll
      for (int j = 0; j < m / 2; ++j) {
        c2<T> t = a[k + j + m / 2];
        if (j != 0) {
          if (4 * j == m) {
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
}

template <int R> struct IsPow2 { static constexpr bool v = R > 0 && (R & (R - 1)) == 0; };

// In-register DFT of length R = 2^k or 3 * 2^k (same conventions as dft_reg).  For 3 * 2^k it is one
// radix-3 decimation-in-time step: the three interleaved subsequences z[3m + r] are transformed with
// dft_reg and combined as Z[k + j R/3] = sum_r w3^(j r) W_R^(k r) E_r[k] (w3 = W_R^(R/3), j = 0, 1, 2).
template <typename T, int R, int NT, bool INV>
__device__ __forceinline__ void dft_any(c2<T> (&z)[R], const c2<T>* __restrict__ twN) {
  if constexpr (IsPow2<R>::v) {
    dft_reg<T, R, NT, INV>(z, twN);
  } else {
    static_assert(R % 3 == 0 && IsPow2<R / 3>::v, "length 2^k or 3 * 2^k");
    constexpr int M = R / 3;
    c2<T> e[3][M];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
#pragma unroll
      for (int m = 0; m < M; ++m) e[r][m] = z[3 * m + r];
      if constexpr (M > 1) dft_reg<T, M, NT, INV>(e[r], twN);
    }
    const c2<T> w3 = twN[M * (NT / R)];             // exp(-2 pi i / 3)
    const T wr = w3.x, wi = INV ? -w3.y : w3.y;
#pragma unroll
    for (int k = 0; k < M; ++k) {
      c2<T> b = e[1][k], c = e[2][k];
      if (k != 0) {
        const c2<T> w1 = twN[k * (NT / R)], w2 = twN[2 * k * (NT / R)];
        b = INV ? cmulc<T>(b, w1) : cmul<T>(b, w1);
        c = INV ? cmulc<T>(c, w2) : cmul<T>(c, w2);
      }
      const c2<T> a = e[0][k];
      const c2<T> s = cadd<T>(b, c), d = csub<T>(b, c);
      // w b + conj(w) c = Re(w) (b + c) + i Im(w) (b - c)
      const c2<T> base = mk2<T>(a.x + wr * s.x, a.y + wr * s.y);
      const c2<T> rot = mk2<T>(-wi * d.y, wi * d.x);
      z[k] = cadd<T>(a, s);
      z[k + M] = cadd<T>(base, rot);
      z[k + 2 * M] = csub<T>(base, rot);
    }
  }
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

// Rows of a shared-memory tile.  Row r = g*RW + j (j < RW) starts at
// base + g*rs_hi + j*rs_lo; element n of a row sits at + n*ES.  RW = 1, ES = 1
// describes the row-major x tile ([t][x], rs_hi = row length); RW = ES = W the
// column layout of the y pass ([c][y][w]: rows are (c, w), rs_hi = n2*W, rs_lo = 1).
template <typename T, int RW, int ES>
struct Rows {
  T* base;
  int rs_hi, rs_lo;
  static constexpr int es = ES;
  __device__ __forceinline__ T* row(int r) const { return base + (r / RW) * rs_hi + (r % RW) * rs_lo; }
};

// Power-of-two DCT via the four-step DFT for a block of NT threads.  PFAST
// selects the work-item order: false = element index fastest (rows contiguous
// in memory), true = row-pair index fastest (rows interleaved, as in the y
// pass).  Pairs are processed in chunks of CP = NT / N1; the scratch holds
// CP * N complex values.  Every index divisor is a compile-time constant.
// PERIODIC = true: the same machinery computes the real Fourier transform of rows of a periodic axis in the
// slot layout of rdft_dense_rows (natural input order; slots 0, 2j-1, 2j, N-1 from the spectrum).
template <typename T, int N1, int N2, bool PFAST, int NT, bool PERIODIC = false>
struct DctPow2 {
  static constexpr int N = N1 * N2;
  static constexpr int CP = NT / N1;
  static_assert(IsPow2<N1>::v && N2 % 2 == 0 && (IsPow2<N2>::v || (N2 % 3 == 0 && IsPow2<N2 / 3>::v)),
                "N1 a power of two, N2 = 2^k or 3 * 2^k (even)");
  static_assert(CP >= 1 && CP * N1 == NT, "block size must be a multiple of N1");

  // scratch address of (pair p, slot j in [0, N))
  __device__ static __forceinline__ int sidx(int p, int j) { return PFAST ? j * CP + p : p * N + j; }
  // transpose slot of (k1, n2) with an XOR swizzle against bank conflicts (element-fast order)
  __device__ static __forceinline__ int tslot(int k1, int n2) {
    return (PFAST || !IsPow2<N2>::v) ? k1 * N2 + n2 : k1 * N2 + (n2 ^ (k1 & (N2 - 1)));
  }
  // split a work item into (pair, index) with `per` indices per pair
  template <int PER>
  __device__ static __forceinline__ void split(int it, int& p, int& j) {
    if (PFAST) { p = it % CP; j = it / CP; } else { p = it / PER; j = it % PER; }
  }

  template <class R>
  __device__ static void forward(const R& rows, int nrows, c2<T>* __restrict__ scr, const c2<T>* __restrict__ tw,
                                 const c2<T>* __restrict__ hw) {
    const int tid = threadIdx.x;
    const int npairs = nrows / 2;
    for (int p0 = 0; p0 < npairs; p0 += CP) {
      const int cp = min(CP, npairs - p0);
      // pass 1: N1-point DFTs over n1 (stride N2), twiddle W_N^{n2 k1}
#pragma unroll
      for (int q = 0; q < (CP * N2 + NT - 1) / NT; ++q) {
        const int it = tid + q * NT;
        int p, n2;
        split<N2>(it, p, n2);
        if (it < CP * N2 && p < cp) {
          const T* ra = rows.row(2 * (p0 + p));
          const T* rb = rows.row(2 * (p0 + p) + 1);
          c2<T> z[N1];
#pragma unroll
          for (int n1 = 0; n1 < N1; ++n1) {
            const int n = N2 * n1 + n2;
            const int e = PERIODIC ? n * R::es : (n1 < N1 / 2 ? 2 * n : 2 * N - 1 - 2 * n) * R::es;   // Makhoul order
            z[n1] = mk2<T>(ra[e], rb[e]);
          }
          dft_reg<T, N1, N, false>(z, tw);
#pragma unroll
          for (int k1 = 0; k1 < N1; ++k1) {
            c2<T> v = z[k1];
            if (k1 != 0) v = cmul<T>(v, tw[n2 * k1]);
            scr[sidx(p, tslot(k1, n2))] = v;
          }
        }
      }
      __syncthreads();
      // pass 2: N2-point DFTs over n2 -> Z[k1 + N1 k2], in place (one item per thread)
      {
        int p, k1;
        split<N1>(tid, p, k1);
        const bool act = p < cp;
        c2<T> y[N2];
        if (act) {
#pragma unroll
          for (int n2 = 0; n2 < N2; ++n2) y[n2] = scr[sidx(p, tslot(k1, n2))];
          dft_any<T, N2, N, false>(y, tw);
        }
        __syncthreads();
        if (act) {
#pragma unroll
          for (int k2 = 0; k2 < N2; ++k2) scr[sidx(p, k1 + N1 * k2)] = y[k2];
        }
      }
      __syncthreads();
      // post: split the packed spectra and rotate by exp(-i pi k / (2N))
#pragma unroll 4
      for (int q = 0; q < CP * N / NT; ++q) {
        const int it = tid + q * NT;
        int p, k;
        split<N>(it, p, k);
        if (p < cp) {
          const c2<T> zk = scr[sidx(p, k)];
          const c2<T> zm = scr[sidx(p, IsPow2<N>::v ? ((N - k) & (N - 1)) : (k == 0 ? 0 : N - k))];
          // V_a = (Z_k + conj Z_m)/2 ; V_b = (Z_k - conj Z_m)/(2i)
          const T vax = T(0.5) * (zk.x + zm.x), vay = T(0.5) * (zk.y - zm.y);
          const T vbx = T(0.5) * (zk.y + zm.y), vby = T(0.5) * (zm.x - zk.x);
          T* ra = rows.row(2 * (p0 + p));
          T* rb = rows.row(2 * (p0 + p) + 1);
          if constexpr (PERIODIC) {
            // V = sum x exp(-2 pi i n k / N): slot 2k-1 = Re V (cos sum), slot 2k = -Im V (sin sum)
            if (k == 0) {
              ra[0] = vax;
              rb[0] = vbx;
            } else if (k < N / 2) {
              ra[(2 * k - 1) * R::es] = vax;
              ra[(2 * k) * R::es] = -vay;
              rb[(2 * k - 1) * R::es] = vbx;
              rb[(2 * k) * R::es] = -vby;
            } else if (k == N / 2) {
              ra[(N - 1) * R::es] = vax;
              rb[(N - 1) * R::es] = vbx;
            }
          } else {
            const c2<T> h = hw[k];  // (cos, -sin) of pi k/(2N)
            ra[k * R::es] = h.x * vax - h.y * vay;
            rb[k * R::es] = h.x * vbx - h.y * vby;
          }
        }
      }
      __syncthreads();
    }
  }

  template <class R>
  __device__ static void inverse(const R& rows, int nrows, c2<T>* __restrict__ scr, const c2<T>* __restrict__ tw,
                                 const c2<T>* __restrict__ hw) {
    const int tid = threadIdx.x;
    const int npairs = nrows / 2;
    const T invN = T(1) / T(N);
    for (int p0 = 0; p0 < npairs; p0 += CP) {
      const int cp = min(CP, npairs - p0);
      // pre + pass 1: V[k] = exp(i pi k/(2N)) (X[k] - i X[N-k]), Z = V_a + i V_b; inverse DFT over n1
#pragma unroll
      for (int q = 0; q < (CP * N2 + NT - 1) / NT; ++q) {
        const int it = tid + q * NT;
        int p, n2;
        split<N2>(it, p, n2);
        if (it < CP * N2 && p < cp) {
          const T* ra = rows.row(2 * (p0 + p));
          const T* rb = rows.row(2 * (p0 + p) + 1);
          c2<T> z[N1];
#pragma unroll
          for (int n1 = 0; n1 < N1; ++n1) {
            const int k = N2 * n1 + n2;
            if constexpr (PERIODIC) {
              // the Hermitian spectrum of each row from its slots: V_k = X[2k-1] - i X[2k], V_{N-k} = conj V_k
              auto spec = [&](const T* r, T& re, T& im) {
                if (k == 0) { re = r[0]; im = T(0); }
                else if (k < N / 2) { re = r[(2 * k - 1) * R::es]; im = -r[(2 * k) * R::es]; }
                else if (k == N / 2) { re = r[(N - 1) * R::es]; im = T(0); }
                else { const int kk = N - k; re = r[(2 * kk - 1) * R::es]; im = r[(2 * kk) * R::es]; }
              };
              T ax, ay, bx, by;
              spec(ra, ax, ay);
              spec(rb, bx, by);
              z[n1] = mk2<T>(ax - by, ay + bx);    // V_a + i V_b
            } else {
              const T xa = ra[k * R::es], xb = rb[k * R::es];
              const T xam = k ? ra[(N - k) * R::es] : T(0);
              const T xbm = k ? rb[(N - k) * R::es] : T(0);
              const c2<T> h = hw[k];                 // conj(h) = (cos, +sin)
              // V_a = (h.x - i h.y) (xa - i xam)
              const T vax = h.x * xa - h.y * xam, vay = -h.x * xam - h.y * xa;
              const T vbx = h.x * xb - h.y * xbm, vby = -h.x * xbm - h.y * xb;
              z[n1] = mk2<T>(vax - vby, vay + vbx);  // V_a + i V_b
            }
          }
          dft_reg<T, N1, N, true>(z, tw);
#pragma unroll
          for (int k1 = 0; k1 < N1; ++k1) {
            c2<T> v = z[k1];
            if (k1 != 0) v = cmulc<T>(v, tw[n2 * k1]);
            scr[sidx(p, tslot(k1, n2))] = v;
          }
        }
      }
      __syncthreads();
      // pass 2: inverse N2-point DFTs; v = IDFT(Z)/N; x[perm(m)] = v[m]
      {
        int p, k1;
        split<N1>(tid, p, k1);
        if (p < cp) {
          c2<T> y[N2];
#pragma unroll
          for (int n2 = 0; n2 < N2; ++n2) y[n2] = scr[sidx(p, tslot(k1, n2))];
          dft_any<T, N2, N, true>(y, tw);
          T* ra = rows.row(2 * (p0 + p));
          T* rb = rows.row(2 * (p0 + p) + 1);
#pragma unroll
          for (int k2 = 0; k2 < N2; ++k2) {
            const int m = k1 + N1 * k2;
            const int e = PERIODIC ? m * R::es : (k2 < N2 / 2 ? 2 * m : 2 * N - 1 - 2 * m) * R::es;
            ra[e] = y[k2].x * invN;
            rb[e] = y[k2].y * invN;
          }
        }
      }
      __syncthreads();
    }
  }
};

// Dense real DFT of arbitrary length along rows, for periodic axes: cs[m] = (cos, sin)(2 pi m / N).
// Forward: slot 0 = sum_n x[n]; slots 2j-1, 2j = sum_n x[n] cos, sin (2 pi n j / N); for even N the
// last slot = sum_n x[n] (-1)^n.  These real Fourier coefficients diagonalise the periodic Laplacian
// (eigenvalue 4 sin^2(pi j / N) for both slots of frequency j).  Inverse:
// x[n] = (1/N) (X[0] + 2 sum_j (X[2j-1] cos + X[2j] sin)(2 pi n j / N) + X[N-1] (-1)^n [even N]).
template <typename T, bool PFAST, class R>
__device__ void rdft_dense_rows(const R& rows, int nrows, int N, bool inverse, T* __restrict__ scr, int scr_cap,
                                const c2<T>* __restrict__ cs) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int CR = max(1, scr_cap / N);
  const bool even = (N & 1) == 0;
  const int last = even ? N - 1 : N;   // slots 1 .. last-1 come in (cos, sin) pairs
  for (int r0 = 0; r0 < nrows; r0 += CR) {
    const int cr = min(CR, nrows - r0);
    for (int it = tid; it < cr * N; it += nt) {
      int r, k;
      if (PFAST) { k = it / cr; r = it - k * cr; } else { r = it / N; k = it - r * N; }
      const T* x = rows.row(r0 + r);
      T acc = 0;
      if (!inverse) {
        if (k == 0) {
          for (int n = 0; n < N; ++n) acc += x[n * R::es];
        } else if (even && k == N - 1) {
          for (int n = 0; n < N; ++n) acc += (n & 1) ? -x[n * R::es] : x[n * R::es];
        } else {
          const int j = (k + 1) >> 1;
          const bool use_cos = k & 1;
          int m = 0;   // n j mod N, stepping n
          for (int n = 0; n < N; ++n) {
            const c2<T> w = cs[m];
            acc += x[n * R::es] * (use_cos ? w.x : w.y);
            m += j;
            if (m >= N) m -= N;
          }
        }
      } else {
        const int n = k;   // output sample; sum over the slots
        T s2 = 0;
        int m = 0;         // n j mod N, stepping j
        for (int slot = 1; slot < last; slot += 2) {
          m += n;
          if (m >= N) m -= N;
          const c2<T> w = cs[m];
          s2 += x[slot * R::es] * w.x + x[(slot + 1) * R::es] * w.y;
        }
        acc = x[0] + T(2) * s2;
        if (even) acc += (n & 1) ? -x[(N - 1) * R::es] : x[(N - 1) * R::es];
        acc *= T(1) / T(N);
      }
      scr[PFAST ? k * cr + r : r * N + k] = acc;
    }
    __syncthreads();
    for (int it = tid; it < cr * N; it += nt) {
      int r, k;
      if (PFAST) { k = it / cr; r = it - k * cr; } else { r = it / N; k = it - r * N; }
      rows.row(r0 + r)[k * R::es] = scr[PFAST ? k * cr + r : r * N + k];
    }
    __syncthreads();
  }
}

// Dense DCT of arbitrary length along rows: cos4[m] = cos(pi m / (2N)), m < 4N.
// scr holds one chunk of rows * N values.  Forward X[k] = sum_n x[n] cos4[k(2n+1) mod 4N];
// inverse x[n] = (1/N) (X[0] + 2 sum_{k>=1} X[k] cos4[k(2n+1) mod 4N]).
template <typename T, bool PFAST, class R>
__device__ void dct_dense_rows(const R& rows, int nrows, int N, bool inverse, T* __restrict__ scr, int scr_cap,
                               const T* __restrict__ cos4) {
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
          acc += x[n * R::es] * cos4[m];
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
          acc += x[j * R::es] * cos4[m];
        }
        acc *= T(2) / T(N);
      }
      scr[PFAST ? k * cr + r : r * N + k] = acc;
    }
    __syncthreads();
    for (int it = tid; it < cr * N; it += nt) {
      int r, k;
      if (PFAST) { k = it / cr; r = it - k * cr; } else { r = it / N; k = it - r * N; }
      rows.row(r0 + r)[k * R::es] = scr[PFAST ? k * cr + r : r * N + k];
    }
    __syncthreads();
  }
}

// Dense transform along columns of a [P][ld] tile (the time axis): every
// thread owns whole columns in registers.  Mt is P x PMAX row-major with zero
// padding: out[k] = sum_t Mt[k*PMAX + t] in[t].
template <typename T, int PMAX>
__device__ void dct_cols(T* __restrict__ buf, int ld, int ncols, int P, const T* __restrict__ Mt) {
  static_assert(PMAX % 4 == 0, "PMAX must be a multiple of 4");
  for (int col = threadIdx.x; col < ncols; col += blockDim.x) {
    T v[PMAX];
#pragma unroll
    for (int t = 0; t < PMAX; ++t) v[t] = (t < P) ? buf[t * ld + col] : T(0);
    for (int k = 0; k < P; ++k) {
      const T* row = Mt + k * PMAX;
      T acc0 = 0, acc1 = 0;
      if constexpr (sizeof(T) == 4) {
        const float4* r4 = reinterpret_cast<const float4*>(row);
#pragma unroll
        for (int t = 0; t < PMAX / 4; ++t) {
          const float4 m = r4[t];
          acc0 = fma(m.x, v[4 * t], acc0);
          acc1 = fma(m.y, v[4 * t + 1], acc1);
          acc0 = fma(m.z, v[4 * t + 2], acc0);
          acc1 = fma(m.w, v[4 * t + 3], acc1);
        }
      } else {
#pragma unroll
        for (int t = 0; t < PMAX; t += 2) {
          acc0 = fma(row[t], v[t], acc0);
          acc1 = fma(row[t + 1], v[t + 1], acc1);
        }
      }
      buf[k * ld + col] = acc0 + acc1;
    }
  }
}

// Register DCT along the columns of a [P][ld] tile for P a power of two: each
// thread owns whole columns.  The row length ld is a compile-time constant so
// that every element address is an immediate offset.  Forward is the unnormalised DCT-II, inverse its
// exact inverse, both by Makhoul's reordering and a P/2-point complex DFT of the
// packed even/odd samples (z[m] = v[2m] + i v[2m+1]).
// twP[j] = exp(-2 pi i j / P), hwP[k] = exp(-i pi k / (2P)).
template <typename T, int P, bool INV, int ld>
__device__ void dct_cols_fft(T* __restrict__ buf, int ncols, const c2<T>* __restrict__ twP,
                             const c2<T>* __restrict__ hwP) {
  constexpr int M = P / 2;
#pragma unroll 1
  for (int col = threadIdx.x; col < ncols; col += blockDim.x) {
    T* cb = buf + col;
    c2<T> z[M];
    if (!INV) {
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const int j0 = 2 * m, j1 = 2 * m + 1;   // v[j] = x[2j] (j < M), x[2(P-1-j)+1] (j >= M)
        const T v0 = cb[(j0 < M ? 2 * j0 : 2 * (P - 1 - j0) + 1) * ld];
        const T v1 = cb[(j1 < M ? 2 * j1 : 2 * (P - 1 - j1) + 1) * ld];
        z[bitrev_c(m, Log2<M>::v)] = mk2<T>(v0, v1);
      }
      dft_reg_br<T, M, P, false>(z, twP);
#pragma unroll
      for (int k = 0; k < M; ++k) {
        const c2<T> zk = z[k];
        const c2<T> zm = z[(M - k) % M];
        // even-sample spectrum E = (Z_k + conj Z_{M-k})/2, odd-sample O = (Z_k - conj Z_{M-k})/(2i)
        const T ex = T(0.5) * (zk.x + zm.x), ey = T(0.5) * (zk.y - zm.y);
        const T ox = T(0.5) * (zk.y + zm.y), oy = T(0.5) * (zm.x - zk.x);
        const c2<T> w = twP[k];
        const T tx = w.x * ox - w.y * oy, ty = w.x * oy + w.y * ox;
        const c2<T> h0 = hwP[k], h1 = hwP[k + M];
        cb[k * ld] = h0.x * (ex + tx) - h0.y * (ey + ty);          // V[k] = E + W^k O
        cb[(k + M) * ld] = h1.x * (ex - tx) - h1.y * (ey - ty);    // V[k+M] = E - W^k O
      }
    } else {
#pragma unroll
      for (int k = 0; k < M; ++k) {
        // V[j] = exp(i pi j / 2P) (X[j] - i X[P-j]) for j = k and j = k + M
        const T a0 = cb[k * ld], b0 = k ? cb[(P - k) * ld] : T(0);
        const T a1 = cb[(k + M) * ld], b1 = cb[(M - k) * ld];
        const c2<T> h0 = hwP[k], h1 = hwP[k + M];
        const T v0x = h0.x * a0 - h0.y * b0, v0y = -h0.x * b0 - h0.y * a0;
        const T v1x = h1.x * a1 - h1.y * b1, v1y = -h1.x * b1 - h1.y * a1;
        const T ex = T(0.5) * (v0x + v1x), ey = T(0.5) * (v0y + v1y);
        const T dx = T(0.5) * (v0x - v1x), dy = T(0.5) * (v0y - v1y);
        const c2<T> w = twP[k];                                   // O = (V[k] - V[k+M])/2 * conj(W^k)
        const T ox = dx * w.x + dy * w.y, oy = dy * w.x - dx * w.y;
        z[bitrev_c(k, Log2<M>::v)] = mk2<T>(ex - oy, ey + ox);   // E + i O
      }
      dft_reg_br<T, M, P, true>(z, twP);
      const T invM = T(1) / T(M);
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const int j0 = 2 * m, j1 = 2 * m + 1;
        cb[(j0 < M ? 2 * j0 : 2 * (P - 1 - j0) + 1) * ld] = z[m].x * invM;
        cb[(j1 < M ? 2 * j1 : 2 * (P - 1 - j1) + 1) * ld] = z[m].y * invM;
      }
    }
  }
}

}  // namespace dynot
