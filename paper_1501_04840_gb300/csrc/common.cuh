// Shared device-side definitions of the dynamic-OT CUDA path.
//
// Layout of every cell-aligned array of one problem (batch index b, half-time
// cell t = 0..P-1, spatial cell s = x + n1*(y + n2*c)):
//     index = ((b*P + t)*S + s),  S = n1*n2*C.
// Faces are stored cell-aligned: component k at index of cell s holds the face
// to the right of s along axis k (between s and s+e_k, wrapping for a periodic
// axis).  For a Neumann axis the last face (i_k = n_k-1) is a boundary face of
// the paper's model (section 2: kappa = 1, m absent there) and is kept at zero.
// f at time (t+1)/P sits at slot t = 0..P-2 of the f array; slot P-1 is zero.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dynot {

constexpr double kPi = 3.141592653589793238462643383279502884;

template <typename T> struct vec2;
template <> struct vec2<float> { using type = float2; };
template <> struct vec2<double> { using type = double2; };
template <typename T> using c2 = typename vec2<T>::type;

template <typename T> __device__ __forceinline__ c2<T> mk2(T a, T b) { c2<T> r; r.x = a; r.y = b; return r; }
template <typename T> __device__ __forceinline__ c2<T> cadd(c2<T> a, c2<T> b) { return mk2<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ c2<T> csub(c2<T> a, c2<T> b) { return mk2<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ c2<T> cmul(c2<T> a, c2<T> b) {
  return mk2<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T> __device__ __forceinline__ c2<T> cmulc(c2<T> a, c2<T> b) {  // a * conj(b)
  return mk2<T>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// Geometry of one problem size on the RGB/grey path (three spatial axes; an
// axis of size 1 is inert) or on the hue path (axis 0 only).
template <typename T>
struct Geo {
  int n1, n2, C;        // cells along x, y, colour
  int per1, per2, perc; // 1 = periodic axis (kappa = 0), 0 = Neumann (kappa = 1)
  int P;                // time intervals
  int S;                // n1*n2*C
  int B;                // problems in the batch (same size)
  long long N;          // P*S cells per problem
  T s1, s2, sc;         // difference factors of D_M per axis (n_k for the unit cube)
  T sp;                 // P, factor of D_F
  T ts;                 // tau*sigma (step 1 of Algorithm 1)
  T sigma;              // step 2 of Algorithm 1
};

template <typename T>
struct CPtr4 {
  const T* p[4];
};

// Device pointers of the iteration state of one plan (all cell-aligned).
template <typename T>
struct Arrays {
  const T* a[4];   // a = x - tau sigma K^T bbar at faces: m_x, m_y, m_c, f
  const T* b[4];   // scaled dual b: b_mx, b_my, b_mc, b_f (cells)
  T* an[4];        // next a
  T* bn[4];        // next b
  const T* phi;    // (A A^T)^+ r of this iteration, physical cells
  const T* f0;     // boundary densities (solver units), [b][s]
  const T* f1;
  T* x[4];         // optional output: x^{r+1} (faces), nullptr when not wanted
};

}  // namespace dynot
