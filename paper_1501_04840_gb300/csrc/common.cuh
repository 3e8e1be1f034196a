// Shared device-side definitions of the dynamic-OT CUDA path.
//
// Layout of every cell-aligned array of one problem (batch index b, half-time
// cell t = 0..P-1, spatial cell s = x + n1*(y + n2*c)):
//     index = ((b*P + t)*S + s),  S = n1*n2*C.
// The iteration state (a and the scaled dual b) and the primal output x hold
// four components per cell, interleaved (one 16-byte vector per cell in FP32):
// (m_x, m_y, m_c, f) for a and x, (b_mx, b_my, b_mc, b_f) for b.
// Faces are stored cell-aligned: component k at index of cell s holds the face
// to the right of s along axis k (between s and s+e_k, wrapping for a periodic
// axis).  For a Neumann axis the last face (i_k = n_k-1) is a boundary face of
// the paper's model (section 2: kappa = 1, m absent there) and is kept at zero.
// f at time (t+1)/P sits in the f component of slot t = 0..P-2; slot P-1 holds zero.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dynot {

// Programmatic dependent launch: a kernel launched with the programmatic-serialisation attribute may
// start while its predecessor in the stream finishes.  pdl_trigger() lets the successor launch once
// every block of this grid has passed it; pdl_wait() blocks until the predecessor grid has completed
// and its writes are visible.  Without the attribute both are no-ops.  Every kernel here reads or
// writes global data only after pdl_wait(); only constant tables are read before it.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// Asynchronous global -> shared copies (cp.async): the loads of a whole tile are in flight at
// once and need no registers; cp_async_wait_all() waits for this thread's copies (a
// __syncthreads() must follow before other threads read them).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
template <int BYTES>
__device__ __forceinline__ void cp_async_small(void* smem, const void* gmem) {
  static_assert(BYTES == 4 || BYTES == 8, "element copies of 4 or 8 bytes");
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Copy nrows rows of len elements from src (row stride src_ld) to shared dst (row stride dst_ld),
// in 16-byte pieces when every row start is 16-byte aligned, element by element otherwise.
template <typename T>
__device__ __forceinline__ void async_rows(T* dst, int dst_ld, const T* src, long long src_ld, int nrows, int len) {
  constexpr int V = 16 / (int)sizeof(T);
  const bool vec = len % V == 0 && dst_ld % V == 0 && src_ld % V == 0 && ((uintptr_t)src & 15) == 0 &&
                   ((uintptr_t)dst & 15) == 0;
  if (vec) {
    const int per = len / V;
    for (int i = threadIdx.x; i < nrows * per; i += blockDim.x) {
      const int r = i / per, k = i - r * per;
      cp_async16(dst + (size_t)r * dst_ld + k * V, src + r * src_ld + k * V);
    }
  } else {
    for (int i = threadIdx.x; i < nrows * len; i += blockDim.x) {
      const int r = i / len, k = i - r * len;
      cp_async_small<sizeof(T)>(dst + (size_t)r * dst_ld + k, src + r * src_ld + k);
    }
  }
}


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
  const int* active;    // per problem: 0 = retired (its blocks return at once); nullptr = all active
};

// A problem of a mixed-size batch that has met its tolerance is retired: every kernel of the iteration
// returns at once for its blocks, so its state stays as it was at the check that retired it.
template <typename T>
__device__ __forceinline__ bool retired(const Geo<T>& g, int b) {
  return g.active != nullptr && g.active[b] == 0;
}

// Four components of one cell, one aligned vector: float4 in FP32, 32-byte aligned in FP64.
struct __align__(32) dvec4 {
  double x, y, z, w;
};
template <typename T> struct vec4;
template <> struct vec4<float> { using type = float4; };
template <> struct vec4<double> { using type = dvec4; };
template <typename T> using v4 = typename vec4<T>::type;

template <typename T>
__host__ __device__ __forceinline__ v4<T> mk4(T a, T b, T c, T d) {
  v4<T> r;
  r.x = a; r.y = b; r.z = c; r.w = d;
  return r;
}
template <typename T>
__host__ __device__ __forceinline__ T cget(const v4<T>& v, int k) {
  return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}
// component k of cell i of an interleaved array, as a scalar load
template <typename T>
__host__ __device__ __forceinline__ T comp(const v4<T>* p, size_t i, int k) {
  return reinterpret_cast<const T*>(p)[4 * i + k];
}

// Device pointers of the iteration state of one plan (all cell-aligned, four components per cell).
template <typename T>
struct Arrays {
  const v4<T>* a;  // a = x - tau sigma K^T bbar at faces: (m_x, m_y, m_c, f)
  const v4<T>* b;  // scaled dual b: (b_mx, b_my, b_mc, b_f) at cells
  v4<T>* an;       // next a
  v4<T>* bn;       // next b
  const T* phi;    // (A A^T)^+ r of this iteration, physical cells
  const T* f0;     // boundary densities (solver units), [b][s]
  const T* f1;
  v4<T>* x;        // optional output: x^{r+1} (faces), nullptr when not wanted
  const v4<T>* w;  // K x0 + (0, f_b^+) at the cells (x0 the least-norm feasible path): the dual value
                   // of a check is sigma <b^{r+1}, w>
};

// Compensated (Kahan) sum in the working precision: the per-thread partial sums of a residual check keep
// about two units in the last place whatever their length; the sums across threads are in FP64.
template <typename T>
struct KSum {
  T s = T(0), c = T(0);
  __device__ __forceinline__ void add(T v) {
    const T y = v - c;
    const T t = s + y;
    c = (t - s) - y;
    s = t;
  }
};

}  // namespace dynot
