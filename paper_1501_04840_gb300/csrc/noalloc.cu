// Projection onto C_d for hue histograms without any device allocation.
//
// Who needs this: code that runs where cudaMalloc is not available or not
// allowed -- for example a host that pre-reserves all device memory for
// itself, an embedding that forbids allocation after start-up, or a caller that
// must not trigger the implicit synchronisation an allocation can cause.
// Such callers cannot create a plan (ot_plan allocates its workspace), so this
// entry point keeps its working memory in a fixed array that lives in the
// library's own device image.  The call only queues its kernel on the caller's
// stream and does not wait for it.
//
// The intermediate spectral array lives in kScratchFloats floats of file-scope
// device memory (16 MiB).  Every GPU that loads this library holds that array
// until the process exits.  All calls share it and each call leaves its own
// data behind; nothing in it has to start at zero because every call writes
// each element before it reads it.  Two calls whose kernels overlap on the GPU
// (different streams, or different host threads) would race on the array, so
// callers must not let them overlap.
#include "../../include/dynot.h"

#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "common.cuh"
#include "plan_base.h"

namespace dynot {
namespace {

constexpr size_t kScratchFloats = size_t(1) << 22;  // 16 MiB of float32
constexpr int kMaxDevices = 64;
constexpr int kMaxBins = 8192;
constexpr int kMaxP = 64;
constexpr float kLamFp64 = 64.f;   // eigenvalues below this are divided in double (the plans' default)

static __device__ __align__(256) float g_noalloc_scratch[kScratchFloats];

// Device address of g_noalloc_scratch for each device, resolved once per device.
float* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

ot_status scratch_for_current_device(float** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return seterr(OT_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return seterr(OT_EUNSUPPORTED, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return seterr(OT_ECUDA, "cudaGetSymbolAddress of the scratch array: %s", cudaGetErrorString(e));
    g_scratch_ptr[dev] = (float*)p;
  }
  *out = g_scratch_ptr[dev];
  return OT_OK;
}

// One block per problem: r = A a - f_b^-, forward real DFT along the bins,
// DCT-II along t with the eigenvalue divide and its inverse, inverse DFT -> phi,
// and x = a - A^T phi.  Tables are computed in shared memory with sincospi.
__global__ void __launch_bounds__(256) k_hue_project_noalloc(int n, int P, double s, const float* __restrict__ f0,
                                                             const float* __restrict__ f1,
                                                             const float* __restrict__ ap, float* __restrict__ xp,
                                                             float* __restrict__ phi, float* __restrict__ scratch) {
  extern __shared__ __align__(16) char sm[];
  const int b = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  float2* cs = (float2*)sm;                     // (cos, sin)(2 pi m / n)
  float* Mt = (float*)(cs + n);                 // [k][t] = cos(pi k (2t+1) / 2P)
  float* lam = Mt + P * P;                      // eigenvalue of each bin slot
  float* lamt = lam + n;                        // eigenvalue of each t mode
  for (int m = tid; m < n; m += nt) {
    double c, si;
    sincospi(2.0 * m / n, &si, &c);
    cs[m] = make_float2((float)c, (float)si);
    int j = (m + 1) / 2;
    if ((n & 1) == 0 && m == n - 1) j = n / 2;
    const double v = sinpi((double)j / n);
    lam[m] = (float)(s * s * 4.0 * v * v);
  }
  for (int i = tid; i < P * P; i += nt) {
    const int k = i / P, t = i % P;
    Mt[i] = (float)cospi((double)k * (2 * t + 1) / (2.0 * P));
  }
  for (int k = tid; k < P; k += nt) {
    const double v = sinpi((double)k / (2.0 * P));
    lamt[k] = (float)((double)P * P * 4.0 * v * v);
  }
  const size_t mlen = (size_t)P * n, flen = (size_t)(P - 1) * n;
  const float* am = ap + (size_t)b * (mlen + flen);
  const float* af = am + mlen;
  float* r = scratch + (size_t)b * 2 * mlen;   // [t][i], then the spectrum [t][slot]
  float* h = r + mlen;
  // r = A a - f_b^-: periodic faces (face i is the left face of bin i)
  for (size_t q = tid; q < mlen; q += nt) {
    const int t = (int)(q / n), i = (int)(q % n);
    const int i1 = i + 1 == n ? 0 : i + 1;
    const float fprev = t == 0 ? f0[(size_t)b * n + i] : af[(size_t)(t - 1) * n + i];
    const float fnext = t == P - 1 ? f1[(size_t)b * n + i] : af[(size_t)t * n + i];
    r[q] = (float)s * (am[(size_t)t * n + i1] - am[(size_t)t * n + i]) + (float)P * (fnext - fprev);
  }
  __syncthreads();
  // forward real DFT along the bins: slot 0, cos/sin pairs, Nyquist for even n
  for (size_t q = tid; q < mlen; q += nt) {
    const int t = (int)(q / n), slot = (int)(q % n);
    const float* row = r + (size_t)t * n;
    float acc = 0.f;
    if (slot == 0) {
      for (int i = 0; i < n; ++i) acc += row[i];
    } else if ((n & 1) == 0 && slot == n - 1) {
      for (int i = 0; i < n; ++i) acc += (i & 1) ? -row[i] : row[i];
    } else {
      const int j = (slot + 1) / 2;
      int m = 0;
      for (int i = 0; i < n; ++i) {
        const float2 w = cs[m];
        acc += row[i] * ((slot & 1) ? w.x : w.y);
        m += j;
        if (m >= n) m -= n;
      }
    }
    h[q] = acc;
  }
  __syncthreads();
  // DCT-II along t, divide by the eigenvalue (zero mode -> 0), exact inverse.  Eigenvalues below
  // lam_fp64 (the hue plan's default threshold of 64) are formed and divided in double, as the plan does.
  for (int slot = tid; slot < n; slot += nt) {
    float v[kMaxP], w[kMaxP];
    for (int t = 0; t < P; ++t) v[t] = h[(size_t)t * n + slot];
    for (int k = 0; k < P; ++k) {
      float acc = 0.f;
      for (int t = 0; t < P; ++t) acc += Mt[k * P + t] * v[t];
      const float l = lam[slot] + lamt[k];
      if (!(l > 0.f)) {
        w[k] = 0.f;
      } else if (l < kLamFp64) {
        int j = (slot + 1) / 2;
        if ((n & 1) == 0 && slot == n - 1) j = n / 2;
        const double vs = sinpi((double)j / n), vt = sinpi((double)k / (2.0 * P));
        const double ld = s * s * 4.0 * vs * vs + (double)P * P * 4.0 * vt * vt;
        w[k] = ld > 0.0 ? (float)((double)acc / ld) : 0.f;
      } else {
        w[k] = acc / l;
      }
    }
    for (int t = 0; t < P; ++t) {
      float acc = 0.f;
      for (int k = 0; k < P; ++k) acc += (k == 0 ? 1.f : 2.f) * Mt[k * P + t] * w[k];
      h[(size_t)t * n + slot] = acc / (float)P;
    }
  }
  __syncthreads();
  // inverse real DFT -> phi: frequency j has the slot pair (2j - 1, 2j) and the basis index
  // i j mod n, which advances by i per frequency
  float* ph = phi + (size_t)b * mlen;
  for (size_t q = tid; q < mlen; q += nt) {
    const int t = (int)(q / n), i = (int)(q % n);
    const float* row = h + (size_t)t * n;
    float acc = row[0];
    const int last = (n & 1) ? n : n - 1;
    int m = 0;
    for (int slot = 1; slot < last; slot += 2) {
      m += i;
      if (m >= n) m -= n;
      const float2 w = cs[m];
      acc += 2.f * (row[slot] * w.x + row[slot + 1] * w.y);
    }
    if ((n & 1) == 0) acc += row[n - 1] * ((i & 1) ? -1.f : 1.f);
    ph[q] = acc / (float)n;
  }
  __syncthreads();
  // x = a - A^T phi: face i gets + s (phi_i - phi_{i-1}); f at time t+1 gets + P (phi_{t+1} - phi_t)
  float* xm = xp + (size_t)b * (mlen + flen);
  float* xf = xm + mlen;
  for (size_t q = tid; q < mlen; q += nt) {
    const int t = (int)(q / n), i = (int)(q % n);
    const int im = i == 0 ? n - 1 : i - 1;
    xm[q] = am[q] + (float)s * (ph[q] - ph[(size_t)t * n + im]);
    if (t < P - 1) xf[q] = af[q] + (float)P * (ph[q + n] - ph[q]);
  }
}

}  // namespace
}  // namespace dynot

using namespace dynot;

extern "C" ot_status ot_hue_project_noalloc(int bins, int P, int batch, double axis_scale, const float* f0,
                                            const float* f1, const float* a_packed, float* x_packed, float* phi,
                                            void* cuda_stream) {
  if (bins < 2 || bins > kMaxBins || P < 2 || P > kMaxP || batch < 1)
    return seterr(OT_EINVAL, "bins must be in [2, %d], P in [2, %d], batch >= 1", kMaxBins, kMaxP);
  if (!f0 || !f1 || !a_packed || !x_packed || !phi) return seterr(OT_EINVAL, "NULL buffer");
  const size_t need = (size_t)batch * 2 * (size_t)bins * P;
  if (need > kScratchFloats)
    return seterr(OT_EINVAL,
                  "batch * 2 * bins * P = %zu floats exceeds the fixed scratch of %zu floats; "
                  "split the batch into smaller calls",
                  need, kScratchFloats);
  if (!(axis_scale >= 0.0) || std::isinf(axis_scale))
    return seterr(OT_EINVAL, "axis_scale must be > 0 (or 0 for the default, bins)");
  const double s = axis_scale > 0 ? axis_scale : (double)bins;
  float* scratch = nullptr;
  ot_status st = scratch_for_current_device(&scratch);
  if (st != OT_OK) return st;
  const size_t smem = sizeof(float2) * bins + sizeof(float) * ((size_t)P * P + bins + P);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute((const void*)k_hue_project_noalloc,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return seterr(OT_ECUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
  }
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  k_hue_project_noalloc<<<batch, 256, smem, stream>>>(bins, P, s, f0, f1, a_packed, x_packed, phi, scratch);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return seterr(OT_ECUDA, "launch: %s", cudaGetErrorString(e));
  return OT_OK;   // queued on the stream; the caller orders its later work (and reads) after it
}
