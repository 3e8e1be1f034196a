// Hue image pipeline of section 5: HSV conversion, hue histograms and the
// periodic exact histogram specification that turns each transported hue
// histogram h^t back into an image (saturation and value kept).
//
// The paper cites, without printing them, an analysis of transport on the
// circle and an exact specification method.  The reading implemented here:
// pixels are ranked by a strict order (hue quantised to 32 bits, then pixel
// index); the target histogram becomes exact integer counts (largest
// remainders, ties to the lower bin); target rank q in bin b gets the hue
// (b + (q - C_b + 1/2) / c_b) / bins; the circle is cut at the cyclic shift s of
// least squared circular distance sum_r d(x_r, y_{(r-s) mod n})^2 over all n
// shifts (ties to the smaller shift).  For sorted points on the circle and a
// cost convex in the circular distance an optimal matching is a cyclic shift of
// the sorted orders, so this cut is the optimal assignment of the source pixels
// to the target hues.
#include "../../include/dynot.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "abi_guard.h"
#include "plan_base.h"

namespace dynot {
namespace {

__global__ void k_rgb_to_hsv(int n, const float* __restrict__ rgb, float* __restrict__ h, float* __restrict__ s,
                             float* __restrict__ v) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float r = rgb[i], g = rgb[(size_t)n + i], b = rgb[2 * (size_t)n + i];
    const float mx = fmaxf(fmaxf(r, g), b), mn = fminf(fminf(r, g), b), d = mx - mn;
    float hh = 0.f;
    if (d > 0.f) {
      if (mx == r) {
        hh = (g - b) / d;
        if (hh < 0.f) hh += 6.f;
      } else if (mx == g) {
        hh = (b - r) / d + 2.f;
      } else {
        hh = (r - g) / d + 4.f;
      }
      hh /= 6.f;
      if (hh >= 1.f) hh -= 1.f;
    }
    h[i] = hh;
    s[i] = mx > 0.f ? d / mx : 0.f;
    v[i] = mx;
  }
}

__global__ void k_hsv_to_rgb(int n, const float* __restrict__ h, const float* __restrict__ s,
                             const float* __restrict__ v, float* __restrict__ rgb) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float h6 = h[i] * 6.f;
    const float fl = floorf(h6);
    const int sec = ((int)fl % 6 + 6) % 6;
    const float f = h6 - fl, vv = v[i], ss = s[i];
    const float p = vv * (1.f - ss), q = vv * (1.f - ss * f), t = vv * (1.f - ss * (1.f - f));
    float r, g, b;
    switch (sec) {
      case 0: r = vv; g = t; b = p; break;
      case 1: r = q; g = vv; b = p; break;
      case 2: r = p; g = vv; b = t; break;
      case 3: r = p; g = q; b = vv; break;
      case 4: r = t; g = p; b = vv; break;
      default: r = vv; g = p; b = q; break;
    }
    rgb[i] = r;
    rgb[(size_t)n + i] = g;
    rgb[2 * (size_t)n + i] = b;
  }
}

__device__ __forceinline__ int hue_bin_of(float h, int bins) {
  return min((int)floor((double)h * bins), bins - 1);
}

// counts (float, exact below 2^24 per bin) then normalisation in a second kernel
__global__ void k_hue_count(int n, const float* __restrict__ h, int bins, float* __restrict__ cnt) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    atomicAdd(&cnt[max(hue_bin_of(h[i], bins), 0)], 1.f);
}
__global__ void k_scale(int n, float* __restrict__ x, float s) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] *= s;
}

// strict order keys: (hue quantised to 32 bits) << 32 | index; padding keys sort last
__global__ void k_hue_keys(int n, int m, const float* __restrict__ h, unsigned long long* __restrict__ key) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    if (i < n) {
      const double q = fmin(floor((double)h[i] * 4294967296.0), 4294967295.0);
      key[i] = ((unsigned long long)q << 32) | (unsigned long long)i;
    } else {
      key[i] = ~0ULL;
    }
  }
}

// one compare-exchange stage (k, j) of an ascending bitonic sort of m = 2^p keys
__global__ void k_bitonic(unsigned long long* __restrict__ key, int m, int k, int j) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const int l = i ^ j;
    if (l > i) {
      const unsigned long long a = key[i], b = key[l];
      const bool up = (i & k) == 0;
      if ((a > b) == up) {
        key[i] = b;
        key[l] = a;
      }
    }
  }
}

// sorted source hues x_r (double) and pixel index of rank r
__global__ void k_sorted_hues(int n, const unsigned long long* __restrict__ key, const float* __restrict__ h,
                              double* __restrict__ x, int* __restrict__ idx) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const int i = (int)(key[r] & 0xffffffffULL);
    idx[r] = i;
    x[r] = (double)h[i];
  }
}

// target hue of rank q: bin b with C_b <= q < C_{b+1}, (b + (q - C_b + 1/2) / c_b) / bins
__global__ void k_target_hues(int n, int bins, const long long* __restrict__ C, double* __restrict__ y) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    int lo = 0, hi = bins;   // largest b with C[b] <= q
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (C[mid] <= q) lo = mid;
      else hi = mid;
    }
    const double cb = (double)(C[lo + 1] - C[lo]);
    y[q] = ((double)lo + ((double)(q - C[lo]) + 0.5) / cb) / bins;
  }
}

// cost[s] = sum_r d(x_r, y_{(r - s) mod n})^2 for every shift s (exhaustive search).  A block takes
// kShiftBlock consecutive shifts, kShiftPer per thread (s = s0 + tid + kShiftThreads u), and walks r in
// tiles of kShiftTile: the tile of x and the window of y that its shifts reach sit in shared memory, x
// read as a broadcast and y at consecutive addresses across the threads.  The target hue is held as a
// float pair (hi + lo = y to about 2^-48), so x - y is formed to about one unit in the last place of
// the difference; the terms of a tile are summed in float, the tiles in double.
constexpr int kShiftThreads = 256, kShiftPer = 4, kShiftBlock = kShiftThreads * kShiftPer, kShiftTile = 256;
constexpr int kShiftWin = kShiftTile + kShiftBlock - 1;

__global__ void __launch_bounds__(kShiftThreads) k_shift_costs(int n, const float* __restrict__ xs,
                                                               const float2* __restrict__ ys,
                                                               double* __restrict__ cost) {
  __shared__ float sx[kShiftTile];
  __shared__ float2 sy[kShiftWin];
  const int s0 = blockIdx.x * kShiftBlock, tid = threadIdx.x;
  double acc[kShiftPer];
#pragma unroll
  for (int u = 0; u < kShiftPer; ++u) acc[u] = 0.0;
  for (int r0 = 0; r0 < n; r0 += kShiftTile) {
    const int len = min(kShiftTile, n - r0);
    __syncthreads();
    for (int i = tid; i < len; i += kShiftThreads) sx[i] = xs[r0 + i];
    // window entry i holds y at q = r0 - s0 - (kShiftBlock - 1) + i (mod n)
    const long long qb = (long long)r0 - s0 - (kShiftBlock - 1);
    for (int i = tid; i < len + kShiftBlock - 1; i += kShiftThreads) {
      long long q = (qb + i) % n;
      if (q < 0) q += n;
      sy[i] = ys[q];
    }
    __syncthreads();
    float part[kShiftPer];
#pragma unroll
    for (int u = 0; u < kShiftPer; ++u) part[u] = 0.f;
    // thread (tid, u) has shift s = s0 + tid + kShiftThreads u; term r reads sy[r - r0 + kShiftBlock - 1 - (s - s0)]
    const int wb = kShiftBlock - 1 - tid;
#pragma unroll 4
    for (int r = 0; r < len; ++r) {
      const float xv = sx[r];
#pragma unroll
      for (int u = 0; u < kShiftPer; ++u) {
        const float2 yv = sy[r + wb - kShiftThreads * u];
        const float e = fabsf((xv - yv.x) - yv.y);
        const float d = fminf(e, 1.f - e);
        part[u] = fmaf(d, d, part[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < kShiftPer; ++u) acc[u] += (double)part[u];
  }
#pragma unroll
  for (int u = 0; u < kShiftPer; ++u) {
    const int s = s0 + tid + kShiftThreads * u;
    if (s < n) cost[s] = acc[u];
  }
}

// the first minimiser of cost over [0, n) (ties to the smaller shift), one block
__global__ void k_argmin_shift(int n, const double* __restrict__ cost, int* __restrict__ best) {
  double bc = INFINITY;
  int bs = n;
  for (int s = threadIdx.x; s < n; s += blockDim.x) {
    const double c = cost[s];
    if (c < bc) { bc = c; bs = s; }   // s increases within a thread: the first minimiser is kept
  }
  __shared__ double rc[1024];
  __shared__ int rs[1024];
  rc[threadIdx.x] = bc;
  rs[threadIdx.x] = bs;
  __syncthreads();
  for (int w = blockDim.x >> 1; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      const double c2 = rc[threadIdx.x + w];
      const int s2 = rs[threadIdx.x + w];
      if (c2 < rc[threadIdx.x] || (c2 == rc[threadIdx.x] && s2 < rs[threadIdx.x])) {
        rc[threadIdx.x] = c2;
        rs[threadIdx.x] = s2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *best = rs[0] < n ? rs[0] : 0;
}

// float source hues of the sorted ranks and the target hues as float pairs
__global__ void k_shift_inputs(int n, const double* __restrict__ x, const double* __restrict__ y,
                               float* __restrict__ xs, float2* __restrict__ ys) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    xs[r] = (float)x[r];
    const float hi = (float)y[r];
    ys[r] = make_float2(hi, (float)(y[r] - (double)hi));
  }
}

// rank r receives target rank (r - s) mod n
__global__ void k_assign(int n, const int* __restrict__ shift, const int* __restrict__ idx,
                         const double* __restrict__ y, float* __restrict__ out) {
  const int s = *shift;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    int q = r - s;
    if (q < 0) q += n;
    out[idx[r]] = (float)y[q];
  }
}

inline int grid_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 152 * 16); }

// the exhaustive shift search costs npix^2 terms (about 0.15 s on one GPU at 2^20 pixels)
constexpr int kMaxSpecifyPixels = 1 << 21;

}  // namespace
}  // namespace dynot

using namespace dynot;

#define HP_CHECK()                                                                 \
  do {                                                                             \
    cudaError_t e_ = cudaGetLastError();                                           \
    if (e_ != cudaSuccess) return seterr(OT_ECUDA, "%s", cudaGetErrorString(e_)); \
  } while (0)

extern "C" {

ot_status ot_rgb_to_hsv(int npix, const float* rgb, float* h, float* s, float* v, void* stream) {
  if (npix < 0 || (npix > 0 && (!rgb || !h || !s || !v))) return seterr(OT_EINVAL, "bad rgb_to_hsv arguments");
  if (npix == 0) return OT_OK;
  k_rgb_to_hsv<<<grid_for(npix), 256, 0, (cudaStream_t)stream>>>(npix, rgb, h, s, v);
  HP_CHECK();
  return OT_OK;
}

ot_status ot_hsv_to_rgb(int npix, const float* h, const float* s, const float* v, float* rgb, void* stream) {
  if (npix < 0 || (npix > 0 && (!rgb || !h || !s || !v))) return seterr(OT_EINVAL, "bad hsv_to_rgb arguments");
  if (npix == 0) return OT_OK;
  k_hsv_to_rgb<<<grid_for(npix), 256, 0, (cudaStream_t)stream>>>(npix, h, s, v, rgb);
  HP_CHECK();
  return OT_OK;
}

ot_status ot_hue_histogram(int npix, const float* h, int bins, float* hist, void* stream) {
  if (npix < 1 || npix >= (1 << 24) || bins < 2 || !h || !hist)
    return seterr(OT_EINVAL, "hue_histogram: need 1 <= npix < 2^24, bins >= 2");
  cudaStream_t st = (cudaStream_t)stream;
  CUDA_OK(cudaMemsetAsync(hist, 0, sizeof(float) * bins, st));
  k_hue_count<<<grid_for(npix), 256, 0, st>>>(npix, h, bins, hist);
  HP_CHECK();
  k_scale<<<grid_for(bins), 256, 0, st>>>(bins, hist, (float)(1.0 / npix));
  HP_CHECK();
  return OT_OK;
}

ot_status ot_hue_specify(int npix, const float* h, int bins, const float* target, float* h_out, void* stream) {
  return ot_guard([&]() -> ot_status {
    if (npix < 1 || npix > kMaxSpecifyPixels || bins < 2 || !h || !target || !h_out)
      return seterr(OT_EINVAL, "hue_specify: need 1 <= npix <= 2^21, bins >= 2");
    cudaStream_t st = (cudaStream_t)stream;
    // exact counts of the target (host: bins values)
    std::vector<float> tg(bins);
    CUDA_OK(cudaMemcpyAsync(tg.data(), target, sizeof(float) * bins, cudaMemcpyDefault, st));
    CUDA_OK(cudaStreamSynchronize(st));
    // negative entries (an unconverged path can hold a few) count as empty; the rest is renormalised
    double mass = 0;
    for (int b = 0; b < bins; ++b) {
      if (!std::isfinite(tg[b])) return seterr(OT_EINVAL, "hue_specify: non-finite target");
      mass += tg[b] > 0.f ? (double)tg[b] : 0.0;
    }
    if (!(mass > 0)) return seterr(OT_EINVAL, "hue_specify: empty target");
    std::vector<long long> cnt(bins);
    std::vector<double> rem(bins);
    long long tot = 0;
    for (int b = 0; b < bins; ++b) {
      const double xb = (tg[b] > 0.f ? (double)tg[b] / mass : 0.0) * npix;
      cnt[b] = (long long)std::floor(xb);
      rem[b] = xb - (double)cnt[b];
      tot += cnt[b];
    }
    long long shortfall = npix - tot;
    if (shortfall < 0 || shortfall > bins) return seterr(OT_EINVAL, "hue_specify: bad target");
    std::vector<int> ord(bins);
    for (int b = 0; b < bins; ++b) ord[b] = b;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int c) { return rem[a] > rem[c]; });
    for (long long k = 0; k < shortfall; ++k) cnt[ord[k]] += 1;
    std::vector<long long> C(bins + 1, 0);
    for (int b = 0; b < bins; ++b) C[b + 1] = C[b] + cnt[b];
    // device workspace
    int m = 1;
    while (m < npix) m <<= 1;
    DevMem ws;
    const size_t bytes = sizeof(unsigned long long) * m + 2 * sizeof(double) * npix + sizeof(int) * npix +
                         sizeof(long long) * (bins + 1) + sizeof(float) * npix + sizeof(float2) * npix +
                         sizeof(double) * npix + 16 * 8 + 64;
    CUDA_OK(cudaMalloc(&ws.p, bytes));
    char* q = (char*)ws.p;
    auto take = [&](size_t b) { char* r = q; q += (b + 15) & ~size_t(15); return r; };
    unsigned long long* key = (unsigned long long*)take(sizeof(unsigned long long) * m);
    double* x = (double*)take(sizeof(double) * npix);
    double* y = (double*)take(sizeof(double) * npix);
    int* idx = (int*)take(sizeof(int) * npix);
    long long* dC = (long long*)take(sizeof(long long) * (bins + 1));
    float* xs = (float*)take(sizeof(float) * npix);
    float2* ys = (float2*)take(sizeof(float2) * npix);
    double* dcost = (double*)take(sizeof(double) * npix);
    int* dbest = (int*)take(sizeof(int));
    // strict order of the source hues
    k_hue_keys<<<grid_for(m), 256, 0, st>>>(npix, m, h, key);
    HP_CHECK();
    for (int k = 2; k <= m; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) k_bitonic<<<grid_for(m), 256, 0, st>>>(key, m, k, j);
    HP_CHECK();
    k_sorted_hues<<<grid_for(npix), 256, 0, st>>>(npix, key, h, x, idx);
    CUDA_OK(cudaMemcpyAsync(dC, C.data(), sizeof(long long) * (bins + 1), cudaMemcpyHostToDevice, st));
    k_target_hues<<<grid_for(npix), 256, 0, st>>>(npix, bins, dC, y);
    HP_CHECK();
    // least-cost cyclic shift over all npix shifts
    k_shift_inputs<<<grid_for(npix), 256, 0, st>>>(npix, x, y, xs, ys);
    HP_CHECK();
    k_shift_costs<<<(npix + kShiftBlock - 1) / kShiftBlock, kShiftThreads, 0, st>>>(npix, xs, ys, dcost);
    HP_CHECK();
    k_argmin_shift<<<1, 1024, 0, st>>>(npix, dcost, dbest);
    HP_CHECK();
    k_assign<<<grid_for(npix), 256, 0, st>>>(npix, dbest, idx, y, h_out);
    HP_CHECK();
    CUDA_OK(cudaStreamSynchronize(st));
    return OT_OK;
  });
}

}  // extern "C"
