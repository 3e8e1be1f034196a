// Kernels of the warm-start network: a 3D U-Net over (t, y, x) that maps the
// boundary densities of an RGB pair to an initial path x0 = (m, f) for
// Algorithm 1.  Activations are channels-last [n][t][y][x][c] in bf16,
// weights [cout][27][cin] in bf16 with fp32 master copies, accumulation fp32.
//
// The 3x3x3 convolutions are implicit GEMMs on the tensor cores
// (mma.sync m16n8k16, bf16 inputs, fp32 accumulators): M = voxels,
// N = output channels, K = 27 taps x input channels.  The data gradient is the
// same convolution with rotated, transposed weights; the weight gradient is a
// second implicit GEMM (M = cout, N = cin, K = voxels) per tap: the tiled
// kernel writes per-block partial sums over voxel chunks that a second kernel
// adds in a fixed order; the direct fallback for unaligned channel slices
// reduces with fp32 atomics.
#include "../../include/dynot.h"

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include <cudaTypedefs.h>

#include <cstdlib>
#include <cstring>

#include "common.cuh"
#include "nn_tcgen05.cuh"
#include "plan_base.h"

namespace dynot {
namespace {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t ld32(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }
__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

struct Vol {
  int N, T, Y, X;
  __host__ __device__ __forceinline__ long long count() const { return (long long)N * T * Y * X; }
};

// Forward 3x3x3 convolution with zero padding; warp tile 16 voxels x (8*NT) channels.
// x: channel stride xs, first channel xo; y: channel stride ys, first channel yo.
template <int NT>
__global__ void __launch_bounds__(128) k_conv3d(Vol v, int Cin, int Cout, const bf16* __restrict__ x, int xs, int xo,
                                                const bf16* __restrict__ w, const float* __restrict__ bias,
                                                void* __restrict__ y, int ys, int yo, int relu, int out_f32) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gid = lane >> 2, tig = lane & 3;
  const long long M = v.count();
  const long long m0 = ((long long)blockIdx.x * 4 + warp) * 16;
  const int co0 = blockIdx.y * 8 * NT;
  if (m0 >= M) return;
  // the two voxels (rows) of this lane
  long long vr[2] = {m0 + gid, m0 + gid + 8};
  int tt[2], yy[2], xx[2], nn[2];
  bool ok[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    ok[r] = vr[r] < M;
    long long q = ok[r] ? vr[r] : 0;
    xx[r] = (int)(q % v.X); q /= v.X;
    yy[r] = (int)(q % v.Y); q /= v.Y;
    tt[r] = (int)(q % v.T);
    nn[r] = (int)(q / v.T);
  }
  float acc[NT][4];
#pragma unroll
  for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
  for (int tap = 0; tap < 27; ++tap) {
    const int dt = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
    const bf16* src[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int t2 = tt[r] + dt, y2 = yy[r] + dy, x2 = xx[r] + dx;
      const bool in = ok[r] && t2 >= 0 && t2 < v.T && y2 >= 0 && y2 < v.Y && x2 >= 0 && x2 < v.X;
      src[r] = in ? x + ((((long long)nn[r] * v.T + t2) * v.Y + y2) * v.X + x2) * xs + xo : nullptr;
    }
    for (int ci = 0; ci < Cin; ci += 16) {
      const int c0 = ci + tig * 2;
      const uint32_t a0 = src[0] ? ld32(src[0] + c0) : 0u;
      const uint32_t a1 = src[1] ? ld32(src[1] + c0) : 0u;
      const uint32_t a2 = src[0] ? ld32(src[0] + c0 + 8) : 0u;
      const uint32_t a3 = src[1] ? ld32(src[1] + c0 + 8) : 0u;
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        const int co = co0 + j * 8 + gid;
        uint32_t b0 = 0u, b1 = 0u;
        if (co < Cout) {
          const bf16* wp = w + ((long long)co * 27 + tap) * Cin + c0;
          b0 = ld32(wp);
          b1 = ld32(wp + 8);
        }
        mma_bf16(acc[j], a0, a1, a2, a3, b0, b1);
      }
    }
  }
  // epilogue: bias, ReLU, store
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    const int co = co0 + j * 8 + tig * 2;
    if (co >= Cout) continue;
    const float bb0 = bias ? bias[co] : 0.f, bb1 = bias ? bias[co + 1] : 0.f;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      if (!ok[r]) continue;
      float u0 = acc[j][2 * r] + bb0, u1 = acc[j][2 * r + 1] + bb1;
      if (relu) {
        u0 = fmaxf(u0, 0.f);
        u1 = fmaxf(u1, 0.f);
      }
      const long long o = vr[r] * ys + yo + co;
      if (out_f32) {
        float* yp = (float*)y + o;
        yp[0] = u0;
        yp[1] = u1;
      } else {
        *reinterpret_cast<uint32_t*>((bf16*)y + o) = pack2(__float2bfloat16(u0), __float2bfloat16(u1));
      }
    }
  }
}

// The same convolution with the input staged in shared memory.  A block computes 4 rows of 32
// voxels (one warp per row, two m16 tiles) for 8 * NT output channels.  For each 16-channel slice
// of the input it stages the zero-padded halo [3][6][34] voxels x 16 channels with cp.async, then
// runs the 27 taps: the A fragments of a tap are ldmatrix loads from the halo rows shifted by the
// tap (no per-tap address or bounds arithmetic), the B fragments come from the weights as above.
// Halo rows are 32 bytes (16 channels); the two 16-byte halves of voxel v are swapped when
// (v >> 2) & 1 so that the eight rows of one ldmatrix hit distinct banks.  Needs the input's
// channel stride and offset to be multiples of 8 (16-byte pieces).
constexpr int kCT_TY = 4, kCT_TX = 32, kCT_HY = kCT_TY + 2, kCT_HX = kCT_TX + 2;
constexpr int kCT_HV = 3 * kCT_HY * kCT_HX;   // halo voxels

__device__ __forceinline__ int ct_half_off(int v, int half) { return v * 32 + ((half ^ ((v >> 2) & 1)) << 4); }

template <int NT>
__global__ void __launch_bounds__(128) k_conv3d_tiled(Vol v, int Cin, int Cout, const bf16* __restrict__ x, int xs,
                                                      int xo, const bf16* __restrict__ w,
                                                      const float* __restrict__ bias, void* __restrict__ y, int ys,
                                                      int yo, int relu, int out_f32) {
  __shared__ __align__(128) unsigned char halo[kCT_HV * 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gid = lane >> 2, tig = lane & 3;
  const int nxb = (v.X + kCT_TX - 1) / kCT_TX;
  const int x0 = (blockIdx.x % nxb) * kCT_TX, y0 = (blockIdx.x / nxb) * kCT_TY;
  const int t = blockIdx.y % v.T, n = blockIdx.y / v.T;
  const int co0 = blockIdx.z * 8 * NT;
  float acc[2][NT][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int j = 0; j < NT; ++j) acc[mt][j][0] = acc[mt][j][1] = acc[mt][j][2] = acc[mt][j][3] = 0.f;
  const unsigned hbase = (unsigned)__cvta_generic_to_shared(halo);
  // ldmatrix row of this lane: matrix (lane >> 3) = (m rows 0-7 | 8-15) x (channels 0-7 | 8-15)
  const int mrow = ((lane >> 3) & 1) * 8 + (lane & 7), mhalf = lane >> 4;
  for (int ci0 = 0; ci0 < Cin; ci0 += 16) {
    // stage the halo of this channel slice (zeros outside the volume)
    for (int i = threadIdx.x; i < kCT_HV * 2; i += blockDim.x) {
      const int hv = i >> 1, half = i & 1;
      const int hx = hv % kCT_HX, hy = (hv / kCT_HX) % kCT_HY, ht = hv / (kCT_HX * kCT_HY);
      const int gx = x0 + hx - 1, gy = y0 + hy - 1, gt = t + ht - 1;
      unsigned char* dst = halo + ct_half_off(hv, half);
      if (gx >= 0 && gx < v.X && gy >= 0 && gy < v.Y && gt >= 0 && gt < v.T) {
        const bf16* src = x + ((((long long)n * v.T + gt) * v.Y + gy) * v.X + gx) * xs + xo + ci0 + half * 8;
        cp_async16(dst, src);
      } else {
        *reinterpret_cast<uint4*>(dst) = make_uint4(0u, 0u, 0u, 0u);
      }
    }
    cp_async_wait_all();
    __syncthreads();
    for (int tap = 0; tap < 27; ++tap) {
      const int dt = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;   // offsets + 1 into the halo
      uint32_t a[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const int hv = (dt * kCT_HY + warp + dy) * kCT_HX + mt * 16 + mrow + dx;
        const unsigned addr = hbase + (unsigned)ct_half_off(hv, mhalf);
        asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                     : "=r"(a[mt][0]), "=r"(a[mt][1]), "=r"(a[mt][2]), "=r"(a[mt][3])
                     : "r"(addr));
      }
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        const int co = co0 + j * 8 + gid;
        uint32_t b0 = 0u, b1 = 0u;
        if (co < Cout) {
          const bf16* wp = w + ((long long)co * 27 + tap) * Cin + ci0 + tig * 2;
          b0 = ld32(wp);
          b1 = ld32(wp + 8);
        }
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) mma_bf16(acc[mt][j], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b0, b1);
      }
    }
    __syncthreads();
  }
  // epilogue: bias, ReLU, store (rows gid, gid + 8 of each m16 tile = voxels x0 + 16 mt + gid (+8))
  const int yy = y0 + warp;
  if (yy >= v.Y) return;
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    const int co = co0 + j * 8 + tig * 2;
    if (co >= Cout) continue;
    const float bb0 = bias ? bias[co] : 0.f, bb1 = bias ? bias[co + 1] : 0.f;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int xx = x0 + mt * 16 + gid + r * 8;
        if (xx >= v.X) continue;
        float u0 = acc[mt][j][2 * r] + bb0, u1 = acc[mt][j][2 * r + 1] + bb1;
        if (relu) {
          u0 = fmaxf(u0, 0.f);
          u1 = fmaxf(u1, 0.f);
        }
        const long long vox = (((long long)n * v.T + t) * v.Y + yy) * v.X + xx;
        const long long o = vox * ys + yo + co;
        if (out_f32) {
          float* yp = (float*)y + o;
          yp[0] = u0;
          yp[1] = u1;
        } else {
          *reinterpret_cast<uint32_t*>((bf16*)y + o) = pack2(__float2bfloat16(u0), __float2bfloat16(u1));
        }
      }
  }
}

// Weight gradient: dw[co][tap][ci] += sum_v dy[v][co] x[v + tap][ci] over a chunk of voxels.
// Block: 4 warps over 4 sub-chunks of the same (tap, co tile of 16, ci tile of 16).  Voxel indices
// are 32-bit (the caller checks N*T*Y*X < 2^31).
__global__ void __launch_bounds__(128) k_conv3d_wgrad(Vol v, int Cin, int Cout, const bf16* __restrict__ x, int xs,
                                                      int xo, const bf16* __restrict__ dy, int dys, int dyo,
                                                      float* __restrict__ dw, int chunk) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gid = lane >> 2, tig = lane & 3;
  const int tap = blockIdx.y;
  const int ntile_ci = Cin / 16;
  const int co0 = (blockIdx.z / ntile_ci) * 16, ci0 = (blockIdx.z % ntile_ci) * 16;
  const int dt = tap / 9 - 1, ddy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
  const int M = (int)v.count();
  const int vbeg = blockIdx.x * chunk;
  const int vend = min(M, vbeg + chunk);
  const int sub = (chunk + 3) / 4;
  const int wb = vbeg + warp * sub, we = min(vend, wb + sub);
  float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
  // element offset of x[vox + tap] (channel 0 of the slice), or -1 outside the volume / chunk
  auto xoff = [&](int vox) -> int {
    if (vox >= we) return -1;
    int q = vox;
    const int x0 = q % v.X; q /= v.X;
    const int y0 = q % v.Y; q /= v.Y;
    const int t0 = q % v.T;
    const int n0 = q / v.T;
    const int t2 = t0 + dt, y2 = y0 + ddy, x2 = x0 + dx;
    if (t2 < 0 || t2 >= v.T || y2 < 0 || y2 >= v.Y || x2 < 0 || x2 >= v.X) return -1;
    return (((n0 * v.T + t2) * v.Y + y2) * v.X + x2) * xs + xo;
  };
  const bf16 zero = __float2bfloat16(0.f);
  auto dyval = [&](int vox, int c) -> bf16 { return vox < we ? dy[(long long)vox * dys + dyo + c] : zero; };
  for (int k0 = wb; k0 < we; k0 += 16) {
    // A = dy^T (rows co, cols voxels): a0 (co gid, vox tig*2 + {0,1}), a1 (co gid+8), a2 (+8 vox), a3
    const int kv = k0 + tig * 2;
    const uint32_t a0 = pack2(dyval(kv, co0 + gid), dyval(kv + 1, co0 + gid));
    const uint32_t a1 = pack2(dyval(kv, co0 + gid + 8), dyval(kv + 1, co0 + gid + 8));
    const uint32_t a2 = pack2(dyval(kv + 8, co0 + gid), dyval(kv + 9, co0 + gid));
    const uint32_t a3 = pack2(dyval(kv + 8, co0 + gid + 8), dyval(kv + 9, co0 + gid + 8));
    const int o0 = xoff(kv), o1 = xoff(kv + 1), o8 = xoff(kv + 8), o9 = xoff(kv + 9);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      // B = shifted x (rows voxels, cols ci): b0 (vox tig*2 + {0,1}, ci gid), b1 (vox + 8)
      const int c = ci0 + j * 8 + gid;
      const uint32_t b0 = pack2(o0 >= 0 ? x[o0 + c] : zero, o1 >= 0 ? x[o1 + c] : zero);
      const uint32_t b1 = pack2(o8 >= 0 ? x[o8 + c] : zero, o9 >= 0 ? x[o9 + c] : zero);
      mma_bf16(acc[j], a0, a1, a2, a3, b0, b1);
    }
  }
  // reduce the 4 warps in shared memory, then one atomic per output element
  __shared__ float red[4][16][16];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    red[warp][gid][j * 8 + tig * 2] = acc[j][0];
    red[warp][gid][j * 8 + tig * 2 + 1] = acc[j][1];
    red[warp][gid + 8][j * 8 + tig * 2] = acc[j][2];
    red[warp][gid + 8][j * 8 + tig * 2 + 1] = acc[j][3];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 256; e += blockDim.x) {
    const int r = e / 16, c = e % 16;
    const float s = red[0][r][c] + red[1][r][c] + red[2][r][c] + red[3][r][c];
    atomicAdd(&dw[((long long)(co0 + r) * 27 + tap) * Cin + ci0 + c], s);
  }
}

// Weight gradient with shared-memory staging.  A block owns one (16 output x 16 input channel) slice
// and a strided set of 4 x 32 voxel tiles; per tile it stages the input halo (as k_conv3d_tiled) and
// the 128 voxels x 16 channels of dy, then every warp forms, for its taps (tap = warp + 4 i), the
// 16 x 16 product dy^T x_shifted over the tile's voxels: A = dy^T and B = shifted x come from
// ldmatrix.trans on the staged rows.  Each block writes its 27 x 16 x 16 partial sums to `part`;
// k_wgrad_reduce adds the blocks' partials into dw (no atomics, a fixed summation order).
constexpr int kWG_TAPS = 7;   // taps per warp (27 over 4 warps)

__global__ void __launch_bounds__(128) k_conv3d_wgrad_tiled(Vol v, int Cin, int Cout, const bf16* __restrict__ x,
                                                            int xs, int xo, const bf16* __restrict__ dy, int dys,
                                                            int dyo, float* __restrict__ part, int ntiles) {
  __shared__ __align__(128) unsigned char halo[kCT_HV * 32];
  __shared__ __align__(128) unsigned char dyt[kCT_TY * kCT_TX * 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gid = lane >> 2, tig = lane & 3;
  const int nci = Cin / 16;
  const int ci0 = (blockIdx.y % nci) * 16, co0 = (blockIdx.y / nci) * 16;
  const int nxb = (v.X + kCT_TX - 1) / kCT_TX, nyb = (v.Y + kCT_TY - 1) / kCT_TY;
  float acc[kWG_TAPS][2][4];
#pragma unroll
  for (int i = 0; i < kWG_TAPS; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[i][j][0] = acc[i][j][1] = acc[i][j][2] = acc[i][j][3] = 0.f;
  const unsigned hbase = (unsigned)__cvta_generic_to_shared(halo);
  const unsigned dbase = (unsigned)__cvta_generic_to_shared(dyt);
  // ldmatrix lane roles: matrix (lane >> 3): voxel block ((lane >> 3) >> 1) * 8, channel half (lane >> 3) & 1
  // for A = dy^T; for B the same split with the channel half selecting the n8 tile
  const int lrow = lane & 7, lmat = lane >> 3;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int xb = tile % nxb, yb = (tile / nxb) % nyb, nt = tile / (nxb * nyb);
    const int x0 = xb * kCT_TX, y0 = yb * kCT_TY, t = nt % v.T, n = nt / v.T;
    for (int i = threadIdx.x; i < kCT_HV * 2; i += blockDim.x) {
      const int hv = i >> 1, half = i & 1;
      const int hx = hv % kCT_HX, hy = (hv / kCT_HX) % kCT_HY, ht = hv / (kCT_HX * kCT_HY);
      const int gx = x0 + hx - 1, gy = y0 + hy - 1, gt = t + ht - 1;
      unsigned char* dst = halo + ct_half_off(hv, half);
      if (gx >= 0 && gx < v.X && gy >= 0 && gy < v.Y && gt >= 0 && gt < v.T)
        cp_async16(dst, x + ((((long long)n * v.T + gt) * v.Y + gy) * v.X + gx) * xs + xo + ci0 + half * 8);
      else
        *reinterpret_cast<uint4*>(dst) = make_uint4(0u, 0u, 0u, 0u);
    }
    for (int i = threadIdx.x; i < kCT_TY * kCT_TX * 2; i += blockDim.x) {
      const int tv = i >> 1, half = i & 1;
      const int gx = x0 + (tv % kCT_TX), gy = y0 + tv / kCT_TX;
      unsigned char* dst = dyt + ct_half_off(tv, half);
      if (gx < v.X && gy < v.Y)
        cp_async16(dst, dy + ((((long long)n * v.T + t) * v.Y + gy) * v.X + gx) * dys + dyo + co0 + half * 8);
      else
        *reinterpret_cast<uint4*>(dst) = make_uint4(0u, 0u, 0u, 0u);
    }
    cp_async_wait_all();
    __syncthreads();
    for (int ks = 0; ks < kCT_TY * kCT_TX / 16; ++ks) {
      const int row = ks >> 1, xk = (ks & 1) * 16;   // 16 voxels x0 + xk .. + 15 of tile row `row`
      // A = dy^T (co x voxel): matrices (voxels 0-7 | 8-15) x (co 0-7 | 8-15), transposed on load
      uint32_t a0, a1, a2, a3;
      {
        const int tv = row * kCT_TX + xk + (lmat >> 1) * 8 + lrow;
        const unsigned addr = dbase + (unsigned)ct_half_off(tv, lmat & 1);
        asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                     : "=r"(a0), "=r"(a1), "=r"(a2), "=r"(a3)
                     : "r"(addr));
      }
#pragma unroll
      for (int i = 0; i < kWG_TAPS; ++i) {
        const int tap = warp + 4 * i;
        if (tap < 27) {
          const int dt = tap / 9, ddy = (tap / 3) % 3, dx = tap % 3;
          // B = shifted x (voxel x ci): matrices (voxels 0-7 | 8-15) x (ci 0-7 | 8-15), transposed on load
          const int hv = (dt * kCT_HY + row + ddy) * kCT_HX + xk + (lmat >> 1) * 8 + lrow + dx;
          const unsigned addr = hbase + (unsigned)ct_half_off(hv, lmat & 1);
          uint32_t b00, b01, b10, b11;
          asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                       : "=r"(b00), "=r"(b10), "=r"(b01), "=r"(b11)
                       : "r"(addr));
          mma_bf16(acc[i][0], a0, a1, a2, a3, b00, b01);
          mma_bf16(acc[i][1], a0, a1, a2, a3, b10, b11);
        }
      }
    }
    __syncthreads();
  }
  // partials: part[block][tap][co 16][ci 16]
  float* pp = part + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * (27 * 256);
#pragma unroll
  for (int i = 0; i < kWG_TAPS; ++i) {
    const int tap = warp + 4 * i;
    if (tap >= 27) continue;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      float* q = pp + tap * 256;
      const int ci = j * 8 + tig * 2;
      q[gid * 16 + ci] = acc[i][j][0];
      q[gid * 16 + ci + 1] = acc[i][j][1];
      q[(gid + 8) * 16 + ci] = acc[i][j][2];
      q[(gid + 8) * 16 + ci + 1] = acc[i][j][3];
    }
  }
}

// dw[co][tap][ci] += sum over the blocks of one channel slice of their partials
__global__ void k_wgrad_reduce(int Cin, int nblk, const float* __restrict__ part, float* __restrict__ dw) {
  const int slice = blockIdx.y, nci = Cin / 16;
  const int ci0 = (slice % nci) * 16, co0 = (slice / nci) * 16;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 27 * 256; e += gridDim.x * blockDim.x) {
    const float* p = part + (size_t)slice * nblk * (27 * 256) + e;
    float s = 0.f;
    for (int k = 0; k < nblk; ++k) s += p[(size_t)k * (27 * 256)];
    const int tap = e / 256, co = (e / 16) % 16, ci = e % 16;
    dw[((size_t)(co0 + co) * 27 + tap) * Cin + ci0 + ci] += s;
  }
}

// dw[co][tap][ci] += sum over the chunks of the tcgen05 weight gradient's partials [chunk][tap][co][ci]
__global__ void k_wgrad_reduce_tc(int Cin, int Cout, int nchunks, const float* __restrict__ part,
                                  float* __restrict__ dw) {
  const int tap = blockIdx.x, co = blockIdx.y;
  for (int ci = threadIdx.x; ci < Cin; ci += blockDim.x) {
    const float* p = part + ((size_t)tap * Cout + co) * Cin + ci;
    float s = 0.f;
    for (int k = 0; k < nchunks; ++k) s += p[(size_t)k * 27 * Cout * Cin];
    dw[((size_t)co * 27 + tap) * Cin + ci] += s;
  }
}

// db[c] += sum_v dy[v][c]
__global__ void k_bias_grad(long long M, int C, const bf16* __restrict__ dy, int dys, int dyo, float* __restrict__ db) {
  const int c = blockIdx.y;
  float s = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x)
    s += __bfloat162float(dy[i * dys + dyo + c]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ float red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    atomicAdd(&db[c], t);
  }
}

// wr[ci][tap][co] = w[co][26 - tap][ci] (weights of the data-gradient convolution)
__global__ void k_rotate_weights(int Cin, int Cout, const bf16* __restrict__ w, bf16* __restrict__ wr) {
  const long long n = (long long)Cin * 27 * Cout;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int co = (int)(i % Cout);
    const int tap = (int)((i / Cout) % 27);
    const int ci = (int)(i / ((long long)Cout * 27));
    wr[i] = w[((long long)co * 27 + (26 - tap)) * Cin + ci];
  }
}

// g[v][c] *= (y[v][c] > 0)  (ReLU backward on the stored activation)
__global__ void k_relu_grad(long long M, int C, bf16* __restrict__ g, int gs, int go, const bf16* __restrict__ y,
                            int ys, int yo) {
  const long long n = M * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long vv = i / C;
    const int c = (int)(i % C);
    if (!(__bfloat162float(y[vv * ys + yo + c]) > 0.f)) g[vv * gs + go + c] = __float2bfloat16(0.f);
  }
}

// 2 x 2 average pooling over (y, x); the inverse spreads a quarter of the gradient.
__global__ void k_pool(Vol vo, int C, const bf16* __restrict__ x, int xs, int xo, bf16* __restrict__ y, int ys,
                       int yo, int backward) {
  const long long n = vo.count() * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    long long q = i / C;
    const int x0 = (int)(q % vo.X); q /= vo.X;
    const int y0 = (int)(q % vo.Y); q /= vo.Y;   // q = n*T + t
    const long long rowbase = q * (2 * vo.Y);
    const long long fine00 = ((rowbase + 2 * y0) * (2 * vo.X) + 2 * x0);
    const long long fine10 = ((rowbase + 2 * y0 + 1) * (2 * vo.X) + 2 * x0);
    const long long coarse = i / C;
    if (!backward) {
      const float s = __bfloat162float(x[fine00 * xs + xo + c]) + __bfloat162float(x[(fine00 + 1) * xs + xo + c]) +
                      __bfloat162float(x[fine10 * xs + xo + c]) + __bfloat162float(x[(fine10 + 1) * xs + xo + c]);
      y[coarse * ys + yo + c] = __float2bfloat16(0.25f * s);
    } else {   // x = coarse gradient, y = fine gradient (overwritten)
      const bf16 gq = __float2bfloat16(0.25f * __bfloat162float(x[coarse * xs + xo + c]));
      y[fine00 * ys + yo + c] = gq;
      y[(fine00 + 1) * ys + yo + c] = gq;
      y[fine10 * ys + yo + c] = gq;
      y[(fine10 + 1) * ys + yo + c] = gq;
    }
  }
}

// nearest 2x upsampling over (y, x); the inverse sums the four fine gradients.
__global__ void k_upsample(Vol vc, int C, const bf16* __restrict__ x, int xs, int xo, bf16* __restrict__ y, int ys,
                           int yo, int backward) {
  const long long n = vc.count() * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    long long q = i / C;
    const int x0 = (int)(q % vc.X); q /= vc.X;
    const int y0 = (int)(q % vc.Y); q /= vc.Y;
    const long long rowbase = q * (2 * vc.Y);
    const long long f00 = ((rowbase + 2 * y0) * (2 * vc.X) + 2 * x0);
    const long long f10 = ((rowbase + 2 * y0 + 1) * (2 * vc.X) + 2 * x0);
    const long long coarse = i / C;
    if (!backward) {   // x coarse -> y fine
      const bf16 val = x[coarse * xs + xo + c];
      y[f00 * ys + yo + c] = val;
      y[(f00 + 1) * ys + yo + c] = val;
      y[f10 * ys + yo + c] = val;
      y[(f10 + 1) * ys + yo + c] = val;
    } else {           // x fine gradient -> y coarse gradient
      const float s = __bfloat162float(x[f00 * xs + xo + c]) + __bfloat162float(x[(f00 + 1) * xs + xo + c]) +
                      __bfloat162float(x[f10 * xs + xo + c]) + __bfloat162float(x[(f10 + 1) * xs + xo + c]);
      y[coarse * ys + yo + c] = __float2bfloat16(s);
    }
  }
}

// y[v][yo + c] += x[v][xo + c]  (gradients meeting at a skip connection)
__global__ void k_add_slice(long long M, int C, const bf16* __restrict__ x, int xs, int xo, bf16* __restrict__ y,
                            int ys, int yo) {
  const long long n = M * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long vv = i / C;
    const int c = (int)(i % C);
    const float s = __bfloat162float(y[vv * ys + yo + c]) + __bfloat162float(x[vv * xs + xo + c]);
    y[vv * ys + yo + c] = __float2bfloat16(s);
  }
}

// loss += sum over v, c < Cv of (out - target)^2 / count; g = 2 (out - target) / count (bf16, gs channels);
// target is bf16 [M][Cv]
__global__ void k_mse(long long M, int Cv, const float* __restrict__ out, int os, const bf16* __restrict__ target,
                      bf16* __restrict__ g, int gs, float inv_count, float* __restrict__ loss) {
  float s = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M * gs; i += (long long)gridDim.x * blockDim.x) {
    const long long vv = i / gs;
    const int c = (int)(i % gs);
    float d = 0.f;
    if (c < Cv) d = out[vv * os + c] - __bfloat162float(target[vv * Cv + c]);
    s += d * d;
    g[i] = __float2bfloat16(2.f * d * inv_count);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ float red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    atomicAdd(loss, t * inv_count);
  }
}

// AdamW (decoupled weight decay) on fp32 master weights; writes the bf16 copy.
__global__ void k_adamw(long long n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                        float* __restrict__ v, bf16* __restrict__ pb, float lr, float b1, float b2, float eps, float wd,
                        float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    float pi = p[i] * (1.f - lr * wd);
    pi -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    if (pb) pb[i] = __float2bfloat16(pi);
  }
}

__global__ void k_to_bf16(long long n, const float* __restrict__ x, bf16* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16(x[i]);
}

// Network input [n][t][y][x][Cp] from densities [n][3][y][x] times the per-problem scale sc (NULL = 1):
// channels 0-2 f0, 3-5 f1, 6-8 the linear interpolation (1 - tau) f0 + tau f1 at the time tau = (t + 1) / P
// of the t-th interior density, 9 the half time (t + 1/2) / P of the momenta, the rest zero.
__global__ void k_make_input(int N, int P, int Y, int X, int Cp, const float* __restrict__ f0,
                             const float* __restrict__ f1, const float* __restrict__ sc, bf16* __restrict__ out) {
  const long long n = (long long)N * P * Y * X;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    long long q = i;
    const int x = (int)(q % X); q /= X;
    const int y = (int)(q % Y); q /= Y;
    const int t = (int)(q % P);
    const int b = (int)(q / P);
    const float s = sc ? sc[b] : 1.f;
    const float tau = (float)(t + 1) / (float)P;
    bf16* o = out + i * Cp;
    for (int c = 0; c < 3; ++c) {
      const long long k = (((long long)b * 3 + c) * Y + y) * X + x;
      const float a0 = f0[k] * s, a1 = f1[k] * s;
      o[c] = __float2bfloat16(a0);
      o[3 + c] = __float2bfloat16(a1);
      o[6 + c] = __float2bfloat16((1.f - tau) * a0 + tau * a1);
    }
    o[9] = __float2bfloat16(((float)t + 0.5f) / (float)P);
    for (int c = 10; c < Cp; ++c) o[c] = __float2bfloat16(0.f);
  }
}

// Compact path (the ABI's packed layout of one problem: m_x | m_y | m_c | f) <-> the 12 cell-aligned
// channels [t][y][x][k*3 + c] (k = x, y, colour faces, f; the face right of the cell, zero where absent).
// With densities f0, f1 (units of the packed path) the f channels hold the deviation from the linear
// interpolation L_t = (1 - tau) f0 + tau f1, tau = (t + 1) / P:  ch = s (packed - L), packed = ch / s + L.
__global__ void k_path_channels(int Y, int X, int P, int to_channels, const float* __restrict__ sc,
                                const float* __restrict__ f0, const float* __restrict__ f1, float* __restrict__ packed,
                                float* __restrict__ ch, int cs, int Nb) {
  const int C = 3;
  const long long offy = (long long)P * C * Y * (X - 1);
  const long long offc = offy + (long long)P * C * (Y - 1) * X;
  const long long offf = offc + (long long)P * C * Y * X;
  const long long total = offf + (long long)(P - 1) * C * Y * X;
  const long long n = (long long)Nb * P * Y * X * 12;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int ch12 = (int)(i % 12);
    long long q = i / 12;
    const int x = (int)(q % X); q /= X;
    const int y = (int)(q % Y); q /= Y;
    const int t = (int)(q % P);
    const int b = (int)(q / P);
    const int k = ch12 / 3, c = ch12 % 3;
    long long idx = -1;
    if (k == 0 && x < X - 1) idx = (((long long)t * C + c) * Y + y) * (X - 1) + x;
    else if (k == 1 && y < Y - 1) idx = offy + (((long long)t * C + c) * (Y - 1) + y) * X + x;
    else if (k == 2) idx = offc + (((long long)t * C + (c + 1) % C) * Y + y) * X + x;   // right face = paper face c+1
    else if (k == 3 && t < P - 1) idx = offf + (((long long)t * C + c) * Y + y) * X + x;
    const float s = sc ? sc[b] : 1.f;
    float L = 0.f;
    if (k == 3 && idx >= 0 && f0) {
      const long long d = (((long long)b * C + c) * Y + y) * X + x;
      const float tau = (float)(t + 1) / (float)P;
      L = (1.f - tau) * f0[d] + tau * f1[d];
    }
    if (idx >= 0) idx += (long long)b * total;
    const long long e = (i / 12) * cs + ch12;   // channel stride cs >= 12
    if (to_channels) ch[e] = idx >= 0 ? (packed[idx] - L) * s : 0.f;
    else if (idx >= 0) packed[idx] = ch[e] / s + L;
  }
}

// Packed dual (the ABI's layout of ot_state_get: per problem the cell arrays b_mx | b_my | b_mc | b_f,
// each [t][c][y][x]) <-> channels co + k*3 + c of [N][P][Y][X][cs].
__global__ void k_dual_channels(int Y, int X, int P, int to_channels, float* __restrict__ packed,
                                float* __restrict__ ch, int cs, int co, int Nb) {
  const long long cells = (long long)P * 3 * Y * X;
  const long long n = (long long)Nb * P * Y * X * 12;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int ch12 = (int)(i % 12);
    long long q = i / 12;
    const int x = (int)(q % X); q /= X;
    const int y = (int)(q % Y); q /= Y;
    const int t = (int)(q % P);
    const int b = (int)(q / P);
    const int k = ch12 / 3, c = ch12 % 3;
    const long long idx = ((long long)b * 4 + k) * cells + (((long long)t * 3 + c) * Y + y) * X + x;
    const long long e = (i / 12) * cs + co + ch12;
    if (to_channels) ch[e] = packed[idx];
    else packed[idx] = ch[e];
  }
}

inline int blocks_for(long long n) { return (int)((n + 255) / 256 < 152 * 32 ? (n + 255) / 256 : 152 * 32); }

}  // namespace
}  // namespace dynot

using namespace dynot;

#define NN_LAUNCH_CHECK()                                                          \
  do {                                                                             \
    cudaError_t e_ = cudaGetLastError();                                           \
    if (e_ != cudaSuccess) return seterr(OT_ECUDA, "%s", cudaGetErrorString(e_)); \
  } while (0)

extern "C" {

// cuTensorMapEncodeTiled from the driver, resolved once through the runtime
static PFN_cuTensorMapEncodeTiled_v12000 nn_tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return (PFN_cuTensorMapEncodeTiled_v12000)f;
  }();
  return fn;
}

// The tcgen05 form of the convolution where its layout rules hold: 16-channel input slices at 16-byte
// offsets, Cout a multiple of 16 up to 256, 16-byte output vectors, and tiles of 128 voxels along x (and y).
// Returns false (nothing launched) where they do not, and for fewer than 32 output channels on rows shorter
// than 128 voxels;
// DYNOT_CONV=mma forces the mma.sync kernels, DYNOT_CONV=tcgen05 the tcgen05 forms wherever their rules
// hold, DYNOT_CONV=tap and =halo the per-tap and the halo-row forms on rows of 128 voxels.
static bool conv3d_tcgen05(int N, int T, int Y, int X, int Cin, int Cout, const void* x, int xs, int xo,
                           const void* w, const float* bias, void* y, int ys, int yo, int relu, int out_f32,
                           cudaStream_t st, ot_status* status) {
  const char* sel = std::getenv("DYNOT_CONV");
  if (sel && std::strcmp(sel, "mma") == 0) return false;
  const bool forced = sel && (std::strcmp(sel, "tcgen05") == 0 || std::strcmp(sel, "tap") == 0 ||
                              std::strcmp(sel, "halo") == 0);
  // with 16 output channels and rows shorter than 128 voxels (per-tap form) an MMA of N = 16 per tap does
  // too little per copy: the mma.sync kernel, which stages one input halo per 16-channel slice, is faster
  // there; rows of 128 voxels take the four-row block form, faster at every width (bench.py --conv)
  if (!forced && Cout < 32 && X % 128 != 0) return false;
  const int vec = out_f32 ? 4 : 8;
  const bool xok = X >= 128 ? X % 128 == 0 : (X >= 1 && 128 % X == 0);
  if (Cin % 16 || Cout % 16 || Cout > 256 || xs % 8 || xo % 8 || ys % vec || yo % vec || !xok ||
      ((uintptr_t)x & 15) || ((uintptr_t)w & 15) || ((uintptr_t)y & 15) || (long long)N * T >= 65536)
    return false;
  auto enc = nn_tensor_map_encoder();
  if (!enc) return false;
  tc::Geom g{N, T, Y, X, 0, 0, 0};
  g.BX = X >= 128 ? 128 : X;
  g.BY = 128 / g.BX;
  g.nxb = X / g.BX;
  const int nyb = (Y + g.BY - 1) / g.BY;
  // rows of 128 voxels along x take the row-block form (Cout <= 64: four output rows per CTA, six input rows
  // per (dt, chunk)) or the halo form (one input row per (dt, dy), three taps per stage)
  const bool tapf = sel && std::strcmp(sel, "tap") == 0, halof = sel && std::strcmp(sel, "halo") == 0;
  const bool rows = g.BX == 128 && Cout <= 64 && !tapf && !halof;
  const bool halo = g.BX == 128 && !tapf && !rows;
  if (rows) {
    CUtensorMap tmR, tmW;
    const cuuint64_t dim[5] = {(cuuint64_t)xs, (cuuint64_t)X, (cuuint64_t)Y, (cuuint64_t)T, (cuuint64_t)N};
    const cuuint64_t str[4] = {2ull * xs, 2ull * xs * X, 2ull * xs * X * Y, 2ull * xs * X * Y * T};
    const bool one_tile = sel && std::strcmp(sel, "rows") == 0, unstacked = sel && std::strcmp(sel, "persist") == 0;
    // Cout 16 and 32: stacked y taps (N = 3 Cout), persistent, 8 and 4 rows per tile (DYNOT_CONV=persist keeps the
    // persistent form with one MMA per tap, DYNOT_CONV=rows one tile per CTA)
    const bool stacked = (Cout == 16 || Cout == 32) && !one_tile && !unstacked;
    const bool persist = Cout <= 16 && !one_tile && !stacked;
    const int rb = stacked ? (Cout == 16 ? 8 : 4) : persist ? 8 : (Cout <= 32 ? 8 : tc::kRB);
    const cuuint32_t box[5] = {8, tc::kHaloRows, (cuuint32_t)(rb + 2), 1, 1};
    const cuuint32_t one[5] = {1, 1, 1, 1, 1};
    const cuuint64_t wdim[3] = {(cuuint64_t)Cin, 27, (cuuint64_t)Cout};
    const cuuint64_t wstr[2] = {2ull * Cin, 2ull * 27 * Cin};
    const cuuint32_t wbox[3] = {16, 1, (cuuint32_t)Cout};
    if (enc(&tmR, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(x), dim, str, box, one,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
        enc(&tmW, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(w), wdim, wstr, wbox, one,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
    if (stacked) {
      const size_t smem = rb == 8 ? tc::rows_s_smem_bytes<8>(Cout) : tc::rows_s_smem_bytes<4>(Cout);
      auto kern = rb == 8 ? tc::k_conv3d_tc_rows_s<8> : tc::k_conv3d_tc_rows_s<4>;
      int dev = 0, nsm = 0;
      cudaError_t e = cudaGetDevice(&dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) {
        const long long ntiles = (long long)g.nxb * ((Y + rb - 1) / rb) * N * T;
        if (ntiles >= (1LL << 31)) return false;
        const int grid = (int)std::min<long long>(ntiles, nsm);   // one CTA per SM (all 512 tensor-memory columns)
        kern<<<grid, 192, smem, st>>>(g, Cin, Cout, xo, (int)ntiles, bias, y, ys, yo, relu, out_f32, tmR, tmW);
        e = cudaGetLastError();
      }
      *status = e == cudaSuccess ? OT_OK : seterr(OT_ECUDA, "conv3d (tcgen05 stacked rows): %s", cudaGetErrorString(e));
      return true;
    }
    if (persist) {
      const size_t smem = rb == 8 ? tc::rows_p_smem_bytes<8>(Cout) : tc::rows_p_smem_bytes<4>(Cout);
      auto kern = rb == 8 ? tc::k_conv3d_tc_rows_p<8> : tc::k_conv3d_tc_rows_p<4>;
      int dev = 0, nsm = 0;
      cudaError_t e = cudaGetDevice(&dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) {
        const long long ntiles = (long long)g.nxb * ((Y + rb - 1) / rb) * N * T;
        if (ntiles >= (1LL << 31)) return false;
        const int grid = (int)std::min<long long>(ntiles, 2LL * nsm);   // two CTAs per SM (tensor memory, shared memory)
        kern<<<grid, 192, smem, st>>>(g, Cin, Cout, xo, (int)ntiles, bias, y, ys, yo, relu, out_f32, tmR, tmW);
        e = cudaGetLastError();
      }
      *status = e == cudaSuccess ? OT_OK : seterr(OT_ECUDA, "conv3d (tcgen05 persistent rows): %s", cudaGetErrorString(e));
      return true;
    }
    const size_t smem = rb == 8 ? tc::rows_smem_bytes<8>(Cout) : tc::rows_smem_bytes<tc::kRB>(Cout);
    auto kern = rb == 8 ? tc::k_conv3d_tc_rows<8> : tc::k_conv3d_tc_rows<tc::kRB>;
    cudaError_t e = cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
      const int nrb = (Y + rb - 1) / rb;
      kern<<<dim3((unsigned)(g.nxb * nrb), (unsigned)(N * T)), 128, smem, st>>>(g, Cin, Cout, xo, bias, y, ys, yo,
                                                                               relu, out_f32, tmR, tmW);
      e = cudaGetLastError();
    }
    *status = e == cudaSuccess ? OT_OK : seterr(OT_ECUDA, "conv3d (tcgen05 rows): %s", cudaGetErrorString(e));
    return true;
  }
  CUtensorMap tmX, tmW;
  {
    const cuuint64_t dim[5] = {(cuuint64_t)xs, (cuuint64_t)X, (cuuint64_t)Y, (cuuint64_t)T, (cuuint64_t)N};
    const cuuint64_t str[4] = {2ull * xs, 2ull * xs * X, 2ull * xs * X * Y, 2ull * xs * X * Y * T};
    const cuuint32_t box[5] = {halo ? 8u : 16u, halo ? tc::kHaloRows : (cuuint32_t)g.BX, (cuuint32_t)g.BY, 1, 1};
    const cuuint32_t one[5] = {1, 1, 1, 1, 1};
    if (enc(&tmX, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(x), dim, str, box, one,
            CU_TENSOR_MAP_INTERLEAVE_NONE, halo ? CU_TENSOR_MAP_SWIZZLE_NONE : CU_TENSOR_MAP_SWIZZLE_32B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  {
    const cuuint64_t dim[3] = {(cuuint64_t)Cin, 27, (cuuint64_t)Cout};
    const cuuint64_t str[2] = {2ull * Cin, 2ull * 27 * Cin};
    const cuuint32_t box[3] = {16, 1, (cuuint32_t)Cout};
    const cuuint32_t one[3] = {1, 1, 1};
    if (enc(&tmW, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(w), dim, str, box, one,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  const size_t smem = tc::smem_bytes(Cout, halo);
  auto kern = halo ? tc::k_conv3d_tc<true> : tc::k_conv3d_tc<false>;
  cudaError_t e = cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) {
    kern<<<dim3((unsigned)(g.nxb * nyb), (unsigned)(N * T)), 128, smem, st>>>(g, Cin, Cout, xo, bias, y, ys, yo, relu,
                                                                              out_f32, tmX, tmW);
    e = cudaGetLastError();
  }
  *status = e == cudaSuccess ? OT_OK : seterr(OT_ECUDA, "conv3d (tcgen05): %s", cudaGetErrorString(e));
  return true;
}

ot_status ot_nn_conv3d(int N, int T, int Y, int X, int Cin, int Cout, const void* x, int xs, int xo, const void* w,
                       const float* bias, void* y, int ys, int yo, int relu, int out_f32, void* stream) {
  if (Cin % 16 || Cout % 8 || xs % 2 || xo % 2 || ys % 2 || yo % 2 || xo < 0 || yo < 0 || Cin + xo > xs ||
      Cout + yo > ys)
    return seterr(OT_EINVAL, "conv3d: channel counts/strides must be multiples of 16/8/2 and fit their tensors");
  const Vol v{N, T, Y, X};
  const long long M = (long long)N * T * Y * X;
  const dim3 blk(128);
  cudaStream_t st = (cudaStream_t)stream;
  ot_status tcs = OT_OK;
  if (conv3d_tcgen05(N, T, Y, X, Cin, Cout, x, xs, xo, w, bias, y, ys, yo, relu, out_f32, st, &tcs)) return tcs;
  if (xs % 8 == 0 && xo % 8 == 0 && ((uintptr_t)x & 15) == 0 && (long long)N * T < 65536) {
    // shared-memory tiled form (16-byte input pieces)
    const int nxb = (X + kCT_TX - 1) / kCT_TX, nyb = (Y + kCT_TY - 1) / kCT_TY;
    if (Cout % 32 == 0) {
      k_conv3d_tiled<4><<<dim3((unsigned)(nxb * nyb), (unsigned)(N * T), Cout / 32), blk, 0, st>>>(
          v, Cin, Cout, (const bf16*)x, xs, xo, (const bf16*)w, bias, y, ys, yo, relu, out_f32);
    } else {
      k_conv3d_tiled<2><<<dim3((unsigned)(nxb * nyb), (unsigned)(N * T), (Cout + 15) / 16), blk, 0, st>>>(
          v, Cin, Cout, (const bf16*)x, xs, xo, (const bf16*)w, bias, y, ys, yo, relu, out_f32);
    }
    NN_LAUNCH_CHECK();
    return OT_OK;
  }
  if (Cout % 32 == 0) {
    k_conv3d<4><<<dim3((unsigned)((M + 63) / 64), Cout / 32), blk, 0, st>>>(
        v, Cin, Cout, (const bf16*)x, xs, xo, (const bf16*)w, bias, y, ys, yo, relu, out_f32);
  } else {
    k_conv3d<2><<<dim3((unsigned)((M + 63) / 64), (Cout + 15) / 16), blk, 0, st>>>(
        v, Cin, Cout, (const bf16*)x, xs, xo, (const bf16*)w, bias, y, ys, yo, relu, out_f32);
  }
  NN_LAUNCH_CHECK();
  return OT_OK;
}

ot_status ot_nn_check(void* stream) {
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return seterr(OT_ECUDA, "nn: %s", cudaGetErrorString(e));
  int flag = 0;
  e = cudaMemcpyFromSymbol(&flag, tc::g_tc_err, sizeof(int));
  if (e != cudaSuccess) return seterr(OT_ECUDA, "nn: %s", cudaGetErrorString(e));
  if (flag) {
    const int zero = 0;
    cudaMemcpyToSymbol(tc::g_tc_err, &zero, sizeof(int));
    return seterr(OT_ETIMEOUT, "a bounded device wait of the tensor-core convolution ran out of its limit");
  }
  return OT_OK;
}

// The weight gradient on tcgen05 (rows of X = 16, 32, 64 or 128 voxels, Cin and Cout multiples of 16, Cout <= 64,
// Cin <= 128: four stages of 210 KB at most):
// per-CTA partial sums of 27 x Cout x Cin, reduced in a fixed order.  false: not this form (DYNOT_CONV=mma, or the
// shapes and alignments do not allow it); then *status is untouched.
static bool wgrad_tcgen05(int N, int T, int Y, int X, int Cin, int Cout, const void* x, int xs, int xo, const void* dy,
                          int dys, int dyo, float* dw, cudaStream_t st, ot_status* status) {
  const char* sel = std::getenv("DYNOT_CONV");
  if (sel && std::strcmp(sel, "mma") == 0) return false;
  // with 16 input or output channels the M = 64 padding or the N = 16 operand leaves the tensor cores idle, and
  // the mma.sync kernels are faster (bench.py --conv, U-Net shapes); DYNOT_CONV=tcgen05 takes this form anyway
  const bool forced = sel && std::strcmp(sel, "tcgen05") == 0;
  if (!forced && (Cin < 32 || Cout < 32)) return false;
  if ((X != 16 && X != 32 && X != 64 && X != 128) || Cin % 16 || Cout % 16 || Cout > 64 || Cin > 128 || xs % 8 ||
      xo % 8 || dys % 8 || dyo % 8 || ((uintptr_t)x & 15) || ((uintptr_t)dy & 15) || (long long)N * T * Y >= (1LL << 31))
    return false;
  const int R = 128 / X;   // rows of one stage
  auto enc = nn_tensor_map_encoder();
  if (!enc) return false;
  CUtensorMap tmX, tmD;
  const cuuint32_t one[5] = {1, 1, 1, 1, 1};
  {
    const cuuint64_t dim[5] = {(cuuint64_t)xs, (cuuint64_t)X, (cuuint64_t)Y, (cuuint64_t)T, (cuuint64_t)N};
    const cuuint64_t str[4] = {2ull * xs, 2ull * xs * X, 2ull * xs * X * Y, 2ull * xs * X * Y * T};
    const cuuint32_t box[5] = {8, (cuuint32_t)(X + 2), (cuuint32_t)R, 1, 1};
    if (enc(&tmX, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(x), dim, str, box, one,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  {
    const cuuint64_t dim[5] = {(cuuint64_t)dys, (cuuint64_t)X, (cuuint64_t)Y, (cuuint64_t)T, (cuuint64_t)N};
    const cuuint64_t str[4] = {2ull * dys, 2ull * dys * X, 2ull * dys * X * Y, 2ull * dys * X * Y * T};
    const cuuint32_t box[5] = {8, (cuuint32_t)X, (cuuint32_t)R, 1, 1};
    if (enc(&tmD, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(dy), dim, str, box, one,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = tc::wg_smem_bytes(Cin);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)tc::k_conv3d_tc_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
  if (e != cudaSuccess) {
    *status = seterr(OT_ECUDA, "conv3d_wgrad (tcgen05): %s", cudaGetErrorString(e));
    return true;
  }
  // CTAs per SM that shared and tensor memory allow, nine (dt, dy) pairs, chunks of voxel rows to fill the SMs
  const int per_sm = (2 * smem + 2048 <= 228 * 1024 && 3 * Cin <= 256) ? 2 : 1;
  const int rows = N * T * ((Y + R - 1) / R);
  int nchunks = std::max(1, std::min(rows, per_sm * nsm / 9));
  const int rpc = (rows + nchunks - 1) / nchunks;
  nchunks = (rows + rpc - 1) / rpc;   // every chunk holds at least one row
  tc::Geom g{N, T, Y, X, X, R, 1};
  float* part = nullptr;
  const size_t bytes = sizeof(float) * (size_t)nchunks * 27 * Cout * Cin;
  e = cudaMallocAsync((void**)&part, bytes, st);
  if (e == cudaSuccess) {
    tc::k_conv3d_tc_wgrad<<<dim3((unsigned)nchunks, 9), 128, smem, st>>>(g, Cin, Cout, xo, dyo, rows, rpc, part, tmX, tmD);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
      k_wgrad_reduce_tc<<<dim3(27, (unsigned)Cout), 128, 0, st>>>(Cin, Cout, nchunks, part, dw);
      e = cudaGetLastError();
    }
    const cudaError_t e2 = cudaFreeAsync(part, st);
    if (e == cudaSuccess) e = e2;
  }
  *status = e == cudaSuccess ? OT_OK : seterr(OT_ECUDA, "conv3d_wgrad (tcgen05): %s", cudaGetErrorString(e));
  return true;
}

ot_status ot_nn_conv3d_wgrad(int N, int T, int Y, int X, int Cin, int Cout, const void* x, int xs, int xo,
                             const void* dy, int dys, int dyo, float* dw, float* db, void* stream) {
  if (Cin % 16 || Cout % 16) return seterr(OT_EINVAL, "conv3d_wgrad: channel counts must be multiples of 16");
  if (xo < 0 || dyo < 0 || Cin + xo > xs || Cout + dyo > dys)
    return seterr(OT_EINVAL, "conv3d_wgrad: channel slices must fit their tensors");
  const Vol v{N, T, Y, X};
  const long long M = (long long)N * T * Y * X;
  cudaStream_t st = (cudaStream_t)stream;
  {
    ot_status s2 = OT_OK;
    if (wgrad_tcgen05(N, T, Y, X, Cin, Cout, x, xs, xo, dy, dys, dyo, dw, st, &s2)) {
      if (s2 != OT_OK) return s2;
      if (db) {
        k_bias_grad<<<dim3(64, Cout), 256, 0, st>>>(M, Cout, (const bf16*)dy, dys, dyo, db);
        NN_LAUNCH_CHECK();
      }
      return OT_OK;
    }
  }
  if (xs % 8 == 0 && xo % 8 == 0 && dys % 8 == 0 && dyo % 8 == 0 && ((uintptr_t)x & 15) == 0 &&
      ((uintptr_t)dy & 15) == 0) {
    // shared-memory tiled form: per-block partials, then a fixed-order reduction into dw
    const int nxb = (X + kCT_TX - 1) / kCT_TX, nyb = (Y + kCT_TY - 1) / kCT_TY;
    const long long ntiles = (long long)N * T * nyb * nxb;
    const int nslices = (Cin / 16) * (Cout / 16);
    const int nblk = (int)std::max<long long>(1, std::min<long long>(ntiles, std::max(1, 4 * 152 / nslices)));
    if (ntiles < (1LL << 31) && nslices < 65536) {
      float* part = nullptr;
      const size_t bytes = sizeof(float) * (size_t)nslices * nblk * 27 * 256;
      CUDA_OK(cudaMallocAsync((void**)&part, bytes, st));
      k_conv3d_wgrad_tiled<<<dim3(nblk, nslices), 128, 0, st>>>(v, Cin, Cout, (const bf16*)x, xs, xo,
                                                                 (const bf16*)dy, dys, dyo, part, (int)ntiles);
      const cudaError_t e1 = cudaGetLastError();
      if (e1 == cudaSuccess) k_wgrad_reduce<<<dim3(27, nslices), 256, 0, st>>>(Cin, nblk, part, dw);
      const cudaError_t e2 = cudaGetLastError();
      CUDA_OK(cudaFreeAsync(part, st));
      if (e1 != cudaSuccess || e2 != cudaSuccess)
        return seterr(OT_ECUDA, "%s", cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
      if (db) {
        k_bias_grad<<<dim3(64, Cout), 256, 0, st>>>(M, Cout, (const bf16*)dy, dys, dyo, db);
        NN_LAUNCH_CHECK();
      }
      return OT_OK;
    }
  }
  if (M * xs >= (1LL << 31)) return seterr(OT_EINVAL, "conv3d_wgrad: tensor too large for 32-bit offsets");
  const int chunk = 4096;
  k_conv3d_wgrad<<<dim3((unsigned)((M + chunk - 1) / chunk), 27, (Cout / 16) * (Cin / 16)), 128, 0, st>>>(
      v, Cin, Cout, (const bf16*)x, xs, xo, (const bf16*)dy, dys, dyo, dw, chunk);
  NN_LAUNCH_CHECK();
  if (db) {
    k_bias_grad<<<dim3(64, Cout), 256, 0, st>>>(M, Cout, (const bf16*)dy, dys, dyo, db);
    NN_LAUNCH_CHECK();
  }
  return OT_OK;
}

ot_status ot_nn_rotate_weights(int Cin, int Cout, const void* w, void* wr, void* stream) {
  k_rotate_weights<<<blocks_for((long long)Cin * 27 * Cout), 256, 0, (cudaStream_t)stream>>>(
      Cin, Cout, (const bf16*)w, (bf16*)wr);
  NN_LAUNCH_CHECK();
  return OT_OK;
}

ot_status ot_nn_relu_grad(long long M, int C, void* g, int gs, int go, const void* y, int ys, int yo, void* stream) {
  k_relu_grad<<<blocks_for(M * C), 256, 0, (cudaStream_t)stream>>>(M, C, (bf16*)g, gs, go, (const bf16*)y, ys, yo);
  NN_LAUNCH_CHECK();
  return OT_OK;
}

ot_status ot_nn_pool(int N, int T, int Yc, int Xc, int C, const void* x, int xs, int xo, void* y, int ys, int yo,
                     int backward, void* stream) {
  const Vol vo{N, T, Yc, Xc};
  k_pool<<<blocks_for(vo.count() * C), 256, 0, (cudaStream_t)stream>>>(vo, C, (const bf16*)x, xs, xo, (bf16*)y, ys,
                                                                          yo, backward);
  NN_LAUNCH_CHECK();
  return OT_OK;
}

ot_status ot_nn_upsample(int N, int T, int Yc, int Xc, int C, const void* x, int xs, int xo, void* y, int ys, int yo,
                         int backward, void* stream) {
  const Vol vc{N, T, Yc, Xc};
  k_upsample<<<blocks_for(vc.count() * C), 256, 0, (cudaStream_t)stream>>>(vc, C, (const bf16*)x, xs, xo, (bf16*)y,
                                                                              ys, yo, backward);
  NN_LAUNCH_CHECK();
  return OT_OK;
}

ot_status ot_nn_add_slice(long long M, int C, const void* x, int xs, int xo, void* y, int ys, int yo, void* stream) {
  k_add_slice<<<blocks_for(M * C), 256, 0, (cudaStream_t)stream>>>(M, C, (const bf16*)x, xs, xo, (bf16*)y, ys, yo);
  NN_LAUNCH_CHECK();
  return OT_OK;
}

ot_status ot_nn_mse(long long M, int Cv, const float* out, int os, const void* target, void* g, int gs, float* loss,
                    void* stream) {
  if (Cv < 1 || Cv > os || Cv > gs) return seterr(OT_EINVAL, "mse: need 1 <= Cv <= os, gs");
  k_mse<<<blocks_for(M * gs), 256, 0, (cudaStream_t)stream>>>(M, Cv, out, os, (const bf16*)target, (bf16*)g, gs,
                                                               1.f / (float)(M * Cv), loss);
  NN_LAUNCH_CHECK();
  return OT_OK;
}

ot_status ot_nn_adamw(long long n, float* p, const float* g, float* m, float* v, void* pb, float lr, float b1,
                      float b2, float eps, float wd, int step, void* stream) {
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  k_adamw<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(n, p, g, m, v, (bf16*)pb, lr, b1, b2, eps, wd, c1, c2);
  NN_LAUNCH_CHECK();
  return OT_OK;
}

ot_status ot_nn_to_bf16(long long n, const float* x, void* y, void* stream) {
  k_to_bf16<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(n, x, (bf16*)y);
  NN_LAUNCH_CHECK();
  return OT_OK;
}

ot_status ot_nn_make_input(int N, int P, int Y, int X, int Cp, const float* f0, const float* f1, const float* scale,
                           void* out, void* stream) {
  if (Cp < 10) return seterr(OT_EINVAL, "make_input needs at least 10 channels");
  k_make_input<<<blocks_for((long long)N * P * Y * X), 256, 0, (cudaStream_t)stream>>>(N, P, Y, X, Cp, f0, f1, scale,
                                                                                        (bf16*)out);
  NN_LAUNCH_CHECK();
  return OT_OK;
}

ot_status ot_nn_path_channels(int N, int Y, int X, int P, int to_channels, const float* scale, const float* f0,
                              const float* f1, float* packed, float* ch, int cs, void* stream) {
  if ((f0 == nullptr) != (f1 == nullptr)) return seterr(OT_EINVAL, "path_channels: give both f0 and f1 or neither");
  if (cs < 12) return seterr(OT_EINVAL, "path_channels: channel stride must be >= 12");
  k_path_channels<<<blocks_for((long long)N * P * Y * X * 12), 256, 0, (cudaStream_t)stream>>>(
      Y, X, P, to_channels, scale, f0, f1, packed, ch, cs, N);
  NN_LAUNCH_CHECK();
  return OT_OK;
}

ot_status ot_nn_dual_channels(int N, int Y, int X, int P, int to_channels, float* packed, float* ch, int cs, int co,
                              void* stream) {
  if (co < 0 || co + 12 > cs) return seterr(OT_EINVAL, "dual_channels: channels co..co+11 must fit the stride");
  k_dual_channels<<<blocks_for((long long)N * P * Y * X * 12), 256, 0, (cudaStream_t)stream>>>(
      Y, X, P, to_channels, packed, ch, cs, co, N);
  NN_LAUNCH_CHECK();
  return OT_OK;
}

}  // extern "C"
