// 3x3x3 convolution on the fifth-generation tensor cores (tcgen05), bf16 in, fp32 accumulate in TMEM.
//
// The implicit GEMM of k_conv3d (M = voxels, N = output channels, K = 27 taps x input channels) with a
// CTA tile of M = 128 voxels (BX x BY of one (n, t) slice, BX * BY = 128) and all N = Cout channels.
// The K loop runs over (tap, 16-channel chunk) pairs.  For each pair a bulk tensor copy brings
//   A: the 128 voxels shifted by the tap, 16 channels each (32-byte rows, 32-byte swizzle; the copy
//      reads zeros outside the volume, which is the convolution's zero padding), and
//   B: the tap's 16-channel slice of every output channel's weights (Cout rows of 32 bytes),
// into one of kTcStages shared-memory stages.  One thread issues the copies, one thread issues one
// tcgen05.mma (M = 128, N = Cout, K = 16) per stage and releases the stage with tcgen05.commit; the
// accumulator lives in tensor memory (Cout columns of 128 lanes).  After the last MMA the four warps
// read their 32 lanes with tcgen05.ld, add the bias, apply ReLU and store bf16 or fp32.
//
// Rows of 128 voxels along x (X a multiple of 128) take the halo form (HALO = true): a stage holds the
// input row of 130 voxels (x0 - 1 .. x0 + 128) of one (dt, dy) and one 16-channel chunk, stored without
// swizzle as two planes of 8 channels (16-byte rows), and the weights of the three taps dx = -1, 0, 1;
// the three MMAs read the row through descriptors that start 0, 1 and 2 rows in, so each input row is
// copied once per (dt, dy) instead of once per tap.
//
// Every mbarrier wait has a time limit; a wait that runs out sets g_tc_err, the kernel writes NaN
// instead of its results, frees its tensor memory and returns.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>

namespace dynot {
namespace tc {

constexpr int kStages = 4;
constexpr int kM = 128;
constexpr unsigned long long kWaitNs = 20000000ull;   // 20 ms

__device__ int g_tc_err = 0;

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}
__device__ __forceinline__ void bar_init(uint32_t b, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(b), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_expect_tx(uint32_t b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(b), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool bar_wait(uint32_t b, uint32_t parity) {
  unsigned long long start = 0;
#pragma unroll 1
  for (int i = 0;; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(b), "r"(parity)
        : "memory");
    if (done) return true;
    if (i == 0) start = now_ns();
    else if ((i & 63) == 0 && now_ns() - start > kWaitNs) return false;
  }
}
// The same for a wait that spans a whole K loop: it runs out only after kWaitNs without progress, i.e. without a
// change of *prog (a stage counter the MMA thread advances), so a long loop is not taken for a stuck one.
__device__ __forceinline__ bool bar_wait_progress(uint32_t b, uint32_t parity, const volatile uint32_t* prog) {
  unsigned long long start = 0;
  uint32_t seen = 0;
#pragma unroll 1
  for (int i = 0;; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(b), "r"(parity)
        : "memory");
    if (done) return true;
    if (i == 0) {
      start = now_ns();
      seen = *prog;
    } else if ((i & 63) == 0) {
      const uint32_t cur = *prog;
      if (cur != seen) {
        seen = cur;
        start = now_ns();
      } else if (now_ns() - start > kWaitNs) {
        return false;
      }
    }
  }
}
__device__ __forceinline__ void tma_5d(uint32_t dst, const CUtensorMap* m, int c0, int c1, int c2, int c3, int c4,
                                       uint32_t b) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
      "%6}], [%7];\n" ::"r"(dst),
      "l"((unsigned long long)m), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(b)
      : "memory");
}
__device__ __forceinline__ void tma_3d(uint32_t dst, const CUtensorMap* m, int c0, int c1, int c2, uint32_t b) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];\n" ::"r"(dst),
      "l"((unsigned long long)m), "r"(c0), "r"(c1), "r"(c2), "r"(b)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major operand in the 32-byte swizzled layout: rows of 32 bytes
// (16 bf16 of K), groups of 8 rows 256 bytes apart (stride byte offset), one swizzle atom across K (the
// leading byte offset is not used), descriptor version 1, layout type 6 (32-byte swizzle).
__device__ __forceinline__ uint64_t desc_k32(uint32_t addr) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(256u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)6 << 61;
  return d;
}
// The same for the layout without swizzle: 8-row core matrices of 16-byte rows (stride byte offset 128 between
// 8-row groups), the two 8-channel halves of K `lbo` bytes apart (leading byte offset), layout type 0.
__device__ __forceinline__ uint64_t desc_k_plain(uint32_t addr, uint32_t lbo) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)(128u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
// Instruction descriptor of kind::f16: fp32 accumulator, bf16 A and B, both K-major, N >> 3 and M >> 4.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__host__ __device__ constexpr uint32_t b_bytes(int cout) { return (uint32_t)((cout * 32 + 1023) & ~1023); }
constexpr uint32_t kHaloRows = 130, kPlane = 2176;   // 130 rows of 16 bytes, padded to 128-byte multiples
constexpr uint32_t kHaloA = 5120;                    // two planes, padded to 1024 bytes
__host__ __device__ constexpr uint32_t stage_bytes(int cout, bool halo) {
  return halo ? kHaloA + 3u * b_bytes(cout) : 4096u + b_bytes(cout);
}
__host__ __device__ constexpr int tmem_cols(int cout) { return cout <= 32 ? 32 : (cout <= 64 ? 64 : (cout <= 128 ? 128 : 256)); }
inline size_t smem_bytes(int cout, bool halo) { return (size_t)kStages * stage_bytes(cout, halo) + 128 + 1024; }

struct Geom {
  int N, T, Y, X;
  int BX, BY, nxb;   // tile of BX x BY voxels (BX * BY = 128); nxb tiles along x
};

template <bool HALO>
__global__ void __launch_bounds__(128) k_conv3d_tc(Geom v, int Cin, int Cout, int xo, const float* __restrict__ bias,
                                                   void* __restrict__ y, int ys, int yo, int relu, int out_f32,
                                                   const __grid_constant__ CUtensorMap tmX,
                                                   const __grid_constant__ CUtensorMap tmW) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int x0 = (blockIdx.x % v.nxb) * v.BX, y0 = (blockIdx.x / v.nxb) * v.BY;
  const int t = blockIdx.y % v.T, n = blockIdx.y / v.T;
  const uint32_t sb = stage_bytes(Cout, HALO), bb = b_bytes(Cout);
  const uint32_t base = saddr(sm);
  const uint32_t bars = base + kStages * sb;   // full[kStages], empty[kStages], done
  auto full = [&](int s) { return bars + 8u * (uint32_t)s; };
  auto empty = [&](int s) { return bars + 8u * (uint32_t)(kStages + s); };
  const uint32_t done = bars + 8u * (2 * kStages);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + kStages * sb + 8 * (2 * kStages + 1));
  const int ncols = tmem_cols(Cout);
  const int chunks = Cin / 16, nk = (HALO ? 9 : 27) * chunks;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      bar_init(full(s), 1);
      bar_init(empty(s), 1);
    }
    bar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(saddr(tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  bool ok = true;
  if (warp == 0 && lane == 0) {
    // producer: the shifted input tile and the weight slice of every (tap, chunk)
    for (int i = 0; i < nk; ++i) {
      const int s = i % kStages;
      if (i >= kStages && ok) ok = bar_wait(empty(s), ((i / kStages) & 1) ^ 1);
      if constexpr (HALO) {
        const int ty = i / chunks, cc = i - ty * chunks;   // ty = 3 (dt + 1) + (dy + 1)
        const int dt = ty / 3 - 1, dy = ty % 3 - 1;
        bar_expect_tx(full(s), 2u * 16u * kHaloRows + 3u * 32u * (uint32_t)Cout);
        for (int h = 0; h < 2; ++h)
          tma_5d(base + s * sb + h * kPlane, &tmX, xo + 16 * cc + 8 * h, x0 - 1, y0 + dy, t + dt, n, full(s));
        for (int q = 0; q < 3; ++q) tma_3d(base + s * sb + kHaloA + q * bb, &tmW, 16 * cc, 3 * ty + q, 0, full(s));
      } else {
        const int tap = i / chunks, cc = i - tap * chunks;
        const int dt = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
        bar_expect_tx(full(s), 4096u + 32u * (uint32_t)Cout);
        tma_5d(base + s * sb, &tmX, xo + 16 * cc, x0 + dx, y0 + dy, t + dt, n, full(s));
        tma_3d(base + s * sb + 4096u, &tmW, 16 * cc, tap, 0, full(s));
      }
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issue: D (tensor memory) += A (128 x 16) B^T (16 x Cout) per stage
    const uint32_t idesc = idesc_bf16(kM, Cout);
    for (int i = 0; i < nk; ++i) {
      const int s = i % kStages;
      if (ok) ok = bar_wait(full(s), (i / kStages) & 1);
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      for (int q = 0; q < (HALO ? 3 : 1); ++q) {
        // halo: the tap dx = q - 1 reads the row from its (q)-th voxel on
        const uint64_t ad = HALO ? desc_k_plain(base + s * sb + 16u * q, kPlane) : desc_k32(base + s * sb);
        const uint64_t bd = desc_k32(base + s * sb + (HALO ? kHaloA + q * bb : 4096u));
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(i > 0 || q > 0 ? 1 : 0)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(empty(s))
                   : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(done)
                 : "memory");
  }
  __syncwarp();
  // epilogue: warp w owns accumulator rows (tensor-memory lanes) 32 w .. 32 w + 31
  if (ok) ok = bar_wait(done, 0);
  __syncwarp();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const int m = 32 * warp + lane;
  const int xx = x0 + m % v.BX, yy = y0 + m / v.BX;
  const bool store = xx < v.X && yy < v.Y;
  const long long vox = (((long long)n * v.T + t) * v.Y + yy) * v.X + xx;
  const float nanv = __int_as_float(0x7fc00000);
  for (int c0 = 0; c0 < Cout; c0 += 16) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
    if (!store) continue;
    float u[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      u[j] = __uint_as_float(r[j]) + (bias ? bias[c0 + j] : 0.f);
      if (relu) u[j] = fmaxf(u[j], 0.f);
      if (!ok) u[j] = nanv;
    }
    const long long o = vox * ys + yo + c0;
    if (out_f32) {
      float4* yp = reinterpret_cast<float4*>((float*)y + o);
#pragma unroll
      for (int q = 0; q < 4; ++q) yp[q] = make_float4(u[4 * q], u[4 * q + 1], u[4 * q + 2], u[4 * q + 3]);
    } else {
      uint4* yp = reinterpret_cast<uint4*>((__nv_bfloat16*)y + o);
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        uint32_t p[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const __nv_bfloat16 lo = __float2bfloat16(u[8 * q + 2 * j]), hi = __float2bfloat16(u[8 * q + 2 * j + 1]);
          p[j] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
        }
        yp[q] = make_uint4(p[0], p[1], p[2], p[3]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncols) : "memory");
  }
  if (!ok) atomicExch(&g_tc_err, 1);
}

// Blocks of kRB = 4 output rows of 128 voxels (X a multiple of 128, Cout <= 64).  One stage holds the six input
// rows y0 - 1 .. y0 + 4 (130 voxels each, two unswizzled 8-channel planes) of one dt and 16-channel chunk, and
// the weights of its nine (dy, dx) taps.  Each stage issues 36 MMAs (4 output rows x 9 taps) into four
// accumulators of Cout columns: every input row is copied once per (dt, chunk) for four output rows and every
// weight slice once per four rows, which cuts the copies per MMA about threefold against the halo row form.
// RB output rows per CTA: 4 for up to 64 output channels, 8 for up to 32 (RB accumulators of at most 64 and 32
// columns fill 256 of the 512 tensor-memory columns, so two CTAs share an SM).
template <int RB>
struct RowsForm {
  static constexpr int in = RB + 2;                                                // input rows per stage
  static constexpr uint32_t plane = ((uint32_t)in * 130u * 16u + 127u) & ~127u;   // one 8-channel plane
  static constexpr uint32_t a_bytes = (2u * plane + 1023u) & ~1023u;
};
constexpr int kRowStages = 2;
template <int RB>
__host__ __device__ constexpr uint32_t rows_stage_bytes(int cout) { return RowsForm<RB>::a_bytes + 9u * b_bytes(cout); }
__host__ __device__ constexpr int rows_col_stride(int cout) { return cout <= 16 ? 16 : (cout <= 32 ? 32 : 64); }
template <int RB>
inline size_t rows_smem_bytes(int cout) { return (size_t)kRowStages * rows_stage_bytes<RB>(cout) + 128 + 1024; }
constexpr int kRB = 4;   // rows per CTA of the wider outputs (the host picks 8 up to 32 output channels)

template <int RB>
__global__ void __launch_bounds__(128) k_conv3d_tc_rows(Geom v, int Cin, int Cout, int xo, const float* __restrict__ bias,
                                                        void* __restrict__ y, int ys, int yo, int relu, int out_f32,
                                                        const __grid_constant__ CUtensorMap tmX,
                                                        const __grid_constant__ CUtensorMap tmW) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  using F = RowsForm<RB>;
  const int x0 = (blockIdx.x % v.nxb) * 128, y0 = (blockIdx.x / v.nxb) * RB;
  const int t = blockIdx.y % v.T, n = blockIdx.y / v.T;
  const uint32_t sb = rows_stage_bytes<RB>(Cout), bb = b_bytes(Cout);
  const uint32_t base = saddr(sm);
  const uint32_t bars = base + kRowStages * sb;   // full[kRowStages], empty[kRowStages], done
  auto full = [&](int s) { return bars + 8u * (uint32_t)s; };
  auto empty = [&](int s) { return bars + 8u * (uint32_t)(kRowStages + s); };
  const uint32_t done = bars + 8u * (2 * kRowStages);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + kRowStages * sb + 8 * (2 * kRowStages + 1));
  const int cs = rows_col_stride(Cout);
  const int ncols = tmem_cols(RB * cs);
  const int chunks = Cin / 16, nk = 3 * chunks;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kRowStages; ++s) {
      bar_init(full(s), 1);
      bar_init(empty(s), 1);
    }
    bar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(saddr(tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  bool ok = true;
  if (warp == 0 && lane == 0) {
    // producer: six input rows of one dt and chunk, and the weights of its nine taps
    for (int i = 0; i < nk; ++i) {
      const int s = i % kRowStages;
      if (i >= kRowStages && ok) ok = bar_wait(empty(s), ((i / kRowStages) & 1) ^ 1);
      const int dt = i / chunks - 1, cc = i % chunks;
      bar_expect_tx(full(s), 2u * F::in * kHaloRows * 16u + 9u * 32u * (uint32_t)Cout);
      for (int h = 0; h < 2; ++h)
        tma_5d(base + s * sb + h * F::plane, &tmX, xo + 16 * cc + 8 * h, x0 - 1, y0 - 1, t + dt, n, full(s));
      for (int q = 0; q < 9; ++q)
        tma_3d(base + s * sb + F::a_bytes + q * bb, &tmW, 16 * cc, 9 * (dt + 1) + q, 0, full(s));
    }
  } else if (warp == 1 && lane == 0) {
    const uint32_t idesc = idesc_bf16(kM, Cout);
    for (int i = 0; i < nk; ++i) {
      const int s = i % kRowStages;
      if (ok) ok = bar_wait(full(s), (i / kRowStages) & 1);
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      // descriptors of the stage's first input voxel and first weight slice; the start-address field counts
      // 16-byte units, so later rows, voxels and slices are added to it
      const uint64_t ad0 = desc_k_plain(base + s * sb, F::plane);
      const uint64_t bd0 = desc_k32(base + s * sb + F::a_bytes);
      for (int r = 0; r < RB; ++r)
        for (int q = 0; q < 9; ++q) {
          // output row r, tap (dy, dx) = (q / 3 - 1, q % 3 - 1): input row r + dy + 1 of the stage, from voxel dx + 1
          const int arow = r + q / 3, ax = q % 3;
          const uint64_t ad = ad0 + (uint64_t)(arow * (int)kHaloRows + ax);
          const uint64_t bd = bd0 + (uint64_t)(q * (bb >> 4));
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + (uint32_t)(r * cs)),
              "l"(ad), "l"(bd), "r"(idesc), "r"(i > 0 || q > 0 ? 1 : 0)
              : "memory");
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(empty(s))
                   : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(done)
                 : "memory");
  }
  __syncwarp();
  if (ok) ok = bar_wait(done, 0);
  __syncwarp();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const int xx = x0 + 32 * warp + lane;
  const float nanv = __int_as_float(0x7fc00000);
  for (int r = 0; r < RB; ++r) {
    const int yy = y0 + r;
    const bool store = xx < v.X && yy < v.Y;
    const long long vox = (((long long)n * v.T + t) * v.Y + yy) * v.X + xx;
    for (int c0 = 0; c0 < Cout; c0 += 16) {
      uint32_t rr[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
          "%15}, [%16];\n"
          : "=r"(rr[0]), "=r"(rr[1]), "=r"(rr[2]), "=r"(rr[3]), "=r"(rr[4]), "=r"(rr[5]), "=r"(rr[6]), "=r"(rr[7]),
            "=r"(rr[8]), "=r"(rr[9]), "=r"(rr[10]), "=r"(rr[11]), "=r"(rr[12]), "=r"(rr[13]), "=r"(rr[14]), "=r"(rr[15])
          : "r"(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(r * cs + c0)));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if (!store) continue;
      float u[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        u[j] = __uint_as_float(rr[j]) + (bias ? bias[c0 + j] : 0.f);
        if (relu) u[j] = fmaxf(u[j], 0.f);
        if (!ok) u[j] = nanv;
      }
      const long long o = vox * ys + yo + c0;
      if (out_f32) {
        float4* yp = reinterpret_cast<float4*>((float*)y + o);
#pragma unroll
        for (int q = 0; q < 4; ++q) yp[q] = make_float4(u[4 * q], u[4 * q + 1], u[4 * q + 2], u[4 * q + 3]);
      } else {
        uint4* yp = reinterpret_cast<uint4*>((__nv_bfloat16*)y + o);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          uint32_t pk[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const __nv_bfloat16 lo = __float2bfloat16(u[8 * q + 2 * j]), hi = __float2bfloat16(u[8 * q + 2 * j + 1]);
            pk[j] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
          }
          yp[q] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncols) : "memory");
  }
  if (!ok) atomicExch(&g_tc_err, 1);
}

// Persistent form of the row blocks for narrow outputs (the host takes it for Cout <= 16).  With 16 output
// channels a CTA of the row form above runs only 3 pipeline stages, so its tensor-memory allocation, pipeline
// fill and epilogue dominate.  Here 2 CTAs per SM stay resident and walk the tiles (RB output rows of 128 voxels) with a stride
// of the grid: warp 0 issues the bulk tensor copies and warp 1 the MMAs, both continuously across tiles through
// the two-stage ring, and warps 2-5 run the epilogue of a tile from one of two accumulators in tensor memory
// while the MMAs of the next tile fill the other.  Barriers: full / empty per stage (copies landed / MMAs done
// reading), and per accumulator acc_full (its last MMA done, by tcgen05.commit) and acc_empty (its four epilogue
// warps done reading).  Every wait has a time limit; a wait that runs out marks the thread's results as NaN,
// stops its waits and sets g_tc_err.
constexpr int kPStages = 2;
template <int RB>
inline size_t rows_p_smem_bytes(int cout) { return (size_t)kPStages * rows_stage_bytes<RB>(cout) + 128 + 1024; }

template <int RB>
__global__ void __launch_bounds__(192) k_conv3d_tc_rows_p(Geom v, int Cin, int Cout, int xo, int ntiles,
                                                          const float* __restrict__ bias, void* __restrict__ y,
                                                          int ys, int yo, int relu, int out_f32,
                                                          const __grid_constant__ CUtensorMap tmX,
                                                          const __grid_constant__ CUtensorMap tmW) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  using F = RowsForm<RB>;
  const uint32_t sb = rows_stage_bytes<RB>(Cout), bb = b_bytes(Cout);
  const uint32_t base = saddr(sm);
  const uint32_t bars = base + kPStages * sb;
  auto full = [&](int s) { return bars + 8u * (uint32_t)s; };
  auto empty = [&](int s) { return bars + 8u * (uint32_t)(kPStages + s); };
  auto acc_full = [&](int a) { return bars + 8u * (uint32_t)(2 * kPStages + a); };
  auto acc_empty = [&](int a) { return bars + 8u * (uint32_t)(2 * kPStages + 2 + a); };
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + kPStages * sb + 8 * (2 * kPStages + 4));
  const int cs = rows_col_stride(Cout);
  const uint32_t acols = (uint32_t)(RB * cs);   // columns of one accumulator
  const int ncols = tmem_cols(2 * RB * cs);
  const int chunks = Cin / 16, nk = 3 * chunks;
  const int nyb = (v.Y + RB - 1) / RB;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kPStages; ++s) {
      bar_init(full(s), 1);
      bar_init(empty(s), 1);
    }
    for (int a = 0; a < 2; ++a) {
      bar_init(acc_full(a), 1);
      bar_init(acc_empty(a), 4);
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(saddr(tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  bool ok = true;
  auto tile_pos = [&](int tile, int& x0, int& y0, int& t, int& n) {
    x0 = (tile % v.nxb) * 128;
    const int rest = tile / v.nxb;
    y0 = (rest % nyb) * RB;
    const int nt = rest / nyb;
    t = nt % v.T;
    n = nt / v.T;
  };
  if (warp == 0) {
    if (lane == 0) {
      int g = 0;   // k-steps issued so far (the ring position)
      for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        int x0, y0, t, n;
        tile_pos(tile, x0, y0, t, n);
        for (int i = 0; i < nk; ++i, ++g) {
          const int s = g % kPStages;
          if (g >= kPStages && ok) ok = bar_wait(empty(s), ((g / kPStages) & 1) ^ 1);
          const int dt = i / chunks - 1, cc = i % chunks;
          bar_expect_tx(full(s), 2u * F::in * kHaloRows * 16u + 9u * 32u * (uint32_t)Cout);
          for (int h = 0; h < 2; ++h)
            tma_5d(base + s * sb + h * F::plane, &tmX, xo + 16 * cc + 8 * h, x0 - 1, y0 - 1, t + dt, n, full(s));
          for (int q = 0; q < 9; ++q)
            tma_3d(base + s * sb + F::a_bytes + q * bb, &tmW, 16 * cc, 9 * (dt + 1) + q, 0, full(s));
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(kM, Cout);
      int g = 0, j = 0;
      for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++j) {
        const int ab = j & 1;
        if (j >= 2 && ok) ok = bar_wait(acc_empty(ab), ((j >> 1) & 1) ^ 1);
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t acc = tmem + (uint32_t)ab * acols;
        for (int i = 0; i < nk; ++i, ++g) {
          const int s = g % kPStages;
          if (ok) ok = bar_wait(full(s), (g / kPStages) & 1);
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
          const uint64_t ad0 = desc_k_plain(base + s * sb, F::plane);
          const uint64_t bd0 = desc_k32(base + s * sb + F::a_bytes);
          for (int r = 0; r < RB; ++r)
            for (int q = 0; q < 9; ++q) {
              const int arow = r + q / 3, ax = q % 3;
              const uint64_t ad = ad0 + (uint64_t)(arow * (int)kHaloRows + ax);
              const uint64_t bd = bd0 + (uint64_t)(q * (bb >> 4));
              asm volatile(
                  "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                  " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc + (uint32_t)(r * cs)),
                  "l"(ad), "l"(bd), "r"(idesc), "r"(i > 0 || q > 0 ? 1 : 0)
                  : "memory");
            }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(empty(s))
                       : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(acc_full(ab))
                     : "memory");
      }
    }
  } else {
    // epilogue: warp w reads the lanes 32 (w % 4) .. 32 (w % 4) + 31 of the accumulator
    const int quad = warp & 3;
    const float nanv = __int_as_float(0x7fc00000);
    int j = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++j) {
      const int ab = j & 1;
      int x0, y0, t, n;
      tile_pos(tile, x0, y0, t, n);
      if (ok) ok = bar_wait(acc_full(ab), (j >> 1) & 1);
      __syncwarp();
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const int xx = x0 + 32 * quad + lane;
      for (int r = 0; r < RB; ++r) {
        const int yy = y0 + r;
        const bool store = xx < v.X && yy < v.Y;
        const long long vox = (((long long)n * v.T + t) * v.Y + yy) * v.X + xx;
        for (int c0 = 0; c0 < Cout; c0 += 16) {
          uint32_t rr[16];
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
              "%14, %15}, [%16];\n"
              : "=r"(rr[0]), "=r"(rr[1]), "=r"(rr[2]), "=r"(rr[3]), "=r"(rr[4]), "=r"(rr[5]), "=r"(rr[6]), "=r"(rr[7]),
                "=r"(rr[8]), "=r"(rr[9]), "=r"(rr[10]), "=r"(rr[11]), "=r"(rr[12]), "=r"(rr[13]), "=r"(rr[14]),
                "=r"(rr[15])
              : "r"(tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)ab * acols + (uint32_t)(r * cs + c0)));
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
          if (!store) continue;
          float u[16];
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            u[q] = __uint_as_float(rr[q]) + (bias ? bias[c0 + q] : 0.f);
            if (relu) u[q] = fmaxf(u[q], 0.f);
            if (!ok) u[q] = nanv;
          }
          const long long o = vox * ys + yo + c0;
          if (out_f32) {
            float4* yp = reinterpret_cast<float4*>((float*)y + o);
#pragma unroll
            for (int q = 0; q < 4; ++q) yp[q] = make_float4(u[4 * q], u[4 * q + 1], u[4 * q + 2], u[4 * q + 3]);
          } else {
            uint4* yp = reinterpret_cast<uint4*>((__nv_bfloat16*)y + o);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              uint32_t pk[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const __nv_bfloat16 lo = __float2bfloat16(u[8 * q + 2 * e]), hi = __float2bfloat16(u[8 * q + 2 * e + 1]);
                pk[e] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
              }
              yp[q] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            }
          }
        }
      }
      // this warp's lanes of accumulator ab are read: hand it back to the MMA warp
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(acc_empty(ab)) : "memory");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncols) : "memory");
  }
  if (!ok) atomicExch(&g_tc_err, 1);
}

// Stacked y taps (persistent, narrow outputs: Cout = 16 with RB = 8 rows per tile, Cout = 32 with RB = 4).
// An input row a of the stage feeds the output rows a, a - 1, a - 2 through its taps dy = -1, 0, 1, so one MMA per
// (input row, dx) with N = 3 Cout -- the weights of the three dy taps of that dx side by side -- does the work of
// three MMAs of N = Cout and reads the 128 x 16 input block once instead of three times.  The accumulator holds
// the rows r = -2 .. RB + 1 at columns (RB + 1 - r) Cout, decreasing with r, so that the three Cout-column
// segments of the MMA of input row a land on rows a, a - 1, a - 2 (rows outside 0 .. RB - 1 collect terms that
// are never read).  In the first stage of a tile the dx = 0 taps go out as three MMAs of N = Cout each, in the
// order that makes each row's first write the one that clears it (row a by its own input row, k = 0).  Weight
// slices are stored dx-major (slot 3 (dx + 1) + dy + 1), Cout rows of 32 bytes each, so the three dy slices of a
// dx are one operand of 3 Cout rows.  One CTA per SM (two accumulators of (RB + 4) Cout columns fill the 512
// tensor-memory columns), four pipeline stages; the warp roles and barriers are those of k_conv3d_tc_rows_p.
constexpr int kSStages = 4;
template <int RB>
__host__ __device__ constexpr uint32_t rows_s_stage_bytes(int cout) {
  return (RowsForm<RB>::a_bytes + 9u * 32u * (uint32_t)cout + 1023u) & ~1023u;
}
template <int RB>
inline size_t rows_s_smem_bytes(int cout) { return (size_t)kSStages * rows_s_stage_bytes<RB>(cout) + 128 + 1024; }

template <int RB>
__global__ void __launch_bounds__(192) k_conv3d_tc_rows_s(Geom v, int Cin, int Cout, int xo, int ntiles,
                                                          const float* __restrict__ bias, void* __restrict__ y,
                                                          int ys, int yo, int relu, int out_f32,
                                                          const __grid_constant__ CUtensorMap tmX,
                                                          const __grid_constant__ CUtensorMap tmW) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  using F = RowsForm<RB>;
  const uint32_t sb = rows_s_stage_bytes<RB>(Cout), bb = 32u * (uint32_t)Cout;
  const uint32_t base = saddr(sm);
  const uint32_t bars = base + kSStages * sb;
  auto full = [&](int s) { return bars + 8u * (uint32_t)s; };
  auto empty = [&](int s) { return bars + 8u * (uint32_t)(kSStages + s); };
  auto acc_full = [&](int a) { return bars + 8u * (uint32_t)(2 * kSStages + a); };
  auto acc_empty = [&](int a) { return bars + 8u * (uint32_t)(2 * kSStages + 2 + a); };
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + kSStages * sb + 8 * (2 * kSStages + 4));
  const uint32_t acols = (uint32_t)((RB + 4) * Cout);   // columns of one accumulator
  const int ncols = 512;
  const int chunks = Cin / 16, nk = 3 * chunks;
  const int nyb = (v.Y + RB - 1) / RB;
  auto col = [&](int r) { return (uint32_t)((RB + 1 - r) * Cout); };
  if (threadIdx.x == 0) {
    for (int s = 0; s < kSStages; ++s) {
      bar_init(full(s), 1);
      bar_init(empty(s), 1);
    }
    for (int a = 0; a < 2; ++a) {
      bar_init(acc_full(a), 1);
      bar_init(acc_empty(a), 4);
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(saddr(tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  bool ok = true;
  auto tile_pos = [&](int tile, int& x0, int& y0, int& t, int& n) {
    x0 = (tile % v.nxb) * 128;
    const int rest = tile / v.nxb;
    y0 = (rest % nyb) * RB;
    const int nt = rest / nyb;
    t = nt % v.T;
    n = nt / v.T;
  };
  if (warp == 0) {
    if (lane == 0) {
      int g = 0;
      for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        int x0, y0, t, n;
        tile_pos(tile, x0, y0, t, n);
        for (int i = 0; i < nk; ++i, ++g) {
          const int s = g % kSStages;
          if (g >= kSStages && ok) ok = bar_wait(empty(s), ((g / kSStages) & 1) ^ 1);
          const int dt = i / chunks - 1, cc = i % chunks;
          bar_expect_tx(full(s), 2u * F::in * kHaloRows * 16u + 9u * 32u * (uint32_t)Cout);
          for (int h = 0; h < 2; ++h)
            tma_5d(base + s * sb + h * F::plane, &tmX, xo + 16 * cc + 8 * h, x0 - 1, y0 - 1, t + dt, n, full(s));
          // weight slot 3 (dx + 1) + (dy + 1) takes tap 9 (dt + 1) + 3 (dy + 1) + (dx + 1)
          for (int dxi = 0; dxi < 3; ++dxi)
            for (int k = 0; k < 3; ++k)
              tma_3d(base + s * sb + F::a_bytes + (uint32_t)(3 * dxi + k) * bb, &tmW, 16 * cc, 9 * (dt + 1) + 3 * k + dxi,
                     0, full(s));
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t id3 = idesc_bf16(kM, 3 * Cout), id1 = idesc_bf16(kM, Cout);
      int g = 0, j = 0;
      for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++j) {
        const int ab = j & 1;
        if (j >= 2 && ok) ok = bar_wait(acc_empty(ab), ((j >> 1) & 1) ^ 1);
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t acc = tmem + (uint32_t)ab * acols;
        for (int i = 0; i < nk; ++i, ++g) {
          const int s = g % kSStages;
          if (ok) ok = bar_wait(full(s), (g / kSStages) & 1);
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
          const uint64_t ad0 = desc_k_plain(base + s * sb, F::plane);
          const uint64_t bd0 = desc_k32(base + s * sb + F::a_bytes);
          for (int dxi = 0; dxi < 3; ++dxi)
            for (int a = 0; a < RB + 2; ++a) {
              const uint64_t ad = ad0 + (uint64_t)(a * (int)kHaloRows + dxi);
              if (i == 0 && dxi == 0) {
                // first writes of the tile: one MMA per dy tap; k = 0 (row a) clears its row
                for (int k = 0; k < 3; ++k) {
                  const uint64_t bd = bd0 + (uint64_t)(k * (bb >> 4));
                  asm volatile(
                      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc + col(a - k)),
                      "l"(ad), "l"(bd), "r"(id1), "r"(k > 0 ? 1 : 0)
                      : "memory");
                }
              } else {
                const uint64_t bd = bd0 + (uint64_t)(3 * dxi * (bb >> 4));
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc + col(a)),
                    "l"(ad), "l"(bd), "r"(id3), "r"(1)
                    : "memory");
              }
            }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(empty(s))
                       : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(acc_full(ab))
                     : "memory");
      }
    }
  } else {
    const int quad = warp & 3;
    const float nanv = __int_as_float(0x7fc00000);
    int j = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++j) {
      const int ab = j & 1;
      int x0, y0, t, n;
      tile_pos(tile, x0, y0, t, n);
      if (ok) ok = bar_wait(acc_full(ab), (j >> 1) & 1);
      __syncwarp();
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const int xx = x0 + 32 * quad + lane;
      for (int r = 0; r < RB; ++r) {
        const int yy = y0 + r;
        const bool store = xx < v.X && yy < v.Y;
        const long long vox = (((long long)n * v.T + t) * v.Y + yy) * v.X + xx;
        for (int c0 = 0; c0 < Cout; c0 += 16) {
          uint32_t rr[16];
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
              "%14, %15}, [%16];\n"
              : "=r"(rr[0]), "=r"(rr[1]), "=r"(rr[2]), "=r"(rr[3]), "=r"(rr[4]), "=r"(rr[5]), "=r"(rr[6]), "=r"(rr[7]),
                "=r"(rr[8]), "=r"(rr[9]), "=r"(rr[10]), "=r"(rr[11]), "=r"(rr[12]), "=r"(rr[13]), "=r"(rr[14]),
                "=r"(rr[15])
              : "r"(tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)ab * acols + col(r) + (uint32_t)c0));
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
          if (!store) continue;
          float u[16];
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            u[q] = __uint_as_float(rr[q]) + (bias ? bias[c0 + q] : 0.f);
            if (relu) u[q] = fmaxf(u[q], 0.f);
            if (!ok) u[q] = nanv;
          }
          const long long o = vox * ys + yo + c0;
          if (out_f32) {
            float4* yp = reinterpret_cast<float4*>((float*)y + o);
#pragma unroll
            for (int q = 0; q < 4; ++q) yp[q] = make_float4(u[4 * q], u[4 * q + 1], u[4 * q + 2], u[4 * q + 3]);
          } else {
            uint4* yp = reinterpret_cast<uint4*>((__nv_bfloat16*)y + o);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              uint32_t pk[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const __nv_bfloat16 lo = __float2bfloat16(u[8 * q + 2 * e]), hi = __float2bfloat16(u[8 * q + 2 * e + 1]);
                pk[e] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
              }
              yp[q] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(acc_empty(ab)) : "memory");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncols) : "memory");
  }
  if (!ok) atomicExch(&g_tc_err, 1);
}

// Weight gradient on the tensor cores: dw[co][tap][ci] = sum over voxels v of dy[v][co] x[v + tap][ci], for rows
// of X voxels along x (X = 16, 32, 64 or 128).  Per tap this is a GEMM with M = output channels (padded to 64),
// N = input channels and K = voxels, both operands MN-major (channels are the contiguous dimension of the
// activations).  A pipeline stage holds R = 128 / X consecutive rows (y) of one (n, t): dy as 8-channel planes of
// 128 voxels of 16 bytes (the planes past Cout stay zero), x as 8-channel planes of the R input rows of one
// (dt, dy) shift with their x halo (X + 2 voxels each), which the three dx taps read through descriptors one voxel
// apart.  A CTA takes one (dt, dy) pair and a chunk of row groups; per stage it issues 3 x 8 MMAs (M = 64,
// N = Cin, K = 16 voxels of one row) into three accumulators (dx = -1, 0, 1) of Cin columns, and at the end
// writes its 3 x Cout x Cin sums to `part`, which a second kernel adds in a fixed order.  The descriptors of MN-major operands without
// swizzle carry the K-group stride (8 voxels, 128 bytes) in bits 16-29 and the 8-channel plane stride in bits
// 32-45; an M = 64 accumulator keeps row r in lane 32 (r / 16) + r % 16.  Waits are time-limited (g_tc_err); the
// wait for the end of the whole K loop runs out only after the MMA thread has made no progress for the limit.
constexpr int kWStages = 4;
constexpr uint32_t kWPlaneA = 128 * 16, kWPlaneB = 2304;   // 128 voxels; R (X + 2) <= 144 voxels, of 16 bytes
__host__ __device__ constexpr uint32_t wg_stage_bytes(int cin) {
  return (8u * kWPlaneA + (uint32_t)(cin / 8) * kWPlaneB + 1023u) & ~1023u;
}
inline size_t wg_smem_bytes(int cin) { return (size_t)kWStages * wg_stage_bytes(cin) + 128 + 1024; }
__device__ __forceinline__ uint64_t desc_mn_plain(uint32_t addr, uint32_t plane) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)(128u >> 4) << 16;                       // K groups of 8 voxels
  d |= (uint64_t)((plane >> 4) & 0x3FFFu) << 32;          // 8-channel planes
  d |= (uint64_t)1 << 46;
  return d;
}

// rows: the N * T * ceil(Y / R) row groups (n, t, y0), chunked over blockIdx.x; blockIdx.y = 3 (dt + 1) + (dy + 1)
__global__ void __launch_bounds__(128) k_conv3d_tc_wgrad(Geom v, int Cin, int Cout, int xo, int dyo, int rows,
                                                         int rows_per_chunk, float* __restrict__ part,
                                                         const __grid_constant__ CUtensorMap tmX,
                                                         const __grid_constant__ CUtensorMap tmD) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t sb = wg_stage_bytes(Cin);
  const uint32_t base = saddr(sm);
  const uint32_t bars = base + kWStages * sb;
  auto full = [&](int s) { return bars + 8u * (uint32_t)s; };
  auto empty = [&](int s) { return bars + 8u * (uint32_t)(kWStages + s); };
  const uint32_t done = bars + 8u * (2 * kWStages);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + kWStages * sb + 8 * (2 * kWStages + 1));
  volatile uint32_t* prog = reinterpret_cast<volatile uint32_t*>(sm + kWStages * sb + 8 * (2 * kWStages + 2));
  const int ncols = tmem_cols(3 * Cin) >= 3 * Cin ? tmem_cols(3 * Cin) : 512;
  const int dt = (int)blockIdx.y / 3 - 1, dy = (int)blockIdx.y % 3 - 1;
  const int r0 = blockIdx.x * rows_per_chunk, r1 = min(rows, r0 + rows_per_chunk);
  const int nrow = max(0, r1 - r0);
  // the A planes past Cout are never copied: zero them in every stage
  for (uint32_t i = threadIdx.x * 16u; i < (uint32_t)kWStages * sb; i += 128u * 16u) {
    if ((i % sb) < 8u * kWPlaneA) *reinterpret_cast<uint4*>(sm + i) = make_uint4(0u, 0u, 0u, 0u);
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  if (threadIdx.x == 0) {
    for (int s = 0; s < kWStages; ++s) {
      bar_init(full(s), 1);
      bar_init(empty(s), 1);
    }
    bar_init(done, 1);
    *prog = 0u;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(saddr(tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  bool ok = true;
  const int pa = Cout / 8, pb = Cin / 8;
  const int X = v.X, R = 128 / X, nyg = (v.Y + R - 1) / R;
  if (warp == 0 && lane == 0) {
    for (int i = 0; i < nrow; ++i) {
      const int s = i % kWStages;
      if (i >= kWStages && ok) ok = bar_wait(empty(s), ((i / kWStages) & 1) ^ 1);
      const int row = r0 + i;
      const int y = (row % nyg) * R, t = (row / nyg) % v.T, n = row / (nyg * v.T);
      bar_expect_tx(full(s), (uint32_t)pa * kWPlaneA + (uint32_t)pb * (uint32_t)(R * (X + 2)) * 16u);
      for (int h = 0; h < pa; ++h) tma_5d(base + s * sb + h * kWPlaneA, &tmD, dyo + 8 * h, 0, y, t, n, full(s));
      for (int h = 0; h < pb; ++h)
        tma_5d(base + s * sb + 8 * kWPlaneA + h * kWPlaneB, &tmX, xo + 8 * h, -1, y + dy, t + dt, n, full(s));
    }
  } else if (warp == 1 && lane == 0) {
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((uint32_t)(Cin >> 3) << 17) |
                           ((uint32_t)(64 >> 4) << 24);
    for (int i = 0; i < nrow; ++i) {
      const int s = i % kWStages;
      if (ok) ok = bar_wait(full(s), (i / kWStages) & 1);
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint64_t ad0 = desc_mn_plain(base + s * sb, kWPlaneA);
      const uint64_t bd0 = desc_mn_plain(base + s * sb + 8 * kWPlaneA, kWPlaneB);
      for (int dxi = 0; dxi < 3; ++dxi)
        for (int k0 = 0; k0 < 8; ++k0) {
          // voxels 16 k0 .. 16 k0 + 15 of the stage: row r = 16 k0 / X, from voxel xk of it
          const int r = (16 * k0) / X, xk = 16 * k0 - r * X;
          const uint64_t ad = ad0 + (uint64_t)(16 * k0);                          // dy rows are contiguous
          const uint64_t bd = bd0 + (uint64_t)(r * (X + 2) + xk + dxi);           // input row r, voxel x + dx + 1
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + (uint32_t)(dxi * Cin)),
              "l"(ad), "l"(bd), "r"(idesc), "r"(i > 0 || k0 > 0 ? 1 : 0)
              : "memory");
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(empty(s))
                   : "memory");
      *prog = (uint32_t)(i + 1);   // progress for the threads that wait for the whole loop
    }
    if (nrow > 0)
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(done)
                   : "memory");
  }
  __syncwarp();
  if (nrow > 0 && ok) ok = bar_wait_progress(done, 0, prog);
  __syncwarp();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  // output channel co = 16 warp + lane sits in lane 32 warp + lane (lanes 0-15 of each quarter)
  const int co = 16 * warp + lane;
  const float nanv = __int_as_float(0x7fc00000);
  for (int dxi = 0; dxi < 3; ++dxi)
    for (int c0 = 0; c0 < Cin; c0 += 16) {
      uint32_t rr[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
          "%15}, [%16];\n"
          : "=r"(rr[0]), "=r"(rr[1]), "=r"(rr[2]), "=r"(rr[3]), "=r"(rr[4]), "=r"(rr[5]), "=r"(rr[6]), "=r"(rr[7]),
            "=r"(rr[8]), "=r"(rr[9]), "=r"(rr[10]), "=r"(rr[11]), "=r"(rr[12]), "=r"(rr[13]), "=r"(rr[14]), "=r"(rr[15])
          : "r"(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(dxi * Cin + c0)));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if (lane >= 16 || co >= Cout) continue;
      const int tap = 9 * (dt + 1) + 3 * (dy + 1) + dxi;
      float* q = part + (((size_t)blockIdx.x * 27 + tap) * Cout + co) * Cin + c0;
#pragma unroll
      for (int j = 0; j < 16; ++j) q[j] = (nrow == 0) ? 0.f : (ok ? __uint_as_float(rr[j]) : nanv);
    }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncols) : "memory");
  }
  if (!ok) atomicExch(&g_tc_err, 1);
}

}  // namespace tc
}  // namespace dynot
