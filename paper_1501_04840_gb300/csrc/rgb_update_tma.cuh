// K_D with its inputs staged by the tensor memory accelerator (FP32, Neumann x and y).
//
// The same steps and the same arithmetic as update_tiled_body (projection
// correction, interpolation, prox, dual update and the next a; steps 1-4 of
// Algorithm 1), on the same overlapping 32 x 8 tiles of (x, y) columns that
// march over a chunk of time planes.  What differs is how a plane reaches the
// threads: one thread issues three bulk tensor copies per plane -- the tile of
// a with the column left of it and the row below it, the tile of b, and the
// tile of phi with a one-cell halo -- into shared-memory slots (two for a and
// b, three for phi, which a plane also reads as the next plane of the plane
// before it), and an mbarrier per slot counts their bytes.  While plane t is
// computed, a and b of plane t + 1 and phi of planes t + 1 and t + 2 are
// already on their way; the threads read their operands from shared memory
// with constant offsets.  Stores go straight from registers as 16-byte vectors.
//
// Every wait on an mbarrier has a time limit.  A wait that runs out sets *err,
// and the thread carries on without waiting again (its results are then
// meaningless, and the plan reports the error), so no block waits forever.
#pragma once
#include <cuda.h>

#include "rgb_kernels.cuh"

namespace dynot {

template <int C>
struct TmaTiles {
  static constexpr int AX = kTX + 1, AY = kTY + 1;   // a: the column left of the tile and the row below it
  static constexpr int PX = kTX + 8, PY = kTY + 2;   // phi: 40 columns from a 16-byte aligned start, rows y-1 .. y+8
  static constexpr size_t a_bytes = sizeof(float4) * AX * AY * C;
  static constexpr size_t b_bytes = sizeof(float4) * kTX * kTY * C;
  static constexpr size_t p_bytes = sizeof(float) * PX * PY * C;
  static constexpr size_t al(size_t n) { return (n + 127) & ~size_t(127); }
  // two slots of (a, b) and three of phi: a plane's phi is read as the next plane of the plane before it
  static constexpr size_t a_off = 0, b_off = al(a_bytes);
  static constexpr size_t ab_bytes = b_off + al(b_bytes);
  static constexpr size_t p_base = 2 * ab_bytes, p_stride = al(p_bytes);
  static constexpr size_t sbb_off = p_base + 3 * p_stride;
  static constexpr size_t sbb_bytes = sizeof(float) * 2 * kTY * kTX * C;
  static constexpr size_t mbar_off = sbb_off + al(sbb_bytes);
  static constexpr size_t total = mbar_off + 64 + 128;   // five mbarriers, and slack to align the base to 128 bytes
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}
// Wait for the phase of the given parity to complete, for at most kWaitNs; false when the limit ran out.
// A plane's copies land within microseconds; the limit only bounds a wait that would otherwise never end.
constexpr unsigned long long kWaitNs = 20000000ull;   // 20 ms
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  unsigned long long start = 0;
#pragma unroll 1
  for (int i = 0;; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (i == 0) start = global_ns();
    else if ((i & 63) == 0 && global_ns() - start > kWaitNs) return false;
  }
}
__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            int c4, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], "
      "[%7];\n" ::"r"(dst),
      "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];\n" ::"r"(dst),
      "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}

template <int C, bool CHECK, bool WRITE_X, bool INTERIOR>
__device__ __forceinline__ void update_tma_body(const Geo<float>& g, const Arrays<float>& A, int TC,
                                                double* __restrict__ part, int* __restrict__ err, char* sm,
                                                const CUtensorMap* tmA, const CUtensorMap* tmB,
                                                const CUtensorMap* tmP, double (&smass)[64]) {
  using L = TmaTiles<C>;
  const int lane = threadIdx.x, row = threadIdx.y;
  const int tid = threadIdx.x + kTX * threadIdx.y;
  const int x0 = blockIdx.x * (kTX - 1), y0 = blockIdx.y * (kTY - 1);
  const int x = x0 + lane, y = y0 + row;
  const int nch = (g.P + TC - 1) / TC;
  const int b = blockIdx.z / nch;
  if (retired(g, b)) return;
  const int t0 = (blockIdx.z % nch) * TC;
  const int tend = min(t0 + TC, g.P);
  const int tlast = min(tend, g.P - 1);
  const bool vx = INTERIOR || x < g.n1, vy = INTERIOR || y < g.n2;
  const bool live = vx && vy;
  const bool out = live && (lane < kTX - 1 || (!INTERIOR && x == g.n1 - 1)) &&
                   (row < kTY - 1 || (!INTERIOR && y == g.n2 - 1));
  const bool hasR = INTERIOR || x < g.n1 - 1, hasL = INTERIOR || x > 0;
  const bool hasU = INTERIOR || y < g.n2 - 1, hasD = INTERIOR || y > 0;
  const int xa = (x0 - 1) & ~3;      // first column of the phi tile (16-byte aligned)
  const int ox = x - xa;             // this cell's column in the phi tile
  float (*sbb)[kTY][kTX][C] = reinterpret_cast<float (*)[kTY][kTX][C]>(sm + L::sbb_off);
  const uint32_t bar0 = smem_u32(sm + L::mbar_off);
  auto bar_ab = [&](int slot) { return bar0 + 8u * (uint32_t)slot; };        // slots 0, 1
  auto bar_p = [&](int slot) { return bar0 + 8u * (uint32_t)(2 + slot); };   // slots 0, 1, 2
  auto sa = [&](int slot) { return reinterpret_cast<const float4*>(sm + slot * L::ab_bytes + L::a_off); };
  auto sbv = [&](int slot) { return reinterpret_cast<const float4*>(sm + slot * L::ab_bytes + L::b_off); };
  auto sp = [&](int slot) { return reinterpret_cast<const float*>(sm + L::p_base + slot * L::p_stride); };
  // copies of the k-th plane of the chunk (plane t0 + k): a and b into slot k % 2 (computed planes), phi into
  // slot k % 3 (computed planes and the plane after the last one)
  auto issue_ab = [&](int k) {
    const int p = t0 + k;
    if (p > tlast) return;
    const int slot = k & 1;
    mbar_expect_tx(bar_ab(slot), (uint32_t)(L::a_bytes + L::b_bytes));
    const int bp = b * g.P + p;
    char* base = sm + slot * L::ab_bytes;
    // rows of a and b are (cell, component) runs: 16 bytes per cell
    tma_load_4d(smem_u32(base + L::a_off), tmA, 4 * (x0 - 1), y0 - 1, 0, bp, bar_ab(slot));
    tma_load_4d(smem_u32(base + L::b_off), tmB, 4 * x0, y0, 0, bp, bar_ab(slot));
  };
  auto issue_p = [&](int k) {
    const int p = t0 + k;
    if (p > tlast + 1 || p >= g.P) return;
    const int slot = k % 3;
    mbar_expect_tx(bar_p(slot), (uint32_t)L::p_bytes);
    tma_load_4d(smem_u32(sm + L::p_base + slot * L::p_stride), tmP, xa, y0 - 1, 0, b * g.P + p, bar_p(slot));
  };
  if (tid == 0) {
    for (int i = 0; i < 5; ++i) mbar_init(bar0 + 8u * (uint32_t)i, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (CHECK)
    for (int i = tid; i < 64; i += kTX * kTY) smass[i] = 0.0;
  __syncthreads();
  pdl_wait();   // phi (inverse x/t pass) and the state are read from here on
  if (tid == 0) {
    issue_ab(0);
    issue_ab(1);
    issue_p(0);
    issue_p(1);
    issue_p(2);
  }

  const int S = g.S, sc = g.n1 * g.n2;
  const size_t col = (size_t)b * g.P * S + min(x, g.n1 - 1) + (size_t)g.n1 * min(y, g.n2 - 1);
  const size_t col2 = (size_t)b * S + min(x, g.n1 - 1) + (size_t)g.n1 * min(y, g.n2 - 1);
  const float* __restrict__ pas = reinterpret_cast<const float*>(A.a + col);
  const float* __restrict__ pph = A.phi + col;
  const float* __restrict__ pf0 = A.f0 + col2;
  const float* __restrict__ pf1 = A.f1 + col2;
  float4* __restrict__ qa = A.an + col;
  float4* __restrict__ qb = A.bn + col;
  const float s1 = g.s1, s2 = g.s2, scl = g.sc, sp_ = g.sp, ts = g.ts, half = 0.5f;
  const float isg = 1.f / g.sigma;
  const bool perc = g.perc;
  KSum<float> r_db, r_kx, r_J, r_w;

  float phic[C], xfp[C], bbfp[C], cax[C], cay[C], cac[C];
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const int o = t0 * S + c * sc;
    phic[c] = pph[o];
    xfp[c] = (t0 == 0) ? pf0[c * sc] : pas[4 * (o - S) + 3] + sp_ * (phic[c] - pph[o - S]);
    bbfp[c] = 0.f;
    cax[c] = cay[c] = cac[c] = 0.f;
  }
  bool ok = true;

#pragma unroll 1
  for (int t = t0; t <= tlast; ++t) {
    const int k = t - t0, slot = k & 1, ps = k % 3, pn = (k + 1) % 3;
    const int pt = t * S;
    const bool write_plane = t < tend;
    const bool tnext = t + 1 < g.P;
    // once a wait has run out, this thread stops waiting (the error is already recorded below)
    if (ok) ok = mbar_wait(bar_ab(slot), (k >> 1) & 1);
    if (ok) ok = mbar_wait(bar_p(ps), (k / 3) & 1);
    if (ok && tnext) ok = mbar_wait(bar_p(pn), ((k + 1) / 3) & 1);
    const float4* ta = sa(slot);
    const float4* tb = sbv(slot);
    const float* tp = sp(ps);
    const float* tpn = sp(pn);
    float bb[C][4], bn[C][4], xr[C][4], phn[C];
    float4 la[C], lb[C];
    float phy[C], phd[C], la1d[C], la0l[C], phl[C], phx[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const int ra = (c * L::AY + row + 1) * L::AX + lane + 1;   // this cell in the a tile
      const int rp = (c * L::PY + row + 1) * L::PX + ox;         // this cell in the phi tile
      la[c] = ta[ra];
      lb[c] = tb[(c * kTY + row) * kTX + lane];
      phn[c] = tnext ? tpn[rp] : 0.f;
      phy[c] = tp[rp + L::PX];
      phd[c] = tp[rp - L::PX];
      phx[c] = tp[rp + 1];
      la1d[c] = ta[ra - L::AX].y;
      la0l[c] = ta[ra - 1].x;
      phl[c] = tp[rp - 1];
    }
    // right faces of x^{r+1}
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const float ph = phic[c];
      xr[c][0] = hasR ? la[c].x + s1 * (phx[c] - ph) : 0.f;
      xr[c][1] = hasU ? la[c].y + s2 * (phy[c] - ph) : 0.f;
      xr[c][3] = tnext ? la[c].w + sp_ * (phn[c] - ph) : pf1[c * sc];
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const int c1 = (c + 1 == C) ? 0 : c + 1;
      const bool hasC = perc || (c + 1 < C);
      xr[c][2] = hasC ? la[c].z + scl * (phic[c1] - phic[c]) : 0.f;
    }
    // left faces, interpolation to the cell, prox, dual update
#pragma unroll
    for (int c = 0; c < C; ++c) {
      float xlx = __shfl_up_sync(0xffffffffu, xr[c][0], 1);
      if (lane == 0) xlx = la0l[c] + s1 * (phic[c] - phl[c]);
      if (!hasL) xlx = 0.f;
      const float xly = hasD ? la1d[c] + s2 * (phic[c] - phd[c]) : 0.f;
      const int cm = (c == 0) ? C - 1 : c - 1;
      const float xlc = (perc || c > 0) ? xr[cm][2] : 0.f;
      const float k0 = half * (xlx + xr[c][0]);
      const float k1 = half * (xly + xr[c][1]);
      const float k2 = half * (xlc + xr[c][2]);
      const float k3 = half * (xfp[c] + xr[c][3]);
      const float lbk[4] = {lb[c].x, lb[c].y, lb[c].z, lb[c].w};
      const float am0 = k0 + lbk[0], am1 = k1 + lbk[1], am2 = k2 + lbk[2], af = k3 + lbk[3];
      float U0, U1, U2, V;
      prox_cell<float>(am0, am1, am2, af, g.sigma, isg, U0, U1, U2, V);
      bn[c][0] = am0 - U0;
      bn[c][1] = am1 - U1;
      bn[c][2] = am2 - U2;
      bn[c][3] = af - V;
#pragma unroll
      for (int q = 0; q < 4; ++q) bb[c][q] = 2.f * bn[c][q] - lbk[q];
      if (CHECK && out && write_plane) {
        float db2 = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float db = bn[c][q] - lbk[q];
          db2 = fmaf(db, db, db2);
        }
        r_db.add(db2);
        r_kx.add(k0 * k0 + k1 * k1 + k2 * k2 + k3 * k3);
        if (V > 0.f) r_J.add(fdiv_fast(U0 * U0 + U1 * U1 + U2 * U2, 2.f * V));
        const float4 wv = A.w[col + pt + c * sc];
        r_w.add(bn[c][0] * wv.x + bn[c][1] * wv.y + bn[c][2] * wv.z + bn[c][3] * wv.w);
      }
    }
    // neighbours' bbar: x+1 by shuffle, y+1 through shared memory
    const int par = t & 1;
#pragma unroll
    for (int c = 0; c < C; ++c) sbb[par][row][lane][c] = bb[c][1];
    __syncthreads();   // every thread is done with a, b of plane t and phi of plane t: refill their slots
    if (tid == 0) {
      issue_ab(k + 2);
      issue_p(k + 3);
    }
    if (out && t > t0) {
#pragma unroll
      for (int c = 0; c < C; ++c)
        qa[pt - S + c * sc] = make_float4(cax[c], cay[c], cac[c], xfp[c] - ts * half * (bbfp[c] + bb[c][3]));
    }
    if (write_plane) {
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const float bxn = __shfl_down_sync(0xffffffffu, bb[c][0], 1);
        const float byn = (row + 1 < kTY) ? sbb[par][row + 1][lane][c] : 0.f;
        const int c1 = (c + 1 == C) ? 0 : c + 1;
        const bool hasC = perc || (c + 1 < C);
        cax[c] = hasR ? xr[c][0] - ts * half * (bb[c][0] + bxn) : 0.f;
        cay[c] = hasU ? xr[c][1] - ts * half * (bb[c][1] + byn) : 0.f;
        cac[c] = hasC ? xr[c][2] - ts * half * (bb[c][2] + bb[c1][2]) : 0.f;
        if (out) {
          const int o = pt + c * sc;
          qb[o] = make_float4(bn[c][0], bn[c][1], bn[c][2], bn[c][3]);
          if (WRITE_X) A.x[col + o] = make_float4(xr[c][0], xr[c][1], xr[c][2], tnext ? xr[c][3] : 0.f);
        }
      }
      if (CHECK && tnext) {
        float mt = 0;
        if (out) {
#pragma unroll
          for (int c = 0; c < C; ++c) mt += xr[c][3];
        }
        double m = (double)mt;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
        if (lane == 0) atomicAdd(&smass[t], m);
      }
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
      xfp[c] = xr[c][3];
      bbfp[c] = bb[c][3];
      phic[c] = phn[c];
    }
  }
  if (out && tlast == tend - 1) {
#pragma unroll
    for (int c = 0; c < C; ++c) qa[tlast * S + c * sc] = make_float4(cax[c], cay[c], cac[c], 0.f);
  }
  if (!ok) atomicExch(err, 1);
  pdl_trigger();
  if (CHECK) block_check_partials<float>(r_db, r_kx, r_J, r_w, lane, row, nch, b, t0, tend, g.P, part, smass);
}

template <int C, bool CHECK, bool WRITE_X>
__global__ void __launch_bounds__(kTX * kTY, DYNOT_UPD_MINB)
    k_update_tma(Geo<float> g, Arrays<float> A, int TC, double* __restrict__ part, int* __restrict__ err,
                 const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                 const __grid_constant__ CUtensorMap tmP) {
  extern __shared__ __align__(128) char smraw[];
  char* sm = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(smraw) + 127) & ~uintptr_t(127));
  __shared__ double smass[64];
  const int x0 = blockIdx.x * (kTX - 1), y0 = blockIdx.y * (kTY - 1);
  const bool interior = x0 >= 1 && x0 + kTX < g.n1 && y0 >= 1 && y0 + kTY < g.n2;
  if (interior) update_tma_body<C, CHECK, WRITE_X, true>(g, A, TC, part, err, sm, &tmA, &tmB, &tmP, smass);
  else update_tma_body<C, CHECK, WRITE_X, false>(g, A, TC, part, err, sm, &tmA, &tmB, &tmP, smass);
}

}  // namespace dynot
