// Templated plan: workspace, transform tables, kernel selection and the
// iteration driver, instantiated for float (plan_f32.cu) and double (plan_f64.cu).
#pragma once
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "fft.cuh"
#include "hue_kernels.cuh"
#include "misc_kernels.cuh"
#include "plan_base.h"
#include "rgb_kernels.cuh"
#include "rgb_update_tma.cuh"

namespace dynot {

constexpr int kThreadsXt = 256;
constexpr int kThreadsUpd = 128;
#ifndef DYNOT_YC_W
#define DYNOT_YC_W 8
#endif
constexpr int kW = DYNOT_YC_W;   // x-strip width of the y/colour pass

inline int pmax_for(int P) { return P <= 16 ? 16 : (P <= 32 ? 32 : 64); }
// lengths with an FFT path: 2^k (64-512) and 3 * 2^k (96 = 16 * 6, 192 = 16 * 12); N1 = fft_n1(n)
inline bool fft_len(int n) { return n == 64 || n == 96 || n == 128 || n == 192 || n == 256 || n == 512; }
inline int fft_n1(int n) { return n == 64 ? 8 : (n == 128 ? 8 : 16); }
// threads per block of the y/colour pass (matches pick_kb)
// threads of the y/colour pass for strips of W columns: 3 W / 2 row pairs of length n2 per FFT chunk
// (NT = 12 N1 at W = 8), 256 on the dense path
constexpr int yc_nt(int m1, int w) { return w == 4 ? 6 * m1 : (w == 8 ? 12 * m1 : 24 * m1); }
inline int yc_threads(int n2, int w = kW) { return fft_len(n2) ? yc_nt(fft_n1(n2), w) : 256; }

inline size_t rnd16(size_t b) { return (b + 15) & ~size_t(15); }

// Launch with programmatic dependent launch allowed (the kernels wait for their predecessor with
// griddepcontrol.wait before touching its data; see pdl_wait): the next pass's blocks can be
// scheduled and load their tables while the previous pass drains.  DYNOT_PDL=0 launches plainly.
#ifndef DYNOT_PDL
#define DYNOT_PDL 1
#endif
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = DYNOT_PDL ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// --------------------------------------------------------------------------
// kernel selection
// --------------------------------------------------------------------------
template <typename T> using KA = void (*)(Geo<T>, const v4<T>*, const T*, const T*, T*, XtTables, int);
template <typename T> using KC = void (*)(Geo<T>, const T*, T*, XtTables, int);
template <typename T> using KB = void (*)(Geo<T>, T*, YcTables, int);
template <typename T> using KH = void (*)(Geo<T>, T*, HueTables);

template <typename T, int PM>
KA<T> pick_ka_p(int n) {
  switch (n) {
    case 64: return k_rhs_fwd_xt<T, 8, 8, PM>;
    case 96: return k_rhs_fwd_xt<T, 16, 6, PM>;
    case 128: return k_rhs_fwd_xt<T, 8, 16, PM>;
    case 192: return k_rhs_fwd_xt<T, 16, 12, PM>;
    case 256: return k_rhs_fwd_xt<T, 16, 16, PM>;
    case 512: return k_rhs_fwd_xt<T, 16, 32, PM>;
    default: return k_rhs_fwd_xt<T, 0, 0, PM>;
  }
}
template <typename T>
KA<T> pick_ka(int n, int pm) {
  return pm == 16 ? pick_ka_p<T, 16>(n) : (pm == 32 ? pick_ka_p<T, 32>(n) : pick_ka_p<T, 64>(n));
}
template <typename T, int PM>
KC<T> pick_kc_p(int n) {
  switch (n) {
    case 64: return k_inv_xt<T, 8, 8, PM>;
    case 96: return k_inv_xt<T, 16, 6, PM>;
    case 128: return k_inv_xt<T, 8, 16, PM>;
    case 192: return k_inv_xt<T, 16, 12, PM>;
    case 256: return k_inv_xt<T, 16, 16, PM>;
    case 512: return k_inv_xt<T, 16, 32, PM>;
    default: return k_inv_xt<T, 0, 0, PM>;
  }
}
template <typename T>
KC<T> pick_kc(int n, int pm) {
  return pm == 16 ? pick_kc_p<T, 16>(n) : (pm == 32 ? pick_kc_p<T, 32>(n) : pick_kc_p<T, 64>(n));
}
template <typename T> using KRX = void (*)(Geo<T>, const T*, T*, XtTables, int);
template <typename T> using KCT = void (*)(Geo<T>, T*, const T*);
template <typename T, bool INV>
KRX<T> pick_krx(int n) {
  switch (n) {
    case 64: return k_rows_x<T, 8, 8, INV>;
    case 96: return k_rows_x<T, 16, 6, INV>;
    case 128: return k_rows_x<T, 8, 16, INV>;
    case 192: return k_rows_x<T, 16, 12, INV>;
    case 256: return k_rows_x<T, 16, 16, INV>;
    case 512: return k_rows_x<T, 16, 32, INV>;
    default: return k_rows_x<T, 0, 0, INV>;
  }
}
template <typename T>
KCT<T> pick_kct(int pm) {
  return pm == 16 ? k_cols_t<T, 16> : (pm == 32 ? k_cols_t<T, 32> : k_cols_t<T, 64>);
}
template <typename T, int W>
KB<T> pick_kb_w(int n) {
  switch (n) {
    case 64: return k_solve_yc<T, 8, 8, W, yc_nt(8, W)>;
    case 96: return k_solve_yc<T, 16, 6, W, yc_nt(16, W)>;
    case 128: return k_solve_yc<T, 8, 16, W, yc_nt(8, W)>;
    case 192: return k_solve_yc<T, 16, 12, W, yc_nt(16, W)>;
    case 256: return k_solve_yc<T, 16, 16, W, yc_nt(16, W)>;
    case 512: return k_solve_yc<T, 16, 32, W, yc_nt(16, W)>;
    default: return k_solve_yc<T, 0, 0, kW, 256>;
  }
}
// strips of 4, 8 or 16 columns on the FFT lengths (FP32; the FP64 plan keeps 8)
template <typename T>
KB<T> pick_kb(int n, int w = kW) {
  if constexpr (std::is_same<T, float>::value) {
    if (fft_len(n) && w == 4) return pick_kb_w<T, 4>(n);
    if (fft_len(n) && w == 16) return pick_kb_w<T, 16>(n);
  }
  return pick_kb_w<T, kW>(n);
}
template <typename T> using KD = void (*)(Geo<T>, Arrays<T>, int, TileLayout, double*);

template <typename T, int C, bool PXY>
KD<T> pick_kd_c(bool check, bool wx) {
  if (check) return wx ? k_update_tiled<T, C, true, true, PXY> : k_update_tiled<T, C, true, false, PXY>;
  return wx ? k_update_tiled<T, C, false, true, PXY> : k_update_tiled<T, C, false, false, PXY>;
}
template <typename T, bool PXY>
KD<T> pick_kd_p(int C, bool check, bool wx) {
  switch (C) {
    case 1: return pick_kd_c<T, 1, PXY>(check, wx);
    case 2: return pick_kd_c<T, 2, PXY>(check, wx);
    case 3: return pick_kd_c<T, 3, PXY>(check, wx);
    default: return pick_kd_c<T, 4, PXY>(check, wx);
  }
}
template <typename T>
KD<T> pick_kd(int C, bool check, bool wx, bool per_xy) {
  return per_xy ? pick_kd_p<T, true>(C, check, wx) : pick_kd_p<T, false>(C, check, wx);
}

// the update kernel with tensor-memory-accelerator staging (FP32, Neumann x and y)
using KDT = void (*)(Geo<float>, Arrays<float>, int, double*, int*, const CUtensorMap, const CUtensorMap,
                     const CUtensorMap);
template <int C>
KDT pick_kdt_c(bool check, bool wx) {
  if (check) return wx ? k_update_tma<C, true, true> : k_update_tma<C, true, false>;
  return wx ? k_update_tma<C, false, true> : k_update_tma<C, false, false>;
}
inline KDT pick_kdt(int C, bool check, bool wx) {
  switch (C) {
    case 1: return pick_kdt_c<1>(check, wx);
    case 2: return pick_kdt_c<2>(check, wx);
    case 3: return pick_kdt_c<3>(check, wx);
    default: return pick_kdt_c<4>(check, wx);
  }
}
inline size_t tma_smem(int C) {
  switch (C) {
    case 1: return TmaTiles<1>::total;
    case 2: return TmaTiles<2>::total;
    case 3: return TmaTiles<3>::total;
    default: return TmaTiles<4>::total;
  }
}
#ifndef DYNOT_UPD_TMA
#define DYNOT_UPD_TMA 1   // 0: the plain-load update kernel everywhere
#endif

// cuTensorMapEncodeTiled from the driver, resolved once through the runtime
inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
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

template <typename T>
KH<T> pick_kh(int pm) {
  return pm == 16 ? k_hue_t<T, 16> : (pm == 32 ? k_hue_t<T, 32> : k_hue_t<T, 64>);
}

template <typename T>
struct Plan final : PlanBase {
  Geo<T> g{};
  DevMem mem;           // one allocation for every array
  v4<T>* a[2]{};        // a = x - tau sigma K^T bbar, two buffers (current and next)
  v4<T>* b[2]{};        // scaled dual b, two buffers
  T* phi = nullptr;
  T* hat = nullptr;
  v4<T>* x = nullptr;   // primal output x of the last check
  v4<T>* w = nullptr;   // K x0 + (0, f_b^+) at the cells (dual value of a check)
  T* f0n = nullptr;
  T* f1n = nullptr;
  float* stage = nullptr;   // float staging: 2*B*S inputs, then path packing
  size_t stage_floats = 0;
  double* acc = nullptr;    // [B][kAcc]
  double* mass = nullptr;   // [B][P]
  double* chk = nullptr;    // [B][kChk]
  double* scl = nullptr;    // [B][2]
  double* part = nullptr;   // per-block partial sums of the residual check
  int* err = nullptr;       // set by a kernel whose bounded device wait ran out (sticky until the next start)
  int* active = nullptr;    // [B] per-problem flags of a retiring batch (g.active points here once enabled)
  std::vector<int> h_active;
  int* h_err = nullptr;     // pinned host copy, read with the residuals
  double* h_acc = nullptr;  // pinned host copies of acc and mass
  double* h_mass = nullptr;
  // transform tables
  DevMem tabmem;
  XtTables xt{};
  YcTables yc{};
  HueTables ht{};
  int pmax = 32;
  int scrA = 0, scrB = 0;
  int yw = kW;              // column-strip width of the y/colour pass (autotuned on the FFT lengths)
  size_t smA = 0, smB = 0, smH = 0, smHt = 0;
  KA<T> ka = nullptr;
  KC<T> kc = nullptr;
  bool split_xt = false;    // separate r, x and t launches (the (t, x) plane exceeds shared memory)
  KRX<T> krx_f = nullptr, krx_i = nullptr;
  KCT<T> kct = nullptr;
  int scrS = 0;
  size_t smR = 0, smT = 0;
  KB<T> kb = nullptr;
  KH<T> kh = nullptr;
  bool hue_gemm = false;    // the hue DFTs as dense matrix products (FP32, bins <= kHueGemmMax)
  const T* hwf = nullptr;   // [slot][bin] forward basis
  const T* hwi = nullptr;   // [bin][slot] inverse
  const T* hmf = nullptr;   // [k][t] forward DCT along t (P x P)
  const T* hmi = nullptr;   // [t][k] its inverse
  bool tiled = false;       // tiled update kernel (up to four colour channels)
  bool use_tma = false;     // the tiled update stages its planes with bulk tensor copies
  CUtensorMap tmA[2]{}, tmB[2]{}, tmP{};   // a[p], b[p] and phi for k_update_tma
  int tc = 0;               // time-chunk length of the tiled update (autotuned)
  int par = 0;              // buffer holding the current state
  bool have_x = false;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  // [parity][lead]: the check iteration (x written) with its reductions and the copies of the results
  // to pinned host memory, optionally preceded by one plain iteration
  cudaGraphExec_t gcheck[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  cudaEvent_t ev[12] = {};

  ~Plan() override {
    for (auto& e : gexec)
      if (e) cudaGraphExecDestroy(e);
    for (auto& row : gcheck)
      for (auto& e : row)
        if (e) cudaGraphExecDestroy(e);
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
    if (h_acc) cudaFreeHost(h_acc);
    if (h_err) cudaFreeHost(h_err);
    if (h_mass) cudaFreeHost(h_mass);
  }

  // the FFT paths cover power-of-two axes (DCT for Neumann, real Fourier slots for periodic ones);
  // other lengths take the dense transforms
  bool x_fft() const { return fft_len(n1); }
  bool y_fft() const { return fft_len(n2); }
  size_t xt_smem() const { return xt_layout<T>(nullptr, nullptr, P, n1, pmax, scrA, !x_fft()); }
  size_t yc_smem() const {
    T *t0, *t1, *t2, *t3;
    c2<T> *c0, *c1, *c3;
    return yc_layout<T>(nullptr, C, n2, yw, scrB, !y_fft(), &t0, &c0, &c1, &c3, &t1, &t2, &t3);
  }

  ot_status init() override {
    CUDA_OK(cudaGetDevice(&device));
    pmax = pmax_for(P);
    g.n1 = n1; g.n2 = n2; g.C = C;
    g.per1 = grid.bc[0] == OT_BC_PERIODIC;
    g.per2 = d >= 2 ? grid.bc[1] == OT_BC_PERIODIC : 0;
    g.perc = d >= 3 ? grid.bc[2] == OT_BC_PERIODIC : 0;
    g.P = P; g.S = S; g.B = B; g.N = N;
    g.s1 = (T)grid.axis_scale[0];
    g.s2 = (T)(d >= 2 ? grid.axis_scale[1] : 1.0);
    g.sc = (T)(d >= 3 ? grid.axis_scale[2] : 1.0);
    g.sp = (T)P;
    g.sigma = (T)grid.sigma;
    g.ts = (T)(grid.tau * grid.sigma);

    // ---- workspace
    const size_t cells = (size_t)B * N;
    const size_t narr = 2 * 4 + 2 * 4 + 2 + 4 + 4;
    // staging holds the inputs (2 B S), a packed path (B total) or a packed dual (B (d+1) N)
    stage_floats = std::max<size_t>({2 * (size_t)B * S, (size_t)B * cp.total, (size_t)B * (d + 1) * (size_t)N});
    size_t bytes = narr * rnd16(cells * sizeof(T)) + 2 * rnd16((size_t)B * S * sizeof(T)) +
                   rnd16(stage_floats * sizeof(float)) + rnd16(sizeof(double) * B * kAcc) +
                   rnd16(sizeof(double) * (size_t)B * P) + rnd16(sizeof(double) * B * kChk) +
                   rnd16(sizeof(double) * B * 2) + rnd16(part_bytes()) + 16 + rnd16(sizeof(int) * B);
    CUDA_OK(cudaMalloc(&mem.p, bytes));
    char* q = (char*)mem.p;
    auto take = [&](size_t nb) { char* r = q; q += rnd16(nb); return r; };
    for (int i = 0; i < 2; ++i) a[i] = (v4<T>*)take(cells * sizeof(v4<T>));
    for (int i = 0; i < 2; ++i) b[i] = (v4<T>*)take(cells * sizeof(v4<T>));
    phi = (T*)take(cells * sizeof(T));
    hat = (T*)take(cells * sizeof(T));
    x = (v4<T>*)take(cells * sizeof(v4<T>));
    w = (v4<T>*)take(cells * sizeof(v4<T>));
    f0n = (T*)take((size_t)B * S * sizeof(T));
    f1n = (T*)take((size_t)B * S * sizeof(T));
    stage = (float*)take(stage_floats * sizeof(float));
    acc = (double*)take(sizeof(double) * B * kAcc);
    mass = (double*)take(sizeof(double) * (size_t)B * P);
    chk = (double*)take(sizeof(double) * B * kChk);
    scl = (double*)take(sizeof(double) * B * 2);
    part = (double*)take(part_bytes());
    err = (int*)take(sizeof(int));
    active = (int*)take(sizeof(int) * B);
    CUDA_OK(cudaMemsetAsync(mem.p, 0, bytes, st));

    OT_TRY(build_tables());
    for (auto& e : ev) CUDA_OK(cudaEventCreate(&e));
    CUDA_OK(cudaMallocHost(&h_acc, sizeof(double) * B * kAcc));
    CUDA_OK(cudaMallocHost(&h_err, sizeof(int)));
    *h_err = 0;
    CUDA_OK(cudaMallocHost(&h_mass, sizeof(double) * (size_t)B * P));
    out_scale.assign(B, 1.0);
    tiled = !hue && C <= 4;
    {
      const char* kind = std::getenv("DYNOT_UPDATE_KERNEL");
      plain_update = kind && std::strcmp(kind, "plain") == 0;
    }
    if constexpr (std::is_same<T, float>::value) {
      // DYNOT_UPDATE_KERNEL=plain selects the plain-load update kernel, =staged the staged one wherever it
      // applies (same arithmetic; for comparisons and profiles)
      const char* kind = std::getenv("DYNOT_UPDATE_KERNEL");
      const bool plain = kind && std::strcmp(kind, "plain") == 0;
      force_staged = kind && std::strcmp(kind, "staged") == 0;
      if (tiled && DYNOT_UPD_TMA && !plain && !g.per1 && !g.per2 && n1 % 4 == 0 && n1 >= kTX && n2 >= kTY)
        OT_TRY(make_tensor_maps());
    }
    OT_TRY(tune());
    {
      // DYNOT_TIME_CHUNK=k: time chunks of k planes in the tiled update instead of the tuned length (comparisons)
      const char* tcs = std::getenv("DYNOT_TIME_CHUNK");
      if (tiled && tcs && std::atoi(tcs) >= 1) tc = std::min(std::atoi(tcs), P);
    }
    return OT_OK;
  }

  // Tensor maps of the TMA-staged update: a and b as float tensors [B P][C][n2][4 n1] (a cell's four components
  // are consecutive, so one box row is one run of 16-byte cells), boxes of 33 x 9 cells (a, with the column left
  // and the row below the 32 x 8 tile) and 32 x 8 cells (b); phi as [B P][C][n2][n1], boxes of 40 x 10 cells.
  // Out-of-range cells read as zero.
  ot_status make_tensor_maps() {
    auto enc = tensor_map_encoder();
    if (!enc) return OT_OK;   // no driver entry point: keep the plain-load update
    const cuuint64_t BP = (cuuint64_t)B * P;
    const cuuint64_t dimS[4] = {4ull * n1, (cuuint64_t)n2, (cuuint64_t)C, BP};
    const cuuint64_t strS[3] = {16ull * n1, 16ull * n1 * n2, 16ull * S};
    const cuuint32_t boxA[4] = {4 * (kTX + 1), kTY + 1, (cuuint32_t)C, 1};
    const cuuint32_t boxB[4] = {4 * kTX, kTY, (cuuint32_t)C, 1};
    const cuuint32_t one[4] = {1, 1, 1, 1};
    for (int i = 0; i < 2; ++i) {
      CUresult r = enc(&tmA[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (void*)a[i], dimS, strS, boxA, one,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return OT_OK;   // the driver cannot describe this tensor: keep the plain-load update
      r = enc(&tmB[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (void*)b[i], dimS, strS, boxB, one,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return OT_OK;
    }
    const cuuint64_t dim4[4] = {(cuuint64_t)n1, (cuuint64_t)n2, (cuuint64_t)C, BP};
    const cuuint64_t str4[3] = {4ull * n1, 4ull * n1 * n2, 4ull * S};
    const cuuint32_t boxP[4] = {kTX + 8, kTY + 2, (cuuint32_t)C, 1};
    CUresult r = enc(&tmP, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (void*)phi, dim4, str4, boxP, one,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return OT_OK;
    const size_t smem = tma_smem(C);
    for (int ck = 0; ck < 2; ++ck)
      for (int wx = 0; wx < 2; ++wx) {
        const void* fn = (const void*)pick_kdt(C, ck, wx);
        CUDA_OK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        // the operands come from shared memory: take the largest shared-memory carve-out of the unified L1
        CUDA_OK(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
      }
    tma_ok = use_tma = true;
    return OT_OK;
  }

  // Autotuner, run once per shape and device (the choice is cached for later plans of the shape):
  //  - the y/colour pass: column strips of 4, 8 or 16 (FFT lengths, FP32) with 6, 12 or 24 row pairs per
  //    FFT chunk;
  //  - the tiled update: staged by bulk tensor copies or with plain loads (where both exist), and time chunks
  //    of P, P/2, P/4 or P/8 planes, each timed over whole iterations (FP32).
  // Each candidate is timed over ten launches (after two untimed ones) on the zeroed workspace (b set so that the prox takes its
  // Newton branch); a later candidate must beat the best by 3 % (1 % for the FP32 update, timed over whole iterations,
  // where the update's share dilutes its differences; ties keep the earlier, simpler one).
  struct Tuned {
    int yw = kW, tc = 0;
    bool tma = false;
  };
  static std::mutex& tune_mu() {
    static std::mutex m;
    return m;
  }
  static std::map<std::string, Tuned>& tune_cache() {
    static std::map<std::string, Tuned> c;
    return c;
  }
  std::string shape_key() const {
    char buf[160];
    std::snprintf(buf, sizeof(buf), "%d:%d:%d:%d:%d:%d:%d%d%d:%d:%d%d", (int)sizeof(T), n1, n2, C, P, B, g.per1, g.per2,
                  g.perc, device, (int)tma_ok, (int)force_staged);
    return buf;
  }
  bool tma_ok = false;      // tensor maps exist: the staged update is a candidate
  bool force_staged = false;
  bool plain_update = false;  // DYNOT_UPDATE_KERNEL=plain: no staged kernel, and hue batches update cell by cell

  // y/colour pass with strips of w columns; false when its shared memory does not fit
  bool set_yw(int w) {
    if (hue) return false;
    const int old = yw;
    yw = w;
    scrB = y_fft() ? (yc_threads(n2, yw) / fft_n1(n2)) * n2 : 4 * n2;
    const size_t need = yc_smem();
    int maxsm = 0;
    if (cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess ||
        (int)need > maxsm) {
      yw = old;
      scrB = y_fft() ? (yc_threads(n2, yw) / fft_n1(n2)) * n2 : 4 * n2;
      return false;
    }
    smB = need;
    kb = pick_kb<T>(y_fft() ? n2 : 0, yw);
    return cudaFuncSetAttribute((const void*)kb, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm) == cudaSuccess;
  }

  template <class F>
  ot_status time_launches(F&& launch, float& ms) {
    launch();   // warm
    launch();
    CUDA_OK(cudaGetLastError());
    CUDA_OK(cudaEventRecord(ev[10], st));
    for (int r = 0; r < 10; ++r) launch();
    CUDA_OK(cudaEventRecord(ev[11], st));
    CUDA_OK(cudaEventSynchronize(ev[11]));
    CUDA_OK(cudaEventElapsedTime(&ms, ev[10], ev[11]));
    return OT_OK;
  }

  ot_status tune() {
    std::vector<int> cands;
    for (int d = 1; d <= 8; d *= 2) {
      const int c = (P + d - 1) / d;
      if (c >= 4 || d == 1)
        if (std::find(cands.begin(), cands.end(), c) == cands.end()) cands.push_back(c);
    }
    tc = cands[0];
    use_tma = tma_ok;
    const std::string key = shape_key();
    {
      std::lock_guard<std::mutex> lk(tune_mu());
      auto it = tune_cache().find(key);
      if (it != tune_cache().end()) {
        if (it->second.yw != yw) set_yw(it->second.yw);
        tc = it->second.tc;
        use_tma = it->second.tma;
        return OT_OK;
      }
    }
    // a state on which the prox takes its Newton branch: b_f = 1, b_m = 0.5, a = phi = 0
    const long long cells = (long long)B * N;
    k_fill<v4<T>><<<grid1d(cells), 256, 0, st>>>(cells, mk4<T>(T(0.5), T(0.5), T(0.5), T(1)), b[0]);
    CUDA_OK(cudaGetLastError());
    if (!hue && y_fft() && std::is_same<T, float>::value) {
      float best = 1e30f;
      int bw = yw;
      for (int w : {kW, 4, 16}) {
        if (!set_yw(w)) continue;
        float ms = 0;
        OT_TRY(time_launches([&] {
          launch_pdl(kb, dim3((n1 + yw - 1) / yw, P, B), dim3(yc_threads(n2, yw)), smB, st, g, hat, yc, scrB);
        }, ms));
        if (ms < 0.97f * best) {
          best = ms;
          bw = w;
        }
      }
      set_yw(bw);
    }
    if (tiled) {
      float best = 1e30f;
      Tuned pick{yw, tc, use_tma};
      for (int kind = 0; kind < (tma_ok && !force_staged ? 2 : 1); ++kind) {
        use_tma = tma_ok && kind == 0;
        for (int c : cands) {
          tc = c;
          float ms = 0;
          // FP32: whole iterations, the update's time with phi just written by the inverse pass, as in a solve
          // (timed alone, on a cold workspace, the ranking of the time chunks differed from the one inside
          // iterations); FP64 (the precision study's reference, whose iterations are long): the update alone
          if (std::is_same<T, float>::value) OT_TRY(time_launches([&] { enqueue_iteration(0, false, false); }, ms));
          else OT_TRY(time_launches([&] { enqueue_update(0, false, false); }, ms));
          if (ms < (std::is_same<T, float>::value ? 0.99f : 0.97f) * best) {   // whole iterations: 1 %
            best = ms;
            pick.tc = c;
            pick.tma = use_tma;
          }
        }
      }
      tc = pick.tc;
      use_tma = pick.tma;
    }
    tune_tc = tc;
    // clear both buffer sets again
    for (int i = 0; i < 2; ++i) {
      CUDA_OK(cudaMemsetAsync(a[i], 0, (size_t)B * N * sizeof(v4<T>), st));
      CUDA_OK(cudaMemsetAsync(b[i], 0, (size_t)B * N * sizeof(v4<T>), st));
    }
    std::lock_guard<std::mutex> lk(tune_mu());
    tune_cache()[key] = Tuned{yw, tc, use_tma};
    return OT_OK;
  }
  int tune_tc = 0;

  // ---- transform tables (computed in double on the host)
  ot_status build_tables() {
    std::vector<char> h;
    auto put = [&](const void* src, size_t nb) {
      size_t off = h.size();
      h.resize(off + rnd16(nb));
      std::memcpy(h.data() + off, src, nb);
      return off;
    };
    auto twid = [&](int n, std::vector<T>& tw, std::vector<T>& hw) {
      tw.resize(2 * n);
      hw.resize(2 * n);
      for (int j = 0; j < n; ++j) {
        tw[2 * j] = (T)std::cos(2 * kPi * j / n);
        tw[2 * j + 1] = (T)-std::sin(2 * kPi * j / n);
        hw[2 * j] = (T)std::cos(kPi * j / (2.0 * n));
        hw[2 * j + 1] = (T)-std::sin(kPi * j / (2.0 * n));
      }
    };
    auto cos4 = [&](int n) {
      std::vector<T> c(4 * n);
      for (int m = 0; m < 4 * n; ++m) c[m] = (T)std::cos(kPi * m / (2.0 * n));
      return c;
    };
    auto neu_lam = [&](int n, double s) {
      std::vector<double> l(n);
      for (int j = 0; j < n; ++j) {
        const double v = std::sin(kPi * j / (2.0 * n));
        l[j] = s * s * 4.0 * v * v;
      }
      return l;
    };
    // periodic axis: eigenvalue of each real-Fourier slot (rdft_dense_rows), frequency (slot + 1) / 2
    auto per_lam = [&](int n, double s) {
      std::vector<double> l(n);
      for (int slot = 0; slot < n; ++slot) {
        const int j = (n % 2 == 0 && slot == n - 1) ? n / 2 : (slot + 1) / 2;
        const double v = std::sin(kPi * j / n);
        l[slot] = s * s * 4.0 * v * v;
      }
      return l;
    };
    // (cos, sin)(2 pi m / n) pairs, padded to the 4 n values of the cosine table they replace
    auto cs_pad = [&](int n) {
      std::vector<T> c(4 * n, T(0));
      for (int m = 0; m < n; ++m) {
        c[2 * m] = (T)std::cos(2 * kPi * m / n);
        c[2 * m + 1] = (T)std::sin(2 * kPi * m / n);
      }
      return c;
    };
    auto toT = [&](const std::vector<double>& v) {
      std::vector<T> r(v.size());
      for (size_t i = 0; i < v.size(); ++i) r[i] = (T)v[i];
      return r;
    };
    // time axis: forward and inverse DCT matrices, padded to pmax columns
    std::vector<T> Mf((size_t)P * pmax, T(0)), Mi((size_t)P * pmax, T(0));
    for (int k = 0; k < P; ++k)
      for (int t = 0; t < P; ++t) {
        const double c = std::cos(kPi * k * (2 * t + 1) / (2.0 * P));
        Mf[(size_t)k * pmax + t] = (T)c;
        Mi[(size_t)t * pmax + k] = (T)((k == 0 ? 1.0 : 2.0) / P * c);
      }
    const std::vector<double> lt = neu_lam(P, (double)P);
    const double thr = grid.precision == OT_PREC_MIXED ? grid.lam_fp64 : 0.0;

    std::vector<T> twt(2 * P), hwt(2 * P);
    for (int j = 0; j < P; ++j) {
      twt[2 * j] = (T)std::cos(2 * kPi * j / P);
      twt[2 * j + 1] = (T)-std::sin(2 * kPi * j / P);
      hwt[2 * j] = (T)std::cos(kPi * j / (2.0 * P));
      hwt[2 * j + 1] = (T)-std::sin(kPi * j / (2.0 * P));
    }
    size_t o_twt = put(twt.data(), twt.size() * sizeof(T));
    size_t o_hwt = put(hwt.data(), hwt.size() * sizeof(T));
    size_t o_Mf = put(Mf.data(), Mf.size() * sizeof(T));
    size_t o_Mi = put(Mi.data(), Mi.size() * sizeof(T));
    std::vector<T> ltT = toT(lt);
    size_t o_lt = put(ltT.data(), P * sizeof(T));
    size_t o_ltd = put(lt.data(), P * sizeof(double));

    size_t o_tw1 = 0, o_hw1 = 0, o_c41 = 0, o_tw2 = 0, o_hw2 = 0, o_c42 = 0, o_l1 = 0, o_l1d = 0, o_l2 = 0,
           o_l2d = 0, o_Q = 0, o_lc = 0, o_lcd = 0, o_cs = 0, o_hl = 0, o_hld = 0, o_wf = 0, o_wi = 0, o_mf = 0,
           o_mi = 0;
    if (!hue) {
      std::vector<T> tw, hw;
      twid(n1, tw, hw);
      o_tw1 = put(tw.data(), tw.size() * sizeof(T));
      o_hw1 = put(hw.data(), hw.size() * sizeof(T));
      std::vector<T> c1 = g.per1 ? cs_pad(n1) : cos4(n1);
      o_c41 = put(c1.data(), c1.size() * sizeof(T));
      twid(n2, tw, hw);
      o_tw2 = put(tw.data(), tw.size() * sizeof(T));
      o_hw2 = put(hw.data(), hw.size() * sizeof(T));
      std::vector<T> c2v = g.per2 ? cs_pad(n2) : cos4(n2);
      o_c42 = put(c2v.data(), c2v.size() * sizeof(T));
      std::vector<double> l1 = g.per1 ? per_lam(n1, grid.axis_scale[0]) : neu_lam(n1, grid.axis_scale[0]);
      const double s2y = d >= 2 ? grid.axis_scale[1] : 1.0;
      std::vector<double> l2 = g.per2 ? per_lam(n2, s2y) : neu_lam(n2, s2y);
      std::vector<T> l1T = toT(l1), l2T = toT(l2);
      o_l1 = put(l1T.data(), n1 * sizeof(T));
      o_l1d = put(l1.data(), n1 * sizeof(double));
      o_l2 = put(l2T.data(), n2 * sizeof(T));
      o_l2d = put(l2.data(), n2 * sizeof(double));
      // colour axis: orthonormal eigenbasis of its 1D Laplacian
      std::vector<double> Q((size_t)C * C, 0.0), lc(C, 0.0);
      const double sc = d >= 3 ? grid.axis_scale[2] : 1.0;
      if (!g.perc) {  // Neumann: DCT-II basis, eigenvalues 4 sin^2(pi j / 2C)
        for (int j = 0; j < C; ++j) {
          const double v = std::sin(kPi * j / (2.0 * C));
          lc[j] = sc * sc * 4 * v * v;
          for (int c = 0; c < C; ++c)
            Q[(size_t)c * C + j] = std::sqrt((j == 0 ? 1.0 : 2.0) / C) * std::cos(kPi * j * (2 * c + 1) / (2.0 * C));
        }
      } else {        // periodic: real Fourier basis, eigenvalues 4 sin^2(pi f / C)
        for (int j = 0; j < C; ++j) {
          const int f = (j + 1) / 2;
          const double v = std::sin(kPi * f / C);
          lc[j] = sc * sc * 4 * v * v;
          for (int c = 0; c < C; ++c) {
            double q;
            if (j == 0) q = 1.0 / std::sqrt((double)C);
            else if (C % 2 == 0 && j == C - 1) q = ((c & 1) ? -1.0 : 1.0) / std::sqrt((double)C);
            else if (j & 1) q = std::sqrt(2.0 / C) * std::cos(2 * kPi * f * c / C);
            else q = std::sqrt(2.0 / C) * std::sin(2 * kPi * f * c / C);
            Q[(size_t)c * C + j] = q;
          }
        }
      }
      std::vector<T> QT = toT(Q), lcT = toT(lc);
      o_Q = put(QT.data(), QT.size() * sizeof(T));
      o_lc = put(lcT.data(), C * sizeof(T));
      o_lcd = put(lc.data(), C * sizeof(double));
    } else {
      const int n = n1;
      std::vector<T> cs(2 * n);
      std::vector<double> hl(n);
      for (int m = 0; m < n; ++m) {
        cs[2 * m] = (T)std::cos(2 * kPi * m / n);
        cs[2 * m + 1] = (T)std::sin(2 * kPi * m / n);
      }
      const double s1 = grid.axis_scale[0];
      for (int slot = 0; slot < n; ++slot) {
        int j = (slot + 1) / 2;
        if (n % 2 == 0 && slot == n - 1) j = n / 2;
        const double v = std::sin(kPi * j / n);
        hl[slot] = s1 * s1 * 4 * v * v;
      }
      std::vector<T> hlT = toT(hl);
      o_cs = put(cs.data(), cs.size() * sizeof(T));
      o_hl = put(hlT.data(), n * sizeof(T));
      o_hld = put(hl.data(), n * sizeof(double));
      hue_gemm = std::is_same<T, float>::value && n <= kHueGemmMax && B * P >= kHueGemmRows;
      if (hue_gemm) {
        // W[slot][i]: 1, cos / sin (2 pi i j / n) of frequency j = (slot + 1) / 2, (-1)^i (Nyquist slot of even n);
        // the inverse, stored [i][slot], weighs the slots 1, 2, ..., 2, (1) and divides by n
        std::vector<T> wf((size_t)n * n), wi((size_t)n * n);
        for (int slot = 0; slot < n; ++slot) {
          const bool nyq = n % 2 == 0 && slot == n - 1;
          const int j = (slot + 1) / 2;
          const double wgt = (slot == 0 || nyq) ? 1.0 : 2.0;
          for (int i = 0; i < n; ++i) {
            double v;
            if (slot == 0) v = 1.0;
            else if (nyq) v = (i & 1) ? -1.0 : 1.0;
            else {
              const double ang = 2 * kPi * (double)(((long long)i * j) % n) / n;
              v = (slot & 1) ? std::cos(ang) : std::sin(ang);
            }
            wf[(size_t)slot * n + i] = (T)v;
            wi[(size_t)i * n + slot] = (T)(wgt * v / n);
          }
        }
        o_wf = put(wf.data(), wf.size() * sizeof(T));
        o_wi = put(wi.data(), wi.size() * sizeof(T));
        // the time DCT and its inverse as P x P matrices (rows of the padded tables above)
        std::vector<T> mf((size_t)P * P), mi((size_t)P * P);
        for (int r = 0; r < P; ++r)
          for (int c = 0; c < P; ++c) {
            mf[(size_t)r * P + c] = Mf[(size_t)r * pmax + c];
            mi[(size_t)r * P + c] = Mi[(size_t)r * pmax + c];
          }
        o_mf = put(mf.data(), mf.size() * sizeof(T));
        o_mi = put(mi.data(), mi.size() * sizeof(T));
      }
    }
    CUDA_OK(cudaMalloc(&tabmem.p, h.size()));
    CUDA_OK(cudaMemcpy(tabmem.p, h.data(), h.size(), cudaMemcpyHostToDevice));
    char* base = (char*)tabmem.p;
    if (!hue) {
      xt.tw = base + o_tw1; xt.hw = base + o_hw1; xt.cos4 = base + o_c41;
      xt.Mt_f = base + o_Mf; xt.Mt_i = base + o_Mi;
      xt.twt = base + o_twt; xt.hwt = base + o_hwt;
      yc.tw = base + o_tw2; yc.hw = base + o_hw2; yc.cos4 = base + o_c42;
      yc.lam1 = base + o_l1; yc.lam2 = base + o_l2; yc.lamt = base + o_lt;
      yc.lam1d = (const double*)(base + o_l1d); yc.lam2d = (const double*)(base + o_l2d);
      yc.lamtd = (const double*)(base + o_ltd);
      yc.Qc = base + o_Q; yc.lamc = base + o_lc; yc.lamcd = (const double*)(base + o_lcd);
      yc.lam_fp64 = thr;
      scrA = x_fft() ? (kThreadsXt / fft_n1(n1)) * n1 : 4 * n1;
      scrB = y_fft() ? (yc_threads(n2, yw) / fft_n1(n2)) * n2 : 4 * n2;
      ka = pick_ka<T>(x_fft() ? n1 : 0, pmax);
      kc = pick_kc<T>(x_fft() ? n1 : 0, pmax);
      kb = pick_kb<T>(y_fft() ? n2 : 0);
      smA = xt_smem();
      smB = yc_smem();
      int maxsm = 0;
      CUDA_OK(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
      // a (t, x) plane too large for one block's shared memory takes the split x/t passes
      // (DYNOT_SPLIT_XT=1 selects them for any grid, for comparisons)
      const char* sx = std::getenv("DYNOT_SPLIT_XT");
      split_xt = (int)smA > maxsm || (sx && std::strcmp(sx, "1") == 0);
      if (split_xt) {
        scrS = x_fft() ? (256 / fft_n1(n1)) * n1 : (kRowsX * n1 + 1) / 2;
        T *t0p, *t1p;
        c2<T> *c0p, *c1p, *c2p;
        smR = rows_x_layout<T>(nullptr, n1, scrS, !x_fft(), &t0p, &c0p, &c1p, &c2p, &t1p);
        smT = sizeof(T) * ((size_t)P * pmax + (size_t)P * kColsT);
        krx_f = pick_krx<T, false>(x_fft() ? n1 : 0);
        krx_i = pick_krx<T, true>(x_fft() ? n1 : 0);
        kct = pick_kct<T>(pmax);
      }
      if ((!split_xt && (int)smA > maxsm) || (int)smB > maxsm || (split_xt && ((int)smR > maxsm || (int)smT > maxsm)))
        return seterr(OT_EUNSUPPORTED, "grid needs %zu / %zu bytes of shared memory per block (max %d)",
                      split_xt ? std::max(smR, smT) : smA, smB, maxsm);
      // The limit is a property of the kernel, shared by every plan that uses it:
      // raise it to the device maximum instead of this plan's size.
      if (split_xt) {
        CUDA_OK(cudaFuncSetAttribute((const void*)krx_f, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
        CUDA_OK(cudaFuncSetAttribute((const void*)krx_i, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
        CUDA_OK(cudaFuncSetAttribute((const void*)kct, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
      } else {
        CUDA_OK(cudaFuncSetAttribute((const void*)ka, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
        CUDA_OK(cudaFuncSetAttribute((const void*)kc, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
      }
      CUDA_OK(cudaFuncSetAttribute((const void*)kb, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
    } else {
      if (hue_gemm) {
        CUDA_OK(cudaFuncSetAttribute((const void*)k_hue_tdiv, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kHueTdivSmem));
        hwf = (const T*)(base + o_wf);
        hwi = (const T*)(base + o_wi);
        hmf = (const T*)(base + o_mf);
        hmi = (const T*)(base + o_mi);
      }
      ht.cs = base + o_cs; ht.lam = base + o_hl; ht.lamd = (const double*)(base + o_hld);
      ht.lamt = base + o_lt; ht.lamtd = (const double*)(base + o_ltd);
      ht.Mt_f = base + o_Mf; ht.Mt_i = base + o_Mi;
      ht.lam_fp64 = thr;
      kh = pick_kh<T>(pmax);
      smH = rnd16(sizeof(T) * n1) + rnd16(sizeof(c2<T>) * n1);
      smHt = hue_t_smem_for<T>(pmax);
      int maxsm = 0;
      CUDA_OK(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
      if ((int)smH > maxsm || (int)smHt > maxsm)
        return seterr(OT_EUNSUPPORTED, "hue grid needs %zu / %zu bytes of shared memory per block (max %d)", smH,
                      smHt, maxsm);
      CUDA_OK(cudaFuncSetAttribute((const void*)k_hue_fwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
      CUDA_OK(cudaFuncSetAttribute((const void*)k_hue_inv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
      CUDA_OK(cudaFuncSetAttribute((const void*)kh, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
    }
    return OT_OK;
  }

  Arrays<T> arrays(int p, bool wx) const {
    Arrays<T> A{};
    A.a = a[p];
    A.b = b[p];
    A.an = a[1 - p];
    A.bn = b[1 - p];
    A.x = wx ? x : nullptr;
    A.w = w;
    A.phi = phi;
    A.f0 = f0n;
    A.f1 = f1n;
    return A;
  }
  const v4<T>* aptr(int p) const { return a[p]; }

  // ---- the Poisson solve phi = (A A^T)^+ (A a - f_b^-) for a in buffer p
  void enqueue_poisson(int p, cudaEvent_t* evs) { enqueue_poisson_src(aptr(p), evs); }
  void enqueue_poisson_src(const v4<T>* asrc, cudaEvent_t* evs) {
    if (!hue) {
      if (evs) cudaEventRecord(evs[0], st);
      if (split_xt) {
        k_rhs_cells<T><<<grid1d((long long)B * N), 256, 0, st>>>(g, asrc, (const T*)f0n, (const T*)f1n, hat);
        launch_pdl(krx_f, dim3((P + kRowsX - 1) / kRowsX, n2 * C, B), dim3(256), smR, st, g, (const T*)hat, hat, xt,
                   scrS);
        launch_pdl(kct, dim3((n1 + kColsT - 1) / kColsT, n2 * C, B), dim3(kColsT), smT, st, g, hat,
                   (const T*)xt.Mt_f);
      } else {
        launch_pdl(ka, dim3(n2, C, B), dim3(kThreadsXt), smA, st, g, asrc, (const T*)f0n, (const T*)f1n, hat, xt,
                   scrA);
      }
      if (evs) cudaEventRecord(evs[1], st);
      launch_pdl(kb, dim3((n1 + yw - 1) / yw, P, B), dim3(yc_threads(y_fft() ? n2 : 0, yw)), smB, st, g, hat, yc,
                 scrB);
      if (evs) cudaEventRecord(evs[2], st);
      if (split_xt) {
        launch_pdl(kct, dim3((n1 + kColsT - 1) / kColsT, n2 * C, B), dim3(kColsT), smT, st, g, hat,
                   (const T*)xt.Mt_i);
        launch_pdl(krx_i, dim3((P + kRowsX - 1) / kRowsX, n2 * C, B), dim3(256), smR, st, g, (const T*)hat, phi, xt,
                   scrS);
      } else {
        launch_pdl(kc, dim3(n2, C, B), dim3(kThreadsXt), smA, st, g, (const T*)hat, phi, xt, scrA);
      }
      if (evs) cudaEventRecord(evs[3], st);
    } else {
      if (evs) cudaEventRecord(evs[0], st);
      const dim3 gg((n1 + 63) / 64, (B * P + 63) / 64);
      if constexpr (std::is_same<T, float>::value) {
        if (hue_gemm) {   // r into phi (overwritten by the inverse below), then R W^T into hat
          k_hue_rhs<T><<<grid1d((long long)B * N), 256, 0, st>>>(g, asrc, f0n, f1n, phi);
          k_gemm_nt<<<gg, 128, 0, st>>>(B * P, n1, n1, phi, hwf, hat);
        }
      }
      if (!hue_gemm) k_hue_fwd<T><<<dim3(P, B), 256, smH, st>>>(g, asrc, f0n, f1n, hat, ht);
      if (evs) cudaEventRecord(evs[1], st);
      bool tdone = false;
      if constexpr (std::is_same<T, float>::value) {
        if (hue_gemm) {   // the time transforms of all slot columns: hat -> phi (with the divide) -> hat
          const dim3 gt((n1 + 63) / 64, (P + 63) / 64, B);
          if (P <= kHueTdivMaxP) {
            k_hue_tdiv<<<dim3((n1 + 63) / 64, B), 256, kHueTdivSmem, st>>>(P, n1, (const float*)hmf,
                                                                           (const float*)hmi, hat, (long long)P * n1, ht);
          } else {
            k_gemm_tn<true><<<gt, 256, 0, st>>>(P, n1, P, (const float*)hmf, hat, phi, (long long)P * n1, ht);
            k_gemm_tn<false><<<gt, 256, 0, st>>>(P, n1, P, (const float*)hmi, phi, hat, (long long)P * n1, ht);
          }
          tdone = true;
        }
      }
      if (!tdone) kh<<<dim3((n1 + 256 / pmax - 1) / (256 / pmax), B), 256, smHt, st>>>(g, hat, ht);
      if (evs) cudaEventRecord(evs[2], st);
      if constexpr (std::is_same<T, float>::value) {
        if (hue_gemm) k_gemm_nt<<<gg, 128, 0, st>>>(B * P, n1, n1, hat, hwi, phi);
      }
      if (!hue_gemm) k_hue_inv<T><<<dim3(P, B), 256, smH, st>>>(g, hat, phi, ht);
      if (evs) cudaEventRecord(evs[3], st);
    }
  }

  // partials for the largest grid the autotuner may pick (time chunks of at least 1 plane)
  size_t part_bytes() const {
    const dim3 g1 = tiled_grid(1);
    return sizeof(double) * (size_t)g1.x * g1.y * g1.z * kPart;
  }

  dim3 tiled_grid(int tchunk) const {
    // a Neumann axis leaves its last cell to the halo lane; a periodic one needs a block past it
    const int nbx = std::max(1, ((g.per1 ? n1 : n1 - 1) + kTX - 2) / (kTX - 1));
    const int nby = std::max(1, ((g.per2 ? n2 : n2 - 1) + kTY - 2) / (kTY - 1));
    const int nch = (P + tchunk - 1) / tchunk;
    return dim3(nbx, nby, B * nch);
  }

  void enqueue_update(int p, bool check, bool wx) {
    const Arrays<T> A = arrays(p, wx);
    if (tiled) {
      const dim3 grd = tiled_grid(tc);
      bool done = false;
      if constexpr (std::is_same<T, float>::value) {
        if (use_tma) {
          launch_pdl(pick_kdt(C, check, wx), grd, dim3(kTX, kTY), tma_smem(C), st, g, A, tc, part, err, tmA[p], tmB[p],
                     tmP);
          done = true;
        }
      }
      if (!done) {
        const TileLayout Lt{S, n1, n1 * n2, (long long)P * S, n1, (long long)S};
        launch_pdl(pick_kd<T>(C, check, wx, g.per1 || g.per2), grd, dim3(kTX, kTY), 0, st, g, A, tc, Lt, part);
      }
      if (check) k_reduce_check<<<B, 512, 0, st>>>(part, (int)(grd.x * grd.y * grd.z / B), P, acc, mass, g.active);
      return;
    }
    if (hue && !check && !wx && !g.active && B >= 8 && !plain_update) {
      // a batch of hue problems: the tiled update with the problems as its rows (no coupling between rows,
      // since the y difference factor is zero and the y components of the state stay zero); checks keep the
      // per-problem kernel below, whose sums are per problem
      Geo<T> gr = g;
      gr.n2 = B;
      gr.B = 1;
      gr.per2 = 0;
      gr.s2 = T(0);
      gr.active = nullptr;
      const TileLayout Lt{n1, P * n1, n1, 0, n1, 0};
      const int tcr = std::max(4, (P + 3) / 4);
      const dim3 grd((n1 + kTX - 2) / (kTX - 1), std::max(1, (B - 1 + kTY - 2) / (kTY - 1)), (P + tcr - 1) / tcr);
      launch_pdl(pick_kd<T>(1, false, false, true), grd, dim3(kTX, kTY), 0, st, gr, A, tcr, Lt, part);
      return;
    }
    const dim3 grd((n1 + kThreadsUpd - 1) / kThreadsUpd, n2, C * P * B);
    if (check) {
      if (wx) k_update<T, true, true><<<grd, kThreadsUpd, 0, st>>>(g, A, acc, mass);
      else k_update<T, true, false><<<grd, kThreadsUpd, 0, st>>>(g, A, acc, mass);
    } else {
      if (wx) k_update<T, false, true><<<grd, kThreadsUpd, 0, st>>>(g, A, acc, mass);
      else k_update<T, false, false><<<grd, kThreadsUpd, 0, st>>>(g, A, acc, mass);
    }
  }

  void enqueue_iteration(int p, bool check, bool wx, cudaEvent_t* evs = nullptr) {
    enqueue_poisson(p, evs);
    enqueue_update(p, check, wx);
    if (evs) cudaEventRecord(evs[4], st);
  }

  ot_status graph_for(int p) {
    if (gexec[p]) return OT_OK;
    cudaGraph_t gr = nullptr;
    CUDA_OK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    enqueue_iteration(p, false, false);
    enqueue_iteration(1 - p, false, false);
    const cudaError_t le = cudaGetLastError();
    cudaError_t e = cudaStreamEndCapture(st, &gr);
    if (le != cudaSuccess) {
      if (gr) cudaGraphDestroy(gr);
      return seterr(OT_ECUDA, "kernel launch during graph capture: %s", cudaGetErrorString(le));
    }
    if (e != cudaSuccess) return seterr(OT_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&gexec[p], gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) return seterr(OT_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    return OT_OK;
  }

  // plain iterations (no residual, no x output), pairs from a graph
  ot_status run_plain(int n) {
    while (n >= 2) {
      OT_TRY(graph_for(par));
      CUDA_OK(cudaGraphLaunch(gexec[par], st));
      n -= 2;
    }
    if (n == 1) {
      enqueue_iteration(par, false, false);
      CUDA_OK(cudaGetLastError());
      par ^= 1;
    }
    return OT_OK;
  }

  struct Check {
    double residual = 0, energy = 0, drift = 0, dual = 0, gap = 0;
  };

  // one iteration with residuals (and x output); results land in pinned host memory
  ot_status enqueue_check(bool wx) {
    CUDA_OK(cudaMemsetAsync(acc, 0, sizeof(double) * B * kAcc, st));
    CUDA_OK(cudaMemsetAsync(mass, 0, sizeof(double) * (size_t)B * P, st));
    enqueue_iteration(par, true, wx);
    CUDA_OK(cudaGetLastError());
    par ^= 1;
    if (wx) have_x = true;
    CUDA_OK(cudaMemcpyAsync(h_acc, acc, sizeof(double) * B * kAcc, cudaMemcpyDeviceToHost, st));
    CUDA_OK(cudaMemcpyAsync(h_mass, mass, sizeof(double) * (size_t)B * P, cudaMemcpyDeviceToHost, st));
    CUDA_OK(cudaMemcpyAsync(h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    return OT_OK;
  }

  // per-problem residual, energy (caller units) and mass drift of the last check (after a sync)
  ot_status collect_check(std::vector<ProblemCheck>& per, Check& out) {
    per.resize(B);
    out = Check{};
    if (*h_err) return seterr(OT_ETIMEOUT, "a bounded device wait of the update kernel ran out of its limit");
    for (int bi = 0; bi < B; ++bi) {
      if (g.active && !h_active[bi]) continue;   // retired: its entry keeps the check that retired it
      const double* q = &h_acc[(size_t)bi * kAcc];
      const double res = std::sqrt(q[0]) / std::max(std::sqrt(q[1]), 1e-300);
      if (!std::isfinite(res) || !std::isfinite(q[2]) || !std::isfinite(q[3]))
        return seterr(OT_ENUMERIC, "non-finite residual in problem %d", bi);
      double M = 0;
      for (int t = 0; t + 1 < P; ++t) M = std::max(M, std::fabs(h_mass[(size_t)bi * P + t] - (double)S));
      per[bi].residual = res;
      per[bi].energy = q[2] / (double)N * out_scale[bi];
      per[bi].dual = (double)g.sigma * q[3] / (double)N * out_scale[bi];
      per[bi].gap = std::fabs(per[bi].energy - per[bi].dual) /
                    std::max(std::max(std::fabs(per[bi].energy), std::fabs(per[bi].dual)), 1e-300);
      per[bi].drift = M / (double)S;
      out.residual = std::max(out.residual, res);
      out.energy += per[bi].energy / B;
      out.dual += per[bi].dual / B;
      out.gap = std::max(out.gap, per[bi].gap);
      out.drift = std::max(out.drift, per[bi].drift);
    }
    return OT_OK;
  }

  // one launch for [plain iteration on p (lead)] + check iteration (x written) + result copies
  ot_status check_graph_for(int p, bool lead) {
    if (gcheck[p][lead]) return OT_OK;
    cudaGraph_t gr = nullptr;
    CUDA_OK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    cudaMemsetAsync(acc, 0, sizeof(double) * B * kAcc, st);
    cudaMemsetAsync(mass, 0, sizeof(double) * (size_t)B * P, st);
    if (lead) enqueue_iteration(p, false, false);
    enqueue_iteration(lead ? 1 - p : p, true, true);
    cudaMemcpyAsync(h_acc, acc, sizeof(double) * B * kAcc, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(h_mass, mass, sizeof(double) * (size_t)B * P, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    const cudaError_t le = cudaGetLastError();
    cudaError_t e = cudaStreamEndCapture(st, &gr);
    if (le != cudaSuccess) {
      if (gr) cudaGraphDestroy(gr);
      return seterr(OT_ECUDA, "launch during check-graph capture: %s", cudaGetErrorString(le));
    }
    if (e != cudaSuccess) return seterr(OT_ECUDA, "check-graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&gcheck[p][lead], gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) return seterr(OT_ECUDA, "check-graph instantiate: %s", cudaGetErrorString(e));
    return OT_OK;
  }

  // n iterations, the last one a check (x written), all from graphs; results collected after a sync
  ot_status run_chunk_with_check(int n, Check& out) {
    const int plain = n - 1;
    OT_TRY(run_plain(plain - (plain & 1)));
    const bool lead = plain & 1;
    OT_TRY(check_graph_for(par, lead));
    CUDA_OK(cudaGraphLaunch(gcheck[par][lead], st));
    if (!lead) par ^= 1;   // with a lead iteration the pair returns to the same buffer
    have_x = true;
    CUDA_OK(cudaStreamSynchronize(st));
    std::vector<ProblemCheck> per;
    return collect_check(per, out);
  }

  ot_status run_check(bool wx, Check& out) {
    OT_TRY(enqueue_check(wx));
    CUDA_OK(cudaStreamSynchronize(st));
    std::vector<ProblemCheck> per;
    return collect_check(per, out);
  }

  ot_status drive(int iters, double tol, int check_every, ot_solve_stats* stats, double fallback = 0.0,
                  int* used_cold = nullptr) {
    if (iters < 1) return seterr(OT_EINVAL, "iters must be >= 1");
    CUDA_OK(cudaEventRecord(ev[10], st));
    int done = 0;
    Check ck;
    bool converged = false;
    const int K = check_every > 0 ? check_every : iters;
    while (done < iters) {
      const int chunk = std::min(K, iters - done);
      const bool last = (done + chunk == iters);
      OT_TRY(run_chunk_with_check(chunk, ck));
      const bool first = (done == 0);
      done += chunk;
      if (first && fallback > 0 && ck.residual > fallback) {
        // the warm start is worse than the threshold: restart from x = 0, b = bbar = 0
        OT_TRY(cold_start());
        if (used_cold) *used_cold = 1;
        continue;
      }
      if (tol > 0 && ck.residual <= tol) {
        converged = true;
        break;
      }
      (void)last;
    }
    CUDA_OK(cudaEventRecord(ev[11], st));
    CUDA_OK(cudaEventSynchronize(ev[11]));
    float ms = 0;
    CUDA_OK(cudaEventElapsedTime(&ms, ev[10], ev[11]));
    if (stats) {
      stats->iterations = done;
      stats->residual = ck.residual;
      stats->energy = ck.energy;
      stats->mass_drift = ck.drift;
      stats->elapsed_ms = ms;
      stats->dual_value = ck.dual;
      stats->gap = ck.gap;
    }
    if (tol > 0 && !converged) return seterr(OT_ENOTCONV, "residual %.3e > tol %.3e after %d iterations",
                                             ck.residual, tol, done);
    return OT_OK;
  }

  // ---- inputs
  ot_status load_boundary(const float* f0, const float* f1, bool normalise) {
    const size_t n = (size_t)B * S;
    CUDA_OK(cudaMemcpyAsync(stage, f0, n * sizeof(float), cudaMemcpyDefault, st));
    CUDA_OK(cudaMemcpyAsync(stage + n, f1, n * sizeof(float), cudaMemcpyDefault, st));
    return validate_scale(normalise);
  }

  // problem bi's densities into the staging area (batches assembled from separate arrays)
  ot_status stage_problem(int bi, const float* f0, const float* f1) override {
    if (bi < 0 || bi >= B || !f0 || !f1) return seterr(OT_EINVAL, "bad problem index or NULL density");
    const size_t n = (size_t)B * S;
    CUDA_OK(cudaMemcpyAsync(stage + (size_t)bi * S, f0, S * sizeof(float), cudaMemcpyDefault, st));
    CUDA_OK(cudaMemcpyAsync(stage + n + (size_t)bi * S, f1, S * sizeof(float), cudaMemcpyDefault, st));
    return OT_OK;
  }

  ot_status prepare_staged() override {
    OT_TRY(validate_scale(true));
    OT_TRY(cold_start());
    return make_dual_weights();
  }

  // validate the staged densities (section 2: f >= 0, equal masses) and rescale (reading of section 4)
  ot_status validate_scale(bool normalise) {
    const size_t n = (size_t)B * S;
    std::vector<double> sc(2 * B, 1.0);
    if (normalise) {
      CUDA_OK(cudaMemsetAsync(chk, 0, sizeof(double) * B * kChk, st));
      // minima start at +inf
      std::vector<double> init((size_t)B * kChk, 0.0);
      for (int bi = 0; bi < B; ++bi) init[(size_t)bi * kChk + 2] = init[(size_t)bi * kChk + 3] = INFINITY;
      CUDA_OK(cudaMemcpyAsync(chk, init.data(), init.size() * sizeof(double), cudaMemcpyHostToDevice, st));
      const int blocks = std::min(1024, (S + 255) / 256);
      k_check_inputs<<<dim3(blocks, B), 256, 0, st>>>(stage, stage + n, S, chk);
      CUDA_OK(cudaGetLastError());
      std::vector<double> h((size_t)B * kChk);
      CUDA_OK(cudaMemcpyAsync(h.data(), chk, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
      CUDA_OK(cudaStreamSynchronize(st));
      for (int bi = 0; bi < B; ++bi) {
        const double* q = &h[(size_t)bi * kChk];
        if (q[4] > 0) return seterr(OT_EMASS, "problem %d: non-finite density values", bi);
        if (q[2] < 0 || q[3] < 0) return seterr(OT_EMASS, "problem %d: negative density values", bi);
        const double M0 = q[0], M1 = q[1];
        if (!(M0 > 0) || !(M1 > 0) || std::fabs(M0 - M1) > 1e-6 * std::max(M0, M1))
          return seterr(OT_EMASS, "problem %d: masses differ (%.9g vs %.9g)", bi, M0, M1);
        sc[2 * bi] = (double)S / M0;
        sc[2 * bi + 1] = (double)S / M1;
        out_scale[bi] = 0.5 * (M0 + M1) / (double)S;
      }
    } else {
      for (int bi = 0; bi < B; ++bi) out_scale[bi] = 1.0;
    }
    CUDA_OK(cudaMemcpyAsync(scl, sc.data(), sc.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    const int blocks = std::min(1024, (S + 255) / 256);
    k_scale_boundary<T><<<dim3(blocks, B), 256, 0, st>>>(stage, stage + n, S, scl, f0n, f1n);
    CUDA_OK(cudaGetLastError());
    return OT_OK;
  }

  int grid1d(long long n) const { return (int)std::min<long long>((n + 255) / 256, 152 * 16); }

  // internal x <- packed (float), solver units
  ot_status unpack_x(const float* packed) {
    const size_t n = (size_t)B * cp.total;
    CUDA_OK(cudaMemcpyAsync(stage, packed, n * sizeof(float), cudaMemcpyDefault, st));
    k_unpack_path<T><<<grid1d((long long)B * N), 256, 0, st>>>(g, cp, stage, 1.0, x);
    CUDA_OK(cudaGetLastError());
    return OT_OK;
  }

  // w = K x0 + (0, f_b^+) for the boundary densities in f0n, f1n, with x0 = Pi_{C_d}(0) the least-norm feasible
  // path (the projection of step 1 applied to a = 0); x serves as the work array.
  ot_status make_dual_weights() {
    const long long cells = (long long)B * N;
    CUDA_OK(cudaMemsetAsync(x, 0, cells * sizeof(v4<T>), st));
    enqueue_poisson_src(x, nullptr);
    Arrays<T> A{};
    A.a = x;
    A.x = x;   // in place: every cell reads only its own a
    A.phi = phi;
    A.f0 = f0n;
    A.f1 = f1n;
    k_correct<T><<<grid1d(cells), 256, 0, st>>>(g, A);
    k_dual_weights<T><<<grid1d(cells), 256, 0, st>>>(g, x, f0n, f1n, w);
    CUDA_OK(cudaGetLastError());
    have_x = false;
    return OT_OK;
  }

  ot_status cold_start() {
    CUDA_OK(cudaMemsetAsync(a[0], 0, (size_t)B * N * sizeof(v4<T>), st));
    CUDA_OK(cudaMemsetAsync(b[0], 0, (size_t)B * N * sizeof(v4<T>), st));
    CUDA_OK(cudaMemsetAsync(b[1], 0, (size_t)B * N * sizeof(v4<T>), st));
    CUDA_OK(cudaMemsetAsync(err, 0, sizeof(int), st));
    *h_err = 0;
    par = 0;
    have_x = false;
    return OT_OK;
  }

  ot_status solve(const float* f0, const float* f1, int iters, double tol, const float* init,
                  const float* init_dual, int dual_init, double dual_support, double fallback, ot_solve_stats* stats,
                  int* used_cold) override {
    if (!f0 || !f1) return seterr(OT_EINVAL, "f0 and f1 are required");
    if (used_cold) *used_cold = 0;
    OT_TRY(load_boundary(f0, f1, true));
    OT_TRY(cold_start());
    OT_TRY(make_dual_weights());
    if (init) {
      // x0 = init (scaled to solver units per problem) into x, then b = bbar = 0 or the fixed-point dual
      const size_t n = (size_t)B * cp.total;
      CUDA_OK(cudaMemcpyAsync(stage, init, n * sizeof(float), cudaMemcpyDefault, st));
      for (int bi = 0; bi < B; ++bi) {   // one scale per problem
        Geo<T> g1 = g;
        g1.B = 1;
        const size_t off = (size_t)bi * N;
        k_unpack_path<T><<<grid1d(N), 256, 0, st>>>(g1, cp, stage + (size_t)bi * cp.total, 1.0 / out_scale[bi],
                                                    x + off);
        CUDA_OK(cudaGetLastError());
      }
      const long long cells = (long long)B * N;
      if (init_dual) {
        OT_TRY(load_dual(init_dual, b[0]));
        CUDA_OK(cudaMemcpyAsync(b[1], b[0], cells * sizeof(v4<T>), cudaMemcpyDeviceToDevice, st));
      } else if (dual_init) {
        // the domain's diameter: extent n_k / scale_k per axis, half of it on periodic axes
        double diam2 = 0;
        for (int k = 0; k < grid.ndim; ++k) {
          const double e = grid.n[k] / grid.axis_scale[k] * (grid.bc[k] == OT_BC_PERIODIC ? 0.5 : 1.0);
          diam2 += e * e;
        }
        k_dual_init<T><<<grid1d(cells), 256, 0, st>>>(g, x, f0n, f1n, T(1.0 / grid.sigma), T(1e-3),
                                                      T(std::sqrt(diam2)), T(dual_support), b[0]);
        CUDA_OK(cudaGetLastError());
        CUDA_OK(cudaMemcpyAsync(b[1], b[0], cells * sizeof(v4<T>), cudaMemcpyDeviceToDevice, st));
      }
      // a = x0 - tau sigma K^T bbar0 (bbar0 = b0)
      k_make_a<T><<<grid1d(cells), 256, 0, st>>>(g, x, b[0], a[0]);
      CUDA_OK(cudaGetLastError());
    }
    return drive(iters, tol, grid.check_every, stats, init ? fallback : 0.0, used_cold);
  }

  // ---- hooks for mixed-size batches (several plans captured into one graph)
  ot_status enqueue_pair() override {
    enqueue_iteration(par, false, false);
    enqueue_iteration(1 - par, false, false);
    CUDA_OK(cudaGetLastError());
    return OT_OK;
  }
  ot_status enqueue_single() override {
    enqueue_iteration(par, false, false);
    CUDA_OK(cudaGetLastError());
    par ^= 1;
    return OT_OK;
  }
  ot_status enqueue_check_async() override { return enqueue_check(true); }
  ot_status collect(std::vector<ProblemCheck>& per) override {
    Check ck;
    return collect_check(per, ck);
  }
  int parity() const override { return par; }

  ot_status enable_retirement() override {
    if (gexec[0] || gexec[1]) return seterr(OT_EINVAL, "retirement must be enabled before graphs are captured");
    h_active.assign(B, 1);
    CUDA_OK(cudaMemcpyAsync(active, h_active.data(), sizeof(int) * B, cudaMemcpyHostToDevice, st));
    CUDA_OK(cudaStreamSynchronize(st));
    g.active = active;
    return OT_OK;
  }
  ot_status set_active(const std::vector<int>& act, cudaStream_t s) override {
    if (!g.active || (int)act.size() != B) return seterr(OT_EINVAL, "retirement is not enabled for this plan");
    h_active = act;
    CUDA_OK(cudaMemcpyAsync(active, h_active.data(), sizeof(int) * B, cudaMemcpyHostToDevice, s));
    CUDA_OK(cudaStreamSynchronize(s));
    return OT_OK;
  }

  ot_status path_one(int bi, float* f, float* m0, float* m1, float* m2) override {
    if (!have_x) return seterr(OT_EINVAL, "no path: run a solve first");
    if (bi < 0 || bi >= B) return seterr(OT_EINVAL, "problem index out of range");
    float* ds[4] = {m0, d >= 2 ? m1 : nullptr, d >= 3 ? m2 : nullptr, f};
    Geo<T> g1 = g;
    g1.B = 1;
    const size_t off = (size_t)bi * N;
    for (int k = 0; k < 4; ++k) {
      if (!ds[k]) continue;
      float* dd[4] = {nullptr, nullptr, nullptr, nullptr};
      dd[k] = stage;
      k_pack_path<T><<<grid1d(N), 256, 0, st>>>(g1, cp, x + off, out_scale[bi], nullptr, dd[0], dd[1], dd[2],
                                                dd[3]);
      CUDA_OK(cudaGetLastError());
      CUDA_OK(cudaMemcpyAsync(ds[k], stage, (size_t)cp.len[k] * sizeof(float), cudaMemcpyDefault, st));
      CUDA_OK(cudaStreamSynchronize(st));
    }
    return OT_OK;
  }

  ot_status path(float* f, float* m0, float* m1, float* m2) override {
    if (!have_x) return seterr(OT_EINVAL, "no path: run ot_solve or ot_iterate first");
    float* ds[4] = {m0, d >= 2 ? m1 : nullptr, d >= 3 ? m2 : nullptr, f};
    for (int k = 0; k < 4; ++k) {
      if (!ds[k]) continue;
      // component k of every problem, scaled back to the caller's units
      for (int bi = 0; bi < B; ++bi) {
        Geo<T> g1 = g;
        g1.B = 1;
        const size_t off = (size_t)bi * N;
        float* dd[4] = {nullptr, nullptr, nullptr, nullptr};
        dd[k] = stage + (size_t)bi * cp.len[k];
        k_pack_path<T><<<grid1d(N), 256, 0, st>>>(g1, cp, x + off, out_scale[bi], nullptr, dd[0], dd[1], dd[2],
                                                  dd[3]);
        CUDA_OK(cudaGetLastError());
      }
      CUDA_OK(cudaMemcpyAsync(ds[k], stage, (size_t)B * cp.len[k] * sizeof(float), cudaMemcpyDefault, st));
      CUDA_OK(cudaStreamSynchronize(st));
    }
    return OT_OK;
  }

  ot_status state_set(const float* f0, const float* f1, const float* xp, const float* bp,
                      const float* bbp) override {
    if (!f0 || !f1 || !xp || !bp) return seterr(OT_EINVAL, "f0, f1, x and b are required");
    OT_TRY(load_boundary(f0, f1, false));
    OT_TRY(make_dual_weights());
    OT_TRY(unpack_x(xp));
    const long long cells = (long long)B * N;
    CUDA_OK(cudaMemsetAsync(err, 0, sizeof(int), st));
    *h_err = 0;
    // b -> b[0]; bbar -> b[1] temporarily
    CUDA_OK(cudaMemsetAsync(b[0], 0, cells * sizeof(v4<T>), st));
    CUDA_OK(cudaMemsetAsync(b[1], 0, cells * sizeof(v4<T>), st));
    OT_TRY(load_dual(bp, b[0]));
    if (bbp) OT_TRY(load_dual(bbp, b[1]));
    else CUDA_OK(cudaMemcpyAsync(b[1], b[0], cells * sizeof(v4<T>), cudaMemcpyDeviceToDevice, st));
    // a[0] = x - tau sigma K^T bbar
    k_make_a<T><<<grid1d(cells), 256, 0, st>>>(g, x, b[1], a[0]);
    CUDA_OK(cudaGetLastError());
    // keep 2 b - bbar in b[1] so that bbar = 2 b[par] - b[1 - par] holds (all four components)
    k_axpby<T><<<grid1d(4 * cells), 256, 0, st>>>(4 * cells, T(2), (const T*)b[0], T(-1), (const T*)b[1],
                                                    (T*)b[1]);
    CUDA_OK(cudaGetLastError());
    par = 0;
    have_x = true;
    CUDA_OK(cudaStreamSynchronize(st));
    return OT_OK;
  }

  // packed dual (float, d+1 components of B*N cells... laid out problem-major) -> internal
  ot_status load_dual(const float* src, v4<T>* dst) {
    const long long cells = (long long)B * N;
    // packed dual: per problem (d+1) components of N cells
    std::vector<int> comp = comps();
    CUDA_OK(cudaMemcpyAsync(stage, src, (size_t)B * (d + 1) * N * sizeof(float), cudaMemcpyDefault, st));
    for (int bi = 0; bi < B; ++bi)
      for (int j = 0; j <= d; ++j) {
        k_comp_in<T><<<grid1d(N), 256, 0, st>>>(N, stage + ((size_t)bi * (d + 1) + j) * N, dst + (size_t)bi * N,
                                                comp[j]);
      }
    CUDA_OK(cudaGetLastError());
    (void)cells;
    return OT_OK;
  }
  std::vector<int> comps() const {
    std::vector<int> c;
    for (int k = 0; k < d; ++k) c.push_back(k);
    c.push_back(3);
    return c;
  }

  ot_status state_get(float* xp, float* bp, float* bbp) override {
    const long long cells = (long long)B * N;
    if (xp) {
      if (!have_x) return seterr(OT_EINVAL, "x is not available: run ot_iterate first");
      k_pack_path<T><<<grid1d(cells), 256, 0, st>>>(g, cp, x, 1.0, stage, nullptr, nullptr, nullptr, nullptr);
      CUDA_OK(cudaGetLastError());
      CUDA_OK(cudaMemcpyAsync(xp, stage, (size_t)B * cp.total * sizeof(float), cudaMemcpyDefault, st));
      CUDA_OK(cudaStreamSynchronize(st));
    }
    std::vector<int> comp = comps();
    for (int which = 0; which < 2; ++which) {
      float* dst = which == 0 ? bp : bbp;
      if (!dst) continue;
      for (int bi = 0; bi < B; ++bi)
        for (int j = 0; j <= d; ++j) {
          const size_t off = (size_t)bi * N;
          float* o = stage + ((size_t)bi * (d + 1) + j) * N;
          if (which == 0) {
            k_comp_out<T><<<grid1d(N), 256, 0, st>>>(N, b[par] + off, comp[j], o);
          } else {
            // bbar = 2 b[par] - b[1-par], computed in T then converted
            k_bbar_out<T><<<grid1d(N), 256, 0, st>>>(N, b[par] + off, b[1 - par] + off, comp[j], o);
          }
        }
      CUDA_OK(cudaGetLastError());
      CUDA_OK(cudaMemcpyAsync(dst, stage, (size_t)B * (d + 1) * N * sizeof(float), cudaMemcpyDefault, st));
      CUDA_OK(cudaStreamSynchronize(st));
    }
    (void)cells;
    return OT_OK;
  }

  ot_status iterate(int iters, ot_solve_stats* stats) override { return drive(iters, 0.0, 0, stats); }

  ot_status project(const float* f0, const float* f1, const float* ap, float* xp, float* phip) override {
    if (!f0 || !f1 || !ap || !xp) return seterr(OT_EINVAL, "f0, f1, a and x are required");
    OT_TRY(load_boundary(f0, f1, false));
    OT_TRY(unpack_x(ap));
    const long long cells = (long long)B * N;
    // a[0] <- unpacked a (stored in x), run the Poisson solve, then x = a - A^T phi
    CUDA_OK(cudaMemcpyAsync(a[0], x, cells * sizeof(v4<T>), cudaMemcpyDeviceToDevice, st));
    enqueue_poisson(0, nullptr);
    Arrays<T> A = arrays(0, true);
    k_correct<T><<<grid1d(cells), 256, 0, st>>>(g, A);
    CUDA_OK(cudaGetLastError());
    k_pack_path<T><<<grid1d(cells), 256, 0, st>>>(g, cp, x, 1.0, stage, nullptr, nullptr, nullptr, nullptr);
    CUDA_OK(cudaGetLastError());
    CUDA_OK(cudaMemcpyAsync(xp, stage, (size_t)B * cp.total * sizeof(float), cudaMemcpyDefault, st));
    if (phip) {
      k_convert<float, T><<<grid1d(cells), 256, 0, st>>>(cells, phi, stage);
      CUDA_OK(cudaMemcpyAsync(phip, stage, cells * sizeof(float), cudaMemcpyDefault, st));
    }
    CUDA_OK(cudaStreamSynchronize(st));
    have_x = false;
    return OT_OK;
  }

  ot_status profile(int iters, double ms[5]) override {
    if (iters < 1) return seterr(OT_EINVAL, "iters must be >= 1");
    double sum[4] = {0, 0, 0, 0};
    for (int i = 0; i < iters; ++i) {
      enqueue_iteration(par, false, false, ev);
      par ^= 1;
      CUDA_OK(cudaGetLastError());
      CUDA_OK(cudaEventSynchronize(ev[4]));
      for (int k = 0; k < 4; ++k) {
        float t = 0;
        CUDA_OK(cudaEventElapsedTime(&t, ev[k], ev[k + 1]));
        sum[k] += t;
      }
    }
    for (int k = 0; k < 4; ++k) ms[k] = sum[k] / iters;
    // whole iterations from the graph
    const int pairs = std::max(1, iters / 2);
    OT_TRY(graph_for(par));
    CUDA_OK(cudaGraphLaunch(gexec[par], st));  // warm
    CUDA_OK(cudaEventRecord(ev[10], st));
    for (int i = 0; i < pairs; ++i) CUDA_OK(cudaGraphLaunch(gexec[par], st));
    CUDA_OK(cudaEventRecord(ev[11], st));
    CUDA_OK(cudaEventSynchronize(ev[11]));
    float t = 0;
    CUDA_OK(cudaEventElapsedTime(&t, ev[10], ev[11]));
    ms[4] = t / (2.0 * pairs);
    return OT_OK;
  }
};


}  // namespace dynot
