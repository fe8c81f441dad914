// fam_internal.cuh -- private host-side definitions shared by the C ABI
// (fam_api.cu) and the per-configuration kernel instantiation units
// (fam_inst.cu): the handle, the launch table and the launchers.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "../../include/fam.h"
#include "fam_kernels1d.cuh"

using namespace fam;

// tile shapes
// 2D tile shapes (one thread per cell), chosen by option "tile2d" or fam_tune:
//   0: 32 x 8 (256 threads, 1 block/SM), 1: 32 x 4 (128 threads, 2 blocks/SM),
//   2: 16 x 8 (128 threads, 2 blocks/SM)
constexpr int kTile2D[3][2] = {{32, 8}, {32, 4}, {16, 8}};
constexpr int TX1 = 128;           // 1D: 128 cells per block

// ---------------------------------------------------------------------------
// per-configuration launchers
// ---------------------------------------------------------------------------
struct Ops {
  int tx = 0, ty = 0;  // tile of the 2D kernels (box of the TMA descriptors)
  cudaError_t (*stage)(struct fam_handle*, int in, int u0, int out, int stage);
  cudaError_t (*oe)(struct fam_handle*, int in, int out, double dt_override);
  cudaError_t (*alpha)(struct fam_handle*, int buf);
  cudaError_t (*prepare)();  // set shared-memory attributes
  // 2D only (null in 1D): final stage + OE in one persistent launch (C -> B
  // -> A with U^n = A), and the resident blocks per SM of that kernel
  cudaError_t (*fused)(struct fam_handle*);
  cudaError_t (*fused_occupancy)(int* blocks_per_sm);
  // BP/PP safeguard (Euler; option "pp_limiter"): before a stage reading
  // buffer buf, the 2D scaling factors of its cells (theta buffer), and with
  // want_dt the step size from the limited point speeds (1D: only the step
  // size; the 1D stage kernel scales inline)
  cudaError_t (*pp_prep)(struct fam_handle*, int buf, bool want_dt);
};

struct fam_handle {
  int d = 1, k = 5, eq = FAM_EULER, bc = FAM_BC_PERIODIC, prec = 64;
  fam_grid grid{};
  Geo geo{};
  int nc = 1, nm = 2, np = 2;
  double gamma = 1.4, ax = 1.0, ay = 1.0;
  int oe_type = 2;
  double gamma_k = 0.0;
  int oe_q6 = 1;
  int smooth_dt = 0;
  double dt_max = 0.0;
  size_t elem = 8;
  size_t buf_elems = 0;
  void* buf[3] = {nullptr, nullptr, nullptr};
  FamCtl* ctl = nullptr;
  double inflow[4][4] = {{0}};   // inflow states per side (conservative averages)
  // front side condition (y-sides, bc kBcFront): behind = inflow[side] left of
  // x = front[0] + front[1] y + front[2] t, front_ahead right of it
  double front[4][3] = {{0}};
  double front_ahead[4][4] = {{0}};
  double* t1_partial = nullptr;  // Type-I OE block partial sums
  int t1_blocks = 0;
  CUtensorMap tm[3];
  CUtensorMap tm_u0[3];  // 2D: U^n rows of a tile (box (tx+4) x ty x planes)
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  bool have_state = false;
  bool dt_valid = false;
  double cfl_set = -1.0;
  double T_set = 0.0;
  std::map<long, cudaGraphExec_t> graphs;
  Ops ops{};
  std::string err;
  int tile2d = 0;  // index into kTile2D
  // opt-in per-kernel timing (option "profile"): 5 events per step bracket
  // the three stage launches and the OE launch of fam_step()
  bool profile = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<char> prof_fused;  // per profiled step: stage 3 and OE ran fused
  size_t ev_used = 0;
  double prof_ms[4] = {0, 0, 0, 0};
  long prof_steps = 0;
  // fused final stage + OE (option "fused_oe"): the task list of the
  // persistent launch, its ticket / tile flags, and its grid size
  int fused_oe = 0;
  int* fz_tasks = nullptr;
  unsigned int* fz_sync = nullptr;
  int fz_ntasks = 0, fz_ntiles = 0, fz_grid = 0;
  bool fz_ready = false;  // task list built for the current tile shape and sides
  // BP/PP safeguard (option "pp_limiter"); 2D: scaling factors, 2 planes
  int pp = 0;
  void* theta = nullptr;
};

inline fam_status fail(fam_handle* h, fam_status s, const std::string& msg) {
  if (h) h->err = msg;
  return s;
}

inline fam_status cuda_fail(fam_handle* h, cudaError_t e, const char* where) {
  return fail(h, FAM_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define FAM_CUDA(h, call)                                   \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call);  \
  } while (0)

template <typename T> inline T* bufp(fam_handle* h, int b) { return reinterpret_cast<T*>(h->buf[b]); }

template <typename T, class PH> PH make_phys(const fam_handle* h);
template <> inline Advection1D<double> make_phys<double, Advection1D<double>>(const fam_handle* h) { return {h->ax}; }
template <> inline Advection1D<float> make_phys<float, Advection1D<float>>(const fam_handle* h) { return {(float)h->ax}; }
template <> inline Burgers1D<double> make_phys<double, Burgers1D<double>>(const fam_handle*) { return {}; }
template <> inline Burgers1D<float> make_phys<float, Burgers1D<float>>(const fam_handle*) { return {}; }
template <> inline BuckleyLeverett1D<double> make_phys<double, BuckleyLeverett1D<double>>(const fam_handle*) {
  return {};
}
template <> inline BuckleyLeverett1D<float> make_phys<float, BuckleyLeverett1D<float>>(const fam_handle*) { return {}; }
template <> inline Euler1D<double> make_phys<double, Euler1D<double>>(const fam_handle* h) {
  return {h->gamma, h->gamma - 1.0, 0.5 * (h->gamma - 1.0)};
}
template <> inline Euler1D<float> make_phys<float, Euler1D<float>>(const fam_handle* h) {
  return {(float)h->gamma, (float)(h->gamma - 1.0), (float)(0.5 * (h->gamma - 1.0))};
}
template <> inline Advection2D<double> make_phys<double, Advection2D<double>>(const fam_handle* h) { return {h->ax, h->ay}; }
template <> inline Advection2D<float> make_phys<float, Advection2D<float>>(const fam_handle* h) {
  return {(float)h->ax, (float)h->ay};
}
template <> inline Burgers2D<double> make_phys<double, Burgers2D<double>>(const fam_handle*) { return {}; }
template <> inline Burgers2D<float> make_phys<float, Burgers2D<float>>(const fam_handle*) { return {}; }
template <> inline Euler2D<double> make_phys<double, Euler2D<double>>(const fam_handle* h) {
  return {h->gamma, h->gamma - 1.0, 0.5 * (h->gamma - 1.0)};
}
template <> inline Euler2D<float> make_phys<float, Euler2D<float>>(const fam_handle* h) {
  return {(float)h->gamma, (float)(h->gamma - 1.0), (float)(0.5 * (h->gamma - 1.0))};
}

inline double default_gamma_k(const fam_handle* h) {
  if (h->gamma_k > 0.0) return h->gamma_k;
  if (h->k <= 4) return 25.0;
  return h->d == 1 ? 12.5 : 15.0;
}

template <typename T, int K, class PH, int TX2, int TY2>
struct Impl2D {
  static constexpr int kTX = TX2, kTY = TY2;
  using S = Smem2D<T, PH::NC, TX2, TY2>;
  using SF = SmemFused<T, PH::NC, TX2, TY2>;
  static cudaError_t prepare() {
    cudaError_t e = cudaFuncSetAttribute(stage2d<T, K, PH, TX2, TY2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)S::bytes_stage);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(stage3_oe2d<T, K, PH, TX2, TY2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)SF::bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(oe2d<T, K, PH, TX2, TY2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)S::bytes_oe);
  }
  static cudaError_t fused_occupancy(int* per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, stage3_oe2d<T, K, PH, TX2, TY2>, TX2 * TY2,
                                                         SF::bytes);
  }
  static cudaError_t fused(fam_handle* h) {
    stage3_oe2d<T, K, PH, TX2, TY2><<<h->fz_grid, TX2 * TY2, SF::bytes, h->stream>>>(
        bufp<T>(h, 2), bufp<T>(h, 0), bufp<T>(h, 1), bufp<T>(h, 0), h->geo, make_phys<T, PH>(h), h->ctl, h->oe_type,
        T(default_gamma_k(h)), h->oe_q6, h->fz_tasks, h->fz_ntasks, h->fz_sync);
    return cudaGetLastError();
  }
  static dim3 grid(const fam_handle* h) {
    return dim3((h->geo.nx + TX2 - 1) / TX2, (h->geo.ny + TY2 - 1) / TY2);
  }
  static cudaError_t stage(fam_handle* h, int in, int u0, int out, int s) {
    stage2d<T, K, PH, TX2, TY2><<<grid(h), TX2 * TY2, S::bytes_stage, h->stream>>>(
        h->tm[in], h->tm_u0[u0], bufp<T>(h, out), h->geo, make_phys<T, PH>(h), h->ctl, s,
        h->pp ? reinterpret_cast<const T*>(h->theta) : nullptr);
    return cudaGetLastError();
  }
  static cudaError_t pp_prep(fam_handle* h, int b, bool want_dt) {
    if constexpr (PH::NC == 4) {
      const long long n = (long long)(h->geo.nx + 2) * (h->geo.ny + 2);
      const int blocks = (int)std::min<long long>((n + 63) / 64, 148LL * 16);
      pp_theta2d<T, K, PH, 64><<<blocks, 64, 0, h->stream>>>(bufp<T>(h, b), reinterpret_cast<T*>(h->theta),
                                                              h->geo, make_phys<T, PH>(h), h->ctl, want_dt ? 1 : 0);
      return cudaGetLastError();
    }
    return cudaErrorNotSupported;
  }
  static cudaError_t oe(fam_handle* h, int in, int out, double dto) {
    oe2d<T, K, PH, TX2, TY2><<<grid(h), TX2 * TY2, S::bytes_oe, h->stream>>>(
        h->tm[in], bufp<T>(h, out), h->geo, make_phys<T, PH>(h), h->ctl, h->oe_type, T(default_gamma_k(h)),
        h->oe_q6, dto);
    return cudaGetLastError();
  }
  static cudaError_t alpha(fam_handle* h, int b) {
    long long n = (long long)h->geo.nx * h->geo.ny;
    int blocks = (int)std::min<long long>((n + 255) / 256, 148LL * 8);
    alpha2d<T, PH, 256><<<blocks, 256, 0, h->stream>>>(bufp<T>(h, b), h->geo, make_phys<T, PH>(h), h->ctl);
    return cudaGetLastError();
  }
};

template <typename T, int K, class PH>
struct Impl1D {
  using S = Smem1D<T, PH::NC, TX1>;
  static cudaError_t prepare() {
    cudaError_t e = cudaFuncSetAttribute(stage1d<T, K, PH, TX1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)S::bytes_stage);
    if (e != cudaSuccess) return e;
    if constexpr (PH::kLimiter != 0) {
      e = cudaFuncSetAttribute(stage1d<T, K, PH, TX1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)S::bytes_stage);
      if (e != cudaSuccess) return e;
    }
    return cudaFuncSetAttribute(oe1d<T, K, PH, TX1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::bytes_oe);
  }
  static dim3 grid(const fam_handle* h) { return dim3((h->geo.nx + TX1 - 1) / TX1); }
  static cudaError_t stage(fam_handle* h, int in, int u0, int out, int s) {
    if constexpr (PH::kLimiter != 0) {
      if (h->pp) {
        stage1d<T, K, PH, TX1, true><<<grid(h), TX1, S::bytes_stage, h->stream>>>(
            h->tm[in], bufp<T>(h, u0), bufp<T>(h, out), h->geo, make_phys<T, PH>(h), h->ctl, s);
        return cudaGetLastError();
      }
    }
    stage1d<T, K, PH, TX1><<<grid(h), TX1, S::bytes_stage, h->stream>>>(
        h->tm[in], bufp<T>(h, u0), bufp<T>(h, out), h->geo, make_phys<T, PH>(h), h->ctl, s);
    return cudaGetLastError();
  }
  static cudaError_t pp_prep(fam_handle* h, int b, bool want_dt) {
    if constexpr (PH::kLimiter != 0) {
      if (!want_dt) return cudaSuccess;  // the stage kernel scales inline
      const int blocks = std::min((h->geo.nx + 127) / 128, 148 * 8);
      pp_alpha1d<T, K, PH, 128><<<blocks, 128, 0, h->stream>>>(bufp<T>(h, b), h->geo, make_phys<T, PH>(h), h->ctl);
      return cudaGetLastError();
    }
    return cudaErrorNotSupported;
  }
  static cudaError_t oe(fam_handle* h, int in, int out, double dto) {
    oe1d<T, K, PH, TX1><<<grid(h), TX1, S::bytes_oe, h->stream>>>(h->tm[in], bufp<T>(h, out), h->geo,
                                                                   make_phys<T, PH>(h), h->ctl, h->oe_type,
                                                                   T(default_gamma_k(h)), dto);
    return cudaGetLastError();
  }
  static cudaError_t alpha(fam_handle* h, int b) {
    int blocks = std::min((h->geo.nx + 255) / 256, 148 * 8);
    alpha1d<T, PH, 256><<<blocks, 256, 0, h->stream>>>(bufp<T>(h, b), h->geo, make_phys<T, PH>(h), h->ctl);
    return cudaGetLastError();
  }
};

template <class I> Ops ops_of() {
  return Ops{0, 0, &I::stage, &I::oe, &I::alpha, &I::prepare, nullptr, nullptr, &I::pp_prep};
}
template <class I> Ops ops_of2d() {
  return Ops{I::kTX, I::kTY, &I::stage, &I::oe, &I::alpha, &I::prepare, &I::fused, &I::fused_occupancy, &I::pp_prep};
}

// per-configuration selectors, one per instantiation unit (fam_inst.cu)
#define FAM_DECL_PICK(D, P, K) bool fam_pick_d##D##_p##P##_k##K(fam_handle* h);
#define FAM_DECL_PICK_K(D, P) FAM_DECL_PICK(D, P, 3) FAM_DECL_PICK(D, P, 4) FAM_DECL_PICK(D, P, 5) FAM_DECL_PICK(D, P, 6)
FAM_DECL_PICK_K(1, 64)
FAM_DECL_PICK_K(1, 32)
FAM_DECL_PICK_K(2, 64)
FAM_DECL_PICK_K(2, 32)
#undef FAM_DECL_PICK_K
#undef FAM_DECL_PICK

// shared host helpers (fam_api.cu)
fam_status refresh_dt_public(fam_handle* h, double cfl);
fam_status fam_internal_step_fixed_dt(fam_handle* h, double dt, void* const* store);
