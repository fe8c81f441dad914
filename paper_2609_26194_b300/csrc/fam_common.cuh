// fam_common.cuh -- shared device helpers of the FAM CUDA library (sm_103a).
//
// Contents: the device control block (time, step size, wave-speed reduction,
// status flags), padded-layout geometry, FP64 reciprocal / reciprocal square
// root by Newton-Raphson refinement of the FP32 hardware approximations,
// TMA + mbarrier wrappers (inline PTX) with bounded waits, and the
// grid-wide max reduction with a last-block epilogue.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fam {

// ---------------------------------------------------------------------------
// status bits written by kernels (read by the host after a step)
// ---------------------------------------------------------------------------
enum : unsigned int {
  kStatusNonFinite = 1u,     // a non-finite value appeared in the state
  kStatusNonPhysical = 2u,   // rho <= 0 or p <= 0 at a cell average
  kStatusTimeout = 4u,       // a bounded wait (TMA barrier) gave up
  kStatusBadLaunch = 8u,     // launch geometry inconsistent with the tile
};

// Device control block: one per handle (or per instance for batched runs).
struct FamCtl {
  double dt;              // step size of the current step (0: finished)
  double t;               // current time
  double T;               // end time (<= 0: no end time)
  double cfl;             // CFL number of the time-step rule
  double dt_max;          // upper bound on dt (<= 0: none)
  double dx, dy;          // mesh widths
  double dxe, dye;        // dx^e, dy^e with e = 1 or k/3 (time-step rule)
  unsigned long long alpha_bits[2];  // running max of Rusanov speeds (x, y) as bits
  double alpha_last[2];   // speeds used for the current dt
  unsigned long long step;
  unsigned int blocks_done;
  unsigned int status;
  int final_step;         // current dt was clamped to reach T
  int dim;                // 1 or 2
  // Type-I OE (Tab. sigma1d / sigma2d): per component, the bit patterns of
  // max |u_p| and of D_Omega = max |u_p - mean| over the grid, and the mean
  unsigned long long t1_maxabs_bits[4];
  unsigned long long t1_dev_bits[4];
  double t1_mean[4];
};

// Padded structure-of-arrays layout.  Plane p = c * nmom + m; within a
// plane, row r (r = j + G in 2D, 0 in 1D) and column q = i + G.
constexpr int G = 2;  // ghost layers per side

struct Geo {
  int nx, ny;        // interior cells (ny = 1 in 1D)
  int px;            // row pitch in elements (>= nx + 2G, multiple of 4)
  int rows;          // ny + 2G in 2D, 1 in 1D
  long long plane;   // elements per plane = px * rows
  int bcx, bcy;      // boundary condition on every side of a direction (0 periodic, 1 outflow)
  double dx, dy;
  double idx, idy;   // 1/dx, 1/dy
  // per-side conditions (x-lo, x-hi, y-lo, y-hi): 0 periodic, 1 outflow,
  // 2 reflective wall, 3 inflow (ghosts hold a fixed state, written once)
  int bc[4];
  int nm;            // moments per component (planes p = c * nm + m)
  int euler;         // component 1 + dir is the normal momentum of a wall
};

enum { kBcPeriodic = 0, kBcOutflow = 1, kBcReflective = 2, kBcInflow = 3 };

// Sign of plane (c, m) in the mirror image across a wall normal to dir: the
// normal momentum and the moment along the normal flip (both: no flip).
__host__ __device__ inline int reflect_sign(const Geo& g, int plane, int dir) {
  const int c = plane / g.nm, m = plane % g.nm;
  const bool normal_mom = g.euler && c == 1 + dir;
  const bool normal_moment = m == 1 + dir;
  return normal_mom != normal_moment ? -1 : 1;
}

__host__ __device__ inline long long cell_index(const Geo& g, int plane, int j, int i) {
  return (long long)plane * g.plane + (long long)((g.rows > 1 ? j + G : 0)) * g.px + (i + G);
}

// ---------------------------------------------------------------------------
// reciprocal and reciprocal square root
// ---------------------------------------------------------------------------
// FP64: the FP32 hardware approximation (rcp.approx / rsqrt.approx, about
// 23 correct bits) is refined by Newton-Raphson steps in FP64, each of which
// doubles the number of correct bits (Newton's method for f(r) = 1/r - x and
// f(r) = 1/r^2 - x; e.g. Markstein, IBM J. Res. Dev. 34 (1990)).  Two steps
// give a result within a few units in the last place.  Inputs are assumed
// to lie in the FP32 normal range (physical densities and pressures).

__device__ __forceinline__ float rcp_approx_f32(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rsqrt_approx_f32(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

template <typename T> struct Fast;

template <> struct Fast<double> {
  static __device__ __forceinline__ double rcp(double x) {
    double r = (double)rcp_approx_f32((float)x);
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    return fma(r, e, r);
  }
  static __device__ __forceinline__ double rsqrt(double x) {
    double r = (double)rsqrt_approx_f32((float)x);
    double hr = 0.5 * r;
    double e = fma(-x * r, r, 1.0);
    r = fma(hr, e, r);
    hr = 0.5 * r;
    e = fma(-x * r, r, 1.0);
    return fma(hr, e, r);
  }
  static __device__ __forceinline__ double sqrt_(double x) { return x * rsqrt(x); }
  static __device__ __forceinline__ double exp_(double x) { return exp(x); }
};

template <> struct Fast<float> {
  static __device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
  static __device__ __forceinline__ float rsqrt(float x) { return rsqrtf(x); }
  static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
  static __device__ __forceinline__ float exp_(float x) { return expf(x); }
};

// ---------------------------------------------------------------------------
// TMA + mbarrier (inline PTX).  Waits are bounded: after kWaitLimitNs the
// kernel records kStatusTimeout and gives up instead of hanging the GPU.
// ---------------------------------------------------------------------------
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s of wall-clock time

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// Returns false once kWaitLimitNs of wall-clock time have passed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase) {
  if (mbar_try_wait(bar, phase)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, phase))
    if (global_ns() - t0 > kWaitLimitNs) return false;
  return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
      "[%2];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(map) : "memory");
}

// ---------------------------------------------------------------------------
// grid-wide max of non-negative speeds and the last-block epilogue
// ---------------------------------------------------------------------------
// Non-negative doubles order like their bit patterns, so atomicMax on the
// 64-bit pattern is an exact, order-independent (deterministic) max.
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* addr, double v) {
  if (!(v >= 0.0)) v = 0.0;  // NaN-safe: non-finite states are flagged elsewhere
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

template <int NT>
__device__ __forceinline__ double block_max(double v, double* scratch /* >= NT/32 */) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  __syncthreads();
  if (l == 0) scratch[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (l < NT / 32) ? scratch[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  }
  return v;  // valid in thread 0
}

// Called by thread 0 of every block after its atomic max.  The last block to
// arrive computes the next step size from the completed maxima (time-step
// rule of Sec. 4), advances the clock and resets the accumulators.
__device__ inline void step_epilogue(FamCtl* ctl, unsigned int nblocks, bool advance_time) {
  __threadfence();
  unsigned int prev = atomicAdd(&ctl->blocks_done, 1u);
  if (prev != nblocks - 1) return;
  __threadfence();
  volatile unsigned long long* ab = ctl->alpha_bits;
  double ax = __longlong_as_double((long long)ab[0]);
  double ay = __longlong_as_double((long long)ab[1]);
  double t = ctl->t;
  if (advance_time && ctl->dt > 0.0) t = ctl->final_step ? ctl->T : t + ctl->dt;
  double dt;
  if (ctl->dim == 1)
    dt = ctl->cfl * ctl->dxe / ax;
  else
    dt = ctl->cfl / (ax / ctl->dxe + ay / ctl->dye);
  if (!(dt > 0.0) || !isfinite(dt)) {
    dt = 0.0;
    ctl->status |= kStatusNonFinite;
  }
  if (ctl->dt_max > 0.0 && dt > ctl->dt_max) dt = ctl->dt_max;
  int fin = 0;
  if (ctl->T > 0.0) {
    if (t >= ctl->T) {
      dt = 0.0;
    } else if (t + dt >= ctl->T) {
      dt = ctl->T - t;
      fin = 1;
    }
  }
  if (advance_time && ctl->dt > 0.0) ctl->step += 1;
  ctl->t = t;
  ctl->dt = dt;
  ctl->final_step = fin;
  ctl->alpha_last[0] = ax;
  ctl->alpha_last[1] = ay;
  ab[0] = 0ull;
  ab[1] = 0ull;
  __threadfence();
  ctl->blocks_done = 0u;
}

}  // namespace fam
