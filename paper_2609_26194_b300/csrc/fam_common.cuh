// fam_common.cuh -- shared device helpers of the FAM CUDA library (sm_103a).
//
// Contents: the device control block (time, step size, wave-speed reduction,
// status flags), padded-layout geometry, FP64 reciprocal / reciprocal square
// root by refinement of the FP32 hardware approximations, the binary64
// multiply on the integer pipes, integer max / sign helpers, TMA + mbarrier
// wrappers (inline PTX) with bounded waits, and the grid-wide max reduction
// with a last-block epilogue.
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
  // face quadrature points at which a Rusanov trace had no spectral radius
  // (NaN |v_n| + c: an Euler trace with gamma p / rho < 0), summed over the
  // residual evaluations since the state was set
  unsigned long long ntrace;
  // where the first bounded wait that gave up was (0: none): wait kind
  // (kWait*), task or tile index, the tile waited for, mbarrier phase
  unsigned int wait_where, wait_task, wait_dep, wait_phase;
  // BP/PP safeguard, step rejection: a stage kernel sets stage_bad when an
  // output average leaves the admissible set; the OE then writes nothing and
  // its epilogue discards the step (no time advance) and halves the step
  // size: the step sizes of the retries are the CFL size times 2^-retry_exp
  // (at most 30 halvings); an accepted step resets retry_exp.  rejected
  // counts the discarded steps since the state was set.
  unsigned int stage_bad;
  unsigned int retry_exp;
  unsigned long long rejected;
};

enum : unsigned int {
  kWaitTileCopy = 1u,   // TMA copy of a tile + halo
  kWaitU0Copy = 2u,     // TMA copy of U^n rows
  kWaitTileFlag = 3u,   // flag of a tile whose final stage an OE task needs
};

// Record the first wait that gave up (later ones keep the first record).
__device__ __forceinline__ void note_wait(FamCtl* ctl, unsigned int where, unsigned int task, unsigned int dep,
                                          unsigned int phase) {
  if (atomicCAS(&ctl->wait_where, 0u, where) == 0u) {
    ctl->wait_task = task;
    ctl->wait_dep = dep;
    ctl->wait_phase = phase;
  }
}

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
  // 2 reflective wall, 3 inflow (ghosts hold a fixed state, written once),
  // 4 front (y-sides: ghosts hold one of two states by a moving straight
  // front, rewritten before every stage and OE; no images)
  int bc[4];
  int nm;            // moments per component (planes p = c * nm + m)
  int euler;         // component 1 + dir is the normal momentum of a wall
  // split[s] > 0: the ghost cells of side s whose nearest interior cell along
  // the side (row for the x-sides, column for the y-sides) has index below
  // split[s] hold the side's inflow state (no images there)
  int split[4] = {0, 0, 0, 0};
};

enum { kBcPeriodic = 0, kBcOutflow = 1, kBcReflective = 2, kBcInflow = 3, kBcFront = 4 };

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
// FP64: a seed from the FP32 hardware approximation (rcp.approx /
// rsqrt.approx) is refined by one third-order step in FP64.  With the seed r
// and its residual e (e = 1 - x r for 1/x, e = 1 - x r^2 for 1/sqrt(x)) the
// exact values are r / (1 - e) and r / sqrt(1 - e); their series in e,
// truncated after the quadratic term (a third-order Householder step),
// r (1 + e + e^2) and r (1 + e/2 + 3 e^2 / 8), leave an error of order e^3.
// The seed carries about 20 correct bits (|e| < 2^-19), so e^3 < 2^-57 and
// the result is within about one unit in the last place.  sqrt(x) folds the
// final product: x r (1 + e/2 + 3 e^2 / 8) with x r computed once.
//
// The seed never passes through the FP64 conversion unit (whose
// conversions share the slow FP64 pipe): the FP32 argument is assembled
// with integer operations from the sign, exponent and leading 20 mantissa
// bits of x's high word, and the FP32 result is widened the same way.  The
// seeds are exact for |x| in [2^-125, 2^126); outside that range (and for
// x <= 0 in rsqrt / sqrt) the result is NaN, which the status word reports
// as a non-finite state.

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

// FP32 number with the sign, exponent and first 20 mantissa bits of the
// double whose high word is hi (exponent rebias 1023 -> 127 done modulo 2^32).
__device__ __forceinline__ float narrow_hi(unsigned hi) {
  return __uint_as_float((((hi & 0x7FFFFFFFu) << 3) + 0x40000000u) | (hi & 0x80000000u));
}
// The double equal to the normal FP32 number f.
__device__ __forceinline__ double widen_f32(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned hi = (((b & 0x7FFFFFFFu) >> 3) + 0x38000000u) | (b & 0x80000000u);
  return __hiloint2double((int)hi, (int)(b << 29));
}
// |x| in [2^-125, 2^126) (biased exponent in [898, 1148]), where the FP32
// argument and result (1/x or 1/sqrt(x)) are normal; the sign is ignored
// (abs) or must be positive (pos)
__device__ __forceinline__ bool seed_range_abs(unsigned hi) {
  return ((hi & 0x7FFFFFFFu) - 0x38200000u) < 0x0FB00000u;
}
__device__ __forceinline__ bool seed_range_pos(unsigned hi) { return (hi - 0x38200000u) < 0x0FB00000u; }
__device__ __forceinline__ double nan_f64() { return __longlong_as_double(0x7FF8000000000000ll); }

// Flip the sign of v where m has the (64-bit) sign mask set; integer-only.
__device__ __forceinline__ double flip_sign(double v, unsigned long long m) {
  return __longlong_as_double(__double_as_longlong(v) ^ (long long)m);
}
__device__ __forceinline__ float flip_sign(float v, unsigned long long m) {
  return __uint_as_float(__float_as_uint(v) ^ (unsigned)(m >> 32));
}

// ---------------------------------------------------------------------------
// binary64 multiply on the integer pipes
// ---------------------------------------------------------------------------
// On this GPU the FP64 unit retires about one warp instruction per 16 SM
// cycles, while the integer pipes sit idle in the FP64 kernels.  dmul_int
// computes the IEEE 754 binary64 product, rounded to nearest with ties to
// even, with 32/64-bit integer instructions only.  The kernels use it for
// products that no multiply-add absorbs and that sit among independent work
// (the volume points and the reconstruction), where it runs beside the FP64
// unit.  Its results equal the FP64 unit's bit for bit: the significand
// product is formed exactly, then rounded on the bits below the 53rd, with a
// sticky bit for the rest.  Zero, subnormal, infinite or NaN operands, and
// products outside the normal range, go to the FP64 unit (__dmul_rn), which
// keeps every special case exact.  (An add built the same way was measured
// slower than the FP64 unit's in these kernels and is not used.)

// a * b.  With the significands left-aligned in 64 bits (ma, mb in
// [2^63, 2^64)), the 128-bit product's high word holds the significand
// product in [2^62, 2^64); its top 53 bits are the result's significand, the
// next bit is the rounding bit, and the remaining high bits plus the low word
// form the sticky bit.
__device__ __forceinline__ double dmul_int(double a, double b) {
  const unsigned long long ia = (unsigned long long)__double_as_longlong(a);
  const unsigned long long ib = (unsigned long long)__double_as_longlong(b);
  const int ea = (int)((ia >> 52) & 0x7FF), eb = (int)((ib >> 52) & 0x7FF);
  const int e = ea + eb - 1023;  // biased exponent for a significand product in [1, 2)
  if ((unsigned)(ea - 1) >= 2046u || (unsigned)(eb - 1) >= 2046u || (unsigned)(e - 1) >= 2044u)
    return __dmul_rn(a, b);
  const unsigned long long top_bit = 0x8000000000000000ull;
  const unsigned long long ma = (ia << 11) | top_bit, mb = (ib << 11) | top_bit;
  const unsigned long long hi = __umul64hi(ma, mb), lo = ma * mb;
  const unsigned carry = (unsigned)(hi >> 63);  // significand product in [2, 4)
  const unsigned drop = 10 + carry;               // bits below the 53-bit significand
  unsigned long long m = hi >> drop;
  const unsigned long long rest = hi << (64 - drop);  // dropped bits, left-aligned
  m += (rest > top_bit || (rest == top_bit && (lo != 0 || (m & 1)))) ? 1ull : 0ull;
  // the hidden bit of m adds one to the exponent field (and a rounding carry
  // to 2^53 one more, with a zero fraction)
  return __longlong_as_double((long long)(((ia ^ ib) & top_bit) |
                                          (((unsigned long long)(e + (int)carry - 1) << 52) + m)));
}

// The kernels' choice of multiply: the integer-pipe one in FP64, the plain
// one in FP32.
__device__ __forceinline__ double pmul(double a, double b) { return dmul_int(a, b); }
__device__ __forceinline__ float pmul(float a, float b) { return a * b; }

// Max and |.| of values >= 0 through their bit patterns (non-negative IEEE
// numbers order like their integer patterns; a NaN operand wins): integer
// operations, off the FP64 pipe.
__device__ __forceinline__ double abs_bits(double v) {
  return __longlong_as_double(__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFll);
}
__device__ __forceinline__ float abs_bits(float v) { return __uint_as_float(__float_as_uint(v) & 0x7FFFFFFFu); }
__device__ __forceinline__ double max_nonneg(double a, double b) {
  const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  return __longlong_as_double(ia > ib ? ia : ib);
}
__device__ __forceinline__ float max_nonneg(float a, float b) {
  const int ia = __float_as_int(a), ib = __float_as_int(b);
  return __int_as_float(ia > ib ? ia : ib);
}
// The Rusanov speed of a face: the larger of the two one-sided spectral
// radii (>= 0), where a NaN radius (a trace with rho <= 0 or p <= 0) is
// ignored in favour of the other one, as IEEE maxNum (C fmax) does.  On the
// bit patterns: adding 2^52 - 1 moves the non-negative numbers (up to +inf)
// to [2^52 - 1, 2^63 - 1] and the NaNs past 2^63, where the signed
// comparison ranks them below every number (NaNs with the sign bit set land
// below 2^52 - 1); two NaNs give a NaN.
// (The addition is unsigned, so the wrap-around is defined.)
__device__ __forceinline__ double rusanov_speed(double aL, double aR) {
  const unsigned long long k = 0x000FFFFFFFFFFFFFull;
  const long long l = (long long)((unsigned long long)__double_as_longlong(aL) + k);
  const long long r = (long long)((unsigned long long)__double_as_longlong(aR) + k);
  return l > r ? aL : aR;
}
__device__ __forceinline__ float rusanov_speed(float aL, float aR) {
  const unsigned k = 0x007FFFFFu;
  const int l = (int)(__float_as_uint(aL) + k), r = (int)(__float_as_uint(aR) + k);
  return l > r ? aL : aR;
}
// a < b for a, b >= 0 (a NaN a compares false, as in IEEE), on bit patterns
__device__ __forceinline__ bool less_nonneg(double a, double b) {
  return __double_as_longlong(a) < __double_as_longlong(b);
}
__device__ __forceinline__ bool less_nonneg(float a, float b) { return __float_as_int(a) < __float_as_int(b); }
// x > 0 and x >= 0 for the step sizes (finite or +0 by construction: the
// epilogue stores 0 for a non-finite step), on the bit pattern: integer
// compares, so that the FP32 kernels keep the slow FP64 pipe free.
__device__ __forceinline__ bool pos_bits(double x) { return __double_as_longlong(x) > 0ll; }
__device__ __forceinline__ bool nonneg_bits(double x) { return __double_as_longlong(x) >= 0ll; }
// isnan on the bit pattern (integer compare)
__device__ __forceinline__ bool nan_bits(double v) {
  return (__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFll) > 0x7FF0000000000000ll;
}
__device__ __forceinline__ bool nan_bits(float v) { return (__float_as_int(v) & 0x7FFFFFFF) > 0x7F800000; }
// Add a per-thread count to *counter (nullptr: no counting) with one atomic
// per warp that has a non-zero sum; every lane of the warp must call it.
__device__ __forceinline__ void warp_count_add(unsigned long long* counter, unsigned n) {
  if (counter == nullptr) return;
  const unsigned tot = __reduce_add_sync(0xffffffffu, n);
  if ((threadIdx.x & 31) == 0 && tot != 0u) atomicAdd(counter, (unsigned long long)tot);
}
// isfinite on the exponent field (integer compare instead of an FP64 one)
__device__ __forceinline__ bool finite_bits(double v) {
  return (__double_as_longlong(v) & 0x7FF0000000000000ll) != 0x7FF0000000000000ll;
}
__device__ __forceinline__ bool finite_bits(float v) { return (__float_as_int(v) & 0x7F800000) != 0x7F800000; }

// Min / max of any two non-NaN values through order-preserving integer keys
// (negative patterns have their magnitude bits flipped).
__device__ __forceinline__ long long order_key(double v) {
  const long long b = __double_as_longlong(v);
  return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFll);
}
__device__ __forceinline__ double from_order_key(long long k) {
  return __longlong_as_double(k ^ ((k >> 63) & 0x7FFFFFFFFFFFFFFFll));
}
__device__ __forceinline__ int order_key(float v) {
  const int b = __float_as_int(v);
  return b ^ ((b >> 31) & 0x7FFFFFFF);
}
__device__ __forceinline__ float from_order_key(int k) { return __int_as_float(k ^ ((k >> 31) & 0x7FFFFFFF)); }
template <typename T> __device__ __forceinline__ T min_ordered(T a, T b) {
  const auto ka = order_key(a), kb = order_key(b);
  return from_order_key(ka < kb ? ka : kb);
}
template <typename T> __device__ __forceinline__ T max_ordered(T a, T b) {
  const auto ka = order_key(a), kb = order_key(b);
  return from_order_key(ka > kb ? ka : kb);
}

template <typename T> struct Fast;

template <> struct Fast<double> {
  static __device__ __forceinline__ double rcp(double x) {
    const unsigned hi = (unsigned)__double2hiint(x);
    double r = widen_f32(rcp_approx_f32(narrow_hi(hi)));
    r = seed_range_abs(hi) ? r : nan_f64();
    const double e = fma(-x, r, 1.0);
    return fma(r, fma(e, e, e), r);
  }
  static __device__ __forceinline__ double rsqrt(double x) {
    const unsigned hi = (unsigned)__double2hiint(x);
    double r = widen_f32(rsqrt_approx_f32(narrow_hi(hi)));
    r = seed_range_pos(hi) ? r : nan_f64();
    const double e = fma(-x * r, r, 1.0);
    return fma(r * e, fma(0.375, e, 0.5), r);
  }
  static __device__ __forceinline__ double sqrt_(double x) {
    const unsigned hi = (unsigned)__double2hiint(x);
    double r = widen_f32(rsqrt_approx_f32(narrow_hi(hi)));
    r = seed_range_pos(hi) ? r : nan_f64();
    const double xr = dmul_int(x, r);
    const double e = fma(-xr, r, 1.0);
    return fma(dmul_int(xr, e), fma(0.375, e, 0.5), xr);
  }
  static __device__ __forceinline__ double exp_(double x) { return exp(x); }
};

// FP32: the hardware approximations, one MUFU instruction each (1/x within
// 1 ulp, sqrt within 2^-23 relative), in place of the correctly rounded
// multi-instruction sequences; the FP32 stage kernel is issue bound, and its
// error against the FP64 oracle is dominated by the accumulated rounding of
// the stage arithmetic.  exp(x) = 2^(x log2 e), with the product rounded
// once (relative error about |x| 2^-24 more, for the OE's damping factor).
template <> struct Fast<float> {
  static __device__ __forceinline__ float rcp(float x) { return rcp_approx_f32(x); }
  static __device__ __forceinline__ float rsqrt(float x) { return rsqrt_approx_f32(x); }
  static __device__ __forceinline__ float sqrt_(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
  }
  static __device__ __forceinline__ float exp_(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x * 1.4426950408889634f));
    return r;
  }
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

// Order this thread's earlier generic-proxy accesses of shared memory before
// later async-proxy (TMA) writes to it (a TMA load reusing a buffer).
__device__ __forceinline__ void fence_proxy_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Flags between CTAs of one launch: release store / acquire load at GPU scope.
__device__ __forceinline__ void st_release_gpu(unsigned int* p, unsigned int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
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

// Warp-wide maximum of values >= 0 on their bit patterns (every lane of the
// warp must call it; NaN or negative counts as 0); valid in every lane.
__device__ __forceinline__ double warp_max_nonneg(double v) {
  long long b = __double_as_longlong(v);
  if (!(b > 0 && b <= 0x7FF0000000000000ll)) b = 0;
  for (int o = 16; o > 0; o >>= 1) {
    const long long c = __shfl_xor_sync(0xffffffffu, b, o);
    b = c > b ? c : b;
  }
  return __longlong_as_double(b);
}

// Block-wide maximum of values >= 0 (speeds, |u|, deviations), on their bit
// patterns with integer operations (the FP64 pipe stays free, which matters
// most to the FP32 kernels).  A NaN or negative input counts as 0, as fmax
// over such data would drop a NaN.
template <int NT>
__device__ __forceinline__ double block_max(double v, double* scratch /* >= NT/32 */) {
  long long b = __double_as_longlong(v);
  if (!(b > 0 && b <= 0x7FF0000000000000ll)) b = 0;  // NaN, negative, -0 -> +0 (+inf kept)
  for (int o = 16; o > 0; o >>= 1) {
    const long long c = __shfl_xor_sync(0xffffffffu, b, o);
    b = c > b ? c : b;
  }
  long long* sc = reinterpret_cast<long long*>(scratch);
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  __syncthreads();
  if (l == 0) sc[w] = b;
  __syncthreads();
  if (w == 0) {
    b = (l < NT / 32) ? sc[l] : 0ll;
    for (int o = 16; o > 0; o >>= 1) {
      const long long c = __shfl_xor_sync(0xffffffffu, b, o);
      b = c > b ? c : b;
    }
  }
  return __longlong_as_double(b);  // valid in thread 0
}
// The same on FP32 values (the FP32 kernels' speeds), kept in FP32 so that
// no thread converts to FP64 (a conversion occupies the slow FP64 pipe).
template <int NT>
__device__ __forceinline__ float block_max(float v, double* scratch /* >= NT/64 */) {
  int b = __float_as_int(v);
  if (!(b > 0 && b <= 0x7F800000)) b = 0;  // NaN, negative, -0 -> +0 (+inf kept)
  for (int o = 16; o > 0; o >>= 1) {
    const int c = __shfl_xor_sync(0xffffffffu, b, o);
    b = c > b ? c : b;
  }
  int* sc = reinterpret_cast<int*>(scratch);
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  __syncthreads();
  if (l == 0) sc[w] = b;
  __syncthreads();
  if (w == 0) {
    b = (l < NT / 32) ? sc[l] : 0;
    for (int o = 16; o > 0; o >>= 1) {
      const int c = __shfl_xor_sync(0xffffffffu, b, o);
      b = c > b ? c : b;
    }
  }
  return __int_as_float(b);  // valid in thread 0
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
  // a step whose stages left the admissible set is discarded (the OE wrote
  // nothing): the clock stays, and the retry takes half the step size
  const bool reject = advance_time && ctl->stage_bad != 0u;
  double t = ctl->t;
  if (advance_time && ctl->dt > 0.0 && !reject) t = ctl->final_step ? ctl->T : t + ctl->dt;
  double dt;
  if (reject) {
    ctl->stage_bad = 0u;
    ctl->rejected += 1ull;
    if (++ctl->retry_exp > 30u) ctl->status |= kStatusNonPhysical;
    // the next step's safeguard kernel recomputes the size from U^n's speeds
    dt = ctl->dt > 0.0 ? 0.5 * ctl->dt : 0.0;
  } else {
    if (advance_time) ctl->retry_exp = 0u;
    if (ctl->dim == 1)
      dt = ctl->cfl * ctl->dxe / ax;
    else
      dt = ctl->cfl / (ax / ctl->dxe + ay / ctl->dye);
    if (!(dt > 0.0) || !isfinite(dt)) {
      dt = 0.0;
      ctl->status |= kStatusNonFinite;
    }
    dt = ldexp(dt, -(int)ctl->retry_exp);
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
  if (advance_time && ctl->dt > 0.0 && !reject) ctl->step += 1;
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
