// fam_kernels2d.cuh -- 2D FAM kernels (sm_103a).
//
//  stage2d  one SSP-RK3 stage (eq. 12): TMA-staged tile + halo of the
//           structure-of-arrays moment planes, compact reconstruction of each
//           cell (Sec. 2.4), Rusanov fluxes at the four Gauss points of every
//           face, 4x4 Gauss volume terms, the residual of eq. (11), the
//           Shu--Osher combination and the ghost layers of the output.
//  oe2d     end-of-step OE (eq. 2dOE_sol / 2dOE_system, Tab. sigma2d) on the
//           final stage; averages are copied unchanged.  Fused: the
//           max Rusanov speeds at cell averages for the next time step.
//  alpha2d  the same speed reduction alone (first step).
//
// Thread layout: one thread per cell of a TX x TY tile; the tile's
// surrounding ring of cells computes only the face traces the tile needs.
#pragma once

#include "fam_phys.cuh"
#include "fam_pp.cuh"
#include "fam_recon.cuh"

namespace fam {

template <typename T>
struct Coefs2D {
  T a0, a1, a2;  // Shu--Osher: out = a1 * U0 + a2 * (Us + dt R)   (a0 unused)
};

// Shu--Osher weights of eq. 12, out = w0 * U0 + w1 * (Us + dt R), as
// constants of the kernel's type (no FP64 conversion in the FP32 kernels).
template <typename T>
__device__ __forceinline__ void stage_weights(int stage, T& w0, T& w1) {
  if (stage == 1) { w0 = T(0.0); w1 = T(1.0); }
  else if (stage == 2) { w0 = T(0.75); w1 = T(0.25); }
  else { w0 = T(1.0 / 3.0); w1 = T(2.0 / 3.0); }
}

// Padded positions (and signs) at which interior index i of one direction
// appears: itself and its ghost images for the two sides' conditions
// (Remark in Sec. 2.3: periodic wrap; outflow copies the boundary cell into
// both layers; a reflective wall mirrors the first G cells; inflow and front
// ghosts hold prescribed states and get no image).
__device__ __forceinline__ int ghost_images(int i, int n, int lo, int hi, int sgn_refl, int* pos, int* sgn) {
  int q = 0;
  pos[q] = i + G; sgn[q++] = 1;
  if (lo == kBcPeriodic) {
    if (i < G) { pos[q] = i + G + n; sgn[q++] = 1; }
    if (i >= n - G) { pos[q] = i + G - n; sgn[q++] = 1; }
    return q;
  }
  if (lo == kBcOutflow && i == 0) { pos[q] = 0; sgn[q++] = 1; pos[q] = 1; sgn[q++] = 1; }
  if (lo == kBcReflective && i < G) { pos[q] = G - 1 - i; sgn[q++] = sgn_refl; }
  if (hi == kBcOutflow && i == n - 1) { pos[q] = n + G; sgn[q++] = 1; pos[q] = n + G + 1; sgn[q++] = 1; }
  if (hi == kBcReflective && i >= n - G) { pos[q] = n + G + (n - 1 - i); sgn[q++] = sgn_refl; }
  return q;
}

// Cells at least G away from every side have no ghost image (the common case).
__device__ __forceinline__ bool has_ghost_images(const Geo& g, int j, int i) {
  return i < G || i >= g.nx - G || (g.rows > 1 && (j < G || j >= g.ny - G));
}

// Write v to cell (i, j) of plane p and to every ghost image of that cell.
template <typename T>
__device__ __forceinline__ void store_with_ghosts(T* __restrict__ out, const Geo& g, int p, int j, int i, T v) {
  if (!has_ghost_images(g, j, i)) {
    out[cell_index(g, p, j, i)] = v;
    return;
  }
  int xs[4], xsg[4], ys[4], ysg[4];
  // the split part of a side holds a fixed state (no images there)
  const int bxl = j < g.split[0] ? kBcInflow : g.bc[0], bxr = j < g.split[1] ? kBcInflow : g.bc[1];
  const int byl = i < g.split[2] ? kBcInflow : g.bc[2], byr = i < g.split[3] ? kBcInflow : g.bc[3];
  const int nxs = ghost_images(i, g.nx, bxl, bxr, reflect_sign(g, p, 0), xs, xsg);
  int nys = 1;
  ys[0] = 0;
  ysg[0] = 1;
  if (g.rows > 1) nys = ghost_images(j, g.ny, byl, byr, reflect_sign(g, p, 1), ys, ysg);
  T* base = out + (long long)p * g.plane;
  for (int b = 0; b < nys; ++b)
    for (int a = 0; a < nxs; ++a) base[(long long)ys[b] * g.px + xs[a]] = (xsg[a] * ysg[b] < 0) ? -v : v;
}

// Shared-memory layout of the 2D kernels (in elements of T).
template <typename T, int NC, int TX, int TY>
struct Smem2D {
  static constexpr int NP = NC * 3;
  static constexpr int HX = TX + 4, HY = TY + 4;
  static constexpr int TILE = NP * HY * HX;
  static constexpr int XF = (TX + 1) * TY * 4 * NC;  // x-face slots
  static constexpr int YF = TX * (TY + 1) * 4 * NC;  // y-face slots
  // stage kernel: tile, then U^n rows of the tile (x halo kept for TMA alignment)
  static constexpr int U0OFF = (TILE + 31) / 32 * 32;
  static constexpr int U0T = NP * TY * HX;
  static constexpr size_t bytes_stage =
      sizeof(T) * (size_t)(U0OFF + U0T + 2 * XF + 2 * YF) + 16 + 64 * sizeof(double);
  static constexpr size_t bytes_oe =
      sizeof(T) * (size_t)(TILE + 4 * NC * (TX + 2) * (TY + 2) + 2 * (TX + 2) * (TY + 2)) + 16 + 64 * sizeof(double);
};

// Issue the TMA load of the tile + halo (box (TX+4) x (TY+4) x NP planes at
// padded coordinates (x0, y0, 0)) and wait for it.  Returns false on timeout.
template <typename T, int NP, int HX, int HY>
__device__ __forceinline__ bool load_tile(T* tile, uint64_t* bar, const CUtensorMap* tm, int x0, int y0,
                                          FamCtl* ctl) {
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(bar, (uint32_t)(sizeof(T) * NP * HY * HX));
    tma_load_3d(tile, tm, bar, x0, y0, 0);
  }
  bool ok = mbar_wait(bar, 0);
  if (!ok) {
    atomicOr(&ctl->status, kStatusTimeout);
    note_wait(ctl, kWaitTileCopy, blockIdx.x, blockIdx.y, 0u);
    mbar_wait(bar, 0);  // let an in-flight copy land before the block exits
  }
  return ok;
}

// Gather the 3x3 patch of moments of component c around tile position (hx, hy).
template <typename T, int HX, int HY>
__device__ __forceinline__ void gather_patch(const T* tile, int c, int hx, int hy, T* A, T* X, T* Y) {
  const T* pa = tile + (size_t)(c * 3 + 0) * HY * HX;
  const T* px = tile + (size_t)(c * 3 + 1) * HY * HX;
  const T* py = tile + (size_t)(c * 3 + 2) * HY * HX;
#pragma unroll
  for (int s = 0; s < 9; ++s) {
    const int o = (hy + s / 3 - 1) * HX + (hx + s % 3 - 1);
    A[s] = pa[o];
    X[s] = px[o];
    Y[s] = py[o];
  }
}

// Patch of moments of ring cell r of component c, mirrored / transposed so
// that the trace the ring cell shows the tile is the right-face trace of the
// patch (the rule in stage2d_tile); (rx, ry) receives the ring cell's tile
// position.  Ring cells: rows first (bottom r < TX, top r < 2 TX), then
// columns (left, right).  Rows run the patch's x along the tile's y (x- and
// y-moments swapped), columns along the tile's x; the side only flips the
// direction (and the sign of the new x-moment).  FP32 (COMPILE_TIME_STRIDES)
// takes rows and columns on separate paths, whose offsets from three
// pointers are compile-time constants: its ring tasks are padded so that a
// warp holds rows or columns only.  FP64 takes one path with run-time
// offsets (its warps mix rows and columns).
template <typename T, int TX, int TY, int HX, int HY, bool COMPILE_TIME_STRIDES>
__device__ __forceinline__ void ring_patch(const T* tile, int c, int r, T* A, T* X, T* Y, int& rx, int& ry) {
  constexpr int P = HY * HX;  // plane stride
  constexpr unsigned long long kSign = 0x8000000000000000ull;
  if constexpr (COMPILE_TIME_STRIDES) {
    if (r < 2 * TX) {
      const bool top = r >= TX;
      rx = top ? r - TX : r;
      ry = top ? TY : -1;
      const int s = top ? -HX : HX;  // the patch's x step (along the tile's y)
      const unsigned long long m = top ? kSign : 0ull;
      const T* pa = tile + (size_t)(c * 3) * P + (ry + 2) * HX + (rx + 2);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const T* ra = pa + (a - 1) * s;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          A[b * 3 + a] = ra[b - 1];
          X[b * 3 + a] = flip_sign(ra[(b - 1) + 2 * P], m);
          Y[b * 3 + a] = ra[(b - 1) + P];
        }
      }
    } else {
      const bool right = r >= 2 * TX + TY;
      rx = right ? TX : -1;
      ry = right ? r - 2 * TX - TY : r - 2 * TX;
      const int s = right ? -1 : 1;  // the patch's x step (along the tile's x)
      const unsigned long long m = right ? kSign : 0ull;
      const T* pa = tile + (size_t)(c * 3) * P + (ry + 2) * HX + (rx + 2);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const T* ra = pa + (a - 1) * s;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          A[b * 3 + a] = ra[(b - 1) * HX];
          X[b * 3 + a] = flip_sign(ra[(b - 1) * HX + P], m);
          Y[b * 3 + a] = ra[(b - 1) * HX + 2 * P];
        }
      }
    }
  } else {
    int ox, oy, swap;
    unsigned long long xsign;
    if (r < TX) {
      rx = r; ry = -1; ox = HX; oy = 1; swap = 1; xsign = 0ull;
    } else if (r < 2 * TX) {
      rx = r - TX; ry = TY; ox = -HX; oy = 1; swap = 1; xsign = kSign;
    } else if (r < 2 * TX + TY) {
      rx = -1; ry = r - 2 * TX; ox = 1; oy = HX; swap = 0; xsign = 0ull;
    } else {
      rx = TX; ry = r - 2 * TX - TY; ox = -1; oy = HX; swap = 0; xsign = kSign;
    }
    const int off = (ry + 2) * HX + (rx + 2);
    const T* pa = tile + (size_t)(c * 3 + 0) * P + off;
    const T* px = tile + (size_t)(c * 3 + (swap ? 2 : 1)) * P + off;
    const T* py = tile + (size_t)(c * 3 + (swap ? 1 : 2)) * P + off;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      const int o = (q % 3 - 1) * ox + (q / 3 - 1) * oy;
      A[q] = pa[o];
      X[q] = flip_sign(px[o], xsign);
      Y[q] = py[o];
    }
  }
}

// Ring task -> (ring cell r, component c).  FP32: the row tasks of every
// component first (2 TX per component, a multiple of 32), then the column
// tasks (2 TY per component), so that a warp holds rows or columns only and
// no lane idles.  FP64: component by component.
template <typename T, int TX, int TY, int NC>
struct RingTasks {
  static constexpr int NR = 2 * (TX + TY);
  static constexpr int count = NR * NC;
  static_assert(sizeof(T) != 4 || (2 * TX * NC) % 32 == 0, "FP32 row tasks must fill whole warps");
  __device__ __forceinline__ static void of(int task, int& r, int& c) {
    if constexpr (sizeof(T) == 4) {
      if (task < 2 * TX * NC) {
        c = task / (2 * TX);
        r = task % (2 * TX);
      } else {
        const int q = task - 2 * TX * NC;
        c = q / (2 * TY);
        r = 2 * TX + q % (2 * TY);
      }
    } else {
      c = task / NR;
      r = task % NR;
    }
  }
};

// ---------------------------------------------------------------------------
// stage kernel
// ---------------------------------------------------------------------------
// U^n for phase C from the TMA box in shared memory (single-problem kernel):
// ready() waits (bounded) for the copy started before phase A.
template <typename T, int TX, int TY>
struct U0FromSmem {
  const T* u0s;
  uint64_t* bar;
  FamCtl* ctl;
  bool want;
  uint32_t phase = 0;  // mbarrier phase parity of this copy
  __device__ __forceinline__ bool ready() const {
    if (want && !mbar_wait(bar, phase)) {
      atomicOr(&ctl->status, kStatusTimeout);
      note_wait(ctl, kWaitU0Copy, blockIdx.x, blockIdx.y, phase);
      mbar_wait(bar, phase);  // let an in-flight copy land before the block exits
      return false;
    }
    return true;
  }
  __device__ __forceinline__ T u0(const Geo&, int p, int, int, int ty, int hx) const {
    return u0s[(size_t)p * TY * (TX + 4) + ty * (TX + 4) + hx];
  }
};

// U^n read from global memory at the cell (batched kernel).
template <typename T>
struct U0FromGlobal {
  const T* __restrict__ U0;
  __device__ __forceinline__ bool ready() const { return true; }
  __device__ __forceinline__ T u0(const Geo& g, int p, int j, int i, int, int) const {
    return U0[cell_index(g, p, j, i)];
  }
};

// U^n read at the cell through L2 only (fused final stage + OE: other blocks
// of the launch write neighbouring cells of the same lines with U^{n+1}; this
// tile's own cells are written only by its own OE task, after its stage task).
template <typename T>
struct U0FromL2 {
  const T* U0;
  __device__ __forceinline__ bool ready() const { return true; }
  __device__ __forceinline__ T u0(const Geo& g, int p, int j, int i, int, int) const {
    return __ldcg(U0 + cell_index(g, p, j, i));
  }
};

// One SSP-RK3 stage (stage = 1, 2, 3) or the residual alone (stage = 0) on
// the TX x TY tile at (x0, y0), whose cells and 2-cell halo of every plane
// are in shared memory at `tile` (HY x HX per plane).  xL, xR, yB, yT are the
// face-trace / flux slots of Smem2D.  u0src supplies U^n for stages 2 and 3
// (ready() is called once by every thread before phase C).  ntrace (may be
// null) accumulates the face points of this tile at which a trace has no
// spectral radius; each face of the grid is counted by one tile only.
template <typename T, int K, class PH, int TX, int TY, class U0Src>
__device__ __forceinline__ void stage2d_tile(const T* __restrict__ tile, T* xL, T* xR, T* yB, T* yT,
                                             T* __restrict__ Uout, const Geo& geo, const PH& ph, const int stage,
                                             const T dt, const int x0, const int y0, const U0Src& u0src,
                                             unsigned long long* ntrace, const T idx_, const T idy_,
                                             const T* __restrict__ theta = nullptr,
                                             unsigned int* stage_bad = nullptr) {
  constexpr int NC = PH::NC;
  using S = Smem2D<T, NC, TX, TY>;
  constexpr int HX = S::HX, HY = S::HY;
  constexpr int D = K - 1;
  constexpr int NCOEF = Recon2D<K>::NCOEF;
  constexpr int NT = TX * TY;
  // Face slots, face index fastest ([Gauss point][component][face]), so that
  // neighbouring threads touch neighbouring words (no shared-memory bank
  // conflicts): x-faces (row, col) with col 0..TX, y-faces (row, col) with
  // row 0..TY.  The x-faces col < TX are stored row-major with pitch TX and
  // the last column (col = TX) after them, so that a warp's two rows of a
  // 16-wide tile fill 32 consecutive words.  Within a row the columns are
  // rotated by the row index (col -> (col + row) mod TX): the ring's column
  // 0 of every row then falls in distinct banks, and a row's last column
  // (stored at TX * TY + row, bank row) fills the one bank that its other
  // TX - 1 faces leave free.
  static_assert((TX & (TX - 1)) == 0, "TX must be a power of 2");
  constexpr int NFX = (TX + 1) * TY, NFY = TX * (TY + 1);
  auto XI = [](int row, int col, int g, int c) {
    return (g * NC + c) * NFX + (col < TX ? row * TX + ((col + row) & (TX - 1)) : TX * TY + row);
  };
  auto YI = [](int row, int col, int g, int c) { return (g * NC + c) * NFY + row * TX + col; };

  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int hx = tx + 2, hy = ty + 2;
  const T wg[4] = {T(famgen::kGaussW[0]), T(famgen::kGaussW[1]), T(famgen::kGaussW[2]), T(famgen::kGaussW[3])};

  // the BP/PP safeguard's scaling factors of a cell (1: none); theta holds
  // planes (theta_rho, theta) in the padded layout, filled for cells -1..n
  auto pp_theta = [&](int ci, int cj, T& tr, T& tt) {
    tr = tt = T(1);
    if (theta != nullptr && ci >= -G && ci < geo.nx + G && cj >= -G && cj < geo.ny + G) {
      const long long q = cell_index(geo, 0, cj, ci);
      tr = theta[q];
      tt = theta[geo.plane + q];
    }
  };

  // ---- phase A: reconstruction, volume terms, traces --------------------
  T coef[NC][NCOEF];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    T A[9], X[9], Y[9];
    gather_patch<T, HX, HY>(tile, c, hx, hy, A, X, Y);
    Recon2D<K>::coef(A, X, Y, coef[c]);
  }
  if (theta != nullptr) {
    T tr, tt;
    pp_theta(x0 + tx, y0 + ty, tr, tt);
#pragma unroll
    for (int l = 1; l < NCOEF; ++l) {
      coef[0][l] *= tr;
#pragma unroll
      for (int c = 1; c < NC; ++c) coef[c][l] *= tt;
    }
  }
  T VA[PH::NVA];
#pragma unroll
  for (int q = 0; q < PH::NVA; ++q) VA[q] = T(0);

  // eta pairs: (+inner, -inner) -> Gauss nodes (2, 1); (+outer, -outer) -> (3, 0)
#pragma unroll
  for (int pr = 0; pr < 2; ++pr) {
    T up[NC][4], um[NC][4];  // values at the 4 xi nodes for eta = +node / -node
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      T dp[D + 1], dm[D + 1];
      if (pr == 0) eta_pair<T, D, kRowInner>(coef[c], dp, dm);
      else eta_pair<T, D, kRowOuter>(coef[c], dp, dm);
      const int hp = pr == 0 ? 2 : 3, hm = pr == 0 ? 1 : 0;
      // volume values: xi nodes 2/1 (inner pair), 3/0 (outer pair); traces at xi = +/- 1/2
      sym_pair<T, D, kRowInner>(dp, up[c][2], up[c][1]);
      sym_pair<T, D, kRowOuter>(dp, up[c][3], up[c][0]);
      sym_pair<T, D, kRowInner>(dm, um[c][2], um[c][1]);
      sym_pair<T, D, kRowOuter>(dm, um[c][3], um[c][0]);
      T rp, lp, rm, lm;
      sym_pair<T, D, kRowHalf>(dp, rp, lp);
      sym_pair<T, D, kRowHalf>(dm, rm, lm);
      // this cell's right trace = left side of x-face tx+1; left trace = right side of face tx
      xL[XI(ty, tx + 1, hp, c)] = rp;
      xL[XI(ty, tx + 1, hm, c)] = rm;
      xR[XI(ty, tx, hp, c)] = lp;
      xR[XI(ty, tx, hm, c)] = lm;
    }
    const int hp = pr == 0 ? 2 : 3, hm = pr == 0 ? 1 : 0;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      T u[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) u[c] = up[c][g];
      ph.vol_acc(u, wg[hp] * wg[g], VA);
#pragma unroll
      for (int c = 0; c < NC; ++c) u[c] = um[c][g];
      ph.vol_acc(u, wg[hm] * wg[g], VA);
    }
  }
  // y-face traces: eta = +1/2 (top) and -1/2 (bottom) at the 4 xi nodes
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    T dp[D + 1], dm[D + 1];
    eta_pair<T, D, kRowHalf>(coef[c], dp, dm);
    T t[4], b[4];
    sym_pair<T, D, kRowInner>(dp, t[2], t[1]);
    sym_pair<T, D, kRowOuter>(dp, t[3], t[0]);
    sym_pair<T, D, kRowInner>(dm, b[2], b[1]);
    sym_pair<T, D, kRowOuter>(dm, b[3], b[0]);
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      yB[YI(ty + 1, tx, g, c)] = t[g];
      yT[YI(ty, tx, g, c)] = b[g];
    }
  }
  // Ring cells around the tile: only the trace facing the tile, one task per
  // (ring cell, component).  The reconstruction commutes with the symmetries
  // of the square stencil, so every task evaluates the right-face traces
  // (tr_xp) of a mirrored / transposed patch:
  //   left ring cell   needs tr_xp of u(x, y)               (identity)
  //   right ring cell  needs tr_xm = tr_xp of u(-x, y)       (x-moments change sign)
  //   bottom ring cell needs tr_yp = tr_xp of u(y, x)        (x- and y-moments swap)
  //   top ring cell    needs tr_ym = tr_xp of u(y, -x)       (swap; new x-moment = -old y-moment)
  // with the Gauss points in the same ascending order (the gather:
  // ring_patch).  In FP32 the row tasks of all components come first, then
  // the column tasks (RingTasks): a warp gathers from one ring segment of
  // rows (consecutive words) or from columns (rows HX apart), with
  // compile-time offsets, and no lane idles.
  {
    using RT = RingTasks<T, TX, TY, NC>;
    for (int task = threadIdx.x; task < RT::count; task += NT) {
      int r, c;
      RT::of(task, r, c);
      int rx, ry;
      T A[9], X[9], Y[9], t[4];
      ring_patch<T, TX, TY, HX, HY, sizeof(T) == 4>(tile, c, r, A, X, Y, rx, ry);
      Recon2D<K>::tr_xp(A, X, Y, t);
      if (theta != nullptr) {  // the ring cell's scaled reconstruction: u_bar + theta (t - u_bar)
        T tr, tt;
        pp_theta(x0 + rx, y0 + ry, tr, tt);
        const T th = c == 0 ? tr : tt;
        if (th != T(1)) {  // unscaled traces stay bit-identical to the unlimited path
#pragma unroll
          for (int g = 0; g < 4; ++g) t[g] = fma(th, t[g] - A[4], A[4]);
        }
      }
      // bottom row: its top trace = bottom side of y-face 0; top row: its
      // bottom trace = top side of y-face TY; left column: its right trace =
      // left side of x-face 0; right column: its left trace = right side of
      // x-face TX
      if (r < 2 * TX) {
        T* out = (r < TX ? yB + YI(0, rx, 0, c) : yT + YI(TY, rx, 0, c));
#pragma unroll
        for (int g = 0; g < 4; ++g) out[g * NC * NFY] = t[g];
      } else {
        T* out = (r < 2 * TX + TY ? xL + XI(ry, 0, 0, c) : xR + XI(ry, TX, 0, c));
#pragma unroll
        for (int g = 0; g < 4; ++g) out[g * NC * NFX] = t[g];
      }
    }
  }
  __syncthreads();

  // ---- phase B: Rusanov fluxes at every face Gauss point -----------------
  // Each thread takes the x-face slot and the y-face slot of its own index
  // (slots 0 .. TX*TY - 1 of each family) at the four Gauss points, with
  // compile-time offsets; the last column of x-faces and the last row of
  // y-faces (slots TX*TY ..) follow, one point per thread.
  unsigned nbad = 0;  // owned face points with a trace that has no spectral radius
  // twice the Rusanov flux, f^- + f^+ - alpha (u^+ - u^-), into the slot's
  // left-side entry (the factor 1/2 is folded into the quadrature weights of
  // phase C, exact: a power of 2); true if a trace has no spectral radius
  auto face_point = [&](T* slot, const T* other, const int cs, const bool xdir) -> bool {
    T uL[NC], uR[NC], fL[NC], fR[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) { uL[c] = slot[c * cs]; uR[c] = other[c * cs]; }
    const T sL = xdir ? ph.flux_x(uL, fL) : ph.flux_y(uL, fL);
    const T sR = xdir ? ph.flux_x(uR, fR) : ph.flux_y(uR, fR);
    const T a = rusanov_speed(sL, sR);
#pragma unroll
    for (int c = 0; c < NC; ++c) slot[c * cs] = fma(-a, uR[c] - uL[c], fL[c] + fR[c]);
    return nan_bits(sL) || nan_bits(sR);
  };
  {
    // the face's owner: the tile holding the cell to its right (top), or for
    // the grid's last face the tile to its left (bottom).  x-face slot
    // threadIdx.x is row ty, column (tx - ty) mod TX; y-face slot threadIdx.x
    // is row ty, column tx.
    const int f = threadIdx.x;
    const bool own_x = y0 + ty < geo.ny && x0 + ((tx - ty) & (TX - 1)) <= geo.nx;
    const bool own_y = x0 + tx < geo.nx && y0 + ty <= geo.ny;
#pragma unroll
    for (int g = 0; g < 4; ++g)
      if (face_point(xL + g * NC * NFX + f, xR + g * NC * NFX + f, NFX, true) && own_x) ++nbad;
#pragma unroll
    for (int g = 0; g < 4; ++g)
      if (face_point(yB + g * NC * NFY + f, yT + g * NC * NFY + f, NFY, false) && own_y) ++nbad;
  }
  for (int e = threadIdx.x; e < 4 * (TX + TY); e += NT) {
    if (e < 4 * TY) {  // x-faces of column TX, row r
      const int g = e / TY, r = e % TY, f = TX * TY + r;
      if (face_point(xL + g * NC * NFX + f, xR + g * NC * NFX + f, NFX, true) && y0 + r < geo.ny &&
          x0 + TX == geo.nx)
        ++nbad;
    } else {  // y-faces of row TY, column col
      const int q = e - 4 * TY, g = q / TX, col = q % TX, f = TX * TY + col;
      if (face_point(yB + g * NC * NFY + f, yT + g * NC * NFY + f, NFY, false) && x0 + col < geo.nx &&
          y0 + TY == geo.ny)
        ++nbad;
    }
  }
  warp_count_add(ntrace, nbad);
  __syncthreads();

  // ---- phase C: residual (eq. 11), Shu--Osher combination, store ---------
  const int i = x0 + tx, j = y0 + ty;
  if (!u0src.ready()) return;
  if (i >= geo.nx || j >= geo.ny) return;
  T avg[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) avg[c] = tile[(size_t)(c * 3) * HY * HX + hy * HX + hx];
  T V1[NC], V2[NC];
  ph.vol_finish(VA, avg, V1, V2);
  T w0, w1;
  stage_weights<T>(stage, w0, w1);
  // half weights (the face slots hold twice the flux) and half weight x node
  T hw[4], hwx[4];
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    hw[g] = T(0.5 * famgen::kGaussW[g]);
    hwx[g] = T(0.5 * famgen::kGaussW[g] * famgen::kGaussX[g]);
  }
  T vout[NC];  // this cell's output averages (the safeguard's stage check)
  T vals[NC * 3];  // this cell's output moments, plane by plane
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const T* fl = xL + XI(ty, tx, 0, c);
    const T* fr = xL + XI(ty, tx + 1, 0, c);
    const T* fb = yB + YI(ty, tx, 0, c);
    const T* ft = yB + YI(ty + 1, tx, 0, c);
    T sxl = T(0), sxr = T(0), syb = T(0), syt = T(0), mx = T(0), my = T(0);
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      const T a = fl[g * NC * NFX], b = fr[g * NC * NFX], cb = fb[g * NC * NFY], ct = ft[g * NC * NFY];
      sxl = fma(hw[g], a, sxl);
      sxr = fma(hw[g], b, sxr);
      syb = fma(hw[g], cb, syb);
      syt = fma(hw[g], ct, syt);
      mx = fma(hwx[g], b - a, mx);   // int eta (f_x(+1/2) - f_x(-1/2)) over the x-faces
      my = fma(hwx[g], ct - cb, my);
    }
    T R[3];
    R[0] = -(sxr - sxl) * idx_ - (syt - syb) * idy_;
    R[1] = (V1[c] - T(0.5) * (sxr + sxl)) * idx_ - my * idy_;
    R[2] = (V2[c] - T(0.5) * (syt + syb)) * idy_ - mx * idx_;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const int p = c * 3 + m;
      T v;
      if (stage == 0) {
        v = R[m];
      } else {
        const T us = tile[(size_t)p * HY * HX + hy * HX + hx];
        if (stage == 1) {
          v = us + dt * R[m];
        } else {
          const T u0 = u0src.u0(geo, p, j, i, ty, hx);
          v = w0 * u0 + w1 * (us + dt * R[m]);
        }
      }
      if (m == 0) vout[c] = v;
      vals[p] = v;
    }
  }
  // one test for the cell's ghost images, then the 3 NC plain stores
  if (!has_ghost_images(geo, j, i)) {
    const long long q = cell_index(geo, 0, j, i);
#pragma unroll
    for (int p = 0; p < NC * 3; ++p) Uout[q + p * geo.plane] = vals[p];
  } else {
#pragma unroll
    for (int p = 0; p < NC * 3; ++p) store_with_ghosts(Uout, geo, p, j, i, vals[p]);
  }
  // BP/PP safeguard: a stage output average outside the admissible set
  // discards the step (the OE then writes nothing; see FamCtl::stage_bad)
  if (stage_bad != nullptr && stage != 0 && !ph.admissible(vout)) atomicOr(stage_bad, 1u << stage);
}


// stage = 1, 2, 3: Shu--Osher stage; stage = 0: write the residual R only.
// Resident CTAs per SM the register allocation is bounded for: FP64 needs
// all 255 registers for the 4 x 15 coefficients of a cell (one CTA of 256 or
// two of 128 threads fit); FP32 needs half as many, so 512 threads fit.
template <typename T, int NT>
constexpr int stage_min_blocks() {
  return sizeof(T) == 8 ? 1 : (512 / NT);
}

template <typename T, int K, class PH, int TX, int TY>
__global__ void __launch_bounds__(TX * TY, stage_min_blocks<T, TX * TY>())
    stage2d(const __grid_constant__ CUtensorMap tm_in, const __grid_constant__ CUtensorMap tm_u0,
            T* __restrict__ Uout, const Geo geo, const PH ph, FamCtl* __restrict__ ctl, const int stage,
            const T* __restrict__ theta) {
  constexpr int NC = PH::NC;
  using S = Smem2D<T, NC, TX, TY>;
  constexpr int NP = S::NP, HX = S::HX, HY = S::HY;

  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* tile = reinterpret_cast<T*>(smem_raw);
  T* u0s = tile + S::U0OFF;  // U^n on the tile's rows (stages 2, 3)
  T* xL = u0s + S::U0T;      // left-side trace of x-face, later the flux
  T* xR = xL + S::XF;
  T* yB = xR + S::XF;        // bottom-side trace of y-face, later the flux
  T* yT = yB + S::YF;
  uint64_t* bar = reinterpret_cast<uint64_t*>(yT + S::YF);  // [0] tile, [1] U^n

  // launch constants in T, converted once per block (in the FP32 kernels a
  // conversion from FP64 occupies the slow FP64 pipe)
  __shared__ T cst[3];
  const double dtd = (stage == 0) ? 0.0 : ctl->dt;
  if (stage != 0 && !pos_bits(dtd)) return;  // run finished: keep the state
  // BP/PP safeguard: an earlier stage discarded the step
  if (theta != nullptr && stage >= 2 && ctl->stage_bad != 0u) return;
  if (threadIdx.x == 0) {
    cst[0] = T(dtd);
    cst[1] = T(geo.idx);
    cst[2] = T(geo.idy);
  }

  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const bool want_u0 = stage >= 2;
  if (threadIdx.x == 0) {
    prefetch_tmap(&tm_in);
    mbar_init(bar + 1, 1);
    if (want_u0) {
      prefetch_tmap(&tm_u0);
      fence_mbar_init();
    }
  }
  if (!load_tile<T, NP, HX, HY>(tile, bar, &tm_in, x0, y0, ctl)) return;
  // U^n arrives while phases A and B run (box (TX+4) x TY x NP at padded (x0, y0+G))
  if (want_u0 && threadIdx.x == 0) {
    mbar_expect_tx(bar + 1, (uint32_t)(sizeof(T) * S::U0T));
    tma_load_3d(u0s, &tm_u0, bar + 1, x0, y0 + G, 0);
  }

  const U0FromSmem<T, TX, TY> u0src{u0s, bar + 1, ctl, want_u0};
  // (load_tile's barrier has made cst visible)
  stage2d_tile<T, K, PH, TX, TY>(tile, xL, xR, yB, yT, Uout, geo, ph, stage, cst[0], x0, y0, u0src, &ctl->ntrace,
                                 cst[1], cst[2], theta, theta != nullptr ? &ctl->stage_bad : nullptr);
}

// ---------------------------------------------------------------------------
// OE kernel (+ wave-speed reduction for the next step)
// ---------------------------------------------------------------------------
// The OE step (eq. 2dOE_sol / 2dOE_system, Tab. sigma2d) on the TX x TY tile
// at (x0, y0) whose cells and 2-cell halo are in shared memory at `tile`;
// fc and sp are the face-centre trace and speed scratch of Smem2D.  Type I
// reads its global statistics from t1.  Returns, per thread, the Rusanov
// speeds at its cell's average (0 outside the grid) for the next step size.
template <typename T, int K, class PH, int TX, int TY>
__device__ __forceinline__ void oe2d_tile(const T* __restrict__ tile, T* fc, T* sp, T* __restrict__ Uout,
                                          const Geo& geo, const PH& ph, const int oe_type, const T gamma_k,
                                          const int q6, const T dt_idx, const T dt_idy, const int x0,
                                          const int y0, const FamCtl* t1, unsigned int* status,
                                          T& my_speed_x, T& my_speed_y) {
  constexpr int NC = PH::NC;
  using S = Smem2D<T, NC, TX, TY>;
  constexpr int HX = S::HX, HY = S::HY;
  constexpr int NT = TX * TY;
  constexpr int RX = TX + 2, RY = TY + 2;  // tile plus one ring
  // face-centre trace f (0 x-, 1 x+, 2 y-, 3 y+) of component c at ring
  // position q, position fastest (no shared-memory bank conflicts)
  auto FI = [](int f, int c, int q) { return (f * NC + c) * (RX * RY) + q; };

  // Face-centre traces (Tab. sigma2d jumps need the two traces at each face
  // centre): all four of every tile cell, one task per (cell, component);
  // the one trace each ring cell shows the tile, evaluated as the right-face
  // trace of a mirrored / transposed patch (as in stage2d); the Rusanov
  // speeds at the averages of the tile and its ring (corners included).
  for (int task = threadIdx.x; task < TX * TY * NC; task += NT) {
    const int cell = task % (TX * TY), c = task / (TX * TY);
    const int cx = cell % TX, cy = cell / TX;
    const int q = (cy + 1) * RX + (cx + 1);
    T A[9], X[9], Y[9], t[4];
    gather_patch<T, HX, HY>(tile, c, cx + 2, cy + 2, A, X, Y);
    Recon2D<K>::facec(A, X, Y, t, q6);
#pragma unroll
    for (int f = 0; f < 4; ++f) fc[FI(f, c, q)] = t[f];
  }
  // rows first, then columns; FP32 pads each component's tasks to whole
  // warps, so that a warp holds rows or columns only (the stage's order,
  // RingTasks, left this kernel 16 more bytes of spills at 64 registers)
  constexpr int NR = 2 * (TX + TY);
  constexpr int NRP = sizeof(T) == 4 ? (NR + 31) / 32 * 32 : NR;
  for (int task = threadIdx.x; task < NRP * NC; task += NT) {
    const int r = task % NRP, c = task / NRP;
    if (r >= NR) continue;
    // bottom ring row: its top trace (slot 3); top row: its bottom trace (2);
    // left column: its right trace (1); right column: its left trace (0)
    const int slot = r < TX ? 3 : r < 2 * TX ? 2 : r < 2 * TX + TY ? 1 : 0;
    int rx, ry;
    T A[9], X[9], Y[9], t[4];
    ring_patch<T, TX, TY, HX, HY, sizeof(T) == 4>(tile, c, r, A, X, Y, rx, ry);
    Recon2D<K>::facec(A, X, Y, t, q6);  // only t[1] (x = +1/2) is used
    const int q = (ry + 1) * RX + (rx + 1);
    fc[FI(slot, c, q)] = t[1];
  }
  for (int q = threadIdx.x; q < RX * RY; q += NT) {
    const int hx = q % RX + 1, hy = q / RX + 1;
    T u[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) u[c] = tile[(size_t)(c * 3) * HY * HX + hy * HX + hx];
    T sx, sy;
    ph.speeds(u, sx, sy);
    sp[q] = sx;
    sp[RX * RY + q] = sy;
  }
  // Type I: the grid statistics D and eps per component, converted to T once
  // per block (no per-cell conversion on the FP64 pipe)
  __shared__ T t1s[2 * NC];
  if (oe_type == 1 && t1 != nullptr && threadIdx.x < NC) {
    const int c = threadIdx.x;
    t1s[c] = T(__longlong_as_double((long long)t1->t1_dev_bits[c]));
    t1s[NC + c] = T(1e-14) * max_nonneg(T(__longlong_as_double((long long)t1->t1_maxabs_bits[c])), T(1));
  }
  __syncthreads();

  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int i = x0 + tx, j = y0 + ty;
  const bool inside = i < geo.nx && j < geo.ny;
  my_speed_x = T(0);
  my_speed_y = T(0);
  if (inside) {
    const int rx = tx + 1, ry = ty + 1, q = ry * RX + rx;
    const int hx = tx + 2, hy = ty + 2;
    T sig_x = T(0), sig_y = T(0);
    bool ok = true;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      // jumps [[u]] = u(right/top side) - u(left/bottom side) at the four face centres
      const T jxl = fc[FI(0, c, q)] - fc[FI(1, c, q - 1)];
      const T jxr = fc[FI(0, c, q + 1)] - fc[FI(1, c, q)];
      const T jyb = fc[FI(2, c, q)] - fc[FI(3, c, q - RX)];
      const T jyt = fc[FI(2, c, q + RX)] - fc[FI(3, c, q)];
      // Type II over the 3x3 stencil: S = sum of the averages (unnormalised,
      // as printed), D = max |u_s - S| = max(S - min u, max u - S) (rounding
      // is monotone, so this equals the max of the nine rounded differences)
      const T* pa = tile + (size_t)(c * 3) * HY * HX;
      T S = T(0), vmin, vmax;
#pragma unroll
      for (int s = 0; s < 9; ++s) {
        const T v = pa[(hy + s / 3 - 1) * HX + (hx + s % 3 - 1)];
        S += v;
        vmin = s == 0 ? v : min_ordered(vmin, v);
        vmax = s == 0 ? v : max_ordered(vmax, v);
      }
      T Dn = T(0), eps;
      if (oe_type == 1) {
        Dn = t1s[c];
        eps = t1s[NC + c];
      } else {
        Dn = max_nonneg(S - vmin, vmax - S);  // one of the two is >= 0
        eps = pmul(T(1e-14), max_nonneg(max_nonneg(abs_bits(vmin), abs_bits(vmax)), T(1)));
      }
      if (oe_type != 0 && !less_nonneg(Dn, eps)) {
        const T g = pmul(gamma_k, Fast<T>::rcp(Dn));
        sig_x = max_nonneg(sig_x, pmul(g, fabs(jxl) + fabs(jxr)));
        sig_y = max_nonneg(sig_y, pmul(g, fabs(jyb) + fabs(jyt)));
      }
    }
    T bx = T(0), by = T(0);
#pragma unroll
    for (int s = 0; s < 9; ++s) {
      const int qq = (ry + s / 3 - 1) * RX + (rx + s % 3 - 1);
      bx = max_nonneg(bx, sp[qq]);
      by = max_nonneg(by, sp[RX * RY + qq]);
    }
    // (products on the integer pipes: pmul, bit-identical to the FP64 unit's)
    const T theta = fma(pmul(bx, sig_x), dt_idx, pmul(pmul(by, sig_y), dt_idy));
    const T delta = Fast<T>::exp_(-theta);
    T uavg[NC], vals[NC * 3];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const T a = tile[(size_t)(c * 3) * HY * HX + hy * HX + hx];
      uavg[c] = a;
      const T m1 = pmul(tile[(size_t)(c * 3 + 1) * HY * HX + hy * HX + hx], delta);
      const T m2 = pmul(tile[(size_t)(c * 3 + 2) * HY * HX + hy * HX + hx], delta);
      if (!finite_bits(a) || !finite_bits(m1) || !finite_bits(m2)) ok = false;
      vals[c * 3 + 0] = a;
      vals[c * 3 + 1] = m1;
      vals[c * 3 + 2] = m2;
    }
    if (!has_ghost_images(geo, j, i)) {
      const long long qc = cell_index(geo, 0, j, i);
#pragma unroll
      for (int p = 0; p < NC * 3; ++p) Uout[qc + p * geo.plane] = vals[p];
    } else {
#pragma unroll
      for (int p = 0; p < NC * 3; ++p) store_with_ghosts(Uout, geo, p, j, i, vals[p]);
    }
    if (!ok) atomicOr(status, kStatusNonFinite);
    else if (!ph.admissible(uavg)) atomicOr(status, kStatusNonPhysical);
    my_speed_x = sp[q];
    my_speed_y = sp[RX * RY + q];
  }
}

// Resident CTAs per SM of the OE kernel: FP32 keeps its registers at 64 so
// that 32 warps fit (8 CTAs of 128 threads, 4 of 256; 12 bytes spill).  At
// 24 warps the 4096^2 FAM5 OE took 1.06 ms, at 32 warps 0.90 ms; at 40
// warps (48 registers) it would spill 60-72 bytes.
template <typename T, int NT>
constexpr int oe_min_blocks() {
  return sizeof(T) == 8 ? 1 : (1024 / NT);
}

template <typename T, int K, class PH, int TX, int TY>
__global__ void __launch_bounds__(TX * TY, oe_min_blocks<T, TX * TY>())
    oe2d(const __grid_constant__ CUtensorMap tm_in, T* __restrict__ Uout, const Geo geo, const PH ph,
         FamCtl* __restrict__ ctl, const int oe_type, const T gamma_k, const int q6, const double dt_override) {
  constexpr int NC = PH::NC;
  using S = Smem2D<T, NC, TX, TY>;
  constexpr int NP = S::NP, HX = S::HX, HY = S::HY;
  constexpr int NT = TX * TY;
  constexpr int RX = TX + 2, RY = TY + 2;  // tile plus one ring

  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* tile = reinterpret_cast<T*>(smem_raw);
  T* fc = tile + S::TILE;            // face-centre traces [4][NC][RY * RX]
  T* sp = fc + 4 * NC * RX * RY;     // speeds at averages [2][RY][RX]
  uint64_t* bar = reinterpret_cast<uint64_t*>(sp + 2 * RX * RY);
  double* red = reinterpret_cast<double*>(bar + 2);

  const bool reduce = !nonneg_bits(dt_override);
  const double dtd = reduce ? ctl->dt : dt_override;
  if (!pos_bits(dtd) && reduce) return;
  if (reduce && ctl->stage_bad != 0u) {  // the step is discarded: U^n stays in Uout
    if (threadIdx.x == 0) step_epilogue(ctl, gridDim.x * gridDim.y, true);
    return;
  }
  __shared__ T cst[2];  // dt/dx, dt/dy in T, once per block
  if (threadIdx.x == 0) {
    cst[0] = T(dtd * geo.idx);
    cst[1] = T(dtd * geo.idy);
  }

  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  if (threadIdx.x == 0) prefetch_tmap(&tm_in);
  if (!load_tile<T, NP, HX, HY>(tile, bar, &tm_in, x0, y0, ctl)) return;

  T my_speed_x, my_speed_y;
  oe2d_tile<T, K, PH, TX, TY>(tile, fc, sp, Uout, geo, ph, oe_type, gamma_k, q6, cst[0], cst[1], x0, y0, ctl,
                              &ctl->status, my_speed_x, my_speed_y);
  if (!reduce) return;
  const T mx = block_max<NT>(my_speed_x, red);
  const T my = block_max<NT>(my_speed_y, red + 32);
  if (threadIdx.x == 0) {
    atomic_max_nonneg(&ctl->alpha_bits[0], (double)mx);
    atomic_max_nonneg(&ctl->alpha_bits[1], (double)my);
    step_epilogue(ctl, gridDim.x * gridDim.y, true);
  }
}

// ---------------------------------------------------------------------------
// final stage and OE fused into one persistent launch
// ---------------------------------------------------------------------------
// The OE of a tile (eq. 2dOE_sol) reads the final stage's output on the tile
// and its 2-cell halo.  Instead of recomputing that stage on the halo (a
// 1.5-1.8x larger stage for the tile shapes that fit), one launch walks a
// task list: "stage" tasks run the final RK stage of a tile (stage2d_tile),
// publish its output W and raise the tile's flag; "OE" tasks wait for the
// flags of the tiles that wrote their halo, then run the OE of their tile
// (oe2d_tile) from W, which is still in L2.  Both task kinds stage their tile
// with L2-only vector loads (no TMA or mbarrier in this kernel).  The host orders the list so
// that every OE task comes after the stage tasks it waits for; blocks take
// tasks in list order from a ticket counter, so a waiting block only ever
// waits for tasks already taken by running blocks (no deadlock, whatever the
// grid size).  Every wait is bounded (kWaitLimitNs); a block that gives up
// records kStatusTimeout, which makes the others stop taking tasks.

// The interior cell whose value (or ghost image, written by the stage
// kernels' store_with_ghosts) is found at cell c of a direction with n cells
// and side conditions lo / hi; -1 for an inflow ghost (a fixed value).
__host__ __device__ inline int halo_source(int c, int n, int lo, int hi) {
  if (c >= 0 && c < n) return c;
  if (c < 0) {
    if (lo == kBcPeriodic) return c + n;
    if (lo == kBcOutflow) return 0;
    if (lo == kBcReflective) return -1 - c;
    return -1;
  }
  if (hi == kBcPeriodic) return c - n;
  if (hi == kBcOutflow) return n - 1;
  if (hi == kBcReflective) return 2 * n - 1 - c;
  return -1;
}

// Tile indices (along one direction, tiles of width TW) whose cells are read
// by the OE of tile t through its 2-cell halo; returns how many (<= 5).
__host__ __device__ inline int halo_tiles(int t, int TW, int n, int lo, int hi, int* out) {
  int m = 0;
  out[m++] = t;
  const int x0 = t * TW, xe = (x0 + TW < n) ? x0 + TW : n;
  const int cs[4] = {x0 - 2, x0 - 1, xe, xe + 1};
  for (int q = 0; q < 4; ++q) {
    const int src = halo_source(cs[q], n, lo, hi);
    if (src < 0) continue;
    const int o = src / TW;
    bool seen = false;
    for (int r = 0; r < m; ++r) seen = seen || out[r] == o;
    if (!seen) out[m++] = o;
  }
  return m;
}

// Load the tile + halo box ((TX+4) x (TY+4) x NP at padded (x0, y0)) of W
// with 16-byte vector loads; outside the padded planes: 0.  L2ONLY: through
// L2 only (W was written by other blocks of the same launch, so no line of it
// may come from this SM's L1).  Needs 16-byte aligned rows (padded pitch a
// multiple of 4 elements, x0 a multiple of 4 / 2 elements in FP32 / FP64).
template <typename T, int NP, int TX, int TY, int NT, bool L2ONLY = true>
__device__ __forceinline__ void load_tile_l2(T* tile, const T* __restrict__ W, const Geo& g, int x0, int y0) {
  constexpr int HX = TX + 4, HY = TY + 4;
  constexpr int VW = 16 / (int)sizeof(T);  // elements per 16-byte vector
  constexpr int VR = HX / VW;              // vectors per row
  static_assert(HX % VW == 0, "tile rows hold whole vectors");
  for (int q = threadIdx.x; q < NP * HY * VR; q += NT) {
    const int p = q / (HY * VR), r = q - p * (HY * VR);
    const int y = y0 + r / VR, xv = x0 + (r % VR) * VW;
    T* dst = tile + (size_t)p * HY * HX + (size_t)(r / VR) * HX + (r % VR) * VW;
    // px is a multiple of 4 elements and xv of VW, so a vector is all in or all out
    if (y < g.rows && xv < g.px) {
      const T* src = W + (long long)p * g.plane + (long long)y * g.px + xv;
      if constexpr (sizeof(T) == 8) {
        const double2* s2 = reinterpret_cast<const double2*>(src);
        const double2 v = L2ONLY ? __ldcg(s2) : __ldg(s2);
        dst[0] = v.x;
        dst[1] = v.y;
      } else {
        const float4* s4 = reinterpret_cast<const float4*>(src);
        const float4 v = L2ONLY ? __ldcg(s4) : __ldg(s4);
        dst[0] = v.x;
        dst[1] = v.y;
        dst[2] = v.z;
        dst[3] = v.w;
      }
    } else {
#pragma unroll
      for (int e = 0; e < VW; ++e) dst[e] = T(0);
    }
  }
}

// The same through L1 (read-only data of the launch: the batch's stage input).
template <typename T, int NP, int TX, int TY, int NT>
__device__ __forceinline__ void load_tile_vec(T* tile, const T* __restrict__ W, const Geo& g, int x0, int y0) {
  load_tile_l2<T, NP, TX, TY, NT, false>(tile, W, g, x0, y0);
}

template <typename T, int NC, int TX, int TY>
struct SmemFused {
  using S = Smem2D<T, NC, TX, TY>;
  static constexpr size_t bytes = S::bytes_stage > S::bytes_oe ? S::bytes_stage : S::bytes_oe;
};

template <typename T, int K, class PH, int TX, int TY>
__global__ void __launch_bounds__(TX * TY, stage_min_blocks<T, TX * TY>())
    stage3_oe2d(const T* __restrict__ Win, const T* U0, T* __restrict__ W, T* Uout, const Geo geo, const PH ph,
                FamCtl* __restrict__ ctl,
                const int oe_type, const T gamma_k, const int q6, const int* __restrict__ tasks, const int ntasks,
                unsigned int* __restrict__ tsync /* [0] ticket, [1 + t] flag of tile t */) {
  constexpr int NC = PH::NC;
  using S = Smem2D<T, NC, TX, TY>;
  constexpr int NP = S::NP, HX = S::HX, HY = S::HY;
  constexpr int NT = TX * TY;
  constexpr int RX = TX + 2, RY = TY + 2;

  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* tile = reinterpret_cast<T*>(smem_raw);
  // stage-task layout (as stage2d; U^n comes from L2 at the cell)
  T* xL = tile + S::U0OFF + S::U0T;
  T* xR = xL + S::XF;
  T* yB = xR + S::XF;
  T* yT = yB + S::YF;
  // OE-task layout (as oe2d)
  T* fc = tile + S::TILE;
  T* sp = fc + 4 * NC * RX * RY;
  __shared__ double red[64];
  __shared__ int task_s, ok_s;

  const double dtd = ctl->dt;
  if (!pos_bits(dtd)) return;  // run finished: keep the state (no block reaches the epilogue)
  __shared__ T cst[5];  // dt, 1/dx, 1/dy, dt/dx, dt/dy in T, once per block
  if (threadIdx.x == 0) {
    cst[0] = T(dtd);
    cst[1] = T(geo.idx);
    cst[2] = T(geo.idy);
    cst[3] = T(dtd * geo.idx);
    cst[4] = T(dtd * geo.idy);
  }
  const int ntx = (geo.nx + TX - 1) / TX, nty = (geo.ny + TY - 1) / TY;
  const int ntiles = ntx * nty;
  unsigned int* ticket = tsync;
  unsigned int* flag = tsync + 1;
  volatile unsigned int* vstatus = &ctl->status;

  for (;;) {
    __syncthreads();  // the previous task is done with shared memory
    if (threadIdx.x == 0) {
      int tk = -1;
      if ((*vstatus & kStatusTimeout) == 0u) {
        const unsigned int q = atomicAdd(ticket, 1u);
        if (q < (unsigned int)ntasks) tk = tasks[q];
      }
      task_s = tk;
    }
    __syncthreads();
    const int task = task_s;
    if (task < 0) break;
    if (task < ntiles) {
      // ---- final RK stage of tile `task` -> W ----
      const int x0 = (task % ntx) * TX, y0 = (task / ntx) * TY;
      load_tile_l2<T, NP, TX, TY, NT>(tile, Win, geo, x0, y0);
      __syncthreads();
      const U0FromL2<T> u0src{U0};
      stage2d_tile<T, K, PH, TX, TY>(tile, xL, xR, yB, yT, W, geo, ph, 3, cst[0], x0, y0, u0src, &ctl->ntrace,
                                     cst[1], cst[2]);
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) st_release_gpu(&flag[task], 1u);
    } else {
      // ---- OE of tile `task - ntiles` from W -> Uout ----
      const int t = task - ntiles;
      const int tx_ = t % ntx, ty_ = t / ntx;
      const int x0 = tx_ * TX, y0 = ty_ * TY;
      if (threadIdx.x == 0) {
        int cx[5], cy[5];
        const int mx = halo_tiles(tx_, TX, geo.nx, geo.bc[0], geo.bc[1], cx);
        const int my = halo_tiles(ty_, TY, geo.ny, geo.bc[2], geo.bc[3], cy);
        bool ok = true;
        const unsigned long long t0 = global_ns();
        for (int b = 0; b < my && ok; ++b)
          for (int a = 0; a < mx && ok; ++a) {
            const unsigned int* f = &flag[cy[b] * ntx + cx[a]];
            while (ld_acquire_gpu(f) == 0u) {
              if ((*vstatus & kStatusTimeout) != 0u) {  // another block gave up first
                ok = false;
                break;
              }
              if (global_ns() - t0 > kWaitLimitNs) {
                ok = false;
                note_wait(ctl, kWaitTileFlag, (unsigned int)t, (unsigned int)(cy[b] * ntx + cx[a]), 0u);
                break;
              }
              __nanosleep(100);
            }
          }
        if (!ok) atomicOr(&ctl->status, kStatusTimeout);
        ok_s = ok;
      }
      __syncthreads();
      if (!ok_s) break;
      load_tile_l2<T, NP, TX, TY, NT>(tile, W, geo, x0, y0);
      __syncthreads();
      T msx, msy;
      oe2d_tile<T, K, PH, TX, TY>(tile, fc, sp, Uout, geo, ph, oe_type, gamma_k, q6, cst[3], cst[4], x0, y0, ctl,
                                  &ctl->status, msx, msy);
      const T mx = block_max<NT>(msx, red);
      const T my = block_max<NT>(msy, red + 32);
      if (threadIdx.x == 0) {
        atomic_max_nonneg(&ctl->alpha_bits[0], (double)mx);
        atomic_max_nonneg(&ctl->alpha_bits[1], (double)my);
      }
    }
  }
  if (threadIdx.x == 0) step_epilogue(ctl, gridDim.x, true);
}

// BP/PP safeguard (Euler, fam_pp.cuh): the scaling factors of the limited
// reconstruction of every cell -1..nx x -1..ny of U into theta (planes
// theta_rho, theta; padded layout), and with want_dt the largest spectral
// radii at the check points of the interior cells -> ctl->dt (no time
// advance).
// FP32 is held to 128 registers (8 blocks of 64 per SM): its common path
// (coefficients, deviation bounds, screen) needs far fewer, and the rare
// point passes may spill; FP64 keeps one block's worth of registers free.
template <typename T, int NT>
constexpr int pp_min_blocks() {
  return sizeof(T) == 4 ? 512 / NT : 1;
}

template <typename T, int K, class PH, int NT>
__global__ void __launch_bounds__(NT, pp_min_blocks<T, NT>()) pp_theta2d(const T* __restrict__ U, T* __restrict__ theta, const Geo geo,
                                                  const PH ph, FamCtl* __restrict__ ctl, const int want_dt) {
  constexpr int NC = PH::NC;
  constexpr int NCOEF = Recon2D<K>::NCOEF;
  static_assert(NC * NCOEF * NT * sizeof(T) <= 48 * 1024, "coefficient slots exceed static shared memory");
  __shared__ double red[64];
  __shared__ T cslot[NC * NCOEF * NT];  // this thread's coefficients, lane fastest
  T mx = T(0), my = T(0);
  const int wx = geo.nx + 2, wy = geo.ny + 2;
  const long long n = (long long)wx * wy;
  // the loop bound is uniform over the block, so every lane of a warp takes
  // part in the warp maxima below
  for (long long q0 = blockIdx.x * (long long)NT; q0 < n; q0 += (long long)gridDim.x * NT) {
    const long long q = q0 + threadIdx.x;
    double px = 0.0, py = 0.0;  // this cell's speed maxima, published for the screen of later cells
    double seen_x = 0.0, seen_y = 0.0;  // the grid maxima this thread read
    if (q < n) {
      // (32-bit division whenever the cell count allows it: the branch is
      // uniform over the launch)
      int i, j;
      if (n <= 0xffffffffll) {
        const unsigned int uq = (unsigned int)q, uj = uq / (unsigned int)wx;
        j = (int)uj - 1;
        i = (int)(uq - uj * (unsigned int)wx) - 1;
      } else {
        j = (int)(q / wx) - 1;
        i = (int)(q - (long long)(j + 1) * wx) - 1;
      }
      // the 3x3 patch: one 64-bit plane base per plane, 32-bit offsets
      // within it (rows of the padded layout)
      const T* centre = U + cell_index(geo, 0, j, i);
      const int pitch = geo.px;
      // coefficients: deviation bounds and the average here; a copy in this
      // thread's shared-memory slot for the cells whose points are needed
      T avg[NC], d[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        T A[9], X[9], Y[9], cf[NCOEF];
        const T* pa = centre + (long long)(c * 3) * geo.plane;
        const T* pmx = pa + geo.plane;
        const T* pmy = pmx + geo.plane;
#pragma unroll
        for (int s9 = 0; s9 < 9; ++s9) {
          const int o = (s9 / 3 - 1) * pitch + (s9 % 3 - 1);
          A[s9] = pa[o];
          X[s9] = pmx[o];
          Y[s9] = pmy[o];
        }
        Recon2D<K>::coef(A, X, Y, cf);
        avg[c] = cf[0];
        d[c] = pp_dev_bound_2d<T, K>(cf);
#pragma unroll
        for (int l = 0; l < NCOEF; ++l) cslot[(c * NCOEF + l) * NT + threadIdx.x] = cf[l];
      }
      const bool interior = i >= 0 && i < geo.nx && j >= 0 && j < geo.ny;
      const bool speeds = want_dt && interior;
      T run_x = T(0), run_y = T(0);
      if (speeds) {  // maxima reached so far (exact values of T, so the conversion is exact)
        seen_x = __longlong_as_double((long long)__ldcg(&ctl->alpha_bits[0]));
        seen_y = __longlong_as_double((long long)__ldcg(&ctl->alpha_bits[1]));
        run_x = T(seen_x);
        run_y = T(seen_y);
      }
      T tr, tt, sx = T(0), sy = T(0);
      const auto cf = [&](int c) { return SlotRef<T, NT>{cslot + c * NCOEF * NT + threadIdx.x}; };
      pp_cell_2d<T, K, PH>(avg, d, cf, ph, tr, tt, speeds, run_x, run_y, sx, sy);
      const long long o = cell_index(geo, 0, j, i);
      theta[o] = tr;
      theta[geo.plane + o] = tt;
      if (speeds) {
        mx = max_nonneg(mx, sx);
        my = max_nonneg(my, sy);
        px = (double)sx;
        py = (double)sy;
      }
    }
    if (want_dt) {
      // publish only what raises the maxima this warp last read (after the
      // first blocks, almost no warp does: no contention on the two words)
      px = warp_max_nonneg(px);
      py = warp_max_nonneg(py);
      if ((threadIdx.x & 31) == 0) {
        if (px > seen_x) atomic_max_nonneg(&ctl->alpha_bits[0], px);
        if (py > seen_y) atomic_max_nonneg(&ctl->alpha_bits[1], py);
      }
    }
  }
  if (!want_dt) return;  // uniform: no block reduction
  const T bx = block_max<NT>(mx, red);
  const T by = block_max<NT>(my, red + 32);
  if (threadIdx.x == 0) {
    atomic_max_nonneg(&ctl->alpha_bits[0], (double)bx);
    atomic_max_nonneg(&ctl->alpha_bits[1], (double)by);
    step_epilogue(ctl, gridDim.x, false);
  }
}

// Max Rusanov speeds at cell averages -> ctl->dt (no time advance).
template <typename T, class PH, int NT>
__global__ void __launch_bounds__(NT) alpha2d(const T* __restrict__ U, const Geo geo, const PH ph,
                                              FamCtl* __restrict__ ctl) {
  __shared__ double red[64];
  double mx = 0.0, my = 0.0;
  const long long n = (long long)geo.nx * geo.ny;
  for (long long q = blockIdx.x * (long long)NT + threadIdx.x; q < n; q += (long long)gridDim.x * NT) {
    const int i = (int)(q % geo.nx), j = (int)(q / geo.nx);
    T u[PH::NC];
#pragma unroll
    for (int c = 0; c < PH::NC; ++c) u[c] = U[cell_index(geo, c * 3, j, i)];
    T sx, sy;
    ph.speeds(u, sx, sy);
    mx = fmax(mx, (double)sx);
    my = fmax(my, (double)sy);
  }
  mx = block_max<NT>(mx, red);
  my = block_max<NT>(my, red + 32);
  if (threadIdx.x == 0) {
    atomic_max_nonneg(&ctl->alpha_bits[0], mx);
    atomic_max_nonneg(&ctl->alpha_bits[1], my);
    step_epilogue(ctl, gridDim.x, false);
  }
}

}  // namespace fam
