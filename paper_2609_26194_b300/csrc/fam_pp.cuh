// fam_pp.cuh -- optional BP/PP safeguard of the FAM stage (Euler).
//
// The paper applies a bound/positivity-preserving limiter after RK substeps
// in the tests that name it, separately from OE (Sec. 2.3 remarks, Alg. 1),
// and takes it from its references without defining it.  This file builds
// the Zhang--Shu construction those references refine: each stage's
// reconstruction of a cell is scaled towards the cell average,
//     p~ = u_bar + theta (p - u_bar),
// density first (theta_rho), then all components (theta), so that the
// density and the pressure are at least eps at every check point:
//   1D  the Gauss--Lobatto nodes of a rule exact on P_{k-1} (3 for k <= 4,
//       4 for k = 5, 6: x = +-1/2, 0 or +-1/2, +-1/(2 sqrt 5)) and the 4
//       Gauss nodes of the volume integral;
//   2D  Lobatto x Gauss, Gauss x Lobatto and Gauss x Gauss points.
// The cell average is a convex combination of the Lobatto x Gauss values
// (and of the Gauss x Lobatto ones), so a forward-Euler step of the averages
// with the Rusanov flux stays admissible when
// (dt/dx) a_x + (dt/dy) a_y <= w_L (1/6 or 1/12), with a the largest
// spectral radius at the check points of the limited reconstructions: with
// the safeguard on, the CFL rule takes its speeds there.
// Targets relative to the cell: density 1e-6 rho_bar and pressure 1e-8
// p_bar in FP64, 1e-4 of each in FP32.  At a point scaled towards vacuum the
// computed density has a relative rounding error of ~u / (density target)
// (u the unit roundoff), which m^2 / (2 rho) carries into the pressure, so
// the product of the two targets must exceed ~u E / p_bar.  The basis has P_0 = 1 and zero-mean higher
// functions, so coefficient 0 is the average and scaling the others scales
// p - u_bar.
#pragma once

#include <type_traits>

#include "fam_recon.cuh"

namespace fam {

template <typename T> struct PPEps;
template <> struct PPEps<double> {
  static __device__ __forceinline__ double rho(double rb) { return 1e-6 * rb; }
  static __device__ __forceinline__ double p_frac() { return 1e-8; }
  // relative margin of the screen's bounds for the rounding of point values
  static __device__ __forceinline__ double tol() { return 1e-12; }
};
// FP32: rho_bar + theta (rho - rho_bar) carries a rounding error of order
// 1e-7 rho_bar
template <> struct PPEps<float> {
  static __device__ __forceinline__ float rho(float rb) { return 1e-4f * rb; }
  static __device__ __forceinline__ float p_frac() { return 1e-4f; }
  static __device__ __forceinline__ float tol() { return 2e-5f; }
};

// Bound of |p(x) - u_bar| over the cell for one component, from its
// coefficients: sum over l >= 1 of |c_l| max|phi_l|.  A monic Legendre
// polynomial on [-1/2, 1/2] is largest in modulus at the ends, so
// max|P_a| = P_a(1/2) (> 0) and max|P_a P_b| <= P_a(1/2) P_b(1/2).
template <typename T, int K>
__device__ __forceinline__ T pp_dev_bound_1d(const T* c) {
  T d = T(0);
#pragma unroll
  for (int a = 1; a < K; ++a) d = fma(fabs(c[a]), T(famgen::kLegAt[kRowHalf][a]), d);
  return d;
}
template <typename T, int K>
__device__ __forceinline__ T pp_dev_bound_2d(const T* c) {
  T d = T(0);
#pragma unroll
  for (int sdeg = 1; sdeg < K; ++sdeg)
#pragma unroll
    for (int a = 0; a <= sdeg; ++a)
      d = fma(fabs(c[cidx(a, sdeg - a)]),
              T(famgen::kLegAt[kRowHalf][a] * famgen::kLegAt[kRowHalf][sdeg - a]), d);
  return d;
}

// Row of the interior Lobatto node(s) for order K
template <int K> struct LobRow {
  static constexpr int row = K <= 4 ? kRowZero : kRowLobatto;
};

// Pressure of an Euler state with NC components (1D: 3, 2D: 4)
template <typename T, int NC>
__device__ __forceinline__ T pp_pressure(T gm1, const T* u) {
  T m2 = u[1] * u[1];
  if (NC == 4) m2 = fma(u[2], u[2], m2);
  return gm1 * (u[NC - 1] - T(0.5) * m2 * Fast<T>::rcp(u[0]));
}

// The t in (0, 1) with p(ub + t dw) = eps, given p(ub) > eps > p(ub + dw):
// the root of rho(t) (E(t) - eps/(gamma-1)) - |m(t)|^2 / 2, a quadratic
// a t^2 + b t + c with c > 0 > a + b + c.
template <typename T, int NC>
__device__ __forceinline__ T pp_pressure_root(T gm1, const T* ub, const T* dw, T eps) {
  const T Eh = ub[NC - 1] - eps * Fast<T>::rcp(gm1);
  T dm2 = dw[1] * dw[1], mdm = ub[1] * dw[1], m2 = ub[1] * ub[1];
  if (NC == 4) {
    dm2 = fma(dw[2], dw[2], dm2);
    mdm = fma(ub[2], dw[2], mdm);
    m2 = fma(ub[2], ub[2], m2);
  }
  const T a = dw[NC - 1] * dw[0] - T(0.5) * dm2;
  const T b = Eh * dw[0] + ub[0] * dw[NC - 1] - mdm;
  const T c = Eh * ub[0] - T(0.5) * m2;
  if (fabs(a) < T(1e-14) * (fabs(b) + fabs(c))) return -c * Fast<T>::rcp(b);
  // roots q / a and c / q, q = -(b + sign(b) sqrt(disc)) / 2: no cancellation
  // in the small root when b^2 >> |4ac|
  const T disc = Fast<T>::sqrt_(fmax(b * b - T(4) * a * c, T(0)));
  const T q = T(-0.5) * (b + copysign(disc, b));
  const T r1 = q * Fast<T>::rcp(a), r2 = c * Fast<T>::rcp(q);
  T t = T(1);
  if (r1 >= T(0) && r1 <= T(1)) t = r1;
  if (r2 >= T(0) && r2 <= T(1) && r2 < t) t = r2;
  return t;
}

// Accumulator of the two passes over the check points.
template <typename T, int NC>
struct PPCell {
  T ub[NC];
  T gm1, eps, epsp, t1, t2;
  T rmin, pmin;
  bool bad_avg;
  __device__ __forceinline__ void init(const T* avg, T gm1_) {
    gm1 = gm1_;
#pragma unroll
    for (int c = 0; c < NC; ++c) ub[c] = avg[c];
    const T pb = ub[0] > T(0) ? pp_pressure<T, NC>(gm1, ub) : T(-1);
    bad_avg = !(ub[0] > T(0)) || !(pb > T(0));
    eps = PPEps<T>::rho(ub[0]);
    epsp = PPEps<T>::p_frac() * pb;
    t1 = t2 = T(1);
    rmin = ub[0];
    pmin = pb;
  }
  // True if every point of the cell is certainly above both targets, from
  // deviation bounds d[c] >= |p_c(x) - ub[c]| (pp_dev_bound_*), with a margin
  // tol for the rounding of the point values: pass 1 would then find no
  // point below target, so theta = 1 without evaluating the points.
  __device__ __forceinline__ bool screen(const T* d) const {
    if (bad_avg) return false;
    const T tol = PPEps<T>::tol();
    const T rlo = ub[0] - d[0] - tol * (ub[0] + d[0]);
    if (!(rlo > eps)) return false;
    T mh = fabs(ub[1]) + d[1];
    T m2 = mh * mh;
    if (NC == 4) {
      mh = fabs(ub[2]) + d[2];
      m2 = fma(mh, mh, m2);
    }
    // (the margin tol also covers the last-place errors of Fast<T>)
    const T kin = T(0.5) * m2 * Fast<T>::rcp(rlo);
    const T plo = gm1 * (ub[NC - 1] - d[NC - 1] - kin) - tol * gm1 * (fabs(ub[NC - 1]) + d[NC - 1] + kin);
    return plo > epsp;
  }
  // Upper bounds of the x / y Rusanov speeds |v_dir| + c anywhere in a cell
  // that passed the screen (density bounded away from 0 there).
  __device__ __forceinline__ void speed_bound(const T* d, T gamma, T& bx, T& by) const {
    const T tol = PPEps<T>::tol();
    const T rlo = ub[0] - d[0] - tol * (ub[0] + d[0]);
    const T rhi = ub[0] + d[0] + tol * (ub[0] + d[0]);
    const T mxh = fabs(ub[1]) + d[1], myh = NC == 4 ? fabs(ub[2]) + d[2] : T(0);
    const T mxl = fmax(fabs(ub[1]) - d[1], T(0)), myl = NC == 4 ? fmax(fabs(ub[2]) - d[2], T(0)) : T(0);
    const T irlo = Fast<T>::rcp(rlo);
    const T phi = gm1 * (ub[NC - 1] + d[NC - 1] - T(0.5) * fma(mxl, mxl, myl * myl) * Fast<T>::rcp(rhi));
    const T c = Fast<T>::sqrt_(fmax(gamma * phi * irlo, T(0)));
    const T f = T(1) + T(8) * tol;
    bx = fma(mxh, irlo, c) * f;
    by = fma(myh, irlo, c) * f;
  }
  // pass 1: the unlimited values
  __device__ __forceinline__ void first(const T* u) {
    rmin = fmin(rmin, u[0]);
    if (u[0] > T(0)) pmin = fmin(pmin, pp_pressure<T, NC>(gm1, u));
    else pmin = T(-1);
  }
  // after pass 1: true if a second pass is needed
  __device__ __forceinline__ bool need_second() {
    if (bad_avg) {
      t1 = t2 = T(0);  // the average itself is not admissible: keep it constant
      return false;
    }
    if (rmin >= eps && pmin >= epsp) return false;
    if (rmin < eps) t1 = (ub[0] - eps) * Fast<T>::rcp(ub[0] - rmin);
    return true;
  }
  // pass 2: pressure at the density-scaled values
  __device__ __forceinline__ void second(const T* u) {
    T w[NC], dw[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) w[c] = u[c];
    w[0] = fma(t1, u[0] - ub[0], ub[0]);
    if (pp_pressure<T, NC>(gm1, w) < epsp) {
#pragma unroll
      for (int c = 0; c < NC; ++c) dw[c] = w[c] - ub[c];
      t2 = fmin(t2, pp_pressure_root<T, NC>(gm1, ub, dw, epsp));
    }
  }
  __device__ __forceinline__ T theta_rho() const { return t1 * t2; }
  __device__ __forceinline__ T theta() const { return t2; }
};

// ---------------------------------------------------------------------------
// 1D: check points of a cell from its coefficients (NC components, K each)
// ---------------------------------------------------------------------------
template <typename T, int K, int NC, class F>
__device__ __forceinline__ void pp_points_1d(const T (&cf)[NC][K], F&& f) {
  constexpr int D = K - 1;
  T vp[NC], vm[NC];
  auto row = [&](auto rowc) {
    constexpr int R = decltype(rowc)::value;
#pragma unroll
    for (int c = 0; c < NC; ++c) sym_pair<T, D, R>(cf[c], vp[c], vm[c]);
    f(vp);
    f(vm);
  };
  row(std::integral_constant<int, kRowHalf>{});
  row(std::integral_constant<int, LobRow<K>::row>{});
  row(std::integral_constant<int, kRowInner>{});
  row(std::integral_constant<int, kRowOuter>{});
}

// Scale the reconstruction of one 1D Euler cell in place (NC = 3); returns
// (theta_rho, theta).
template <typename T, int K, int NC>
__device__ __forceinline__ void pp_limit_1d(T (&cf)[NC][K], T gm1, T& th_rho, T& th) {
  PPCell<T, NC> s;
  T avg[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) avg[c] = cf[c][0];
  s.init(avg, gm1);
  T d[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) d[c] = pp_dev_bound_1d<T, K>(cf[c]);
  if (!s.screen(d)) {  // a cell that passes the screen keeps theta = 1 without its points
    pp_points_1d<T, K, NC>(cf, [&](const T* u) { s.first(u); });
    if (s.need_second()) pp_points_1d<T, K, NC>(cf, [&](const T* u) { s.second(u); });
  }
  th_rho = s.theta_rho();
  th = s.theta();
  if (th_rho != T(1) || th != T(1)) {
#pragma unroll
    for (int l = 1; l < K; ++l) {
      cf[0][l] *= th_rho;
#pragma unroll
      for (int c = 1; c < NC; ++c) cf[c][l] *= th;
    }
  }
}

// Bound-preserving scaling of a scalar reconstruction to [0, 1]
// (Buckley-Leverett): theta = min(1, (1 - u_bar) / (M - u_bar),
// u_bar / (u_bar - m)), M and m the largest and smallest value at the 1D
// check points.  A cell whose deviation bound keeps every point inside
// [0, 1] (with the rounding margin) is left alone without its points.
template <typename T, int K>
__device__ __forceinline__ void bp_limit_scalar_1d(T (&cf)[1][K]) {
  const T ub = cf[0][0];
  const T d = pp_dev_bound_1d<T, K>(cf[0]);
  const T tol = PPEps<T>::tol();
  const T margin = tol * (fabs(ub) + d);
  if (ub - d - margin >= T(0) && ub + d + margin <= T(1)) return;
  T M = ub, m = ub;
  pp_points_1d<T, K, 1>(cf, [&](const T* u) {
    M = fmax(M, u[0]);
    m = fmin(m, u[0]);
  });
  T th = T(1);
  if (!(ub >= T(0) && ub <= T(1))) {
    th = T(0);
  } else {
    if (M > T(1)) th = fmin(th, (T(1) - ub) / (M - ub));
    if (m < T(0)) th = fmin(th, ub / (ub - m));
  }
  if (th != T(1)) {
#pragma unroll
    for (int l = 1; l < K; ++l) cf[0][l] *= th;
  }
}

// The safeguard of a 1D physics on one cell's coefficients (kLimiter of
// fam_phys.cuh: 1 positivity, 2 bounds [0, 1]).
template <typename T, int K, class PH>
__device__ __forceinline__ void pp_limit_any_1d(T (&cf)[PH::NC][K], const PH& ph) {
  if constexpr (PH::kLimiter == 1) {
    T tr, tt;
    pp_limit_1d<T, K, PH::NC>(cf, ph.gm1, tr, tt);
  } else if constexpr (PH::kLimiter == 2) {
    bp_limit_scalar_1d<T, K>(cf);
  }
}

// ---------------------------------------------------------------------------
// 2D: check points from the coefficients of the 4 components
// ---------------------------------------------------------------------------
// Coefficient l of a component held in a shared-memory slot with stride NT
// (one slot per thread, lane fastest).
template <typename T, int NT>
struct SlotRef {
  const T* p;
  __device__ __forceinline__ T operator[](int l) const { return p[l * NT]; }
};

// Points on the eta lines +-node(EROW); x at the rows listed (Gauss always,
// the Lobatto rows when LOBX).  cf(c) gives component c's coefficients.
template <typename T, int K, int EROW, bool LOBX, class CF, class F>
__device__ __forceinline__ void pp_eta_line(const CF& cf, F& f) {
  constexpr int D = K - 1;
  T dp[4][D + 1], dm[4][D + 1];
#pragma unroll
  for (int c = 0; c < 4; ++c) eta_pair<T, D, EROW>(cf(c), dp[c], dm[c]);
  T a[4], b[4], e[4], g[4];
  auto xrow = [&](auto rowc) {
    constexpr int R = decltype(rowc)::value;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      sym_pair<T, D, R>(dp[c], a[c], b[c]);
      sym_pair<T, D, R>(dm[c], e[c], g[c]);
    }
    f(a);
    f(b);
    f(e);
    f(g);
  };
  xrow(std::integral_constant<int, kRowInner>{});
  xrow(std::integral_constant<int, kRowOuter>{});
  if constexpr (LOBX) {
    xrow(std::integral_constant<int, kRowHalf>{});
    xrow(std::integral_constant<int, LobRow<K>::row>{});
  }
}

template <typename T, int K, class CF, class F>
__device__ __forceinline__ void pp_points_2d(const CF& cf, F&& f) {
  pp_eta_line<T, K, kRowInner, true>(cf, f);  // Gauss eta: Gauss and Lobatto x
  pp_eta_line<T, K, kRowOuter, true>(cf, f);
  pp_eta_line<T, K, kRowHalf, false>(cf, f);  // Lobatto eta: Gauss x
  pp_eta_line<T, K, LobRow<K>::row, false>(cf, f);
}

// (theta_rho, theta) of one 2D Euler cell from its average and deviation
// bounds d (pp_dev_bound_2d), and optionally the largest x / y spectral
// radii at the check points of the limited reconstruction.  A cell that
// passes the screen gets theta = 1 without its points; with want_speeds, its
// points are skipped too when its speed bounds do not exceed run_x / run_y,
// values the grid's maxima already reached (they only grow, so the maxima
// come out the same).  Only a cell that needs its points reads its
// coefficients, through cf(c) (component c, indexable by coefficient).
template <typename T, int K, class PH, class CF>
__device__ __forceinline__ void pp_cell_2d(const T* avg, const T* d, const CF& cf, const PH& ph, T& th_rho, T& th,
                                           bool want_speeds, T run_x, T run_y, T& sx_max, T& sy_max) {
  PPCell<T, 4> s;
  s.init(avg, ph.gm1);
  const bool clear = s.screen(d);
  bool skip = true;
  if (want_speeds) {
    ph.speeds(avg, sx_max, sy_max);
    skip = false;
    if (clear) {
      T bx, by;
      s.speed_bound(d, ph.g, bx, by);
      skip = bx <= run_x && by <= run_y;
    }
  }
  if (!clear || !skip) {
    if (!clear) {
      pp_points_2d<T, K>(cf, [&](const T* u) { s.first(u); });
      if (s.need_second()) pp_points_2d<T, K>(cf, [&](const T* u) { s.second(u); });
    }
    if (!skip) {
      const T tr = s.theta_rho(), tt = s.theta();
      const bool unit = tr == T(1) && tt == T(1);
      pp_points_2d<T, K>(cf, [&](const T* u) {
        T w[4];
        if (unit) {
#pragma unroll
          for (int c = 0; c < 4; ++c) w[c] = u[c];
        } else {
          w[0] = fma(tr, u[0] - avg[0], avg[0]);
#pragma unroll
          for (int c = 1; c < 4; ++c) w[c] = fma(tt, u[c] - avg[c], avg[c]);
        }
        T bx, by;
        ph.speeds(w, bx, by);
        sx_max = max_nonneg(sx_max, bx);
        sy_max = max_nonneg(sy_max, by);
      });
    }
  }
  th_rho = s.theta_rho();
  th = s.theta();
}

}  // namespace fam
