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
// Targets: density min(1e-13, rho_bar) in FP64, 1e-4 rho_bar in FP32;
// pressure a fraction of p_bar (1e-10 in FP64, 1e-4 in FP32), above the
// rounding of E - |m|^2/(2 rho) at a point scaled to a small density.  The basis has P_0 = 1 and zero-mean higher
// functions, so coefficient 0 is the average and scaling the others scales
// p - u_bar.
#pragma once

#include <type_traits>

#include "fam_recon.cuh"

namespace fam {

template <typename T> struct PPEps;
template <> struct PPEps<double> {
  static __device__ __forceinline__ double rho(double rb) { return fmin(1e-13, rb); }
  static __device__ __forceinline__ double p_frac() { return 1e-10; }
};
// FP32: the density target too is a fraction of the average, since
// rho_bar + theta (rho - rho_bar) carries a rounding error of order
// 1e-7 rho_bar, far above 1e-13
template <> struct PPEps<float> {
  static __device__ __forceinline__ float rho(float rb) { return 1e-4f * rb; }
  static __device__ __forceinline__ float p_frac() { return 1e-4f; }
};

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
  pp_points_1d<T, K, NC>(cf, [&](const T* u) { s.first(u); });
  if (s.need_second()) pp_points_1d<T, K, NC>(cf, [&](const T* u) { s.second(u); });
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

// ---------------------------------------------------------------------------
// 2D: check points from the coefficients of the 4 components
// ---------------------------------------------------------------------------
// Points on the eta lines +-node(EROW); x at the rows listed (Gauss always,
// the Lobatto rows when LOBX).
template <typename T, int K, int EROW, bool LOBX, class F>
__device__ __forceinline__ void pp_eta_line(const T (&coef)[4][K * (K + 1) / 2], F& f) {
  constexpr int D = K - 1;
  T dp[4][D + 1], dm[4][D + 1];
#pragma unroll
  for (int c = 0; c < 4; ++c) eta_pair<T, D, EROW>(coef[c], dp[c], dm[c]);
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

template <typename T, int K, class F>
__device__ __forceinline__ void pp_points_2d(const T (&coef)[4][K * (K + 1) / 2], F&& f) {
  pp_eta_line<T, K, kRowInner, true>(coef, f);  // Gauss eta: Gauss and Lobatto x
  pp_eta_line<T, K, kRowOuter, true>(coef, f);
  pp_eta_line<T, K, kRowHalf, false>(coef, f);  // Lobatto eta: Gauss x
  pp_eta_line<T, K, LobRow<K>::row, false>(coef, f);
}

// (theta_rho, theta) of one 2D Euler cell, and optionally the largest x / y
// spectral radii at the check points of the limited reconstruction.
template <typename T, int K, class PH>
__device__ __forceinline__ void pp_cell_2d(const T (&coef)[4][K * (K + 1) / 2], const PH& ph, T& th_rho, T& th,
                                           bool want_speeds, T& sx_max, T& sy_max) {
  PPCell<T, 4> s;
  const T avg[4] = {coef[0][0], coef[1][0], coef[2][0], coef[3][0]};
  s.init(avg, ph.gm1);
  pp_points_2d<T, K>(coef, [&](const T* u) { s.first(u); });
  if (s.need_second()) pp_points_2d<T, K>(coef, [&](const T* u) { s.second(u); });
  th_rho = s.theta_rho();
  th = s.theta();
  if (want_speeds) {
    T ax, ay;
    ph.speeds(avg, ax, ay);
    sx_max = ax;
    sy_max = ay;
    const T tr = th_rho, tt = th;
    pp_points_2d<T, K>(coef, [&](const T* u) {
      T w[4];
      w[0] = fma(tr, u[0] - avg[0], avg[0]);
#pragma unroll
      for (int c = 1; c < 4; ++c) w[c] = fma(tt, u[c] - avg[c], avg[c]);
      T bx, by;
      ph.speeds(w, bx, by);
      sx_max = max_nonneg(sx_max, bx);
      sy_max = max_nonneg(sy_max, by);
    });
  }
}

}  // namespace fam
