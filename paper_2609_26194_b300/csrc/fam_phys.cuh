// fam_phys.cuh -- physical fluxes, Rusanov wave speeds and volume-integral
// accumulation for the FAM stage kernels.
//
// Scalar laws: linear advection f = a u (Sec. 3), Burgers f = u^2/2
// (Example 4.1), Buckley-Leverett f = 4u^2 / (4u^2 + (1-u)^2) (Example 4.3).  Euler equations with ratio of specific heats gamma in
// conservative variables (Sec. 2.3): 1D (rho, rho u, E), 2D (rho, rho u,
// rho v, E), p = (gamma - 1)(E - rho |v|^2 / 2), spectral radius of the flux
// Jacobian |v_n| + c with c = sqrt(gamma p / rho).
//
// Conventions:
//   flux_x / flux_y return the spectral radius and write the flux.
//   vol_acc accumulates w * f at a volume quadrature point into VA (a
//   physics-specific packing); vol_finish unpacks VA into the volume terms
//   V1[c] = sum w f_1,c and V2[c] = sum w f_2,c.  Components whose flux is a
//   conserved variable itself (rho u, rho v for the mass equation) take the
//   exact integral, which is the cell average because the reconstruction
//   reproduces it and the Gauss rule integrates it exactly.
#pragma once

#include "fam_common.cuh"

namespace fam {

enum Equation { kAdvection = 0, kBurgers = 1, kEuler = 2, kBuckley = 3 };

// kLimiter: the optional safeguard a physics has (fam_pp.cuh): 0 none,
// 1 positivity of density and pressure (Euler), 2 bounds [0, 1] (a scalar
// whose solution stays there, Buckley-Leverett).

// ----------------------------------------------------------------------------
// 1D
// ----------------------------------------------------------------------------
template <typename T> struct Advection1D {
  static constexpr int NC = 1, NVA = 1, kLimiter = 0;
  T a;
  __device__ __forceinline__ T flux_x(const T* u, T* f) const { f[0] = a * u[0]; return fabs(a); }
  __device__ __forceinline__ T speed_x(const T* u) const { return fabs(a); }
  __device__ __forceinline__ void vol_acc(const T* u, T w, T* VA) const { VA[0] = fma(w, u[0], VA[0]); }
  __device__ __forceinline__ void vol_finish(const T* VA, const T* avg, T* V1) const { V1[0] = a * VA[0]; }
  __device__ __forceinline__ bool admissible(const T* u) const { return true; }
};

template <typename T> struct Burgers1D {
  static constexpr int NC = 1, NVA = 1, kLimiter = 0;
  __device__ __forceinline__ T flux_x(const T* u, T* f) const { f[0] = T(0.5) * u[0] * u[0]; return fabs(u[0]); }
  __device__ __forceinline__ T speed_x(const T* u) const { return fabs(u[0]); }
  __device__ __forceinline__ void vol_acc(const T* u, T w, T* VA) const { VA[0] = fma(w * u[0], u[0], VA[0]); }
  __device__ __forceinline__ void vol_finish(const T* VA, const T* avg, T* V1) const { V1[0] = T(0.5) * VA[0]; }
  __device__ __forceinline__ bool admissible(const T* u) const { return true; }
};

// Buckley-Leverett (Example 4.3).  f'(u) = 8u(1-u) / (5u^2 - 2u + 1)^2
// vanishes at u = 0 and 1, the states of the initial data, so every speed
// (Rusanov, OE beta, time step) is the bound max |f'| over all u: f'(u*),
// u* the root in (0, 1) of 10u^3 - 15u^2 + 1 (where f'' = 0).
template <typename T> struct BuckleyLeverett1D {
  static constexpr int NC = 1, NVA = 1, kLimiter = 2;
  static __device__ __forceinline__ T flux(T u) {
    const T a = T(4) * u * u, b = (T(1) - u) * (T(1) - u);
    return a / (a + b);
  }
  static __device__ __forceinline__ T bound() { return T(2.332030375854268710378); }
  __device__ __forceinline__ T flux_x(const T* u, T* f) const { f[0] = flux(u[0]); return bound(); }
  __device__ __forceinline__ T speed_x(const T* u) const { return bound(); }
  __device__ __forceinline__ void vol_acc(const T* u, T w, T* VA) const { VA[0] = fma(w, flux(u[0]), VA[0]); }
  __device__ __forceinline__ void vol_finish(const T* VA, const T* avg, T* V1) const { V1[0] = VA[0]; }
  __device__ __forceinline__ bool admissible(const T* u) const { return true; }
};

template <typename T> struct Euler1D {
  static constexpr int NC = 3, NVA = 2, kLimiter = 1;
  T g, gm1, hgm1;  // gamma, gamma - 1, (gamma - 1)/2
  __device__ __forceinline__ T flux_x(const T* u, T* f) const {
    const T r = Fast<T>::rcp(u[0]);
    const T vel = u[1] * r;
    const T mu = u[1] * vel;
    const T p = fma(-hgm1, mu, gm1 * u[2]);
    f[0] = u[1];
    f[1] = mu + p;
    f[2] = (u[2] + p) * vel;
    return fabs(vel) + Fast<T>::sqrt_(g * p * r);
  }
  __device__ __forceinline__ T speed_x(const T* u) const {
    const T r = Fast<T>::rcp(u[0]);
    const T vel = u[1] * r;
    const T p = fma(-hgm1, u[1] * vel, gm1 * u[2]);
    return fabs(vel) + Fast<T>::sqrt_(g * p * r);
  }
  __device__ __forceinline__ void vol_acc(const T* u, T w, T* VA) const {
    const T r = Fast<T>::rcp(u[0]);
    const T vel = u[1] * r;
    const T mu = u[1] * vel;
    const T p = fma(-hgm1, mu, gm1 * u[2]);
    VA[0] = fma(w, mu + p, VA[0]);
    VA[1] = fma(w, (u[2] + p) * vel, VA[1]);
  }
  __device__ __forceinline__ void vol_finish(const T* VA, const T* avg, T* V1) const {
    V1[0] = avg[1];
    V1[1] = VA[0];
    V1[2] = VA[1];
  }
  __device__ __forceinline__ bool admissible(const T* u) const {
    // rho > 0 and rho E - |rho u|^2 / 2 > 0 (p > 0 without a division)
    return u[0] > T(0) && u[0] * u[2] - T(0.5) * u[1] * u[1] > T(0);
  }
};

// ----------------------------------------------------------------------------
// 2D
// ----------------------------------------------------------------------------
template <typename T> struct Advection2D {
  static constexpr int NC = 1, NVA = 1;
  T ax, ay;
  __device__ __forceinline__ T flux_x(const T* u, T* f) const { f[0] = ax * u[0]; return fabs(ax); }
  __device__ __forceinline__ T flux_y(const T* u, T* f) const { f[0] = ay * u[0]; return fabs(ay); }
  __device__ __forceinline__ void speeds(const T* u, T& sx, T& sy) const { sx = fabs(ax); sy = fabs(ay); }
  __device__ __forceinline__ void vol_acc(const T* u, T w, T* VA) const { VA[0] = fma(w, u[0], VA[0]); }
  __device__ __forceinline__ void vol_finish(const T* VA, const T* avg, T* V1, T* V2) const {
    V1[0] = ax * VA[0];
    V2[0] = ay * VA[0];
  }
  __device__ __forceinline__ bool admissible(const T* u) const { return true; }
};

template <typename T> struct Burgers2D {
  static constexpr int NC = 1, NVA = 1;
  __device__ __forceinline__ T flux_x(const T* u, T* f) const { f[0] = T(0.5) * u[0] * u[0]; return fabs(u[0]); }
  __device__ __forceinline__ T flux_y(const T* u, T* f) const { f[0] = T(0.5) * u[0] * u[0]; return fabs(u[0]); }
  __device__ __forceinline__ void speeds(const T* u, T& sx, T& sy) const { sx = sy = fabs(u[0]); }
  __device__ __forceinline__ void vol_acc(const T* u, T w, T* VA) const { VA[0] = fma(w * u[0], u[0], VA[0]); }
  __device__ __forceinline__ void vol_finish(const T* VA, const T* avg, T* V1, T* V2) const {
    V1[0] = V2[0] = T(0.5) * VA[0];
  }
  __device__ __forceinline__ bool admissible(const T* u) const { return true; }
};

template <typename T> struct Euler2D {
  static constexpr int NC = 4, NVA = 5;
  T g, gm1, hgm1;
  __device__ __forceinline__ T flux_x(const T* u, T* f) const {
    const T r = Fast<T>::rcp(u[0]);
    const T vx = u[1] * r, vy = u[2] * r;
    const T p = fma(-hgm1, fma(u[1], vx, u[2] * vy), gm1 * u[3]);
    f[0] = u[1];
    f[1] = fma(u[1], vx, p);
    f[2] = u[2] * vx;
    f[3] = (u[3] + p) * vx;
    return fabs(vx) + Fast<T>::sqrt_(g * p * r);
  }
  __device__ __forceinline__ T flux_y(const T* u, T* f) const {
    const T r = Fast<T>::rcp(u[0]);
    const T vx = u[1] * r, vy = u[2] * r;
    const T p = fma(-hgm1, fma(u[1], vx, u[2] * vy), gm1 * u[3]);
    f[0] = u[2];
    f[1] = u[1] * vy;
    f[2] = fma(u[2], vy, p);
    f[3] = (u[3] + p) * vy;
    return fabs(vy) + Fast<T>::sqrt_(g * p * r);
  }
  __device__ __forceinline__ void speeds(const T* u, T& sx, T& sy) const {
    const T r = Fast<T>::rcp(u[0]);
    const T vx = u[1] * r, vy = u[2] * r;
    const T p = fma(-hgm1, fma(u[1], vx, u[2] * vy), gm1 * u[3]);
    const T c = Fast<T>::sqrt_(g * p * r);
    sx = fabs(vx) + c;
    sy = fabs(vy) + c;
  }
  // VA = {sum w (rho u^2 + p), sum w rho u v, sum w (E+p) u, sum w (rho v^2 + p), sum w (E+p) v}
  // The products that no multiply-add absorbs run on the integer pipes
  // (pmul, bit-identical): the 16 volume points of a cell are independent,
  // so these overlap the FP64 unit's work.  The face fluxes keep the FP64
  // unit: their dependent chains would wait on the longer integer latency.
  __device__ __forceinline__ void vol_acc(const T* u, T w, T* VA) const {
    const T r = Fast<T>::rcp(u[0]);
    const T vx = pmul(u[1], r), vy = pmul(u[2], r);
    const T p = fma(-hgm1, fma(u[1], vx, pmul(u[2], vy)), pmul(gm1, u[3]));
    const T wh = pmul(w, u[3] + p);
    VA[0] = fma(w, fma(u[1], vx, p), VA[0]);
    VA[1] = fma(pmul(w, u[2]), vx, VA[1]);
    VA[2] = fma(wh, vx, VA[2]);
    VA[3] = fma(w, fma(u[2], vy, p), VA[3]);
    VA[4] = fma(wh, vy, VA[4]);
  }
  __device__ __forceinline__ void vol_finish(const T* VA, const T* avg, T* V1, T* V2) const {
    V1[0] = avg[1];
    V1[1] = VA[0];
    V1[2] = VA[1];
    V1[3] = VA[2];
    V2[0] = avg[2];
    V2[1] = VA[1];
    V2[2] = VA[3];
    V2[3] = VA[4];
  }
  __device__ __forceinline__ bool admissible(const T* u) const {
    return u[0] > T(0) && u[0] * u[3] - T(0.5) * (u[1] * u[1] + u[2] * u[2]) > T(0);
  }

  // ---- derivatives for the adjoint ------------------------------------------
  // ub += (d f_dir / d u)^T w  (flux Jacobian-transpose product)
  __device__ __forceinline__ void flux_vjp(int dir, const T* u, const T* w, T* ub) const {
    const T r = Fast<T>::rcp(u[0]);
    const T vx = u[1] * r, vy = u[2] * r;
    const T q2 = vx * vx + vy * vy;
    const T p = gm1 * (u[3] - T(0.5) * u[0] * q2);
    const T H = (u[3] + p) * r;
    if (dir == 0) {
      ub[0] += w[1] * (hgm1 * q2 - vx * vx) - w[2] * vx * vy + w[3] * vx * (hgm1 * q2 - H);
      ub[1] += w[0] + w[1] * (T(2) - gm1) * vx + w[2] * vy + w[3] * (H - gm1 * vx * vx);
      ub[2] += -w[1] * gm1 * vy + w[2] * vx - w[3] * gm1 * vx * vy;
      ub[3] += w[1] * gm1 + w[3] * g * vx;
    } else {
      ub[0] += -w[1] * vx * vy + w[2] * (hgm1 * q2 - vy * vy) + w[3] * vy * (hgm1 * q2 - H);
      ub[1] += w[1] * vy - w[2] * gm1 * vx - w[3] * gm1 * vx * vy;
      ub[2] += w[0] + w[1] * vx + w[2] * (T(2) - gm1) * vy + w[3] * (H - gm1 * vy * vy);
      ub[3] += w[2] * gm1 + w[3] * g * vy;
    }
  }
  // spectral radius |v_dir| + c and its gradient with respect to u
  __device__ __forceinline__ T speed_grad(int dir, const T* u, T* gr) const {
    const T r = Fast<T>::rcp(u[0]);
    const T vx = u[1] * r, vy = u[2] * r;
    const T q2 = vx * vx + vy * vy;
    const T p = gm1 * (u[3] - T(0.5) * u[0] * q2);
    const T c = Fast<T>::sqrt_(g * p * r);
    const T vn = dir == 0 ? vx : vy;
    const T sg = vn > T(0) ? T(1) : (vn < T(0) ? T(-1) : T(0));
    const T kc = T(0.5) * g * r * Fast<T>::rcp(c);   // dc = kc (dp - (p/rho) drho), kc = g / (2 c rho)
    // dp/du = gm1 (q2/2, -vx, -vy, 1); dvn/du = (-vn/rho, [dir==0]/rho, [dir==1]/rho, 0)
    gr[0] = -sg * vn * r + kc * (hgm1 * q2 - p * r);
    gr[1] = (dir == 0 ? sg * r : T(0)) - kc * gm1 * vx;
    gr[2] = (dir == 1 ? sg * r : T(0)) - kc * gm1 * vy;
    gr[3] = kc * gm1;
    return fabs(vn) + c;
  }
};

}  // namespace fam
