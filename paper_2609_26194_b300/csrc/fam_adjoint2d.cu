// fam_adjoint2d.cu -- reverse sweep of the 2D Euler FAM time step.
//
// Not in the paper: the adjoint (transpose of the linearised step) of the
// SSP-RK3 stages of eq. (12) and of the OE step of eq. (2dOE_system), with
// the step sizes of the forward run held fixed.  Given the cotangent of the
// state after a step it returns the cotangent of the state before it; with
// checkpoints of the forward states every m steps and recomputation of each
// segment, fam_adjoint() returns dJ/dU^0 for a terminal functional J(U^T).
//
// Transposes, cell by cell (one thread per cell, periodic grids):
//   residual eq. (11): v = cotangent of R(c) ->
//     face flux cotangents (the two cells sharing a face), Rusanov flux
//     Jacobian-transpose products (subgradient of the max wave speed to the
//     side that attains it, left/bottom on ties), Euler flux
//     Jacobian-transposes at the 4x4 volume points, transpose of the point
//     evaluation of p, transpose of the reconstruction (generated), gather
//     of the 3x3 patch contributions;
//   OE: d(m e^-theta) = e^-theta dm - m e^-theta dtheta, theta through the
//     jumps (transposed face-centre traces), the Type-II denominator D and
//     the local speed maxima beta (subgradients at the maximisers).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "fam_internal.cuh"

namespace {

using fam::cidx;

// ------------------------------------------------------------------------
// point slots of a cell, in a fixed order:
//   slots 0..15  volume (b*4 + a): xi node a, eta node b (ascending nodes)
//   slots 16..19 x-face -1/2 (eta node g), 20..23 x-face +1/2,
//   slots 24..27 y-face -1/2 (xi node g), 28..31 y-face +1/2
// ------------------------------------------------------------------------

template <int K> struct RT;
#define FAM_RT(K, FCT)                                                                         \
  template <> struct RT<K> {                                                                   \
    template <typename T> static __device__ void coefT(const T* cb, T* g) { fam2d_coefT_k##K(cb, g); } \
    template <typename T> static __device__ void facecT(const T* tb, T* g, int q6) { FCT; }    \
  };
FAM_RT(3, fam2d_facecT_k3p(tb, g))
FAM_RT(4, fam2d_facecT_k4p(tb, g))
FAM_RT(5, fam2d_facecT_k5p(tb, g))
FAM_RT(6, if (q6) fam2d_facecT_k6q(tb, g); else fam2d_facecT_k6p(tb, g))
#undef FAM_RT

struct AGeo {
  Geo g;          // padded layout of the stored forward states
  long long n;    // cells
};

__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

template <typename T>
__device__ __forceinline__ void gather_patch_g(const T* __restrict__ U, const Geo& g, int c, int j, int i, T* A,
                                               T* X, T* Y) {
#pragma unroll
  for (int s = 0; s < 9; ++s) {
    const int jj = j + s / 3 - 1, ii = i + s % 3 - 1;  // ghosts hold the periodic images
    A[s] = U[cell_index(g, c * 3 + 0, jj, ii)];
    X[s] = U[cell_index(g, c * 3 + 1, jj, ii)];
    Y[s] = U[cell_index(g, c * 3 + 2, jj, ii)];
  }
}

// ------------------------------------------------------------------------
// residual transpose
// ------------------------------------------------------------------------
// TR[(f*4 + g)*NC + comp][cell]: the cell's own trace on face f (0 = x-,
// 1 = x+, 2 = y-, 3 = y+) at Gauss point g.
template <typename T, int K, class PH>
__global__ void __launch_bounds__(128) adj_traces(const T* __restrict__ U, const Geo geo, T* __restrict__ TR) {
  constexpr int NC = PH::NC;
  constexpr int D = K - 1;
  constexpr int NCO = K * (K + 1) / 2;
  const long long n = (long long)geo.nx * geo.ny;
  const long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (cell >= n) return;
  const int i = (int)(cell % geo.nx), j = (int)(cell / geo.nx);
  auto put = [&](int f, int g, int c, T v) { TR[((long long)(f * 4 + g) * NC + c) * n + cell] = v; };
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    T A[9], X[9], Y[9], coef[NCO];
    gather_patch_g(U, geo, c, j, i, A, X, Y);
    Recon2D<K>::coef(A, X, Y, coef);
    // x-faces at the eta nodes: pairs (+inner, -inner) = nodes (2, 1), (+outer, -outer) = (3, 0)
#pragma unroll
    for (int pr = 0; pr < 2; ++pr) {
      T dp[D + 1], dm[D + 1];
      if (pr == 0) eta_pair<T, D, kRowInner>(coef, dp, dm);
      else eta_pair<T, D, kRowOuter>(coef, dp, dm);
      const int hp = pr == 0 ? 2 : 3, hm = pr == 0 ? 1 : 0;
      T rp, lp, rm, lm;
      sym_pair<T, D, kRowHalf>(dp, rp, lp);
      sym_pair<T, D, kRowHalf>(dm, rm, lm);
      put(1, hp, c, rp);
      put(0, hp, c, lp);
      put(1, hm, c, rm);
      put(0, hm, c, lm);
    }
    // y-faces at the xi nodes: eta = +1/2 (top, face 3) and -1/2 (bottom, face 2)
    T dp[D + 1], dm[D + 1], t[4], b[4];
    eta_pair<T, D, kRowHalf>(coef, dp, dm);
    sym_pair<T, D, kRowInner>(dp, t[2], t[1]);
    sym_pair<T, D, kRowOuter>(dp, t[3], t[0]);
    sym_pair<T, D, kRowInner>(dm, b[2], b[1]);
    sym_pair<T, D, kRowOuter>(dm, b[3], b[0]);
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      put(3, g, c, t[g]);
      put(2, g, c, b[g]);
    }
  }
}

// Cotangent of the Rusanov flux F(uL, uR) with respect to this cell's trace
// (side = 0: this cell is the left/bottom one, 1: right/top one).
template <typename T, class PH>
__device__ __forceinline__ void llf_vjp(const PH& ph, int dir, const T* uL, const T* uR, const T* Fb, int side,
                                        T* ub) {
  constexpr int NC = PH::NC;
  T gL[NC], gR[NC];
  const T sL = ph.speed_grad(dir, uL, gL);
  const T sR = ph.speed_grad(dir, uR, gR);
  const bool left_max = sL >= sR;
  const T a = left_max ? sL : sR;
  T d = T(0);
#pragma unroll
  for (int c = 0; c < NC; ++c) d = fma(Fb[c], uR[c] - uL[c], d);
  T hf[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) hf[c] = T(0.5) * Fb[c];
  const T* u = side == 0 ? uL : uR;
  ph.flux_vjp(dir, u, hf, ub);
  const T sgn = side == 0 ? T(1) : T(-1);
#pragma unroll
  for (int c = 0; c < NC; ++c) ub[c] += sgn * T(0.5) * a * Fb[c];
  if ((side == 0) == left_max) {
    const T* gr = side == 0 ? gL : gR;
#pragma unroll
    for (int c = 0; c < NC; ++c) ub[c] -= T(0.5) * d * gr[c];
  }
}

// PB[(s*3 + m)*NC + comp][cell]: cotangent of this cell's patch input
// (neighbour s of the 3x3 patch, moment m) from R^T v.
//
// Point cotangents (16 volume points, 16 face Gauss points; slots as
// listed at the top of this file) go to shared memory, [q][c][thread]; each component's
// coefficient cotangents are then the transposed sum-factorised evaluation
// (sym_pair_T / eta_pair_T mirror the forward evaluation of stage2d).
constexpr int kAdjBS = 64;  // threads per block of adj_residual_local

template <typename T, int K, class PH>
__global__ void __launch_bounds__(kAdjBS) adj_residual_local(const T* __restrict__ U, const Geo geo,
                                                             const T* __restrict__ TR, const T* __restrict__ V,
                                                             const PH ph, T* __restrict__ PB) {
  constexpr int NC = PH::NC;
  constexpr int D = K - 1;
  constexpr int NCO = K * (K + 1) / 2;
  extern __shared__ __align__(16) unsigned char adj_smem[];
  T* vbs = reinterpret_cast<T*>(adj_smem);  // [32][NC][kAdjBS]
  auto VB = [&](int q, int c) -> T& { return vbs[(q * NC + c) * kAdjBS + threadIdx.x]; };
  const long long n = (long long)geo.nx * geo.ny;
  const long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (cell >= n) return;  // no block-wide barrier below
  const int i = (int)(cell % geo.nx), j = (int)(cell / geo.nx);
  const T idx_ = T(geo.idx), idy_ = T(geo.idy);
  const double* X = famgen::kGaussX;
  const double* W = famgen::kGaussW;
  auto vat = [&](int c, int m, int jj, int ii) -> T {
    return V[(long long)(c * 3 + m) * n + (long long)wrap(jj, geo.ny) * geo.nx + wrap(ii, geo.nx)];
  };
  auto trat = [&](int f, int g, int c, int jj, int ii) -> T {
    return TR[(long long)((f * 4 + g) * NC + c) * n + (long long)wrap(jj, geo.ny) * geo.nx + wrap(ii, geo.nx)];
  };
  // ---- volume points: flux Jacobian-transposes weighted by v1/dx, v2/dy ----
  {
    T coef[NC][NCO];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      T A[9], Xm[9], Ym[9];
      gather_patch_g(U, geo, c, j, i, A, Xm, Ym);
      Recon2D<K>::coef(A, Xm, Ym, coef[c]);
    }
    T v1[NC], v2[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      v1[c] = vat(c, 1, j, i) * idx_;
      v2[c] = vat(c, 2, j, i) * idy_;
    }
#pragma unroll
    for (int pr = 0; pr < 2; ++pr) {
      T up[NC][4], um[NC][4];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        T dp[D + 1], dm[D + 1];
        if (pr == 0) eta_pair<T, D, kRowInner>(coef[c], dp, dm);
        else eta_pair<T, D, kRowOuter>(coef[c], dp, dm);
        sym_pair<T, D, kRowInner>(dp, up[c][2], up[c][1]);
        sym_pair<T, D, kRowOuter>(dp, up[c][3], up[c][0]);
        sym_pair<T, D, kRowInner>(dm, um[c][2], um[c][1]);
        sym_pair<T, D, kRowOuter>(dm, um[c][3], um[c][0]);
      }
      const int hp = pr == 0 ? 2 : 3, hm = pr == 0 ? 1 : 0;
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const int b = side == 0 ? hp : hm;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const T wq = T(W[a] * W[b]);
          T u[NC], ub[NC], w1[NC], w2[NC];
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            u[c] = side == 0 ? up[c][a] : um[c][a];
            ub[c] = T(0);
            w1[c] = wq * v1[c];
            w2[c] = wq * v2[c];
          }
          ph.flux_vjp(0, u, w1, ub);
          ph.flux_vjp(1, u, w2, ub);
#pragma unroll
          for (int c = 0; c < NC; ++c) VB(b * 4 + a, c) = ub[c];
        }
      }
    }
  }
  // ---- faces.  x-face between L and R at Gauss node g (eta):
  //   Fbar = (w_g/dx)[-v0_L - v1_L/2 - eta_g v2_L + v0_R - v1_R/2 + eta_g v2_R]
  // y-face between B and T at xi node g:
  //   Fbar = (w_g/dy)[-v0_B - v2_B/2 - xi_g v1_B + v0_T - v2_T/2 + xi_g v1_T]
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const int dir = f / 2;
    const int side = (f % 2 == 0) ? 1 : 0;          // face - : this cell is right/top; face + : left/bottom
    const int di = dir == 0 ? (f == 0 ? -1 : 1) : 0;
    const int dj = dir == 1 ? (f == 2 ? -1 : 1) : 0;
    const int nbf = f ^ 1;                           // the neighbour's face opposite
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      T own[NC], oth[NC], Fb[NC], ub[NC];
      const T wg = T(W[g]) * (dir == 0 ? idx_ : idy_);
      const T xg = T(X[g]);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        own[c] = trat(f, g, c, j, i);
        oth[c] = trat(nbf, g, c, j + dj, i + di);
        // L/B cell and R/T cell of this face
        const int jl = side == 0 ? j : j + dj, il = side == 0 ? i : i + di;
        const int jr = side == 0 ? j + dj : j, ir = side == 0 ? i + di : i;
        T fb;
        if (dir == 0)
          fb = -vat(c, 0, jl, il) - T(0.5) * vat(c, 1, jl, il) - xg * vat(c, 2, jl, il) + vat(c, 0, jr, ir) -
               T(0.5) * vat(c, 1, jr, ir) + xg * vat(c, 2, jr, ir);
        else
          fb = -vat(c, 0, jl, il) - T(0.5) * vat(c, 2, jl, il) - xg * vat(c, 1, jl, il) + vat(c, 0, jr, ir) -
               T(0.5) * vat(c, 2, jr, ir) + xg * vat(c, 1, jr, ir);
        Fb[c] = wg * fb;
        ub[c] = T(0);
      }
      if (side == 0) llf_vjp(ph, dir, own, oth, Fb, 0, ub);
      else llf_vjp(ph, dir, oth, own, Fb, 1, ub);
#pragma unroll
      for (int c = 0; c < NC; ++c) VB(16 + f * 4 + g, c) = ub[c];
    }
  }
  // ---- transpose of the point evaluation, then of the reconstruction ----
#pragma unroll 1
  for (int c = 0; c < NC; ++c) {
    T cb[NCO];
#pragma unroll
    for (int l = 0; l < NCO; ++l) cb[l] = T(0);
#pragma unroll
    for (int pr = 0; pr < 2; ++pr) {
      const int hp = pr == 0 ? 2 : 3, hm = pr == 0 ? 1 : 0;
      T dpb[D + 1], dmb[D + 1];
#pragma unroll
      for (int a = 0; a <= D; ++a) dpb[a] = dmb[a] = T(0);
      // volume values at eta = +node (row hp) and -node (row hm)
      sym_pair_T<T, D, kRowInner>(VB(hp * 4 + 2, c), VB(hp * 4 + 1, c), dpb);
      sym_pair_T<T, D, kRowOuter>(VB(hp * 4 + 3, c), VB(hp * 4 + 0, c), dpb);
      sym_pair_T<T, D, kRowInner>(VB(hm * 4 + 2, c), VB(hm * 4 + 1, c), dmb);
      sym_pair_T<T, D, kRowOuter>(VB(hm * 4 + 3, c), VB(hm * 4 + 0, c), dmb);
      // x-face traces (xi = +1/2: slot 20 + node, -1/2: slot 16 + node) on the same eta rows
      sym_pair_T<T, D, kRowHalf>(VB(20 + hp, c), VB(16 + hp, c), dpb);
      sym_pair_T<T, D, kRowHalf>(VB(20 + hm, c), VB(16 + hm, c), dmb);
      if (pr == 0) eta_pair_T<T, D, kRowInner>(dpb, dmb, cb);
      else eta_pair_T<T, D, kRowOuter>(dpb, dmb, cb);
    }
    {
      // y-face traces: eta = +1/2 (slots 28 + xi node), -1/2 (slots 24 + xi node)
      T dpb[D + 1], dmb[D + 1];
#pragma unroll
      for (int a = 0; a <= D; ++a) dpb[a] = dmb[a] = T(0);
      sym_pair_T<T, D, kRowInner>(VB(28 + 2, c), VB(28 + 1, c), dpb);
      sym_pair_T<T, D, kRowOuter>(VB(28 + 3, c), VB(28 + 0, c), dpb);
      sym_pair_T<T, D, kRowInner>(VB(24 + 2, c), VB(24 + 1, c), dmb);
      sym_pair_T<T, D, kRowOuter>(VB(24 + 3, c), VB(24 + 0, c), dmb);
      eta_pair_T<T, D, kRowHalf>(dpb, dmb, cb);
    }
    T gp[27];
    RT<K>::coefT(cb, gp);
#pragma unroll
    for (int s2 = 0; s2 < 9; ++s2)
#pragma unroll
      for (int m = 0; m < 3; ++m) PB[(long long)((s2 * 3 + m) * NC + c) * n + cell] = gp[m * 9 + s2];
  }
}

// Gather the patch cotangents onto each cell and apply the Shu--Osher
// transpose: out_in = w1 (v + dt R^T v); acc0 += w0 v (+ out_in for stage 1).
template <typename T, int NC>
__global__ void adj_gather(const T* __restrict__ PB, const T* __restrict__ V, const Geo geo, T dt, T w0, T w1,
                           int stage, T* __restrict__ out_in, T* __restrict__ acc0) {
  const long long n = (long long)geo.nx * geo.ny;
  const long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (cell >= n) return;
  const int i = (int)(cell % geo.nx), j = (int)(cell / geo.nx);
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      T rt = T(0);
#pragma unroll
      for (int s = 0; s < 9; ++s) {
        // cell (j,i) is patch position s of the cell at (j,i) - offset(s)
        const int jj = wrap(j - (s / 3 - 1), geo.ny), ii = wrap(i - (s % 3 - 1), geo.nx);
        rt += PB[(long long)((s * 3 + m) * NC + c) * n + (long long)jj * geo.nx + ii];
      }
      const long long o = (long long)(c * 3 + m) * n + cell;
      const T v = V[o];
      const T in = w1 * (v + dt * rt);
      if (stage == 1) {
        acc0[o] += in;
      } else {
        out_in[o] = in;
        acc0[o] += w0 * v;
      }
    }
}

// ------------------------------------------------------------------------
// OE transpose
// ------------------------------------------------------------------------
// TRC[(f*NC + comp)][cell] face-centre traces; SP[dir][cell] speeds at averages
template <typename T, int K, class PH>
__global__ void adj_oe_prep(const T* __restrict__ U, const Geo geo, const PH ph, int q6, T* __restrict__ TRC,
                            T* __restrict__ SP) {
  constexpr int NC = PH::NC;
  const long long n = (long long)geo.nx * geo.ny;
  const long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (cell >= n) return;
  const int i = (int)(cell % geo.nx), j = (int)(cell / geo.nx);
  T u[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    T A[9], X[9], Y[9], t[4];
    gather_patch_g(U, geo, c, j, i, A, X, Y);
    Recon2D<K>::facec(A, X, Y, t, q6);
#pragma unroll
    for (int f = 0; f < 4; ++f) TRC[(long long)(f * NC + c) * n + cell] = t[f];
    u[c] = A[4];
  }
  T gr[NC];
  SP[cell] = ph.speed_grad(0, u, gr);
  SP[n + cell] = ph.speed_grad(1, u, gr);
}

// Per cell: JB[(f*NC + comp)][cell] jump cotangents (f = xl, xr, yb, yt),
// AVB[(s*NC + comp)][cell] cotangent contributions to the averages of the
// 3x3 neighbourhood (position s), and the moment part of the result.
template <typename T, int K, class PH>
__global__ void adj_oe_local(const T* __restrict__ U, const Geo geo, const PH ph, const T* __restrict__ TRC,
                             const T* __restrict__ SP, const T* __restrict__ LAM, T dt, T gamma_k,
                             T* __restrict__ JB, T* __restrict__ AVB, T* __restrict__ OUT) {
  constexpr int NC = PH::NC;
  const long long n = (long long)geo.nx * geo.ny;
  const long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (cell >= n) return;
  const int i = (int)(cell % geo.nx), j = (int)(cell / geo.nx);
  auto at = [&](int jj, int ii) -> long long { return (long long)wrap(jj, geo.ny) * geo.nx + wrap(ii, geo.nx); };
  const T idx_ = T(geo.idx), idy_ = T(geo.idy);
  // jumps, denominators, sigma per component
  T jx[NC][2], jy[NC][2], Dn[NC], sxc[NC], syc[NC];
  int pstar[NC];
  T sgnp[NC];
  bool act[NC];
  T lam[NC][9];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    jx[c][0] = TRC[(long long)(0 * NC + c) * n + cell] - TRC[(long long)(1 * NC + c) * n + at(j, i - 1)];
    jx[c][1] = TRC[(long long)(0 * NC + c) * n + at(j, i + 1)] - TRC[(long long)(1 * NC + c) * n + cell];
    jy[c][0] = TRC[(long long)(2 * NC + c) * n + cell] - TRC[(long long)(3 * NC + c) * n + at(j - 1, i)];
    jy[c][1] = TRC[(long long)(2 * NC + c) * n + at(j + 1, i)] - TRC[(long long)(3 * NC + c) * n + cell];
    T S = T(0), mabs = T(0);
#pragma unroll
    for (int s = 0; s < 9; ++s) {
      lam[c][s] = U[cell_index(geo, c * 3, j + s / 3 - 1, i + s % 3 - 1)];
      S += lam[c][s];
      mabs = fmax(mabs, fabs(lam[c][s]));
    }
    T d = T(-1);
    int ps = 0;
#pragma unroll
    for (int s = 0; s < 9; ++s) {
      const T t = fabs(lam[c][s] - S);
      if (t > d) { d = t; ps = s; }
    }
    Dn[c] = d;
    pstar[c] = ps;
    sgnp[c] = (lam[c][ps] - S) >= T(0) ? T(1) : T(-1);
    act[c] = !(d < T(1e-14) * fmax(mabs, T(1)));
    const T gd = act[c] ? gamma_k * Fast<T>::rcp(d) : T(0);
    sxc[c] = act[c] ? gd * (fabs(jx[c][0]) + fabs(jx[c][1])) : T(0);
    syc[c] = act[c] ? gd * (fabs(jy[c][0]) + fabs(jy[c][1])) : T(0);
  }
  int lx = 0, ly = 0;
  T sx = T(0), sy = T(0);
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    if (sxc[c] > sx) { sx = sxc[c]; lx = c; }
    if (syc[c] > sy) { sy = syc[c]; ly = c; }
  }
  T bx = T(0), by = T(0);
  int kx = 4, ky = 4;
#pragma unroll
  for (int s = 0; s < 9; ++s) {
    const T a = SP[at(j + s / 3 - 1, i + s % 3 - 1)];
    const T b = SP[n + at(j + s / 3 - 1, i + s % 3 - 1)];
    if (a > bx) { bx = a; kx = s; }
    if (b > by) { by = b; ky = s; }
  }
  const T theta = bx * dt * sx * idx_ + by * dt * sy * idy_;
  const T delta = exp(-theta);
  // g = dJ/dtheta = -delta sum lambda_mom * mom
  T gth = T(0);
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int m = 1; m < 3; ++m) {
      const long long o = (long long)(c * 3 + m) * n + cell;
      gth = fma(LAM[o], U[cell_index(geo, c * 3 + m, j, i)], gth);
      OUT[o] = delta * LAM[o];
    }
  gth = -delta * gth;
  const T sxb = gth * bx * dt * idx_, syb = gth * by * dt * idy_;
  const T bxb = gth * dt * sx * idx_, byb = gth * dt * sy * idy_;
  T jb[4][NC];
  T avb[9][NC];
#pragma unroll
  for (int f = 0; f < 4; ++f)
#pragma unroll
    for (int c = 0; c < NC; ++c) jb[f][c] = T(0);
#pragma unroll
  for (int s = 0; s < 9; ++s)
#pragma unroll
    for (int c = 0; c < NC; ++c) avb[s][c] = T(0);
  T Db[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) Db[c] = T(0);
  if (sx > T(0)) {
    const int c = lx;
    const T iD = Fast<T>::rcp(Dn[c]);
    const T k = sxb * gamma_k * iD;
    jb[0][c] += k * (jx[c][0] > T(0) ? T(1) : (jx[c][0] < T(0) ? T(-1) : T(0)));
    jb[1][c] += k * (jx[c][1] > T(0) ? T(1) : (jx[c][1] < T(0) ? T(-1) : T(0)));
    Db[c] -= sxb * sx * iD;
  }
  if (sy > T(0)) {
    const int c = ly;
    const T iD = Fast<T>::rcp(Dn[c]);
    const T k = syb * gamma_k * iD;
    jb[2][c] += k * (jy[c][0] > T(0) ? T(1) : (jy[c][0] < T(0) ? T(-1) : T(0)));
    jb[3][c] += k * (jy[c][1] > T(0) ? T(1) : (jy[c][1] < T(0) ? T(-1) : T(0)));
    Db[c] -= syb * sy * iD;
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    if (Db[c] != T(0)) {
      const T t = Db[c] * sgnp[c];
      avb[pstar[c]][c] += t;
#pragma unroll
      for (int s = 0; s < 9; ++s) avb[s][c] -= t;
    }
  }
  if (bxb != T(0) && sx > T(0)) {
    T u[NC], gr[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) u[c] = lam[c][kx];
    ph.speed_grad(0, u, gr);
#pragma unroll
    for (int c = 0; c < NC; ++c) avb[kx][c] += bxb * gr[c];
  }
  if (byb != T(0) && sy > T(0)) {
    T u[NC], gr[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) u[c] = lam[c][ky];
    ph.speed_grad(1, u, gr);
#pragma unroll
    for (int c = 0; c < NC; ++c) avb[ky][c] += byb * gr[c];
  }
#pragma unroll
  for (int f = 0; f < 4; ++f)
#pragma unroll
    for (int c = 0; c < NC; ++c) JB[(long long)(f * NC + c) * n + cell] = jb[f][c];
#pragma unroll
  for (int s = 0; s < 9; ++s)
#pragma unroll
    for (int c = 0; c < NC; ++c) AVB[(long long)(s * NC + c) * n + cell] = avb[s][c];
}

// trace cotangents from the jump cotangents -> patch cotangents PB
template <typename T, int K, int NC>
__global__ void adj_oe_traces(const Geo geo, const T* __restrict__ JB, int q6, T* __restrict__ PB) {
  const long long n = (long long)geo.nx * geo.ny;
  const long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (cell >= n) return;
  const int i = (int)(cell % geo.nx), j = (int)(cell / geo.nx);
  auto at = [&](int jj, int ii) -> long long { return (long long)wrap(jj, geo.ny) * geo.nx + wrap(ii, geo.nx); };
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    auto J = [&](int f, long long q) -> T { return JB[(long long)(f * NC + c) * n + q]; };
    T tb[4];
    // xm(c) in Jxl(c) (+) and Jxr(c-1) (+); xp(c) in Jxr(c) (-) and Jxl(c+1) (-)
    tb[0] = J(0, cell) + J(1, at(j, i - 1));
    tb[1] = -(J(1, cell) + J(0, at(j, i + 1)));
    tb[2] = J(2, cell) + J(3, at(j - 1, i));
    tb[3] = -(J(3, cell) + J(2, at(j + 1, i)));
    T gp[27];
    RT<K>::facecT(tb, gp, q6);
#pragma unroll
    for (int s = 0; s < 9; ++s)
#pragma unroll
      for (int m = 0; m < 3; ++m) PB[(long long)((s * 3 + m) * NC + c) * n + cell] = gp[m * 9 + s];
  }
}

// final OE transpose: out += avg cotangent + gathered average contributions + patch gathers
template <typename T, int NC>
__global__ void adj_oe_gather(const T* __restrict__ PB, const T* __restrict__ AVB, const T* __restrict__ LAM,
                              const Geo geo, T* __restrict__ OUT) {
  const long long n = (long long)geo.nx * geo.ny;
  const long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (cell >= n) return;
  const int i = (int)(cell % geo.nx), j = (int)(cell / geo.nx);
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      T r = m == 0 ? LAM[(long long)(c * 3) * n + cell] : OUT[(long long)(c * 3 + m) * n + cell];
#pragma unroll
      for (int s = 0; s < 9; ++s) {
        const int jj = wrap(j - (s / 3 - 1), geo.ny), ii = wrap(i - (s % 3 - 1), geo.nx);
        const long long q = (long long)jj * geo.nx + ii;
        r += PB[(long long)((s * 3 + m) * NC + c) * n + q];
        if (m == 0) r += AVB[(long long)(s * NC + c) * n + q];
      }
      OUT[(long long)(c * 3 + m) * n + cell] = r;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------
struct AdjBuffers {
  size_t ncells = 0, bytes_state = 0;
  std::vector<void*> ckpt, seg;  // padded states
  double *lam = nullptr, *acc = nullptr, *tmp = nullptr;
  double *TR = nullptr, *PB = nullptr, *TRC = nullptr, *SP = nullptr, *JB = nullptr, *AVB = nullptr;
  void release() {
    for (void* p : ckpt) cudaFree(p);
    for (void* p : seg) cudaFree(p);
    ckpt.clear();
    seg.clear();
    for (double** p : {&lam, &acc, &tmp, &TR, &PB, &TRC, &SP, &JB, &AVB})
      if (*p) { cudaFree(*p); *p = nullptr; }
  }
};

template <int K>
static cudaError_t adj_step(fam_handle* h, AdjBuffers& B, const void* const* S /*U0..U3*/, double dt) {
  using PH = Euler2D<double>;
  PH ph{h->gamma, h->gamma - 1.0, 0.5 * (h->gamma - 1.0)};
  const Geo geo = h->geo;
  const long long n = (long long)geo.nx * geo.ny;
  const int bs = 128;
  const int grid = (int)((n + bs - 1) / bs);
  const double gk = h->gamma_k > 0.0 ? h->gamma_k : (K <= 4 ? 25.0 : 15.0);
  const double* U3 = reinterpret_cast<const double*>(S[3]);
  const size_t adj_res_smem = sizeof(double) * 32 * PH::NC * kAdjBS;  // 64 KB: above the default 48 KB
  {
    // per call (cheap), so that it holds on whichever device is current
    cudaError_t ea = cudaFuncSetAttribute(adj_residual_local<double, K, PH>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)adj_res_smem);
    if (ea != cudaSuccess) return ea;
  }
  // OE transpose: lam (post-OE) -> tmp (pre-OE)
  adj_oe_prep<double, K, PH><<<grid, bs, 0, h->stream>>>(U3, geo, ph, h->oe_q6, B.TRC, B.SP);
  adj_oe_local<double, K, PH><<<grid, bs, 0, h->stream>>>(U3, geo, ph, B.TRC, B.SP, B.lam, dt, gk, B.JB, B.AVB,
                                                          B.tmp);
  adj_oe_traces<double, K, 4><<<grid, bs, 0, h->stream>>>(geo, B.JB, h->oe_q6, B.PB);
  adj_oe_gather<double, 4><<<grid, bs, 0, h->stream>>>(B.PB, B.AVB, B.lam, geo, B.tmp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (h->oe_type == 0) {  // no OE: the transpose is the identity
    e = cudaMemcpyAsync(B.tmp, B.lam, sizeof(double) * n * 12, cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) return e;
  }
  // stages 3, 2, 1: v = tmp (cotangent of the stage output)
  e = cudaMemsetAsync(B.acc, 0, sizeof(double) * n * 12, h->stream);
  if (e != cudaSuccess) return e;
  const double w0s[4] = {0, 0.0, 0.75, 1.0 / 3.0}, w1s[4] = {0, 1.0, 0.25, 2.0 / 3.0};
  for (int s = 3; s >= 1; --s) {
    const double* Us = reinterpret_cast<const double*>(S[s - 1]);
    adj_traces<double, K, PH><<<grid, bs, 0, h->stream>>>(Us, geo, B.TR);
    adj_residual_local<double, K, PH><<<(int)((n + kAdjBS - 1) / kAdjBS), kAdjBS, adj_res_smem, h->stream>>>(
        Us, geo, B.TR, B.tmp, ph, B.PB);
    // out_in goes to lam (reused as the next v); acc collects U^n cotangents
    adj_gather<double, 4><<<grid, bs, 0, h->stream>>>(B.PB, B.tmp, geo, dt, w0s[s], w1s[s], s, B.lam, B.acc);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (s > 1) std::swap(B.lam, B.tmp);
  }
  // cotangent of the state before the step
  std::swap(B.lam, B.acc);
  return cudaSuccess;
}

static cudaError_t adj_dispatch(fam_handle* h, AdjBuffers& B, const void* const* S, double dt) {
  switch (h->k) {
    case 3: return adj_step<3>(h, B, S, dt);
    case 4: return adj_step<4>(h, B, S, dt);
    case 5: return adj_step<5>(h, B, S, dt);
    default: return adj_step<6>(h, B, S, dt);
  }
}

// padded <-> unpadded copies of the 12 planes
static cudaError_t copy_planes(fam_handle* h, void* dst, const void* src, bool to_padded, cudaMemcpyKind kind) {
  const Geo& g = h->geo;
  const size_t row = (size_t)g.nx * 8;
  for (int p = 0; p < h->np; ++p) {
    char* pad = nullptr;
    const char* cpad = nullptr;
    const size_t off = ((size_t)p * g.plane + (size_t)G * g.px + G) * 8;
    if (to_padded) {
      pad = reinterpret_cast<char*>(dst) + off;
      cudaError_t e = cudaMemcpy2DAsync(pad, (size_t)g.px * 8, reinterpret_cast<const char*>(src) + p * row * g.ny,
                                        row, row, g.ny, kind, h->stream);
      if (e != cudaSuccess) return e;
    } else {
      cpad = reinterpret_cast<const char*>(src) + off;
      cudaError_t e = cudaMemcpy2DAsync(reinterpret_cast<char*>(dst) + p * row * g.ny, row, cpad, (size_t)g.px * 8,
                                        row, g.ny, kind, h->stream);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}


extern "C" fam_status fam_adjoint(fam_t h, long nsteps, double cfl, int ckpt_every, const void* U0,
                                  const void* dJdUT, void* dJdU0, int on_device) {
  if (!h || !U0 || !dJdUT || !dJdU0) return FAM_E_INVAL;
  bool periodic = true;
  for (int q = 0; q < 4; ++q) periodic = periodic && h->geo.bc[q] == kBcPeriodic;
  if (h->d != 2 || h->eq != FAM_EULER || h->prec != 64 || !periodic || h->pp)
    return fail(h, FAM_E_UNSUPPORTED, "the adjoint is built for 2D Euler, FP64, periodic grids, without the BP/PP safeguard");
  if (nsteps < 1 || ckpt_every < 1) return fail(h, FAM_E_INVAL, "nsteps and ckpt_every must be >= 1");
  const Geo& g = h->geo;
  const long long n = (long long)g.nx * g.ny;
  const size_t sb = h->buf_elems * 8;
  AdjBuffers B;
  auto bail = [&](fam_status s, const std::string& m) {
    cudaStreamSynchronize(h->stream);
    B.release();
    return fail(h, s, m);
  };
  const long nck = (nsteps + ckpt_every - 1) / ckpt_every;
  for (long q = 0; q < nck; ++q) {
    void* p = nullptr;
    if (cudaMalloc(&p, sb) != cudaSuccess) return bail(FAM_E_NOMEM, "checkpoint allocation");
    B.ckpt.push_back(p);
  }
  for (long q = 0; q < 4 * (long)ckpt_every; ++q) {
    void* p = nullptr;
    if (cudaMalloc(&p, sb) != cudaSuccess) return bail(FAM_E_NOMEM, "segment allocation");
    B.seg.push_back(p);
  }
  const size_t sn = sizeof(double) * (size_t)n;
  if (cudaMalloc(&B.lam, 12 * sn) || cudaMalloc(&B.acc, 12 * sn) || cudaMalloc(&B.tmp, 12 * sn) ||
      cudaMalloc(&B.TR, 64 * sn) || cudaMalloc(&B.PB, 108 * sn) || cudaMalloc(&B.TRC, 16 * sn) ||
      cudaMalloc(&B.SP, 2 * sn) || cudaMalloc(&B.JB, 16 * sn) || cudaMalloc(&B.AVB, 36 * sn))
    return bail(FAM_E_NOMEM, "adjoint work buffers");
  // forward run with checkpoints; record the step sizes
  fam_status s = fam_set_state(h, U0, on_device);
  if (s) return bail(s, h->err);
  s = refresh_dt_public(h, cfl);
  if (s) return bail(s, h->err);
  std::vector<double> dts(nsteps);
  for (long q = 0; q < nsteps; ++q) {
    FamCtl c;
    if (cudaMemcpyAsync(&c, h->ctl, sizeof(c), cudaMemcpyDeviceToHost, h->stream) ||
        cudaStreamSynchronize(h->stream))
      return bail(FAM_E_CUDA, "control block read");
    dts[q] = c.dt;
    if (q % ckpt_every == 0 &&
        cudaMemcpyAsync(B.ckpt[q / ckpt_every], h->buf[0], sb, cudaMemcpyDeviceToDevice, h->stream))
      return bail(FAM_E_CUDA, "checkpoint copy");
    s = fam_internal_step_fixed_dt(h, dts[q], nullptr);
    if (s) return bail(s, h->err);
  }
  // reverse sweep
  const cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  for (int p = 0; p < 12; ++p)
    if (cudaMemcpyAsync(B.lam + p * n, reinterpret_cast<const char*>(dJdUT) + p * sn, sn, kin, h->stream))
      return bail(FAM_E_CUDA, "cotangent upload");
  std::vector<double> save_state;
  void* final_state = nullptr;
  if (cudaMalloc(&final_state, sb)) return bail(FAM_E_NOMEM, "final state");
  cudaMemcpyAsync(final_state, h->buf[0], sb, cudaMemcpyDeviceToDevice, h->stream);
  for (long seg = nck - 1; seg >= 0; --seg) {
    const long q0 = seg * ckpt_every, q1 = std::min(nsteps, q0 + ckpt_every);
    cudaMemcpyAsync(h->buf[0], B.ckpt[seg], sb, cudaMemcpyDeviceToDevice, h->stream);
    for (long q = q0; q < q1; ++q) {
      void* st[4] = {B.seg[4 * (q - q0) + 0], B.seg[4 * (q - q0) + 1], B.seg[4 * (q - q0) + 2],
                     B.seg[4 * (q - q0) + 3]};
      s = fam_internal_step_fixed_dt(h, dts[q], st);
      if (s) { cudaFree(final_state); return bail(s, h->err); }
    }
    for (long q = q1 - 1; q >= q0; --q) {
      const void* st[4] = {B.seg[4 * (q - q0) + 0], B.seg[4 * (q - q0) + 1], B.seg[4 * (q - q0) + 2],
                           B.seg[4 * (q - q0) + 3]};
      if (adj_dispatch(h, B, st, dts[q]) != cudaSuccess) { cudaFree(final_state); return bail(FAM_E_CUDA, "adjoint kernels"); }
    }
  }
  const cudaMemcpyKind kout = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  for (int p = 0; p < 12; ++p)
    if (cudaMemcpyAsync(reinterpret_cast<char*>(dJdU0) + p * sn, B.lam + p * n, sn, kout, h->stream)) {
      cudaFree(final_state);
      return bail(FAM_E_CUDA, "gradient download");
    }
  cudaMemcpyAsync(h->buf[0], final_state, sb, cudaMemcpyDeviceToDevice, h->stream);
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
    cudaFree(final_state);
    return bail(FAM_E_CUDA, "adjoint synchronisation");
  }
  cudaFree(final_state);
  B.release();
  return FAM_OK;
}
