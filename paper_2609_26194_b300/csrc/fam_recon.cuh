// fam_recon.cuh -- evaluation of the FAM reconstructions at the points the
// kernels need (Gauss points of the volume and face integrals, face traces).
//
// The coefficients come from fam_recon_gen.cuh (derived from the moment
// systems of Sec. 2.4).  Polynomials are held in the tensor Legendre basis
// P_a(xi) P_b(eta) with P_a monic orthogonal on [-1/2,1/2]; since
// P_a(-x) = (-1)^a P_a(x), a value pair at +x and -x costs one even and one
// odd partial sum (sum factorisation with symmetric pairs).  The product
// opening each odd sum runs on the integer pipes (pmul: bit-identical to the
// FP64 unit's), beside the FP64 unit's multiply-adds.
#pragma once

#include "fam_common.cuh"
#include "fam_recon_gen.cuh"

namespace fam {

// Rows of famgen::kLegAt: P_a at the inner Gauss node, the outer Gauss node,
// at 1/2, at 0, and at the interior node 1/(2 sqrt 5) of the 4-point
// Gauss--Lobatto rule.  Gauss nodes ascending: {-outer, -inner, +inner, +outer}.
enum { kRowInner = 0, kRowOuter = 1, kRowHalf = 2, kRowZero = 3, kRowLobatto = 4 };

__host__ __device__ constexpr int cidx(int a, int b) { return (a + b) * (a + b + 1) / 2 + a; }

// Value pair of sum_a d[a] P_a(x) at x = +node(ROW) and x = -node(ROW).
template <typename T, int D, int ROW>
__device__ __forceinline__ void sym_pair(const T* d, T& vp, T& vm) {
  T e = d[0];
  T o = T(0);
#pragma unroll
  for (int a = 1; a <= D; ++a) {
    const T L = T(famgen::kLegAt[ROW][a]);
    if (a & 1)
      o = (a == 1) ? pmul(d[a], L) : fma(d[a], L, o);
    else
      e = fma(d[a], L, e);
  }
  if (D >= 1) {
    vp = e + o;
    vm = e - o;
  } else {
    vp = vm = e;
  }
}

// 2D: partial sums over eta at eta = +/- node(ROW): dp[a] = sum_b c_ab P_b(+y).
// c is anything indexable by the coefficient index (an array, a pointer, a
// strided view of shared memory).
template <typename T, int D, int ROW, typename C>
__device__ __forceinline__ void eta_pair(const C& c, T* dp, T* dm) {
#pragma unroll
  for (int a = 0; a <= D; ++a) {
    T e = c[cidx(a, 0)];
    T o = T(0);
    bool odd = false;
#pragma unroll
    for (int b = 1; a + b <= D; ++b) {
      const T L = T(famgen::kLegAt[ROW][b]);
      if (b & 1) {
        o = odd ? fma(c[cidx(a, b)], L, o) : pmul(c[cidx(a, b)], L);
        odd = true;
      } else {
        e = fma(c[cidx(a, b)], L, e);
      }
    }
    if (odd) {
      dp[a] = e + o;
      dm[a] = e - o;
    } else {
      dp[a] = dm[a] = e;
    }
  }
}

// Transposes (for the adjoint): given the cotangents vpb, vmb of the pair
// (vp, vm) of sym_pair, accumulate the cotangents of d; given dpb, dmb of
// eta_pair's outputs, accumulate the cotangents of the coefficients c.
template <typename T, int D, int ROW>
__device__ __forceinline__ void sym_pair_T(T vpb, T vmb, T* db) {
  const T e = vpb + vmb, o = vpb - vmb;
  db[0] += e;
#pragma unroll
  for (int a = 1; a <= D; ++a) db[a] = fma(T(famgen::kLegAt[ROW][a]), (a & 1) ? o : e, db[a]);
}

template <typename T, int D, int ROW>
__device__ __forceinline__ void eta_pair_T(const T* dpb, const T* dmb, T* cb) {
#pragma unroll
  for (int a = 0; a <= D; ++a) {
    const T e = dpb[a] + dmb[a], o = dpb[a] - dmb[a];
    cb[cidx(a, 0)] += e;
#pragma unroll
    for (int b = 1; a + b <= D; ++b) cb[cidx(a, b)] = fma(T(famgen::kLegAt[ROW][b]), (b & 1) ? o : e, cb[cidx(a, b)]);
  }
}

// ---------------------------------------------------------------------------
// dispatch to the generated operators
// ---------------------------------------------------------------------------
template <int K> struct Recon1D;
#define FAM_RECON1D(K)                                                                             \
  template <> struct Recon1D<K> {                                                                  \
    template <typename T>                                                                          \
    static __device__ __forceinline__ void coef(T am, T a0, T ap, T mm, T m0, T mp, T* c) {        \
      fam1d_coef_k##K(am, a0, ap, mm, m0, mp, c);                                                  \
    }                                                                                              \
  };
FAM_RECON1D(3)
FAM_RECON1D(4)
FAM_RECON1D(5)
FAM_RECON1D(6)
#undef FAM_RECON1D

template <int K> struct Recon2D;
#define FAM_RECON2D(K, FC)                                                                          \
  template <> struct Recon2D<K> {                                                                   \
    static constexpr int NCOEF = K * (K + 1) / 2;                                                   \
    template <typename T>                                                                           \
    static __device__ __forceinline__ void coef(const T* A, const T* X, const T* Y, T* c) {         \
      fam2d_coef_k##K(A, X, Y, c);                                                                  \
    }                                                                                               \
    template <typename T>                                                                           \
    static __device__ __forceinline__ void tr_xm(const T* A, const T* X, const T* Y, T* t) {        \
      fam2d_tr_xm_k##K(A, X, Y, t);                                                                 \
    }                                                                                               \
    template <typename T>                                                                           \
    static __device__ __forceinline__ void tr_xp(const T* A, const T* X, const T* Y, T* t) {        \
      fam2d_tr_xp_k##K(A, X, Y, t);                                                                 \
    }                                                                                               \
    template <typename T>                                                                           \
    static __device__ __forceinline__ void tr_ym(const T* A, const T* X, const T* Y, T* t) {        \
      fam2d_tr_ym_k##K(A, X, Y, t);                                                                 \
    }                                                                                               \
    template <typename T>                                                                           \
    static __device__ __forceinline__ void tr_yp(const T* A, const T* X, const T* Y, T* t) {        \
      fam2d_tr_yp_k##K(A, X, Y, t);                                                                 \
    }                                                                                               \
    template <typename T>                                                                           \
    static __device__ __forceinline__ void facec(const T* A, const T* X, const T* Y, T* t, int q6) { \
      FC;                                                                                           \
    }                                                                                               \
  };
FAM_RECON2D(3, fam2d_facec_k3p(A, X, Y, t))
FAM_RECON2D(4, fam2d_facec_k4p(A, X, Y, t))
FAM_RECON2D(5, fam2d_facec_k5p(A, X, Y, t))
FAM_RECON2D(6, if (q6) fam2d_facec_k6q(A, X, Y, t); else fam2d_facec_k6p(A, X, Y, t))
#undef FAM_RECON2D

}  // namespace fam
