/*
 * fam_oracle.c -- plain FP64 CPU oracle of the compact FAM time step.
 *
 * TEST INFRASTRUCTURE ONLY (see fam_oracle.h).  Written from the paper, step
 * by step, with no blocking or fusion:
 *   - reconstruction coefficients: App. B (1D) and App. I (2D), transcribed;
 *   - semi-discrete residual: eq. (1dSemi) in 1D, eq. (11) in 2D, with the
 *     Rusanov flux and four-point Gauss quadrature per direction (Remark in
 *     Sec. 2.3);
 *   - SSP-RK3 in Shu--Osher form: eq. (3) / eq. (12);
 *   - end-of-step OE: eq. (9) and Tab. sigma1d (1D), eq. (2dOE_sol) and
 *     Tab. sigma2d (2D), system forms eq. (1dOE_system) / eq. (2dOE_system);
 *     interface jumps are evaluated from the reconstructed polynomials;
 *   - time step: Sec. 4, "Time stepping".
 * Readings where the paper is not explicit are listed where they are used.
 */
#include "fam_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define G 4 /* ghost layers held by the padded work arrays */

int or_ncomp(const or_problem* P) { return P->eq == OR_EULER ? P->d + 2 : 1; }
int or_nmom(const or_problem* P) { return P->d + 1; }

/* ------------------------------------------------------------------ */
/* Bases (App. B, App. I) and Gauss rule                               */
/* ------------------------------------------------------------------ */

static double leg2(double t) { return t * t - 1.0 / 12.0; }
static double leg3(double t) { return t * t * t - 3.0 / 20.0 * t; }
static double leg4(double t) { return t * t * t * t - 3.0 / 14.0 * t * t + 3.0 / 560.0; }
static double leg5(double t) {
  return t * t * t * t * t - 5.0 / 18.0 * t * t * t + 5.0 / 336.0 * t;
}

double or_basis1d(int l, double xi) {
  switch (l) {
    case 0: return 1.0;
    case 1: return xi;
    case 2: return leg2(xi);
    case 3: return leg3(xi);
    case 4: return leg4(xi);
    case 5: return leg5(xi);
  }
  return 0.0;
}

double or_basis2d(int l, double x, double y) {
  switch (l) {
    case 0: return 1.0;
    case 1: return x;
    case 2: return y;
    case 3: return leg2(x);
    case 4: return x * y;
    case 5: return leg2(y);
    case 6: return leg3(x);
    case 7: return leg2(x) * y;
    case 8: return x * leg2(y);
    case 9: return leg3(y);
    case 10: return leg2(x) * leg2(y);
    case 11: return leg4(x);
    case 12: return leg3(x) * y;
    case 13: return x * leg3(y);
    case 14: return leg4(y);
    case 15: return leg5(x);
    case 16: return leg4(x) * y;
    case 17: return leg3(x) * leg2(y);
    case 18: return leg2(x) * leg3(y);
    case 19: return x * leg4(y);
    case 20: return leg5(y);
    case 21: return leg4(x) * leg2(y);
    case 22: return leg2(x) * leg4(y);
  }
  return 0.0;
}

double or_eval1d(int ncoef, const double* c, double xi) {
  double s = 0.0;
  for (int l = 0; l < ncoef; ++l) s += c[l] * or_basis1d(l, xi);
  return s;
}

double or_eval2d(int ncoef, const double* c, double xi, double eta) {
  double s = 0.0;
  for (int l = 0; l < ncoef; ++l) s += c[l] * or_basis2d(l, xi, eta);
  return s;
}

/* Nodes +-sqrt(3/7 -+ (2/7) sqrt(6/5)) on [-1,1], mapped to [-1/2,1/2];
 * weights (18 +- sqrt(30))/36 halved so that they sum to one. */
void or_gauss4(double node[4], double weight[4]) {
  double a = sqrt(3.0 / 7.0 - 2.0 / 7.0 * sqrt(6.0 / 5.0));
  double b = sqrt(3.0 / 7.0 + 2.0 / 7.0 * sqrt(6.0 / 5.0));
  double wa = (18.0 + sqrt(30.0)) / 72.0;
  double wb = (18.0 - sqrt(30.0)) / 72.0;
  node[0] = -0.5 * b; weight[0] = wb;
  node[1] = -0.5 * a; weight[1] = wa;
  node[2] = 0.5 * a;  weight[2] = wa;
  node[3] = 0.5 * b;  weight[3] = wb;
}

/* ------------------------------------------------------------------ */
/* Reconstructions                                                      */
/* ------------------------------------------------------------------ */

/* App. B.  um/u0/up = (average, scaled moment) of cells i-1, i, i+1. */
int or_recon1d(int k, const double um[2], const double u0[2], const double up[2], double c[6]) {
  for (int l = 0; l < 6; ++l) c[l] = 0.0;
  double a_m = um[0], a_0 = u0[0], a_p = up[0];
  double m_m = um[1], m_0 = u0[1], m_p = up[1];
  c[0] = a_0;
  c[1] = 12.0 * m_0;
  if (k == 3 || k == 4) {
    /* cubic auxiliary Q, eq. (5) */
    c[2] = 0.5 * (a_m - 2.0 * a_0 + a_p);
    c[3] = 5.0 / 11.0 * (a_p - a_m) - 120.0 / 11.0 * m_0;
  } else {
    /* quintic auxiliary Q, eq. (6) */
    c[2] = 73.0 / 56.0 * (a_m - 2.0 * a_0 + a_p) + 135.0 / 28.0 * (m_m - m_p);
    c[3] = 595.0 / 324.0 * (a_p - a_m) - 985.0 / 162.0 * (m_m + m_p) - 2585.0 / 81.0 * m_0;
    c[4] = -5.0 / 8.0 * (a_m - 2.0 * a_0 + a_p) - 15.0 / 4.0 * (m_m - m_p);
    c[5] = 35.0 / 36.0 * (a_m - a_p) + 77.0 / 18.0 * (m_m + m_p) + 133.0 / 9.0 * m_0;
  }
  return k; /* p_{k-1} uses c_0 .. c_{k-1} */
}

/* App. I.  a, mx, my: averages, x-moments and y-moments of the 3x3 patch
 * numbered I1..I9 row by row from (i-1,j-1) (index 0) to (i+1,j+1) (index 8). */
int or_recon2d(int k, const double a[9], const double mx[9], const double my[9], double c[23]) {
  for (int l = 0; l < 23; ++l) c[l] = 0.0;
  /* 1-based names as in the paper */
  double u1 = a[0], u2 = a[1], u3 = a[2], u4 = a[3], u5 = a[4], u6 = a[5], u7 = a[6], u8 = a[7], u9 = a[8];
  double x1 = mx[0], x2 = mx[1], x3 = mx[2], x4 = mx[3], x5 = mx[4], x6 = mx[5], x7 = mx[6], x8 = mx[7],
         x9 = mx[8];
  double y1 = my[0], y2 = my[1], y3 = my[2], y4 = my[3], y5 = my[4], y6 = my[5], y7 = my[6], y8 = my[7],
         y9 = my[8];
  (void)x2; (void)x8; (void)y4; (void)y6;
  c[0] = u5;
  c[1] = 12.0 * x5;
  c[2] = 12.0 * y5;
  if (k == 3 || k == 4) {
    /* incomplete quartic Q4, eq. (Qxy_quartic) */
    c[3] = 0.5 * (u4 - 2.0 * u5 + u6);
    c[4] = 0.25 * (u1 - u3 - u7 + u9);
    c[5] = 0.5 * (u2 - 2.0 * u5 + u8);
    c[6] = 5.0 / 11.0 * (-u4 + u6) - 120.0 / 11.0 * x5;
    c[7] = 0.25 * (-u1 + 2.0 * u2 - u3 + u7 - 2.0 * u8 + u9);
    c[8] = 0.25 * (-u1 + u3 + 2.0 * u4 - 2.0 * u6 - u7 + u9);
    c[9] = 5.0 / 11.0 * (-u2 + u8) - 120.0 / 11.0 * y5;
    c[10] = 0.25 * (u1 - 2.0 * u2 + u3 - 2.0 * u4 + 4.0 * u5 - 2.0 * u6 + u7 - 2.0 * u8 + u9);
    return k == 3 ? 6 : 10;
  }
  /* incomplete degree-six Q6, eq. (Qxy_quintic) */
  c[3] = 73.0 / 56.0 * (u4 - 2.0 * u5 + u6) + 135.0 / 28.0 * (x4 - x6);
  c[4] = 41.0 / 76.0 * (u1 - u3 - u7 + u9) + 33.0 / 19.0 * (x1 + x3 - x7 - x9 + y1 - y3 + y7 - y9);
  c[5] = 73.0 / 56.0 * (u2 - 2.0 * u5 + u8) + 135.0 / 28.0 * (y2 - y8);
  c[6] = 595.0 / 324.0 * (-u4 + u6) - 985.0 / 162.0 * (x4 + x6) - 2585.0 / 81.0 * x5;
  c[7] = 1695.0 / 2128.0 * (-u1 + 2.0 * u2 - u3 + u7 - 2.0 * u8 + u9) +
         135.0 / 56.0 * (-x1 + x3 + x7 - x9) +
         33.0 / 19.0 * (-y1 + 2.0 * y2 - y3 - y7 + 2.0 * y8 - y9);
  c[8] = 1695.0 / 2128.0 * (-u1 + u3 + 2.0 * u4 - 2.0 * u6 - u7 + u9) +
         33.0 / 19.0 * (-x1 - x3 + 2.0 * x4 + 2.0 * x6 - x7 - x9) +
         135.0 / 56.0 * (-y1 + y3 + y7 - y9);
  c[9] = 595.0 / 324.0 * (-u2 + u8) - 985.0 / 162.0 * (y2 + y8) - 2585.0 / 81.0 * y5;
  c[10] = 59.0 / 56.0 * (u1 - 2.0 * u2 + u3 - 2.0 * u4 + 4.0 * u5 - 2.0 * u6 + u7 - 2.0 * u8 + u9) +
          135.0 / 56.0 * (x1 - x3 - 2.0 * x4 + 2.0 * x6 + x7 - x9 + y1 - 2.0 * y2 + y3 - y7 + 2.0 * y8 - y9);
  c[11] = 5.0 / 8.0 * (-u4 + 2.0 * u5 - u6) + 15.0 / 4.0 * (-x4 + x6);
  c[12] = 5.0 / 38.0 * (-u1 + u3 + u7 - u9) + 30.0 / 19.0 * (-x1 - x3 + x7 + x9);
  c[13] = 5.0 / 38.0 * (-u1 + u3 + u7 - u9) + 30.0 / 19.0 * (-y1 + y3 - y7 + y9);
  c[14] = 5.0 / 8.0 * (-u2 + 2.0 * u5 - u8) + 15.0 / 4.0 * (-y2 + y8);
  c[15] = 35.0 / 36.0 * (u4 - u6) + 77.0 / 18.0 * (x4 + x6) + 133.0 / 9.0 * x5;
  c[16] = 5.0 / 16.0 * (u1 - 2.0 * u2 + u3 - u7 + 2.0 * u8 - u9) + 15.0 / 8.0 * (x1 - x3 - x7 + x9);
  c[17] = 5.0 / 38.0 * (u1 - u3 - 2.0 * u4 + 2.0 * u6 + u7 - u9) +
          30.0 / 19.0 * (x1 + x3 - 2.0 * x4 - 2.0 * x6 + x7 + x9);
  c[18] = 5.0 / 38.0 * (u1 - 2.0 * u2 + u3 - u7 + 2.0 * u8 - u9) +
          30.0 / 19.0 * (y1 - 2.0 * y2 + y3 + y7 - 2.0 * y8 + y9);
  c[19] = 5.0 / 16.0 * (u1 - u3 - 2.0 * u4 + 2.0 * u6 + u7 - u9) + 15.0 / 8.0 * (y1 - y3 - y7 + y9);
  c[20] = 35.0 / 36.0 * (u2 - u8) + 77.0 / 18.0 * (y2 + y8) + 133.0 / 9.0 * y5;
  c[21] = 5.0 / 16.0 * (-u1 + 2.0 * u2 - u3 + 2.0 * u4 - 4.0 * u5 + 2.0 * u6 - u7 + 2.0 * u8 - u9) +
          15.0 / 8.0 * (-x1 + x3 + 2.0 * x4 - 2.0 * x6 - x7 + x9);
  c[22] = 5.0 / 16.0 * (-u1 + 2.0 * u2 - u3 + 2.0 * u4 - 4.0 * u5 + 2.0 * u6 - u7 + 2.0 * u8 - u9) +
          15.0 / 8.0 * (-y1 + 2.0 * y2 - y3 + y7 - 2.0 * y8 + y9);
  return k == 5 ? 15 : 21;
}

/* ------------------------------------------------------------------ */
/* Physics: fluxes and spectral radii                                   */
/* ------------------------------------------------------------------ */

/* Flux in direction dir (0 = x, 1 = y) and spectral radius of its Jacobian. */
static void phys_flux(const or_problem* P, int dir, const double* u, double* f) {
  if (P->eq == OR_ADVECTION) {
    f[0] = (dir == 0 ? P->ax : P->ay) * u[0];
    return;
  }
  if (P->eq == OR_BURGERS) {
    f[0] = 0.5 * u[0] * u[0];
    return;
  }
  if (P->eq == OR_BUCKLEY) {  /* Example 4.3: f = 4 u^2 / (4 u^2 + (1 - u)^2) */
    const double a = 4.0 * u[0] * u[0], b = (1.0 - u[0]) * (1.0 - u[0]);
    f[0] = a / (a + b);
    return;
  }
  double g = P->gamma;
  if (P->d == 1) {
    double rho = u[0], mom = u[1], E = u[2];
    double vel = mom / rho;
    double p = (g - 1.0) * (E - 0.5 * mom * vel);
    f[0] = mom;
    f[1] = mom * vel + p;
    f[2] = (E + p) * vel;
    return;
  }
  double rho = u[0], mu = u[1], mv = u[2], E = u[3];
  double vx = mu / rho, vy = mv / rho;
  double p = (g - 1.0) * (E - 0.5 * (mu * vx + mv * vy));
  double vn = dir == 0 ? vx : vy;
  f[0] = rho * vn;
  f[1] = mu * vn + (dir == 0 ? p : 0.0);
  f[2] = mv * vn + (dir == 1 ? p : 0.0);
  f[3] = (E + p) * vn;
}

static double phys_speed(const or_problem* P, int dir, const double* u) {
  if (P->eq == OR_ADVECTION) return fabs(dir == 0 ? P->ax : P->ay);
  if (P->eq == OR_BURGERS) return fabs(u[0]);
  /* Buckley-Leverett: f'(u) = 8 u (1 - u) / (5 u^2 - 2 u + 1)^2 vanishes at
   * u = 0 and 1, the states of the initial data, so every speed the method
   * takes (Rusanov, OE beta, time step) is the bound max |f'| over all u,
   * f'(u*) with u* the root in (0, 1) of 10 u^3 - 15 u^2 + 1 = 0 (where
   * f'' = 0; |f'| -> 0 as |u| -> infinity and is smaller at the other two
   * roots), a Lax-Friedrichs speed */
  if (P->eq == OR_BUCKLEY) return 2.332030375854268710378;
  double g = P->gamma;
  if (P->d == 1) {
    double rho = u[0], vel = u[1] / rho, E = u[2];
    double p = (g - 1.0) * (E - 0.5 * rho * vel * vel);
    return fabs(vel) + sqrt(g * p / rho);
  }
  double rho = u[0], vx = u[1] / rho, vy = u[2] / rho, E = u[3];
  double p = (g - 1.0) * (E - 0.5 * rho * (vx * vx + vy * vy));
  double c = sqrt(g * p / rho);
  return fabs(dir == 0 ? vx : vy) + c;
}

/* Rusanov / local Lax-Friedrichs flux; the wave speed is the larger spectral
 * radius of the two one-sided traces (reading of "Rusanov flux").  A trace
 * with rho <= 0 or p <= 0 (possible without the paper's positivity limiter,
 * while the averages stay admissible) has no spectral radius (NaN): the
 * larger radius is then the other trace's, as IEEE maxNum (C fmax) gives. */
static int llf(const or_problem* P, int dir, const double* uL, const double* uR, double* fh) {
  int nc = or_ncomp(P);
  double fL[4], fR[4];
  phys_flux(P, dir, uL, fL);
  phys_flux(P, dir, uR, fR);
  double aL = phys_speed(P, dir, uL), aR = phys_speed(P, dir, uR);
  double a = fmax(aL, aR);
  for (int c = 0; c < nc; ++c) fh[c] = 0.5 * (fL[c] + fR[c]) - 0.5 * a * (uR[c] - uL[c]);
  /* 1 when a trace has no spectral radius (counted by the residuals) */
  return isnan(aL) || isnan(aR);
}

/* Face quadrature points at which a one-sided trace had no spectral radius,
 * summed over every residual evaluation since the last or_trace_reset(). */
static long long g_nonphys_traces = 0;
long long or_trace_count(void) { return g_nonphys_traces; }
void or_trace_reset(void) { g_nonphys_traces = 0; }

/* ------------------------------------------------------------------ */
/* Ghost cells (Remark in Sec. 2.3)                                     */
/* ------------------------------------------------------------------ */

typedef struct {
  int nx, ny, nxp, nyp, gy, nc, nm;
  double* v;
} padded;

static double* pv(padded* A, int c, int m, int j, int i) {
  return &A->v[(((size_t)(c * A->nm + m) * A->nyp + (j + A->gy)) * A->nxp) + (i + G)];
}

/* Copy ghost cell (gj,gi) from interior cell (sj,si); reflect across the
 * boundary normal to direction dir when refl != 0; inflow when infl != NULL.
 * Reflection mirrors the field: the normal momentum changes sign, and the
 * moment along the normal direction changes sign (the two flips cancel for the
 * normal momentum's normal moment). */
static void ghost_from(const or_problem* P, padded* A, int gj, int gi, int sj, int si, int dir, int refl,
                       const double* infl) {
  for (int c = 0; c < A->nc; ++c)
    for (int m = 0; m < A->nm; ++m) {
      double v;
      if (infl) {
        v = (m == 0) ? infl[c] : 0.0;
      } else {
        v = *pv(A, c, m, sj, si);
        if (refl) {
          int normal_mom = (P->eq == OR_EULER) && (c == 1 + dir);
          int normal_moment = (m == 1 + dir);
          if (normal_mom != normal_moment) v = -v;
        }
      }
      *pv(A, c, m, gj, gi) = v;
    }
}

/* Centre of interior cell i (clamped to the grid) along x, of row j along y. */
static double centre_x(const or_problem* P, int i) {
  if (i < 0) i = 0;
  if (i > P->nx - 1) i = P->nx - 1;
  return P->x0 + (i + 0.5) * (P->x1 - P->x0) / P->nx;
}
static double centre_y(const or_problem* P, int j) {
  if (j < 0) j = 0;
  if (j > P->ny - 1) j = P->ny - 1;
  return P->y0 + (j + 0.5) * (P->y1 - P->y0) / P->ny;
}

/* The fixed state a ghost cell of side s holds, or NULL when the side's own
 * condition applies there: the split part of the side (along-side centre
 * below split[s]) and the front condition.  a = along-side index of the
 * ghost cell, q = its layer (0 next to the grid). */
static const double* side_state(const or_problem* P, int s, int a, int q) {
  const double along = s < 2 ? centre_y(P, a) : centre_x(P, a);
  if (P->split[s] > 0.0 && along < P->split[s]) return P->inflow[s];
  if (P->bc[s] == OR_BC_FRONT) {
    const double dy = (P->y1 - P->y0) / P->ny;
    const double y = s == 2 ? P->y0 - (q + 0.5) * dy : P->y1 + (q + 0.5) * dy;
    const double x = P->x0 + (a + 0.5) * (P->x1 - P->x0) / P->nx;  /* the ghost column's own centre */
    return x < P->front[0] + P->front[1] * y + P->front[2] * P->time ? P->inflow[s] : P->front_ahead;
  }
  return NULL;
}

static void fill_ghosts(const or_problem* P, padded* A) {
  int nx = A->nx, ny = A->ny;
  /* x-direction, interior rows */
  for (int j = 0; j < ny; ++j)
    for (int q = 0; q < G; ++q) {
      int gl = -1 - q, gr = nx + q;
      const double* fl = side_state(P, 0, j, q);
      const double* fr = side_state(P, 1, j, q);
      if (fl) ghost_from(P, A, j, gl, j, 0, 0, 0, fl);
      else switch (P->bc[0]) {
        case OR_BC_PERIODIC: ghost_from(P, A, j, gl, j, ((gl % nx) + nx) % nx, 0, 0, NULL); break;
        case OR_BC_OUTFLOW: ghost_from(P, A, j, gl, j, 0, 0, 0, NULL); break;
        case OR_BC_REFLECTIVE: ghost_from(P, A, j, gl, j, q < nx ? q : nx - 1, 0, 1, NULL); break;
        default: ghost_from(P, A, j, gl, j, 0, 0, 0, P->inflow[0]); break;
      }
      if (fr) ghost_from(P, A, j, gr, j, nx - 1, 0, 0, fr);
      else switch (P->bc[1]) {
        case OR_BC_PERIODIC: ghost_from(P, A, j, gr, j, gr % nx, 0, 0, NULL); break;
        case OR_BC_OUTFLOW: ghost_from(P, A, j, gr, j, nx - 1, 0, 0, NULL); break;
        case OR_BC_REFLECTIVE: ghost_from(P, A, j, gr, j, nx - 1 - q >= 0 ? nx - 1 - q : 0, 0, 1, NULL); break;
        default: ghost_from(P, A, j, gr, j, nx - 1, 0, 0, P->inflow[1]); break;
      }
    }
  if (P->d == 1) return;
  /* y-direction, all columns including x-ghosts */
  for (int i = -G; i < nx + G; ++i)
    for (int q = 0; q < G; ++q) {
      int gl = -1 - q, gr = ny + q;
      const double* fb = side_state(P, 2, i, q);
      const double* ft = side_state(P, 3, i, q);
      if (fb) ghost_from(P, A, gl, i, 0, i, 1, 0, fb);
      else switch (P->bc[2]) {
        case OR_BC_PERIODIC: ghost_from(P, A, gl, i, ((gl % ny) + ny) % ny, i, 1, 0, NULL); break;
        case OR_BC_OUTFLOW: ghost_from(P, A, gl, i, 0, i, 1, 0, NULL); break;
        case OR_BC_REFLECTIVE: ghost_from(P, A, gl, i, q < ny ? q : ny - 1, i, 1, 1, NULL); break;
        default: ghost_from(P, A, gl, i, 0, i, 1, 0, P->inflow[2]); break;
      }
      if (ft) ghost_from(P, A, gr, i, ny - 1, i, 1, 0, ft);
      else switch (P->bc[3]) {
        case OR_BC_PERIODIC: ghost_from(P, A, gr, i, gr % ny, i, 1, 0, NULL); break;
        case OR_BC_OUTFLOW: ghost_from(P, A, gr, i, ny - 1, i, 1, 0, NULL); break;
        case OR_BC_REFLECTIVE: ghost_from(P, A, gr, i, ny - 1 - q >= 0 ? ny - 1 - q : 0, i, 1, 1, NULL); break;
        default: ghost_from(P, A, gr, i, ny - 1, i, 1, 0, P->inflow[3]); break;
      }
    }
}

static int pad_state(const or_problem* P, const double* U, padded* A) {
  A->nx = P->nx;
  A->ny = P->d == 1 ? 1 : P->ny;
  A->gy = P->d == 1 ? 0 : G;
  A->nxp = A->nx + 2 * G;
  A->nyp = A->ny + 2 * A->gy;
  A->nc = or_ncomp(P);
  A->nm = or_nmom(P);
  A->v = (double*)calloc((size_t)A->nc * A->nm * A->nyp * A->nxp, sizeof(double));
  if (!A->v) return -1;
  for (int c = 0; c < A->nc; ++c)
    for (int m = 0; m < A->nm; ++m)
      for (int j = 0; j < A->ny; ++j)
        for (int i = 0; i < A->nx; ++i)
          *pv(A, c, m, j, i) = U[(((size_t)(c * A->nm + m) * A->ny + j) * A->nx) + i];
  fill_ghosts(P, A);
  return 0;
}

/* Reconstruction coefficients of cell (j, i) for component c. */
static int cell_coeffs(const or_problem* P, padded* A, int c, int j, int i, double* cf) {
  if (P->d == 1) {
    double um[2] = {*pv(A, c, 0, 0, i - 1), *pv(A, c, 1, 0, i - 1)};
    double u0[2] = {*pv(A, c, 0, 0, i), *pv(A, c, 1, 0, i)};
    double up[2] = {*pv(A, c, 0, 0, i + 1), *pv(A, c, 1, 0, i + 1)};
    return or_recon1d(P->k, um, u0, up, cf);
  }
  double a[9], mx[9], my[9];
  for (int s = 0; s < 3; ++s)
    for (int r = 0; r < 3; ++r) {
      a[3 * s + r] = *pv(A, c, 0, j - 1 + s, i - 1 + r);
      mx[3 * s + r] = *pv(A, c, 1, j - 1 + s, i - 1 + r);
      my[3 * s + r] = *pv(A, c, 2, j - 1 + s, i - 1 + r);
    }
  return or_recon2d(P->k, a, mx, my, cf);
}

/* ------------------------------------------------------------------ */
/* Residual                                                             */
/* ------------------------------------------------------------------ */

/* ------------------------------------------------------------------ */
/* Optional BP/PP safeguard (Sec. 2.3 remarks, Alg. 1; the paper cites its */
/* limiter, CDW1/CDW2, without defining it): the Zhang-Shu scaling of a    */
/* cell's reconstruction towards its average, p~ = u_bar + theta (p -     */
/* u_bar), so that every point of a cell-average decomposition and every  */
/* volume Gauss point holds an admissible Euler state.                    */
/* ------------------------------------------------------------------ */

/* Gauss-Lobatto nodes on [-1/2,1/2] whose rule is exact on P_{k-1}: 3 points
 * for k <= 4, 4 points for k = 5, 6. */
static int lobatto_nodes(int k, double* x) {
  if (k <= 4) {
    x[0] = -0.5; x[1] = 0.0; x[2] = 0.5;
    return 3;
  }
  x[0] = -0.5; x[1] = -0.5 / sqrt(5.0); x[2] = 0.5 / sqrt(5.0); x[3] = 0.5;
  return 4;
}

/* Points of the check: 1D the Lobatto nodes and the 4 Gauss nodes; 2D the
 * Lobatto x Gauss, Gauss x Lobatto and Gauss x Gauss products.  Returns the
 * number of points (at most 48). */
static int pp_points(int d, int k, double* xi, double* eta) {
  double gl[4], g[4], w[4];
  int nl = lobatto_nodes(k, gl);
  or_gauss4(g, w);
  int n = 0;
  if (d == 1) {
    for (int a = 0; a < nl; ++a) { xi[n] = gl[a]; eta[n++] = 0.0; }
    for (int a = 0; a < 4; ++a) { xi[n] = g[a]; eta[n++] = 0.0; }
    return n;
  }
  for (int a = 0; a < nl; ++a)
    for (int b = 0; b < 4; ++b) { xi[n] = gl[a]; eta[n++] = g[b]; }
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < nl; ++b) { xi[n] = g[a]; eta[n++] = gl[b]; }
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) { xi[n] = g[a]; eta[n++] = g[b]; }
  return n;
}

static double pressure(double gm1, int d, const double* u) {
  double m2 = u[1] * u[1] + (d == 2 ? u[2] * u[2] : 0.0);
  return gm1 * (u[d + 1] - 0.5 * m2 / u[0]);
}

/* The t in [0, 1] with p(ub + t dw) = eps, given p(ub) > eps > p(ub + dw):
 * the root in (0, 1) of rho(t) (E(t) - eps/(gamma-1)) - |m(t)|^2 / 2. */
static double pressure_root(double gm1, int d, const double* ub, const double* dw, double eps) {
  int e = d + 1;
  double Eh = ub[e] - eps / gm1, dm2 = dw[1] * dw[1], mdm = ub[1] * dw[1], m2 = ub[1] * ub[1];
  if (d == 2) { dm2 += dw[2] * dw[2]; mdm += ub[2] * dw[2]; m2 += ub[2] * ub[2]; }
  double a = dw[e] * dw[0] - 0.5 * dm2;
  double b = Eh * dw[0] + ub[0] * dw[e] - mdm;
  double c = Eh * ub[0] - 0.5 * m2;
  if (fabs(a) < 1e-14 * (fabs(b) + fabs(c))) return -c / b;
  /* roots q / a and c / q with q = -(b + sign(b) sqrt(disc)) / 2: the same
   * pair as (-b -+ sqrt(disc)) / 2a without the cancellation of -b + sqrt
   * when b^2 >> |4ac| (the small root, the one wanted, would lose digits) */
  double disc = sqrt(fmax(b * b - 4.0 * a * c, 0.0));
  double q = -0.5 * (b + copysign(disc, b));
  double r1 = q / a, r2 = c / q;
  double t = 1.0;
  if (r1 >= 0.0 && r1 <= 1.0) t = r1;
  if (r2 >= 0.0 && r2 <= 1.0 && r2 < t) t = r2;
  return t;
}

/* Scale the Euler reconstruction of one cell, given as nc coefficient arrays
 * (coefficient 0 is the cell average; basis functions 1.. have zero mean):
 * density first (theta1), then all components (theta2). */
static void pp_limit_cell(const or_problem* P, int ncoef, double* const* cf, double* smax);

/* Rusanov speeds (x, y) maxed over the check points of the limited
 * reconstruction of every cell: the wave speeds of the CFL condition under
 * which the scaled reconstruction keeps the averages admissible (Zhang-Shu). */
static void pp_max_speed(const or_problem* P, const double* U, double* ax, double* ay) {
  padded A;
  double mx = 0.0, my = 0.0;
  if (pad_state(P, U, &A)) { *ax = *ay = NAN; return; }
  int nc = A.nc, ny = P->d == 1 ? 1 : P->ny;
  int ncoef = P->d == 1 ? P->k : (P->k == 3 ? 6 : P->k == 4 ? 10 : P->k == 5 ? 15 : 21);
#pragma omp parallel for reduction(max : mx, my)
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < P->nx; ++i) {
      double cbuf[4][23], *cf[4], sm[2];
      for (int c = 0; c < nc; ++c) {
        cf[c] = cbuf[c];
        cell_coeffs(P, &A, c, j, i, cf[c]);
      }
      pp_limit_cell(P, ncoef, cf, sm);
      if (sm[0] > mx) mx = sm[0];
      if (sm[1] > my) my = sm[1];
    }
  free(A.v);
  *ax = mx;
  *ay = my;
}

/* Bound-preserving scaling of a scalar reconstruction (Buckley-Leverett,
 * whose solution stays in [0, 1]): theta = min(1, (1 - u_bar) / (M - u_bar),
 * u_bar / (u_bar - m)) with M, m the largest and smallest value at the check
 * points; smax (if not NULL) gets the largest |f'| at the check points of the
 * scaled reconstruction and at the average. */
static void bp_limit_scalar(const or_problem* P, int ncoef, double* cf, double* smax) {
  double xi[48], eta[48];
  int np = pp_points(1, P->k, xi, eta);
  const double ub = cf[0];
  double M = ub, m = ub;
  for (int q = 0; q < np; ++q) {
    const double v = or_eval1d(ncoef, cf, xi[q]);
    if (v > M) M = v;
    if (v < m) m = v;
  }
  double theta = 1.0;
  if (!(ub >= 0.0 && ub <= 1.0)) theta = 0.0;
  else {
    if (M > 1.0) theta = fmin(theta, (1.0 - ub) / (M - ub));
    if (m < 0.0) theta = fmin(theta, ub / (ub - m));
  }
  if (theta != 1.0)
    for (int l = 1; l < ncoef; ++l) cf[l] *= theta;
  if (smax) {
    smax[0] = phys_speed(P, 0, &ub);
    smax[1] = 0.0;
    for (int q = 0; q < np; ++q) {
      const double v = or_eval1d(ncoef, cf, xi[q]);
      const double sq = phys_speed(P, 0, &v);
      if (sq > smax[0]) smax[0] = sq;
    }
  }
}

static void pp_limit_cell(const or_problem* P, int ncoef, double* const* cf, double* smax) {
  if (P->eq == OR_BUCKLEY) {
    bp_limit_scalar(P, ncoef, cf[0], smax);
    return;
  }
  int d = P->d, nc = d + 2;
  double gm1 = P->gamma - 1.0;
  double xi[48], eta[48];
  int np = pp_points(d, P->k, xi, eta);
  double ub[4];
  for (int c = 0; c < nc; ++c) ub[c] = cf[c][0];
  double pb = ub[0] > 0.0 ? pressure(gm1, d, ub) : -1.0;
  double t1 = 1.0, t2 = 1.0;
  if (!(ub[0] > 0.0) || !(pb > 0.0)) {
    t1 = t2 = 0.0;  /* the average itself is not admissible: keep it constant */
  } else {
    /* targets relative to the cell: density 1e-6 rho_bar, pressure 1e-8
     * p_bar.  At a check point scaled towards vacuum the computed density
     * carries a relative rounding error of ~1e-16 / (density target), which
     * m^2 / (2 rho) carries into the pressure: the pressure target must stay
     * above ~1e-16 E / (relative density target), so the two targets' product
     * must exceed ~1e-16 E / p_bar (the absolute 1e-13 density of Zhang-Shu
     * with 1e-10 p_bar left limited points at p < 0 in the multiscale Lax
     * problem of Example 4.6) */
    double eps = 1e-6 * ub[0], epsp = 1e-8 * pb;
    double u[48][4];
    double rmin = ub[0];
    for (int q = 0; q < np; ++q) {
      for (int c = 0; c < nc; ++c)
        u[q][c] = d == 1 ? or_eval1d(ncoef, cf[c], xi[q]) : or_eval2d(ncoef, cf[c], xi[q], eta[q]);
      if (u[q][0] < rmin) rmin = u[q][0];
    }
    if (rmin < eps) t1 = (ub[0] - eps) / (ub[0] - rmin);
    for (int q = 0; q < np; ++q) {
      double w[4], dw[4];
      for (int c = 0; c < nc; ++c) w[c] = u[q][c];
      w[0] = ub[0] + t1 * (u[q][0] - ub[0]);
      if (pressure(gm1, d, w) < epsp) {
        for (int c = 0; c < nc; ++c) dw[c] = w[c] - ub[c];
        double t = pressure_root(gm1, d, ub, dw, epsp);
        if (t < t2) t2 = t;
      }
    }
  }
  if (!(t1 == 1.0 && t2 == 1.0))
    for (int l = 1; l < ncoef; ++l) {
      cf[0][l] *= t1 * t2;
      for (int c = 1; c < nc; ++c) cf[c][l] *= t2;
    }
  if (smax) {
    smax[0] = phys_speed(P, 0, ub);
    smax[1] = d == 2 ? phys_speed(P, 1, ub) : 0.0;
    for (int q = 0; q < np; ++q) {
      double u[4];
      for (int c = 0; c < nc; ++c)
        u[c] = d == 1 ? or_eval1d(ncoef, cf[c], xi[q]) : or_eval2d(ncoef, cf[c], xi[q], eta[q]);
      double sx = phys_speed(P, 0, u);
      if (sx > smax[0]) smax[0] = sx;
      if (d == 2) {
        double sy = phys_speed(P, 1, u);
        if (sy > smax[1]) smax[1] = sy;
      }
    }
  }
}

static int residual_1d(const or_problem* P, padded* A, double* R) {
  int nx = P->nx, nc = A->nc;
  double dx = (P->x1 - P->x0) / nx;
  double gx[4], gw[4];
  or_gauss4(gx, gw);
  /* coefficients of cells -1..nx */
  double* C = (double*)malloc(sizeof(double) * (size_t)(nx + 2) * nc * 6);
  double* F = (double*)malloc(sizeof(double) * (size_t)(nx + 1) * nc);
  if (!C || !F) { free(C); free(F); return -1; }
  int ncoef = P->k;
#pragma omp parallel for
  for (int i = -1; i <= nx; ++i) {
    for (int c = 0; c < nc; ++c) cell_coeffs(P, A, c, 0, i, &C[((size_t)(i + 1) * nc + c) * 6]);
    if (P->pp_limiter && (P->eq == OR_EULER || P->eq == OR_BUCKLEY)) {
      double* cf[4];
      for (int c = 0; c < nc; ++c) cf[c] = &C[((size_t)(i + 1) * nc + c) * 6];
      pp_limit_cell(P, ncoef, cf, NULL);
    }
  }
  /* face f sits between cells f-1 and f */
  long long bad = 0;
#pragma omp parallel for reduction(+ : bad)
  for (int f = 0; f <= nx; ++f) {
    double uL[4], uR[4];
    for (int c = 0; c < nc; ++c) {
      uL[c] = or_eval1d(ncoef, &C[((size_t)(f) * nc + c) * 6], 0.5);
      uR[c] = or_eval1d(ncoef, &C[((size_t)(f + 1) * nc + c) * 6], -0.5);
    }
    bad += llf(P, 0, uL, uR, &F[(size_t)f * nc]);
  }
  g_nonphys_traces += bad;
#pragma omp parallel for
  for (int i = 0; i < nx; ++i) {
    double vol[4] = {0, 0, 0, 0};
    for (int g = 0; g < 4; ++g) {
      double u[4], fl[4];
      for (int c = 0; c < nc; ++c) u[c] = or_eval1d(ncoef, &C[((size_t)(i + 1) * nc + c) * 6], gx[g]);
      phys_flux(P, 0, u, fl);
      for (int c = 0; c < nc; ++c) vol[c] += gw[g] * fl[c];
    }
    for (int c = 0; c < nc; ++c) {
      double fr = F[(size_t)(i + 1) * nc + c], fl = F[(size_t)i * nc + c];
      R[((size_t)(c * 2 + 0)) * nx + i] = -(fr - fl) / dx;
      R[((size_t)(c * 2 + 1)) * nx + i] = (vol[c] - 0.5 * (fr + fl)) / dx;
    }
  }
  free(C);
  free(F);
  return 0;
}

static int residual_2d(const or_problem* P, padded* A, double* R) {
  int nx = P->nx, ny = P->ny, nc = A->nc;
  double dx = (P->x1 - P->x0) / nx, dy = (P->y1 - P->y0) / ny;
  double gx[4], gw[4];
  or_gauss4(gx, gw);
  int ncoef = P->k == 3 ? 6 : P->k == 4 ? 10 : P->k == 5 ? 15 : 21;
  size_t ncell = (size_t)(nx + 2) * (ny + 2);
  double* C = (double*)malloc(sizeof(double) * ncell * nc * 23);
  /* Fx[j][f][g][c], f = 0..nx ; Fy[f][i][g][c], f = 0..ny */
  double* Fx = (double*)malloc(sizeof(double) * (size_t)ny * (nx + 1) * 4 * nc);
  double* Fy = (double*)malloc(sizeof(double) * (size_t)(ny + 1) * nx * 4 * nc);
  if (!C || !Fx || !Fy) { free(C); free(Fx); free(Fy); return -1; }
#define CC(j, i, c) (&C[(((size_t)((j) + 1) * (nx + 2) + ((i) + 1)) * nc + (c)) * 23])
#pragma omp parallel for
  for (int j = -1; j <= ny; ++j)
    for (int i = -1; i <= nx; ++i) {
      for (int c = 0; c < nc; ++c) cell_coeffs(P, A, c, j, i, CC(j, i, c));
      if (P->pp_limiter && P->eq == OR_EULER) {
        double* cf[4];
        for (int c = 0; c < nc; ++c) cf[c] = CC(j, i, c);
        pp_limit_cell(P, ncoef, cf, NULL);
      }
    }
  long long bad = 0;
#pragma omp parallel for reduction(+ : bad)
  for (int j = 0; j < ny; ++j)
    for (int f = 0; f <= nx; ++f)
      for (int g = 0; g < 4; ++g) {
        double uL[4], uR[4];
        for (int c = 0; c < nc; ++c) {
          uL[c] = or_eval2d(ncoef, CC(j, f - 1, c), 0.5, gx[g]);
          uR[c] = or_eval2d(ncoef, CC(j, f, c), -0.5, gx[g]);
        }
        bad += llf(P, 0, uL, uR, &Fx[(((size_t)j * (nx + 1) + f) * 4 + g) * nc]);
      }
#pragma omp parallel for reduction(+ : bad)
  for (int f = 0; f <= ny; ++f)
    for (int i = 0; i < nx; ++i)
      for (int g = 0; g < 4; ++g) {
        double uB[4], uT[4];
        for (int c = 0; c < nc; ++c) {
          uB[c] = or_eval2d(ncoef, CC(f - 1, i, c), gx[g], 0.5);
          uT[c] = or_eval2d(ncoef, CC(f, i, c), gx[g], -0.5);
        }
        bad += llf(P, 1, uB, uT, &Fy[(((size_t)f * nx + i) * 4 + g) * nc]);
      }
  g_nonphys_traces += bad;
#pragma omp parallel for
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      double v1[4] = {0, 0, 0, 0}, v2[4] = {0, 0, 0, 0};
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
          double u[4], f1[4], f2[4];
          for (int c = 0; c < nc; ++c) u[c] = or_eval2d(ncoef, CC(j, i, c), gx[a], gx[b]);
          phys_flux(P, 0, u, f1);
          phys_flux(P, 1, u, f2);
          for (int c = 0; c < nc; ++c) {
            v1[c] += gw[a] * gw[b] * f1[c];
            v2[c] += gw[a] * gw[b] * f2[c];
          }
        }
      for (int c = 0; c < nc; ++c) {
        double xr = 0, xl = 0, yt = 0, yb = 0, xr_w = 0, xl_w = 0, yt_w = 0, yb_w = 0;
        for (int g = 0; g < 4; ++g) {
          double fxr = Fx[(((size_t)j * (nx + 1) + i + 1) * 4 + g) * nc + c];
          double fxl = Fx[(((size_t)j * (nx + 1) + i) * 4 + g) * nc + c];
          double fyt = Fy[(((size_t)(j + 1) * nx + i) * 4 + g) * nc + c];
          double fyb = Fy[(((size_t)j * nx + i) * 4 + g) * nc + c];
          xr += gw[g] * fxr; xl += gw[g] * fxl;
          yt += gw[g] * fyt; yb += gw[g] * fyb;
          xr_w += gw[g] * gx[g] * fxr; xl_w += gw[g] * gx[g] * fxl;
          yt_w += gw[g] * gx[g] * fyt; yb_w += gw[g] * gx[g] * fyb;
        }
        size_t o = (size_t)j * nx + i, plane = (size_t)nx * ny;
        R[(size_t)(c * 3 + 0) * plane + o] = -(xr - xl) / dx - (yt - yb) / dy;
        R[(size_t)(c * 3 + 1) * plane + o] = (v1[c] - 0.5 * (xr + xl)) / dx - (yt_w - yb_w) / dy;
        R[(size_t)(c * 3 + 2) * plane + o] = (v2[c] - 0.5 * (yt + yb)) / dy - (xr_w - xl_w) / dx;
      }
    }
#undef CC
  free(C);
  free(Fx);
  free(Fy);
  return 0;
}

int or_residual(const or_problem* P, const double* U, double* R) {
  padded A;
  if (pad_state(P, U, &A)) return -1;
  int rc = P->d == 1 ? residual_1d(P, &A, R) : residual_2d(P, &A, R);
  free(A.v);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Wave speeds and time step                                            */
/* ------------------------------------------------------------------ */

static void cell_average_vec(const or_problem* P, const double* U, size_t cell, double* u) {
  int nc = or_ncomp(P), nm = or_nmom(P);
  size_t plane = (size_t)P->nx * (P->d == 1 ? 1 : P->ny);
  for (int c = 0; c < nc; ++c) u[c] = U[(size_t)(c * nm) * plane + cell];
}

void or_max_speed(const or_problem* P, const double* U, double* ax, double* ay) {
  size_t n = (size_t)P->nx * (P->d == 1 ? 1 : P->ny);
  double mx = 0.0, my = 0.0;
  for (size_t q = 0; q < n; ++q) {
    double u[4];
    cell_average_vec(P, U, q, u);
    double sx = phys_speed(P, 0, u);
    if (sx > mx) mx = sx;
    if (P->d == 2) {
      double sy = phys_speed(P, 1, u);
      if (sy > my) my = sy;
    }
  }
  *ax = mx;
  *ay = my;
}

double or_dt(const or_problem* P, const double* U, double cfl, int smooth) {
  double ax, ay;
  if (P->pp_limiter && (P->eq == OR_EULER || P->eq == OR_BUCKLEY)) pp_max_speed(P, U, &ax, &ay);
  else or_max_speed(P, U, &ax, &ay);
  double dx = (P->x1 - P->x0) / P->nx;
  double e = smooth ? P->k / 3.0 : 1.0;
  if (P->d == 1) return cfl * pow(dx, e) / ax;
  double dy = (P->y1 - P->y0) / P->ny;
  return cfl / (ax / pow(dx, e) + ay / pow(dy, e));
}

/* ------------------------------------------------------------------ */
/* OE                                                                   */
/* ------------------------------------------------------------------ */

static double default_gamma_k(const or_problem* P) {
  if (P->gamma_k > 0.0) return P->gamma_k;
  if (P->k <= 4) return 25.0;
  return P->d == 1 ? 12.5 : 15.0;
}

/* Type-II denominator D and tolerance eps over the stencil Lambda of averages
 * vals[0..n-1] (Tab. sigma1d / sigma2d; S_Lambda is the unnormalised sum, as
 * printed; mean != 0 selects the alternative reading S_Lambda / |Lambda|). */
static void type2_den(const double* vals, int n, int mean, double* D, double* eps) {
  double S = 0.0, mabs = 0.0, d = 0.0;
  for (int q = 0; q < n; ++q) S += vals[q];
  if (mean) S /= (double)n;
  for (int q = 0; q < n; ++q) {
    double t = fabs(vals[q] - S);
    if (t > d) d = t;
    if (fabs(vals[q]) > mabs) mabs = fabs(vals[q]);
  }
  *D = d;
  *eps = 1e-14 * (mabs > 1.0 ? mabs : 1.0);
}

int or_oe(const or_problem* P, double dt, double* U, double* theta) {
  if (P->oe_type == OR_OE_NONE) {
    if (theta) {
      size_t n = (size_t)P->nx * (P->d == 1 ? 1 : P->ny);
      for (size_t q = 0; q < n; ++q) theta[q] = 0.0;
    }
    return 0;
  }
  padded A;
  if (pad_state(P, U, &A)) return -1;
  int nc = A.nc, nm = A.nm, nx = P->nx, ny = A.ny;
  double gk = default_gamma_k(P);
  size_t plane = (size_t)nx * ny;
  /* Type I: global denominators per component */
  double DO[4] = {0, 0, 0, 0}, eO[4] = {0, 0, 0, 0};
  if (P->oe_type == OR_OE_TYPE1) {
    for (int c = 0; c < nc; ++c) {
      const double* a = &U[(size_t)(c * nm) * plane];
      double mean = 0.0, mabs = 0.0, d = 0.0;
      for (size_t q = 0; q < plane; ++q) mean += a[q];
      mean /= (double)plane;
      for (size_t q = 0; q < plane; ++q) {
        if (fabs(a[q] - mean) > d) d = fabs(a[q] - mean);
        if (fabs(a[q]) > mabs) mabs = fabs(a[q]);
      }
      DO[c] = d;
      eO[c] = 1e-14 * (mabs > 1.0 ? mabs : 1.0);
    }
  }
  double dx = (P->x1 - P->x0) / nx;
  double dy = P->d == 2 ? (P->y1 - P->y0) / ny : 1.0;
  if (P->d == 1) {
    int ncoef = P->k;
    double* C = (double*)malloc(sizeof(double) * (size_t)(nx + 2) * nc * 6);
    if (!C) { free(A.v); return -1; }
#pragma omp parallel for
    for (int i = -1; i <= nx; ++i)
      for (int c = 0; c < nc; ++c) cell_coeffs(P, &A, c, 0, i, &C[((size_t)(i + 1) * nc + c) * 6]);
#pragma omp parallel for
    for (int i = 0; i < nx; ++i) {
      double sig = 0.0;
      for (int c = 0; c < nc; ++c) {
        const double* cm = &C[((size_t)(i) * nc + c) * 6];
        const double* c0 = &C[((size_t)(i + 1) * nc + c) * 6];
        const double* cp = &C[((size_t)(i + 2) * nc + c) * 6];
        double jl = or_eval1d(ncoef, c0, -0.5) - or_eval1d(ncoef, cm, 0.5);
        double jr = or_eval1d(ncoef, cp, -0.5) - or_eval1d(ncoef, c0, 0.5);
        double D, eps;
        if (P->oe_type == OR_OE_TYPE1) {
          D = DO[c];
          eps = eO[c];
        } else {
          double v[3] = {*pv(&A, c, 0, 0, i - 1), *pv(&A, c, 0, 0, i), *pv(&A, c, 0, 0, i + 1)};
          type2_den(v, 3, P->oe_mean, &D, &eps);
        }
        double s = (D < eps) ? 0.0 : gk * (fabs(jl) + fabs(jr)) / D;
        if (s > sig) sig = s;
      }
      double beta = 0.0;
      for (int q = -1; q <= 1; ++q) {
        double u[4];
        for (int c = 0; c < nc; ++c) u[c] = *pv(&A, c, 0, 0, i + q);
        double s = phys_speed(P, 0, u);
        if (s > beta) beta = s;
      }
      double th = beta * dt * sig / dx;
      double damp = exp(-th);
      for (int c = 0; c < nc; ++c) U[(size_t)(c * nm + 1) * plane + i] *= damp;
      if (theta) theta[i] = th;
    }
    free(C);
  } else {
    /* Jumps at face centres use p_k, except that for k=6 the reading
     * oe_jump_q6=1 uses the full auxiliary Q6 (this reproduces the printed
     * matrices A_6, B_6, C_6 of the 2D jump table). */
    int ncoef = P->k == 3 ? 6 : P->k == 4 ? 10 : P->k == 5 ? 15 : (P->oe_jump_q6 ? 23 : 21);
    size_t ncell = (size_t)(nx + 2) * (ny + 2);
    double* C = (double*)malloc(sizeof(double) * ncell * nc * 23);
    if (!C) { free(A.v); return -1; }
#define CC(j, i, c) (&C[(((size_t)((j) + 1) * (nx + 2) + ((i) + 1)) * nc + (c)) * 23])
#pragma omp parallel for
    for (int j = -1; j <= ny; ++j)
      for (int i = -1; i <= nx; ++i)
        for (int c = 0; c < nc; ++c) cell_coeffs(P, &A, c, j, i, CC(j, i, c));
#pragma omp parallel for
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double sx = 0.0, sy = 0.0;
        for (int c = 0; c < nc; ++c) {
          double jxl = or_eval2d(ncoef, CC(j, i, c), -0.5, 0.0) - or_eval2d(ncoef, CC(j, i - 1, c), 0.5, 0.0);
          double jxr = or_eval2d(ncoef, CC(j, i + 1, c), -0.5, 0.0) - or_eval2d(ncoef, CC(j, i, c), 0.5, 0.0);
          double jyb = or_eval2d(ncoef, CC(j, i, c), 0.0, -0.5) - or_eval2d(ncoef, CC(j - 1, i, c), 0.0, 0.5);
          double jyt = or_eval2d(ncoef, CC(j + 1, i, c), 0.0, -0.5) - or_eval2d(ncoef, CC(j, i, c), 0.0, 0.5);
          double D, eps;
          if (P->oe_type == OR_OE_TYPE1) {
            D = DO[c];
            eps = eO[c];
          } else {
            double v[9];
            for (int s = 0; s < 3; ++s)
              for (int r = 0; r < 3; ++r) v[3 * s + r] = *pv(&A, c, 0, j - 1 + s, i - 1 + r);
            type2_den(v, 9, P->oe_mean, &D, &eps);
          }
          double ssx = 0.0, ssy = 0.0;
          if (!(D < eps)) {
            ssx = gk * (fabs(jxl) + fabs(jxr)) / D;
            ssy = gk * (fabs(jyb) + fabs(jyt)) / D;
          }
          if (ssx > sx) sx = ssx;
          if (ssy > sy) sy = ssy;
        }
        double bx = 0.0, by = 0.0;
        for (int s = -1; s <= 1; ++s)
          for (int r = -1; r <= 1; ++r) {
            double u[4];
            for (int c = 0; c < nc; ++c) u[c] = *pv(&A, c, 0, j + s, i + r);
            double qx = phys_speed(P, 0, u), qy = phys_speed(P, 1, u);
            if (qx > bx) bx = qx;
            if (qy > by) by = qy;
          }
        double th = bx * dt * sx / dx + by * dt * sy / dy;
        double damp = exp(-th);
        size_t o = (size_t)j * nx + i;
        for (int c = 0; c < nc; ++c) {
          U[(size_t)(c * nm + 1) * plane + o] *= damp;
          U[(size_t)(c * nm + 2) * plane + o] *= damp;
        }
        if (theta) theta[o] = th;
      }
#undef CC
    free(C);
  }
  free(A.v);
  return 0;
}

/* ------------------------------------------------------------------ */
/* SSP-RK3 step and time loop                                           */
/* ------------------------------------------------------------------ */

static size_t state_len(const or_problem* P);

/* Number of cells whose averages are not an admissible Euler state: rho <= 0
 * or p <= 0, i.e. rho E - |rho v|^2 / 2 <= 0 (Sec. 2.3; 0 for scalar laws)
 * or that hold a non-finite value in any plane. */
long long or_inadmissible(const or_problem* P, const double* U) {
  size_t cells = (size_t)P->nx * (P->d == 1 ? 1 : P->ny);
  int nm = or_nmom(P), nc = or_ncomp(P);
  long long bad = 0;
  for (size_t q = 0; q < cells; ++q) {
    int ok = 1;
    for (int p = 0; p < nc * nm; ++p)
      if (!isfinite(U[(size_t)p * cells + q])) ok = 0;
    if (ok && P->eq == OR_EULER) {
      double rho = U[q], E = U[(size_t)(nc - 1) * nm * cells + q];
      double m2 = 0.0;
      for (int c = 1; c < nc - 1; ++c) {
        double m = U[(size_t)c * nm * cells + q];
        m2 += m * m;
      }
      if (!(rho > 0.0) || !(rho * E - 0.5 * m2 > 0.0)) ok = 0;
    }
    bad += !ok;
  }
  return bad;
}

static size_t state_len(const or_problem* P) {
  return (size_t)or_ncomp(P) * or_nmom(P) * P->nx * (P->d == 1 ? 1 : P->ny);
}

/* Averages of state V inadmissible anywhere (Euler: rho <= 0 or
 * rho E - |m|^2 / 2 <= 0, NaN included)? */
static int averages_inadmissible(const or_problem* P, const double* V) {
  return P->eq == OR_EULER && or_inadmissible(P, V) > 0;
}

/* One step; with check != 0, returns 1 (U unchanged) as soon as a stage's
 * averages leave the admissible set. */
static int step_impl(const or_problem* P, double* U, double dt, int check);

int or_step(const or_problem* P, double* U, double dt) { return step_impl(P, U, dt, 0); }

static long g_rejected = 0;
long or_rejected_steps(int reset) {
  long v = g_rejected;
  if (reset) g_rejected = 0;
  return v;
}

static int step_impl(const or_problem* P, double* U, double dt, int check) {
  size_t n = state_len(P);
  double* U0 = (double*)malloc(sizeof(double) * n);
  double* Us = (double*)malloc(sizeof(double) * n);
  double* R = (double*)malloc(sizeof(double) * n);
  if (!U0 || !Us || !R) { free(U0); free(Us); free(R); return -1; }
  memcpy(U0, U, sizeof(double) * n);
  int rc = 0;
  /* the stage states' times (they matter only to a front side condition) */
  or_problem Q = *P;
  int bad = 0;
  /* stage 1: U1 = U0 + dt R(U0), U0 at time t */
  rc |= or_residual(&Q, U0, R);
  for (size_t q = 0; q < n; ++q) Us[q] = U0[q] + dt * R[q];
  bad = check && averages_inadmissible(P, Us);
  /* stage 2: U2 = 3/4 U0 + 1/4 (U1 + dt R(U1)), U1 at t + dt */
  if (!bad) {
    Q.time = P->time + dt;
    rc |= or_residual(&Q, Us, R);
    for (size_t q = 0; q < n; ++q) Us[q] = 0.75 * U0[q] + 0.25 * (Us[q] + dt * R[q]);
    bad = check && averages_inadmissible(P, Us);
  }
  /* stage 3: Un = 1/3 U0 + 2/3 (U2 + dt R(U2)), U2 at t + dt/2 */
  if (!bad) {
    Q.time = P->time + 0.5 * dt;
    rc |= or_residual(&Q, Us, R);
    for (size_t q = 0; q < n; ++q) U[q] = 1.0 / 3.0 * U0[q] + 2.0 / 3.0 * (Us[q] + dt * R[q]);
    bad = check && averages_inadmissible(P, U);
  }
  if (bad) {  /* discard the step: U keeps U^n */
    memcpy(U, U0, sizeof(double) * n);
    free(U0);
    free(Us);
    free(R);
    return rc ? -1 : 1;
  }
  /* end-of-step OE on the state at t + dt */
  Q.time = P->time + dt;
  rc |= or_oe(&Q, dt, U, NULL);
  free(U0);
  free(Us);
  free(R);
  return rc ? -1 : 0;
}

int or_run(const or_problem* P, double* U, double T, long nsteps, double cfl, int smooth, double* t_out,
           long* nsteps_out) {
  size_t n = state_len(P);
  double t = 0.0;  /* time since the start (the states' times are P->time + t) */
  long s = 0;
  int rc = 0;
  or_problem Q = *P;
  /* With the BP/PP safeguard (Euler), a step whose stage averages leave the
   * admissible set is discarded and retried with half the step size (the
   * forward-Euler bound holds only for the speeds of each stage's input,
   * which may exceed those of U^n the step size came from); r halvings so
   * far, at most 30; an accepted step resets r. */
  const int check = P->pp_limiter && P->eq == OR_EULER;
  int r = 0;
  for (;;) {
    if (T > 0.0) {
      if (t >= T) break;
    } else if (s >= nsteps) {
      break;
    }
    Q.time = P->time + t;
    double dt = or_dt(&Q, U, cfl, smooth);
    if (!(dt > 0.0) || !isfinite(dt)) { rc = -1; break; }
    dt = ldexp(dt, -r);
    if (T > 0.0 && t + dt >= T) dt = T - t;
    int st = step_impl(&Q, U, dt, check);
    if (st == 1) {
      ++g_rejected;
      if (++r > 30) { rc = -1; break; }
      continue;
    }
    if (st) { rc = -1; break; }
    r = 0;
    t = (T > 0.0 && t + dt >= T) ? T : t + dt;
    ++s;
    for (size_t q = 0; q < n; ++q)
      if (!isfinite(U[q])) { rc = -1; break; }
    if (rc) break;
  }
  if (t_out) *t_out = t;
  if (nsteps_out) *nsteps_out = s;
  return rc;
}
