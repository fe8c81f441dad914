/*
 * fam_oracle.h -- plain, slow, FP64 CPU oracle for the compact FAM time step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA implementation: every coefficient
 * below is transcribed by hand from the paper (Fan & Wu, "Compact
 * Finite-Average-Moment Schemes with Single-Step Oscillation Elimination").
 *
 * Layout of a state array (no ghost cells):
 *     U[((c * nmom + m) * ny + j) * nx + i]
 * c = conserved component (1 for scalar laws, d+2 for Euler),
 * m = moment (0 = cell average, 1 = scaled x-moment, 2 = scaled y-moment),
 * ny = 1 in one dimension.
 *
 * Parity status (see the pins in tests/test_oracle_pins.py): every function is
 * pinned except the shock-run solution values themselves, which the paper does
 * not print; those are covered only by invariants (conservation, OE
 * properties) -- "parity unpinned" for shock-run values.
 */
#ifndef FAM_ORACLE_H
#define FAM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_ADVECTION = 0, OR_BURGERS = 1, OR_EULER = 2, OR_BUCKLEY = 3 };
enum { OR_BC_PERIODIC = 0, OR_BC_OUTFLOW = 1, OR_BC_REFLECTIVE = 2, OR_BC_INFLOW = 3, OR_BC_FRONT = 4 };
enum { OR_OE_NONE = 0, OR_OE_TYPE1 = 1, OR_OE_TYPE2 = 2 };

typedef struct {
  int d;              /* 1 or 2 */
  int nx, ny;         /* ny = 1 when d = 1 */
  double x0, x1, y0, y1;
  int k;              /* FAM order 3..6 */
  int eq;             /* OR_ADVECTION / OR_BURGERS / OR_EULER */
  int bc[4];          /* x-lo, x-hi, y-lo, y-hi */
  double inflow[4][4];/* conservative inflow state per side (averages) */
  double gamma;       /* Euler: ratio of specific heats */
  double ax, ay;      /* advection velocity */
  int oe_type;        /* OR_OE_NONE / OR_OE_TYPE1 / OR_OE_TYPE2 */
  double gamma_k;     /* OE constant; <= 0 selects the paper's default */
  int oe_jump_q6;     /* 2D k=6: 1 = jumps of full Q6 (printed matrices), 0 = of p6 */
  int oe_mean;        /* Type II: 0 = S_Lambda the unnormalised sum (as printed),
                         1 = the mean over Lambda (an alternative reading) */
  int pp_limiter;     /* Buckley-Leverett (1D): 1 = scale every stage's reconstruction
                         towards the cell average until every check point lies in
                         [0, 1] (the bound-preserving form for a scalar);
                         Euler: 1 = scale every stage's reconstruction towards the
                         cell average until rho, p >= eps at the points of a
                         Gauss-Lobatto decomposition and the volume Gauss points
                         (the BP/PP safeguard the paper cites; Zhang-Shu scaling) */
  /* Side conditions that vary along a side or in time (the double Mach
   * reflection set-up of Example 4.8).  split[s] > 0: the ghost cells of
   * side s whose cell centre along the side (x for the y-sides, y for the
   * x-sides; ghost columns and rows take the centre of the nearest interior
   * one) lies below split[s] hold inflow[s]; the others follow bc[s].
   * bc[s] = OR_BC_FRONT (y-sides only): a ghost cell with centre (x, y) holds
   * inflow[s] if x < front[0] + front[1] y + front[2] time, front_ahead
   * otherwise (a straight front moving along x).  time: the time of the state
   * passed to or_residual / or_oe / or_dt; or_step evaluates its stages at
   * time, time + dt, time + dt/2 and the OE at time + dt; or_run starts at
   * time. */
  double split[4];
  double front[3];
  double front_ahead[4];
  double time;
} or_problem;

int or_ncomp(const or_problem* P);
int or_nmom(const or_problem* P);

/* Reconstruction (App. B / App. I).  Returns the number of coefficients of
 * the FAM-k polynomial (k in 1D; 6, 10, 15, 21 in 2D).  c must hold 6 (1D) or
 * 23 (2D) entries; all auxiliary coefficients are filled as well. */
int or_recon1d(int k, const double um[2], const double u0[2], const double up[2], double c[6]);
int or_recon2d(int k, const double a[9], const double mx[9], const double my[9], double c[23]);
double or_basis1d(int l, double xi);
double or_basis2d(int l, double xi, double eta);
double or_eval1d(int ncoef, const double* c, double xi);
double or_eval2d(int ncoef, const double* c, double xi, double eta);

/* Four-point Gauss-Legendre rule on [-1/2, 1/2] (weights sum to 1). */
void or_gauss4(double node[4], double weight[4]);

/* Semi-discrete right-hand side R(U) of eq. (1dSemi) / eq. (11). */
int or_residual(const or_problem* P, const double* U, double* R);

/* Face quadrature points (1D: faces) at which one of the two traces of the
 * Rusanov flux has no spectral radius -- an Euler trace with gamma p / rho < 0
 * (rho <= 0 or p <= 0 without a positivity limiter), whose radius |v_n| + c
 * evaluates to NaN -- summed over every residual evaluation (stages of
 * or_step / or_run and or_residual) since the last or_trace_reset().  The
 * faces counted are the x-faces 0..nx of every row and the y-faces 0..ny of
 * every column (a periodic grid counts its boundary face twice). */
long long or_trace_count(void);
void or_trace_reset(void);

/* Cells whose averages are not admissible (Euler: rho <= 0 or p <= 0) or
 * hold a non-finite value; 0 when the state is admissible. */
long long or_inadmissible(const or_problem* P, const double* U);

/* Maximum Rusanov wave speeds over the mesh from cell averages. */
void or_max_speed(const or_problem* P, const double* U, double* ax, double* ay);

/* Time-step rule of Sec. 4 ("Time stepping"); smooth != 0 uses dx^(k/3). */
double or_dt(const or_problem* P, const double* U, double cfl, int smooth);

/* End-of-step OE, in place (eq. 9 / eq. 1dOE_system / eq. 2dOE_system).
 * If theta != NULL it receives the damping exponent per cell. */
int or_oe(const or_problem* P, double dt, double* U, double* theta);

/* One SSP-RK3 step (eq. 3 / eq. 12) followed by OE, in place. */
int or_step(const or_problem* P, double* U, double dt);
/* Steps or_run discarded since the last reset (the safeguard's retries with
 * half the step size). */
long or_rejected_steps(int reset);

/* Advance to time T (last step clamped).  max_steps <= 0: unlimited.
 * nsteps_or_T: if T <= 0, runs exactly nsteps accepted steps instead.  With
 * pp_limiter (Euler), a step whose stage averages leave the admissible set is
 * discarded and retried with the step size halved (again and again, at most
 * 30 times; an accepted step restores the full size).  Returns 0 on success,
 * -1 on a non-finite value or after 30 halvings. */
int or_run(const or_problem* P, double* U, double T, long nsteps, double cfl, int smooth,
           double* t_out, long* nsteps_out);

#ifdef __cplusplus
}
#endif
#endif
