/*
 * orc.h -- plain FP64 CPU oracle for the MUSCL-Hancock step of the
 * vibrationally excited gas model (Khrapov & Khoperskov 2018).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header or constant with the CUDA path.
 *
 * Model (Sec. 2.1): eqs. 1-5 (continuity, momentum, total energy with pump Q
 * and sink I, vibrational energy relaxing with time tau), eq. 6 (power-law
 * closures tau, Q, I in rho and T), eq. 7 (p = R rho T).  Units (Sec. 2.3,
 * normalisation paragraph): rho0 = p0 = R = 1, so T0 = 1; tau0 is kept as a
 * free parameter and Q0 = I0 = S / tau0 (the definition of S under eq. 8 with
 * the equilibrium condition Q0 = I0 of eq. 3).
 *
 * Conserved state per cell, d = dim:  (rho, rho*v_1 .. rho*v_d, E, E_nu),
 * nf = d + 3 fields.  Arrays are field-major structure-of-arrays:
 * U[f * ncell + idx], idx = i + nx * (j + ny * k).  Periodic in every axis.
 */
#ifndef ORC_H
#define ORC_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MINMOD  0
#define ORC_VANLEER 1
#define ORC_MC      2

typedef struct {
  double gamma;     /* adiabatic exponent, eq. 5 */
  double Ck;        /* C_k = dE_nue / (R dT), under eq. 8 */
  double S;         /* degree of non-equilibrium S = tau0 Q0 / (R T0), under eq. 8 */
  double tau0;      /* relaxation time at equilibrium; +inf = frozen limit */
  double tau_rho, tau_T, Q_rho, Q_T, I_rho, I_T;   /* eq. 6 exponents */
  double cfl;       /* factor applied to the eq. 16 bound */
  double c_tau;     /* dt <= c_tau * min tau (explicit source bound) */
  int limiter;      /* ORC_MINMOD (default), ORC_VANLEER, ORC_MC */
} orc_params;

/* Pointwise pieces (one cell state u[nf], dim = 1..3). */
double orc_pressure(const orc_params* P, int dim, const double* u);          /* eq. 5 */
void   orc_flux(const orc_params* P, int dim, int axis, const double* u, double* F); /* F, G, H of eq. 15 */
void   orc_source(const orc_params* P, int dim, const double* u, double* Y); /* Y of eq. 15, eq. 6 */
void   orc_hll(const orc_params* P, int dim, int axis, const double* uL, const double* uR, double* F); /* eq. 13 */
double orc_limiter(int limiter, double a, double b);                          /* TVD slope limiter */
int    orc_physical(const orc_params* P, int dim, const double* u);           /* rho > 0, p > 0, finite */

/* One MUSCL-Hancock step (eqs. 13-15, xi = 0) on a periodic grid.
   n[0..dim-1] = cells per axis, h = cell size, U and Unew are nf*ncell arrays.
   Returns 0, or -1 if any new state is non-physical (rho <= 0, p <= 0, NaN),
   or -2 on allocation failure. */
int orc_step(const orc_params* P, int dim, const long* n, double h, double dt,
             const double* U, double* Unew);

/* The same step for one cell `idx` only, recomputing its neighbourhood; out[nf].
   Bitwise identical to orc_step's value at that cell. */
void orc_step_cell(const orc_params* P, int dim, const long* n, double h, double dt,
                   const double* U, long idx, double* out);

/* Time step of eq. 16 times cfl, capped by c_tau * min tau. */
double orc_dt(const orc_params* P, int dim, const long* n, double h, const double* U);

/* Advance U in place until t_end (last step clamped) or max_steps steps.
   Writes the reached time and the number of steps taken. Returns 0, -1 on a
   non-physical state (stops there), -2 on allocation failure. */
int orc_run(const orc_params* P, int dim, const long* n, double h, double* U,
            double t0, double t_end, long max_steps, double* t_out, long* steps_out);

/* 1D boundary conditions (per side). */
#define ORC_BC_PERIODIC 0
#define ORC_BC_REFLECT  1   /* solid wall: mirrored ghost cells, velocity reversed */
#define ORC_BC_OUTFLOW  2   /* zero-gradient ghost cells */
#define ORC_BC_DRIVEN   3   /* x = 0 only: ghost cells hold a prescribed wave */

/* Prescribed wave of the driven boundary: a ghost cell at x (< 0) holds
   U(x, t) = base + Re(amp e^{i (k x - omega t)}), k = k_re + i k_im. */
typedef struct {
  double omega, k_re, k_im;
  double base[4], amp_re[4], amp_im[4];
} orc_drive;

/* As orc_step_bc1 / orc_run_bc1 with a driven boundary at x = 0 (bc_lo =
   ORC_BC_DRIVEN) evaluated at the step's start time t. */
int orc_step_bc1d(const orc_params* P, long N, double h, double dt, int bc_lo, int bc_hi,
                  const orc_drive* drive, double t, const double* U, double* Unew);
int orc_run_bc1d(const orc_params* P, long N, double h, int bc_lo, int bc_hi,
                 const orc_drive* drive, double* U, double t0, double t_end, long max_steps,
                 double* t_out, long* steps_out);

/* One 1D step (and a run to t_end) with the boundary conditions bc_lo at
   x = 0 and bc_hi at x = L, on two ghost cells per side.  N >= 2.
   Returns as orc_step / orc_run, and -3 for N < 2. */
int orc_step_bc1(const orc_params* P, long N, double h, double dt, int bc_lo, int bc_hi,
                 const double* U, double* Unew);
int orc_run_bc1(const orc_params* P, long N, double h, int bc_lo, int bc_hi, double* U,
                double t0, double t_end, long max_steps, double* t_out, long* steps_out);

/* Heun (SSP-RK2) time integration of the same spatial operator on a periodic
   grid: U* = U + dt L(U), U^{n+1} = (U + U*)/2 + dt/2 L(U*), with L the
   flux divergence of eq. 13/14 faces at the stage's own time level plus Y.
   Returns and runs as orc_step / orc_run. */
int orc_step_heun(const orc_params* P, int dim, const long* n, double h, double dt,
                  const double* U, double* Unew);
int orc_run_heun(const orc_params* P, int dim, const long* n, double h, double* U,
                 double t0, double t_end, long max_steps, double* t_out, long* steps_out);

/* 2D problems with boundaries, a map of the active medium and driven cells
   (the paper's two-dimensional active-sector problem, Sec. 3).
   bc[0], bc[1]: x = 0, x = Lx; bc[2], bc[3]: y = 0, y = Ly; each
   ORC_BC_PERIODIC, ORC_BC_REFLECT (solid wall: mirrored ghosts with the
   normal momentum reversed) or ORC_BC_OUTFLOW (zero-gradient ghosts); a
   non-periodic axis needs n >= 2.
   Medium: row j (0 <= j < ny) is the active medium of P (relaxation, pump
   and sink) in the cells act_lo[j] <= i < act_hi[j] and frozen (no
   relaxation, pump or sink: Y = 0) elsewhere; act_lo == NULL: active
   everywhere.  The rest state rho = p = 1, v = 0, E_nu = C_k + S is steady in
   both.  A ghost cell takes the medium of the cell whose state it holds.
   Driven cells: drv_lo[j] <= i < drv_hi[j] (drv_lo == NULL: none) hold, at
   every new time level t, rho = 1 + amp sin(omega t), v = 0,
   p = 1 + gamma amp sin(omega t), E_nu = rho (C_k + S): a pulsating acoustic
   source (frozen sound speed c0^2 = gamma at rho0 = p0 = 1). */
typedef struct {
  const int* act_lo;
  const int* act_hi;
  const int* drv_lo;
  const int* drv_hi;
  double omega, amp;
} orc_medium2;

/* One step of the 2D problem (fields rho, rho u, rho v, E, E_nu; U[f*nx*ny +
   i + nx*j]) from time t with time step dt.  Returns as orc_step, -3 on a
   bad argument. */
int orc_step2m(const orc_params* P, long nx, long ny, double h, double dt, const int* bc,
               const orc_medium2* M, double t, const double* U, double* Unew);
int orc_run2m(const orc_params* P, long nx, long ny, double h, const int* bc,
              const orc_medium2* M, double* U, double t0, double t_end, long max_steps,
              double* t_out, long* steps_out);

/* Number of OpenMP threads the array loops use (1 without OpenMP), and a
   way to change it (timing only: results do not depend on it). */
int orc_threads(void);
void orc_set_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
