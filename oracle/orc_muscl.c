/*
 * orc_muscl.c -- plain FP64 CPU oracle of the MUSCL-Hancock step
 * (Khrapov & Khoperskov 2018, Sec. 2.3, eqs. 13-16).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.  Built with
 * -O2 -ffp-contract=off and no fast-math so every operation is a plain IEEE
 * double operation in source order.
 *
 * The step, in the paper's order (eq. 14 with xi = 0, eq. 15, eq. 13):
 *   1. slopes:   Theta_j h = lim(U_j - U_{j-1}, U_{j+1} - U_j) per conserved
 *                field and axis (eq. 14 reconstructs U; the limiter is not
 *                named, minmod by default);
 *                if an extrapolated state U_j +- Theta_j h / 2 of any axis is
 *                non-physical, all slopes of that cell are set to zero;
 *   2. predictor (the half step of the "two-step predictor-corrector"):
 *                U^{n+1/2}_j = U_j - dt/(2h) sum_axes [F(U_j + Th/2) - F(U_j - Th/2)]
 *                              + dt/2 Y(U_j);
 *   3. face states (eq. 14, xi = 0):
 *                U^L_{j+1/2} = U^{n+1/2}_j + Theta_j h/2,
 *                U^R_{j+1/2} = U^{n+1/2}_{j+1} - Theta_{j+1} h/2;
 *                a face with a non-physical state uses U_j, U_{j+1} instead;
 *   4. HLL flux (eq. 13) with S_L = min(u_L - c_L, u_R - c_R),
 *                S_R = max(u_L + c_L, u_R + c_R), c = sqrt(gamma p / rho);
 *   5. corrector (eq. 15):
 *                U^{n+1}_j = U_j - dt/h sum_axes (F_{j+1/2} - F_{j-1/2})
 *                            + dt Y(U^{n+1/2}_j).
 * Source Y (the MUSCL Y vector of Sec. 2.3 with f = 0):
 *   Y = (0, 0.., rho (Q - I), (rho C_k T - E_nu)/tau + rho Q),
 * tau, Q, I from eq. 6, T = p / rho (eq. 7, R = 1), p from eq. 5.
 */
#include "orc.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NF_MAX 6

int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* eq. 5: E = p/(gamma-1) + rho |v|^2 / 2 + E_nu  ->  p */
double orc_pressure(const orc_params* P, int dim, const double* u) {
  double rho = u[0];
  double kin = 0.0;
  for (int a = 0; a < dim; ++a) kin += u[1 + a] * u[1 + a];
  kin = 0.5 * kin / rho;
  return (P->gamma - 1.0) * (u[1 + dim] - kin - u[2 + dim]);
}

int orc_physical(const orc_params* P, int dim, const double* u) {
  double p = orc_pressure(P, dim, u);
  return isfinite(u[0]) && isfinite(p) && u[0] > 0.0 && p > 0.0;
}

/* Flux along `axis`: F (x), G (y) of eq. 15, and the analogous z flux. */
void orc_flux(const orc_params* P, int dim, int axis, const double* u, double* F) {
  double rho = u[0];
  double va = u[1 + axis] / rho;
  double p = orc_pressure(P, dim, u);
  F[0] = u[1 + axis];
  for (int b = 0; b < dim; ++b) F[1 + b] = u[1 + b] * va + (b == axis ? p : 0.0);
  F[1 + dim] = va * (u[1 + dim] + p);
  F[2 + dim] = va * u[2 + dim];
}

/* Y of eq. 15 with f = 0, closures of eq. 6, T from eq. 7 with R = 1. */
void orc_source(const orc_params* P, int dim, const double* u, double* Y) {
  int nf = dim + 3;
  double rho = u[0];
  double p = orc_pressure(P, dim, u);
  double T = p / rho;
  double Q0 = P->S / P->tau0;   /* S = tau0 Q0 / (R T0) */
  double I0 = Q0;               /* equilibrium of eq. 3 */
  double tau = P->tau0 * pow(rho, P->tau_rho) * pow(T, P->tau_T);
  double Q = Q0 * pow(rho, P->Q_rho) * pow(T, P->Q_T);
  double I = I0 * pow(rho, P->I_rho) * pow(T, P->I_T);
  for (int f = 0; f < nf; ++f) Y[f] = 0.0;
  Y[1 + dim] = rho * (Q - I);
  Y[2 + dim] = (rho * P->Ck * T - u[2 + dim]) / tau + rho * Q;
}

/* eq. 13 */
void orc_hll(const orc_params* P, int dim, int axis, const double* uL, const double* uR, double* F) {
  int nf = dim + 3;
  double FL[NF_MAX], FR[NF_MAX];
  double pL = orc_pressure(P, dim, uL), pR = orc_pressure(P, dim, uR);
  double vL = uL[1 + axis] / uL[0], vR = uR[1 + axis] / uR[0];
  double cL = sqrt(P->gamma * pL / uL[0]), cR = sqrt(P->gamma * pR / uR[0]);
  double SL = fmin(vL - cL, vR - cR);
  double SR = fmax(vL + cL, vR + cR);
  orc_flux(P, dim, axis, uL, FL);
  orc_flux(P, dim, axis, uR, FR);
  if (0.0 < SL) {
    for (int f = 0; f < nf; ++f) F[f] = FL[f];
  } else if (0.0 > SR) {
    for (int f = 0; f < nf; ++f) F[f] = FR[f];
  } else {
    for (int f = 0; f < nf; ++f)
      F[f] = (SR * FL[f] - SL * FR[f] + SL * SR * (uR[f] - uL[f])) / (SR - SL);
  }
}

double orc_limiter(int limiter, double a, double b) {
  if (a * b <= 0.0) return 0.0;
  double s = a > 0.0 ? 1.0 : -1.0;
  switch (limiter) {
    case ORC_VANLEER:
      return 2.0 * a * b / (a + b);
    case ORC_MC: {
      double m = fmin(2.0 * fabs(a), 2.0 * fabs(b));
      return s * fmin(m, 0.5 * fabs(a + b));
    }
    default:
      return s * fmin(fabs(a), fabs(b));
  }
}

/* ---------------------------------------------------------------- grid */

typedef struct {
  int dim, nf;
  long n[3];
  long ncell;
} grid_t;

static grid_t make_grid(int dim, const long* n) {
  grid_t g;
  g.dim = dim;
  g.nf = dim + 3;
  g.n[0] = g.n[1] = g.n[2] = 1;
  g.ncell = 1;
  for (int a = 0; a < dim; ++a) { g.n[a] = n[a]; g.ncell *= n[a]; }
  return g;
}

/* periodic neighbour of cell idx along axis a at offset s (|s| <= 2) */
static long neighbour(const grid_t* g, long idx, int a, int s) {
  long c[3];
  c[0] = idx % g->n[0];
  c[1] = (idx / g->n[0]) % g->n[1];
  c[2] = idx / (g->n[0] * g->n[1]);
  c[a] = ((c[a] + s) % g->n[a] + g->n[a]) % g->n[a];
  return c[0] + g->n[0] * (c[1] + g->n[1] * c[2]);
}

static void gather(const grid_t* g, const double* U, long idx, double* u) {
  for (int f = 0; f < g->nf; ++f) u[f] = U[(long)f * g->ncell + idx];
}

/* Steps 1-2 for cell q: slopes dU[a][f] (= Theta h) and the half-step state uh. */
static void predict(const orc_params* P, const grid_t* g, double h, double dt,
                    const double* U, long q, double dU[3][NF_MAX], double* uh) {
  int dim = g->dim, nf = g->nf;
  double u[NF_MAX], um[NF_MAX], up[NF_MAX];
  gather(g, U, q, u);
  int ok = 1;
  for (int a = 0; a < dim; ++a) {
    gather(g, U, neighbour(g, q, a, -1), um);
    gather(g, U, neighbour(g, q, a, +1), up);
    for (int f = 0; f < nf; ++f) dU[a][f] = orc_limiter(P->limiter, u[f] - um[f], up[f] - u[f]);
  }
  for (int a = 0; a < dim && ok; ++a) {
    for (int f = 0; f < nf; ++f) { um[f] = u[f] - 0.5 * dU[a][f]; up[f] = u[f] + 0.5 * dU[a][f]; }
    if (!orc_physical(P, dim, um) || !orc_physical(P, dim, up)) ok = 0;
  }
  if (!ok)
    for (int a = 0; a < dim; ++a)
      for (int f = 0; f < nf; ++f) dU[a][f] = 0.0;

  double Y[NF_MAX], Fm[NF_MAX], Fp[NF_MAX], div[NF_MAX];
  for (int f = 0; f < nf; ++f) div[f] = 0.0;
  for (int a = 0; a < dim; ++a) {
    for (int f = 0; f < nf; ++f) { um[f] = u[f] - 0.5 * dU[a][f]; up[f] = u[f] + 0.5 * dU[a][f]; }
    orc_flux(P, dim, a, up, Fp);
    orc_flux(P, dim, a, um, Fm);
    for (int f = 0; f < nf; ++f) div[f] += Fp[f] - Fm[f];
  }
  orc_source(P, dim, u, Y);
  for (int f = 0; f < nf; ++f) uh[f] = u[f] - dt / (2.0 * h) * div[f] + 0.5 * dt * Y[f];
}

/* Steps 3-4 for the face between cell l and its +axis neighbour r. */
static void face_flux(const orc_params* P, const grid_t* g, const double* U, int a,
                      long l, const double dUl[3][NF_MAX], const double* uhl,
                      long r, const double dUr[3][NF_MAX], const double* uhr, double* F) {
  int nf = g->nf, dim = g->dim;
  double uL[NF_MAX], uR[NF_MAX];
  for (int f = 0; f < nf; ++f) {
    uL[f] = uhl[f] + 0.5 * dUl[a][f];
    uR[f] = uhr[f] - 0.5 * dUr[a][f];
  }
  if (!orc_physical(P, dim, uL) || !orc_physical(P, dim, uR)) {
    gather(g, U, l, uL);
    gather(g, U, r, uR);
  }
  orc_hll(P, dim, a, uL, uR, F);
}

/* Step 5 for one cell. */
static void correct(const orc_params* P, const grid_t* g, double h, double dt,
                    const double* u, const double* uh, double Fp[3][NF_MAX],
                    double Fm[3][NF_MAX], double* out) {
  int nf = g->nf, dim = g->dim;
  double Y[NF_MAX], div[NF_MAX];
  for (int f = 0; f < nf; ++f) div[f] = 0.0;
  for (int a = 0; a < dim; ++a)
    for (int f = 0; f < nf; ++f) div[f] += Fp[a][f] - Fm[a][f];
  orc_source(P, dim, uh, Y);
  for (int f = 0; f < nf; ++f) out[f] = u[f] - dt / h * div[f] + dt * Y[f];
}

int orc_step(const orc_params* P, int dim, const long* n, double h, double dt,
             const double* U, double* Unew) {
  grid_t g = make_grid(dim, n);
  int nf = g.nf;
  long N = g.ncell;
  double (*dU)[3][NF_MAX] = malloc(sizeof(double[3][NF_MAX]) * (size_t)N);
  double (*uh)[NF_MAX] = malloc(sizeof(double[NF_MAX]) * (size_t)N);
  double (*Fface)[3][NF_MAX] = malloc(sizeof(double[3][NF_MAX]) * (size_t)N);
  if (!dU || !uh || !Fface) { free(dU); free(uh); free(Fface); return -2; }

#pragma omp parallel for schedule(static)
  for (long q = 0; q < N; ++q) predict(P, &g, h, dt, U, q, dU[q], uh[q]);

#pragma omp parallel for schedule(static)
  for (long q = 0; q < N; ++q)
    for (int a = 0; a < dim; ++a) {
      long r = neighbour(&g, q, a, +1);
      face_flux(P, &g, U, a, q, dU[q], uh[q], r, dU[r], uh[r], Fface[q][a]);
    }

  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (long q = 0; q < N; ++q) {
    double u[NF_MAX], out[NF_MAX], Fp[3][NF_MAX], Fm[3][NF_MAX];
    gather(&g, U, q, u);
    for (int a = 0; a < dim; ++a) {
      long l = neighbour(&g, q, a, -1);
      memcpy(Fp[a], Fface[q][a], sizeof(double) * NF_MAX);
      memcpy(Fm[a], Fface[l][a], sizeof(double) * NF_MAX);
    }
    correct(P, &g, h, dt, u, uh[q], Fp, Fm, out);
    for (int f = 0; f < nf; ++f) Unew[(long)f * N + q] = out[f];
    if (!orc_physical(P, dim, out)) bad = 1;
  }
  free(dU); free(uh); free(Fface);
  return bad ? -1 : 0;
}

void orc_step_cell(const orc_params* P, int dim, const long* n, double h, double dt,
                   const double* U, long idx, double* out) {
  grid_t g = make_grid(dim, n);
  double dUc[3][NF_MAX], uhc[NF_MAX], dUn[3][NF_MAX], uhn[NF_MAX];
  double Fp[3][NF_MAX], Fm[3][NF_MAX], u[NF_MAX];
  predict(P, &g, h, dt, U, idx, dUc, uhc);
  for (int a = 0; a < dim; ++a) {
    long r = neighbour(&g, idx, a, +1);
    predict(P, &g, h, dt, U, r, dUn, uhn);
    face_flux(P, &g, U, a, idx, dUc, uhc, r, dUn, uhn, Fp[a]);
    long l = neighbour(&g, idx, a, -1);
    predict(P, &g, h, dt, U, l, dUn, uhn);
    face_flux(P, &g, U, a, l, dUn, uhn, idx, dUc, uhc, Fm[a]);
  }
  gather(&g, U, idx, u);
  correct(P, &g, h, dt, u, uhc, Fp, Fm, out);
}

/* eq. 16: dt < min_j min(h / (2|v_j|), h / (|v_j| + c_j)), times cfl;
   then dt <= c_tau * min_j tau_j (the explicit source needs it when tau is short). */
double orc_dt(const orc_params* P, int dim, const long* n, double h, const double* U) {
  grid_t g = make_grid(dim, n);
  double smax = 0.0, taumin = INFINITY;
  for (long q = 0; q < g.ncell; ++q) {
    double u[NF_MAX];
    gather(&g, U, q, u);
    double p = orc_pressure(P, dim, u);
    double v2 = 0.0;
    for (int a = 0; a < dim; ++a) v2 += (u[1 + a] / u[0]) * (u[1 + a] / u[0]);
    double v = sqrt(v2);
    double c = sqrt(P->gamma * p / u[0]);
    double s = fmax(2.0 * v, v + c);
    if (s > smax) smax = s;
    double T = p / u[0];
    double tau = P->tau0 * pow(u[0], P->tau_rho) * pow(T, P->tau_T);
    if (tau < taumin) taumin = tau;
  }
  double dt = P->cfl * h / smax;
  if (isfinite(taumin) && P->c_tau * taumin < dt) dt = P->c_tau * taumin;
  return dt;
}

int orc_run(const orc_params* P, int dim, const long* n, double h, double* U,
            double t0, double t_end, long max_steps, double* t_out, long* steps_out) {
  grid_t g = make_grid(dim, n);
  size_t bytes = sizeof(double) * (size_t)g.nf * (size_t)g.ncell;
  double* tmp = malloc(bytes);
  if (!tmp) return -2;
  double t = t0;
  long k = 0;
  int rc = 0;
  while (t < t_end && k < max_steps) {
    double dt = orc_dt(P, dim, n, h, U);
    int last = 0;
    if (dt >= t_end - t) { dt = t_end - t; last = 1; }
    rc = orc_step(P, dim, n, h, dt, U, tmp);
    memcpy(U, tmp, bytes);
    t = last ? t_end : t + dt;
    ++k;
    if (rc != 0) break;
  }
  free(tmp);
  *t_out = t;
  *steps_out = k;
  return rc;
}

/* ------------------------------------------------------------ 1D boundaries */

/* One 1D step with boundary conditions at x = 0 (bc_lo) and x = L (bc_hi):
   ORC_BC_PERIODIC, ORC_BC_REFLECT (solid wall: mirrored ghost cells with the
   velocity reversed) or ORC_BC_OUTFLOW (zero-gradient ghost cells).  The grid
   is extended by two ghost cells per side filled by those rules; the predictor
   runs on cells -1..N, the faces -1/2..N-1/2, the update on 0..N-1, with the
   same functions as the periodic step. */
static void fill_ghost(const grid_t* g, const double* U, int bc, long src_near, long src_far,
                       double* near, double* far) {
  for (int f = 0; f < g->nf; ++f) {
    if (bc == ORC_BC_OUTFLOW) {
      near[f] = U[(long)f * g->ncell + src_near];
      far[f] = near[f];
    } else {
      near[f] = U[(long)f * g->ncell + src_near];
      far[f] = U[(long)f * g->ncell + src_far];
    }
  }
  if (bc == ORC_BC_REFLECT) {
    near[1] = -near[1];
    far[1] = -far[1];
  }
}

/* Ghost cell at position x of the driven boundary at time t. */
static void drive_state(const orc_drive* d, double x, double t, double* u) {
  const double env = exp(-d->k_im * x);
  const double ph = d->k_re * x - d->omega * t;
  const double c = cos(ph), s = sin(ph);
  for (int f = 0; f < 4; ++f) u[f] = d->base[f] + env * (d->amp_re[f] * c - d->amp_im[f] * s);
}

int orc_step_bc1(const orc_params* P, long N, double h, double dt, int bc_lo, int bc_hi,
                 const double* U, double* Unew) {
  return orc_step_bc1d(P, N, h, dt, bc_lo, bc_hi, NULL, 0.0, U, Unew);
}

int orc_step_bc1d(const orc_params* P, long N, double h, double dt, int bc_lo, int bc_hi,
                  const orc_drive* drive, double t, const double* U, double* Unew) {
  if (bc_lo == ORC_BC_DRIVEN && !drive) return -3;
  if (bc_hi == ORC_BC_DRIVEN) return -3;
  if (N < 2) return -3;
  const long n1 = N;
  grid_t g = make_grid(1, &n1);
  const long ne = N + 4;
  grid_t ge = make_grid(1, &ne);
  const int nf = 4;
  double* Ue = malloc(sizeof(double) * (size_t)nf * (size_t)ne);
  double (*dU)[3][NF_MAX] = malloc(sizeof(double[3][NF_MAX]) * (size_t)ne);
  double (*uh)[NF_MAX] = malloc(sizeof(double[NF_MAX]) * (size_t)ne);
  double (*Fface)[NF_MAX] = malloc(sizeof(double[NF_MAX]) * (size_t)ne);
  if (!Ue || !dU || !uh || !Fface) { free(Ue); free(dU); free(uh); free(Fface); return -2; }
  for (int f = 0; f < nf; ++f)
    for (long j = 0; j < N; ++j) Ue[(long)f * ne + j + 2] = U[(long)f * N + j];
  double gn[NF_MAX], gf[NF_MAX];
  /* left ghosts: extended index 1 (cell -1) and 0 (cell -2) */
  if (bc_lo == ORC_BC_PERIODIC) fill_ghost(&g, U, bc_lo, N - 1, N - 2, gn, gf);
  else if (bc_lo == ORC_BC_DRIVEN) {
    drive_state(drive, -0.5 * h, t, gn);   /* cell -1 centre */
    drive_state(drive, -1.5 * h, t, gf);   /* cell -2 centre */
  } else fill_ghost(&g, U, bc_lo, 0, 1, gn, gf);
  for (int f = 0; f < nf; ++f) { Ue[(long)f * ne + 1] = gn[f]; Ue[(long)f * ne + 0] = gf[f]; }
  /* right ghosts: extended index N+2 (cell N) and N+3 (cell N+1) */
  if (bc_hi == ORC_BC_PERIODIC) fill_ghost(&g, U, bc_hi, 0, 1, gn, gf);
  else fill_ghost(&g, U, bc_hi, N - 1, N - 2, gn, gf);
  for (int f = 0; f < nf; ++f) { Ue[(long)f * ne + N + 2] = gn[f]; Ue[(long)f * ne + N + 3] = gf[f]; }

  for (long q = 1; q <= N + 2; ++q) predict(P, &ge, h, dt, Ue, q, dU[q], uh[q]);
  for (long q = 1; q <= N + 1; ++q)
    face_flux(P, &ge, Ue, 0, q, dU[q], uh[q], q + 1, dU[q + 1], uh[q + 1], Fface[q]);
  int bad = 0;
  for (long q = 2; q <= N + 1; ++q) {
    double u[NF_MAX], out[NF_MAX], Fp[3][NF_MAX], Fm[3][NF_MAX];
    gather(&ge, Ue, q, u);
    memcpy(Fp[0], Fface[q], sizeof(double) * NF_MAX);
    memcpy(Fm[0], Fface[q - 1], sizeof(double) * NF_MAX);
    correct(P, &ge, h, dt, u, uh[q], Fp, Fm, out);
    for (int f = 0; f < nf; ++f) Unew[(long)f * N + q - 2] = out[f];
    if (!orc_physical(P, 1, out)) bad = 1;
  }
  free(Ue); free(dU); free(uh); free(Fface);
  return bad ? -1 : 0;
}

int orc_run_bc1(const orc_params* P, long N, double h, int bc_lo, int bc_hi, double* U,
                double t0, double t_end, long max_steps, double* t_out, long* steps_out) {
  return orc_run_bc1d(P, N, h, bc_lo, bc_hi, NULL, U, t0, t_end, max_steps, t_out, steps_out);
}

int orc_run_bc1d(const orc_params* P, long N, double h, int bc_lo, int bc_hi,
                 const orc_drive* drive, double* U, double t0, double t_end, long max_steps,
                 double* t_out, long* steps_out) {
  size_t bytes = sizeof(double) * 4 * (size_t)N;
  double* tmp = malloc(bytes);
  if (!tmp) return -2;
  const long n1 = N;
  double t = t0;
  long k = 0;
  int rc = 0;
  while (t < t_end && k < max_steps) {
    double dt = orc_dt(P, 1, &n1, h, U);
    int last = 0;
    if (dt >= t_end - t) { dt = t_end - t; last = 1; }
    rc = orc_step_bc1d(P, N, h, dt, bc_lo, bc_hi, drive, t, U, tmp);
    memcpy(U, tmp, bytes);
    t = last ? t_end : t + dt;
    ++k;
    if (rc != 0) break;
  }
  free(tmp);
  *t_out = t;
  *steps_out = k;
  return rc;
}

/* ------------------------------------------------- 2D boundaries, medium map, drive */

/* Cell (0..n-1) whose state position j (-2..n+1) holds along an axis of n
   cells, and whether its normal momentum is reversed (solid wall). */
static long ghost_map(long j, long n, int bc_lo, int bc_hi, int* flip) {
  *flip = 0;
  if (j >= 0 && j < n) return j;
  const int bc = j < 0 ? bc_lo : bc_hi;
  if (bc == ORC_BC_PERIODIC) return ((j % n) + n) % n;
  if (bc == ORC_BC_REFLECT) {
    *flip = 1;
    return j < 0 ? -1 - j : 2 * n - 1 - j;
  }
  return j < 0 ? 0 : n - 1;   /* outflow: zero gradient */
}

static int active_cell(const orc_medium2* M, long i, long j) {
  if (!M || !M->act_lo) return 1;
  return i >= M->act_lo[j] && i < M->act_hi[j];
}

static int driven_cell(const orc_medium2* M, long i, long j) {
  if (!M || !M->drv_lo) return 0;
  return i >= M->drv_lo[j] && i < M->drv_hi[j];
}

/* The pulsating source at time t. */
static void pulse_state(const orc_params* P, const orc_medium2* M, double t, double* u) {
  const double s = M->amp * sin(M->omega * t);
  const double rho = 1.0 + s, p = 1.0 + P->gamma * s;
  const double Ev = rho * (P->Ck + P->S);
  u[0] = rho;
  u[1] = 0.0;
  u[2] = 0.0;
  u[3] = p / (P->gamma - 1.0) + Ev;
  u[4] = Ev;
}

/* The grid is extended by two ghost layers per side; position (a, b) of the
   extended grid holds cell (map_x(a - 2), map_y(b - 2)) with the momenta of
   the wall-mirrored axes reversed (so corner ghosts are mirrored in both).
   Predictors run on positions 1..n+2 of both axes, faces on those that
   bound a grid cell, updates on the grid cells, each with the functions of
   the periodic step and the cell's own medium. */
int orc_step2m(const orc_params* P, long nx, long ny, double h, double dt, const int* bc,
               const orc_medium2* M, double t, const double* U, double* Unew) {
  if (!bc || nx < 1 || ny < 1) return -3;
  for (int k = 0; k < 4; ++k)
    if (bc[k] < ORC_BC_PERIODIC || bc[k] > ORC_BC_OUTFLOW) return -3;
  if ((bc[0] != ORC_BC_PERIODIC || bc[1] != ORC_BC_PERIODIC) && nx < 2) return -3;
  if ((bc[2] != ORC_BC_PERIODIC || bc[3] != ORC_BC_PERIODIC) && ny < 2) return -3;
  if (M && M->drv_lo && !(M->omega == M->omega)) return -3;
  const int nf = 5;
  const long N = nx * ny, ex = nx + 4, ey = ny + 4, NE = ex * ey;
  const long ne[2] = {ex, ey};
  grid_t ge = make_grid(2, ne);
  orc_params Pp = *P;
  Pp.tau0 = INFINITY;                           /* the passive medium: frozen, Y = 0 */
  double* Ue = malloc(sizeof(double) * (size_t)nf * (size_t)NE);
  unsigned char* act = malloc((size_t)NE);
  double (*dU)[3][NF_MAX] = malloc(sizeof(double[3][NF_MAX]) * (size_t)NE);
  double (*uh)[NF_MAX] = malloc(sizeof(double[NF_MAX]) * (size_t)NE);
  double (*Fface)[3][NF_MAX] = malloc(sizeof(double[3][NF_MAX]) * (size_t)NE);
  if (!Ue || !act || !dU || !uh || !Fface) {
    free(Ue); free(act); free(dU); free(uh); free(Fface);
    return -2;
  }
  for (long b = 0; b < ey; ++b)
    for (long a = 0; a < ex; ++a) {
      int fx, fy;
      const long i = ghost_map(a - 2, nx, bc[0], bc[1], &fx);
      const long j = ghost_map(b - 2, ny, bc[2], bc[3], &fy);
      const long e = a + ex * b, q = i + nx * j;
      for (int f = 0; f < nf; ++f) Ue[(long)f * NE + e] = U[(long)f * N + q];
      if (fx) Ue[1 * NE + e] = -Ue[1 * NE + e];
      if (fy) Ue[2 * NE + e] = -Ue[2 * NE + e];
      act[e] = (unsigned char)active_cell(M, i, j);
    }

#pragma omp parallel for schedule(static)
  for (long b = 1; b <= ny + 2; ++b)
    for (long a = 1; a <= nx + 2; ++a) {
      const long e = a + ex * b;
      predict(act[e] ? P : &Pp, &ge, h, dt, Ue, e, dU[e], uh[e]);
    }

#pragma omp parallel for schedule(static)
  for (long b = 1; b <= ny + 1; ++b)
    for (long a = 1; a <= nx + 1; ++a) {
      const long e = a + ex * b;
      if (b >= 2)   /* x face between (a, b) and (a + 1, b) */
        face_flux(P, &ge, Ue, 0, e, dU[e], uh[e], e + 1, dU[e + 1], uh[e + 1], Fface[e][0]);
      if (a >= 2)   /* y face between (a, b) and (a, b + 1) */
        face_flux(P, &ge, Ue, 1, e, dU[e], uh[e], e + ex, dU[e + ex], uh[e + ex], Fface[e][1]);
    }

  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (long j = 0; j < ny; ++j)
    for (long i = 0; i < nx; ++i) {
      const long e = (i + 2) + ex * (j + 2), q = i + nx * j;
      double u[NF_MAX], out[NF_MAX], Fp[3][NF_MAX], Fm[3][NF_MAX];
      gather(&ge, Ue, e, u);
      memcpy(Fp[0], Fface[e][0], sizeof(double) * NF_MAX);
      memcpy(Fm[0], Fface[e - 1][0], sizeof(double) * NF_MAX);
      memcpy(Fp[1], Fface[e][1], sizeof(double) * NF_MAX);
      memcpy(Fm[1], Fface[e - ex][1], sizeof(double) * NF_MAX);
      correct(act[e] ? P : &Pp, &ge, h, dt, u, uh[e], Fp, Fm, out);
      if (driven_cell(M, i, j)) pulse_state(P, M, t + dt, out);
      for (int f = 0; f < nf; ++f) Unew[(long)f * N + q] = out[f];
      if (!orc_physical(P, 2, out)) bad = 1;
    }
  free(Ue); free(act); free(dU); free(uh); free(Fface);
  return bad ? -1 : 0;
}

int orc_run2m(const orc_params* P, long nx, long ny, double h, const int* bc,
              const orc_medium2* M, double* U, double t0, double t_end, long max_steps,
              double* t_out, long* steps_out) {
  const size_t bytes = sizeof(double) * 5 * (size_t)nx * (size_t)ny;
  double* tmp = malloc(bytes);
  if (!tmp) return -2;
  const long n2[2] = {nx, ny};
  double t = t0;
  long k = 0;
  int rc = 0;
  while (t < t_end && k < max_steps) {
    double dt = orc_dt(P, 2, n2, h, U);
    int last = 0;
    if (dt >= t_end - t) {
      dt = t_end - t;
      last = 1;
    }
    rc = orc_step2m(P, nx, ny, h, dt, bc, M, t, U, tmp);
    if (rc == -2 || rc == -3) break;
    memcpy(U, tmp, bytes);
    t = last ? t_end : t + dt;
    ++k;
    if (rc != 0) break;
  }
  free(tmp);
  *t_out = t;
  *steps_out = k;
  return rc;
}

/* ------------------------------------------------------------ Heun / SSP-RK2 */

/* Spatial operator of the method of lines on a periodic grid:
   L(U)_j = -1/h sum_axes (F_{j+1/2} - F_{j-1/2}) + Y(U_j), with the faces of
   eq. 13 between the piecewise-linear states of eq. 14 taken at time level n
   (U_j +- Theta_j h / 2, no half step), the same limiter and positivity guard
   as the MUSCL-Hancock step. */
static int rhs(const orc_params* P, const grid_t* g, double h, const double* U, double* Lu) {
  const int dim = g->dim, nf = g->nf;
  const long N = g->ncell;
  double (*dU)[3][NF_MAX] = malloc(sizeof(double[3][NF_MAX]) * (size_t)N);
  double (*Fface)[3][NF_MAX] = malloc(sizeof(double[3][NF_MAX]) * (size_t)N);
  double (*u0)[NF_MAX] = malloc(sizeof(double[NF_MAX]) * (size_t)N);
  if (!dU || !Fface || !u0) { free(dU); free(Fface); free(u0); return -2; }
  /* slopes: the predictor with dt = 0 leaves the state unchanged (U^{n+1/2} = U) */
#pragma omp parallel for schedule(static)
  for (long q = 0; q < N; ++q) predict(P, g, h, 0.0, U, q, dU[q], u0[q]);
#pragma omp parallel for schedule(static)
  for (long q = 0; q < N; ++q)
    for (int a = 0; a < dim; ++a) {
      long r = neighbour(g, q, a, +1);
      face_flux(P, g, U, a, q, dU[q], u0[q], r, dU[r], u0[r], Fface[q][a]);
    }
#pragma omp parallel for schedule(static)
  for (long q = 0; q < N; ++q) {
    double u[NF_MAX], Y[NF_MAX], div[NF_MAX];
    gather(g, U, q, u);
    for (int f = 0; f < nf; ++f) div[f] = 0.0;
    for (int a = 0; a < dim; ++a) {
      long l = neighbour(g, q, a, -1);
      for (int f = 0; f < nf; ++f) div[f] += Fface[q][a][f] - Fface[l][a][f];
    }
    orc_source(P, dim, u, Y);
    for (int f = 0; f < nf; ++f) Lu[(long)f * N + q] = -div[f] / h + Y[f];
  }
  free(dU); free(Fface); free(u0);
  return 0;
}

/* One Heun step (the two-stage predictor-corrector of eqs. 10-11 applied to
   the whole MUSCL operator):
     U*      = U^n + dt L(U^n)
     U^{n+1} = (U^n + U*) / 2 + dt/2 L(U*). */
int orc_step_heun(const orc_params* P, int dim, const long* n, double h, double dt,
                  const double* U, double* Unew) {
  grid_t g = make_grid(dim, n);
  const long M = (long)g.nf * g.ncell;
  double* Lu = malloc(sizeof(double) * (size_t)M);
  double* Us = malloc(sizeof(double) * (size_t)M);
  if (!Lu || !Us) { free(Lu); free(Us); return -2; }
  int rc = rhs(P, &g, h, U, Lu);
  if (rc == 0) {
    for (long i = 0; i < M; ++i) Us[i] = U[i] + dt * Lu[i];
    rc = rhs(P, &g, h, Us, Lu);
  }
  int bad = 0;
  if (rc == 0) {
    for (long i = 0; i < M; ++i) Unew[i] = 0.5 * (U[i] + Us[i]) + 0.5 * dt * Lu[i];
    for (long q = 0; q < g.ncell && !bad; ++q) {
      double u[NF_MAX];
      gather(&g, Unew, q, u);
      if (!orc_physical(P, dim, u)) bad = 1;
    }
  }
  free(Lu); free(Us);
  return rc ? rc : (bad ? -1 : 0);
}

int orc_run_heun(const orc_params* P, int dim, const long* n, double h, double* U,
                 double t0, double t_end, long max_steps, double* t_out, long* steps_out) {
  grid_t g = make_grid(dim, n);
  size_t bytes = sizeof(double) * (size_t)g.nf * (size_t)g.ncell;
  double* tmp = malloc(bytes);
  if (!tmp) return -2;
  double t = t0;
  long k = 0;
  int rc = 0;
  while (t < t_end && k < max_steps) {
    double dt = orc_dt(P, dim, n, h, U);
    int last = 0;
    if (dt >= t_end - t) { dt = t_end - t; last = 1; }
    rc = orc_step_heun(P, dim, n, h, dt, U, tmp);
    memcpy(U, tmp, bytes);
    t = last ? t_end : t + dt;
    ++k;
    if (rc != 0) break;
  }
  free(tmp);
  *t_out = t;
  *steps_out = k;
  return rc;
}
