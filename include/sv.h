/*
 * sv.h -- C ABI of libsv.so: a GB300 (sm_103a) solver for the MUSCL-Hancock
 * finite-volume step of the vibrationally excited gas model of
 * Khrapov & Khoperskov (2018), "Dynamics of unstable sound waves in a
 * non-equilibrium medium at the nonlinear stage".
 *
 * Problem (Sec. 2.1): eqs. 1-4 -- continuity, momentum, total energy E with
 * pump Q and heat sink I, vibrational energy E_nu relaxing to its equilibrium
 * with time tau; eq. 5 (E = p/(gamma-1) + rho|v|^2/2 + E_nu); eq. 6 (tau, Q, I
 * as power laws of rho and T about the equilibrium); eq. 7 (p = R rho T).
 * Units (Sec. 2.3, normalisation): rho0 = p0 = R = T0 = 1; tau0 is a free
 * parameter; Q0 = I0 = S / tau0 (S as defined under eq. 8, Q0 = I0 by the
 * energy balance of eq. 3 at equilibrium); the equilibrium vibrational energy
 * is E_nue = C_k rho T (C_k under eq. 8), relaxation term (rho C_k T - E_nu)/tau.
 *
 * Method (Sec. 2.3): MUSCL with a two-step predictor-corrector (read as
 * MUSCL-Hancock), piecewise-linear reconstruction of the conserved variables
 * with a TVD limiter (eq. 14, xi = 0), HLL interface fluxes (eq. 13), update
 * with the source Y at the half step (eq. 15), time step from eq. 16.
 *
 * Layout.  The state has nf = dim + 3 conserved fields, in this order:
 *   rho, rho*v_x [, rho*v_y [, rho*v_z]], E, E_nu.
 * Host buffers are always double, field-major structure-of-arrays:
 *   buf[f * ncell + idx], idx = i + n[0] * (j + n[1] * k), x fastest.
 * Periodic boundaries in every axis, except that a 1D grid may have solid
 * walls or free outflow at either end (two ghost cells per side, as needed
 * by the five-point stencil).  All axes share one cell size h = L[0] / n[0]
 * (the equal-step grid of Sec. 2.3).
 *
 * Errors.  Every call returns an int status, 0 on success, never throws.
 * Ownership.  Host buffers belong to the caller.  Device memory belongs to
 * the library unless the caller hands a device block to sv_init.
 * Threading.  One handle is used by one host thread at a time.  All device
 * work is enqueued on the CUDA stream given at sv_init; the read calls and
 * sv_status synchronise that stream.
 */
#ifndef SV_H
#define SV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes */
#define SV_OK          0
#define SV_EINVAL     -1   /* bad argument (null pointer, size, parameter) */
#define SV_ENOMEM     -2   /* device allocation failed / caller block too small */
#define SV_ECUDA      -3   /* a CUDA runtime call failed */
#define SV_ENONPHYS   -4   /* a cell reached rho <= 0, p <= 0 or a non-finite value */
#define SV_EDT        -5   /* the time step collapsed (dt <= 0 or non-finite) */
#define SV_EMAXSTEPS  -7   /* sv_run_to stopped at max_steps before t_end */
#define SV_ESIZE      -8   /* a size beyond the stated maximum of an entry point */
#define SV_ESTALL     -9   /* a grid-wide wait of the persistent step loop timed out */

/* ---- status flag bits (sv_status) */
#define SV_FLAG_NONPHYS  1u
#define SV_FLAG_DT       2u
#define SV_FLAG_MAXSTEPS 4u   /* batched runs: step budget exhausted before t_end */
#define SV_FLAG_STALL    8u   /* persistent step loop: a grid-wide wait gave up after ~2 s */

/* ---- limiters (the paper asks for "TVD limiters" without naming one) */
#define SV_MINMOD   0
#define SV_VANLEER  1
#define SV_MC       2

/* ---- arithmetic of the step kernels */
#define SV_FP32     0   /* float state and arithmetic */
#define SV_FP64     1   /* double state and arithmetic */
#define SV_FP32_P64 2   /* float state, pressure recovery of eq. 5 in double */
#define SV_FP32_PC  3   /* float state, pressure recovery of eq. 5 in compensated float:
                           the exact E - rho v^2/2 - E_nu of the float operands (two
                           error-free float sums), times gamma - 1, rounded once; the
                           same p as SV_FP32_P64 to within its last bit, at float speed */
#define SV_FP32_PS  4   /* MUSCL-Hancock (1D, 2D, 3D): float perturbations about the uniform
                           equilibrium (rho = p = 1, v = 0, E_nu = C_k + S) on the device, the
                           fluxes and the source Y written so that the equilibrium part cancels
                           exactly; host I/O stays full double states.  Float rounding then
                           scales with the perturbation instead of the O(1) background */

/* ---- time integration */
#define SV_HANCOCK  0   /* MUSCL-Hancock: half-step predictor + corrector (eqs. 14-15) */
#define SV_HEUN     1   /* Heun / SSP-RK2 (the predictor-corrector of eqs. 10-11) over the
                           same spatial operator; 1D periodic grids, SV_FP32 or SV_FP64 */

typedef struct {
  double gamma;                 /* adiabatic exponent (eq. 5) */
  double Ck;                    /* C_k = dE_nue/(R dT) (under eq. 8) */
  double S;                     /* degree of non-equilibrium (under eq. 8) */
  double tau0;                  /* equilibrium relaxation time; +inf: frozen
                                   limit (Q = I = 0, no relaxation) */
  double tau_rho, tau_T;        /* eq. 6 exponents of tau */
  double Q_rho, Q_T;            /* eq. 6 exponents of the pump Q */
  double I_rho, I_T;            /* eq. 6 exponents of the sink I */
  double cfl;                   /* factor on the eq. 16 bound, e.g. 0.4 */
  double c_tau;                 /* dt <= c_tau * min tau (explicit source), e.g. 0.5 */
  int limiter;                  /* SV_MINMOD, SV_VANLEER, SV_MC */
  int precision;                /* SV_FP32, SV_FP64, SV_FP32_P64, SV_FP32_PC, SV_FP32_PS */
  int method;                   /* SV_HANCOCK (0) or SV_HEUN */
} sv_params;

/* ---- boundary conditions (1D and 2D grids; 3D grids are periodic) */
#define SV_BC_PERIODIC 0
#define SV_BC_REFLECT  1   /* solid wall: mirrored ghost cells with the velocity reversed */
#define SV_BC_OUTFLOW  2   /* zero-gradient ghost cells (free outflow) */
#define SV_BC_DRIVEN   3   /* x = 0 only: ghost cells hold a prescribed wave (sv_set_drive),
                              the forced source of the paper's Sec. 3 runs */

typedef struct {
  int dim;                      /* 1, 2 or 3 */
  int64_t n[3];                 /* cells per axis (unused axes ignored) */
  double L[3];                  /* domain length per axis; L[a]/n[a] must agree */
  int bc[4];                    /* SV_BC_* at x = 0, x = L[0], y = 0, y = L[1].
                                   1D: bc[0], bc[1] (SV_BC_DRIVEN only at x = 0),
                                   bc[2], bc[3] ignored.  2D: periodic, wall or
                                   outflow per side (a non-periodic axis needs >= 2
                                   cells).  3D: all SV_BC_PERIODIC (0). */
} sv_grid;

typedef struct sv_solver sv_solver;

/* Bytes of device memory one solver needs for (params, grid): two state
   buffers, a double staging buffer for host I/O, the control block and the
   reduction scratch.  Returns SV_EINVAL on a bad grid or parameter. */
int sv_required_bytes(const sv_params* p, const sv_grid* g, size_t* bytes);

/* Create a solver.  `cuda_stream` is a cudaStream_t (NULL: legacy default
   stream).  `device_mem` is either NULL (the library allocates and later frees
   its memory) or a caller-owned device block of `device_bytes` >=
   sv_required_bytes(), 256-byte aligned, that must outlive the solver.  The
   state starts at the uniform equilibrium rho = p = 1, v = 0,
   E_nu = C_k + S, t = 0. */
int sv_init(const sv_params* p, const sv_grid* g, void* cuda_stream,
            void* device_mem, size_t device_bytes, sv_solver** out);

/* Upload a state (host double SoA, nf * ncell values) and set the time to t.
   Clears the status flags and computes the next dt (eq. 16 with the tau cap). */
int sv_write_state(sv_solver* s, const double* host_soa, double t);

/* Download the current state into host_soa (nf * ncell doubles) and its time. */
int sv_read_state(sv_solver* s, double* host_soa, double* t);

/* The same with float host buffers (nf * ncell floats, same layout): half the
   bytes over the host link.  For the float policies (SV_FP32, SV_FP32_P64,
   SV_FP32_PC) the device state is float, so a float buffer carries it
   exactly both ways; SV_FP32_PS forms U - U_ref in double from the float
   values and adds U_ref back in double before rounding to float; SV_FP64
   widens on upload and rounds to nearest on download.  Page-locked (mapped)
   buffers are read / written by the conversion kernels directly, others go
   through the solver's staging area.  Errors: SV_EINVAL (null argument),
   SV_ECUDA. */
int sv_write_state_f32(sv_solver* s, const float* host_soa, double t);
int sv_read_state_f32(sv_solver* s, float* host_soa, double* t);

/* The dt the next step will take: cfl * h / max_j max(2|v_j|, |v_j| + c_j)
   (eq. 16), capped by c_tau * min_j tau_j and by the pending t_end. */
int sv_dt_cfl(sv_solver* s, double* dt);

/* Advance exactly nsteps MUSCL-Hancock steps (eqs. 13-15), each with the dt
   computed on the device from the state it starts from.  Asynchronous on the
   solver's stream; errors of the steps show up in sv_status. */
int sv_step(sv_solver* s, int64_t nsteps);

/* How the steps of a solver are launched (sv_set_launch).
   SV_LAUNCH_PER_STEP: one kernel launch per step (two for SV_HEUN), replayed
     from a CUDA graph of 32 steps.
   SV_LAUNCH_PERSISTENT: 1D MUSCL-Hancock only -- one cooperative launch runs
     up to 65536 steps, its blocks resident throughout; the block that
     finishes a step last computes the next dt and releases the others (a
     grid-wide barrier).  Bitwise the same results as per-step launches.
     Every barrier wait gives up after about 2 s with SV_FLAG_STALL, which
     sv_run_to reports as SV_ESTALL.
   SV_LAUNCH_AUTO (default): persistent for 1D MUSCL-Hancock grids of at most
     one 64-cell chunk per two SMs (4864 cells on a GB300), where a step is
     short enough for the gap between launches to matter; per-step launches
     otherwise. */
#define SV_LAUNCH_AUTO       0
#define SV_LAUNCH_PER_STEP   1
#define SV_LAUNCH_PERSISTENT 2

/* Choose the launch mode.  SV_EINVAL for an unknown mode, or for
   SV_LAUNCH_PERSISTENT on a solver that cannot use it (not 1D MUSCL-Hancock,
   or no cooperative launch on the device).  Takes effect at the next step. */
int sv_set_launch(sv_solver* s, int mode);

/* The mode the next steps will use (SV_LAUNCH_PER_STEP or
   SV_LAUNCH_PERSISTENT; AUTO resolved). */
int sv_get_launch(sv_solver* s, int* mode);

/* Bound of the persistent loop's grid-barrier waits, for exercising its
   failure path: every wait gives up after `polls` polls of the barrier
   generation (or the ~2 s time limit, whichever comes first); 0 (the default)
   restores the limit of 2^24 polls.  A wait that gives up raises
   SV_FLAG_STALL and leaves the launch, so sv_step / sv_run_to end with
   SV_ESTALL and the state is undefined until the next sv_write_state (which
   also clears the flag).  Per-step launches do not wait and ignore it.
   Errors: SV_EINVAL (null solver, polls < 0). */
int sv_set_wait_limit(sv_solver* s, int polls);

/* ------------------------------------------------------------------------
 * Launch configurations and the autotuner.  A solver's per-step kernel comes
 * in a few launch configurations that compute bitwise the same states and
 * differ only in speed:
 *   1D float MUSCL-Hancock, >= 4096 cells: 512-cell block tiles at a register
 *     budget of 3 blocks/SM (default), 2 or 4 blocks/SM, 1024-cell tiles with
 *     two cell pairs per thread, or warps sliding over 64-cell chunks (the
 *     kernel of every other 1D solver, its only config);
 *   2D / 3D: planes per block along the marching axis, 64 / 128 / 256 / 512.
 * sv_autotune times each configuration on the solver's current state and
 * keeps the fastest; the state, time and status are restored afterwards.
 * ------------------------------------------------------------------------ */

/* Number of launch configurations of this solver (>= 1). */
int sv_num_configs(sv_solver* s, int* count);

/* Current configuration index and its description (desc may be NULL;
   truncated to cap bytes including the terminating zero). */
int sv_get_config(sv_solver* s, int* index, char* desc, size_t cap);

/* Description of configuration `index`. */
int sv_config_desc(sv_solver* s, int index, char* desc, size_t cap);

/* Make configuration `index` current (SV_EINVAL if out of range). */
int sv_set_config(sv_solver* s, int index);

/* Time every configuration over `steps` per-step launches (after 2 warm-up
   launches) with CUDA events on the solver's stream, restoring the state and
   control block after each trial, and make the fastest current.  *best
   (may be NULL) receives its index; us_per_step (may be NULL, else
   sv_num_configs entries) the microseconds per step of each configuration,
   +inf where the trial stopped early (t_end reached or a non-physical
   state).  steps < 0 times -steps launches one by one, each after a write
   of a 256 MiB scratch buffer (allocated for the call) that evicts the state
   from L2: the conditions of a measurement that flushes L2 between steps,
   where back-to-back steps find part of the state still in L2.
   Synchronous. */
int sv_autotune(sv_solver* s, int steps, int* best, double* us_per_step);

/* Advance until t_end, the last step clamped to land on t_end, or until
   max_steps steps.  Synchronous.  Returns SV_EMAXSTEPS if stopped early,
   SV_ENONPHYS / SV_EDT if the run failed (the state of the failing step is
   kept), SV_ESTALL if a persistent launch lost its barrier (the state is
   then undefined).  *steps_taken (may be NULL) receives the number of steps. */
int sv_run_to(sv_solver* s, double t_end, int64_t max_steps, int64_t* steps_taken);

/* Current time and number of steps taken since the last sv_write_state. */
int sv_time(sv_solver* s, double* t, int64_t* steps);

/* Sums over all cells of each conserved field (nf doubles), accumulated in
   double with compensated (Neumaier) summation.  Synchronous. */
int sv_conservation(sv_solver* s, double* sums);

/* Status flags (SV_FLAG_*) accumulated since the last sv_write_state.
   Synchronous. */
int sv_status(sv_solver* s, uint32_t* flags);

/* Device pointer of the current state buffer (nf * ncell elements of the
   solver's precision, field-major), valid until the next step.  For callers
   that keep data on the device.  Under SV_FP32_PS the buffer holds U - U_ref
   (U_ref: rho = 1, zero momenta, E = 1/(gamma-1) + C_k + S, E_nu = C_k + S). */
int sv_state_device(sv_solver* s, void** dev_ptr, int* elem_bytes);

/* Release the solver (waits for its stream). */
void sv_free(sv_solver* s);

/* ------------------------------------------------------------------------
 * Batched sweep: many independent 1D periodic runs of uneven sizes and
 * parameters (a stability map over S, tau0, the eq. 6 exponents and the
 * wavenumber), advanced to their own t_end by one persistent launch that is
 * replayed from a CUDA graph.  Every run uses the same per-cell arithmetic as
 * a single 1D solver with the same parameters, so a batched run and a looped
 * sv_run_to of that run give identical results.
 * ------------------------------------------------------------------------ */

typedef struct {
  int64_t n;            /* cells (1 .. 2^24) */
  double L;             /* domain length, h = L / n */
  double t_end;         /* end time of the run */
  double S, tau0;       /* degree of non-equilibrium, relaxation time (+inf: frozen) */
  double tau_rho, tau_T, Q_rho, Q_T, I_rho, I_T;   /* eq. 6 exponents */
  int mode;             /* index m of the logged Fourier amplitude of the velocity,
                           a_m(t) = (1/n) sum_j v_j exp(-i 2 pi m (j + 1/2) / n);
                           0: no log */
} sv_run;

typedef struct sv_batch sv_batch;

/* Device bytes for the batch: two state buffers (each run's 4 fields padded
   to a multiple of 32 cells), run records, order, queue and mode logs. */
int sv_batch_required_bytes(const sv_params* common, const sv_run* runs, int64_t nruns,
                            int log_cap, size_t* bytes);

/* Create a batch.  `common` supplies gamma, C_k, cfl, c_tau, limiter and
   precision (its S, tau0 and exponents are ignored: each run has its own).
   `host_states`: the runs' initial states, concatenated in run order, each
   a (4, n) field-major double block (rho, rho v, E, E_nu).  `log_cap`:
   samples of a_m kept per run (at t = 0, every t_end / (log_cap - 1) and at
   the end).  `max_steps_per_run` caps each run (SV_FLAG_MAXSTEPS).
   Stream and device memory as for sv_init. */
int sv_batch_init(const sv_params* common, const sv_run* runs, int64_t nruns,
                  const double* host_states, int log_cap, int64_t max_steps_per_run,
                  void* cuda_stream, void* device_mem, size_t device_bytes, sv_batch** out);

/* Re-upload initial states (same layout as sv_batch_init), times back to 0. */
int sv_batch_reset(sv_batch* b, const double* host_states);

/* Advance every run to its t_end: one persistent kernel launch, replayed from
   a CUDA graph.  Asynchronous on the batch's stream. */
int sv_batch_run(sv_batch* b);

/* Wait for the batch's stream. */
int sv_batch_sync(sv_batch* b);

/* State (4 * n doubles, may be NULL), time, steps and flags of one run.
   Synchronous. */
int sv_batch_read(sv_batch* b, int64_t run, double* host_soa, double* t, int64_t* steps,
                  uint32_t* flags);

/* Up to `cap` logged samples (t, Re a_m, Im a_m) of one run; *count gets the
   number written.  Synchronous. */
int sv_batch_mode_log(sv_batch* b, int64_t run, double* t, double* re, double* im, int64_t cap,
                      int64_t* count);

void sv_batch_free(sv_batch* b);

/* Launch configurations of a batch: the block size per run, 256 (default) or
   128 threads.  Same results, different speed: smaller blocks keep more runs
   in flight and idle fewer warps on small runs.  Set before sv_batch_run. */
int sv_batch_num_configs(sv_batch* b, int* count);
int sv_batch_set_config(sv_batch* b, int index);
int sv_batch_get_config(sv_batch* b, int* index, char* desc, size_t cap);

/* ------------------------------------------------------------------------
 * Allocation-free 1D step.  The paper has no counterpart: this is a service
 * of the library for callers that cannot allocate device memory -- processes
 * whose device memory is a fixed pool handed out at start-up and that forbid
 * allocation afterwards, and hosts that must not allocate on their stepping
 * path (a device allocation can synchronise the device and takes unbounded
 * time).  Such a caller owns the two state buffers; the small
 * control block the fused kernel needs (time, dt, the eq.-16 reduction keys,
 * the block-completion ticket) lives in a file-scope static device array of
 * SV_NOALLOC_SCRATCH_BYTES bytes that every GPU loading libsv.so holds until
 * the process exits.
 * ------------------------------------------------------------------------ */
#define SV_NOALLOC_SCRATCH_BYTES 256
#define SV_NOALLOC_MAX_CELLS ((1 << 29) - 1)   /* largest grid (32-bit offsets) */

/* One MUSCL-Hancock step of a 1D periodic grid of n cells (length L) from the
   caller's device buffer U_in to the caller's device buffer U_out (each
   4 * n elements of float for SV_FP32 / SV_FP32_P64 / SV_FP32_PC or double for SV_FP64,
   field-major rho, rho v, E, E_nu; buffers sharing any byte return
   SV_EINVAL), with dt from eq. 16 (capped by c_tau * min tau) on U_in.  The
   same dt and, bit for bit, the same state as sv_step on a solver holding
   U_in: it runs the sliding-warp kernel, whose per-cell arithmetic every 1D
   kernel of the solver shares.  Allocates nothing and calls no allocating
   routine.
   dt_used / flags (host pointers, each may be NULL) receive the dt taken and
   the SV_FLAG_* bits of the step; giving either makes the call wait for the
   stream, otherwise it is asynchronous on cuda_stream.
   The first call on a device (and the first with each precision, limiter
   and source variant) looks up the device address of the static array
   (cudaGetSymbolAddress, with that device current) and the step kernel's
   launch grid; later calls reuse them.  Every call resets the control block it
   finds, since the array keeps the previous call's contents; calls that
   overlap on the GPU (other streams, other host threads) share that one
   array and race.  n beyond SV_NOALLOC_MAX_CELLS returns SV_ESIZE. */
int sv_step1d_noalloc(const sv_params* p, int64_t n, double L, const void* U_in, void* U_out,
                      double* dt_used, uint32_t* flags, void* cuda_stream);

/* Medium map and driven cells of a 2D solver (the paper's two-dimensional
   active-sector problem, Sec. 3: the active medium fills a sector, a source
   drives acoustic waves, walls and free outflow bound the domain).  All
   arrays have n[1] entries (one per row j = 0..ny-1) and are copied.
     active_lo / active_hi: row j is the active medium of the solver's
       parameters (relaxation, pump and sink) in the cells
       active_lo[j] <= i < active_hi[j] and frozen (no relaxation, pump or sink)
       elsewhere; NULL: active everywhere.  The rest state rho = p = 1, v = 0,
       E_nu = C_k + S is steady in both.  A ghost cell takes the medium of the
       cell whose state it holds.
     driven_lo / driven_hi: cells driven_lo[j] <= i < driven_hi[j] hold, at
       every new time level t, the pulsating source rho = 1 + amp sin(omega t),
       v = 0, p = 1 + gamma amp sin(omega t), E_nu = rho (C_k + S); NULL: none.
   0 <= lo <= hi <= n[0] in every row. */
typedef struct {
  const int32_t* active_lo;
  const int32_t* active_hi;
  const int32_t* driven_lo;
  const int32_t* driven_hi;
  double omega, amp;
} sv_medium2d;

/* Install (or, with every table NULL, remove) the medium map and driven
   cells of a 2D solver; the library keeps device copies (4 n[1] int32) until
   sv_free.  SV_EINVAL if the solver is not 2D or a table is out of range.
   Synchronous. */
int sv_set_medium2d(sv_solver* s, const sv_medium2d* m);

/* Prescribed wave of an SV_BC_DRIVEN boundary: the ghost cell centred at x < 0
   holds U(x, t) = base + Re(amp e^{i (k x - omega t)}), k = k_re + i k_im,
   evaluated at the start time of each step (conserved variables rho, rho v,
   E, E_nu). */
typedef struct {
  double omega, k_re, k_im;
  double base[4], amp_re[4], amp_im[4];
} sv_drive;

/* Set the wave of a 1D solver whose grid has bc[0] = SV_BC_DRIVEN (until it
   is set the ghost cells hold the uniform equilibrium).  SV_EINVAL for other
   grids. */
int sv_set_drive(sv_solver* s, const sv_drive* d);

/* Human-readable name of a status code. */
const char* sv_strerror(int code);

/* ------------------------------------------------------------------------
 * Measurement utility (not part of the paper's method).  The FP64 step
 * kernels are bound by the GPU's double-precision pipe rather than by HBM;
 * this measures that pipe's throughput on the current device, the
 * denominator of their roofline: independent DFMA chains (8 per thread, 4
 * blocks of 256 threads per SM, an exact count of FMAs at 2 flops each), the
 * best of three launches timed with CUDA events on cuda_stream, after one
 * warm-up launch.  Writes TFLOP/s to *tflops (host pointer); synchronous.
 * Errors: SV_EINVAL (null tflops), SV_ECUDA.
 * ------------------------------------------------------------------------ */
int sv_measure_fp64_peak(void* cuda_stream, double* tflops);

#ifdef __cplusplus
}
#endif
#endif
