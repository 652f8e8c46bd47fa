// sv_model.cuh -- device-side physics of the vibrationally excited gas model
// (Khrapov & Khoperskov 2018) used by every step kernel.
//
//   eq. 5   pressure recovery      p = (gamma-1) (E - rho|v|^2/2 - E_nu)
//   eq. 7   temperature            T = p / rho              (R = 1)
//   eq. 6   closures               tau = tau0 rho^tau_rho T^tau_T, Q, I alike
//   MUSCL Y (Sec. 2.3, f = 0)      Y_E    = rho (Q - I)
//                                  Y_E_nu = (rho C_k T - E_nu) / tau + rho Q
//   F/G of eq. 15                  (rho v_a, rho v v_a + p e_a, v_a (E + p), v_a E_nu)
//   eq. 13                         HLL flux with Davis speed estimates
//
// Everything is templated on the arithmetic type R (float or double).  The
// float instantiation uses the SFU approximations (rcp, rsqrt, lg2, ex2); the
// double instantiation uses IEEE division, sqrt and pow.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <type_traits>

namespace sv {

// Kernel-side parameter block, passed by value.
struct KParams {
  double gamma, g1, Ck, Q0, tau0, inv_tau0;
  double tau_rho, tau_T, Q_rho, Q_T, I_rho, I_T;
  double h, cfl, c_tau;
  int limiter;   // 0 minmod, 1 van Leer, 2 MC
  int frozen;    // 1: no source at all (Q = I = 0, 1/tau = 0)
  int qi_zero;   // 1: all Q and I exponents are zero (Q = I = Q0)
  int bc_lo, bc_hi;   // boundary conditions at x = 0 / x = Lx (BC_*)
  int bc_ylo, bc_yhi; // 2D: boundary conditions at y = 0 / y = Ly
  int stall_polls;     // persistent loop: polls before a grid-barrier wait gives up (0: default)
  // driven boundary wave: U = base + Re(amp e^{i (k x - omega t)})
  double drv_omega, drv_kre, drv_kim, drv_base[4], drv_are[4], drv_aim[4];
  // 2D medium map (device arrays of ny entries, null when unused): row j is
  // active (relaxation, pump, sink) for act_lo[j] <= i < act_hi[j] and frozen
  // elsewhere; cells drv_lo[j] <= i < drv_hi[j] hold the pulsating source
  // rho = 1 + pul_amp sin(pul_omega t), v = 0, p = 1 + gamma (rho - 1),
  // E_nu = rho (C_k + S) at every new time level
  const int* act_lo;
  const int* act_hi;
  const int* pul_lo;
  const int* pul_hi;
  double pul_omega, pul_amp, pul_ev;   // pul_ev = C_k + S
  // float copies for the float kernels (kparams_finish): the twelve values
  // above, then log2(1/tau0) (0 in the frozen limit), -tau_rho, -tau_T, and
  // the low part of g1 (g1 - (float)g1, for the compensated pressure)
  float f[16];
  // float constants of the dt rule of the float solvers: cfl h, 1/h, 1/(2h),
  // c_tau tau0 (0 in the frozen limit)
  float fdt[4];
  // degree of non-equilibrium S, and the uniform equilibrium rho = p = T = 1,
  // v = 0, E_nu = C_k + S that the perturbation layout (SV_FP32_PS) subtracts:
  // ref = (rho, rho v, E, E_nu); fps = (E + p, E_nu, S) of it in float
  double S;
  double ref[4];
  float fps[4];
};

// Fill the float copies once on the host, so float kernels convert nothing.
inline void kparams_finish(KParams& k) {
  const double v[12] = {k.gamma, k.g1, k.Ck, k.Q0, k.tau0, k.inv_tau0,
                        k.tau_rho, k.tau_T, k.Q_rho, k.Q_T, k.I_rho, k.I_T};
  for (int i = 0; i < 12; ++i) k.f[i] = (float)v[i];
  k.f[12] = k.inv_tau0 > 0.0 ? (float)log2(k.inv_tau0) : 0.0f;
  k.f[13] = (float)(-k.tau_rho);
  k.f[14] = (float)(-k.tau_T);
  k.f[15] = (float)(k.g1 - (double)k.f[1]);
  k.fdt[0] = (float)(k.cfl * k.h);
  k.fdt[1] = (float)(1.0 / k.h);
  k.fdt[2] = (float)(0.5 / k.h);
  k.fdt[3] = k.frozen ? 0.0f : (float)(k.c_tau * k.tau0);
  const double ev0 = k.Ck + k.S;
  k.ref[0] = 1.0;
  k.ref[1] = 0.0;
  k.ref[2] = 1.0 / k.g1 + ev0;
  k.ref[3] = ev0;
  k.fps[0] = (float)(k.ref[2] + 1.0);
  k.fps[1] = (float)ev0;
  k.fps[2] = (float)k.S;
  k.fps[3] = 0.0f;
}

// Entry f of the perturbation layout's reference state U_ref for nf = DIM + 3
// fields (ref holds its 1D form: rho, rho v, E, E_nu).
__host__ __device__ __forceinline__ double ref_field(const double (&ref)[4], int f, int nf) {
  if (f == 0) return ref[0];
  if (f == nf - 2) return ref[2];
  if (f == nf - 1) return ref[3];
  return 0.0;
}

// Programmatic dependent launch: a step kernel launched with the programmatic
// stream-serialization attribute (the graph-replayed steps of a solver) may
// start while the previous step's grid is still finishing.  pdl_wait blocks
// until that grid has completed and its memory is visible -- every step
// kernel calls it before reading the control block or the state; launched
// without the attribute it returns at once.  pdl_trigger lets the next grid
// launch once every block of this one has called it or exited (its blocks
// then wait in pdl_wait for this grid to complete).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Device control block: time, step size and the reductions of one solver.
struct Ctl {
  double t;            // current time
  double dt;           // dt of the next step (0: stopped / reached t_end)
  double dtdx, dt_2h, dt_2;   // dt / h, dt / (2h), dt / 2 of the next step
  float fdt, fdtdx, fdt_2h, fdt_2;   // the same rounded to float
  double dt_cfl;       // unclamped eq.-16 dt of the current state
  double t_end;        // target time of the running sv_run_to (+inf otherwise)
  int64_t nsteps;      // steps taken since the last state upload
  uint32_t cur;        // which of the two state buffers is current
  uint32_t last;       // 1: the next step lands exactly on t_end
  uint32_t flags;      // SV_FLAG_* bits
  uint32_t ticket;     // blocks finished in the running launch
  uint64_t smax_key;   // order-preserving key of max signal speed
  uint64_t tau_key;    // order-preserving key of the tau bound (see finalize)
  uint32_t gen;        // grid-barrier generation of the persistent step loop
  uint32_t pad32;
  double pad[3];
};

// 1D boundary conditions (the values of SV_BC_* in sv.h).
constexpr int BC_PERIODIC = 0, BC_REFLECT = 1, BC_OUTFLOW = 2, BC_DRIVEN = 3;

constexpr uint32_t FLAG_NONPHYS = 1u;
constexpr uint32_t FLAG_DT = 2u;
constexpr uint32_t FLAG_STALL = 8u;   // a grid-barrier wait ran out (sv.h SV_FLAG_STALL)

// ---------------------------------------------------------------- arithmetic

template <typename R> struct Ar;

// The float kernels use the SFU approximations directly (PTX rcp/rsqrt/lg2/ex2
// .approx.ftz, each within a few ulp; subnormal inputs are flushed, which a
// physical state never produces).
template <> struct Ar<float> {
  static __device__ __forceinline__ float rcp(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
  }
  static __device__ __forceinline__ float rsqrt(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
  }
  static __device__ __forceinline__ float sqrt_pos(float x) { return x * rsqrt(x); }
  static __device__ __forceinline__ float lg2(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
  }
  static __device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
  }
};

// The double kernels' reciprocal: the SFU's approximate 1/x refined by two
// Newton-Raphson steps y <- y + y (1 - x y) (each doubling the correct bits;
// within an ulp or two of 1/x for the positive normal densities and speed sums
// it is used on): four FMAs instead of an IEEE division on GB300's narrow FP64
// pipe.  A non-positive density still raises SV_FLAG_NONPHYS through the
// physicality checks, which test rho itself.
template <> struct Ar<double> {
  static __device__ __forceinline__ double rcp(double x) {
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    y = fma(y, fma(-x, y, 1.0), y);
    return fma(y, fma(-x, y, 1.0), y);
  }
  static __device__ __forceinline__ double sqrt_pos(double x) { return sqrt(x); }
};

// Parameters converted once to the kernel's arithmetic type.
template <typename R> struct P;

template <> struct P<double> {
  double gamma, g1, Ck, Q0, inv_tau0, tau0;
  double tau_rho, tau_T, Q_rho, Q_T, I_rho, I_T;
  int limiter, frozen, qi_zero, bc_lo, bc_hi;
  // eq. 6 exponents that are multiples of 1/2 (the paper's tau_rho = -1,
  // tau_T = -1.5): twice each exponent (tau_rho, tau_T, Q_rho, Q_T, I_rho,
  // I_T), and whether the tau pair / the Q and I exponents all qualify
  // (|exponent| <= 4), so that the power laws are products and square roots
  int hk[6];
  bool half_tau, half_qi;
  __device__ __forceinline__ explicit P(const KParams& k)
      : gamma(k.gamma), g1(k.g1), Ck(k.Ck), Q0(k.Q0), inv_tau0(k.inv_tau0), tau0(k.tau0),
        tau_rho(k.tau_rho), tau_T(k.tau_T), Q_rho(k.Q_rho), Q_T(k.Q_T), I_rho(k.I_rho),
        I_T(k.I_T), limiter(k.limiter), frozen(k.frozen), qi_zero(k.qi_zero), bc_lo(k.bc_lo),
        bc_hi(k.bc_hi) {
    const double e[6] = {tau_rho, tau_T, Q_rho, Q_T, I_rho, I_T};
    bool ok[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const double t = 2.0 * e[i], r = rint(t);
      ok[i] = t == r && fabs(r) <= 8.0;
      hk[i] = ok[i] ? (int)r : 0;
    }
    half_tau = ok[0] && ok[1];
    half_qi = ok[2] && ok[3] && ok[4] && ok[5];
  }
};

// rho^(kr/2) T^(kT/2) for integers |kr|, |kT| <= 8, given sr = sqrt(rho) and
// sT = sqrt(T) where kr / kT is odd: whole powers by repeated multiplication,
// the negative ones gathered into one reciprocal.  Each product rounds once,
// so the result stays within a few ulp of pow's.
__device__ __forceinline__ double half_powers(double rho, double sr, int kr, double T, double sT,
                                              int kT);

template <> struct P<float> {
  float gamma, g1, Ck, Q0, inv_tau0, tau0;
  float tau_rho, tau_T, Q_rho, Q_T, I_rho, I_T;
  float l2_inv_tau0, ntau_rho, ntau_T;   // log2(1/tau0), -tau_rho, -tau_T
  float g1lo;                            // g1 - (float)g1
  float h0, ev0, S;                      // perturbation layout: E + p, E_nu, S of the reference
  int limiter, frozen, qi_zero, bc_lo, bc_hi;
  __device__ __forceinline__ explicit P(const KParams& k)
      : gamma(k.f[0]), g1(k.f[1]), Ck(k.f[2]), Q0(k.f[3]), inv_tau0(k.f[5]), tau0(k.f[4]),
        tau_rho(k.f[6]), tau_T(k.f[7]), Q_rho(k.f[8]), Q_T(k.f[9]), I_rho(k.f[10]),
        I_T(k.f[11]), l2_inv_tau0(k.f[12]), ntau_rho(k.f[13]), ntau_T(k.f[14]), g1lo(k.f[15]),
        h0(k.fps[0]), ev0(k.fps[1]), S(k.fps[2]),
        limiter(k.limiter), frozen(k.frozen), qi_zero(k.qi_zero), bc_lo(k.bc_lo),
        bc_hi(k.bc_hi) {}
};

// The control-block fields a step kernel reads: written by the previous
// launch (or, in the persistent loop, by another block), so read with volatile
// loads -- by one thread per block, which publishes them in shared memory.
// (Every thread reading them itself sends tens of thousands of requests per
// launch to the one L2 line of the control block.)
struct StepCtl {
  double t, dt, dtdx, dt_2h, dt_2;
  float fdt, fdtdx, fdt_2h, fdt_2;
  uint32_t cur, gen;
};

// Must be called by every thread of the block; ends with a block barrier.
__device__ __forceinline__ StepCtl block_step_ctl(const Ctl* ctl) {
  __shared__ StepCtl s;
  if (threadIdx.x == 0) {
    const volatile Ctl* c = (const volatile Ctl*)ctl;
    s.t = c->t;
    s.dt = c->dt;
    s.dtdx = c->dtdx;
    s.dt_2h = c->dt_2h;
    s.dt_2 = c->dt_2;
    s.fdt = c->fdt;
    s.fdtdx = c->fdtdx;
    s.fdt_2h = c->fdt_2h;
    s.fdt_2 = c->fdt_2;
    s.cur = c->cur;
    s.gen = c->gen;
  }
  __syncthreads();
  return s;
}

// The dt-derived factors of the next step in the kernel's arithmetic type.
// Float solvers form them in float from the float dt (a product by the
// stored 1/h and 1/(2h): no FP64 divide on the step's serial path).
template <typename R> struct StepDt;
template <> struct StepDt<double> {
  double dt, dtdx, dt_2h, dt_2;
  __device__ __forceinline__ explicit StepDt(const StepCtl& c)
      : dt(c.dt), dtdx(c.dtdx), dt_2h(c.dt_2h), dt_2(c.dt_2) {}
  __device__ __forceinline__ StepDt(double d, const KParams& kp)
      : dt(d), dtdx(d / kp.h), dt_2h(d / (2.0 * kp.h)), dt_2(0.5 * d) {}
};
template <> struct StepDt<float> {
  float dt, dtdx, dt_2h, dt_2;
  __device__ __forceinline__ explicit StepDt(const StepCtl& c)
      : dt(c.fdt), dtdx(c.fdtdx), dt_2h(c.fdt_2h), dt_2(c.fdt_2) {}
  __device__ __forceinline__ StepDt(double d, const KParams& kp)
      : dt((float)d), dtdx(dt * kp.fdt[1]), dt_2h(dt * kp.fdt[2]), dt_2(0.5f * dt) {}
};

// ---------------------------------------------------------------- eq. 5

// Pressure policies of the float kernels: PP = 0 all-float, PP = 1 the
// subtraction of eq. 5 carried out in double, PP = 2 the same subtraction in
// compensated float: E - kin2/2 - E_nu of the float operands is formed exactly
// as an unevaluated sum t + e by two of Dekker's fast two-sums (exact when
// |E| >= E_nu and E - E_nu >= kin2/2, i.e. for every state with p >= 0), then
// multiplied by g1 held as two floats (g1 + g1lo) with one final rounding.  The
// result is the double policy's p to within its last bit, at the cost of eleven
// float operations (three for PP = 0) instead of a trip through GB300's narrow
// FP64 pipe.
template <typename R, int PP>
__device__ __forceinline__ R pressure(const P<R>& k, R kin2, R E, R Ev) {
  // kin2 = rho |v|^2 (twice the kinetic energy density)
  if constexpr (PP == 1) {
    return (R)((double)k.g1 * ((double)E - 0.5 * (double)kin2 - (double)Ev));
  } else if constexpr (PP == 2) {
    static_assert(std::is_same<R, float>::value, "compensated pressure is a float policy");
    const float h = 0.5f * kin2;
    const float s = __fsub_rn(E, Ev);
    const float e1 = __fsub_rn(__fsub_rn(E, s), Ev);
    const float t = __fsub_rn(s, h);
    const float e2 = __fsub_rn(__fsub_rn(s, t), h);
    return __fmaf_rn(k.g1, t, __fmaf_rn(k.g1lo, t, __fmul_rn(k.g1, __fadd_rn(e1, e2))));
  } else if constexpr (std::is_same<R, float>::value) {
    // The cancelling pair first: E - E_nu is exact whenever E_nu >= E / 2
    // (Sterbenz), which is where the cancellation bites, so p stays within
    // ~1.4 ulp of the exact value of the float operands however large E_nu
    // is (the order E - kin2/2 - E_nu loses log2(E / p) bits there).
    return k.g1 * fmaf(kin2, -0.5f, E - Ev);
  } else {
    return k.g1 * (E - (R)0.5 * kin2 - Ev);
  }
}

// ---------------------------------------------------------------- limiter

// minmod(a, b): the argument of smaller magnitude when a and b have the same
// sign, else 0.
// float: min.xorsign.abs gives min(|a|, |b|) with the sign of a xor b, i.e.
// negative exactly when the signs differ; max with 0 clears that case and the
// sign of a is put back (three ALU instructions).
__device__ __forceinline__ float minmod(float a, float b) {
  float m;
  asm("min.xorsign.abs.f32 %0, %1, %2;" : "=f"(m) : "f"(a), "f"(b));
  return copysignf(fmaxf(m, 0.0f), a);
}
// double: the same decision on the bit patterns (for doubles of one sign the
// integer order of the magnitudes' bits is their order), on the integer pipe
// rather than GB300's narrow FP64 pipe.  A zero argument gives a zero of a's
// sign.
__device__ __forceinline__ double minmod(double a, double b) {
  const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  if ((ia ^ ib) < 0) return 0.0;
  const long long ma = ia & 0x7fffffffffffffffll, mb = ib & 0x7fffffffffffffffll;
  return __longlong_as_double((ma < mb ? ma : mb) | (ia & (long long)0x8000000000000000ull));
}

// Whether four values (densities and pressures of two states) are all > 0.
// float: the minimum against 0.  double: the signed high words of the bit
// patterns are all > 0 (integer pipe; a positive double below ~1e-313 counts
// as not positive, far below any density or pressure of a state).
__device__ __forceinline__ bool all_positive(float a, float b, float c, float d) {
  return fminf(fminf(a, b), fminf(c, d)) > 0.0f;
}
__device__ __forceinline__ bool all_positive(double a, double b, double c, double d) {
  const int ha = __double2hiint(a), hb = __double2hiint(b);
  const int hc = __double2hiint(c), hd = __double2hiint(d);
  return min(min(ha, hb), min(hc, hd)) > 0;
}
__device__ __forceinline__ bool both_positive(float a, float b) { return (a > 0.0f) && (b > 0.0f); }
__device__ __forceinline__ bool both_positive(double a, double b) {
  return min(__double2hiint(a), __double2hiint(b)) > 0;
}

// TVD slope limiters on the two one-sided differences a, b (eq. 14 asks for
// "limiter functions" without naming one): LIM 0 minmod, 1 van Leer, 2 MC.
template <int LIM, typename R>
__device__ __forceinline__ R limit(R a, R b) {
  if constexpr (LIM == 0) {
    return minmod(a, b);
  } else {
    const R ab = a * b;
    R m;
    if (LIM == 1) {
      if constexpr (std::is_same<R, float>::value) m = __fdividef(2.0f * ab, fabsf(a + b));
      else m = (R)2 * ab / fabs(a + b);
    } else {
      m = fmin(fabs(a), fabs(b));
      m = fmin((R)2 * m, (R)0.5 * fabs(a + b));
    }
    return ab > (R)0 ? copysign(m, a) : (R)0;
  }
}

// ---------------------------------------------------------------- source Y

// Components E and E_nu of Y (the others vanish with f = 0).
// SRC 0: frozen limit (no source); 1: Q and I exponents all zero (Q = I = Q0,
// so rho (Q - I) = 0); 2: general closures of eq. 6.
template <typename R, int SRC> struct Src;

template <int SRC> struct Src<float, SRC> {
  static __device__ __forceinline__ void eval(const P<float>& k, float rho, float T, float Ev,
                                              float& yE, float& yEv) {
    if (SRC == 0) {
      yE = yEv = 0.0f;
      return;
    }
    // 1/tau = (1/tau0) rho^-tau_rho T^-tau_T = 2^(log2(1/tau0) - tau_rho lg rho - tau_T lg T)
    const float lr = Ar<float>::lg2(rho), lT = Ar<float>::lg2(T);
    const float inv_tau = Ar<float>::ex2(fmaf(k.ntau_rho, lr, fmaf(k.ntau_T, lT, k.l2_inv_tau0)));
    float Q = k.Q0;
    yE = 0.0f;
    if (SRC == 2) {
      Q = k.Q0 * Ar<float>::ex2(fmaf(k.Q_rho, lr, k.Q_T * lT));
      const float I = k.Q0 * Ar<float>::ex2(fmaf(k.I_rho, lr, k.I_T * lT));
      yE = rho * (Q - I);
    }
    yEv = fmaf(rho * k.Ck, T, -Ev) * inv_tau + rho * Q;
  }
};

__device__ __forceinline__ double half_powers(double rho, double sr, int kr, double T, double sT,
                                              int kT) {
  double num = 1.0, den = 1.0;
  const int ar = kr < 0 ? -kr : kr, aT = kT < 0 ? -kT : kT;
  double pr = (ar & 1) ? sr : 1.0, pT = (aT & 1) ? sT : 1.0;
  for (int i = 0; i < (ar >> 1); ++i) pr *= rho;
  for (int i = 0; i < (aT >> 1); ++i) pT *= T;
  if (kr < 0) den *= pr; else num *= pr;
  if (kT < 0) den *= pT; else num *= pT;
  return (kr < 0 || kT < 0) ? num * Ar<double>::rcp(den) : num;
}

template <int SRC> struct Src<double, SRC> {
  static __device__ __forceinline__ void eval(const P<double>& k, double rho, double T, double Ev,
                                              double& yE, double& yEv) {
    if (SRC == 0) {
      yE = yEv = 0.0;
      return;
    }
    double inv_tau, Q = k.Q0, I = k.Q0;
    if (k.half_tau && (SRC == 1 || k.half_qi)) {
      // exponents that are multiples of 1/2: products and at most one square
      // root per variable, in place of logarithms and exponentials on GB300's
      // narrow FP64 pipe
      const bool odd_r = ((k.hk[0] | (SRC == 2 ? k.hk[2] | k.hk[4] : 0)) & 1) != 0;
      const bool odd_T = ((k.hk[1] | (SRC == 2 ? k.hk[3] | k.hk[5] : 0)) & 1) != 0;
      const double sr = odd_r ? sqrt(rho) : 1.0, sT = odd_T ? sqrt(T) : 1.0;
      inv_tau = k.inv_tau0 * half_powers(rho, sr, -k.hk[0], T, sT, -k.hk[1]);
      if (SRC == 2) {
        Q = k.Q0 * half_powers(rho, sr, k.hk[2], T, sT, k.hk[3]);
        I = k.Q0 * half_powers(rho, sr, k.hk[4], T, sT, k.hk[5]);
      }
    } else {
      // the power laws of eq. 6 as exp of a linear form in ln rho, ln T: two
      // logarithms per state instead of two pow per closure (GB300's FP64 rate)
      const double lr = log(rho), lT = log(T);
      inv_tau = exp(-fma(k.tau_rho, lr, k.tau_T * lT)) * k.inv_tau0;
      if (SRC == 2) {
        Q = k.Q0 * exp(fma(k.Q_rho, lr, k.Q_T * lT));
        I = k.Q0 * exp(fma(k.I_rho, lr, k.I_T * lT));
      }
    }
    yE = rho * (Q - I);
    yEv = (rho * k.Ck * T - Ev) * inv_tau + rho * Q;
  }
};

// Order-preserving unsigned keys so that atomicMax/atomicMin order floats.
__device__ __forceinline__ uint64_t key_of(double x) {
  uint64_t b = (uint64_t)__double_as_longlong(x);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__host__ __device__ __forceinline__ double key_to_double(uint64_t k) {
  uint64_t b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double d;
  memcpy(&d, &b, sizeof d);
  return d;
#endif
}

}  // namespace sv
