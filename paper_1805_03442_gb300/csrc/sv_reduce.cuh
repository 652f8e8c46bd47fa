// sv_reduce.cuh -- the time-step reduction shared by the step kernels.
//
// Every step kernel ends by folding, over the cells it wrote, the two
// quantities that bound the next time step:
//   s_j  = max(2|v_j|, |v_j| + c_j)           (eq. 16, c the frozen sound speed)
//   a tau bound per cell (see TauKey below)    (explicit source: dt <= c_tau tau)
// Warp shuffles, then shared memory, then one atomicMax per block into the
// solver's control block.  The last block to finish (ticket counter, with a
// fence before the ticket) turns the maxima into the next dt, advances t and
// flips the current state buffer: the host never has to read anything to keep
// stepping, so K steps can be replayed from a CUDA graph.
#pragma once

#include "sv_model.cuh"

namespace sv {

// The tau bound is folded as a maximum:
//   float kernels:  a_j = -(tau_rho log2 rho + tau_T log2 T), tau_j = tau0 2^-a_j
//   double kernels: a_j = -tau_j (tau_j from pow, as in the closure of eq. 6)
template <typename R> struct TauKey;
template <> struct TauKey<float> {
  static __device__ __forceinline__ float of(const P<float>& k, float rho, float T) {
    return -fmaf(k.tau_rho, Ar<float>::lg2(rho), k.tau_T * Ar<float>::lg2(T));
  }
};
template <> struct TauKey<double> {
  static __device__ __forceinline__ double of(const P<double>& k, double rho, double T) {
    if (k.half_tau) {
      const double sr = (k.hk[0] & 1) ? sqrt(rho) : 1.0, sT = (k.hk[1] & 1) ? sqrt(T) : 1.0;
      return -(k.tau0 * half_powers(rho, sr, k.hk[0], T, sT, k.hk[1]));
    }
    return -(k.tau0 * exp(fma(k.tau_rho, log(rho), k.tau_T * log(T))));
  }
};

// |v| from v.v for the eq. 16 bound of 2D / 3D states.  In float,
// x * rsqrt(x) of a subnormal v.v (the far tail of a wave still spreading into
// gas at rest) flushes the rsqrt argument to zero and gives +inf; a speed
// below 1e-19 cannot change max(2|v|, |v| + c) in float, so it counts as 0.
template <typename R>
__device__ __forceinline__ R speed_of(R v2) {
  if (std::is_same<R, float>::value) return v2 >= (R)1.17549435e-38 ? Ar<R>::sqrt_pos(v2) : (R)0;
  return v2 > (R)0 ? Ar<R>::sqrt_pos(v2) : (R)0;
}

// Signal speed, tau key and physicality of one updated state (dim-generic),
// folded into per-thread maxima of the kernel's own type.
// `kin2` = rho |v|^2, `vmag` = |v|.  SRC 0 (frozen) has no tau bound.
template <typename R, int PP, int SRC>
__device__ __forceinline__ void cfl_cell(const P<R>& k, R rho, R kin2, R vmag, R E, R Ev,
                                         R& smax, R& akey, uint32_t& flags) {
  const R p = pressure<R, PP>(k, kin2, E, Ev);
  const R ir = Ar<R>::rcp(rho);
  if (!both_positive(rho, p)) {
    flags |= FLAG_NONPHYS;
    return;
  }
  const R c = Ar<R>::sqrt_pos(k.gamma * p * ir);
  smax = fmax(smax, fmax((R)2 * vmag, vmag + c));
  if (SRC != 0) akey = fmax(akey, TauKey<R>::of(k, rho, p * ir));
}

// eq. 16 times cfl from the maximal signal speed, capped by c_tau * min tau;
// raises FLAG_DT if the result is not a positive finite number.  One thread
// per step evaluates it on the step's serial path, in the solver's own type:
// float solvers stay off the narrow FP64 pipe, whose divide and exp2 take
// microseconds of latency on one thread.
__device__ __forceinline__ double dt_from_maxima(const KParams& kp, double smax, double akey,
                                                 uint32_t& flags) {
  double dt = kp.cfl * kp.h / smax;
  if (!kp.frozen) {
    const double cap = kp.c_tau * -akey;          // akey = -min tau
    if (cap < dt) dt = cap;
  }
  if (!(dt > 0.0) || !isfinite(dt)) flags |= FLAG_DT;
  return dt;
}
__device__ __forceinline__ double dt_from_maxima(const KParams& kp, float smax, float akey,
                                                 uint32_t& flags) {
  float dt = __fdiv_rn(kp.fdt[0], smax);
  if (!kp.frozen) {
    const float cap = kp.fdt[3] * Ar<float>::ex2(-akey);   // c_tau tau0 2^-a = c_tau min tau
    if (cap < dt) dt = cap;
  }
  if (!(dt > 0.0f) || !isfinite(dt)) flags |= FLAG_DT;
  return (double)dt;
}

// Store the next step's dt and its derived factors (StepDt of the solver's
// type; the other type's copies are conversions of those).
template <typename R>
__device__ __forceinline__ void set_step_dt(Ctl* ctl, double dt, const KParams& kp) {
  const StepDt<R> s(dt, kp);
  ctl->dt = dt;
  ctl->dtdx = (double)s.dtdx;
  ctl->dt_2h = (double)s.dt_2h;
  ctl->dt_2 = (double)s.dt_2;
  ctl->fdt = (float)s.dt;
  ctl->fdtdx = (float)s.dtdx;
  ctl->fdt_2h = (float)s.dt_2h;
  ctl->fdt_2 = (float)s.dt_2;
}

// A zero step (no step pending).
__device__ __forceinline__ void clear_step_dt(Ctl* ctl) {
  ctl->dt = ctl->dtdx = ctl->dt_2h = ctl->dt_2 = 0.0;
  ctl->fdt = ctl->fdtdx = ctl->fdt_2h = ctl->fdt_2 = 0.0f;
}

// Read a control field written by other blocks in this launch or by the
// previous launch, bypassing L1.
template <typename T>
__device__ __forceinline__ T vload(const T* p) {
  return *(const volatile T*)p;
}

// Ticket of a block: atomic add with acquire-release semantics at GPU scope.
// Release: this block's folds of the maxima and flags (and, through the block
// barrier before it, every thread's stores) are visible to whoever acquires a
// later ticket; acquire: the block that takes the last ticket sees every other
// block's folds.  One round trip instead of a fence followed by an atomic.
__device__ __forceinline__ uint32_t ticket_acq_rel(uint32_t* p) {
  uint32_t v;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Turn the reduced maxima into the next dt (eq. 16 capped by c_tau tau and by
// t_end).  `advance` = the kernel just completed a step.  Runs on one thread
// of the block that took the last ticket (ticket_acq_rel): every other block
// has folded its maxima, so the keys, the flags and the time are read with
// plain loads issued together (one round trip) and reset with plain stores;
// the next launch (kernel boundary) or, in the persistent loop, the caller's
// fence before the barrier bump publishes them.
template <typename R>
__device__ void finalize(Ctl* ctl, const KParams& kp, bool advance, bool flip = true) {
  const uint64_t sk = vload(&ctl->smax_key), tk = vload(&ctl->tau_key);
  uint32_t flags = vload(&ctl->flags);
  double t = vload(&ctl->t);
  const double t_end = vload(&ctl->t_end);
  const uint32_t was_last = vload(&ctl->last), cur = vload(&ctl->cur);
  const double dt_taken = vload(&ctl->dt);
  const int64_t nsteps = vload(&ctl->nsteps);
  ctl->smax_key = key_of(0.0);
  ctl->tau_key = key_of(-INFINITY);
  const double dt = dt_from_maxima(kp, (R)key_to_double(sk), (R)key_to_double(tk), flags);
  if (advance) {
    t = was_last ? t_end : t + dt_taken;
    if (flip) ctl->cur = cur ^ 1u;
    ctl->nsteps = nsteps + 1;
  }
  uint32_t last = 0;
  double dtn = dt;
  if (flags) {
    dtn = 0.0;
  } else if (!(t < t_end)) {
    dtn = 0.0;
  } else if (dt >= t_end - t) {
    dtn = t_end - t;
    last = 1;
  }
  ctl->t = t;
  ctl->dt_cfl = dt;
  set_step_dt<R>(ctl, dtn, kp);
  ctl->last = last;
  ctl->flags = flags;
  ctl->ticket = 0u;
}

// Block-wide fold of (smax, akey, flags) into the control block, then this
// block's ticket.  The fold runs in the kernel's own type T (float kernels
// stay off the narrow FP64 pipe; widening to double after the maximum gives
// the same key as before it).  Returns, in every thread, whether this block
// was the last of the launch to arrive.  Must be called by every thread of
// the block, after its last store.
template <int NT, typename T>
__device__ __forceinline__ bool block_arrive(Ctl* ctl, T smax, T akey, uint32_t flags) {
  __shared__ T s_s[NT / 32], s_a[NT / 32];
  __shared__ uint32_t s_f[NT / 32];
  __shared__ bool s_last;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
    akey = fmax(akey, __shfl_xor_sync(0xffffffffu, akey, o));
    flags |= __shfl_xor_sync(0xffffffffu, flags, o);
  }
  // fmax drops NaN: a non-physical cell already raised its flag.
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    s_s[w] = smax;
    s_a[w] = akey;
    s_f[w] = flags;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < NT / 32; ++i) {
      smax = fmax(smax, s_s[i]);
      akey = fmax(akey, s_a[i]);
      flags |= s_f[i];
    }
    atomicMax((unsigned long long*)&ctl->smax_key, (unsigned long long)key_of((double)smax));
    atomicMax((unsigned long long*)&ctl->tau_key, (unsigned long long)key_of((double)akey));
    if (flags) atomicOr(&ctl->flags, flags);
    const uint32_t ticket = ticket_acq_rel(&ctl->ticket);
    s_last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  return s_last;
}

// block_arrive followed by the last block's finalize.
template <typename R, int NT>
__device__ __forceinline__ void reduce_and_finalize(Ctl* ctl, const KParams& kp, R smax, R akey,
                                                    uint32_t flags, bool advance,
                                                    bool flip = true) {
  const bool last = block_arrive<NT, R>(ctl, smax, akey, flags);
  if (last && threadIdx.x == 0) finalize<R>(ctl, kp, advance, flip);
}

// The index type of a call, taken from its first argument only.
template <typename T> struct index_of { using type = T; };

// Periodic index for |j| within a few periods of [0, N), in the type of j
// (int64_t, or int where the caller's grid fits).
template <typename I>
__device__ __forceinline__ I wrap(I j, typename index_of<I>::type N) {
  if (j >= 0 && j < N) return j;
  j %= N;
  return j < 0 ? j + N : j;
}

}  // namespace sv
