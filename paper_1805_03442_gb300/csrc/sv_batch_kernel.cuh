// sv_batch_kernel.cuh -- the persistent kernel of the batched stability sweep
// (see sv_batch.cu), templated on its block size so that each size compiles
// in a translation unit of its own.
#pragma once

#include "sv.h"
#include "sv_internal.h"
#include "sv_step1d.cuh"

namespace sv {

struct RunDev {
  KParams kp;            // per-run parameters (h = L / n)
  int64_t off;           // element offset of the run's block (4 fields x stride)
  int n, stride, mode, log_count;
  int src, pad2;         // source variant of the run (as a single solver would pick it)
  double t, t_end;
  int64_t steps;
  uint32_t flags, cur, pad0, pad1;
};

constexpr uint32_t FLAG_MAXSTEPS = SV_FLAG_MAXSTEPS;

template <int NT, typename R>
__device__ __forceinline__ void block_max(R& smax, R& akey, uint32_t& flags, R* s_a, R* s_b,
                                          uint32_t* s_f) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
    akey = fmax(akey, __shfl_xor_sync(0xffffffffu, akey, o));
    flags |= __shfl_xor_sync(0xffffffffu, flags, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    s_a[w] = smax;
    s_b[w] = akey;
    s_f[w] = flags;
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int i = 1; i < NT / 32; ++i) {
      smax = fmax(smax, s_a[i]);
      akey = fmax(akey, s_b[i]);
      flags |= s_f[i];
    }
}

template <int NT, typename R>
__device__ __forceinline__ void block_sum2(R& a, R& b, R* s_a, R* s_b) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    s_a[w] = a;
    s_b[w] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int i = 1; i < NT / 32; ++i) {
      a += s_a[i];
      b += s_b[i];
    }
}

// Every run is stepped with the source variant a single 1D solver with the
// same parameters would use (none in the frozen limit, pump = sink for zero
// exponents, general otherwise), chosen per run at run time, so that a batched
// run and a looped solver run execute the same instructions.
template <typename R, int PP, int LIM, int NTB, int MINB>
__global__ void __launch_bounds__(NTB, MINB)
batch_kernel(RunDev* __restrict__ runs, const int* __restrict__ order, int nruns,
             int* __restrict__ queue, R* __restrict__ bufA, R* __restrict__ bufB,
             double* __restrict__ logs, int log_cap, int64_t max_steps) {
  __shared__ R s_a[NTB / 32], s_b[NTB / 32];
  __shared__ uint32_t s_f[NTB / 32];
  __shared__ int s_run, s_stop, s_last, s_log;
  __shared__ double s_dt, s_t;
  __shared__ R s_step[4];               // dt, dt/h, dt/(2h), dt/2 of the next step
  extern __shared__ __align__(16) unsigned char smemb[];   // per-warp rings
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  R* ring = reinterpret_cast<R*>(smemb) + warp * (ring1d_bytes<R>() / sizeof(R));

  for (;;) {
    if (threadIdx.x == 0) s_run = atomicAdd(queue, 1);
    __syncthreads();
    const int qi = s_run;
    if (qi >= nruns) break;
    RunDev* rd = runs + order[qi];
    const KParams& kp = rd->kp;
    const P<R> k(kp);
    const int n = rd->n, stride = rd->stride, mode = rd->mode, src = rd->src;
    const double t_end = rd->t_end;
    R* A = bufA + rd->off;
    R* B = bufB + rd->off;
    const int nchunk = (n + 63) / 64;
    const int c0 = warp * nchunk / (NTB / 32), c1 = (warp + 1) * nchunk / (NTB / 32);
    double* lg = logs + (int64_t)(order[qi]) * log_cap * 3;
    const double log_dt = log_cap > 1 ? t_end / (double)(log_cap - 1) : INFINITY;

    // logging of a_m at the current state (buffer U)
    auto log_mode = [&](const R* U, double t, int slot) {
      R re = 0, im = 0;
      for (int j = threadIdx.x; j < n; j += NTB) {
        const R v = U[stride + j] / (PP == 3 ? (R)1 + U[j] : U[j]);   // PP 3: perturbations
        R sn, cs;
        const R ph = (R)(2.0 * mode) * ((R)j + (R)0.5) / (R)n;
        if constexpr (sizeof(R) == 4) sincospif(ph, &sn, &cs);
        else sincospi(ph, &sn, &cs);
        re += v * cs;
        im -= v * sn;
      }
      block_sum2<NTB>(re, im, s_a, s_b);
      if (threadIdx.x == 0) {
        lg[3 * slot + 0] = t;
        lg[3 * slot + 1] = (double)re / n;
        lg[3 * slot + 2] = (double)im / n;
      }
      __syncthreads();
    };

    // dt of the initial state (same per-cell bound as every step)
    {
      R smax = 0, akey = -INFINITY;
      uint32_t flags = 0;
      for (int j = threadIdx.x; j < n; j += NTB) {
        const R u[4] = {A[j], A[stride + j], A[2 * stride + j], A[3 * stride + j]};
        cell_bound<R, PP, 1>(k, u, smax, akey, flags);
      }
      block_max<NTB>(smax, akey, flags, s_a, s_b, s_f);
      if (threadIdx.x == 0) {
        const double dt = dt_from_maxima(kp, smax, akey, flags);
        double t = rd->t;
        rd->flags = flags;
        s_t = t;
        s_stop = flags != 0 || !(t < t_end);
        s_last = 0;
        s_dt = dt;
        if (!s_stop && dt >= t_end - t) {
          s_dt = t_end - t;
          s_last = 1;
        }
        const StepDt<R> sd(s_dt, kp);
        s_step[0] = sd.dt;
        s_step[1] = sd.dtdx;
        s_step[2] = sd.dt_2h;
        s_step[3] = sd.dt_2;
      }
      __syncthreads();
    }
    int log_count = 0;
    double next_log = s_t;
    if (mode > 0 && log_cap > 0) {
      log_mode(A, s_t, 0);
      log_count = 1;
      next_log = s_t + log_dt;
    }
    uint32_t cur = 0;
    int64_t steps = 0;
    while (!s_stop) {
      const double dtd = s_dt;
      const R dt = s_step[0], dtdx = s_step[1], dt_2h = s_step[2], dt_2 = s_step[3];
      const R* Uin = cur ? B : A;
      R* Uout = cur ? A : B;
      R smax = 0, akey = -INFINITY;
      uint32_t flags = 0;
      if (src == 0)
        step1d_warp<R, PP, LIM, 0>(k, Uin, Uout, n, stride, c0, c1, lane, dt, dtdx, dt_2h, dt_2,
                                   smax, akey, flags, ring, kp, s_t);
      else if (src == 1)
        step1d_warp<R, PP, LIM, 1>(k, Uin, Uout, n, stride, c0, c1, lane, dt, dtdx, dt_2h, dt_2,
                                   smax, akey, flags, ring, kp, s_t);
      else
        step1d_warp<R, PP, LIM, 2>(k, Uin, Uout, n, stride, c0, c1, lane, dt, dtdx, dt_2h, dt_2,
                                   smax, akey, flags, ring, kp, s_t);
      // the barrier inside block_max also orders this step's stores before the
      // next step's loads of neighbouring warps' cells
      block_max<NTB>(smax, akey, flags, s_a, s_b, s_f);
      cur ^= 1u;
      ++steps;
      if (threadIdx.x == 0) {
        const double dt_next = dt_from_maxima(kp, smax, akey, flags);
        const double t = s_last ? t_end : s_t + dtd;
        s_t = t;
        if (steps >= max_steps && t < t_end) flags |= FLAG_MAXSTEPS;
        rd->flags = flags;
        s_stop = flags != 0 || !(t < t_end);
        s_last = 0;
        s_dt = dt_next;
        if (!s_stop && dt_next >= t_end - t) {
          s_dt = t_end - t;
          s_last = 1;
        }
        const StepDt<R> sd(s_dt, kp);
        s_step[0] = sd.dt;
        s_step[1] = sd.dtdx;
        s_step[2] = sd.dt_2h;
        s_step[3] = sd.dt_2;
        s_log = mode > 0 && log_count < log_cap && (t >= next_log || s_stop);
      }
      __syncthreads();
      if (s_log) {
        log_mode(cur ? B : A, s_t, log_count);
        ++log_count;
        while (next_log <= s_t) next_log += log_dt;
      }
    }
    if (threadIdx.x == 0) {
      rd->t = s_t;
      rd->steps = steps;
      rd->cur = cur;
      rd->log_count = log_count;
    }
    __syncthreads();
  }
}

// Kernel of the given block size for (limiter, precision).
template <int NTB, typename R, int PP, int LIM>
struct KB {
  // double and the perturbation layout take the whole register file (one
  // block per SM) rather than spill
  static constexpr int MINB = (sizeof(R) == 8 || PP == 3) ? 1 : 256 / NTB * 2;
  static constexpr auto fn = batch_kernel<R, PP, LIM, NTB, MINB>;
};

template <int NTB, int LIM>
void* bpick_prec(int precision) {
  switch (precision) {
    case PREC_FP64: return (void*)KB<NTB, double, 0, LIM>::fn;
    case PREC_FP32_P64: return (void*)KB<NTB, float, 1, LIM>::fn;
    case PREC_FP32_PC: return (void*)KB<NTB, float, 2, LIM>::fn;
    case PREC_FP32_PS: return (void*)KB<NTB, float, 3, LIM>::fn;
    default: return (void*)KB<NTB, float, 0, LIM>::fn;
  }
}
template <int NTB>
void* bpick(int limiter, int precision) {
  switch (limiter) {
    case 1: return bpick_prec<NTB, 1>(precision);
    case 2: return bpick_prec<NTB, 2>(precision);
    default: return bpick_prec<NTB, 0>(precision);
  }
}

}  // namespace sv
