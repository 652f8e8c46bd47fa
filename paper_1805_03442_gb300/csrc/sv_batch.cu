// sv_batch.cu -- batched stability sweep: thousands of independent 1D
// periodic runs of uneven sizes and parameters advanced to their own t_end by
// ONE persistent launch.
//
// Each CTA takes a run from a device work queue (runs ordered by decreasing
// estimated cost, n^2 t_end / L, so the longest runs start first), steps it
// to completion with the same per-warp MUSCL-Hancock body as the single-grid
// kernel (sv_step1d.cuh), and only then takes the next run.  A run's dt
// reduction is CTA-local (shared memory + __syncthreads): there is no grid
// barrier and no host round trip per step.  At sampled times the CTA
// projects the velocity on the logged Fourier mode m,
//   a_m(t) = (1/n) sum_j v_j exp(-i 2 pi m (j + 1/2) / n),
// which is what a growth-rate fit of the linear stage needs.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "sv.h"
#include "sv_internal.h"
#include "sv_step1d.cuh"

namespace sv {

constexpr int NTB = 256;

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

template <typename R>
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
    for (int i = 1; i < NTB / 32; ++i) {
      smax = fmax(smax, s_a[i]);
      akey = fmax(akey, s_b[i]);
      flags |= s_f[i];
    }
}

template <typename R>
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
    for (int i = 1; i < NTB / 32; ++i) {
      a += s_a[i];
      b += s_b[i];
    }
}

// Every run is stepped with the source variant a single 1D solver with the
// same parameters would use (none in the frozen limit, pump = sink for zero
// exponents, general otherwise), chosen per run at run time, so that a batched
// run and a looped solver run execute the same instructions.
template <typename R, int PP, int LIM, int MINB>
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
        const R v = U[stride + j] / U[j];
        R sn, cs;
        const R ph = (R)(2.0 * mode) * ((R)j + (R)0.5) / (R)n;
        if constexpr (sizeof(R) == 4) sincospif(ph, &sn, &cs);
        else sincospi(ph, &sn, &cs);
        re += v * cs;
        im -= v * sn;
      }
      block_sum2(re, im, s_a, s_b);
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
        const R rho = A[j], m = A[stride + j];
        const R ir = Ar<R>::rcp(rho);
        const R v = m * ir;
        cfl_cell<R, PP, 1>(k, rho, m * v, fabs(m * ir), A[2 * stride + j], A[3 * stride + j], smax,
                           akey, flags);
      }
      block_max(smax, akey, flags, s_a, s_b, s_f);
      if (threadIdx.x == 0) {
        const double dt = dt_from_maxima<R>(kp, (double)smax, (double)akey, flags);
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
        const StepDt<R> sd(s_dt, kp.h);
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
      block_max(smax, akey, flags, s_a, s_b, s_f);
      cur ^= 1u;
      ++steps;
      if (threadIdx.x == 0) {
        const double dt_next = dt_from_maxima<R>(kp, (double)smax, (double)akey, flags);
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
        const StepDt<R> sd(s_dt, kp.h);
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

template <typename R, int PP, int LIM>
struct KB {
  static constexpr int MINB = sizeof(R) == 8 ? 1 : 2;
  static constexpr auto fn = batch_kernel<R, PP, LIM, MINB>;
};

template <int LIM>
static void* bpick_prec(int precision) {
  switch (precision) {
    case PREC_FP64: return (void*)KB<double, 0, LIM>::fn;
    case PREC_FP32_P64: return (void*)KB<float, 1, LIM>::fn;
    default: return (void*)KB<float, 0, LIM>::fn;
  }
}
static void* bpick(int limiter, int precision) {
  switch (limiter) {
    case 1: return bpick_prec<1>(precision);
    case 2: return bpick_prec<2>(precision);
    default: return bpick_prec<0>(precision);
  }
}

}  // namespace sv

using namespace sv;

struct sv_batch {
  sv_params p;
  int64_t nruns = 0;
  int log_cap = 0;
  int esize = 4;
  cudaStream_t stream = nullptr, cap_stream = nullptr;
  void* mem = nullptr;
  bool owns_mem = false;
  void* buf[2] = {nullptr, nullptr};
  RunDev* runs = nullptr;
  int* order = nullptr;
  int* queue = nullptr;
  double* logs = nullptr;
  std::vector<RunDev> host_runs;
  std::vector<int64_t> n;
  int64_t total_elems = 0;
  int grid = 0;
  void* fn = nullptr;
  cudaGraphExec_t graph = nullptr;
  int64_t max_steps = 0;
};

namespace {

constexpr size_t kAlignB = 256;
size_t alb(size_t x) { return (x + kAlignB - 1) / kAlignB * kAlignB; }

struct BLayout {
  size_t state, runs, order, queue, logs, total;
};

int64_t stride_of(int64_t n) { return (n + 31) / 32 * 32; }

int check_batch(const sv_params* p, const sv_run* r, int64_t nruns, int log_cap) {
  if (!p || !r || nruns < 1 || nruns > (1 << 30) || log_cap < 0) return SV_EINVAL;
  if (!(p->gamma > 1.0) || !(p->cfl > 0.0) || !(p->c_tau > 0.0)) return SV_EINVAL;
  if (p->limiter < SV_MINMOD || p->limiter > SV_MC) return SV_EINVAL;
  if (p->precision < SV_FP32 || p->precision > SV_FP32_P64) return SV_EINVAL;
  if (p->method != SV_HANCOCK) return SV_EINVAL;
  for (int64_t i = 0; i < nruns; ++i) {
    if (r[i].n < 1 || r[i].n > (1 << 24) || !(r[i].L > 0.0) || !(r[i].tau0 > 0.0) ||
        !(r[i].t_end >= 0.0) || r[i].mode < 0)
      return SV_EINVAL;
  }
  return SV_OK;
}

BLayout blayout(const sv_params* p, const sv_run* r, int64_t nruns, int log_cap) {
  int64_t elems = 0;
  for (int64_t i = 0; i < nruns; ++i) elems += 4 * stride_of(r[i].n);
  const size_t es = p->precision == SV_FP64 ? 8 : 4;
  BLayout L;
  L.state = alb((size_t)elems * es);
  L.runs = alb(sizeof(RunDev) * (size_t)nruns);
  L.order = alb(sizeof(int) * (size_t)nruns);
  L.queue = alb(sizeof(int));
  L.logs = alb(sizeof(double) * 3 * (size_t)log_cap * (size_t)nruns);
  L.total = 2 * L.state + L.runs + L.order + L.queue + L.logs;
  return L;
}

#define SVB_TRY(expr)                        \
  do {                                       \
    cudaError_t e_ = (expr);                 \
    if (e_ != cudaSuccess) return SV_ECUDA;  \
  } while (0)

int upload(sv_batch* b, const double* host) {
  // host: concatenation over runs of (4, n_r) field-major blocks
  const size_t es = (size_t)b->esize;
  std::vector<unsigned char> tmp((size_t)b->total_elems * es, 0);
  int64_t src = 0;
  for (int64_t i = 0; i < b->nruns; ++i) {
    const int64_t n = b->n[i], st = stride_of(n), off = b->host_runs[i].off;
    for (int f = 0; f < 4; ++f)
      for (int64_t j = 0; j < n; ++j) {
        const double v = host[src + f * n + j];
        const size_t at = (size_t)(off + f * st + j);
        if (es == 8) memcpy(&tmp[at * 8], &v, 8);
        else {
          const float fv = (float)v;
          memcpy(&tmp[at * 4], &fv, 4);
        }
      }
    src += 4 * n;
  }
  SVB_TRY(cudaMemcpyAsync(b->buf[0], tmp.data(), tmp.size(), cudaMemcpyHostToDevice, b->stream));
  for (auto& r : b->host_runs) {
    r.t = 0.0;
    r.steps = 0;
    r.flags = 0;
    r.cur = 0;
    r.log_count = 0;
  }
  SVB_TRY(cudaMemcpyAsync(b->runs, b->host_runs.data(), sizeof(RunDev) * b->host_runs.size(),
                          cudaMemcpyHostToDevice, b->stream));
  return cudaStreamSynchronize(b->stream) == cudaSuccess ? SV_OK : SV_ECUDA;
}

size_t batch_smem(int precision) {
  return (size_t)(NTB / 32) * (precision == SV_FP64 ? ring1d_bytes<double>() : ring1d_bytes<float>());
}

cudaError_t launch_batch(sv_batch* b, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(b->queue, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  int nr = (int)b->nruns;
  int lc = b->log_cap;
  int64_t ms = b->max_steps;
  void* args[] = {&b->runs, &b->order, &nr, &b->queue, &b->buf[0], &b->buf[1], &b->logs, &lc, &ms};
  return cudaLaunchKernel(b->fn, dim3(b->grid), dim3(NTB), args, batch_smem(b->p.precision), st);
}

int read_runs(sv_batch* b) {
  SVB_TRY(cudaMemcpyAsync(b->host_runs.data(), b->runs, sizeof(RunDev) * b->host_runs.size(),
                          cudaMemcpyDeviceToHost, b->stream));
  SVB_TRY(cudaStreamSynchronize(b->stream));
  return SV_OK;
}

}  // namespace

extern "C" {

int sv_batch_required_bytes(const sv_params* p, const sv_run* runs, int64_t nruns, int log_cap,
                            size_t* bytes) {
  int rc = check_batch(p, runs, nruns, log_cap);
  if (rc != SV_OK) return rc;
  if (!bytes) return SV_EINVAL;
  *bytes = blayout(p, runs, nruns, log_cap).total;
  return SV_OK;
}

int sv_batch_init(const sv_params* p, const sv_run* runs, int64_t nruns,
                  const double* host_states, int log_cap, int64_t max_steps_per_run,
                  void* cuda_stream, void* device_mem, size_t device_bytes, sv_batch** out) {
  if (!out || !host_states || max_steps_per_run < 1) return SV_EINVAL;
  *out = nullptr;
  int rc = check_batch(p, runs, nruns, log_cap);
  if (rc != SV_OK) return rc;
  const BLayout L = blayout(p, runs, nruns, log_cap);
  if (device_mem && (device_bytes < L.total || ((uintptr_t)device_mem % kAlignB) != 0))
    return SV_ENOMEM;
  sv_batch* b = new (std::nothrow) sv_batch();
  if (!b) return SV_ENOMEM;
  b->p = *p;
  b->nruns = nruns;
  b->log_cap = log_cap;
  b->esize = p->precision == SV_FP64 ? 8 : 4;
  b->stream = (cudaStream_t)cuda_stream;
  b->max_steps = max_steps_per_run;
  b->host_runs.resize((size_t)nruns);
  b->n.resize((size_t)nruns);
  int64_t off = 0;
  for (int64_t i = 0; i < nruns; ++i) {
    const sv_run& r = runs[i];
    RunDev d;
    memset(&d, 0, sizeof d);
    KParams& k = d.kp;
    k.gamma = p->gamma;
    k.g1 = p->gamma - 1.0;
    k.Ck = p->Ck;
    k.frozen = isinf(r.tau0) ? 1 : 0;
    k.tau0 = r.tau0;
    k.inv_tau0 = k.frozen ? 0.0 : 1.0 / r.tau0;
    k.Q0 = k.frozen ? 0.0 : r.S / r.tau0;
    k.tau_rho = r.tau_rho;
    k.tau_T = r.tau_T;
    k.Q_rho = r.Q_rho;
    k.Q_T = r.Q_T;
    k.I_rho = r.I_rho;
    k.I_T = r.I_T;
    k.qi_zero = (r.Q_rho == 0.0 && r.Q_T == 0.0 && r.I_rho == 0.0 && r.I_T == 0.0) ? 1 : 0;
    k.h = r.L / (double)r.n;
    k.cfl = p->cfl;
    k.c_tau = p->c_tau;
    k.limiter = p->limiter;
    kparams_finish(k);
    d.src = k.frozen ? 0 : (k.qi_zero ? 1 : 2);
    d.off = off;
    d.n = (int)r.n;
    d.stride = (int)stride_of(r.n);
    d.mode = r.mode;
    d.t_end = r.t_end;
    b->host_runs[(size_t)i] = d;
    b->n[(size_t)i] = r.n;
    off += 4 * stride_of(r.n);
  }
  b->total_elems = off;
  b->fn = bpick(p->limiter, p->precision);

  if (device_mem) b->mem = device_mem;
  else {
    if (cudaMalloc(&b->mem, L.total) != cudaSuccess) {
      delete b;
      return SV_ENOMEM;
    }
    b->owns_mem = true;
  }
  char* m = (char*)b->mem;
  b->buf[0] = m;
  b->buf[1] = m + L.state;
  b->runs = (RunDev*)(m + 2 * L.state);
  b->order = (int*)(m + 2 * L.state + L.runs);
  b->queue = (int*)(m + 2 * L.state + L.runs + L.order);
  b->logs = (double*)(m + 2 * L.state + L.runs + L.order + L.queue);

  // longest runs first: cost ~ n * steps ~ n^2 t_end / L
  std::vector<int> order((size_t)nruns);
  std::iota(order.begin(), order.end(), 0);
  std::vector<double> cost((size_t)nruns);
  for (int64_t i = 0; i < nruns; ++i)
    cost[(size_t)i] = (double)runs[i].n * (double)runs[i].n * runs[i].t_end / runs[i].L;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost[a] > cost[c]; });

  rc = SV_OK;
  int dev = 0, sms = 0, per = 0;
  if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaFuncSetAttribute(b->fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)batch_smem(p->precision)) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, b->fn, NTB, batch_smem(p->precision)) !=
          cudaSuccess ||
      cudaMemcpyAsync(b->order, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice,
                      b->stream) != cudaSuccess)
    rc = SV_ECUDA;
  if (rc == SV_OK) {
    b->grid = sms * (per < 1 ? 1 : per);
    if ((int64_t)b->grid > nruns) b->grid = (int)nruns;
    rc = upload(b, host_states);
  }
  if (rc != SV_OK) {
    sv_batch_free(b);
    return rc;
  }
  *out = b;
  return SV_OK;
}

int sv_batch_reset(sv_batch* b, const double* host_states) {
  if (!b || !host_states) return SV_EINVAL;
  return upload(b, host_states);
}

int sv_batch_run(sv_batch* b) {
  if (!b) return SV_EINVAL;
  if (!b->graph) {
    cudaGraph_t g = nullptr;
    SVB_TRY(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t le = launch_batch(b, b->cap_stream);
    cudaError_t ee = cudaStreamEndCapture(b->cap_stream, &g);
    if (le != cudaSuccess || ee != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return SV_ECUDA;
    }
    cudaError_t ie = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
      b->graph = nullptr;
      return SV_ECUDA;
    }
  }
  SVB_TRY(cudaGraphLaunch(b->graph, b->stream));
  return SV_OK;
}

int sv_batch_sync(sv_batch* b) {
  if (!b) return SV_EINVAL;
  SVB_TRY(cudaStreamSynchronize(b->stream));
  return SV_OK;
}

int sv_batch_read(sv_batch* b, int64_t run, double* host_soa, double* t, int64_t* steps,
                  uint32_t* flags) {
  if (!b || run < 0 || run >= b->nruns) return SV_EINVAL;
  int rc = read_runs(b);
  if (rc != SV_OK) return rc;
  const RunDev& d = b->host_runs[(size_t)run];
  if (t) *t = d.t;
  if (steps) *steps = d.steps;
  if (flags) *flags = d.flags;
  if (host_soa) {
    const int64_t n = d.n, st = d.stride;
    const size_t es = (size_t)b->esize;
    std::vector<unsigned char> tmp((size_t)(4 * st) * es);
    const char* src = (const char*)b->buf[d.cur ? 1 : 0] + (size_t)d.off * es;
    SVB_TRY(cudaMemcpyAsync(tmp.data(), src, tmp.size(), cudaMemcpyDeviceToHost, b->stream));
    SVB_TRY(cudaStreamSynchronize(b->stream));
    for (int f = 0; f < 4; ++f)
      for (int64_t j = 0; j < n; ++j) {
        const size_t at = (size_t)(f * st + j);
        if (es == 8) memcpy(&host_soa[f * n + j], &tmp[at * 8], 8);
        else {
          float fv;
          memcpy(&fv, &tmp[at * 4], 4);
          host_soa[f * n + j] = fv;
        }
      }
  }
  return SV_OK;
}

int sv_batch_mode_log(sv_batch* b, int64_t run, double* t, double* re, double* im, int64_t cap,
                      int64_t* count) {
  if (!b || run < 0 || run >= b->nruns || cap < 0) return SV_EINVAL;
  int rc = read_runs(b);
  if (rc != SV_OK) return rc;
  const int64_t c = std::min<int64_t>(b->host_runs[(size_t)run].log_count, cap);
  if (count) *count = c;
  if (c > 0) {
    std::vector<double> tmp((size_t)c * 3);
    SVB_TRY(cudaMemcpyAsync(tmp.data(), b->logs + run * (int64_t)b->log_cap * 3,
                            sizeof(double) * tmp.size(), cudaMemcpyDeviceToHost, b->stream));
    SVB_TRY(cudaStreamSynchronize(b->stream));
    for (int64_t i = 0; i < c; ++i) {
      if (t) t[i] = tmp[(size_t)(3 * i)];
      if (re) re[i] = tmp[(size_t)(3 * i + 1)];
      if (im) im[i] = tmp[(size_t)(3 * i + 2)];
    }
  }
  return SV_OK;
}

void sv_batch_free(sv_batch* b) {
  if (!b) return;
  if (b->stream || b->mem) cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  if (b->owns_mem && b->mem) cudaFree(b->mem);
  delete b;
}

}  // extern "C"
