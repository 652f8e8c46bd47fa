// sv_batch.cu -- batched stability sweep: thousands of independent 1D
// periodic runs of uneven sizes and parameters advanced to their own t_end by
// ONE persistent launch.
//
// Each CTA takes a run from a device work queue (the runs of >= 8192 cells
// first, largest first, then the others by decreasing estimated cost,
// n^2 t_end / L, so that the longest runs start first), steps it
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

#include "sv_batch_kernel.cuh"

namespace sv {

// Kernels of the two block sizes: 256 threads here, 128 in sv_batch128.cu.
void* batch_pick256(int limiter, int precision) { return bpick<256>(limiter, precision); }

}  // namespace sv

using namespace sv;

struct sv_batch {
  sv_params p;
  int64_t nruns = 0;
  int log_cap = 0;
  int esize = 4;
  bool ps = false;                    // perturbation layout (SV_FP32_PS)
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
  int nt = 256;                       // threads per run (block size)
  int config = 0;                     // index into kBatchConfigs
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

// Runs of at least this many cells lead the queue (sv_batch_init).
constexpr int64_t kBigRun = 8192;

int64_t stride_of(int64_t n) { return (n + 31) / 32 * 32; }

int check_batch(const sv_params* p, const sv_run* r, int64_t nruns, int log_cap) {
  if (!p || !r || nruns < 1 || nruns > (1 << 30) || log_cap < 0) return SV_EINVAL;
  if (!(p->gamma > 1.0) || !(p->cfl > 0.0) || !(p->c_tau > 0.0)) return SV_EINVAL;
  if (p->limiter < SV_MINMOD || p->limiter > SV_MC) return SV_EINVAL;
  if (p->precision < SV_FP32 || p->precision > SV_FP32_PS) return SV_EINVAL;
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
    const double* ref = b->host_runs[i].kp.ref;
    for (int f = 0; f < 4; ++f)
      for (int64_t j = 0; j < n; ++j) {
        // the perturbation layout holds U - ref (difference in double)
        const double v = host[src + f * n + j] - (b->ps ? ref[f] : 0.0);
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

// Launch configurations of the batch kernel (sv_batch_set_config): block size
// per run.  Smaller blocks keep more runs in flight and idle fewer warps on
// small runs; larger ones finish each run sooner.
struct BatchConfig {
  int nt;
  const char* desc;
};
constexpr BatchConfig kBatchConfigs[] = {
    {256, "batch: 256 threads (8 warps) per run, 64-cell chunks, 2 cells per thread"},
    {128, "batch: 128 threads (4 warps) per run, 64-cell chunks, 2 cells per thread"},
};
constexpr int kNumBatchConfigs = (int)(sizeof(kBatchConfigs) / sizeof(kBatchConfigs[0]));

size_t batch_smem(int precision, int nt) {
  return (size_t)(nt / 32) * (precision == SV_FP64 ? ring1d_bytes<double>() : ring1d_bytes<float>());
}

// Pick the kernel of configuration c, set its shared-memory limit and the
// persistent grid (host side, outside any capture).
int apply_config(sv_batch* b, int c) {
  const int nt = kBatchConfigs[c].nt;
  void* fn = nt == 128 ? batch_pick128(b->p.limiter, b->p.precision)
                       : batch_pick256(b->p.limiter, b->p.precision);
  int dev = 0, sms = 0, per = 0;
  const size_t smem = batch_smem(b->p.precision, nt);
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, nt, smem) != cudaSuccess)
    return SV_ECUDA;
  if (b->graph) {
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return SV_ECUDA;
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  b->fn = fn;
  b->nt = nt;
  b->config = c;
  b->grid = sms * (per < 1 ? 1 : per);
  if ((int64_t)b->grid > b->nruns) b->grid = (int)b->nruns;
  return SV_OK;
}

cudaError_t launch_batch(sv_batch* b, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(b->queue, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  int nr = (int)b->nruns;
  int lc = b->log_cap;
  int64_t ms = b->max_steps;
  void* args[] = {&b->runs, &b->order, &nr, &b->queue, &b->buf[0], &b->buf[1], &b->logs, &lc, &ms};
  return cudaLaunchKernel(b->fn, dim3(b->grid), dim3(b->nt), args, batch_smem(b->p.precision, b->nt),
                          st);
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
  b->ps = p->precision == SV_FP32_PS;
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
    k.S = r.S;
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

  // Queue order.  The runs of >= kBigRun cells first, largest first: a run's
  // worst case is the step cap, whose cost grows with n alone, and the few
  // large runs that reach it (their dt collapses long after the start, which
  // no estimate from the initial state foresees) set the sweep's end unless
  // they start early.  Then the others, longest first by the estimated cost
  // n * steps ~ n^2 t_end / L.
  std::vector<int> order((size_t)nruns);
  std::iota(order.begin(), order.end(), 0);
  std::vector<double> cost((size_t)nruns);
  for (int64_t i = 0; i < nruns; ++i)
    cost[(size_t)i] = (double)runs[i].n * (double)runs[i].n * runs[i].t_end / runs[i].L;
  auto big = [&](int i) { return runs[i].n >= kBigRun; };
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
    if (big(a) != big(c)) return big(a);
    return big(a) ? runs[a].n > runs[c].n : cost[a] > cost[c];
  });

  rc = SV_OK;
  if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMemcpyAsync(b->order, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice,
                      b->stream) != cudaSuccess)
    rc = SV_ECUDA;
  if (rc == SV_OK) rc = apply_config(b, 0);
  if (rc == SV_OK) rc = upload(b, host_states);
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
          host_soa[f * n + j] = (b->ps ? d.kp.ref[f] : 0.0) + (double)fv;
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

int sv_batch_num_configs(sv_batch* b, int* count) {
  if (!b || !count) return SV_EINVAL;
  *count = kNumBatchConfigs;
  return SV_OK;
}

int sv_batch_set_config(sv_batch* b, int index) {
  if (!b || index < 0 || index >= kNumBatchConfigs) return SV_EINVAL;
  return apply_config(b, index);
}

int sv_batch_get_config(sv_batch* b, int* index, char* desc, size_t cap) {
  if (!b) return SV_EINVAL;
  if (index) *index = b->config;
  if (desc && cap > 0) {
    strncpy(desc, kBatchConfigs[b->config].desc, cap - 1);
    desc[cap - 1] = 0;
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
