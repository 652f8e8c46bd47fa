// sv_api.cu -- host runtime behind the C ABI of include/sv.h.
//
// One solver = one device block carved into: two state buffers (ping-pong),
// a double staging buffer for host I/O, the control block (time, dt,
// reductions, current buffer, flags) and the scratch of the conservation sums.
// Steps are launched on the caller's stream; runs of steps are replayed from a
// CUDA graph captured once per solver.  The device decides dt, the clamp to
// t_end and the buffer flip, so nothing is read back between steps.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "sv.h"
#include "sv_internal.h"
#include "sv_model.cuh"

using namespace sv;

// One launch configuration of a solver's per-step kernel (sv_set_config).
struct SolverConfig {
  int kind;        // CFG_TILE, CFG_SLIDE or CFG_ND
  int param;       // TILE: 10 x cell pairs per thread + blocks per SM; ND: planes per segment
  const char* desc;
};
enum { CFG_TILE = 0, CFG_SLIDE = 1, CFG_ND = 2 };

struct sv_solver {
  sv_params p;
  sv_grid g;
  int dim = 1, nf = 4, esize = 4;
  int64_t ncell = 0;
  double h = 0;
  KParams kp;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;   // private stream used only to capture graphs
  void* mem = nullptr;
  bool owns_mem = false;
  void* buf[2] = {nullptr, nullptr};
  double* staging = nullptr;
  Ctl* ctl = nullptr;
  double* partial = nullptr;
  double* sums_out = nullptr;
  Ctl* host_ctl = nullptr;             // pinned mirror of the control block
  int* medium_dev = nullptr;           // 2D medium map and driven cells: 4 x ny int32
  double* host_sums = nullptr;
  int grid = 0;
  int tile_grid = 0;                   // grid of the block-tile kernel of the current config
  std::vector<SolverConfig> cfgs;      // launch configurations of the per-step kernel
  int config = 0;                      // current index into cfgs
  int loop_grid = 0;                   // persistent 1D loop: blocks (0 = not available)
  bool loop_fits = false;              // ... at most one 64-cell chunk per SM
  int launch = SV_LAUNCH_AUTO;
  cudaGraphExec_t graph = nullptr;
  int graph_len = 0;
};

namespace {

constexpr size_t kAlign = 256;
constexpr int kGraphLen = 32;
constexpr int64_t kLoopChunk = 1 << 16;   // steps per persistent launch at most

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Layout {
  size_t state, staging, ctl, partial, sums, total;
};

int check_inputs(const sv_params* p, const sv_grid* g) {
  if (!p || !g) return SV_EINVAL;
  if (g->dim < 1 || g->dim > 3) return SV_EINVAL;
  for (int a = 0; a < g->dim; ++a)
    if (g->n[a] < 1 || !(g->L[a] > 0.0)) return SV_EINVAL;
  const double h = g->L[0] / (double)g->n[0];
  for (int a = 1; a < g->dim; ++a)
    if (fabs(g->L[a] / (double)g->n[a] - h) > 1e-12 * h) return SV_EINVAL;
  if (!(p->gamma > 1.0) || !(p->cfl > 0.0) || !(p->c_tau > 0.0) || !(p->tau0 > 0.0))
    return SV_EINVAL;
  if (p->limiter < SV_MINMOD || p->limiter > SV_MC) return SV_EINVAL;
  if (p->precision < SV_FP32 || p->precision > SV_FP32_PS) return SV_EINVAL;
  // the perturbation layout: MUSCL-Hancock
  if (p->precision == SV_FP32_PS && p->method != SV_HANCOCK) return SV_EINVAL;
  for (int side = 0; side < 2; ++side)
    if (g->bc[side] < SV_BC_PERIODIC || g->bc[side] > SV_BC_DRIVEN) return SV_EINVAL;
  if (g->bc[1] == SV_BC_DRIVEN) return SV_EINVAL;
  if (g->dim == 2) {
    // walls and outflow on any side; the driven boundary is 1D only
    for (int side = 0; side < 4; ++side)
      if (g->bc[side] < SV_BC_PERIODIC || g->bc[side] > SV_BC_OUTFLOW) return SV_EINVAL;
    for (int a = 0; a < 2; ++a)
      if ((g->bc[2 * a] != SV_BC_PERIODIC || g->bc[2 * a + 1] != SV_BC_PERIODIC) && g->n[a] < 2)
        return SV_EINVAL;
  }
  if (g->dim == 3)
    for (int side = 0; side < 4; ++side)
      if (g->bc[side] != SV_BC_PERIODIC) return SV_EINVAL;
  if (p->method != SV_HANCOCK && p->method != SV_HEUN) return SV_EINVAL;
  if (p->method == SV_HEUN &&
      (g->dim != 1 || g->bc[0] != SV_BC_PERIODIC || g->bc[1] != SV_BC_PERIODIC ||
       p->precision == SV_FP32_P64 || p->precision == SV_FP32_PC))
    return SV_EINVAL;
  if (g->dim == 1 && (g->bc[0] != SV_BC_PERIODIC || g->bc[1] != SV_BC_PERIODIC) && g->n[0] < 2)
    return SV_EINVAL;
  return SV_OK;
}

Layout layout(const sv_params* p, const sv_grid* g) {
  int64_t ncell = 1;
  for (int a = 0; a < g->dim; ++a) ncell *= g->n[a];
  const int nf = g->dim + 3;
  const size_t es = p->precision == SV_FP64 ? 8 : 4;
  Layout L;
  L.state = align_up((size_t)nf * (size_t)ncell * es);
  L.staging = align_up((size_t)nf * (size_t)ncell * 8);
  L.ctl = align_up(sizeof(Ctl));
  L.partial = align_up((size_t)sums_blocks() * (size_t)nf * 2 * 8);
  L.sums = align_up(8 * 8);
  L.total = 2 * L.state + L.staging + L.ctl + L.partial + L.sums;
  return L;
}

#define SV_TRY(expr)                         \
  do {                                       \
    cudaError_t e_ = (expr);                 \
    if (e_ != cudaSuccess) return SV_ECUDA;  \
  } while (0)

// One step's launches; pdl: the 1D step kernels with the programmatic
// stream-serialization attribute (recorded so in the step graph: a step may
// launch while the previous one finishes and waits in pdl_wait).
cudaError_t launch_step(sv_solver* s, cudaStream_t st, bool pdl = false) {
  if (s->dim == 1 && s->p.method == SV_HEUN) {
    cudaError_t e = heun1d_launch(s->p.precision, 1, s->kp, s->buf[0], s->buf[1], s->ctl, s->ncell,
                                  s->grid, st);
    if (e != cudaSuccess) return e;
    return heun1d_launch(s->p.precision, 2, s->kp, s->buf[0], s->buf[1], s->ctl, s->ncell, s->grid,
                         st);
  }
  const SolverConfig& c = s->cfgs[(size_t)s->config];
  if (c.kind == CFG_TILE)
    return tile1d_launch(s->kp, s->p.precision, c.param, s->buf[0], s->buf[1], s->ctl, s->ncell,
                         s->tile_grid, st, pdl);
  if (c.kind == CFG_SLIDE)
    return step1d_launch(s->p.precision, s->kp, s->buf[0], s->buf[1], s->ctl, s->ncell, s->grid, st,
                         pdl);
  return stepnd_launch(s->dim, s->p.precision, s->kp, s->buf[0], s->buf[1], s->ctl, s->g.n,
                       c.param, st);
}

int ensure_graph(sv_solver* s) {
  if (s->graph) return SV_OK;
  cudaGraph_t gr = nullptr;
  SV_TRY(cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t le = cudaSuccess;
  for (int i = 0; i < kGraphLen && le == cudaSuccess; ++i) le = launch_step(s, s->cap_stream, true);
  cudaError_t ee = cudaStreamEndCapture(s->cap_stream, &gr);
  if (le != cudaSuccess || ee != cudaSuccess) {
    if (gr) cudaGraphDestroy(gr);
    return SV_ECUDA;
  }
  cudaError_t ie = cudaGraphInstantiate(&s->graph, gr, 0);
  cudaGraphDestroy(gr);
  if (ie != cudaSuccess) {
    s->graph = nullptr;
    return SV_ECUDA;
  }
  s->graph_len = kGraphLen;
  return SV_OK;
}

// The persistent loop serves 1D MUSCL-Hancock solvers: always when asked for,
// by default on grids of at most one 64-cell chunk per two SMs, where a step
// is short enough for the gap between launches to matter (measured on a
// GB300 with the float finalize: 7.8 instead of 10.1 us per float step at 200
// cells, equal at 1600-5000 cells, 25-33% slower from 2e4 cells on).
bool use_loop(const sv_solver* s) {
  if (s->loop_grid < 1) return false;
  return s->launch == SV_LAUNCH_PERSISTENT || (s->launch == SV_LAUNCH_AUTO && s->loop_fits);
}

// Launch configurations a solver can choose from, the default first.
const char* seg_desc(int seg) {
  switch (seg) {
    case 64: return "2D/3D: marching segments of 64 planes per block";
    case 128: return "2D/3D: marching segments of 128 planes per block";
    case 256: return "2D/3D: marching segments of 256 planes per block";
    default: return "2D/3D: marching segments of 512 planes per block";
  }
}

void build_configs(sv_solver* s) {
  s->cfgs.clear();
  if (s->dim == 1) {
    if (s->p.method == SV_HANCOCK &&
        (s->p.precision == SV_FP32 || s->p.precision == SV_FP32_PC ||
         s->p.precision == SV_FP32_PS) &&
        s->ncell >= kTile1dMinCells) {
      s->cfgs.push_back({CFG_TILE, 13,
                         "1D: 512-cell block tiles, 2 cells per thread, 78 registers, 3 blocks/SM"});
      s->cfgs.push_back({CFG_TILE, 12, "1D: 512-cell block tiles, 2 cells per thread, 2 blocks/SM"});
      s->cfgs.push_back({CFG_TILE, 22, "1D: 1024-cell block tiles, 4 cells per thread, 2 blocks/SM"});
      s->cfgs.push_back({CFG_TILE, 14,
                         "1D: 512-cell block tiles, 2 cells per thread, 64 registers, 4 blocks/SM"});
    }
    s->cfgs.push_back({CFG_SLIDE, 0, "1D: warps sliding over 64-cell chunks, 2 cells per thread"});
  } else {
    const int d = stepnd_default_seg(s->dim, s->p.precision);
    s->cfgs.push_back({CFG_ND, d, seg_desc(d)});
    for (int seg : {64, 128, 256, 512})
      if (seg != d) s->cfgs.push_back({CFG_ND, seg, seg_desc(seg)});
  }
}

// Make configuration idx current (host side, outside any capture); the
// captured step graph holds the old kernel, so it is dropped.
int apply_config(sv_solver* s, int idx) {
  const SolverConfig& c = s->cfgs[(size_t)idx];
  int tg = 0;
  if (c.kind == CFG_TILE) {
    tg = tile1d_grid(s->kp, s->p.precision, c.param);
    if (tg < 1) return SV_ECUDA;
  }
  if (s->graph) {
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return SV_ECUDA;
    cudaGraphExecDestroy(s->graph);
    s->graph = nullptr;
  }
  s->config = idx;
  s->tile_grid = tg;
  return SV_OK;
}

int issue_steps(sv_solver* s, int64_t n) {
  if (n <= 0) return SV_OK;
  if (use_loop(s)) {
    while (n > 0) {
      const int64_t m = n < kLoopChunk ? n : kLoopChunk;
      SV_TRY(loop1d_launch(s->p.precision, s->kp, s->buf[0], s->buf[1], s->ctl, s->ncell,
                           s->loop_grid, m, s->stream));
      n -= m;
    }
    return SV_OK;
  }
  if (n >= kGraphLen) {
    int rc = ensure_graph(s);
    if (rc != SV_OK) return rc;
    while (n >= s->graph_len) {
      SV_TRY(cudaGraphLaunch(s->graph, s->stream));
      n -= s->graph_len;
    }
  }
  for (int64_t i = 0; i < n; ++i) SV_TRY(launch_step(s, s->stream));
  return SV_OK;
}

// The device address of page-locked host memory (cudaHostAlloc or
// cudaHostRegister, mapped), or null for any other pointer.
const void* mapped_view(const void* host) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
    cudaGetLastError();                  // not a sticky error: clear it for later checks
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

int read_ctl(sv_solver* s) {
  SV_TRY(cudaMemcpyAsync(s->host_ctl, s->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s->stream));
  SV_TRY(cudaStreamSynchronize(s->stream));
  return SV_OK;
}

int flags_to_status(uint32_t f) {
  if (f & FLAG_STALL) return SV_ESTALL;
  if (f & FLAG_NONPHYS) return SV_ENONPHYS;
  if (f & FLAG_DT) return SV_EDT;
  return SV_OK;
}

// Upload / download of the state in host format H (double, or float).
template <typename H>
int write_state_host(sv_solver* s, const H* host_soa, double t) {
  if (!s || !host_soa) return SV_EINVAL;
  const size_t count = (size_t)s->nf * (size_t)s->ncell;
  // pinned host memory: the conversion kernel reads it over the host link
  // itself (one pass instead of a copy into staging and a second pass); the
  // staging buffer holds count doubles, room for either format
  const H* src = (const H*)mapped_view(host_soa);
  if (!src) {
    SV_TRY(cudaMemcpyAsync(s->staging, host_soa, count * sizeof(H), cudaMemcpyHostToDevice,
                           s->stream));
    src = (const H*)s->staging;
  }
  SV_TRY(ctl_reset_launch(s->ctl, t, s->stream));
  SV_TRY(to_state_launch(s->p.precision, src, s->buf[0], s->buf[1], s->ctl, (int64_t)count,
                         s->stream, s->kp.ref, s->nf));
  SV_TRY(dt_reduce_launch(s->p.precision, s->dim, s->kp, s->buf[0], s->buf[1], s->ctl, s->ncell,
                          s->stream));
  return SV_OK;
}

template <typename H>
int read_state_host(sv_solver* s, H* host_soa, double* t) {
  if (!s || !host_soa) return SV_EINVAL;
  const size_t count = (size_t)s->nf * (size_t)s->ncell;
  // pinned host memory: the conversion kernel writes it over the host link
  H* dst = (H*)mapped_view(host_soa);
  SV_TRY(from_state_launch(s->p.precision, s->buf[0], s->buf[1], s->ctl,
                           dst ? dst : (H*)s->staging, (int64_t)count, s->stream, s->kp.ref,
                           s->nf));
  if (!dst)
    SV_TRY(cudaMemcpyAsync(host_soa, s->staging, count * sizeof(H), cudaMemcpyDeviceToHost,
                           s->stream));
  int rc = read_ctl(s);
  if (rc != SV_OK) return rc;
  if (t) *t = s->host_ctl->t;
  return SV_OK;
}

}  // namespace

extern "C" {

int sv_required_bytes(const sv_params* p, const sv_grid* g, size_t* bytes) {
  int rc = check_inputs(p, g);
  if (rc != SV_OK) return rc;
  if (!bytes) return SV_EINVAL;
  *bytes = layout(p, g).total;
  return SV_OK;
}

int sv_init(const sv_params* p, const sv_grid* g, void* cuda_stream, void* device_mem,
            size_t device_bytes, sv_solver** out) {
  if (!out) return SV_EINVAL;
  *out = nullptr;
  int rc = check_inputs(p, g);
  if (rc != SV_OK) return rc;
  const Layout L = layout(p, g);
  if (device_mem && (device_bytes < L.total || ((uintptr_t)device_mem % kAlign) != 0))
    return SV_ENOMEM;

  sv_solver* s = new (std::nothrow) sv_solver();
  if (!s) return SV_ENOMEM;
  s->p = *p;
  s->g = *g;
  s->dim = g->dim;
  s->nf = g->dim + 3;
  s->esize = p->precision == SV_FP64 ? 8 : 4;
  s->ncell = 1;
  for (int a = 0; a < g->dim; ++a) s->ncell *= g->n[a];
  s->h = g->L[0] / (double)g->n[0];
  s->stream = (cudaStream_t)cuda_stream;

  KParams& k = s->kp;
  k.gamma = p->gamma;
  k.g1 = p->gamma - 1.0;
  k.Ck = p->Ck;
  k.S = p->S;
  k.frozen = isinf(p->tau0) ? 1 : 0;
  k.tau0 = p->tau0;
  k.inv_tau0 = k.frozen ? 0.0 : 1.0 / p->tau0;
  k.Q0 = k.frozen ? 0.0 : p->S / p->tau0;   // S = tau0 Q0 / (R T0), R = T0 = 1
  k.tau_rho = p->tau_rho;
  k.tau_T = p->tau_T;
  k.Q_rho = p->Q_rho;
  k.Q_T = p->Q_T;
  k.I_rho = p->I_rho;
  k.I_T = p->I_T;
  k.qi_zero = (p->Q_rho == 0.0 && p->Q_T == 0.0 && p->I_rho == 0.0 && p->I_T == 0.0) ? 1 : 0;
  k.h = s->h;
  k.cfl = p->cfl;
  k.c_tau = p->c_tau;
  k.limiter = p->limiter;
  k.bc_lo = g->dim <= 2 ? g->bc[0] : SV_BC_PERIODIC;
  k.bc_hi = g->dim <= 2 ? g->bc[1] : SV_BC_PERIODIC;
  k.bc_ylo = g->dim == 2 ? g->bc[2] : SV_BC_PERIODIC;
  k.bc_yhi = g->dim == 2 ? g->bc[3] : SV_BC_PERIODIC;
  k.act_lo = k.act_hi = k.pul_lo = k.pul_hi = nullptr;
  k.pul_omega = k.pul_amp = 0.0;
  k.pul_ev = p->Ck + p->S;
  {   // a driven boundary holds the uniform equilibrium until sv_set_drive
    const double ev0 = p->Ck + p->S;
    const double base[4] = {1.0, 0.0, 1.0 / (p->gamma - 1.0) + ev0, ev0};
    for (int f = 0; f < 4; ++f) k.drv_base[f] = base[f];
  }
  kparams_finish(k);

  if (device_mem) {
    s->mem = device_mem;
  } else {
    if (cudaMalloc(&s->mem, L.total) != cudaSuccess) {
      delete s;
      return SV_ENOMEM;
    }
    s->owns_mem = true;
  }
  char* m = (char*)s->mem;
  s->buf[0] = m;
  s->buf[1] = m + L.state;
  s->staging = (double*)(m + 2 * L.state);
  s->ctl = (Ctl*)(m + 2 * L.state + L.staging);
  s->partial = (double*)(m + 2 * L.state + L.staging + L.ctl);
  s->sums_out = (double*)(m + 2 * L.state + L.staging + L.ctl + L.partial);

  rc = SV_OK;
  if (cudaMallocHost((void**)&s->host_ctl, sizeof(Ctl)) != cudaSuccess ||
      cudaMallocHost((void**)&s->host_sums, 8 * sizeof(double)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    rc = SV_ECUDA;
  if (rc == SV_OK) {
    s->grid = s->dim == 1 ? (p->method == SV_HEUN ? heun1d_grid(s->kp, p->precision)
                                                  : step1d_grid(s->kp, p->precision))
                          : stepnd_grid(s->dim, p->precision, s->kp);
    if (s->grid < 1) rc = SV_ECUDA;
  }
  if (rc == SV_OK) {
    build_configs(s);
    rc = apply_config(s, 0);
  }
  if (rc == SV_OK && s->dim == 1 && p->method == SV_HANCOCK) {
    // 0 where the device has no cooperative launch: the per-step path remains
    int dev = 0, sms = 0, cap = 0;
    s->loop_grid = loop1d_grid(s->kp, p->precision, s->ncell, &cap);
    if (cudaGetDevice(&dev) == cudaSuccess)
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    s->loop_fits = s->loop_grid > 0 && 2 * ((s->ncell + 63) / 64) <= (int64_t)sms;
  }
  if (rc == SV_OK) {
    // uniform equilibrium start: rho = p = 1, v = 0, E_nu = C_k + S
    if (ctl_reset_launch(s->ctl, 0.0, s->stream) != cudaSuccess ||
        fill_equilibrium_launch(s->p.precision, s->buf[0], s->nf, s->ncell, p->gamma,
                                p->Ck + p->S, s->stream) != cudaSuccess ||
        dt_reduce_launch(s->p.precision, s->dim, s->kp, s->buf[0], s->buf[1], s->ctl, s->ncell,
                         s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
      rc = SV_ECUDA;
  }
  if (rc != SV_OK) {
    sv_free(s);
    return rc;
  }
  *out = s;
  return SV_OK;
}

int sv_write_state(sv_solver* s, const double* host_soa, double t) {
  return write_state_host<double>(s, host_soa, t);
}

int sv_read_state(sv_solver* s, double* host_soa, double* t) {
  return read_state_host<double>(s, host_soa, t);
}

int sv_write_state_f32(sv_solver* s, const float* host_soa, double t) {
  return write_state_host<float>(s, host_soa, t);
}

int sv_read_state_f32(sv_solver* s, float* host_soa, double* t) {
  return read_state_host<float>(s, host_soa, t);
}

int sv_dt_cfl(sv_solver* s, double* dt) {
  if (!s || !dt) return SV_EINVAL;
  int rc = read_ctl(s);
  if (rc != SV_OK) return rc;
  *dt = s->host_ctl->dt;
  return SV_OK;
}

int sv_step(sv_solver* s, int64_t nsteps) {
  if (!s || nsteps < 0) return SV_EINVAL;
  return issue_steps(s, nsteps);
}

int sv_run_to(sv_solver* s, double t_end, int64_t max_steps, int64_t* steps_taken) {
  if (!s || max_steps < 0 || isnan(t_end)) return SV_EINVAL;
  SV_TRY(set_target_launch(s->p.precision, s->ctl, t_end, s->kp, s->stream));
  int rc = read_ctl(s);
  if (rc != SV_OK) return rc;
  const int64_t n0 = s->host_ctl->nsteps;
  int64_t issued = 0;
  int status = SV_OK;
  for (;;) {
    const Ctl& c = *s->host_ctl;
    const int64_t done = c.nsteps - n0;
    if (c.flags) { status = flags_to_status(c.flags); break; }
    if (!(c.t < t_end) || !(c.dt > 0.0)) break;
    if (done >= max_steps) { status = SV_EMAXSTEPS; break; }
    // steps still needed at the current dt, bounded by the remaining budget;
    // launches issued after the run ends return at once on the device.
    double est = ceil((t_end - c.t) / (c.dt_cfl > 0.0 ? c.dt_cfl : c.dt));
    if (!(est >= 1.0)) est = 1.0;
    int64_t n = est > 1e15 ? (int64_t)1e15 : (int64_t)est;
    n = n > 4096 ? 4096 : n;
    // the persistent loop stops by itself at t_end: no estimate needed
    if (use_loop(s)) n = kLoopChunk;
    if (n > max_steps - done) n = max_steps - done;
    if (n < 1) n = 1;
    rc = issue_steps(s, n);
    if (rc != SV_OK) return rc;
    issued += n;
    rc = read_ctl(s);
    if (rc != SV_OK) return rc;
  }
  (void)issued;
  if (steps_taken) *steps_taken = s->host_ctl->nsteps - n0;
  // clear the target so that later sv_step calls are not clamped
  SV_TRY(set_target_launch(s->p.precision, s->ctl, INFINITY, s->kp, s->stream));
  return status;
}

int sv_num_configs(sv_solver* s, int* count) {
  if (!s || !count) return SV_EINVAL;
  *count = (int)s->cfgs.size();
  return SV_OK;
}

int sv_get_config(sv_solver* s, int* index, char* desc, size_t cap) {
  if (!s) return SV_EINVAL;
  if (index) *index = s->config;
  if (desc && cap > 0) {
    strncpy(desc, s->cfgs[(size_t)s->config].desc, cap - 1);
    desc[cap - 1] = 0;
  }
  return SV_OK;
}

int sv_config_desc(sv_solver* s, int index, char* desc, size_t cap) {
  if (!s || !desc || cap == 0 || index < 0 || index >= (int)s->cfgs.size()) return SV_EINVAL;
  strncpy(desc, s->cfgs[(size_t)index].desc, cap - 1);
  desc[cap - 1] = 0;
  return SV_OK;
}

int sv_set_config(sv_solver* s, int index) {
  if (!s || index < 0 || index >= (int)s->cfgs.size()) return SV_EINVAL;
  return apply_config(s, index);
}

int sv_autotune(sv_solver* s, int steps, int* best, double* us_per_step) {
  const bool cold = steps < 0;
  if (cold) steps = -steps;
  if (!s || steps < 1) return SV_EINVAL;
  const int ncfg = (int)s->cfgs.size();
  const size_t count = (size_t)s->nf * (size_t)s->ncell;
  // keep the state (a raw copy of the current buffer into the staging area,
  // which holds count doubles) and the control block; every trial is undone
  // before the next one
  Ctl saved;
  const int64_t state_bytes = (int64_t)count * s->esize;
  SV_TRY(raw_state_launch(s->buf[0], s->buf[1], s->ctl, s->staging, state_bytes, true, s->stream));
  SV_TRY(cudaMemcpyAsync(&saved, s->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s->stream));
  SV_TRY(cudaStreamSynchronize(s->stream));
  auto restore = [&]() -> int {
    SV_TRY(cudaMemcpyAsync(s->ctl, &saved, sizeof(Ctl), cudaMemcpyHostToDevice, s->stream));
    SV_TRY(raw_state_launch(s->buf[0], s->buf[1], s->ctl, s->staging, state_bytes, false,
                            s->stream));
    SV_TRY(cudaStreamSynchronize(s->stream));
    return SV_OK;
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return SV_ECUDA;
  }
  // cold trials: an L2-sized write before every timed launch
  constexpr size_t kFlushBytes = size_t(256) << 20;
  void* flush = nullptr;
  if (cold && cudaMalloc(&flush, kFlushBytes) != cudaSuccess) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return SV_ENOMEM;
  }
  const int warm = 2;
  const int start = s->config;
  int pick = start, rc = SV_OK;
  double best_us = INFINITY;
  for (int c = 0; c < ncfg && rc == SV_OK; ++c) {
    double us = INFINITY;
    rc = apply_config(s, c);
    for (int i = 0; i < warm && rc == SV_OK; ++i)
      if (launch_step(s, s->stream) != cudaSuccess) rc = SV_ECUDA;
    float ms = 0.0f;
    if (!cold) {
      if (rc == SV_OK && cudaEventRecord(e0, s->stream) != cudaSuccess) rc = SV_ECUDA;
      for (int i = 0; i < steps && rc == SV_OK; ++i)
        if (launch_step(s, s->stream) != cudaSuccess) rc = SV_ECUDA;
      if (rc == SV_OK && (cudaEventRecord(e1, s->stream) != cudaSuccess ||
                          cudaEventSynchronize(e1) != cudaSuccess ||
                          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        rc = SV_ECUDA;
    } else {
      for (int i = 0; i < steps && rc == SV_OK; ++i) {
        float one = 0.0f;
        if (cudaMemsetAsync(flush, i & 0xff, kFlushBytes, s->stream) != cudaSuccess ||
            cudaEventRecord(e0, s->stream) != cudaSuccess ||
            launch_step(s, s->stream) != cudaSuccess ||
            cudaEventRecord(e1, s->stream) != cudaSuccess ||
            cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&one, e0, e1) != cudaSuccess)
          rc = SV_ECUDA;
        ms += one;
      }
    }
    if (rc == SV_OK) {
      // a trial whose steps stopped (t_end reached, non-physical state) timed
      // nothing useful
      if (rc == SV_OK) rc = read_ctl(s);
      if (rc == SV_OK && s->host_ctl->flags == 0 && s->host_ctl->nsteps == saved.nsteps + warm + steps)
        us = 1e3 * (double)ms / steps;
    }
    if (us_per_step) us_per_step[c] = us;
    if (us < best_us) {
      best_us = us;
      pick = c;
    }
    const int rr = restore();
    if (rc == SV_OK) rc = rr;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (flush) cudaFree(flush);
  const int ra = apply_config(s, rc == SV_OK ? pick : start);
  if (rc == SV_OK) rc = ra;
  if (best) *best = s->config;
  return rc;
}

int sv_set_launch(sv_solver* s, int mode) {
  if (!s || mode < SV_LAUNCH_AUTO || mode > SV_LAUNCH_PERSISTENT) return SV_EINVAL;
  if (mode == SV_LAUNCH_PERSISTENT && s->loop_grid < 1) return SV_EINVAL;
  s->launch = mode;
  return SV_OK;
}

int sv_set_wait_limit(sv_solver* s, int polls) {
  if (!s || polls < 0) return SV_EINVAL;
  s->kp.stall_polls = polls;   // read by the persistent loop only, which is never captured
  return SV_OK;
}

int sv_get_launch(sv_solver* s, int* mode) {
  if (!s || !mode) return SV_EINVAL;
  *mode = use_loop(s) ? SV_LAUNCH_PERSISTENT : SV_LAUNCH_PER_STEP;
  return SV_OK;
}

int sv_set_medium2d(sv_solver* s, const sv_medium2d* m) {
  if (!s || !m || s->dim != 2) return SV_EINVAL;
  const int64_t nx = s->g.n[0], ny = s->g.n[1];
  const int32_t* tab[4] = {m->active_lo, m->active_hi, m->driven_lo, m->driven_hi};
  if ((tab[0] == nullptr) != (tab[1] == nullptr) || (tab[2] == nullptr) != (tab[3] == nullptr))
    return SV_EINVAL;
  for (int t = 0; t < 4; t += 2)
    if (tab[t])
      for (int64_t j = 0; j < ny; ++j)
        if (tab[t][j] < 0 || tab[t][j] > tab[t + 1][j] || tab[t + 1][j] > nx) return SV_EINVAL;
  if (tab[2] && (!isfinite(m->omega) || !isfinite(m->amp))) return SV_EINVAL;
  if (!s->medium_dev && (tab[0] || tab[2])) {
    if (cudaMalloc((void**)&s->medium_dev, sizeof(int) * 4 * (size_t)ny) != cudaSuccess) {
      s->medium_dev = nullptr;
      return SV_ENOMEM;
    }
  }
  // the captured graph and running steps use the old tables
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return SV_ECUDA;
  if (s->graph) {
    cudaGraphExecDestroy(s->graph);
    s->graph = nullptr;
  }
  int* dst[4] = {nullptr, nullptr, nullptr, nullptr};
  for (int t = 0; t < 4; ++t) {
    if (!tab[t]) continue;
    dst[t] = s->medium_dev + (size_t)t * (size_t)ny;
    SV_TRY(cudaMemcpy(dst[t], tab[t], sizeof(int) * (size_t)ny, cudaMemcpyHostToDevice));
  }
  s->kp.act_lo = dst[0];
  s->kp.act_hi = dst[1];
  s->kp.pul_lo = dst[2];
  s->kp.pul_hi = dst[3];
  s->kp.pul_omega = tab[2] ? m->omega : 0.0;
  s->kp.pul_amp = tab[2] ? m->amp : 0.0;
  return SV_OK;
}

int sv_set_drive(sv_solver* s, const sv_drive* d) {
  if (!s || !d || s->dim != 1 || s->kp.bc_lo != SV_BC_DRIVEN) return SV_EINVAL;
  if (!isfinite(d->omega) || !isfinite(d->k_re) || !isfinite(d->k_im)) return SV_EINVAL;
  s->kp.drv_omega = d->omega;
  s->kp.drv_kre = d->k_re;
  s->kp.drv_kim = d->k_im;
  for (int f = 0; f < 4; ++f) {
    s->kp.drv_base[f] = d->base[f];
    s->kp.drv_are[f] = d->amp_re[f];
    s->kp.drv_aim[f] = d->amp_im[f];
  }
  // the captured graph holds the old parameters: capture again on next use
  if (s->graph) {
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return SV_ECUDA;
    cudaGraphExecDestroy(s->graph);
    s->graph = nullptr;
  }
  return SV_OK;
}

int sv_time(sv_solver* s, double* t, int64_t* steps) {
  if (!s) return SV_EINVAL;
  int rc = read_ctl(s);
  if (rc != SV_OK) return rc;
  if (t) *t = s->host_ctl->t;
  if (steps) *steps = s->host_ctl->nsteps;
  return SV_OK;
}

int sv_conservation(sv_solver* s, double* sums) {
  if (!s || !sums) return SV_EINVAL;
  SV_TRY(sums_launch(s->p.precision, s->buf[0], s->buf[1], s->ctl, s->nf, s->ncell, s->partial,
                     sums_blocks(), s->sums_out, s->stream));
  SV_TRY(cudaMemcpyAsync(s->host_sums, s->sums_out, s->nf * sizeof(double), cudaMemcpyDeviceToHost,
                         s->stream));
  SV_TRY(cudaStreamSynchronize(s->stream));
  memcpy(sums, s->host_sums, s->nf * sizeof(double));
  if (s->p.precision == SV_FP32_PS)      // the device holds U - ref
    for (int f = 0; f < s->nf; ++f) sums[f] += (double)s->ncell * ref_field(s->kp.ref, f, s->nf);
  return SV_OK;
}

int sv_status(sv_solver* s, uint32_t* flags) {
  if (!s || !flags) return SV_EINVAL;
  int rc = read_ctl(s);
  if (rc != SV_OK) return rc;
  *flags = s->host_ctl->flags;
  return SV_OK;
}

int sv_state_device(sv_solver* s, void** dev_ptr, int* elem_bytes) {
  if (!s || !dev_ptr) return SV_EINVAL;
  int rc = read_ctl(s);
  if (rc != SV_OK) return rc;
  *dev_ptr = s->buf[s->host_ctl->cur ? 1 : 0];
  if (elem_bytes) *elem_bytes = s->esize;
  return SV_OK;
}

void sv_free(sv_solver* s) {
  if (!s) return;
  if (s->stream || s->mem) cudaStreamSynchronize(s->stream);
  if (s->graph) cudaGraphExecDestroy(s->graph);
  if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
  if (s->owns_mem && s->mem) cudaFree(s->mem);
  if (s->medium_dev) cudaFree(s->medium_dev);
  if (s->host_ctl) cudaFreeHost(s->host_ctl);
  if (s->host_sums) cudaFreeHost(s->host_sums);
  delete s;
}

const char* sv_strerror(int code) {
  switch (code) {
    case SV_OK: return "ok";
    case SV_EINVAL: return "invalid argument";
    case SV_ENOMEM: return "out of device memory or caller block too small";
    case SV_ECUDA: return "CUDA runtime error";
    case SV_ENONPHYS: return "non-physical state (rho <= 0, p <= 0 or non-finite)";
    case SV_EDT: return "time step collapsed";
    case SV_EMAXSTEPS: return "max_steps reached before t_end";
    case SV_ESIZE: return "size beyond the maximum of this entry point";
    case SV_ESTALL: return "a grid-wide wait of the persistent step loop timed out";
    default: return "unknown status";
  }
}

}  // extern "C"
