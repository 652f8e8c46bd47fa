// sv_noalloc.cu -- a 1D step entry point that allocates no memory at all.
//
// The regular solver (sv_init) owns a device block that holds, besides the
// two state buffers, a small control block: time, dt, the eq.-16 reduction
// keys and the completion ticket that the fused step kernel updates.  Some
// callers cannot provide that block through cudaMalloc: processes whose device
// memory is a fixed pool handed out at start-up and that forbid allocation
// afterwards, and hosts that must not allocate on their stepping path (a
// device allocation can synchronise the device and takes unbounded time).
// For them sv_step1d_noalloc takes the state buffers from the caller and
// keeps the control block in the file-scope array below instead.
//
// The array is a static __device__ object: every GPU that loads libsv.so
// holds it (SV_NOALLOC_SCRATCH_BYTES) until the process exits.  Host code
// cannot use its name as a device address; its address is obtained with
// cudaGetSymbolAddress, once per device, the first time the entry point runs
// on that device, together with the launch grid of each step kernel it uses.
#include <mutex>

#include "sv.h"
#include "sv_internal.h"
#include "sv_model.cuh"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[SV_NOALLOC_SCRATCH_BYTES];

static_assert(sizeof(sv::Ctl) <= SV_NOALLOC_SCRATCH_BYTES, "control block must fit the scratch");

constexpr int kMaxDevices = 64;
constexpr int kKernels = 4 * 3 * 3;   // precision (SV_FP32 .. SV_FP32_PC) x limiter x source
std::mutex g_mutex;
void* g_addr[kMaxDevices] = {};
int g_grid[kMaxDevices][kKernels] = {};

// Device address of the scratch array and the persistent grid of the step
// kernel of k on the current device (set-up on the first call per device and
// kernel, with that device current; the kernel's shared-memory attribute is
// set then and stays set).
int setup(const sv::KParams& k, int precision, void** addr, int* grid) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return SV_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return SV_EINVAL;
  const int src = k.frozen ? 0 : (k.qi_zero ? 1 : 2);
  const int kid = (precision * 3 + k.limiter) * 3 + src;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SV_ECUDA;
    g_addr[dev] = p;
  }
  if (g_grid[dev][kid] < 1) {
    const int g = sv::step1d_grid(k, precision);
    if (g < 1) return SV_ECUDA;
    g_grid[dev][kid] = g;
  }
  *addr = g_addr[dev];
  *grid = g_grid[dev][kid];
  return SV_OK;
}

// Whether the byte ranges [a, a + n) and [b, b + n) share a byte.
bool overlap(const void* a, const void* b, uint64_t n) {
  const uint64_t x = (uint64_t)(uintptr_t)a, y = (uint64_t)(uintptr_t)b;
  return x < y ? y - x < n : x - y < n;
}

}  // namespace

extern "C" int sv_step1d_noalloc(const sv_params* p, int64_t n, double L, const void* U_in,
                                 void* U_out, double* dt_used, uint32_t* flags,
                                 void* cuda_stream) {
  using namespace sv;
  if (!p || !U_in || !U_out) return SV_EINVAL;
  if (n > SV_NOALLOC_MAX_CELLS) return SV_ESIZE;
  if (n < 1 || !(L > 0.0)) return SV_EINVAL;
  if (!(p->gamma > 1.0) || !(p->cfl > 0.0) || !(p->c_tau > 0.0) || !(p->tau0 > 0.0) ||
      p->limiter < SV_MINMOD || p->limiter > SV_MC || p->precision < SV_FP32 ||
      p->precision > SV_FP32_PC || p->method != SV_HANCOCK)   // not the perturbation layout
    return SV_EINVAL;
  // the fused step reads U_in's neighbours after other blocks wrote U_out:
  // the two 4 n-element buffers must not share a byte
  const uint64_t span = 4ull * (uint64_t)n * (p->precision == SV_FP64 ? 8u : 4u);
  if (overlap(U_in, U_out, span)) return SV_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;

  KParams k;
  memset(&k, 0, sizeof k);
  k.gamma = p->gamma;
  k.g1 = p->gamma - 1.0;
  k.Ck = p->Ck;
  k.S = p->S;
  k.frozen = isinf(p->tau0) ? 1 : 0;
  k.tau0 = p->tau0;
  k.inv_tau0 = k.frozen ? 0.0 : 1.0 / p->tau0;
  k.Q0 = k.frozen ? 0.0 : p->S / p->tau0;
  k.tau_rho = p->tau_rho;
  k.tau_T = p->tau_T;
  k.Q_rho = p->Q_rho;
  k.Q_T = p->Q_T;
  k.I_rho = p->I_rho;
  k.I_T = p->I_T;
  k.qi_zero = (p->Q_rho == 0.0 && p->Q_T == 0.0 && p->I_rho == 0.0 && p->I_T == 0.0) ? 1 : 0;
  k.h = L / (double)n;
  k.cfl = p->cfl;
  k.c_tau = p->c_tau;
  k.limiter = p->limiter;
  kparams_finish(k);

  void* scratch = nullptr;
  int grid = 0;
  const int rc = setup(k, p->precision, &scratch, &grid);
  if (rc != SV_OK) return rc;
  Ctl* ctl = (Ctl*)scratch;
  // The scratch keeps whatever the previous call left: reset the control block
  // (time 0, ticket 0, reduction keys, flags, current buffer = U_in) first.
  if (ctl_reset_launch(ctl, 0.0, st) != cudaSuccess) return SV_ECUDA;
  // dt of U_in (eq. 16 with the tau cap), then one fused step U_in -> U_out
  if (dt_reduce_launch(p->precision, 1, k, U_in, U_out, ctl, n, st) != cudaSuccess)
    return SV_ECUDA;
  if (step1d_launch(p->precision, k, (void*)U_in, U_out, ctl, n, grid, st) != cudaSuccess)
    return SV_ECUDA;
  if (dt_used || flags) {
    // the step advanced the control block's time from 0 by the dt it took
    double t = 0.0;
    uint32_t f = 0;
    if (cudaMemcpyAsync(&t, &ctl->t, sizeof t, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&f, &ctl->flags, sizeof f, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return SV_ECUDA;
    if (dt_used) *dt_used = t;
    if (flags) *flags = f;
  }
  return SV_OK;
}
