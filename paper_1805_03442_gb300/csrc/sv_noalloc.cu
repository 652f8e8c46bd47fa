// sv_noalloc.cu -- a 1D step entry point that allocates no memory at all.
//
// The regular solver (sv_init) owns a device block that holds, besides the
// two state buffers, a small control block: time, dt, the eq.-16 reduction
// keys and the completion ticket that the fused step kernel updates.  Some
// callers cannot provide that block through cudaMalloc -- code that runs
// inside another framework's CUDA graph capture (where allocation is not
// allowed), processes with a fixed memory pool that forbids allocation after
// start-up, or hosts that must not allocate on their stepping path.  For
// them sv_step1d_noalloc takes the state buffers from the caller and keeps
// the control block in the file-scope array below instead.
//
// The array is a static __device__ object: every GPU that loads libsv.so
// holds it (SV_NOALLOC_SCRATCH_BYTES) until the process exits.  Host code
// cannot use its name as a device address; its address is obtained with
// cudaGetSymbolAddress, once per device, the first time the entry point runs
// on that device.
#include <mutex>

#include "sv.h"
#include "sv_internal.h"
#include "sv_model.cuh"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[SV_NOALLOC_SCRATCH_BYTES];

static_assert(sizeof(sv::Ctl) <= SV_NOALLOC_SCRATCH_BYTES, "control block must fit the scratch");

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set-up on the
// first call per device, with that device current).
int scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return SV_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return SV_EINVAL;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SV_ECUDA;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return SV_OK;
}

}  // namespace

extern "C" int sv_step1d_noalloc(const sv_params* p, int64_t n, double L, const void* U_in,
                                 void* U_out, double* dt_used, uint32_t* flags,
                                 void* cuda_stream) {
  using namespace sv;
  if (!p || !U_in || !U_out || U_in == U_out) return SV_EINVAL;
  if (n > SV_NOALLOC_MAX_CELLS) return SV_ESIZE;
  if (n < 1 || !(L > 0.0)) return SV_EINVAL;
  if (!(p->gamma > 1.0) || !(p->cfl > 0.0) || !(p->c_tau > 0.0) || !(p->tau0 > 0.0) ||
      p->limiter < SV_MINMOD || p->limiter > SV_MC || p->precision < SV_FP32 ||
      p->precision > SV_FP32_PC || p->method != SV_HANCOCK)   // not the perturbation layout
    return SV_EINVAL;
  void* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc != SV_OK) return rc;
  Ctl* ctl = (Ctl*)scratch;
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

  // The scratch keeps whatever the previous call left: reset the control block
  // (time 0, ticket 0, reduction keys, flags, current buffer = U_in) first.
  const int grid = step1d_grid(k, p->precision);
  if (grid < 1) return SV_ECUDA;
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
