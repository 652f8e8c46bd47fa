// sv_step1d.cu -- fused 1D MUSCL-Hancock step (Sec. 2.3: eqs. 13-15 with
// xi = 0, source Y, eq. 16 reduction) for sm_103a.
//
// The per-warp body lives in sv_step1d.cuh; this file holds the single-grid
// persistent kernel and its launcher.
//
// The current buffer and dt are read from the device control block, so the
// same launch can be replayed from a CUDA graph.
#include "sv_internal.h"
#include "sv_step1d.cuh"

namespace sv {

constexpr int NT1 = 256;

template <typename R, int PP, int LIM, int SRC, int MINB>
__global__ void __launch_bounds__(NT1, MINB)
step1d_kernel(const KParams kp, R* __restrict__ bufA, R* __restrict__ bufB, Ctl* __restrict__ ctl,
              int N) {
  pdl_wait();                                     // the previous step's grid has completed
  const StepCtl sc = block_step_ctl(ctl);
  if (!(sc.dt > 0.0)) return;                     // stopped, or t_end reached
  const R* __restrict__ Uin = sc.cur ? bufB : bufA;
  R* __restrict__ Uout = sc.cur ? bufA : bufB;

  const P<R> k(kp);
  const StepDt<R> sd(sc);
  const R dt = sd.dt, dtdx = sd.dtdx, dt_2h = sd.dt_2h, dt_2 = sd.dt_2;
  extern __shared__ __align__(16) unsigned char smem1d[];   // per-warp rings
  R* ring = reinterpret_cast<R*>(smem1d) + (threadIdx.x >> 5) * (ring1d_bytes<R>() / sizeof(R));

  const int lane = threadIdx.x & 31;
  const int nwarps = gridDim.x * (NT1 / 32);
  const int warp = blockIdx.x * (NT1 / 32) + (threadIdx.x >> 5);
  const int nchunk = (N + 63) / 64;
  const int c0 = (int)((int64_t)warp * nchunk / nwarps);
  const int c1 = (int)((int64_t)(warp + 1) * nchunk / nwarps);

  R smax = 0, akey = -INFINITY;
  uint32_t flags = 0;

  step1d_warp<R, PP, LIM, SRC>(k, Uin, Uout, N, N, c0, c1, lane, dt, dtdx, dt_2h, dt_2, smax, akey,
                               flags, ring, kp, sc.t);
  pdl_trigger();                                  // the next step may launch and wait
  reduce_and_finalize<R, NT1>(ctl, kp, smax, akey, flags, true);
}

// Kernel variants: arithmetic (float / double / float with double or
// compensated-float pressure),
// limiter and source kind are compile-time; one of them is chosen per solver.
template <typename R, int PP, int LIM, int SRC>
struct K1 {
  static constexpr int MINB = sizeof(R) == 8 ? 1 : 2;
  static constexpr auto fn = step1d_kernel<R, PP, LIM, SRC, MINB>;
};

template <int LIM, int SRC>
static void* pick_prec(int precision) {
  switch (precision) {
    case PREC_FP64: return (void*)K1<double, 0, LIM, SRC>::fn;
    case PREC_FP32_P64: return (void*)K1<float, 1, LIM, SRC>::fn;
    case PREC_FP32_PC: return (void*)K1<float, 2, LIM, SRC>::fn;
    case PREC_FP32_PS: return (void*)K1<float, 3, LIM, SRC>::fn;
    default: return (void*)K1<float, 0, LIM, SRC>::fn;
  }
}

template <int LIM>
static void* pick_src(int precision, int src) {
  switch (src) {
    case 0: return pick_prec<LIM, 0>(precision);
    case 1: return pick_prec<LIM, 1>(precision);
    default: return pick_prec<LIM, 2>(precision);
  }
}

static void* pick(const KParams& kp, int precision) {
  const int src = kp.frozen ? 0 : (kp.qi_zero ? 1 : 2);
  switch (kp.limiter) {
    case 1: return pick_src<1>(precision, src);
    case 2: return pick_src<2>(precision, src);
    default: return pick_src<0>(precision, src);
  }
}

static size_t smem_bytes(int precision) {
  return (size_t)(NT1 / 32) * (precision == PREC_FP64 ? ring1d_bytes<double>() : ring1d_bytes<float>());
}

// Sets the kernel's dynamic shared-memory limit (host side, outside any stream
// capture) and returns the persistent grid size.
int step1d_grid(const KParams& kp, int precision) {
  int dev = 0, sms = 0, per = 0;
  const void* fn = pick(kp, precision);
  const size_t smem = smem_bytes(precision);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, NT1, smem);
  if (per < 1) per = 1;
  return sms * per;
}

cudaError_t step1d_launch(int precision, const KParams& kp, void* a, void* b, Ctl* ctl, int64_t N,
                          int grid, cudaStream_t st, bool pdl) {
  if (N >= (1LL << 31) / 4) return cudaErrorInvalidValue;
  int n32 = (int)N;
  void* args[] = {(void*)&kp, &a, &b, &ctl, &n32};
  return launch_kernel(pick(kp, precision), dim3(grid), dim3(NT1), args, smem_bytes(precision), st,
                       pdl);
}

}  // namespace sv
