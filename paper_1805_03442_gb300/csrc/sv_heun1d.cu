// sv_heun1d.cu -- Heun (SSP-RK2) time integration of the 1D MUSCL operator:
// the two-stage predictor-corrector of eqs. 10-11 applied to the whole
// spatial operator L (flux divergence of eq. 13 faces between the eq. 14
// states at the stage's own time level, plus the source Y):
//   stage 1:  U*      = U^n + dt L(U^n)                 (into the other buffer)
//   stage 2:  U^{n+1} = (U^n + U*) / 2 + dt/2 L(U*)     (in place over U^n)
// Two launches per step with the per-warp body of sv_step1d.cuh; the second
// folds the next dt and advances the time without flipping the buffers.
#include "sv_internal.h"
#include "sv_step1d.cuh"

namespace sv {

constexpr int NTH = 256;

template <typename R, int PP, int LIM, int SRC, int MODE, int MINB>
__global__ void __launch_bounds__(NTH, MINB)
heun1d_kernel(const KParams kp, R* __restrict__ bufA, R* __restrict__ bufB, Ctl* __restrict__ ctl,
              int N) {
  const StepCtl sc = block_step_ctl(ctl);
  if (!(sc.dt > 0.0)) return;
  R* Un = sc.cur ? bufB : bufA;     // U^n (and U^{n+1} after stage 2)
  R* Us = sc.cur ? bufA : bufB;     // U*
  const R* Uin = MODE == MODE_HEUN1 ? Un : Us;
  R* Uout = MODE == MODE_HEUN1 ? Us : Un;

  const P<R> k(kp);
  const StepDt<R> sd(sc);
  extern __shared__ __align__(16) unsigned char smemh[];
  R* ring = reinterpret_cast<R*>(smemh) + (threadIdx.x >> 5) * (ring1d_bytes<R>() / sizeof(R));

  const int lane = threadIdx.x & 31;
  const int nwarps = gridDim.x * (NTH / 32);
  const int warp = blockIdx.x * (NTH / 32) + (threadIdx.x >> 5);
  const int nchunk = (N + 63) / 64;
  const int c0 = (int)((int64_t)warp * nchunk / nwarps);
  const int c1 = (int)((int64_t)(warp + 1) * nchunk / nwarps);
  R smax = 0, akey = -INFINITY;
  uint32_t flags = 0;
  step1d_warp<R, PP, LIM, SRC, MODE>(k, Uin, Uout, N, N, c0, c1, lane, sd.dt, sd.dtdx, sd.dt_2h,
                                     sd.dt_2, smax, akey, flags, ring, kp, sc.t, Un);
  if (MODE == MODE_HEUN2)
    reduce_and_finalize<R, NTH>(ctl, kp, smax, akey, flags, true, false);
}

template <typename R, int LIM, int SRC, int MODE>
struct KH {
  static constexpr auto fn = heun1d_kernel<R, 0, LIM, SRC, MODE, sizeof(R) == 8 ? 1 : 2>;
};

template <int LIM, int SRC, int MODE>
static void* hpick_prec(int precision) {
  return precision == PREC_FP64 ? (void*)KH<double, LIM, SRC, MODE>::fn
                                : (void*)KH<float, LIM, SRC, MODE>::fn;
}
template <int LIM, int MODE>
static void* hpick_src(int precision, int src) {
  switch (src) {
    case 0: return hpick_prec<LIM, 0, MODE>(precision);
    case 1: return hpick_prec<LIM, 1, MODE>(precision);
    default: return hpick_prec<LIM, 2, MODE>(precision);
  }
}
template <int MODE>
static void* hpick_lim(const KParams& kp, int precision) {
  const int src = kp.frozen ? 0 : (kp.qi_zero ? 1 : 2);
  switch (kp.limiter) {
    case 1: return hpick_src<1, MODE>(precision, src);
    case 2: return hpick_src<2, MODE>(precision, src);
    default: return hpick_src<0, MODE>(precision, src);
  }
}
static void* hpick(const KParams& kp, int precision, int stage) {
  return stage == 1 ? hpick_lim<MODE_HEUN1>(kp, precision) : hpick_lim<MODE_HEUN2>(kp, precision);
}

static size_t hsmem(int precision) {
  return (size_t)(NTH / 32) * (precision == PREC_FP64 ? ring1d_bytes<double>() : ring1d_bytes<float>());
}

int heun1d_grid(const KParams& kp, int precision) {
  int dev = 0, sms = 0, per = 0, per2 = 0;
  const size_t smem = hsmem(precision);
  for (int stage = 1; stage <= 2; ++stage)
    if (cudaFuncSetAttribute(hpick(kp, precision, stage), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
      return 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, hpick(kp, precision, 1), NTH, smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per2, hpick(kp, precision, 2), NTH, smem);
  if (per2 < per) per = per2;
  if (per < 1) per = 1;
  return sms * per;
}

cudaError_t heun1d_launch(int precision, int stage, const KParams& kp, void* a, void* b, Ctl* ctl,
                          int64_t N, int grid, cudaStream_t st) {
  if (N >= (1LL << 31) / 4) return cudaErrorInvalidValue;
  int n32 = (int)N;
  void* args[] = {(void*)&kp, &a, &b, &ctl, &n32};
  return cudaLaunchKernel(hpick(kp, precision, stage), dim3(grid), dim3(NTH), args, hsmem(precision),
                          st);
}

}  // namespace sv
