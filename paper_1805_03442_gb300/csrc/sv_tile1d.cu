// sv_tile1d.cu -- the block-tile 1D step (sv_tile1d.cuh): the float-pressure
// kernels and the host entry points tile1d_grid / tile1d_launch.
#include "sv_tile1d.cuh"

namespace sv {

namespace {

void* pick(const KParams& kp, int precision, int var) {
  if (precision == PREC_FP32_PC) return tile1d_pick_pc(kp, var);
  if (precision == PREC_FP32_PS) return tile1d_pick_ps(kp, var);
  return pick_lim<0>(kp, var);
}

}  // namespace

// Sets the kernel's shared-memory limit (host side, outside any capture) and
// returns the persistent grid size of variant `var`, 0 on failure.
int tile1d_grid(const KParams& kp, int precision, int var) {
  int dev = 0, sms = 0, per = 0;
  const void* fn = pick(kp, precision, var);
  const size_t smem = smem_of(var);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads_of(var), smem) != cudaSuccess)
    return 0;
  if (per < 1) per = 1;
  return sms * per;
}

cudaError_t tile1d_launch(const KParams& kp, int precision, int var, void* a, void* b, Ctl* ctl,
                          int64_t N, int grid, cudaStream_t st, bool pdl) {
  if (N >= (1LL << 31) / 4 || N < kTile1dMinCells || grid < 1) return cudaErrorInvalidValue;
  int n32 = (int)N;
  void* args[] = {(void*)&kp, &a, &b, &ctl, &n32};
  return launch_kernel(pick(kp, precision, var), dim3(grid), dim3(threads_of(var)), args,
                       smem_of(var), st, pdl);
}

}  // namespace sv
