// sv_internal.h -- declarations shared by the host runtime and the kernel
// translation units of libsv.so (not part of the public C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sv {

struct KParams;
struct Ctl;

enum { PREC_FP32 = 0, PREC_FP64 = 1, PREC_FP32_P64 = 2, PREC_FP32_PC = 3, PREC_FP32_PS = 4 };

// A kernel launch; pdl = with the programmatic stream-serialization
// attribute (for kernels that call pdl_wait before reading what the previous
// kernel wrote: the 1D step kernels), as the solver's step graph records them.
inline cudaError_t launch_kernel(const void* fn, dim3 grid, dim3 block, void** args, size_t smem,
                                 cudaStream_t st, bool pdl) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = pdl ? attr : nullptr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

// 1D fused step (sv_step1d.cu)
int step1d_grid(const KParams& kp, int precision);
cudaError_t step1d_launch(int precision, const KParams& kp, void* a, void* b, Ctl* ctl, int64_t N,
                          int grid, cudaStream_t st, bool pdl = false);

// Float 1D MUSCL-Hancock step on block tiles (sv_tile1d.cu), grids of at
// least kTile1dMinCells cells; precision PREC_FP32, PREC_FP32_PC or PREC_FP32_PS
constexpr int64_t kTile1dMinCells = 4096;
// var = 10 * (cell pairs per thread) + (blocks per SM of the register budget):
// 13, 12 or 22
int tile1d_grid(const KParams& kp, int precision, int var);
cudaError_t tile1d_launch(const KParams& kp, int precision, int var, void* a, void* b, Ctl* ctl,
                          int64_t N, int grid, cudaStream_t st, bool pdl = false);

// 1D persistent loop of up to nmax steps (sv_loop1d.cu); grid 0 = unavailable
int loop1d_grid(const KParams& kp, int precision, int64_t N, int* cap);
cudaError_t loop1d_launch(int precision, const KParams& kp, void* a, void* b, Ctl* ctl, int64_t N,
                          int grid, int64_t nmax, cudaStream_t st);

// 1D Heun (SSP-RK2) stages (sv_heun1d.cu); stage 1 or 2
int heun1d_grid(const KParams& kp, int precision);
cudaError_t heun1d_launch(int precision, int stage, const KParams& kp, void* a, void* b, Ctl* ctl,
                          int64_t N, int grid, cudaStream_t st);

// 2D / 3D fused steps (sv_stepnd.cu); n[] cells per axis; seg = planes per
// block along the marching axis (0: default)
int stepnd_grid(int dim, int precision, const KParams& kp);
int stepnd_default_seg(int dim, int precision);
cudaError_t stepnd_launch(int dim, int precision, const KParams& kp, void* a, void* b, Ctl* ctl,
                          const int64_t* n, int seg, cudaStream_t st);
// The float 2D step marching plane pairs (sv_stepnd_pair.cu), precision
// PREC_FP32 or PREC_FP32_PC; n == nullptr sets the kernels' shared-memory limits
int stepnd_pair_default_seg(int dim);
cudaError_t stepnd_pair_launch(int dim, int precision, const KParams& kp, void* a, void* b, Ctl* ctl,
                               const int64_t* n, int seg, cudaStream_t st);

// The float 3D step with the fields in packed pairs (sv_stepnd3f.cu),
// precision PREC_FP32, PREC_FP32_PC or PREC_FP32_PS (the last compiled in
// sv_stepnd3f_ps.cu); n == nullptr sets the kernels' shared-memory limits
int stepnd3f_default_seg();
cudaError_t stepnd3f_launch(int precision, const KParams& kp, void* a, void* b, Ctl* ctl,
                            const int64_t* n, int seg, cudaStream_t st);
cudaError_t stepnd3f_launch_ps(const KParams& kp, void* a, void* b, Ctl* ctl, const int64_t* n,
                               int seg, cudaStream_t st);

// Batched sweep kernels of 256 (sv_batch.cu) and 128 (sv_batch128.cu) threads
void* batch_pick256(int limiter, int precision);
void* batch_pick128(int limiter, int precision);

// Utility kernels (sv_util.cu)
cudaError_t ctl_reset_launch(Ctl* ctl, double t, cudaStream_t st);
cudaError_t dt_reduce_launch(int precision, int dim, const KParams& kp, const void* a,
                             const void* b, Ctl* ctl, int64_t ncell, cudaStream_t st);
cudaError_t set_target_launch(int precision, Ctl* ctl, double t_end, const KParams& kp,
                              cudaStream_t st);
// Host-format (double, full state) <-> device state; `ref` (4 values) is the
// reference state the perturbation layout PREC_FP32_PS subtracts, unused otherwise.
cudaError_t to_state_launch(int precision, const double* src, void* a, void* b, Ctl* ctl,
                            int64_t count, cudaStream_t st, const double* ref = nullptr,
                            int nf = 4);
cudaError_t from_state_launch(int precision, const void* a, const void* b, const Ctl* ctl,
                              double* dst, int64_t count, cudaStream_t st,
                              const double* ref = nullptr, int nf = 4);
// The same with float host-format buffers (sv_write_state_f32 / sv_read_state_f32).
cudaError_t to_state_launch(int precision, const float* src, void* a, void* b, Ctl* ctl,
                            int64_t count, cudaStream_t st, const double* ref, int nf);
cudaError_t from_state_launch(int precision, const void* a, const void* b, const Ctl* ctl,
                              float* dst, int64_t count, cudaStream_t st, const double* ref,
                              int nf);
// Exact copy of the current state buffer's `bytes` to (save) or from `other`.
cudaError_t raw_state_launch(void* a, void* b, const Ctl* ctl, void* other, int64_t bytes,
                             bool save, cudaStream_t st);
cudaError_t sums_launch(int precision, const void* a, const void* b, const Ctl* ctl, int nf,
                        int64_t ncell, double* partial, int nblocks, double* out,
                        cudaStream_t st);
int sums_blocks();
cudaError_t fill_equilibrium_launch(int precision, void* a, int nf, int64_t ncell, double gamma,
                                    double ev0, cudaStream_t st);

}  // namespace sv
