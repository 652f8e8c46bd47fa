// sv_util.cu -- small kernels of the runtime: control-block reset, the
// eq.-16 dt reduction of an uploaded state, the t_end clamp, host I/O
// conversion and the compensated conservation sums.
#include "sv_internal.h"
#include "sv_reduce.cuh"
#include "sv_pertnd.cuh"

namespace sv {

constexpr int NTU = 256;

__global__ void ctl_reset_kernel(Ctl* ctl, double t) {
  ctl->t = t;
  clear_step_dt(ctl);
  ctl->dt_cfl = 0.0;
  ctl->t_end = INFINITY;
  ctl->nsteps = 0;
  ctl->cur = 0;
  ctl->last = 0;
  ctl->flags = 0;
  ctl->ticket = 0;
  ctl->smax_key = key_of(0.0);
  ctl->tau_key = key_of(-INFINITY);
}

cudaError_t ctl_reset_launch(Ctl* ctl, double t, cudaStream_t st) {
  ctl_reset_kernel<<<1, 1, 0, st>>>(ctl, t);
  return cudaGetLastError();
}

// Sets the target time and re-clamps the pending dt (same rule as the
// step finalize: the step that would reach or pass t_end lands on it).
template <typename R>
__global__ void set_target_kernel(Ctl* ctl, double t_end, const KParams kp) {
  const double t = ctl->t, dt = ctl->dt_cfl;
  ctl->t_end = t_end;
  uint32_t last = 0;
  double dtn = dt;
  if (ctl->flags || !(t < t_end)) {
    dtn = 0.0;
  } else if (dt >= t_end - t) {
    dtn = t_end - t;
    last = 1;
  }
  set_step_dt<R>(ctl, dtn, kp);
  ctl->last = last;
}

cudaError_t set_target_launch(int precision, Ctl* ctl, double t_end, const KParams& kp,
                              cudaStream_t st) {
  if (precision == PREC_FP64)
    set_target_kernel<double><<<1, 1, 0, st>>>(ctl, t_end, kp);
  else
    set_target_kernel<float><<<1, 1, 0, st>>>(ctl, t_end, kp);
  return cudaGetLastError();
}

// dt of the current state (no step): same per-cell bound and finalize as the
// step kernels.
template <typename R, int PP>
__global__ void __launch_bounds__(NTU) dt_reduce_kernel(const KParams kp, const R* a, const R* b,
                                                        Ctl* ctl, int dim, int64_t ncell) {
  const R* U = vload(&ctl->cur) ? b : a;
  const P<R> k(kp);
  R smax = 0, akey = -INFINITY;
  uint32_t flags = 0;
  if constexpr (PP == 3) {        // perturbation layout
    for (int64_t i = (int64_t)blockIdx.x * NTU + threadIdx.x; i < ncell;
         i += (int64_t)gridDim.x * NTU) {
      if (dim == 1) {
        const R u[4] = {U[i], U[ncell + i], U[2 * ncell + i], U[3 * ncell + i]};
        cell_bound<R, 3, 1>(k, u, smax, akey, flags);
      } else if (dim == 2) {
        float u[5];
        for (int f = 0; f < 5; ++f) u[f] = U[f * ncell + i];
        psn::bound<2, 1>(k, u, smax, akey, flags);
      } else {
        float u[6];
        for (int f = 0; f < 6; ++f) u[f] = U[f * ncell + i];
        psn::bound<3, 1>(k, u, smax, akey, flags);
      }
    }
    reduce_and_finalize<R, NTU>(ctl, kp, smax, akey, flags, false);
    return;
  }
  for (int64_t i = (int64_t)blockIdx.x * NTU + threadIdx.x; i < ncell;
       i += (int64_t)gridDim.x * NTU) {
    const R rho = U[i];
    const R ir = Ar<R>::rcp(rho);
    R kin2 = 0, v2 = 0;
    for (int d = 0; d < dim; ++d) {
      const R m = U[(1 + d) * ncell + i], v = m * ir;
      kin2 += m * v;
      v2 += v * v;
    }
    const R vmag = dim == 1 ? fabs(U[ncell + i] * ir) : speed_of<R>(v2);
    cfl_cell<R, PP, 1>(k, rho, kin2, vmag, U[(1 + dim) * ncell + i], U[(2 + dim) * ncell + i],
                       smax, akey, flags);
  }
  reduce_and_finalize<R, NTU>(ctl, kp, smax, akey, flags, false);
}

static int grid_small(int64_t count) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t g = (count + NTU - 1) / NTU;
  if (g > 4LL * sms) g = 4LL * sms;
  return g < 1 ? 1 : (int)g;
}

cudaError_t dt_reduce_launch(int precision, int dim, const KParams& kp, const void* a,
                             const void* b, Ctl* ctl, int64_t ncell, cudaStream_t st) {
  const int g = grid_small(ncell);
  switch (precision) {
    case PREC_FP64:
      dt_reduce_kernel<double, 0><<<g, NTU, 0, st>>>(kp, (const double*)a, (const double*)b, ctl,
                                                     dim, ncell);
      break;
    case PREC_FP32_P64:
      dt_reduce_kernel<float, 1><<<g, NTU, 0, st>>>(kp, (const float*)a, (const float*)b, ctl,
                                                    dim, ncell);
      break;
    case PREC_FP32_PC:
      dt_reduce_kernel<float, 2><<<g, NTU, 0, st>>>(kp, (const float*)a, (const float*)b, ctl,
                                                    dim, ncell);
      break;
    case PREC_FP32_PS:
      dt_reduce_kernel<float, 3><<<g, NTU, 0, st>>>(kp, (const float*)a, (const float*)b, ctl,
                                                    dim, ncell);
      break;
    default:
      dt_reduce_kernel<float, 0><<<g, NTU, 0, st>>>(kp, (const float*)a, (const float*)b, ctl,
                                                    dim, ncell);
  }
  return cudaGetLastError();
}

// Host-format (double) <-> state conversion.  `src` / `dst` is a device
// staging buffer or the device view of mapped pinned host memory (then the
// kernel itself moves the bytes over the host link).  Pairs of elements go as
// one 16-byte double2 access where both sides are aligned for it.
template <typename R> struct Vec2;
template <> struct Vec2<float> { using T = float2; };
template <> struct Vec2<double> { using T = double2; };

template <typename H, typename R>
__global__ void to_state_kernel(const H* src, R* a, R* b, const Ctl* ctl, int64_t count) {
  R* U = vload(&ctl->cur) ? b : a;
  using R2 = typename Vec2<R>::T;
  using H2 = typename Vec2<H>::T;
  const int64_t i0 = (int64_t)blockIdx.x * NTU + threadIdx.x, di = (int64_t)gridDim.x * NTU;
  if (((uintptr_t)src & (sizeof(H2) - 1)) == 0 && ((uintptr_t)U & (sizeof(R2) - 1)) == 0) {
    const int64_t n2 = count / 2;
    for (int64_t i = i0; i < n2; i += di) {
      const H2 v = reinterpret_cast<const H2*>(src)[i];
      R2 w;
      w.x = (R)v.x;
      w.y = (R)v.y;
      reinterpret_cast<R2*>(U)[i] = w;
    }
    if (i0 == 0 && (count & 1)) U[count - 1] = (R)src[count - 1];
  } else {
    for (int64_t i = i0; i < count; i += di) U[i] = (R)src[i];
  }
}

template <typename H, typename R>
__global__ void from_state_kernel(const R* a, const R* b, const Ctl* ctl, H* dst, int64_t count) {
  const R* U = vload(&ctl->cur) ? b : a;
  using R2 = typename Vec2<R>::T;
  using H2 = typename Vec2<H>::T;
  const int64_t i0 = (int64_t)blockIdx.x * NTU + threadIdx.x, di = (int64_t)gridDim.x * NTU;
  if (((uintptr_t)dst & (sizeof(H2) - 1)) == 0 && ((uintptr_t)U & (sizeof(R2) - 1)) == 0) {
    const int64_t n2 = count / 2;
    for (int64_t i = i0; i < n2; i += di) {
      const R2 w = reinterpret_cast<const R2*>(U)[i];
      H2 v;
      v.x = (H)w.x;
      v.y = (H)w.y;
      reinterpret_cast<H2*>(dst)[i] = v;
    }
    if (i0 == 0 && (count & 1)) dst[count - 1] = (H)U[count - 1];
  } else {
    for (int64_t i = i0; i < count; i += di) dst[i] = (H)U[i];
  }
}

// The perturbation layout (SV_FP32_PS): element i of field f = i / ncell holds
// (float)(U - ref[f]) (the difference taken in double); nf = 4, 5 or 6 fields.
struct RefN {
  double v[6];
};

RefN ref_of(const double* ref, int nf) {
  RefN r{};
  const double four[4] = {ref[0], ref[1], ref[2], ref[3]};
  for (int f = 0; f < nf; ++f) r.v[f] = ref_field(four, f, nf);
  return r;
}

template <typename H>
__global__ void to_state_ps_kernel(const H* src, float* a, float* b, const Ctl* ctl,
                                   int64_t count, int64_t ncell, RefN ref) {
  float* U = vload(&ctl->cur) ? b : a;
  for (int64_t i = (int64_t)blockIdx.x * NTU + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * NTU)
    U[i] = (float)((double)src[i] - ref.v[i / ncell]);
}

template <typename H>
__global__ void from_state_ps_kernel(const float* a, const float* b, const Ctl* ctl, H* dst,
                                     int64_t count, int64_t ncell, RefN ref) {
  const float* U = vload(&ctl->cur) ? b : a;
  for (int64_t i = (int64_t)blockIdx.x * NTU + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * NTU)
    dst[i] = (H)(ref.v[i / ncell] + (double)U[i]);
}

// Raw copies of the current state buffer (`words` 4-byte words) to / from
// `other` (the autotuner's exact save and restore).
__global__ void raw_state_kernel(uint32_t* a, uint32_t* b, const Ctl* ctl, uint32_t* other,
                                 int64_t words, bool save) {
  uint32_t* U = vload(&ctl->cur) ? b : a;
  for (int64_t i = (int64_t)blockIdx.x * NTU + threadIdx.x; i < words;
       i += (int64_t)gridDim.x * NTU) {
    if (save) other[i] = U[i];
    else U[i] = other[i];
  }
}

cudaError_t raw_state_launch(void* a, void* b, const Ctl* ctl, void* other, int64_t bytes,
                             bool save, cudaStream_t st) {
  const int64_t words = bytes / 4;
  raw_state_kernel<<<grid_small(words), NTU, 0, st>>>((uint32_t*)a, (uint32_t*)b, ctl,
                                                      (uint32_t*)other, words, save);
  return cudaGetLastError();
}

template <typename H>
cudaError_t to_state_impl(int precision, const H* src, void* a, void* b, Ctl* ctl, int64_t count,
                          cudaStream_t st, const double* ref, int nf) {
  const int g = grid_small(count);
  if (precision == PREC_FP32_PS) {
    to_state_ps_kernel<H><<<g, NTU, 0, st>>>(src, (float*)a, (float*)b, ctl, count, count / nf,
                                             ref_of(ref, nf));
    return cudaGetLastError();
  }
  if (precision == PREC_FP64)
    to_state_kernel<H, double><<<g, NTU, 0, st>>>(src, (double*)a, (double*)b, ctl, count);
  else
    to_state_kernel<H, float><<<g, NTU, 0, st>>>(src, (float*)a, (float*)b, ctl, count);
  return cudaGetLastError();
}

template <typename H>
cudaError_t from_state_impl(int precision, const void* a, const void* b, const Ctl* ctl, H* dst,
                            int64_t count, cudaStream_t st, const double* ref, int nf) {
  const int g = grid_small(count);
  if (precision == PREC_FP32_PS) {
    from_state_ps_kernel<H><<<g, NTU, 0, st>>>((const float*)a, (const float*)b, ctl, dst, count,
                                               count / nf, ref_of(ref, nf));
    return cudaGetLastError();
  }
  if (precision == PREC_FP64)
    from_state_kernel<H, double><<<g, NTU, 0, st>>>((const double*)a, (const double*)b, ctl, dst,
                                                    count);
  else
    from_state_kernel<H, float><<<g, NTU, 0, st>>>((const float*)a, (const float*)b, ctl, dst,
                                                   count);
  return cudaGetLastError();
}

cudaError_t to_state_launch(int precision, const double* src, void* a, void* b, Ctl* ctl,
                            int64_t count, cudaStream_t st, const double* ref, int nf) {
  return to_state_impl<double>(precision, src, a, b, ctl, count, st, ref, nf);
}
cudaError_t to_state_launch(int precision, const float* src, void* a, void* b, Ctl* ctl,
                            int64_t count, cudaStream_t st, const double* ref, int nf) {
  return to_state_impl<float>(precision, src, a, b, ctl, count, st, ref, nf);
}
cudaError_t from_state_launch(int precision, const void* a, const void* b, const Ctl* ctl,
                              double* dst, int64_t count, cudaStream_t st, const double* ref,
                              int nf) {
  return from_state_impl<double>(precision, a, b, ctl, dst, count, st, ref, nf);
}
cudaError_t from_state_launch(int precision, const void* a, const void* b, const Ctl* ctl,
                              float* dst, int64_t count, cudaStream_t st, const double* ref,
                              int nf) {
  return from_state_impl<float>(precision, a, b, ctl, dst, count, st, ref, nf);
}

// Uniform equilibrium rho = p = 1, v = 0, E_nu = ev0 into buffer a.
template <typename R>
__global__ void fill_equilibrium_kernel(R* a, int nf, int64_t ncell, double gamma, double ev0) {
  for (int64_t i = (int64_t)blockIdx.x * NTU + threadIdx.x; i < (int64_t)nf * ncell;
       i += (int64_t)gridDim.x * NTU) {
    const int f = (int)(i / ncell);
    double v = 0.0;
    if (f == 0) v = 1.0;
    else if (f == nf - 2) v = 1.0 / (gamma - 1.0) + ev0;
    else if (f == nf - 1) v = ev0;
    a[i] = (R)v;
  }
}

cudaError_t fill_equilibrium_launch(int precision, void* a, int nf, int64_t ncell, double gamma,
                                    double ev0, cudaStream_t st) {
  const int g = grid_small((int64_t)nf * ncell);
  if (precision == PREC_FP32_PS)      // the equilibrium is the layout's reference: all zero
    return cudaMemsetAsync(a, 0, sizeof(float) * (size_t)nf * (size_t)ncell, st);
  if (precision == PREC_FP64)
    fill_equilibrium_kernel<double><<<g, NTU, 0, st>>>((double*)a, nf, ncell, gamma, ev0);
  else
    fill_equilibrium_kernel<float><<<g, NTU, 0, st>>>((float*)a, nf, ncell, gamma, ev0);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- sums

// Neumaier compensated addition of x into (s, c).
__device__ __forceinline__ void neumaier(double& s, double& c, double x) {
  const double t = s + x;
  if (fabs(s) >= fabs(x)) c += (s - t) + x;
  else c += (x - t) + s;
  s = t;
}

constexpr int SUM_BLOCKS = 512;
int sums_blocks() { return SUM_BLOCKS; }

// Pass 1: per block and field, a compensated partial (sum, compensation).
template <typename R>
__global__ void __launch_bounds__(NTU) sums_kernel(const R* a, const R* b, const Ctl* ctl, int nf,
                                                   int64_t ncell, double* partial) {
  const R* U = vload(&ctl->cur) ? b : a;
  __shared__ double sh_s[NTU], sh_c[NTU];
  for (int f = 0; f < nf; ++f) {
    double s = 0.0, c = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * NTU + threadIdx.x; i < ncell;
         i += (int64_t)gridDim.x * NTU)
      neumaier(s, c, (double)U[f * ncell + i]);
    sh_s[threadIdx.x] = s;
    sh_c[threadIdx.x] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
      double S = 0.0, C = 0.0;
      for (int i = 0; i < NTU; ++i) {
        neumaier(S, C, sh_s[i]);
        C += sh_c[i];
      }
      partial[(blockIdx.x * nf + f) * 2 + 0] = S;
      partial[(blockIdx.x * nf + f) * 2 + 1] = C;
    }
    __syncthreads();
  }
}

// Pass 2: fold the block partials (one thread per field).
__global__ void sums_fold_kernel(const double* partial, int nblocks, int nf, double* out) {
  const int f = threadIdx.x;
  if (f >= nf) return;
  double S = 0.0, C = 0.0;
  for (int bk = 0; bk < nblocks; ++bk) {
    neumaier(S, C, partial[(bk * nf + f) * 2 + 0]);
    C += partial[(bk * nf + f) * 2 + 1];
  }
  out[f] = S + C;
}

cudaError_t sums_launch(int precision, const void* a, const void* b, const Ctl* ctl, int nf,
                        int64_t ncell, double* partial, int nblocks, double* out,
                        cudaStream_t st) {
  if (precision == PREC_FP64)
    sums_kernel<double><<<nblocks, NTU, 0, st>>>((const double*)a, (const double*)b, ctl, nf,
                                                 ncell, partial);
  else
    sums_kernel<float><<<nblocks, NTU, 0, st>>>((const float*)a, (const float*)b, ctl, nf, ncell,
                                                partial);
  sums_fold_kernel<<<1, 32, 0, st>>>(partial, nblocks, nf, out);
  return cudaGetLastError();
}

}  // namespace sv
