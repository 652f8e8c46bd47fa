// sv_loop1d.cu -- many 1D MUSCL-Hancock steps (Sec. 2.3: eqs. 13-15 with
// xi = 0, source Y, eq. 16 reduction) in one persistent launch.
//
// On the grids of the paper's own experiments (a few hundred to 10^5 cells)
// one step is a chain of latencies -- loading a chunk, three sliding
// iterations of one warp, the block fold and the serial dt finalize -- rather
// than a throughput problem, and a kernel boundary per step adds to it.  This
// kernel keeps its blocks resident for a whole run of steps instead:
//   - every block computes its chunks of the step with the same per-warp body
//     as the one-step kernel (sv_step1d.cuh), so each cell gets the same
//     operations in the same order and the results are bitwise equal;
//   - every block folds its dt bounds into the control block and takes a
//     ticket; the last block to arrive turns the maxima into the next dt,
//     advances t, flips the buffers (finalize) and then bumps the barrier
//     generation; the other blocks wait for that bump before the next step.
// Co-residency of all blocks is guaranteed by a cooperative launch.  Each wait
// is bounded in time: a block that gives up raises FLAG_STALL (which stops the
// run on the next finalize) and leaves the loop, so a broken barrier ends the
// launch with an error status instead of hanging it.
#include "sv_internal.h"
#include "sv_step1d.cuh"

namespace sv {

namespace {

constexpr int NTL = 256;
constexpr uint64_t kStallNs = 2000000000ull;   // give up a barrier wait after 2 s
constexpr uint32_t kStallIters = 1u << 24;      // ... or after this many polls

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait (one thread) until the barrier generation moves past gen0.  Returns
// false if the wait ran out: after `polls` polls (0: kStallIters) or kStallNs.
__device__ bool wait_generation(Ctl* ctl, uint32_t gen0, int polls) {
  const uint64_t t0 = globaltimer();
  const uint32_t limit = polls > 0 ? (uint32_t)polls : kStallIters;
  for (uint32_t it = 0; it < limit; ++it) {
    if (ld_acquire(&ctl->gen) != gen0) {
      __threadfence();
      return true;
    }
    if (it >= 256) {
      __nanosleep(64);
      if ((it & 255) == 0 && globaltimer() - t0 > kStallNs) break;
    }
  }
  atomicOr(&ctl->flags, FLAG_STALL);
  return false;
}

// Up to nmax steps; stops early once the device-side dt is 0 (t_end reached or
// a flag raised).  bufA / bufB alternate as input and output from step to step.
template <typename R, int PP, int LIM, int SRC, int MINB>
__global__ void __launch_bounds__(NTL, MINB)
loop1d_kernel(const KParams kp, R* bufA, R* bufB, Ctl* ctl, int N, long long nmax) {
  extern __shared__ __align__(16) unsigned char smem1d[];   // per-warp rings
  R* ring = reinterpret_cast<R*>(smem1d) + (threadIdx.x >> 5) * (ring1d_bytes<R>() / sizeof(R));
  __shared__ int s_stop;

  const P<R> k(kp);
  const int lane = threadIdx.x & 31;
  const int nwarps = gridDim.x * (NTL / 32);
  const int warp = blockIdx.x * (NTL / 32) + (threadIdx.x >> 5);
  const int nchunk = (N + 63) / 64;
  const int c0 = (int)((int64_t)warp * nchunk / nwarps);
  const int c1 = (int)((int64_t)(warp + 1) * nchunk / nwarps);

  for (long long s = 0; s < nmax; ++s) {
    // ctl changes only inside the barrier below: every block sees the same
    // dt here and leaves the loop at the same step.
    const StepCtl sc = block_step_ctl(ctl);
    if (!(sc.dt > 0.0)) break;
    const uint32_t gen0 = sc.gen;
    const R* Uin = sc.cur ? bufB : bufA;
    R* Uout = sc.cur ? bufA : bufB;
    const StepDt<R> sd(sc);
    R smax = 0, akey = -INFINITY;
    uint32_t flags = 0;
    step1d_warp<R, PP, LIM, SRC>(k, Uin, Uout, N, N, c0, c1, lane, sd.dt, sd.dtdx, sd.dt_2h,
                                 sd.dt_2, smax, akey, flags, ring, kp, sc.t);
    const bool last = block_arrive<NTL, R>(ctl, smax, akey, flags);
    if (threadIdx.x == 0) {
      bool ok = true;
      if (last) {
        finalize<R>(ctl, kp, true);
        __threadfence();
        atomicAdd(&ctl->gen, 1u);
      } else {
        ok = wait_generation(ctl, gen0, kp.stall_polls);
      }
      s_stop = ok ? 0 : 1;
    }
    __syncthreads();
    if (s_stop) break;
  }
}

template <typename R, int PP, int LIM, int SRC>
struct KL {
  static constexpr int MINB = sizeof(R) == 8 ? 1 : 2;
  static constexpr auto fn = loop1d_kernel<R, PP, LIM, SRC, MINB>;
};

template <int LIM, int SRC>
void* pick_prec(int precision) {
  switch (precision) {
    case PREC_FP64: return (void*)KL<double, 0, LIM, SRC>::fn;
    case PREC_FP32_P64: return (void*)KL<float, 1, LIM, SRC>::fn;
    case PREC_FP32_PC: return (void*)KL<float, 2, LIM, SRC>::fn;
    case PREC_FP32_PS: return (void*)KL<float, 3, LIM, SRC>::fn;
    default: return (void*)KL<float, 0, LIM, SRC>::fn;
  }
}

template <int LIM>
void* pick_src(int precision, int src) {
  switch (src) {
    case 0: return pick_prec<LIM, 0>(precision);
    case 1: return pick_prec<LIM, 1>(precision);
    default: return pick_prec<LIM, 2>(precision);
  }
}

void* pick(const KParams& kp, int precision) {
  const int src = kp.frozen ? 0 : (kp.qi_zero ? 1 : 2);
  switch (kp.limiter) {
    case 1: return pick_src<1>(precision, src);
    case 2: return pick_src<2>(precision, src);
    default: return pick_src<0>(precision, src);
  }
}

size_t smem_bytes(int precision) {
  return (size_t)(NTL / 32) *
         (precision == PREC_FP64 ? ring1d_bytes<double>() : ring1d_bytes<float>());
}

}  // namespace

// Grid of the persistent loop for N cells: one block per 64-cell chunk while
// the device holds that many, so that the few busy warps of a small grid sit
// on different SMs (each warp's critical path is its own chunk; in double the
// SM's FP64 pipe, not latency, bounds it); beyond that as many blocks as fit
// at once, every warp sliding over several chunks.  Sets the kernel's
// shared-memory limit (host side, outside any capture).  Returns 0 if the
// device cannot launch it cooperatively; *cap receives the co-resident limit.
int loop1d_grid(const KParams& kp, int precision, int64_t N, int* cap) {
  int dev = 0, sms = 0, per = 0, coop = 0;
  const void* fn = pick(kp, precision);
  const size_t smem = smem_bytes(precision);
  if (cap) *cap = 0;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, NTL, smem) != cudaSuccess) return 0;
  if (!coop || per < 1 || sms < 1) return 0;
  const int64_t want = (N + 63) / 64;
  const int64_t limit = (int64_t)sms * per;
  if (cap) *cap = (int)limit;
  return (int)(want < limit ? (want < 1 ? 1 : want) : limit);
}

cudaError_t loop1d_launch(int precision, const KParams& kp, void* a, void* b, Ctl* ctl, int64_t N,
                          int grid, int64_t nmax, cudaStream_t st) {
  if (N >= (1LL << 31) / 4 || grid < 1) return cudaErrorInvalidValue;
  int n32 = (int)N;
  long long nm = (long long)nmax;
  void* args[] = {(void*)&kp, &a, &b, &ctl, &n32, &nm};
  return cudaLaunchCooperativeKernel(pick(kp, precision), dim3(grid), dim3(NTL), args,
                                     smem_bytes(precision), st);
}

}  // namespace sv
