// sv_step1d.cu -- fused 1D MUSCL-Hancock step (Sec. 2.3: eqs. 13-15 with
// xi = 0, source Y, eq. 16 reduction) for sm_103a.
//
// Work decomposition.  The grid is persistent (a few blocks per SM); each warp
// owns a contiguous run of 32-cell chunks and slides along it, lane i <-> cell
// chunk_base + i.  Per chunk the warp
//   1. reads the 4 conserved fields (one coalesced 128-byte load per field,
//      prefetched PF chunks ahead, no shared memory),
//   2. takes U_{j-1}, U_{j+1} from the neighbouring lanes (shuffles; the edge
//      lanes take them from the previous / next chunk still in registers),
//   3. limited slopes, positivity guard and the half-step predictor of the
//      chunk's cells (each cell's predictor exactly once),
//   4. the HLL flux of each cell's left face (each face exactly once; the left
//      state comes from lane-1, for lane 0 from the previous chunk),
//   5. the conservative update and half-step source of the PREVIOUS chunk,
//      whose right-most face needed this chunk's first flux,
//   6. the signal speed / tau bound of the updated cells for the next dt.
// Only the two chunks around each warp's run are computed twice.
//
// The current buffer and dt are read from the device control block, so the
// same launch can be replayed from a CUDA graph.
#include "sv_internal.h"
#include "sv_reduce.cuh"

namespace sv {

constexpr int NT1 = 256;

// Offsets are 32-bit: the host rejects grids with nf * ncell >= 2^31.
template <typename R>
__device__ __forceinline__ void load_cell(const R* __restrict__ U, int N, int i, R (&u)[4]) {
#pragma unroll
  for (int f = 0; f < 4; ++f) u[f] = __ldg(U + f * N + i);
}

// Steps 1-3 for one cell: slopes d (= Theta h), predictor, face states
// wp = U^{n+1/2} + d/2 (right face), wm = U^{n+1/2} - d/2 (left face), and the
// source at U^{n+1/2} (E and E_nu components).
template <typename R, int PP, int LIM, int SRC>
__device__ __forceinline__ void predict(const P<R>& k, const R (&u)[4], const R (&um)[4],
                                        const R (&up)[4], R dt_2h, R dt_2, R (&wp)[4], R (&wm)[4],
                                        R& yEh, R& yEvh) {
  R d[4], a[4], b[4];
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    d[f] = limit<LIM, R>(u[f] - um[f], up[f] - u[f]);
    a[f] = u[f] + (R)0.5 * d[f];
    b[f] = u[f] - (R)0.5 * d[f];
  }
  const R va = a[1] * Ar<R>::rcp(a[0]);
  const R pa = pressure<R, PP>(k, a[1] * va, a[2], a[3]);
  const R vb = b[1] * Ar<R>::rcp(b[0]);
  const R pb = pressure<R, PP>(k, b[1] * vb, b[2], b[3]);
  R dF[4];
  dF[0] = a[1] - b[1];
  dF[1] = (a[1] * va + pa) - (b[1] * vb + pb);
  dF[2] = va * (a[2] + pa) - vb * (b[2] + pb);
  dF[3] = va * a[3] - vb * b[3];
  if (!((a[0] > (R)0) && (pa > (R)0) && (b[0] > (R)0) && (pb > (R)0))) {
#pragma unroll
    for (int f = 0; f < 4; ++f) d[f] = dF[f] = (R)0;
  }
  R yE = 0, yEv = 0;
  if (SRC != 0) {
    const R ir = Ar<R>::rcp(u[0]);
    const R p = pressure<R, PP>(k, u[1] * (u[1] * ir), u[2], u[3]);
    Src<R, SRC>::eval(k, u[0], p * ir, u[3], yE, yEv);
  }
  R uh[4];
  uh[0] = u[0] - dt_2h * dF[0];
  uh[1] = u[1] - dt_2h * dF[1];
  uh[2] = u[2] - dt_2h * dF[2] + dt_2 * yE;
  uh[3] = u[3] - dt_2h * dF[3] + dt_2 * yEv;
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    wp[f] = uh[f] + (R)0.5 * d[f];
    wm[f] = uh[f] - (R)0.5 * d[f];
  }
  yEh = yEvh = (R)0;
  if (SRC != 0) {
    const R irh = Ar<R>::rcp(uh[0]);
    const R ph = pressure<R, PP>(k, uh[1] * (uh[1] * irh), uh[2], uh[3]);
    Src<R, SRC>::eval(k, uh[0], ph * irh, uh[3], yEh, yEvh);
  }
}

// eq. 13 at one face; a face with a non-physical state uses the cell values
// (fl, fr) instead.
template <typename R, int PP>
__device__ __forceinline__ void hll(const P<R>& k, const R (&l)[4], const R (&r)[4],
                                    const R (&fl)[4], const R (&fr)[4], R (&F)[4]) {
  R L[4], Rr[4];
#pragma unroll
  for (int f = 0; f < 4; ++f) { L[f] = l[f]; Rr[f] = r[f]; }
  R irL = Ar<R>::rcp(L[0]), uL = L[1] * irL, pL = pressure<R, PP>(k, L[1] * uL, L[2], L[3]);
  R irR = Ar<R>::rcp(Rr[0]), uR = Rr[1] * irR, pR = pressure<R, PP>(k, Rr[1] * uR, Rr[2], Rr[3]);
  if (!((L[0] > (R)0) && (pL > (R)0) && (Rr[0] > (R)0) && (pR > (R)0))) {
#pragma unroll
    for (int f = 0; f < 4; ++f) { L[f] = fl[f]; Rr[f] = fr[f]; }
    irL = Ar<R>::rcp(L[0]); uL = L[1] * irL; pL = pressure<R, PP>(k, L[1] * uL, L[2], L[3]);
    irR = Ar<R>::rcp(Rr[0]); uR = Rr[1] * irR; pR = pressure<R, PP>(k, Rr[1] * uR, Rr[2], Rr[3]);
  }
  const R cL = Ar<R>::sqrt_pos(k.gamma * pL * irL);
  const R cR = Ar<R>::sqrt_pos(k.gamma * pR * irR);
  const R sl = fmin(fmin(uL - cL, uR - cR), (R)0);   // min(S_L, 0)
  const R sr = fmax(fmax(uL + cL, uR + cR), (R)0);   // max(S_R, 0)
  const R FL[4] = {L[1], L[1] * uL + pL, uL * (L[2] + pL), uL * L[3]};
  const R FR[4] = {Rr[1], Rr[1] * uR + pR, uR * (Rr[2] + pR), uR * Rr[3]};
  const R inv = Ar<R>::rcp(sr - sl), slsr = sl * sr;
#pragma unroll
  for (int f = 0; f < 4; ++f) F[f] = (sr * FL[f] - sl * FR[f] + slsr * (Rr[f] - L[f])) * inv;
}

template <typename R>
__device__ __forceinline__ R shfl(R v, int src) {
  return __shfl_sync(0xffffffffu, v, src);
}

template <typename R, int PP, int LIM, int SRC, int MINB>
__global__ void __launch_bounds__(NT1, MINB)
step1d_kernel(const KParams kp, R* __restrict__ bufA, R* __restrict__ bufB, Ctl* __restrict__ ctl,
              int N) {
  const double dtd = vload(&ctl->dt);
  if (!(dtd > 0.0)) return;                       // stopped, or t_end reached
  const uint32_t cur = vload(&ctl->cur);
  const R* __restrict__ Uin = cur ? bufB : bufA;
  R* __restrict__ Uout = cur ? bufA : bufB;

  const P<R> k(kp);
  const R dt = (R)dtd, dtdx = (R)(dtd / kp.h), dt_2h = (R)(dtd / (2.0 * kp.h)), dt_2 = (R)(0.5 * dtd);

  const int lane = threadIdx.x & 31;
  const int nwarps = gridDim.x * (NT1 / 32);
  const int warp = blockIdx.x * (NT1 / 32) + (threadIdx.x >> 5);
  const int nchunk = (N + 31) / 32;
  const int c0 = (int)((int64_t)warp * nchunk / nwarps);
  const int c1 = (int)((int64_t)(warp + 1) * nchunk / nwarps);

  R smax = 0, akey = -INFINITY;
  uint32_t flags = 0;

  if (c1 > c0) {
    // cells c0*32-64 .. (c1+2)*32-1 are read; no index wrap needed inside [0, N)
    const bool nowrap = c0 >= 2 && (c1 + 2) * 32 <= N;
    auto idx = [&](int j) { return nowrap ? j : (int)wrap(j, N); };
    const int src_m = (lane + 31) & 31, src_p = (lane + 1) & 31;
    R Uprev[4], Uc[4], Un[4], Un2[4];
    R Wp_prev[4] = {0, 0, 0, 0}, F_prev[4] = {0, 0, 0, 0}, yE_prev = 0, yEv_prev = 0;
    const int base = c0 * 32 + lane;
    load_cell(Uin, N, idx(base - 64), Uprev);
    load_cell(Uin, N, idx(base - 32), Uc);
    load_cell(Uin, N, idx(base), Un);
    load_cell(Uin, N, idx(base + 32), Un2);
    // chunk index kk runs from c0-1 (warm-up) to c1 (trailing faces)
    for (int kk = c0 - 1; kk <= c1; ++kk) {
      const int j = kk * 32 + lane;
      R Um[4], Up[4];
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        Um[f] = shfl(lane == 31 ? Uprev[f] : Uc[f], src_m);
        Up[f] = shfl(lane == 0 ? Un[f] : Uc[f], src_p);
      }
      R Wp[4], Wm[4], yEh, yEvh;
      predict<R, PP, LIM, SRC>(k, Uc, Um, Up, dt_2h, dt_2, Wp, Wm, yEh, yEvh);
      R F[4] = {0, 0, 0, 0};
      if (kk >= c0) {
        R WL[4];
#pragma unroll
        for (int f = 0; f < 4; ++f) WL[f] = shfl(lane == 31 ? Wp_prev[f] : Wp[f], src_m);
        hll<R, PP>(k, WL, Wm, Um, Uc, F);          // face j - 1/2
      }
      if (kk > c0) {
        // update of cell j - 32 (previous chunk)
        R FR[4];
#pragma unroll
        for (int f = 0; f < 4; ++f) FR[f] = shfl(lane == 0 ? F[f] : F_prev[f], src_p);
        const int jo = j - 32;
        if (jo < N) {
          R un[4];
          un[0] = Uprev[0] - dtdx * (FR[0] - F_prev[0]);
          un[1] = Uprev[1] - dtdx * (FR[1] - F_prev[1]);
          un[2] = Uprev[2] - dtdx * (FR[2] - F_prev[2]) + dt * yE_prev;
          un[3] = Uprev[3] - dtdx * (FR[3] - F_prev[3]) + dt * yEv_prev;
#pragma unroll
          for (int f = 0; f < 4; ++f) Uout[f * N + jo] = un[f];
          const R v = un[1] * Ar<R>::rcp(un[0]);
          cfl_cell<R, PP, SRC>(k, un[0], un[1] * v, fabs(v), un[2], un[3], smax, akey, flags);
        }
      }
      // rotate the window
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        Uprev[f] = Uc[f];
        Uc[f] = Un[f];
        Un[f] = Un2[f];
        Wp_prev[f] = Wp[f];
        F_prev[f] = F[f];
      }
      yE_prev = yEh;
      yEv_prev = yEvh;
      if (kk + 3 <= c1 + 1) load_cell(Uin, N, idx(j + 96), Un2);
    }
  }
  reduce_and_finalize<R, NT1>(ctl, kp, (double)smax, (double)akey, flags, true);
}

// Kernel variants: arithmetic (float / double / float with double pressure),
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

int step1d_grid(const KParams& kp, int precision) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, pick(kp, precision), NT1, 0);
  if (per < 1) per = 1;
  return sms * per;
}

cudaError_t step1d_launch(int precision, const KParams& kp, void* a, void* b, Ctl* ctl, int64_t N,
                          int grid, cudaStream_t st) {
  if (N >= (1LL << 31) / 4) return cudaErrorInvalidValue;
  int n32 = (int)N;
  void* args[] = {(void*)&kp, &a, &b, &ctl, &n32};
  return cudaLaunchKernel(pick(kp, precision), dim3(grid), dim3(NT1), args, 0, st);
}

}  // namespace sv
