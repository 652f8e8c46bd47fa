// sv_step1d.cuh -- the per-warp body of the fused 1D MUSCL-Hancock step
// (Sec. 2.3: eqs. 13-15 with xi = 0, source Y), shared by the single-grid
// kernel and the batched sweep kernel so that both compute every cell with
// the same operations in the same order.
//
// A warp owns the 32-cell chunks [c0, c1) of a periodic grid of N cells and
// slides along them, lane i <-> cell chunk_base + i.  Per chunk it
//   1. streams the 4 conserved fields through a per-warp ring of RS chunks in
//      shared memory (cp.async, one coalesced 128-byte copy per field and
//      chunk, RS - 3 chunks in flight ahead of the one being computed),
//   2. reads U_j and its neighbours U_{j-1}, U_{j+1} from the ring,
//   3. limited slopes, positivity guard and the half-step predictor of the
//      chunk's cells (each cell's predictor exactly once),
//   4. the HLL flux of each cell's left face (each face exactly once; the left
//      state comes from lane-1, for lane 0 from the previous chunk),
//   5. the conservative update and half-step source of the PREVIOUS chunk,
//      whose right-most face needed this chunk's first flux,
//   6. the signal speed / tau bound of the updated cells for the next dt.
// Only the two chunks around each warp's run are computed twice.
#pragma once

#include "sv_reduce.cuh"

namespace sv {

// Offsets are 32-bit: the host rejects grids with nf * ncell >= 2^31.

// Ring depth (chunks) per warp: deep for float (memory-bound), shallow for
// double (arithmetic-bound).
template <typename R> struct Ring { static constexpr int RS = sizeof(R) == 4 ? 8 : 4; };

// Asynchronous global -> shared copy of one element (cp.async, L1-allocating).
template <typename R>
__device__ __forceinline__ void cp_async_elem(R* smem, const R* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (sizeof(R) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
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

// One warp's share of a step: chunks [c0, c1) of the periodic grid of N cells
// Uin -> Uout (fields `stride` elements apart).  `ring` is this warp's shared
// buffer of 4 * RS * 32 elements.  Folds the updated cells' signal speed /
// tau key / flags into the per-thread accumulators.
template <typename R, int PP, int LIM, int SRC>
__device__ __forceinline__ void step1d_warp(const P<R>& k, const R* __restrict__ Uin,
                                            R* __restrict__ Uout, int N, int stride, int c0, int c1,
                                            int lane, R dt, R dtdx, R dt_2h, R dt_2, R& smax,
                                            R& akey, uint32_t& flags, R* __restrict__ ring) {
  constexpr int RS = Ring<R>::RS, RN = RS * 32, MASK = RN - 1;
  if (c1 <= c0) return;
  // cells c0*32-64 .. (c1+2)*32-1 are read; no index wrap needed inside [0, N)
  const bool nowrap = c0 >= 2 && (c1 + 2) * 32 <= N;
  // copy chunk c (if it is needed at all) into its ring slot; always commit a
  // group so that the wait counts below stay exact
  auto issue = [&](int c) {
    if (c <= c1 + 1) {
      const int j = c * 32 + lane;
      const int i = nowrap ? j : (int)wrap(j, N);
      R* dst = ring + (c & (RS - 1)) * 32 + lane;
#pragma unroll
      for (int f = 0; f < 4; ++f) cp_async_elem(dst + f * RN, Uin + f * stride + i);
    }
    cp_async_commit();
  };
  for (int c = c0 - 2; c <= c0 + RS - 4; ++c) issue(c);   // RS - 1 chunks ahead

  R Wp_prev[4] = {0, 0, 0, 0}, F_prev[4] = {0, 0, 0, 0}, yE_prev = 0, yEv_prev = 0;
  const int src_m = (lane + 31) & 31, src_p = (lane + 1) & 31;
  // chunk index kk runs from c0-1 (warm-up) to c1 (trailing faces)
  for (int kk = c0 - 1; kk <= c1; ++kk) {
    cp_async_wait<RS - 4>();     // chunks up to kk+1 have landed for this lane ...
    __syncwarp();                // ... and for the warp; chunk kk-2 is no longer read
    issue(kk + RS - 2);          // reuses the slot of chunk kk-2
    const int pos = (kk & (RS - 1)) * 32 + lane;
    R Uc[4], Um[4], Up[4], Uprev[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const R* rf = ring + f * RN;
      Uc[f] = rf[pos];
      Um[f] = rf[(pos - 1) & MASK];
      Up[f] = rf[(pos + 1) & MASK];
      Uprev[f] = rf[(pos - 32) & MASK];
    }
    const int j = kk * 32 + lane;
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
        for (int f = 0; f < 4; ++f) Uout[f * stride + jo] = un[f];
        const R v = un[1] * Ar<R>::rcp(un[0]);
        cfl_cell<R, PP, SRC>(k, un[0], un[1] * v, fabs(v), un[2], un[3], smax, akey, flags);
      }
    }
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      Wp_prev[f] = Wp[f];
      F_prev[f] = F[f];
    }
    yE_prev = yEh;
    yEv_prev = yEvh;
  }
  cp_async_wait<0>();            // nothing in flight when the warp moves on
  __syncwarp();
}

}  // namespace sv
