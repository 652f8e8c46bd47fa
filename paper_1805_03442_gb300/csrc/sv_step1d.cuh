// sv_step1d.cuh -- the per-warp body of the fused 1D MUSCL-Hancock step
// (Sec. 2.3: eqs. 13-15 with xi = 0, source Y), shared by the single-grid
// kernel and the batched sweep kernel so that both compute every cell with
// the same operations in the same order.
//
// A warp owns the 64-cell chunks [c0, c1) of a periodic grid of N cells and
// slides along them; lane i holds the cell pair (2i, 2i+1) of the chunk.
// Per chunk it
//   1. streams the 4 conserved fields through a per-warp ring of RS chunks in
//      shared memory (cp.async, one coalesced 256-byte copy per field and
//      chunk, RS - 3 chunks in flight ahead of the one being computed),
//   2. reads its pair and the two outer neighbours U_{2i-1}, U_{2i+2} from the
//      ring,
//   3. limited slopes, positivity guard and the half-step predictor of both
//      cells (each cell's predictor exactly once),
//   4. the HLL fluxes of the pair's inner face and of its left face (each face
//      exactly once; the left state of the left face comes from lane-1, for
//      lane 0 from the previous chunk),
//   5. the conservative update and half-step source of the PREVIOUS chunk,
//      whose right-most face needed this chunk's first flux,
//   6. the signal speed / tau bound of the updated cells for the next dt.
// Only the two chunks around each warp's run are computed twice.
// In float (all-float pressure, MUSCL-Hancock) steps 3-6 run on the lane's
// two cells at once in packed f32x2 arithmetic (sv_pair1d.cuh); there both
// faces of step 4 are one packed HLL evaluation.
#pragma once

#include <type_traits>

#include "sv_pair1d.cuh"
#include "sv_pert1d.cuh"
#include "sv_reduce.cuh"

namespace sv {

// Offsets are 32-bit: the host rejects grids with nf * ncell >= 2^31.

// Ring depth (64-cell chunks) per warp.
constexpr int kRing1d = 8;

template <typename R> struct Pair;
template <> struct Pair<float> { using T = float2; };
template <> struct Pair<double> { using T = double2; };

// Bytes of the per-warp ring: 4 fields x kRing1d chunks x 64 cells.
template <typename R>
constexpr int ring1d_bytes() { return 4 * kRing1d * 64 * (int)sizeof(R); }

// Asynchronous global -> shared copy of BYTES bytes (cp.async, L1-allocating).
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(BYTES)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Primitive recovery (eq. 5, eq. 7): 1/rho, v, rho v^2, p.
template <typename R, int PP>
__device__ __forceinline__ void prim1(const P<R>& k, const R (&u)[4], R& ir, R& v, R& kin2, R& p) {
  ir = Ar<R>::rcp(u[0]);
  v = u[1] * ir;
  kin2 = u[1] * v;
  p = pressure<R, PP>(k, kin2, u[2], u[3]);
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
  R ira, va, ka, pa, irb, vb, kb, pb;
  prim1<R, PP>(k, a, ira, va, ka, pa);
  prim1<R, PP>(k, b, irb, vb, kb, pb);
  R dF[4];
  dF[0] = a[1] - b[1];
  dF[1] = (ka + pa) - (kb + pb);
  dF[2] = va * (a[2] + pa) - vb * (b[2] + pb);
  dF[3] = va * a[3] - vb * b[3];
  // positivity guard: a non-physical extrapolated state drops the slopes
  if (!all_positive(a[0], pa, b[0], pb)) {
#pragma unroll
    for (int f = 0; f < 4; ++f) d[f] = dF[f] = (R)0;
  }
  R yE = 0, yEv = 0;
  if (SRC != 0) {
    R ir, v, kin2, p;
    prim1<R, PP>(k, u, ir, v, kin2, p);
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
    R ir, v, kin2, p;
    prim1<R, PP>(k, uh, ir, v, kin2, p);
    Src<R, SRC>::eval(k, uh[0], p * ir, uh[3], yEh, yEvh);
  }
}

// Heun stages: slopes with the same guard, face states at the stage's own time
// level (wp = u + d/2, wm = u - d/2) and the source Y(u) for the update.
template <typename R, int PP, int LIM, int SRC>
__device__ __forceinline__ void level_states(const P<R>& k, const R (&u)[4], const R (&um)[4],
                                             const R (&up)[4], R (&wp)[4], R (&wm)[4], R& yE,
                                             R& yEv) {
  R d[4], a[4], b[4];
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    d[f] = limit<LIM, R>(u[f] - um[f], up[f] - u[f]);
    a[f] = u[f] + (R)0.5 * d[f];
    b[f] = u[f] - (R)0.5 * d[f];
  }
  R ira, va, ka, pa, irb, vb, kb, pb;
  prim1<R, PP>(k, a, ira, va, ka, pa);
  prim1<R, PP>(k, b, irb, vb, kb, pb);
  if (!all_positive(a[0], pa, b[0], pb)) {
#pragma unroll
    for (int f = 0; f < 4; ++f) a[f] = b[f] = u[f];
  }
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    wp[f] = a[f];
    wm[f] = b[f];
  }
  yE = yEv = (R)0;
  if (SRC != 0) {
    R ir, v, kin2, p;
    prim1<R, PP>(k, u, ir, v, kin2, p);
    Src<R, SRC>::eval(k, u[0], p * ir, u[3], yE, yEv);
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
  R irL, uL, kL, pL, irR, uR, kR, pR;
  prim1<R, PP>(k, L, irL, uL, kL, pL);
  prim1<R, PP>(k, Rr, irR, uR, kR, pR);
  if (!all_positive(L[0], pL, Rr[0], pR)) {
#pragma unroll
    for (int f = 0; f < 4; ++f) { L[f] = fl[f]; Rr[f] = fr[f]; }
    prim1<R, PP>(k, L, irL, uL, kL, pL);
    prim1<R, PP>(k, Rr, irR, uR, kR, pR);
  }
  const R cL = Ar<R>::sqrt_pos(k.gamma * pL * irL);
  const R cR = Ar<R>::sqrt_pos(k.gamma * pR * irR);
  const R sl = fmin(fmin(uL - cL, uR - cR), (R)0);   // min(S_L, 0)
  const R sr = fmax(fmax(uL + cL, uR + cR), (R)0);   // max(S_R, 0)
  const R FL[4] = {L[1], kL + pL, uL * (L[2] + pL), uL * L[3]};
  const R FR[4] = {Rr[1], kR + pR, uR * (Rr[2] + pR), uR * Rr[3]};
  const R inv = Ar<R>::rcp(sr - sl);
  const R wl = sr * inv, wr = -sl * inv, wd = sl * sr * inv;
#pragma unroll
  for (int f = 0; f < 4; ++f) F[f] = wl * FL[f] + wr * FR[f] + wd * (Rr[f] - L[f]);
}

// Cell whose state fills position j of a 1D grid of N cells: periodic wrap,
// wall mirror (ghost -1-g holds cell g with the velocity reversed: *flip) or
// outflow copy of the boundary cell.  Ghosts deeper than the two the stencil
// uses are clamped into the grid; their values never reach an updated cell.
__device__ __forceinline__ int bc_index(int j, int N, int bc_lo, int bc_hi, bool& flip) {
  flip = false;
  if (j >= 0 && j < N) return j;
  const int bc = j < 0 ? bc_lo : bc_hi;
  if (bc == BC_PERIODIC) return (int)wrap(j, N);
  int m;
  if (bc == BC_REFLECT) {
    flip = true;
    m = j < 0 ? -1 - j : 2 * N - 1 - j;
  } else {
    m = j < 0 ? 0 : N - 1;
  }
  return m < 0 ? 0 : (m >= N ? N - 1 : m);
}

template <typename R>
__device__ __forceinline__ R shfl(R v, int src) {
  return __shfl_sync(0xffffffffu, v, src);
}

// Conservative update (eq. 15) of one cell and, with CFL, its next-dt bound.
template <typename R, int PP, int SRC, bool CFL = true>
__device__ __forceinline__ void update_cell(const P<R>& k, const R (&u)[4], const R (&Fl)[4],
                                            const R (&Fr)[4], R yE, R yEv, R dt, R dtdx,
                                            R (&un)[4], R& smax, R& akey, uint32_t& flags) {
  un[0] = u[0] - dtdx * (Fr[0] - Fl[0]);
  un[1] = u[1] - dtdx * (Fr[1] - Fl[1]);
  un[2] = u[2] - dtdx * (Fr[2] - Fl[2]) + dt * yE;
  un[3] = u[3] - dtdx * (Fr[3] - Fl[3]) + dt * yEv;
  if (CFL) cell_bound<R, PP, SRC>(k, un, smax, akey, flags);
}

// State of the driven boundary's ghost cell centred at x at time t (double).
__device__ __forceinline__ void drive_state(const KParams& kp, double x, double t, double (&u)[4]) {
  const double env = exp(-kp.drv_kim * x);
  double s, c;
  sincos(kp.drv_kre * x - kp.drv_omega * t, &s, &c);
#pragma unroll
  for (int f = 0; f < 4; ++f) u[f] = kp.drv_base[f] + env * (kp.drv_are[f] * c - kp.drv_aim[f] * s);
}

// One warp's share of a step: chunks [c0, c1) (64 cells each) of the periodic
// grid of N cells Uin -> Uout (fields `stride` elements apart).  `ring` is this
// warp's shared buffer (ring1d_bytes<R>()).  Folds the updated cells' signal
// speed / tau key / flags into the per-thread accumulators.
// Step modes: the MUSCL-Hancock step, or one of the two stages of the Heun
// (SSP-RK2) integration of the same spatial operator L:
//   stage 1: Uout = Uin + dt L(Uin)
//   stage 2: Uout = (U0 + Uin) / 2 + dt/2 L(Uin)   (U0 read cell by cell; Uout
//            may be U0: each cell reads its own U0 before writing it)
enum { MODE_HANCOCK = 0, MODE_HEUN1 = 1, MODE_HEUN2 = 2 };

// `kp` and `t` (the step's start time) only serve a driven boundary.
template <typename R, int PP, int LIM, int SRC, int MODE = MODE_HANCOCK>
__device__ __forceinline__ void step1d_warp(const P<R>& k, const R* __restrict__ Uin, R* Uout,
                                            int N, int stride, int c0, int c1, int lane, R dt,
                                            R dtdx, R dt_2h, R dt_2, R& smax, R& akey,
                                            uint32_t& flags, R* __restrict__ ring,
                                            const KParams& kp, double t, const R* U0 = nullptr) {
  using R2 = typename Pair<R>::T;
  constexpr int RS = kRing1d, RN = RS * 64, MASK = RN - 1;
  if (c1 <= c0) return;
  // cells c0*64-128 .. (c1+2)*64-1 are read; inside [0, N) no index wraps
  const bool nowrap = c0 >= 2 && (c1 + 2) * 64 <= N;
  const bool pairs = nowrap && (stride % 2) == 0;    // 2-element copies are aligned
  // copy chunk c (if it is needed at all) into its ring slot; always commit a
  // group so that the wait counts below stay exact
  auto issue = [&](int c) {
    if (c <= c1 + 1) {
      const int j = c * 64 + 2 * lane;
      R* dst = ring + (c & (RS - 1)) * 64 + 2 * lane;
      if (pairs) {
#pragma unroll
        for (int f = 0; f < 4; ++f) cp_async<2 * sizeof(R)>(dst + f * RN, Uin + f * stride + j);
      } else {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          if (j + e < 0 && k.bc_lo == BC_DRIVEN) {
            double u[4];
            drive_state(kp, ((double)(j + e) + 0.5) * kp.h, t, u);
#pragma unroll
            for (int f = 0; f < 4; ++f) dst[f * RN + e] = (R)(PP == 3 ? u[f] - kp.ref[f] : u[f]);
          } else {
            bool fl;
            const int i = bc_index(j + e, N, k.bc_lo, k.bc_hi, fl);
#pragma unroll
            for (int f = 0; f < 4; ++f) cp_async<sizeof(R)>(dst + f * RN + e, Uin + f * stride + i);
          }
        }
      }
    }
    cp_async_commit();
  };
  // wall ghosts: reverse the velocity of the landed copies of chunk c (each
  // lane its own pair; a __syncwarp must follow)
  const bool walls = !nowrap && (k.bc_lo == BC_REFLECT || k.bc_hi == BC_REFLECT);
  auto flip_ghosts = [&](int c) {
    const int j = c * 64 + 2 * lane;
    R* m = ring + RN + (c & (RS - 1)) * 64 + 2 * lane;
    bool f0, f1;
    bc_index(j, N, k.bc_lo, k.bc_hi, f0);
    bc_index(j + 1, N, k.bc_lo, k.bc_hi, f1);
    if (f0) m[0] = -m[0];
    if (f1) m[1] = -m[1];
  };
  for (int c = c0 - 2; c <= c0 + RS - 4; ++c) issue(c);   // RS - 1 chunks ahead
  if (walls) {
    cp_async_wait<RS - 3>();     // chunks c0-2 and c0-1 have landed
    flip_ghosts(c0 - 2);
    flip_ghosts(c0 - 1);
  }

  R Wp1_prev[4] = {0, 0, 0, 0}, Fa_prev[4] = {0, 0, 0, 0}, Fb_prev[4] = {0, 0, 0, 0};
  R y0E_prev = 0, y0Ev_prev = 0, y1E_prev = 0, y1Ev_prev = 0;
  const int src_m = (lane + 31) & 31, src_p = (lane + 1) & 31;
  // The float MUSCL-Hancock step (float or compensated-float pressure, or the
  // perturbation layout) runs both cells of a lane in packed f32x2 arithmetic
  // (sv_pair1d.cuh, sv_pert1d.cuh); double, double-pressure and Heun stay
  // scalar.
  constexpr bool PACKED = std::is_same<R, float>::value && (PP == 0 || PP == 2 || PP == 3) &&
                          MODE == MODE_HANCOCK;
  constexpr int PPK = PP == 1 ? 0 : PP;     // the packed policy (unused when not PACKED)
  using pk::f2;
  // carried from chunk to chunk: the odd cell's right face state (its first
  // use, by lane 0 of the warm-up chunk, only needs to be physical), the
  // (left, inner) face fluxes and the half-step sources of the pair
  float Wy_prev[4] = {1.0f, 0.0f, 1.0f, 0.0f};
  f2 F_prev[4] = {}, YE_prev = {}, YEv_prev = {};
  const f2 dt2 = pk::splat((float)dt), ndtdx2 = pk::splat(-(float)dtdx);
  const f2 ndt_2h2 = pk::splat(-(float)dt_2h), dt_22 = pk::splat((float)dt_2);
  // chunk index kk runs from c0-1 (warm-up) to c1 (trailing faces)
  for (int kk = c0 - 1; kk <= c1; ++kk) {
    cp_async_wait<RS - 4>();     // chunks up to kk+1 have landed for this lane ...
    if (walls) flip_ghosts(kk + 1);
    __syncwarp();                // ... and for the warp; chunk kk-2 is no longer read
    issue(kk + RS - 2);          // reuses the slot of chunk kk-2
    const int pos = (kk & (RS - 1)) * 64 + 2 * lane;
    if constexpr (PACKED) {
      f2 X[4], A[4], B[4], Qp[4];
      float xl[4];
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const float* rf = reinterpret_cast<const float*>(ring) + f * RN;
        X[f] = *reinterpret_cast<const f2*>(rf + pos);
        Qp[f] = *reinterpret_cast<const f2*>(rf + ((pos - 64) & MASK));   // previous chunk's pair
        xl[f] = rf[(pos - 1) & MASK];
        // one-sided differences, the inner one shared by both cells (scalar:
        // the limiter takes them component by component)
        const float c = X[f].y - X[f].x;
        A[f] = pk::pair(X[f].x - xl[f], c);
        B[f] = pk::pair(c, rf[(pos + 2) & MASK] - X[f].y);
      }
      f2 WP[4], WM[4], YE, YEv, L[4], F[4];
      pkx::predict<PPK, LIM, SRC>(k, X, A, B, ndt_2h2, dt_22, WP, WM, YE, YEv);
#pragma unroll
      for (int f = 0; f < 4; ++f) L[f] = pk::pair(shfl(lane == 31 ? Wy_prev[f] : WP[f].y, src_m), WP[f].x);
      pkx::hll<PPK>(k, L, WM, xl, X, F);            // faces 2i - 1/2 and 2i + 1/2
      if (kk > c0) {
        // update of the pair of chunk kk-1: left faces F_prev, right faces
        // (inner face, next lane's left face)
        f2 FRt[4];
#pragma unroll
        for (int f = 0; f < 4; ++f)
          FRt[f] = pk::pair(F_prev[f].y, shfl(lane == 0 ? F[f].x : F_prev[f].x, src_p));
        const int jo = (kk - 1) * 64 + 2 * lane;
        if (jo < N) {
          f2 Nw[4];
          pk::update<SRC>(Qp, F_prev, FRt, YE_prev, YEv_prev, dt2, ndtdx2, Nw);
          const bool two = jo + 1 < N;
          pkx::cfl<PPK, SRC>(k, Nw, two ? 3 : 1, smax, akey, flags);
          if (two && (stride % 2) == 0) {
#pragma unroll
            for (int f = 0; f < 4; ++f) *reinterpret_cast<f2*>(Uout + f * stride + jo) = Nw[f];
          } else {
#pragma unroll
            for (int f = 0; f < 4; ++f) {
              Uout[f * stride + jo] = Nw[f].x;
              if (two) Uout[f * stride + jo + 1] = Nw[f].y;
            }
          }
        }
      }
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        Wy_prev[f] = WP[f].y;
        F_prev[f] = F[f];
      }
      YE_prev = YE;
      YEv_prev = YEv;
    } else {
      R x0[4], x1[4], um[4], up[4], q0[4], q1[4];
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const R* rf = ring + f * RN;
        const R2 c2 = *reinterpret_cast<const R2*>(rf + pos);
        const R2 p2 = *reinterpret_cast<const R2*>(rf + ((pos - 64) & MASK));
        x0[f] = c2.x;
        x1[f] = c2.y;
        q0[f] = p2.x;                // the previous chunk's pair (updated below)
        q1[f] = p2.y;
        um[f] = rf[(pos - 1) & MASK];
        up[f] = rf[(pos + 2) & MASK];
      }
      R Wp0[4], Wm0[4], Wp1[4], Wm1[4], y0E, y0Ev, y1E, y1Ev;
      if (MODE == MODE_HANCOCK) {
        predict<R, PP, LIM, SRC>(k, x0, um, x1, dt_2h, dt_2, Wp0, Wm0, y0E, y0Ev);
        predict<R, PP, LIM, SRC>(k, x1, x0, up, dt_2h, dt_2, Wp1, Wm1, y1E, y1Ev);
      } else {
        level_states<R, PP, LIM, SRC>(k, x0, um, x1, Wp0, Wm0, y0E, y0Ev);
        level_states<R, PP, LIM, SRC>(k, x1, x0, up, Wp1, Wm1, y1E, y1Ev);
      }
      R Fa[4] = {0, 0, 0, 0}, Fb[4];
      hll<R, PP>(k, Wp0, Wm1, x0, x1, Fb);            // face 2i + 1/2
      if (kk >= c0) {
        R WL[4];
#pragma unroll
        for (int f = 0; f < 4; ++f) WL[f] = shfl(lane == 31 ? Wp1_prev[f] : Wp1[f], src_m);
        hll<R, PP>(k, WL, Wm0, um, x0, Fa);           // face 2i - 1/2
      }
      if (kk > c0) {
        // update of the pair of chunk kk-1
        R FR[4];
#pragma unroll
        for (int f = 0; f < 4; ++f) FR[f] = shfl(lane == 0 ? Fa[f] : Fa_prev[f], src_p);
        const int jo = (kk - 1) * 64 + 2 * lane;
        R n0[4], n1[4];
        if (jo < N) {
          if (MODE == MODE_HEUN2) {
            // (U0 + U*)/2 + dt/2 L(U*) = (U0 + U*)/2 - dt/(2h) dF + dt/2 Y(U*)
#pragma unroll
            for (int f = 0; f < 4; ++f) {
              // plain loads: U0 may be the buffer this kernel writes
              q0[f] = (R)0.5 * (U0[f * stride + jo] + q0[f]);
              if (jo + 1 < N) q1[f] = (R)0.5 * (U0[f * stride + jo + 1] + q1[f]);
            }
          }
          const R udt = MODE == MODE_HEUN2 ? dt_2 : dt, udx = MODE == MODE_HEUN2 ? dt_2h : dtdx;
          update_cell<R, PP, SRC, MODE != MODE_HEUN1>(k, q0, Fa_prev, Fb_prev, y0E_prev, y0Ev_prev,
                                                       udt, udx, n0, smax, akey, flags);
          if (jo + 1 < N) {
            update_cell<R, PP, SRC, MODE != MODE_HEUN1>(k, q1, Fb_prev, FR, y1E_prev, y1Ev_prev, udt,
                                                         udx, n1, smax, akey, flags);
            if ((stride % 2) == 0) {
#pragma unroll
              for (int f = 0; f < 4; ++f)
                *reinterpret_cast<R2*>(Uout + f * stride + jo) = R2{n0[f], n1[f]};
            } else {
#pragma unroll
              for (int f = 0; f < 4; ++f) {
                Uout[f * stride + jo] = n0[f];
                Uout[f * stride + jo + 1] = n1[f];
              }
            }
          } else {
#pragma unroll
            for (int f = 0; f < 4; ++f) Uout[f * stride + jo] = n0[f];
          }
        }
      }
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        Wp1_prev[f] = Wp1[f];
        Fa_prev[f] = Fa[f];
        Fb_prev[f] = Fb[f];
      }
      y0E_prev = y0E;
      y0Ev_prev = y0Ev;
      y1E_prev = y1E;
      y1Ev_prev = y1Ev;
    }   // scalar body
  }
  cp_async_wait<0>();            // nothing in flight when the warp moves on
  __syncwarp();
}

}  // namespace sv
