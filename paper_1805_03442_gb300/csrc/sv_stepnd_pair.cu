// sv_stepnd_pair.cu -- the float 2D unsplit MUSCL-Hancock step (Sec. 2.3:
// eq. 15 with the F and G flux differences in one update, eq. 14 face states
// per axis with xi = 0, eq. 13 HLL per axis, source Y at the half step, eq. 16
// reduction) marching two rows per iteration.  (The template is written for
// 3D too, where it needs 242 registers and loses to one cell per thread.)
//
// Same work decomposition as the scalar marching-plane kernel (sv_stepnd.cu):
// a block owns a transverse tile with a one-cell halo ring and a segment of
// planes along the outermost axis, each thread one column.  Here each
// iteration takes the planes (q, q+1) of the column as one pair of cells and
// runs their arithmetic in packed f32x2 operations (sv_pairnd.cuh):
//   a. the column's planes q-1 .. q+2 come from a per-thread cp.async ring
//      that stores the planes as pairs (q, q+1); planes q and q+1 (with the
//      halo's second ring) are published in shared memory, also as pairs, so
//      that every shared-memory access of the step moves both cells;
//   b. slopes on every axis, guard, half-step predictor of both cells; the
//      + states of the transverse axes are published;
//   c. transverse faces (left neighbour's + states of both planes against the
//      own - states), one packed HLL per transverse axis;
//   d. transverse flux divergence of both cells;
//   e. marching-axis faces q - 1/2 (its left state carried from the previous
//      iteration) and q + 1/2, one packed HLL;
//   f. update of the previous pair (planes q-2, q-1), whose last face is
//      q - 1/2, and its eq. 16 bound.
// Three block barriers per iteration, i.e. per two planes.  Each cell gets the
// same operations whatever the segmentation, so every segment length gives
// bitwise the same states.
#include "sv_internal.h"
#include "sv_ndbnd.cuh"
#include "sv_pairnd.cuh"
#include "sv_pertnd.cuh"
#include "sv_step1d.cuh"      // cp.async helpers, wrap

namespace sv {

namespace {

using pk::f2;

constexpr int kPairRing = 8;   // planes per thread ring (four plane pairs)

template <int DIM, int TX, int TY> struct PairHalo {
  static constexpr int N = 2 * TY + (DIM == 3 ? 2 * TX : 0);
};

// Shared memory, all in pairs of planes (q, q+1) -- a thread's two cells --
// so that each access moves both: sU[NF][SY][TX+2] (the tile row with its
// halo), sW and sF [DIM-1][NF][NT] (+ states, fluxes), sR[D/2][NF][NT]
// (own-column ring), sH[D/2][NF][NH] (the halo's second ring).
template <int DIM, int TX, int TY>
constexpr size_t pair_smem() {
  constexpr size_t NF = DIM + 3, SY = DIM == 3 ? TY + 2 : 1, NT = (size_t)TX * TY;
  return sizeof(pk::f2) * (NF * SY * (TX + 2) + 2 * (DIM - 1) * NF * NT +
                           (size_t)(kPairRing / 2) * NF * NT +
                           (size_t)(kPairRing / 2) * NF * PairHalo<DIM, TX, TY>::N);
}

// component h of pair slot s as a float address (cp.async destination)
__device__ __forceinline__ float* half_of(pk::f2* s, int h) {
  return reinterpret_cast<float*>(s) + h;
}

template <int PP, int LIM, int SRC, int DIM, int TX, int TY, int MINB, bool BND>
__global__ void __launch_bounds__(TX * TY, MINB)
stepnd_pair_kernel(const KParams kp, float* __restrict__ bufA, float* __restrict__ bufB,
                   Ctl* __restrict__ ctl, int64_t nx, int64_t ny, int64_t nz, int tiles_x,
                   int tiles_y, int nseg) {
  static_assert(!BND || DIM == 2, "boundaries and media are 2D only");
  constexpr int NF = DIM + 3, NT = TX * TY, SY = DIM == 3 ? TY + 2 : 1, AM = DIM - 1;
  constexpr int DP = kPairRing / 2, NH = PairHalo<DIM, TX, TY>::N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  f2 (*sU)[SY][TX + 2] = reinterpret_cast<f2 (*)[SY][TX + 2]>(smem_raw);
  size_t off = sizeof(f2) * NF * SY * (TX + 2);
  f2 (*sW)[NF][NT] = reinterpret_cast<f2 (*)[NF][NT]>(smem_raw + off);
  off += sizeof(f2) * (DIM - 1) * NF * NT;
  f2 (*sF)[NF][NT] = reinterpret_cast<f2 (*)[NF][NT]>(smem_raw + off);
  off += sizeof(f2) * (DIM - 1) * NF * NT;
  f2 (*sR)[NF][NT] = reinterpret_cast<f2 (*)[NF][NT]>(smem_raw + off);
  off += sizeof(f2) * DP * NF * NT;
  f2 (*sH)[NF][NH] = reinterpret_cast<f2 (*)[NF][NH]>(smem_raw + off);

  const StepCtl sc = block_step_ctl(ctl);
  if (!(sc.dt > 0.0)) return;
  const float* __restrict__ Uin = sc.cur ? bufB : bufA;
  float* __restrict__ Uout = sc.cur ? bufA : bufB;
  const P<float> k(kp);
  const StepDt<float> sd(sc);
  const f2 dt2 = pk::splat(sd.dt), ndtdx2 = pk::splat(-sd.dtdx);
  const f2 ndt_2h2 = pk::splat(-sd.dt_2h), dt_22 = pk::splat(sd.dt_2);
  const f2 half = pk::splat(0.5f), nhalf = pk::splat(-0.5f);

  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int seg = blockIdx.x % nseg;
  const int tile = blockIdx.x / nseg;
  const int tile_x = tile % tiles_x, tile_y = tile / tiles_x;
  // Cell and field offsets in 32 bits: the launch admits grids whose fields
  // hold fewer than 2^31 values in all (stepnd_launch), and 64-bit offsets
  // cost the issue-bound kernel a tenth of its instructions.
  using I = int;
  const I gx = (I)tile_x * (TX - 2) - 1 + tx;
  const I gy = DIM == 3 ? (I)tile_y * (TY - 2) - 1 + ty : 0;
  const I M = (I)(DIM == 3 ? nz : ny);                      // planes
  const I plane = (I)(DIM == 3 ? nx * ny : nx);             // cells per plane
  const I ncell = plane * M;
  const I q0 = (I)((int64_t)seg * M / nseg), q1 = (I)((int64_t)(seg + 1) * M / nseg);
  const I nxi = (I)nx, nyi = (I)ny;
  const bool interior = tx >= 1 && tx <= TX - 2 && gx < nxi &&
                        (DIM == 2 || (ty >= 1 && ty <= TY - 2 && gy < nyi));
  bool fx_own = false, fx_rx = false;
  const I wx = BND ? map_axis(gx, nxi, kp.bc_lo, kp.bc_hi, fx_own) : wrap(gx, nxi);
  const I wy = DIM == 3 ? wrap(gy, nyi) : 0;
  const I col = DIM == 3 ? wy * nxi + wx : wx;
  const bool ringx = (tx == 0) || (tx == TX - 1);
  const I col_rx = (DIM == 3 ? wy * nxi : 0) +
                   (BND ? map_axis(gx + (tx == 0 ? -1 : 1), nxi, kp.bc_lo, kp.bc_hi, fx_rx)
                        : wrap(gx + (tx == 0 ? -1 : 1), nxi));
  const bool ringy = DIM == 3 && ((ty == 0) || (ty == TY - 1));
  const I col_ry = DIM == 3 ? wrap(gy + (ty == 0 ? -1 : 1), nyi) * nxi + wx : 0;
  const int oy = DIM == 3 ? ty + 1 : 0;
  auto plane_of = [&](I p, bool& fy) -> I {
    if (!BND) {
      fy = false;
      return wrap(p, M);
    }
    return map_axis(p, M, kp.bc_ylo, kp.bc_yhi, fy);
  };
  const bool medium = BND && kp.act_lo != nullptr;
  const bool pulses = BND && kp.pul_lo != nullptr;
  auto active = [&](I jrow) {
    return !medium || (wx >= __ldg(kp.act_lo + jrow) && wx < __ldg(kp.act_hi + jrow));
  };

  float smax = 0.0f, akey = -INFINITY;
  uint32_t flags = 0;

  const int tid = threadIdx.x;
  const int hx = ty * 2 + (tx == 0 ? 0 : 1);
  const int hy = 2 * TY + tx * 2 + (ty == 0 ? 0 : 1);
  // The iterations take the planes in pairs (q, q+1) with q - q0 even, so
  // plane p lives in component (p - q0) & 1 of ring pair (p - q0 + 4) / 2
  // mod D/2.  Copy plane p of the own column (p <= q1 + 3) and of the second
  // ring (p <= q1 + 2) into its place; always commit a group.
  auto issue = [&](I p) {
    const int r = (int)(p - q0 + 4), ps = (r >> 1) & (DP - 1), h = r & 1;
    if (p <= q1 + 3) {
      bool fy;
      const I o = plane_of(p, fy) * plane;
#pragma unroll
      for (int f = 0; f < NF; ++f) cp_async<4>(half_of(&sR[ps][f][tid], h), Uin + f * ncell + o + col);
      if (p <= q1 + 2) {
        if (ringx)
#pragma unroll
          for (int f = 0; f < NF; ++f)
            cp_async<4>(half_of(&sH[ps][f][hx], h), Uin + f * ncell + o + col_rx);
        if (ringy)
#pragma unroll
          for (int f = 0; f < NF; ++f)
            cp_async<4>(half_of(&sH[ps][f][hy], h), Uin + f * ncell + o + col_ry);
      }
    }
    cp_async_commit();
  };

  // carried from pair to pair: the upper plane's + state on the marching
  // axis (its first use, in the warm-up iteration, only needs to be physical),
  // the marching faces, the transverse divergence and the half-step sources
  float wpm_prev[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) wpm_prev[f] = (f == 0 || f == NF - 2) ? 1.0f : 0.0f;
  f2 H_prev[NF], D_prev[NF], YE_prev = pk::splat(0.0f), YEv_prev = pk::splat(0.0f);
#pragma unroll
  for (int f = 0; f < NF; ++f) H_prev[f] = D_prev[f] = pk::splat(0.0f);

  // invariant at the top of iteration q: planes up to q + 3 issued
  for (I p = q0 - 3; p <= q0 + 1; ++p) issue(p);

  for (I q = q0 - 2; q - 2 < q1; q += 2) {
    // a. planes q-1 .. q+2 of the own column and q, q+1 of the second ring
    //    have landed; publish planes q and q+1
    cp_async_wait<1>();
    // ring pairs (q-2, q-1), (q, q+1) and (q+2, q+3)
    const int pq = (int)(((q - q0 + 4) >> 1) & (DP - 1));
    const int pm = (pq + DP - 1) & (DP - 1), pn = (pq + 1) & (DP - 1);
    bool fym, fy0, fy1, fy2;
    plane_of(q - 1, fym);
    const I j0 = plane_of(q, fy0), j1 = plane_of(q + 1, fy1);
    plane_of(q + 2, fy2);
    // the column's planes q-1 .. q+2 (X = planes q, q+1), wall ghosts with
    // their momenta reversed
    f2 X[NF];
    float um[NF], u2[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      X[f] = sR[pq][f][tid];
      um[f] = sR[pm][f][tid].y;
      u2[f] = sR[pn][f][tid].x;
    }
    if (BND) {
      if (fx_own) {
        X[1] = pk::mul(X[1], pk::splat(-1.0f));
        um[1] = -um[1];
        u2[1] = -u2[1];
      }
      if (fym) um[2] = -um[2];
      if (fy0) X[2].x = -X[2].x;
      if (fy1) X[2].y = -X[2].y;
      if (fy2) u2[2] = -u2[2];
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      sU[f][oy][tx + 1] = X[f];
      if (ringx) {
        f2 a = sH[pq][f][hx];
        if (BND) {
          if (f == 1 && fx_rx) a = pk::mul(a, pk::splat(-1.0f));
          if (f == 2 && fy0) a.x = -a.x;
          if (f == 2 && fy1) a.y = -a.y;
        }
        sU[f][oy][tx == 0 ? 0 : TX + 1] = a;
      }
      if (DIM == 3 && ringy) sU[f][ty == 0 ? 0 : SY - 1][tx + 1] = sH[pq][f][hy];
    }
    issue(q + 4);        // the pair of planes q-4, q-3: no longer read
    issue(q + 5);
    __syncthreads();

    // b. slopes on every axis, guard, predictor of the pair
    f2 d[DIM][NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      {
        const f2 A = pk::sub(X[f], sU[f][oy][tx]);
        const f2 B = pk::sub(sU[f][oy][tx + 2], X[f]);
        d[0][f] = pk::pair(pk::slope<LIM>(A.x, B.x), pk::slope<LIM>(A.y, B.y));
      }
      if (DIM == 3) {
        const f2 A = pk::sub(X[f], sU[f][oy - 1][tx + 1]);
        const f2 B = pk::sub(sU[f][oy + 1][tx + 1], X[f]);
        d[1][f] = pk::pair(pk::slope<LIM>(A.x, B.x), pk::slope<LIM>(A.y, B.y));
      }
      {
        const f2 A = pk::sub(X[f], pk::pair(um[f], X[f].x));
        const f2 B = pk::sub(pk::pair(X[f].y, u2[f]), X[f]);
        d[AM][f] = pk::pair(pk::slope<LIM>(A.x, B.x), pk::slope<LIM>(A.y, B.y));
      }
    }
    f2 div[NF], dF[NF];
    bool ok0 = true, ok1 = true;
    pknx::dflux<DIM, PP, 0>(k, X, d[0], div, ok0, ok1);
    pknx::dflux<DIM, PP, 1>(k, X, d[1], dF, ok0, ok1);
#pragma unroll
    for (int f = 0; f < NF; ++f) div[f] = pk::add(div[f], dF[f]);
    if (DIM == 3) {
      pknx::dflux<DIM, PP, DIM == 3 ? 2 : 1>(k, X, d[AM], dF, ok0, ok1);
#pragma unroll
      for (int f = 0; f < NF; ++f) div[f] = pk::add(div[f], dF[f]);
    }
    if (!(ok0 && ok1)) {
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        if (!ok0) {
          div[f].x = 0.0f;
#pragma unroll
          for (int a = 0; a < DIM; ++a) d[a][f].x = 0.0f;
        }
        if (!ok1) {
          div[f].y = 0.0f;
#pragma unroll
          for (int a = 0; a < DIM; ++a) d[a][f].y = 0.0f;
        }
      }
    }
    // the cells' media (2D map: frozen cells have no source)
    const bool act0 = active(j0), act1 = active(j1);
    f2 yE, yEv;
    pknx::source<DIM, PP, SRC>(k, X, yE, yEv);
    if (!act0) yE.x = yEv.x = 0.0f;
    if (!act1) yE.y = yEv.y = 0.0f;
    f2 uh[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) uh[f] = pk::fma(ndt_2h2, div[f], X[f]);
    if (SRC == 2) uh[1 + DIM] = pk::fma(dt_22, yE, uh[1 + DIM]);
    if (SRC != 0) uh[2 + DIM] = pk::fma(dt_22, yEv, uh[2 + DIM]);
    f2 yEh, yEvh;
    pknx::source<DIM, PP, SRC>(k, uh, yEh, yEvh);
    if (!act0) yEh.x = yEvh.x = 0.0f;
    if (!act1) yEh.y = yEvh.y = 0.0f;

    // publish the + states of the transverse axes
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      sW[0][f][tid] = pk::fma(half, d[0][f], uh[f]);
      if (DIM == 3) sW[DIM == 3 ? 1 : 0][f][tid] = pk::fma(half, d[1][f], uh[f]);
    }
    __syncthreads();

    // c. transverse faces of both planes
    f2 Fx[NF], Fy[NF];
    {
      f2 L[NF], Rr[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        L[f] = sW[0][f][tx > 0 ? tid - 1 : tid];
        Rr[f] = pk::fma(nhalf, d[0][f], uh[f]);
      }
      // a face with a non-physical state: the cells left and right of it
      pknx::hll<DIM, PP, 0>(k, L, Rr,
                            [&](f2 (&cl)[NF], f2 (&cr)[NF]) {
#pragma unroll
                              for (int f = 0; f < NF; ++f) {
                                cl[f] = sU[f][oy][tx];
                                cr[f] = X[f];
                              }
                            },
                            Fx);
      if (DIM == 3) {
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          L[f] = sW[DIM == 3 ? 1 : 0][f][ty > 0 ? tid - TX : tid];
          Rr[f] = pk::fma(nhalf, d[1][f], uh[f]);
        }
        pknx::hll<DIM, PP, DIM == 3 ? 1 : 0>(k, L, Rr,
                                             [&](f2 (&cl)[NF], f2 (&cr)[NF]) {
#pragma unroll
                                               for (int f = 0; f < NF; ++f) {
                                                 cl[f] = sU[f][oy > 0 ? oy - 1 : oy][tx + 1];
                                                 cr[f] = X[f];
                                               }
                                             },
                                             Fy);
      }
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      sF[0][f][tid] = Fx[f];
      if (DIM == 3) sF[DIM == 3 ? 1 : 0][f][tid] = Fy[f];
    }
    __syncthreads();

    // d. transverse flux divergence of both cells
    f2 Dq[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      Dq[f] = pk::sub(sF[0][f][tx < TX - 1 ? tid + 1 : tid], Fx[f]);
      if (DIM == 3)
        Dq[f] = pk::add(Dq[f], pk::sub(sF[DIM == 3 ? 1 : 0][f][ty < TY - 1 ? tid + TX : tid], Fy[f]));
    }

    // e. marching faces q - 1/2 and q + 1/2
    f2 Hq[NF];
    float wpm_next[NF];
    {
      f2 L[NF], Rr[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const f2 wp = pk::fma(half, d[AM][f], uh[f]);
        Rr[f] = pk::fma(nhalf, d[AM][f], uh[f]);
        L[f] = pk::pair(wpm_prev[f], wp.x);
        wpm_next[f] = wp.y;
      }
      pknx::hll<DIM, PP, AM>(k, L, Rr,
                             [&](f2 (&cl)[NF], f2 (&cr)[NF]) {
#pragma unroll
                               for (int f = 0; f < NF; ++f) {
                                 cl[f] = pk::pair(um[f], X[f].x);
                                 cr[f] = X[f];
                               }
                             },
                             Hq);
    }

    // f. update of planes q-2 and q-1 (interior planes: no ghosts)
    if (q - 2 >= q0 && interior) {
      const bool two = q - 1 < q1;
      f2 Nw[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const f2 Q = sR[pm][f][tid];           // planes q-2, q-1 (never ghosts here)
        const f2 FR = pk::pair(H_prev[f].y, Hq[f].x);
        Nw[f] = pk::fma(ndtdx2, pk::add(D_prev[f], pk::sub(FR, H_prev[f])), Q);
      }
      if (SRC == 2) Nw[1 + DIM] = pk::fma(dt2, YE_prev, Nw[1 + DIM]);
      if (SRC != 0) Nw[2 + DIM] = pk::fma(dt2, YEv_prev, Nw[2 + DIM]);
      if (pulses) {
        // driven cells hold the pulsating source at the new time level
        float pu[NF];
        const bool d0 = gx >= __ldg(kp.pul_lo + (q - 2)) && gx < __ldg(kp.pul_hi + (q - 2));
        const bool d1 = two && gx >= __ldg(kp.pul_lo + (q - 1)) && gx < __ldg(kp.pul_hi + (q - 1));
        if (d0 || d1) {
          if constexpr (PP == 3) pulse_state_ps<NF>(kp, sc.t + sc.dt, pu);
          else pulse_state<float, NF>(kp, sc.t + sc.dt, pu);
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            if (d0) Nw[f].x = pu[f];
            if (d1) Nw[f].y = pu[f];
          }
        }
      }
      bool fy;
      const I oa = plane_of(q - 2, fy) * plane + col, ob = plane_of(q - 1, fy) * plane + col;
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        Uout[f * ncell + oa] = Nw[f].x;
        if (two) Uout[f * ncell + ob] = Nw[f].y;
      }
      pknx::cfl<DIM, PP, SRC>(k, Nw, two ? 3 : 1, smax, akey, flags);
    }

#pragma unroll
    for (int f = 0; f < NF; ++f) {
      wpm_prev[f] = wpm_next[f];
      H_prev[f] = Hq[f];
      D_prev[f] = Dq[f];
    }
    YE_prev = yEh;
    YEv_prev = yEvh;
  }
  cp_async_wait<0>();
  reduce_and_finalize<float, NT>(ctl, kp, smax, akey, flags, true);
}

// Tiles of the pair kernel: 128 threads along x (126 interior cells), 166-168
// registers, 3 blocks per SM (a budget of 4 spills).
template <int DIM> struct PairCfg;
template <> struct PairCfg<2> { static constexpr int TX = 128, TY = 1, MINB = 3, SEG = 128; };

template <int PP, int LIM, int SRC, int DIM>
cudaError_t launch_pair(const KParams& kp, void* a, void* b, Ctl* ctl, const int64_t* n, int seg,
                        cudaStream_t st) {
  using G = PairCfg<DIM>;
  constexpr size_t smem = pair_smem<DIM, G::TX, G::TY>();
  if (!n) {
    cudaError_t e = cudaFuncSetAttribute(stepnd_pair_kernel<PP, LIM, SRC, DIM, G::TX, G::TY, G::MINB, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess || DIM != 2) return e;
    return cudaFuncSetAttribute(stepnd_pair_kernel<PP, LIM, SRC, DIM, G::TX, G::TY, G::MINB, DIM == 2>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
  const bool bnd = DIM == 2 && (kp.bc_lo != BC_PERIODIC || kp.bc_hi != BC_PERIODIC ||
                                kp.bc_ylo != BC_PERIODIC || kp.bc_yhi != BC_PERIODIC ||
                                kp.act_lo != nullptr || kp.pul_lo != nullptr);
  auto fn = bnd ? stepnd_pair_kernel<PP, LIM, SRC, DIM, G::TX, G::TY, G::MINB, DIM == 2>
                : stepnd_pair_kernel<PP, LIM, SRC, DIM, G::TX, G::TY, G::MINB, false>;
  const int64_t nx = n[0], ny = n[1], nz = DIM == 3 ? n[2] : 1;
  const int tiles_x = (int)((nx + G::TX - 3) / (G::TX - 2));
  const int tiles_y = DIM == 3 ? (int)((ny + G::TY - 3) / (G::TY - 2)) : 1;
  const int64_t M = DIM == 3 ? nz : ny;
  const int64_t sl = seg > 0 ? seg : G::SEG;
  int64_t nseg64 = (M + sl - 1) / sl;
  if (nseg64 > M) nseg64 = M;
  const int nseg = (int)nseg64;
  const int64_t blocks = (int64_t)tiles_x * tiles_y * nseg;
  if (blocks > 0x7fffffff) return cudaErrorInvalidConfiguration;
  fn<<<(int)blocks, G::TX * G::TY, smem, st>>>(kp, (float*)a, (float*)b, ctl, nx, ny, nz, tiles_x,
                                               tiles_y, nseg);
  return cudaGetLastError();
}

template <int PP, int DIM>
cudaError_t pair_by_kind(const KParams& kp, void* a, void* b, Ctl* ctl, const int64_t* n, int seg,
                         cudaStream_t st) {
  const int src = kp.frozen ? 0 : (kp.qi_zero ? 1 : 2);
#define SV_PAIR_SRC(LIM)                                                   \
  switch (src) {                                                           \
    case 0: return launch_pair<PP, LIM, 0, DIM>(kp, a, b, ctl, n, seg, st);    \
    case 1: return launch_pair<PP, LIM, 1, DIM>(kp, a, b, ctl, n, seg, st);    \
    default: return launch_pair<PP, LIM, 2, DIM>(kp, a, b, ctl, n, seg, st);   \
  }
  switch (kp.limiter) {
    case 1: SV_PAIR_SRC(1)
    case 2: SV_PAIR_SRC(2)
    default: SV_PAIR_SRC(0)
  }
#undef SV_PAIR_SRC
}

}  // namespace

int stepnd_pair_default_seg(int) { return PairCfg<2>::SEG; }

// n == nullptr: set the kernels' shared-memory limits (host side, at set-up).
// 2D only: in 3D the pair kernel needs 242 registers (one 8-warp block per SM)
// and loses to one cell per thread.
cudaError_t stepnd_pair_launch(int dim, int precision, const KParams& kp, void* a, void* b, Ctl* ctl,
                               const int64_t* n, int seg, cudaStream_t st) {
  if (dim == 2)
    switch (precision) {
      case PREC_FP32_PC: return pair_by_kind<2, 2>(kp, a, b, ctl, n, seg, st);
      case PREC_FP32_PS: return pair_by_kind<3, 2>(kp, a, b, ctl, n, seg, st);
      default: return pair_by_kind<0, 2>(kp, a, b, ctl, n, seg, st);
    }
  return cudaErrorInvalidValue;
}

}  // namespace sv
