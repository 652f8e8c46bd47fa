// sv_stepnd.cu -- fused 2D / 3D unsplit MUSCL-Hancock steps (Sec. 2.3:
// eq. 15 with both flux differences F and G -- and the analogous z flux in
// 3D -- in one update; eq. 14 face states per axis with xi = 0; eq. 13 HLL per
// axis; source Y at the half step; eq. 16 reduction).
//
// Work decomposition ("marching planes").  Each block owns a transverse tile
// (TX threads along x in 2D; TX x TY threads over x-y in 3D) and a segment of
// planes along the outermost axis (y in 2D, z in 3D).  Thread (tx, ty) owns
// the column of cells at one transverse position; the outer ring of threads is
// a one-cell halo whose predictors feed the tile's faces but which update
// nothing.  Per plane q the block
//   a. publishes plane q's states in shared memory (the halo threads also load
//      the second ring, needed by their slopes),
//   b. computes slopes (all axes; the marching-axis slope from the planes
//      q-1, q, q+1 held in registers), the positivity guard and the half-step
//      predictor of plane q -- once per cell,
//   c. publishes the +face states of the transverse axes and computes each
//      cell's left transverse faces (HLL, once per face),
//   d. publishes those fluxes and forms the transverse flux divergence,
//   e. computes the marching-axis face between planes q-1 and q,
//   f. updates plane q-1 (all its faces are now known) and folds its
//      signal speed / tau bound for the next dt.
// Three barriers per plane.  Each thread streams its own column (and the halo
// threads their second-ring cells) through a per-thread ring of kPlaneRing
// planes in shared memory with cp.async, four planes ahead of the one being
// computed; copies are coalesced along x.
#include "sv_internal.h"
#include "sv_ndbnd.cuh"
#include "sv_step1d.cuh"      // cp.async helpers

namespace sv {

template <typename R, int PP, int DIM, int SRC>
struct Nd {
  static constexpr int NF = DIM + 3;
  using V = R[NF];

  static __device__ __forceinline__ void prim(const P<R>& k, const V& u, R& ir, R (&v)[DIM], R& p) {
    ir = Ar<R>::rcp(u[0]);
    R kin2 = 0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      v[a] = u[1 + a] * ir;
      kin2 += u[1 + a] * v[a];
    }
    p = pressure<R, PP>(k, kin2, u[1 + DIM], u[2 + DIM]);
  }

  template <int A>
  static __device__ __forceinline__ void flux(const V& u, const R (&v)[DIM], R p, V& F) {
    F[0] = u[1 + A];
#pragma unroll
    for (int b = 0; b < DIM; ++b) F[1 + b] = u[1 + b] * v[A] + (b == A ? p : (R)0);
    F[1 + DIM] = v[A] * (u[1 + DIM] + p);
    F[2 + DIM] = v[A] * u[2 + DIM];
  }

  // F(u + d/2) - F(u - d/2) along axis A; returns false if a state is non-physical
  template <int A>
  static __device__ __forceinline__ bool dflux(const P<R>& k, const V& u, const V& d, V& dF) {
    V a, b;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      a[f] = u[f] + (R)0.5 * d[f];
      b[f] = u[f] - (R)0.5 * d[f];
    }
    R ira, irb, pa, pb, va[DIM], vb[DIM];
    prim(k, a, ira, va, pa);
    prim(k, b, irb, vb, pb);
    V Fa, Fb;
    flux<A>(a, va, pa, Fa);
    flux<A>(b, vb, pb, Fb);
#pragma unroll
    for (int f = 0; f < NF; ++f) dF[f] = Fa[f] - Fb[f];
    return all_positive(a[0], pa, b[0], pb);
  }

  // Y of a cell of the active medium; a frozen cell (active = false) has none.
  static __device__ __forceinline__ void source(const P<R>& k, const V& u, R& yE, R& yEv,
                                                bool active = true) {
    yE = yEv = (R)0;
    if (SRC == 0 || !active) return;
    R ir, p, v[DIM];
    prim(k, u, ir, v, p);
    Src<R, SRC>::eval(k, u[0], p * ir, u[2 + DIM], yE, yEv);
  }

  // eq. 13 along axis A
  template <int A>
  static __device__ __forceinline__ void hll(const P<R>& k, const V& l, const V& r, const V& fl,
                                             const V& fr, V& F) {
    V L, Rr;
#pragma unroll
    for (int f = 0; f < NF; ++f) { L[f] = l[f]; Rr[f] = r[f]; }
    R irL, pL, vL[DIM], irR, pR, vR[DIM];
    prim(k, L, irL, vL, pL);
    prim(k, Rr, irR, vR, pR);
    if (!all_positive(L[0], pL, Rr[0], pR)) {
#pragma unroll
      for (int f = 0; f < NF; ++f) { L[f] = fl[f]; Rr[f] = fr[f]; }
      prim(k, L, irL, vL, pL);
      prim(k, Rr, irR, vR, pR);
    }
    const R cL = Ar<R>::sqrt_pos(k.gamma * pL * irL);
    const R cR = Ar<R>::sqrt_pos(k.gamma * pR * irR);
    const R sl = fmin(fmin(vL[A] - cL, vR[A] - cR), (R)0);
    const R sr = fmax(fmax(vL[A] + cL, vR[A] + cR), (R)0);
    V FL, FR;
    flux<A>(L, vL, pL, FL);
    flux<A>(Rr, vR, pR, FR);
    const R inv = Ar<R>::rcp(sr - sl);
    const R wl = sr * inv, wr = -sl * inv, wd = sl * sr * inv;
#pragma unroll
    for (int f = 0; f < NF; ++f) F[f] = wl * FL[f] + wr * FR[f] + wd * (Rr[f] - L[f]);
  }
};

// Planes per thread ring (a power of two; four planes are in flight).
constexpr int kPlaneRing = 8;

// Slots of the second-ring cells: two per tile row (x ring) and, in 3D, two
// per tile column (y ring).
template <int DIM, int TX, int TY> struct HaloSlots {
  static constexpr int N = 2 * TY + (DIM == 3 ? 2 * TX : 0);
};

template <typename R, int DIM, int TX, int TY>
constexpr size_t stepnd_smem() {
  constexpr int NF = DIM + 3, SY = DIM == 3 ? TY + 2 : 1, NT = TX * TY;
  return sizeof(R) * ((size_t)NF * SY * (TX + 2) + 2 * (size_t)(DIM - 1) * NF * TY * TX +
                      (size_t)kPlaneRing * NF * NT + (size_t)kPlaneRing * NF * HaloSlots<DIM, TX, TY>::N);
}

// DIM 2: TY must be 1; marching axis y.  DIM 3: marching axis z.
// BND: a 2D grid with walls or outflow on some side, or a medium map / driven
// cells; without it every axis is periodic (the compiled-out general path
// costs the periodic kernel 8%).
template <typename R, int PP, int LIM, int SRC, int DIM, int TX, int TY, int MINB, bool BND>
__global__ void __launch_bounds__(TX * TY, MINB)
stepnd_kernel(const KParams kp, R* __restrict__ bufA, R* __restrict__ bufB, Ctl* __restrict__ ctl,
              int64_t nx, int64_t ny, int64_t nz, int tiles_x, int tiles_y, int nseg) {
  using C = Nd<R, PP, DIM, SRC>;
  constexpr int NF = DIM + 3;
  constexpr int NT = TX * TY;
  constexpr int SY = DIM == 3 ? TY + 2 : 1;     // rows of the shared state plane
  constexpr int AM = DIM - 1;                   // marching axis
  // dynamic shared memory: sU[NF][SY][TX+2], sW[DIM-1][NF][TY][TX],
  // sF[DIM-1][NF][TY][TX], sR[D][NF][NT] (own-column ring), sH[D][NF][NH]
  // (second-ring cells of the halo threads)
  constexpr int D = kPlaneRing, NH = HaloSlots<DIM, TX, TY>::N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R (*sU)[SY][TX + 2] = reinterpret_cast<R (*)[SY][TX + 2]>(smem_raw);
  R (*sW)[NF][TY][TX] = reinterpret_cast<R (*)[NF][TY][TX]>(smem_raw + sizeof(R) * NF * SY * (TX + 2));
  R (*sF)[NF][TY][TX] = reinterpret_cast<R (*)[NF][TY][TX]>(
      smem_raw + sizeof(R) * (NF * SY * (TX + 2) + (DIM - 1) * NF * TY * TX));
  R (*sR)[NF][NT] = reinterpret_cast<R (*)[NF][NT]>(
      smem_raw + sizeof(R) * (NF * SY * (TX + 2) + 2 * (DIM - 1) * NF * TY * TX));
  R (*sH)[NF][NH] = reinterpret_cast<R (*)[NF][NH]>(
      smem_raw + sizeof(R) * (NF * SY * (TX + 2) + 2 * (DIM - 1) * NF * TY * TX + D * NF * NT));

  const StepCtl sc = block_step_ctl(ctl);
  if (!(sc.dt > 0.0)) return;
  const R* __restrict__ Uin = sc.cur ? bufB : bufA;
  R* __restrict__ Uout = sc.cur ? bufA : bufB;
  const P<R> k(kp);
  const StepDt<R> sd(sc);
  const R dt = sd.dt, dtdx = sd.dtdx, dt_2h = sd.dt_2h, dt_2 = sd.dt_2;

  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int seg = blockIdx.x % nseg;
  const int tile = blockIdx.x / nseg;
  const int tile_x = tile % tiles_x, tile_y = tile / tiles_x;
  // Cell and field offsets in 32 bits: the launch admits grids whose fields
  // hold fewer than 2^31 values in all (stepnd_launch).
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
  // 2D boundaries: x sides kp.bc_lo / bc_hi, y sides (the marching axis)
  // kp.bc_ylo / bc_yhi; 3D is periodic.  Ghost positions load the mapped cell;
  // the reversed momenta of wall ghosts are applied when the planes are read.
  static_assert(!BND || DIM == 2, "boundaries and media are 2D only");
  bool fx_own = false, fx_rx = false;
  const I wx = BND ? map_axis(gx, nxi, kp.bc_lo, kp.bc_hi, fx_own) : wrap(gx, nxi);
  const I wy = DIM == 3 ? wrap(gy, nyi) : 0;
  const I col = DIM == 3 ? wy * nxi + wx : wx;               // index within a plane
  // second-ring positions loaded by the halo threads
  const bool ringx = (tx == 0) || (tx == TX - 1);
  const I col_rx = (DIM == 3 ? wy * nxi : 0) +
                   (BND ? map_axis(gx + (tx == 0 ? -1 : 1), nxi, kp.bc_lo, kp.bc_hi, fx_rx)
                        : wrap(gx + (tx == 0 ? -1 : 1), nxi));
  // plane of the marching axis holding position p, and whether it is a wall ghost
  auto plane_of = [&](I p, bool& fy) -> I {
    if (!BND) {
      fy = false;
      return wrap(p, M);
    }
    return map_axis(p, M, kp.bc_ylo, kp.bc_yhi, fy);
  };
  const bool medium = BND && kp.act_lo != nullptr;
  const bool pulses = BND && kp.pul_lo != nullptr;
  const bool ringy = DIM == 3 && ((ty == 0) || (ty == TY - 1));
  const I col_ry = DIM == 3 ? wrap(gy + (ty == 0 ? -1 : 1), nyi) * nxi + wx : 0;
  const int oy = DIM == 3 ? ty + 1 : 0;

  R smax = 0, akey = -INFINITY;
  uint32_t flags = 0;

  const int tid = threadIdx.x;
  const int hx = ty * 2 + (tx == 0 ? 0 : 1);                              // x-ring slot
  const int hy = 2 * TY + tx * 2 + (ty == 0 ? 0 : 1);                     // y-ring slot
  // copy plane p of the own column (p <= q1 + 1) and of the second ring
  // (p <= q1) into ring slot p mod D; always commit a group
  auto issue = [&](I p) {
    const int sl = (int)(p & (D - 1));
    if (p <= q1 + 1) {
      bool fy;
      const I o = plane_of(p, fy) * plane;
#pragma unroll
      for (int f = 0; f < NF; ++f) cp_async<sizeof(R)>(&sR[sl][f][tid], Uin + f * ncell + o + col);
      if (p <= q1) {
        if (ringx)
#pragma unroll
          for (int f = 0; f < NF; ++f) cp_async<sizeof(R)>(&sH[sl][f][hx], Uin + f * ncell + o + col_rx);
        if (ringy)
#pragma unroll
          for (int f = 0; f < NF; ++f) cp_async<sizeof(R)>(&sH[sl][f][hy], Uin + f * ncell + o + col_ry);
      }
    }
    cp_async_commit();
  };

  R Um1[NF], Uq[NF], Up1[NF];
  R Wm_prev[NF], D_prev[NF], H_prev[NF], yE_prev = 0, yEv_prev = 0;
#pragma unroll
  for (int f = 0; f < NF; ++f) Wm_prev[f] = D_prev[f] = H_prev[f] = (R)0;
  auto pidx = [&](I q) {
    bool fy;
    return plane_of(q, fy) * plane;
  };
  for (I p = q0 - 2; p <= q0 + D - 4; ++p) issue(p);    // D - 1 planes ahead

  for (I q = q0 - 1; q <= q1; ++q) {
    // a. planes q-1, q, q+1 of the own column and plane q's second ring have
    //    landed; publish plane q
    cp_async_wait<D - 4>();
    const int sm = (int)((q - 1) & (D - 1)), s0 = (int)(q & (D - 1)), sp = (int)((q + 1) & (D - 1));
    bool fym, fy0, fyp;
    const I jq = plane_of(q, fy0);
    plane_of(q - 1, fym);
    plane_of(q + 1, fyp);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      Um1[f] = sR[sm][f][tid];
      Uq[f] = sR[s0][f][tid];
      Up1[f] = sR[sp][f][tid];
    }
    if (BND) {
      if (fx_own) {
        Um1[1] = -Um1[1];
        Uq[1] = -Uq[1];
        Up1[1] = -Up1[1];
      }
      if (fym) Um1[2] = -Um1[2];
      if (fy0) Uq[2] = -Uq[2];
      if (fyp) Up1[2] = -Up1[2];
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      sU[f][oy][tx + 1] = Uq[f];
      if (ringx) {
        R v = sH[s0][f][hx];
        if (BND && ((f == 1 && fx_rx) || (f == 2 && fy0))) v = -v;
        sU[f][oy][tx == 0 ? 0 : TX + 1] = v;
      }
      if (DIM == 3 && ringy) sU[f][ty == 0 ? 0 : SY - 1][tx + 1] = sH[s0][f][hy];
    }
    // medium of this cell (the mapped cell of a ghost): active or frozen
    const bool active = !medium || (wx >= __ldg(kp.act_lo + jq) && wx < __ldg(kp.act_hi + jq));
    issue(q + D - 2);    // reuses the slot of plane q-2 (read one barrier ago)
    __syncthreads();

    // b. slopes and predictor of plane q
    R d[DIM][NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      d[0][f] = limit<LIM, R>(Uq[f] - sU[f][oy][tx], sU[f][oy][tx + 2] - Uq[f]);
      if (DIM == 3) d[1][f] = limit<LIM, R>(Uq[f] - sU[f][oy - 1][tx + 1], sU[f][oy + 1][tx + 1] - Uq[f]);
      d[AM][f] = limit<LIM, R>(Uq[f] - Um1[f], Up1[f] - Uq[f]);
    }
    R div[NF], dF[NF];
    bool ok = C::template dflux<0>(k, Uq, d[0], div);
    ok = C::template dflux<1>(k, Uq, d[1], dF) && ok;
#pragma unroll
    for (int f = 0; f < NF; ++f) div[f] += dF[f];
    if (DIM == 3) {
      ok = C::template dflux<DIM == 3 ? 2 : 1>(k, Uq, d[AM], dF) && ok;
#pragma unroll
      for (int f = 0; f < NF; ++f) div[f] += dF[f];
    }
    if (!ok) {
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        div[f] = (R)0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) d[a][f] = (R)0;
      }
    }
    R yE, yEv;
    C::source(k, Uq, yE, yEv, active);
    R uh[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) uh[f] = Uq[f] - dt_2h * div[f];
    uh[1 + DIM] += dt_2 * yE;
    uh[2 + DIM] += dt_2 * yEv;
    R yEh, yEvh;
    C::source(k, uh, yEh, yEvh, active);

    // c. transverse faces: publish +states, take the left neighbour's
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      sW[0][f][ty][tx] = uh[f] + (R)0.5 * d[0][f];
      if (DIM == 3) sW[DIM == 3 ? 1 : 0][f][ty][tx] = uh[f] + (R)0.5 * d[1][f];
    }
    __syncthreads();
    R Fx[NF], Fy[NF];
    {
      R l[NF], r[NF], fl[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        l[f] = sW[0][f][ty][tx > 0 ? tx - 1 : tx];
        r[f] = uh[f] - (R)0.5 * d[0][f];
        fl[f] = sU[f][oy][tx];
      }
      C::template hll<0>(k, l, r, fl, Uq, Fx);
      if (DIM == 3) {
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          l[f] = sW[DIM == 3 ? 1 : 0][f][ty > 0 ? ty - 1 : ty][tx];
          r[f] = uh[f] - (R)0.5 * d[1][f];
          fl[f] = sU[f][oy > 0 ? oy - 1 : oy][tx + 1];
        }
        C::template hll<1>(k, l, r, fl, Uq, Fy);
      }
    }
    // d. transverse flux divergence of plane q
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      sF[0][f][ty][tx] = Fx[f];
      if (DIM == 3) sF[DIM == 3 ? 1 : 0][f][ty][tx] = Fy[f];
    }
    __syncthreads();
    R Dq[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      Dq[f] = sF[0][f][ty][tx < TX - 1 ? tx + 1 : tx] - Fx[f];
      if (DIM == 3) Dq[f] += sF[DIM == 3 ? 1 : 0][f][ty < TY - 1 ? ty + 1 : ty][tx] - Fy[f];
    }

    // e. marching-axis face between planes q-1 and q
    R Wm[NF], Hq[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) Wm[f] = uh[f] - (R)0.5 * d[AM][f];
    C::template hll<AM>(k, Wm_prev, Wm, Um1, Uq, Hq);

    // f. update of plane q-1
    if (q > q0 && interior) {
      R un[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) un[f] = Um1[f] - dtdx * (D_prev[f] + Hq[f] - H_prev[f]);
      un[1 + DIM] += dt * yE_prev;
      un[2 + DIM] += dt * yEv_prev;
      // a driven cell holds the pulsating source at the new time level
      if (pulses && gx >= __ldg(kp.pul_lo + (q - 1)) && gx < __ldg(kp.pul_hi + (q - 1)))
        pulse_state<R, NF>(kp, sc.t + sc.dt, un);
      const I o = pidx(q - 1) + col;
#pragma unroll
      for (int f = 0; f < NF; ++f) Uout[f * ncell + o] = un[f];
      R ir, p, v[DIM];
      C::prim(k, un, ir, v, p);
      R v2 = 0;
#pragma unroll
      for (int a = 0; a < DIM; ++a) v2 += v[a] * v[a];
      const R vmag = speed_of<R>(v2);
      R kin2 = 0;
#pragma unroll
      for (int a = 0; a < DIM; ++a) kin2 += un[1 + a] * v[a];
      cfl_cell<R, PP, SRC>(k, un[0], kin2, vmag, un[1 + DIM], un[2 + DIM], smax, akey, flags);
    }

    // rotate the plane window
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      Wm_prev[f] = uh[f] + (R)0.5 * d[AM][f];
      D_prev[f] = Dq[f];
      H_prev[f] = Hq[f];
    }
    yE_prev = yEh;
    yEv_prev = yEvh;
  }
  cp_async_wait<0>();
  reduce_and_finalize<R, NT>(ctl, kp, smax, akey, flags, true);
}

// ------------------------------------------------------------------ launch

template <int DIM, int PREC> struct Cfg;
template <> struct Cfg<2, PREC_FP32_P64> { static constexpr int TX = 256, TY = 1, MINB = 2, SEG = 256; };
template <> struct Cfg<2, PREC_FP64> { static constexpr int TX = 128, TY = 1, MINB = 2, SEG = 256; };
template <> struct Cfg<3, PREC_FP32_P64> { static constexpr int TX = 34, TY = 15, MINB = 1, SEG = 128; };
template <> struct Cfg<3, PREC_FP64> { static constexpr int TX = 16, TY = 16, MINB = 1, SEG = 128; };

// With `n` null only the kernel's shared-memory attribute is set (done once per
// solver at init, outside any stream capture).  `seg` = planes per block along
// the marching axis (0: the default of Cfg); each segment pays a warm-up of
// two planes, shorter segments give more blocks.
template <typename R, int PP, int LIM, int SRC, int DIM, int PREC>
static cudaError_t launch_nd(const KParams& kp, void* a, void* b, Ctl* ctl, const int64_t* n,
                            int seg, cudaStream_t st) {
  using G = Cfg<DIM, PREC>;
  constexpr size_t smem = stepnd_smem<R, DIM, G::TX, G::TY>();
  const bool bnd = DIM == 2 && (kp.bc_lo != BC_PERIODIC || kp.bc_hi != BC_PERIODIC ||
                                kp.bc_ylo != BC_PERIODIC || kp.bc_yhi != BC_PERIODIC ||
                                kp.act_lo != nullptr || kp.pul_lo != nullptr);
  auto fn = bnd ? stepnd_kernel<R, PP, LIM, SRC, DIM, G::TX, G::TY, G::MINB, DIM == 2>
                : stepnd_kernel<R, PP, LIM, SRC, DIM, G::TX, G::TY, G::MINB, false>;
  if (!n) {
    cudaError_t e = cudaFuncSetAttribute(stepnd_kernel<R, PP, LIM, SRC, DIM, G::TX, G::TY, G::MINB, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess || DIM != 2) return e;
    return cudaFuncSetAttribute(stepnd_kernel<R, PP, LIM, SRC, DIM, G::TX, G::TY, G::MINB, DIM == 2>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
  const int64_t nx = n[0], ny = n[1], nz = DIM == 3 ? n[2] : 1;
  const int tiles_x = (int)((nx + G::TX - 3) / (G::TX - 2));
  const int tiles_y = DIM == 3 ? (int)((ny + G::TY - 3) / (G::TY - 2)) : 1;
  const int64_t M = DIM == 3 ? nz : ny;
  const int64_t sl = seg > 0 ? seg : G::SEG;
  int64_t nseg64 = (M + sl - 1) / sl;
  if (nseg64 > M) nseg64 = M;
  int nseg = (int)nseg64;
  if (nseg < 1) nseg = 1;
  const int64_t blocks = (int64_t)tiles_x * tiles_y * nseg;
  if (blocks > 0x7fffffff) return cudaErrorInvalidConfiguration;
  fn<<<(int)blocks, G::TX * G::TY, smem, st>>>(kp, (R*)a, (R*)b, ctl, nx, ny, nz, tiles_x, tiles_y,
                                               nseg);
  return cudaGetLastError();
}

template <int LIM, int SRC, int DIM>
static cudaError_t by_prec(int precision, const KParams& kp, void* a, void* b, Ctl* ctl,
                           const int64_t* n, int seg, cudaStream_t st) {
  switch (precision) {
    case PREC_FP64: return launch_nd<double, 0, LIM, SRC, DIM, PREC_FP64>(kp, a, b, ctl, n, seg, st);
    case PREC_FP32_P64: return launch_nd<float, 1, LIM, SRC, DIM, PREC_FP32_P64>(kp, a, b, ctl, n, seg, st);
    default:
      // the other float policies: in 2D packed plane pairs
      // (sv_stepnd_pair.cu); in 3D each cell's fields in packed pairs
      // (sv_stepnd3f.cu: plane pairs need 242 registers there, one block per
      // SM, and ran 17% slower than one cell per thread)
      if constexpr (DIM == 2) return stepnd_pair_launch(DIM, precision, kp, a, b, ctl, n, seg, st);
      else return stepnd3f_launch(precision, kp, a, b, ctl, n, seg, st);
  }
}

template <int LIM, int DIM>
static cudaError_t by_src(int precision, const KParams& kp, void* a, void* b, Ctl* ctl,
                          const int64_t* n, int seg, cudaStream_t st) {
  if (kp.frozen) return by_prec<LIM, 0, DIM>(precision, kp, a, b, ctl, n, seg, st);
  if (kp.qi_zero) return by_prec<LIM, 1, DIM>(precision, kp, a, b, ctl, n, seg, st);
  return by_prec<LIM, 2, DIM>(precision, kp, a, b, ctl, n, seg, st);
}

template <int DIM>
static cudaError_t by_lim(int precision, const KParams& kp, void* a, void* b, Ctl* ctl,
                          const int64_t* n, int seg, cudaStream_t st) {
  switch (kp.limiter) {
    case 1: return by_src<1, DIM>(precision, kp, a, b, ctl, n, seg, st);
    case 2: return by_src<2, DIM>(precision, kp, a, b, ctl, n, seg, st);
    default: return by_src<0, DIM>(precision, kp, a, b, ctl, n, seg, st);
  }
}

// Default planes per block segment along the marching axis.
int stepnd_default_seg(int dim, int precision) {
  if ((precision == PREC_FP32 || precision == PREC_FP32_PC || precision == PREC_FP32_PS) &&
      dim == 2)
    return stepnd_pair_default_seg(dim);
  if (dim == 2) return precision == PREC_FP64 ? Cfg<2, PREC_FP64>::SEG : Cfg<2, PREC_FP32_P64>::SEG;
  if (precision == PREC_FP32_P64) return Cfg<3, PREC_FP32_P64>::SEG;
  return precision == PREC_FP64 ? Cfg<3, PREC_FP64>::SEG : stepnd3f_default_seg();
}

int stepnd_grid(int dim, int precision, const KParams& kp) {
  cudaError_t e = cudaErrorInvalidValue;
  if (dim == 2) e = by_lim<2>(precision, kp, nullptr, nullptr, nullptr, nullptr, 0, nullptr);
  if (dim == 3) e = by_lim<3>(precision, kp, nullptr, nullptr, nullptr, nullptr, 0, nullptr);
  return e == cudaSuccess ? 1 : 0;
}

cudaError_t stepnd_launch(int dim, int precision, const KParams& kp, void* a, void* b, Ctl* ctl,
                          const int64_t* n, int seg, cudaStream_t st) {
  if (!n) return cudaErrorInvalidValue;
  int64_t ncell = n[0] * n[1] * (dim == 3 ? n[2] : 1);
  if (ncell * (dim + 3) >= (1LL << 31)) return cudaErrorInvalidValue;
  if (dim == 2) return by_lim<2>(precision, kp, a, b, ctl, n, seg, st);
  if (dim == 3) return by_lim<3>(precision, kp, a, b, ctl, n, seg, st);
  return cudaErrorInvalidValue;
}

}  // namespace sv
