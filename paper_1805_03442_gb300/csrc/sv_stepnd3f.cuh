// sv_stepnd3f.cuh -- the float 3D unsplit MUSCL-Hancock step (Sec. 2.3: eq. 15
// with the F, G and H flux differences in one update, eq. 14 face states per
// axis with xi = 0, eq. 13 HLL per axis, source Y at the half step, eq. 16
// reduction) with each cell's six conserved fields held as three packed
// pairs: (rho, rho v_x), (rho v_y, rho v_z), (E, E_nu).
//
// Same marching-plane decomposition as the scalar kernel of sv_stepnd.cu: a
// block owns a TX x TY tile of columns with a one-cell halo ring and a
// segment of z planes, one thread per column, three block barriers per plane.
// What the pairs change: every operation that treats the six fields alike --
// the one-sided differences, the extrapolations u +- d/2, the flux
// differences and their sum, the half-step predictor, the face states, the
// HLL combination, the flux divergence and the update -- is one packed f32x2
// instruction (FADD2 / FMUL2 / FFMA2) per pair of fields instead of two, and
// every shared-memory access moves a pair (8-byte loads and stores).  The
// primitive recovery, the signal speeds, the limiter, the positivity tests
// and the source stay scalar.  A thread holds the same values as in the
// scalar kernel, so it needs about the same registers and runs the same tile.
//
// Each packed operation rounds each component as the scalar one does; the
// results differ from the scalar kernel's only where the compiler fuses a
// multiply and an add differently.
//
// The kernel is instantiated for float and compensated-float pressure in
// sv_stepnd3f.cu and for the perturbation layout in sv_stepnd3f_ps.cu.
//
// Pressure policies PP: 0 float, 2 compensated float, 3 the perturbation
// layout (the state holds u = U - U_ref, sv_pertnd.cuh: rho = 1 + u_rho, the
// fluxes less F(U_ref), the source from the perturbation series of psn::).
#pragma once

#include "sv_internal.h"
#include "sv_pair1d.cuh"      // packed f32x2 helpers
#include "sv_pertnd.cuh"      // perturbation layout (psn::)
#include "sv_step1d.cuh"      // cp.async helpers, wrap

namespace sv {

namespace {

using pk::f2;

constexpr int NP = 3;         // field pairs of a 3D state
constexpr int kRing3 = 8;     // planes per thread ring (four in flight)

// Primitive recovery (eq. 5, eq. 7) of a state: rho, 1/rho, v, rho |v|^2, p
// and pf, the pressure term of the fluxes (p; in the perturbation layout
// p - 1, the fluxes there being those less F(U_ref)).
struct Pr3 {
  float rho, ir, vx, kin2, p, pf;
  f2 vyz;
};

template <int PP>
__device__ __forceinline__ Pr3 prim3(const P<float>& k, const f2 (&u)[NP]) {
  Pr3 q;
  q.rho = PP == 3 ? 1.0f + u[0].x : u[0].x;
  q.ir = Ar<float>::rcp(q.rho);
  q.vx = u[0].y * q.ir;
  q.vyz = pk::pair(u[1].x * q.ir, u[1].y * q.ir);
  q.kin2 = fmaf(u[1].y, q.vyz.y, fmaf(u[1].x, q.vyz.x, u[0].y * q.vx));
  if constexpr (PP == 3) {
    q.pf = k.g1 * fmaf(q.kin2, -0.5f, u[2].x - u[2].y);
    q.p = 1.0f + q.pf;
  } else {
    q.p = q.pf = pressure<float, PP>(k, q.kin2, u[2].x, u[2].y);
  }
  return q;
}

// the state's six fields as an array (the scalar helpers of the
// perturbation layout take one)
__device__ __forceinline__ void fields6(const f2 (&u)[NP], float (&v)[2 * NP]) {
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    v[2 * p] = u[p].x;
    v[2 * p + 1] = u[p].y;
  }
}

template <int A>
__device__ __forceinline__ float vel(const Pr3& q) {
  return A == 0 ? q.vx : (A == 1 ? q.vyz.x : q.vyz.y);
}

// Flux along axis A (F, G, H of eq. 15) in field pairs, component by
// component (a packed product here would first have to copy v into a pair);
// in the perturbation layout the flux less F(U_ref).
template <int PP, int A>
__device__ __forceinline__ void flux3(const P<float>& k, const f2 (&u)[NP], const Pr3& q,
                                      f2 (&F)[NP]) {
  const float v = vel<A>(q);
  const float mA = A == 0 ? u[0].y : (A == 1 ? u[1].x : u[1].y);
  F[0] = pk::pair(mA, A == 0 ? fmaf(u[0].y, v, q.pf) : u[0].y * v);
  F[1] = pk::pair(A == 1 ? fmaf(u[1].x, v, q.pf) : u[1].x * v,
                  A == 2 ? fmaf(u[1].y, v, q.pf) : u[1].y * v);
  if constexpr (PP == 3) F[2] = pk::pair(v * (k.h0 + (u[2].x + q.pf)), v * (k.ev0 + u[2].y));
  else F[2] = pk::pair(v * (u[2].x + q.p), v * u[2].y);
}

// F(u + d/2) - F(u - d/2) along axis A; false if either state is non-physical.
template <int PP, int A>
__device__ __forceinline__ bool dflux3(const P<float>& k, const f2 (&u)[NP], const f2 (&d)[NP],
                                       f2 (&dF)[NP]) {
  f2 a[NP], b[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    a[p] = pk::fma(pk::splat(0.5f), d[p], u[p]);
    b[p] = pk::fma(pk::splat(-0.5f), d[p], u[p]);
  }
  const Pr3 qa = prim3<PP>(k, a), qb = prim3<PP>(k, b);
  f2 Fa[NP], Fb[NP];
  flux3<PP, A>(k, a, qa, Fa);
  flux3<PP, A>(k, b, qb, Fb);
#pragma unroll
  for (int p = 0; p < NP; ++p) dF[p] = pk::sub(Fa[p], Fb[p]);
  return all_positive(qa.rho, qa.p, qb.rho, qb.p);
}

// (Y_E, Y_Enu) of a state (eq. 6 closures).
template <int PP, int SRC>
__device__ __forceinline__ f2 source3(const P<float>& k, const f2 (&u)[NP]) {
  if (SRC == 0) return pk::splat(0.0f);
  float yE, yEv;
  if constexpr (PP == 3) {
    float v[2 * NP];
    fields6(u, v);
    psn::source<3, SRC>(k, v, psn::prim<3>(k, v), yE, yEv);
  } else {
    const Pr3 q = prim3<PP>(k, u);
    Src<float, SRC>::eval(k, u[0].x, q.p * q.ir, u[2].y, yE, yEv);
  }
  return pk::pair(yE, yEv);
}

// eq. 13 along axis A with left state L and right state R; a face with a
// non-physical state takes the cell values, which `fallback(L, R)` loads
// (only then: it is the rare path).
template <int PP, int A, typename FB>
__device__ __forceinline__ void hll3(const P<float>& k, f2 (&L)[NP], f2 (&R)[NP], FB&& fallback,
                                     f2 (&F)[NP]) {
  Pr3 ql = prim3<PP>(k, L), qr = prim3<PP>(k, R);
  if (!all_positive(ql.rho, ql.p, qr.rho, qr.p)) {
    fallback(L, R);
    ql = prim3<PP>(k, L);
    qr = prim3<PP>(k, R);
  }
  const float cL = Ar<float>::sqrt_pos(k.gamma * ql.p * ql.ir);
  const float cR = Ar<float>::sqrt_pos(k.gamma * qr.p * qr.ir);
  const float vl = vel<A>(ql), vr = vel<A>(qr);
  const float sl = fminf(fminf(vl - cL, vr - cR), 0.0f);
  const float sr = fmaxf(fmaxf(vl + cL, vr + cR), 0.0f);
  f2 FL[NP], FR[NP];
  flux3<PP, A>(k, L, ql, FL);
  flux3<PP, A>(k, R, qr, FR);
  const float inv = Ar<float>::rcp(sr - sl);
  const f2 wl = pk::splat(sr * inv), wr = pk::splat(-sl * inv), wd = pk::splat(sl * sr * inv);
#pragma unroll
  for (int p = 0; p < NP; ++p) F[p] = pk::fma(wd, pk::sub(R[p], L[p]), pk::fma(wl, FL[p], pk::mul(wr, FR[p])));
}

// Limited slopes of one pair of fields from its one-sided differences.
template <int LIM>
__device__ __forceinline__ f2 slope2(f2 a, f2 b) {
  return pk::pair(limit<LIM, float>(a.x, b.x), limit<LIM, float>(a.y, b.y));
}

// Shared memory: sU[NP][TY+2][TX+2] (plane q with the second ring), sW and sF
// [2][NP][NT] (x and y + states, x and y fluxes), sR[D][NP][NT] (own-column
// ring), sH[D][NP][NH] (second-ring ring); all field pairs.
template <int TX, int TY>
struct Lay3 {
  static constexpr int NT = TX * TY, SY = TY + 2, NH = 2 * TY + 2 * TX, D = kRing3;
  static constexpr size_t bytes =
      sizeof(f2) * ((size_t)NP * SY * (TX + 2) + 4 * (size_t)NP * NT + (size_t)D * NP * NT +
                    (size_t)D * NP * NH);
};

// field f of pair slot s as a float address (cp.async destination)
__device__ __forceinline__ float* half_of(f2* s, int f) {
  return reinterpret_cast<float*>(s) + (f & 1);
}

template <int PP, int LIM, int SRC, int TX, int TY, int MINB>
__global__ void __launch_bounds__(TX * TY, MINB)
stepnd3f_kernel(const KParams kp, float* __restrict__ bufA, float* __restrict__ bufB,
                Ctl* __restrict__ ctl, int64_t nx64, int64_t ny64, int64_t nz64, int tiles_x,
                int tiles_y, int nseg) {
  using G = Lay3<TX, TY>;
  constexpr int NT = G::NT, SY = G::SY, NH = G::NH, D = G::D;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  f2 (*sU)[SY][TX + 2] = reinterpret_cast<f2 (*)[SY][TX + 2]>(smem_raw);
  size_t off = sizeof(f2) * NP * SY * (TX + 2);
  f2 (*sW)[NP][NT] = reinterpret_cast<f2 (*)[NP][NT]>(smem_raw + off);
  off += sizeof(f2) * 2 * NP * NT;
  f2 (*sF)[NP][NT] = reinterpret_cast<f2 (*)[NP][NT]>(smem_raw + off);
  off += sizeof(f2) * 2 * NP * NT;
  f2 (*sR)[NP][NT] = reinterpret_cast<f2 (*)[NP][NT]>(smem_raw + off);
  off += sizeof(f2) * D * NP * NT;
  f2 (*sH)[NP][NH] = reinterpret_cast<f2 (*)[NP][NH]>(smem_raw + off);

  const StepCtl sc = block_step_ctl(ctl);
  if (!(sc.dt > 0.0)) return;
  const float* __restrict__ Uin = sc.cur ? bufB : bufA;
  float* __restrict__ Uout = sc.cur ? bufA : bufB;
  const P<float> k(kp);
  const StepDt<float> sd(sc);
  const f2 ndtdx = pk::splat(-sd.dtdx), ndt_2h = pk::splat(-sd.dt_2h);
  const f2 dt2 = pk::splat(sd.dt), dt_22 = pk::splat(sd.dt_2);
  const f2 half = pk::splat(0.5f), nhalf = pk::splat(-0.5f);

  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int seg = blockIdx.x % nseg;
  const int tile = blockIdx.x / nseg;
  const int tile_x = tile % tiles_x, tile_y = tile / tiles_x;
  // 32-bit offsets: the launch admits grids whose fields hold fewer than 2^31
  // values in all
  const int nx = (int)nx64, ny = (int)ny64, M = (int)nz64;
  const int gx = tile_x * (TX - 2) - 1 + tx, gy = tile_y * (TY - 2) - 1 + ty;
  const int plane = nx * ny, ncell = plane * M;
  const int q0 = (int)((int64_t)seg * M / nseg), q1 = (int)((int64_t)(seg + 1) * M / nseg);
  const bool interior = tx >= 1 && tx <= TX - 2 && gx < nx && ty >= 1 && ty <= TY - 2 && gy < ny;
  const int wx = wrap(gx, nx), wy = wrap(gy, ny);
  const int col = wy * nx + wx;
  // second-ring positions loaded by the halo threads
  const bool ringx = (tx == 0) || (tx == TX - 1), ringy = (ty == 0) || (ty == TY - 1);
  const int col_rx = wy * nx + wrap(gx + (tx == 0 ? -1 : 1), nx);
  const int col_ry = wrap(gy + (ty == 0 ? -1 : 1), ny) * nx + wx;
  const int oy = ty + 1;
  const int tid = threadIdx.x;
  const int hx = ty * 2 + (tx == 0 ? 0 : 1);                  // x-ring slot
  const int hy = 2 * TY + tx * 2 + (ty == 0 ? 0 : 1);         // y-ring slot

  float smax = 0.0f, akey = -INFINITY;
  uint32_t flags = 0;

  // copy plane p of the own column (p <= q1 + 1) and of the second ring
  // (p <= q1) into ring slot p mod D; always commit a group
  auto issue = [&](int p) {
    const int sl = p & (D - 1);
    if (p <= q1 + 1) {
      const int o = wrap(p, M) * plane;
#pragma unroll
      for (int f = 0; f < 2 * NP; ++f)
        cp_async<4>(half_of(&sR[sl][f >> 1][tid], f), Uin + f * ncell + o + col);
      if (p <= q1) {
        if (ringx)
#pragma unroll
          for (int f = 0; f < 2 * NP; ++f)
            cp_async<4>(half_of(&sH[sl][f >> 1][hx], f), Uin + f * ncell + o + col_rx);
        if (ringy)
#pragma unroll
          for (int f = 0; f < 2 * NP; ++f)
            cp_async<4>(half_of(&sH[sl][f >> 1][hy], f), Uin + f * ncell + o + col_ry);
      }
    }
    cp_async_commit();
  };

  f2 Wm_prev[NP], D_prev[NP], H_prev[NP], Y_prev = pk::splat(0.0f);
#pragma unroll
  for (int p = 0; p < NP; ++p) Wm_prev[p] = D_prev[p] = H_prev[p] = pk::splat(0.0f);
  for (int p = q0 - 2; p <= q0 + D - 4; ++p) issue(p);    // D - 1 planes ahead

  for (int q = q0 - 1; q <= q1; ++q) {
    // a. planes q-1, q, q+1 of the own column and plane q's second ring have
    //    landed; publish plane q
    cp_async_wait<D - 4>();
    const int sm = (q - 1) & (D - 1), s0 = q & (D - 1), sp = (q + 1) & (D - 1);
    f2 Um1[NP], Uq[NP], Up1[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      Um1[p] = sR[sm][p][tid];
      Uq[p] = sR[s0][p][tid];
      Up1[p] = sR[sp][p][tid];
      sU[p][oy][tx + 1] = Uq[p];
      if (ringx) sU[p][oy][tx == 0 ? 0 : TX + 1] = sH[s0][p][hx];
      if (ringy) sU[p][ty == 0 ? 0 : SY - 1][tx + 1] = sH[s0][p][hy];
    }
    issue(q + D - 2);    // reuses the slot of plane q-2 (read one barrier ago)
    __syncthreads();

    // b. slopes on the three axes, guard and half-step predictor of plane q
    f2 d[3][NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      d[0][p] = slope2<LIM>(pk::sub(Uq[p], sU[p][oy][tx]), pk::sub(sU[p][oy][tx + 2], Uq[p]));
      d[1][p] = slope2<LIM>(pk::sub(Uq[p], sU[p][oy - 1][tx + 1]), pk::sub(sU[p][oy + 1][tx + 1], Uq[p]));
      d[2][p] = slope2<LIM>(pk::sub(Uq[p], Um1[p]), pk::sub(Up1[p], Uq[p]));
    }
    f2 div[NP], dF[NP];
    bool ok = dflux3<PP, 0>(k, Uq, d[0], div);
    ok = dflux3<PP, 1>(k, Uq, d[1], dF) && ok;
#pragma unroll
    for (int p = 0; p < NP; ++p) div[p] = pk::add(div[p], dF[p]);
    ok = dflux3<PP, 2>(k, Uq, d[2], dF) && ok;
#pragma unroll
    for (int p = 0; p < NP; ++p) div[p] = pk::add(div[p], dF[p]);
    if (!ok) {
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        div[p] = pk::splat(0.0f);
#pragma unroll
        for (int a = 0; a < 3; ++a) d[a][p] = pk::splat(0.0f);
      }
    }
    f2 uh[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) uh[p] = pk::fma(ndt_2h, div[p], Uq[p]);
    if (SRC != 0) uh[2] = pk::fma(dt_22, source3<PP, SRC>(k, Uq), uh[2]);
    const f2 Yh = source3<PP, SRC>(k, uh);

    // c. transverse faces: publish the + states, take the left neighbour's
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      sW[0][p][tid] = pk::fma(half, d[0][p], uh[p]);
      sW[1][p][tid] = pk::fma(half, d[1][p], uh[p]);
    }
    __syncthreads();
    f2 Fx[NP], Fy[NP];
    {
      f2 l[NP], r[NP];
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        l[p] = sW[0][p][tx > 0 ? tid - 1 : tid];
        r[p] = pk::fma(nhalf, d[0][p], uh[p]);
      }
      hll3<PP, 0>(k, l, r,
                  [&](f2 (&L)[NP], f2 (&R)[NP]) {
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                      L[p] = sU[p][oy][tx];
                      R[p] = Uq[p];
                    }
                  },
                  Fx);
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        l[p] = sW[1][p][ty > 0 ? tid - TX : tid];
        r[p] = pk::fma(nhalf, d[1][p], uh[p]);
      }
      hll3<PP, 1>(k, l, r,
                  [&](f2 (&L)[NP], f2 (&R)[NP]) {
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                      L[p] = sU[p][oy - 1][tx + 1];
                      R[p] = Uq[p];
                    }
                  },
                  Fy);
    }
    // d. transverse flux divergence of plane q
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      sF[0][p][tid] = Fx[p];
      sF[1][p][tid] = Fy[p];
    }
    __syncthreads();
    f2 Dq[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p)
      Dq[p] = pk::add(pk::sub(sF[0][p][tx < TX - 1 ? tid + 1 : tid], Fx[p]),
                      pk::sub(sF[1][p][ty < TY - 1 ? tid + TX : tid], Fy[p]));

    // e. z face between planes q-1 and q
    f2 Hq[NP];
    {
      f2 Wm[NP];
#pragma unroll
      for (int p = 0; p < NP; ++p) Wm[p] = pk::fma(nhalf, d[2][p], uh[p]);
      hll3<PP, 2>(k, Wm_prev, Wm,
                  [&](f2 (&L)[NP], f2 (&R)[NP]) {
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                      L[p] = Um1[p];
                      R[p] = Uq[p];
                    }
                  },
                  Hq);
    }

    // f. update of plane q-1 and its eq. 16 bound
    if (q > q0 && interior) {
      f2 un[NP];
#pragma unroll
      for (int p = 0; p < NP; ++p)
        un[p] = pk::fma(ndtdx, pk::sub(pk::add(D_prev[p], Hq[p]), H_prev[p]), Um1[p]);
      if (SRC != 0) un[2] = pk::fma(dt2, Y_prev, un[2]);
      const int o = wrap(q - 1, M) * plane + col;
#pragma unroll
      for (int f = 0; f < 2 * NP; ++f) Uout[f * ncell + o] = (f & 1) ? un[f >> 1].y : un[f >> 1].x;
      if constexpr (PP == 3) {
        float v[2 * NP];
        fields6(un, v);
        psn::bound<3, SRC>(k, v, smax, akey, flags);
      } else {
        const Pr3 qn = prim3<PP>(k, un);
        const float v2 = fmaf(qn.vyz.y, qn.vyz.y, fmaf(qn.vyz.x, qn.vyz.x, qn.vx * qn.vx));
        cfl_cell<float, PP, SRC>(k, un[0].x, qn.kin2, speed_of<float>(v2), un[2].x, un[2].y,
                                 smax, akey, flags);
      }
    }

    // rotate the plane window
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      Wm_prev[p] = pk::fma(half, d[2][p], uh[p]);
      D_prev[p] = Dq[p];
      H_prev[p] = Hq[p];
    }
    Y_prev = Yh;
  }
  cp_async_wait<0>();
  reduce_and_finalize<float, NT>(ctl, kp, smax, akey, flags, true);
}

// The tile: 34 x 15 threads, 32 x 13 written columns (16 x-tiles on 512
// cells), one block per SM (about 128 registers per thread).
struct Tile3f {
  static constexpr int TX = 34, TY = 15, MINB = 1, SEG = 128;
};

template <int PP, int LIM, int SRC>
cudaError_t launch3f(const KParams& kp, void* a, void* b, Ctl* ctl, const int64_t* n, int seg,
                     cudaStream_t st) {
  using T = Tile3f;
  constexpr size_t smem = Lay3<T::TX, T::TY>::bytes;
  auto fn = stepnd3f_kernel<PP, LIM, SRC, T::TX, T::TY, T::MINB>;
  if (!n) return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int64_t nx = n[0], ny = n[1], nz = n[2];
  const int tiles_x = (int)((nx + T::TX - 3) / (T::TX - 2));
  const int tiles_y = (int)((ny + T::TY - 3) / (T::TY - 2));
  const int64_t sl = seg > 0 ? seg : T::SEG;
  int64_t nseg64 = (nz + sl - 1) / sl;
  if (nseg64 > nz) nseg64 = nz;
  const int nseg = nseg64 < 1 ? 1 : (int)nseg64;
  const int64_t blocks = (int64_t)tiles_x * tiles_y * nseg;
  if (blocks > 0x7fffffff) return cudaErrorInvalidConfiguration;
  fn<<<(int)blocks, T::TX * T::TY, smem, st>>>(kp, (float*)a, (float*)b, ctl, nx, ny, nz, tiles_x,
                                               tiles_y, nseg);
  return cudaGetLastError();
}

template <int PP, int LIM>
cudaError_t by_src3f(const KParams& kp, void* a, void* b, Ctl* ctl, const int64_t* n, int seg,
                     cudaStream_t st) {
  if (kp.frozen) return launch3f<PP, LIM, 0>(kp, a, b, ctl, n, seg, st);
  if (kp.qi_zero) return launch3f<PP, LIM, 1>(kp, a, b, ctl, n, seg, st);
  return launch3f<PP, LIM, 2>(kp, a, b, ctl, n, seg, st);
}

template <int PP>
cudaError_t by_lim3f(const KParams& kp, void* a, void* b, Ctl* ctl, const int64_t* n, int seg,
                     cudaStream_t st) {
  switch (kp.limiter) {
    case 1: return by_src3f<PP, 1>(kp, a, b, ctl, n, seg, st);
    case 2: return by_src3f<PP, 2>(kp, a, b, ctl, n, seg, st);
    default: return by_src3f<PP, 0>(kp, a, b, ctl, n, seg, st);
  }
}

}  // namespace
}  // namespace sv
