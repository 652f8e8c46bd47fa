// sv_pairnd.cuh -- the float 2D / 3D MUSCL-Hancock arithmetic (Sec. 2.3:
// eq. 14 reconstruction per axis with xi = 0, the unsplit half-step predictor,
// eq. 13 HLL per axis, eq. 15 update with the source Y, eq. 16 bound) on a
// pair of cells at once in packed f32x2 operations (FFMA2 / FADD2 / FMUL2).
//
// The pair is one thread's cells in two consecutive planes of the marching
// axis (sv_stepnd_pair.cu): component .x the lower plane, .y the upper one.
// Fields are (rho, rho v_1 .. rho v_DIM, E, E_nu), NF = DIM + 3; states are
// f2[NF] (field f of both cells in one register pair).
#pragma once

#include "sv_pair1d.cuh"
#include "sv_reduce.cuh"

namespace sv {
namespace pkn {

using pk::f2;
using pk::add;
using pk::fma;
using pk::mul;
using pk::pair;
using pk::rcp;
using pk::splat;
using pk::sub;

template <int DIM>
struct Prim {
  f2 ir, v[DIM], kin2, p;
};

// Primitive recovery (eq. 5, eq. 7) of two states; PP the pressure policy
// (pk::pressure: 0 float, 2 compensated float).
template <int DIM, int PP>
__device__ __forceinline__ Prim<DIM> prim(const P<float>& k, const f2 (&u)[DIM + 3]) {
  Prim<DIM> q;
  q.ir = rcp(u[0]);
#pragma unroll
  for (int a = 0; a < DIM; ++a) q.v[a] = mul(u[1 + a], q.ir);
  q.kin2 = mul(u[1], q.v[0]);
#pragma unroll
  for (int a = 1; a < DIM; ++a) q.kin2 = fma(u[1 + a], q.v[a], q.kin2);
  q.p = pk::pressure<PP>(k, q.kin2, u[1 + DIM], u[2 + DIM]);
  return q;
}

// Flux along axis A (F, G, H of eq. 15) of two states.
template <int DIM, int A>
__device__ __forceinline__ void flux(const f2 (&u)[DIM + 3], const Prim<DIM>& q, f2 (&F)[DIM + 3]) {
  F[0] = u[1 + A];
#pragma unroll
  for (int b = 0; b < DIM; ++b) F[1 + b] = b == A ? fma(u[1 + b], q.v[A], q.p) : mul(u[1 + b], q.v[A]);
  F[1 + DIM] = mul(q.v[A], add(u[1 + DIM], q.p));
  F[2 + DIM] = mul(q.v[A], u[2 + DIM]);
}

// F(u + d/2) - F(u - d/2) along axis A; ok0 / ok1 stay true while both
// extrapolated states of that cell are physical.
template <int DIM, int PP, int A>
__device__ __forceinline__ void dflux(const P<float>& k, const f2 (&u)[DIM + 3], const f2 (&d)[DIM + 3],
                                      f2 (&dF)[DIM + 3], bool& ok0, bool& ok1) {
  constexpr int NF = DIM + 3;
  f2 a[NF], b[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    a[f] = fma(splat(0.5f), d[f], u[f]);
    b[f] = fma(splat(-0.5f), d[f], u[f]);
  }
  const Prim<DIM> pa = prim<DIM, PP>(k, a), pb = prim<DIM, PP>(k, b);
  f2 Fa[NF], Fb[NF];
  flux<DIM, A>(a, pa, Fa);
  flux<DIM, A>(b, pb, Fb);
#pragma unroll
  for (int f = 0; f < NF; ++f) dF[f] = sub(Fa[f], Fb[f]);
  ok0 = ok0 && fminf(fminf(a[0].x, pa.p.x), fminf(b[0].x, pb.p.x)) > 0.0f;
  ok1 = ok1 && fminf(fminf(a[0].y, pa.p.y), fminf(b[0].y, pb.p.y)) > 0.0f;
}

// Components E and E_nu of Y (eq. 6 closures) of two states.
template <int DIM, int PP, int SRC>
__device__ __forceinline__ void source(const P<float>& k, const f2 (&u)[DIM + 3], f2& yE, f2& yEv) {
  yE = yEv = splat(0.0f);
  if (SRC == 0) return;
  const Prim<DIM> q = prim<DIM, PP>(k, u);
  pk::source<SRC>(k, u[0], mul(q.p, q.ir), u[2 + DIM], yE, yEv);
}

// eq. 13 along axis A at two faces with left states L and right states R; a
// face with a non-physical state uses the cell values, which `cells(fl, fr)`
// supplies (called on that rare path only, so a caller whose cell values sit
// in shared memory loads them only then).  Weights as in pk::hll (all
// non-negative).
template <int DIM, int PP, int A, typename CV>
__device__ __forceinline__ void hll(const P<float>& k, f2 (&L)[DIM + 3], f2 (&R)[DIM + 3],
                                    CV&& cells, f2 (&F)[DIM + 3]) {
  constexpr int NF = DIM + 3;
  Prim<DIM> pl = prim<DIM, PP>(k, L), pr = prim<DIM, PP>(k, R);
  const bool g0 = fminf(fminf(L[0].x, pl.p.x), fminf(R[0].x, pr.p.x)) > 0.0f;
  const bool g1 = fminf(fminf(L[0].y, pl.p.y), fminf(R[0].y, pr.p.y)) > 0.0f;
  if (!(g0 && g1)) {
    f2 fl[NF], fr[NF];
    cells(fl, fr);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      if (!g0) { L[f].x = fl[f].x; R[f].x = fr[f].x; }
      if (!g1) { L[f].y = fl[f].y; R[f].y = fr[f].y; }
    }
    pl = prim<DIM, PP>(k, L);
    pr = prim<DIM, PP>(k, R);
  }
  const f2 gam = splat(k.gamma);
  const f2 cL = pk::sqrt_pos(mul(mul(gam, pl.p), pl.ir));
  const f2 cR = pk::sqrt_pos(mul(mul(gam, pr.p), pr.ir));
  const f2 mL = sub(cL, pl.v[A]), mR = sub(cR, pr.v[A]);
  const f2 qL = add(pl.v[A], cL), qR = add(pr.v[A], cR);
  const f2 nsl = pair(fmaxf(fmaxf(mL.x, mR.x), 0.0f), fmaxf(fmaxf(mL.y, mR.y), 0.0f));
  const f2 sr = pair(fmaxf(fmaxf(qL.x, qR.x), 0.0f), fmaxf(fmaxf(qL.y, qR.y), 0.0f));
  f2 FL[NF], FR[NF];
  flux<DIM, A>(L, pl, FL);
  flux<DIM, A>(R, pr, FR);
  const f2 inv = rcp(add(sr, nsl));
  const f2 wl = mul(sr, inv), wr = mul(nsl, inv), wd = mul(mul(nsl, sr), inv);
#pragma unroll
  for (int f = 0; f < NF; ++f) F[f] = fma(wd, sub(L[f], R[f]), fma(wl, FL[f], mul(wr, FR[f])));
}

// eq. 16 signal speed and tau key of two updated states, folded for the cells
// whose mask bit is set (bit 0: .x, bit 1: .y).
template <int DIM, int PP, int SRC>
__device__ __forceinline__ void cfl(const P<float>& k, const f2 (&N)[DIM + 3], int mask, float& smax,
                                    float& akey, uint32_t& flags) {
  const Prim<DIM> q = prim<DIM, PP>(k, N);
  const f2 c = pk::sqrt_pos(mul(mul(splat(k.gamma), q.p), q.ir));
  f2 v2 = mul(q.v[0], q.v[0]);
#pragma unroll
  for (int a = 1; a < DIM; ++a) v2 = fma(q.v[a], q.v[a], v2);
  f2 key = splat(-INFINITY);
  if (SRC != 0) key = fma(splat(k.ntau_rho), pk::lg2(N[0]), mul(splat(k.ntau_T), pk::lg2(mul(q.p, q.ir))));
  const float vx = speed_of<float>(v2.x), vy = speed_of<float>(v2.y);
  if (mask & 1) {
    if ((N[0].x > 0.0f) && (q.p.x > 0.0f)) {
      smax = fmaxf(smax, fmaxf(2.0f * vx, vx + c.x));
      if (SRC != 0) akey = fmaxf(akey, key.x);
    } else {
      flags |= FLAG_NONPHYS;
    }
  }
  if (mask & 2) {
    if ((N[0].y > 0.0f) && (q.p.y > 0.0f)) {
      smax = fmaxf(smax, fmaxf(2.0f * vy, vy + c.y));
      if (SRC != 0) akey = fmaxf(akey, key.y);
    } else {
      flags |= FLAG_NONPHYS;
    }
  }
}

}  // namespace pkn
}  // namespace sv
