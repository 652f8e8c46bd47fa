// sv_pertnd.cuh -- the perturbation layout (SV_FP32_PS) of the 2D / 3D
// unsplit steps: the arithmetic of sv_pert1d.cuh with DIM velocity
// components, for one cell (psn::, the source and the eq. 16 bound of the 3D
// field-pair kernel and of the dt of an uploaded state) and for a thread's
// two cells in packed f32x2 (pknps::, the 2D plane-pair kernel).  The 3D
// kernel forms its fluxes in field pairs itself (sv_stepnd3f.cuh).
//
// u = U - U_ref, U_ref = (1, 0 .. 0, E0, E_nu0); fields (rho, rho v_1 ..
// rho v_DIM, E, E_nu), NF = DIM + 3.  Along axis A the flux less F(U_ref)
// (whose only non-zero entry is p0 = 1 in the momentum of axis A) is
//   (m_A, m_b v_A + (p - 1) [b = A], v_A (E0 + p0 + dE + (p - 1)), v_A (E_nu0 + dE_nu)).
#pragma once

#include "sv_pairnd.cuh"
#include "sv_pert1d.cuh"

namespace sv {

// The pulsating source of the 2D medium map (pulse_state of sv_ndbnd.cuh) as
// a perturbation: each field's difference to U_ref taken in double.
template <int NF>
__device__ __forceinline__ void pulse_state_ps(const KParams& kp, double t, float (&u)[NF]) {
  const double s = kp.pul_amp * sin(kp.pul_omega * t);
  const double rho = 1.0 + s, p = 1.0 + kp.gamma * s, Ev = rho * kp.pul_ev;
#pragma unroll
  for (int f = 0; f < NF; ++f) u[f] = 0.0f;
  u[0] = (float)s;
  u[NF - 2] = (float)((p / kp.g1 + Ev) - kp.ref[2]);
  u[NF - 1] = (float)(Ev - kp.ref[3]);
}

namespace psn {

template <int DIM>
struct Prim {
  float rho, ir, v[DIM], v2, kin2, dp, p;
};

template <int DIM>
__device__ __forceinline__ Prim<DIM> prim(const P<float>& k, const float (&u)[DIM + 3]) {
  Prim<DIM> q;
  q.rho = 1.0f + u[0];
  q.ir = Ar<float>::rcp(q.rho);
  q.kin2 = 0.0f;
  q.v2 = 0.0f;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    q.v[a] = u[1 + a] * q.ir;
    q.kin2 += u[1 + a] * q.v[a];
    q.v2 += q.v[a] * q.v[a];
  }
  q.dp = k.g1 * fmaf(q.kin2, -0.5f, u[1 + DIM] - u[2 + DIM]);
  q.p = 1.0f + q.dp;
  return q;
}

template <int DIM, int SRC>
__device__ __forceinline__ void source(const P<float>& k, const float (&u)[DIM + 3],
                                       const Prim<DIM>& q, float& yE, float& yEv) {
  yE = yEv = 0.0f;
  if (SRC == 0) return;
  const float lr = ps::ln1p(u[0]);
  const float lT = ps::ln1p((q.dp - u[0]) * q.ir);
  const float inv_tau =
      Ar<float>::ex2(fmaf(1.44269504f, fmaf(k.ntau_rho, lr, k.ntau_T * lT), k.l2_inv_tau0));
  const float a = 1.0f + k.Q_rho + k.tau_rho, b = k.Q_T + k.tau_T;
  const float relax = fmaf(k.Ck, q.dp, -u[2 + DIM]) + k.S * ps::em1(fmaf(a, lr, b * lT));
  yEv = relax * inv_tau;
  if (SRC == 2)
    yE = q.rho * k.Q0 *
         (ps::em1(fmaf(k.Q_rho, lr, k.Q_T * lT)) - ps::em1(fmaf(k.I_rho, lr, k.I_T * lT)));
}

template <int DIM, int SRC>
__device__ __forceinline__ void bound(const P<float>& k, const float (&u)[DIM + 3], float& smax,
                                      float& akey, uint32_t& flags) {
  const Prim<DIM> q = prim<DIM>(k, u);
  if (!((q.rho > 0.0f) && (q.p > 0.0f))) {
    flags |= FLAG_NONPHYS;
    return;
  }
  const float vmag = speed_of<float>(q.v2);
  const float c = Ar<float>::sqrt_pos(k.gamma * q.p * q.ir);
  smax = fmaxf(smax, fmaxf(2.0f * vmag, vmag + c));
  if (SRC != 0) akey = fmaxf(akey, TauKey<float>::of(k, q.rho, q.p * q.ir));
}

}  // namespace psn

// ------------------------------------------------------------------ packed
namespace pknps {

using pk::add;
using pk::f2;
using pk::fma;
using pk::mul;
using pk::pair;
using pk::rcp;
using pk::splat;
using pk::sub;

template <int DIM>
struct Prim {
  f2 rho, ir, v[DIM], kin2, dp, p;
};

template <int DIM>
__device__ __forceinline__ Prim<DIM> prim(const P<float>& k, const f2 (&u)[DIM + 3]) {
  Prim<DIM> q;
  q.rho = add(splat(1.0f), u[0]);
  q.ir = rcp(q.rho);
#pragma unroll
  for (int a = 0; a < DIM; ++a) q.v[a] = mul(u[1 + a], q.ir);
  q.kin2 = mul(u[1], q.v[0]);
#pragma unroll
  for (int a = 1; a < DIM; ++a) q.kin2 = fma(u[1 + a], q.v[a], q.kin2);
  q.dp = mul(splat(k.g1), fma(q.kin2, splat(-0.5f), sub(u[1 + DIM], u[2 + DIM])));
  q.p = add(splat(1.0f), q.dp);
  return q;
}

template <int DIM, int A>
__device__ __forceinline__ void flux(const P<float>& k, const f2 (&u)[DIM + 3], const Prim<DIM>& q,
                                     f2 (&F)[DIM + 3]) {
  F[0] = u[1 + A];
#pragma unroll
  for (int b = 0; b < DIM; ++b) F[1 + b] = b == A ? fma(u[1 + b], q.v[A], q.dp) : mul(u[1 + b], q.v[A]);
  F[1 + DIM] = mul(q.v[A], add(splat(k.h0), add(u[1 + DIM], q.dp)));
  F[2 + DIM] = mul(q.v[A], add(splat(k.ev0), u[2 + DIM]));
}

template <int DIM, int A>
__device__ __forceinline__ void dflux(const P<float>& k, const f2 (&u)[DIM + 3],
                                      const f2 (&d)[DIM + 3], f2 (&dF)[DIM + 3], bool& ok0,
                                      bool& ok1) {
  constexpr int NF = DIM + 3;
  f2 a[NF], b[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    a[f] = fma(splat(0.5f), d[f], u[f]);
    b[f] = fma(splat(-0.5f), d[f], u[f]);
  }
  const Prim<DIM> pa = prim<DIM>(k, a), pb = prim<DIM>(k, b);
  f2 Fa[NF], Fb[NF];
  flux<DIM, A>(k, a, pa, Fa);
  flux<DIM, A>(k, b, pb, Fb);
#pragma unroll
  for (int f = 0; f < NF; ++f) dF[f] = sub(Fa[f], Fb[f]);
  ok0 = ok0 && fminf(fminf(pa.rho.x, pa.p.x), fminf(pb.rho.x, pb.p.x)) > 0.0f;
  ok1 = ok1 && fminf(fminf(pa.rho.y, pa.p.y), fminf(pb.rho.y, pb.p.y)) > 0.0f;
}

template <int DIM, int SRC>
__device__ __forceinline__ void source(const P<float>& k, const f2 (&u)[DIM + 3], f2& yE, f2& yEv) {
  yE = yEv = splat(0.0f);
  if (SRC == 0) return;
  const Prim<DIM> q = prim<DIM>(k, u);
  const f2 lr = pkps::ln1p(u[0]);
  const f2 lT = pkps::ln1p(mul(sub(q.dp, u[0]), q.ir));
  const f2 inv_tau = pk::ex2(fma(splat(1.44269504f), fma(splat(k.ntau_rho), lr, mul(splat(k.ntau_T), lT)),
                                 splat(k.l2_inv_tau0)));
  const float a = 1.0f + k.Q_rho + k.tau_rho, b = k.Q_T + k.tau_T;
  const f2 relax = fma(splat(k.S), pkps::em1(fma(splat(a), lr, mul(splat(b), lT))),
                       fma(splat(k.Ck), q.dp, mul(u[2 + DIM], splat(-1.0f))));
  yEv = mul(relax, inv_tau);
  if (SRC == 2)
    yE = mul(mul(q.rho, splat(k.Q0)), sub(pkps::em1(fma(splat(k.Q_rho), lr, mul(splat(k.Q_T), lT))),
                                          pkps::em1(fma(splat(k.I_rho), lr, mul(splat(k.I_T), lT)))));
}

template <int DIM, int A, typename CV>
__device__ __forceinline__ void hll(const P<float>& k, f2 (&L)[DIM + 3], f2 (&R)[DIM + 3],
                                    CV&& cells, f2 (&F)[DIM + 3]) {
  constexpr int NF = DIM + 3;
  Prim<DIM> pl = prim<DIM>(k, L), pr = prim<DIM>(k, R);
  const bool g0 = fminf(fminf(pl.rho.x, pl.p.x), fminf(pr.rho.x, pr.p.x)) > 0.0f;
  const bool g1 = fminf(fminf(pl.rho.y, pl.p.y), fminf(pr.rho.y, pr.p.y)) > 0.0f;
  if (!(g0 && g1)) {
    f2 fl[NF], fr[NF];
    cells(fl, fr);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      if (!g0) { L[f].x = fl[f].x; R[f].x = fr[f].x; }
      if (!g1) { L[f].y = fl[f].y; R[f].y = fr[f].y; }
    }
    pl = prim<DIM>(k, L);
    pr = prim<DIM>(k, R);
  }
  const f2 gam = splat(k.gamma);
  const f2 cL = pk::sqrt_pos(mul(mul(gam, pl.p), pl.ir));
  const f2 cR = pk::sqrt_pos(mul(mul(gam, pr.p), pr.ir));
  const f2 mL = sub(cL, pl.v[A]), mR = sub(cR, pr.v[A]);
  const f2 qL = add(pl.v[A], cL), qR = add(pr.v[A], cR);
  const f2 nsl = pair(fmaxf(fmaxf(mL.x, mR.x), 0.0f), fmaxf(fmaxf(mL.y, mR.y), 0.0f));
  const f2 sr = pair(fmaxf(fmaxf(qL.x, qR.x), 0.0f), fmaxf(fmaxf(qL.y, qR.y), 0.0f));
  f2 FL[NF], FR[NF];
  flux<DIM, A>(k, L, pl, FL);
  flux<DIM, A>(k, R, pr, FR);
  const f2 inv = rcp(add(sr, nsl));
  const f2 wl = mul(sr, inv), wr = mul(nsl, inv), wd = mul(mul(nsl, sr), inv);
#pragma unroll
  for (int f = 0; f < NF; ++f) F[f] = fma(wd, sub(L[f], R[f]), fma(wl, FL[f], mul(wr, FR[f])));
}

template <int DIM, int SRC>
__device__ __forceinline__ void cfl(const P<float>& k, const f2 (&N)[DIM + 3], int mask, float& smax,
                                    float& akey, uint32_t& flags) {
  const Prim<DIM> q = prim<DIM>(k, N);
  const f2 c = pk::sqrt_pos(mul(mul(splat(k.gamma), q.p), q.ir));
  f2 v2 = mul(q.v[0], q.v[0]);
#pragma unroll
  for (int a = 1; a < DIM; ++a) v2 = fma(q.v[a], q.v[a], v2);
  f2 key = splat(-INFINITY);
  if (SRC != 0)
    key = fma(splat(k.ntau_rho), pk::lg2(q.rho), mul(splat(k.ntau_T), pk::lg2(mul(q.p, q.ir))));
  const float vx = speed_of<float>(v2.x), vy = speed_of<float>(v2.y);
  if (mask & 1) {
    if ((q.rho.x > 0.0f) && (q.p.x > 0.0f)) {
      smax = fmaxf(smax, fmaxf(2.0f * vx, vx + c.x));
      if (SRC != 0) akey = fmaxf(akey, key.x);
    } else {
      flags |= FLAG_NONPHYS;
    }
  }
  if (mask & 2) {
    if ((q.rho.y > 0.0f) && (q.p.y > 0.0f)) {
      smax = fmaxf(smax, fmaxf(2.0f * vy, vy + c.y));
      if (SRC != 0) akey = fmaxf(akey, key.y);
    } else {
      flags |= FLAG_NONPHYS;
    }
  }
}

}  // namespace pknps
}  // namespace sv

namespace sv {

// The packed 2D step functions by pressure policy / layout: PP 0 and 2 the
// full-state pair arithmetic (sv_pairnd.cuh), PP 3 the perturbation layout.
namespace pknx {

template <int DIM, int PP, int A>
__device__ __forceinline__ void dflux(const P<float>& k, const pk::f2 (&u)[DIM + 3],
                                      const pk::f2 (&d)[DIM + 3], pk::f2 (&dF)[DIM + 3], bool& ok0,
                                      bool& ok1) {
  if constexpr (PP == 3) pknps::dflux<DIM, A>(k, u, d, dF, ok0, ok1);
  else pkn::dflux<DIM, PP, A>(k, u, d, dF, ok0, ok1);
}

template <int DIM, int PP, int SRC>
__device__ __forceinline__ void source(const P<float>& k, const pk::f2 (&u)[DIM + 3], pk::f2& yE,
                                       pk::f2& yEv) {
  if constexpr (PP == 3) pknps::source<DIM, SRC>(k, u, yE, yEv);
  else pkn::source<DIM, PP, SRC>(k, u, yE, yEv);
}

template <int DIM, int PP, int A, typename CV>
__device__ __forceinline__ void hll(const P<float>& k, pk::f2 (&L)[DIM + 3], pk::f2 (&R)[DIM + 3],
                                    CV&& cells, pk::f2 (&F)[DIM + 3]) {
  if constexpr (PP == 3) pknps::hll<DIM, A>(k, L, R, cells, F);
  else pkn::hll<DIM, PP, A>(k, L, R, cells, F);
}

template <int DIM, int PP, int SRC>
__device__ __forceinline__ void cfl(const P<float>& k, const pk::f2 (&N)[DIM + 3], int mask,
                                    float& smax, float& akey, uint32_t& flags) {
  if constexpr (PP == 3) pknps::cfl<DIM, SRC>(k, N, mask, smax, akey, flags);
  else pkn::cfl<DIM, PP, SRC>(k, N, mask, smax, akey, flags);
}

}  // namespace pknx
}  // namespace sv
