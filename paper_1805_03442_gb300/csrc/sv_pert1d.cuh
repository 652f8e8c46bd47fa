// sv_pert1d.cuh -- the float 1D MUSCL-Hancock arithmetic on perturbations
// about the uniform equilibrium (precision SV_FP32_PS): Sec. 2.3, eq. 14
// reconstruction with xi = 0, half-step predictor, eq. 13 HLL, eq. 15 update,
// the source Y of eqs. 4 and 6, and the eq. 16 bound.
//
// The device holds u = U - U_ref with U_ref = (1, 0, E0, E_nu0) the
// equilibrium rho = p = T = 1, v = 0, E_nu0 = C_k + S (R = 1; E0 = 1/(gamma-1)
// + E_nu0).  A float state of the full fields is rounded at ~6e-8 of the O(1)
// background every step; here the rounding scales with the perturbation.  Every
// quantity the step needs is formed so that the equilibrium part cancels
// algebraically before any rounding:
//   p - 1           = (gamma - 1)((dE - dE_nu) - rho v^2 / 2)
//   flux - F(U_ref) = (m, rho v^2 + (p - 1), v (E0 + p0 + dE + (p - 1)), v (E_nu0 + dE_nu))
//                     (the constant F(U_ref) = (0, 1, 0, 0) cancels in flux
//                     differences and passes through HLL, whose weights sum to 1)
//   rho C_k T - E_nu + rho Q tau = C_k (p - 1) - dE_nu + S expm1(a ln rho + b ln T),
//                     a = 1 + Q_rho + tau_rho, b = Q_T + tau_T (rho Q tau = S rho^a T^b
//                     with Q0 tau0 = S), so Y_Enu = (that) / tau
//   rho (Q - I)     = rho Q0 (expm1(Q_rho ln rho + Q_T ln T) - expm1(I_rho ln rho + I_T ln T))
// with ln rho = ln(1 + d rho) and ln T = ln(1 + (dp - d rho) / rho).  Only rates
// (1/tau, the sound speed, 1/rho) are formed from full values: they multiply
// perturbation-sized quantities, so their relative rounding stays relative.
#pragma once

#include "sv_model.cuh"
#include "sv_pair1d.cuh"
#include "sv_reduce.cuh"

namespace sv {
namespace ps {

struct Prim {
  float rho, ir, v, kin2, dp, p;
};

__device__ __forceinline__ Prim prim(const P<float>& k, const float (&u)[4]) {
  Prim q;
  q.rho = 1.0f + u[0];
  q.ir = Ar<float>::rcp(q.rho);
  q.v = u[1] * q.ir;
  q.kin2 = u[1] * q.v;
  q.dp = k.g1 * fmaf(q.kin2, -0.5f, u[2] - u[3]);
  q.p = 1.0f + q.dp;
  return q;
}

// ln(1 + x) and exp(y) - 1 with relative accuracy near 0.  Perturbations of
// the linear stage are small, so the Mercator series of ln(1 + x) and the
// exponential series (textbook Taylor coefficients 1/n and 1/n!, Horner form)
// cover |x| < 1/16 with a truncation below 1e-8 relative (six terms: (1/16)^6
// / 7 and (1/16)^6 / 7!); larger arguments go to the CUDA math library.
__device__ __forceinline__ float ln1p(float x) {
  if (fabsf(x) < 0.0625f) {
    float s = -1.0f / 6.0f;
    s = fmaf(s, x, 1.0f / 5.0f);
    s = fmaf(s, x, -1.0f / 4.0f);
    s = fmaf(s, x, 1.0f / 3.0f);
    s = fmaf(s, x, -1.0f / 2.0f);
    s = fmaf(s, x, 1.0f);
    return s * x;
  }
  return log1pf(x);
}
__device__ __forceinline__ float em1(float y) {
  if (fabsf(y) < 0.0625f) {
    float s = 1.0f / 720.0f;
    s = fmaf(s, y, 1.0f / 120.0f);
    s = fmaf(s, y, 1.0f / 24.0f);
    s = fmaf(s, y, 1.0f / 6.0f);
    s = fmaf(s, y, 1.0f / 2.0f);
    s = fmaf(s, y, 1.0f);
    return s * y;
  }
  return expm1f(y);
}

// eq. 16 bound and physicality of one perturbed state.
template <int SRC>
__device__ __forceinline__ void bound(const P<float>& k, const float (&u)[4], float& smax,
                                      float& akey, uint32_t& flags) {
  const Prim q = prim(k, u);
  if (!((q.rho > 0.0f) && (q.p > 0.0f))) {
    flags |= FLAG_NONPHYS;
    return;
  }
  const float vmag = fabsf(q.v);
  const float c = Ar<float>::sqrt_pos(k.gamma * q.p * q.ir);
  smax = fmaxf(smax, fmaxf(2.0f * vmag, vmag + c));
  if (SRC != 0) akey = fmaxf(akey, TauKey<float>::of(k, q.rho, q.p * q.ir));
}

}  // namespace ps

// ------------------------------------------------------------------ packed
// The step itself runs on a lane's two cells in packed f32x2 operations (as
// sv_pair1d.cuh does for the full-state policies): component .x the even
// cell, .y the odd one.  The one-cell ps:: functions above serve the eq. 16
// bound of an uploaded state and the per-component fallback of the series.
namespace pkps {

using pk::add;
using pk::f2;
using pk::fma;
using pk::mul;
using pk::pair;
using pk::rcp;
using pk::splat;
using pk::sub;

struct Prim {
  f2 rho, ir, v, kin2, dp, p;
};

__device__ __forceinline__ Prim prim(const P<float>& k, const f2 (&u)[4]) {
  Prim q;
  q.rho = add(splat(1.0f), u[0]);
  q.ir = rcp(q.rho);
  q.v = mul(u[1], q.ir);
  q.kin2 = mul(u[1], q.v);
  q.dp = mul(splat(k.g1), fma(q.kin2, splat(-0.5f), sub(u[2], u[3])));
  q.p = add(splat(1.0f), q.dp);
  return q;
}

__device__ __forceinline__ void flux(const P<float>& k, const f2 (&u)[4], const Prim& q,
                                     f2 (&F)[4]) {
  F[0] = u[1];
  F[1] = add(q.kin2, q.dp);
  F[2] = mul(q.v, add(splat(k.h0), add(u[2], q.dp)));
  F[3] = mul(q.v, add(splat(k.ev0), u[3]));
}

// ps::ln1p / ps::em1 on a pair: the series in packed form when both
// arguments are small, else per component.
__device__ __forceinline__ f2 ln1p(f2 x) {
  if (fabsf(x.x) < 0.0625f && fabsf(x.y) < 0.0625f) {
    f2 s = splat(-1.0f / 6.0f);
    s = fma(s, x, splat(1.0f / 5.0f));
    s = fma(s, x, splat(-1.0f / 4.0f));
    s = fma(s, x, splat(1.0f / 3.0f));
    s = fma(s, x, splat(-1.0f / 2.0f));
    s = fma(s, x, splat(1.0f));
    return mul(s, x);
  }
  return pair(ps::ln1p(x.x), ps::ln1p(x.y));
}
__device__ __forceinline__ f2 em1(f2 y) {
  if (fabsf(y.x) < 0.0625f && fabsf(y.y) < 0.0625f) {
    f2 s = splat(1.0f / 720.0f);
    s = fma(s, y, splat(1.0f / 120.0f));
    s = fma(s, y, splat(1.0f / 24.0f));
    s = fma(s, y, splat(1.0f / 6.0f));
    s = fma(s, y, splat(1.0f / 2.0f));
    s = fma(s, y, splat(1.0f));
    return mul(s, y);
  }
  return pair(ps::em1(y.x), ps::em1(y.y));
}

template <int SRC>
__device__ __forceinline__ void source(const P<float>& k, const f2 (&u)[4], const Prim& q, f2& yE,
                                       f2& yEv) {
  yE = yEv = splat(0.0f);
  if (SRC == 0) return;
  const f2 lr = ln1p(u[0]);
  const f2 lT = ln1p(mul(sub(q.dp, u[0]), q.ir));
  const f2 inv_tau = pk::ex2(fma(splat(1.44269504f), fma(splat(k.ntau_rho), lr, mul(splat(k.ntau_T), lT)),
                                 splat(k.l2_inv_tau0)));
  const float a = 1.0f + k.Q_rho + k.tau_rho, b = k.Q_T + k.tau_T;
  const f2 relax = fma(splat(k.S), em1(fma(splat(a), lr, mul(splat(b), lT))),
                       fma(splat(k.Ck), q.dp, mul(u[3], splat(-1.0f))));
  yEv = mul(relax, inv_tau);
  if (SRC == 2)
    yE = mul(mul(q.rho, splat(k.Q0)), sub(em1(fma(splat(k.Q_rho), lr, mul(splat(k.Q_T), lT))),
                                          em1(fma(splat(k.I_rho), lr, mul(splat(k.I_T), lT)))));
}

template <int LIM, int SRC>
__device__ __forceinline__ void predict(const P<float>& k, const f2 (&X)[4], const f2 (&A)[4],
                                        const f2 (&B)[4], f2 ndt_2h, f2 dt_2, f2 (&WP)[4],
                                        f2 (&WM)[4], f2& yEh, f2& yEvh) {
  f2 d[4], a[4], b[4];
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    d[f] = pair(pk::slope<LIM>(A[f].x, B[f].x), pk::slope<LIM>(A[f].y, B[f].y));
    a[f] = fma(splat(0.5f), d[f], X[f]);
    b[f] = fma(splat(-0.5f), d[f], X[f]);
  }
  const Prim qa = prim(k, a), qb = prim(k, b);
  f2 Fa[4], Fb[4], dF[4];
  flux(k, a, qa, Fa);
  flux(k, b, qb, Fb);
#pragma unroll
  for (int f = 0; f < 4; ++f) dF[f] = sub(Fa[f], Fb[f]);
  const bool g0 = fminf(fminf(qa.rho.x, qa.p.x), fminf(qb.rho.x, qb.p.x)) > 0.0f;
  const bool g1 = fminf(fminf(qa.rho.y, qa.p.y), fminf(qb.rho.y, qb.p.y)) > 0.0f;
  if (!(g0 && g1)) {
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      if (!g0) d[f].x = dF[f].x = 0.0f;
      if (!g1) d[f].y = dF[f].y = 0.0f;
    }
  }
  f2 yE = splat(0.0f), yEv = splat(0.0f);
  if (SRC != 0) source<SRC>(k, X, prim(k, X), yE, yEv);
  f2 uh[4];
  uh[0] = fma(ndt_2h, dF[0], X[0]);
  uh[1] = fma(ndt_2h, dF[1], X[1]);
  uh[2] = fma(ndt_2h, dF[2], X[2]);
  if (SRC == 2) uh[2] = fma(dt_2, yE, uh[2]);
  uh[3] = fma(dt_2, yEv, fma(ndt_2h, dF[3], X[3]));
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    WP[f] = fma(splat(0.5f), d[f], uh[f]);
    WM[f] = fma(splat(-0.5f), d[f], uh[f]);
  }
  yEh = yEvh = splat(0.0f);
  if (SRC != 0) source<SRC>(k, uh, prim(k, uh), yEh, yEvh);
}

__device__ __forceinline__ void hll(const P<float>& k, f2 (&L)[4], f2 (&R)[4], const float (&xl)[4],
                                    const f2 (&X)[4], f2 (&F)[4]) {
  Prim ql = prim(k, L), qr = prim(k, R);
  const bool g0 = fminf(fminf(ql.rho.x, ql.p.x), fminf(qr.rho.x, qr.p.x)) > 0.0f;
  const bool g1 = fminf(fminf(ql.rho.y, ql.p.y), fminf(qr.rho.y, qr.p.y)) > 0.0f;
  if (!(g0 && g1)) {
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      if (!g0) { L[f].x = xl[f]; R[f].x = X[f].x; }
      if (!g1) { L[f].y = X[f].x; R[f].y = X[f].y; }
    }
    ql = prim(k, L);
    qr = prim(k, R);
  }
  const f2 gam = splat(k.gamma);
  const f2 cL = pk::sqrt_pos(mul(mul(gam, ql.p), ql.ir));
  const f2 cR = pk::sqrt_pos(mul(mul(gam, qr.p), qr.ir));
  const f2 mL = sub(cL, ql.v), mR = sub(cR, qr.v);
  const f2 qL = add(ql.v, cL), qR = add(qr.v, cR);
  const f2 nsl = pair(fmaxf(fmaxf(mL.x, mR.x), 0.0f), fmaxf(fmaxf(mL.y, mR.y), 0.0f));
  const f2 sr = pair(fmaxf(fmaxf(qL.x, qR.x), 0.0f), fmaxf(fmaxf(qL.y, qR.y), 0.0f));
  f2 FL[4], FR[4];
  flux(k, L, ql, FL);
  flux(k, R, qr, FR);
  const f2 inv = rcp(add(sr, nsl));
  const f2 wl = mul(sr, inv), wr = mul(nsl, inv), wd = mul(mul(nsl, sr), inv);
#pragma unroll
  for (int f = 0; f < 4; ++f) F[f] = fma(wd, sub(L[f], R[f]), fma(wl, FL[f], mul(wr, FR[f])));
}

template <int SRC>
__device__ __forceinline__ void cfl(const P<float>& k, const f2 (&N)[4], int mask, float& smax,
                                    float& akey, uint32_t& flags) {
  const Prim q = prim(k, N);
  const f2 c = pk::sqrt_pos(mul(mul(splat(k.gamma), q.p), q.ir));
  f2 key = splat(-INFINITY);
  if (SRC != 0)
    key = fma(splat(k.ntau_rho), pk::lg2(q.rho), mul(splat(k.ntau_T), pk::lg2(mul(q.p, q.ir))));
  const float vx = fabsf(q.v.x), vy = fabsf(q.v.y);
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

}  // namespace pkps

// The packed step functions by pressure policy / layout: PP 0 and 2 the
// full-state pair arithmetic (sv_pair1d.cuh), PP 3 the perturbation layout.
namespace pkx {

template <int PP, int LIM, int SRC>
__device__ __forceinline__ void predict(const P<float>& k, const pk::f2 (&X)[4],
                                        const pk::f2 (&A)[4], const pk::f2 (&B)[4], pk::f2 ndt_2h,
                                        pk::f2 dt_2, pk::f2 (&WP)[4], pk::f2 (&WM)[4],
                                        pk::f2& yEh, pk::f2& yEvh) {
  if constexpr (PP == 3) pkps::predict<LIM, SRC>(k, X, A, B, ndt_2h, dt_2, WP, WM, yEh, yEvh);
  else pk::predict<PP, LIM, SRC>(k, X, A, B, ndt_2h, dt_2, WP, WM, yEh, yEvh);
}

template <int PP>
__device__ __forceinline__ void hll(const P<float>& k, pk::f2 (&L)[4], pk::f2 (&R)[4],
                                    const float (&xl)[4], const pk::f2 (&X)[4], pk::f2 (&F)[4]) {
  if constexpr (PP == 3) pkps::hll(k, L, R, xl, X, F);
  else pk::hll<PP>(k, L, R, xl, X, F);
}

template <int PP, int SRC>
__device__ __forceinline__ void cfl(const P<float>& k, const pk::f2 (&N)[4], int mask,
                                    float& smax, float& akey, uint32_t& flags) {
  if constexpr (PP == 3) pkps::cfl<SRC>(k, N, mask, smax, akey, flags);
  else pk::cfl<PP, SRC>(k, N, mask, smax, akey, flags);
}

}  // namespace pkx

// eq. 16 bound of one 1D cell state u (rho, rho v, E, E_nu), or of its
// perturbation (PP = 3), folded into the caller's maxima.
template <typename R, int PP, int SRC>
__device__ __forceinline__ void cell_bound(const P<R>& k, const R (&u)[4], R& smax, R& akey,
                                           uint32_t& flags) {
  if constexpr (PP == 3) {
    ps::bound<SRC>(k, u, smax, akey, flags);
  } else {
    const R v = u[1] * Ar<R>::rcp(u[0]);
    cfl_cell<R, PP, SRC>(k, u[0], u[1] * v, fabs(v), u[2], u[3], smax, akey, flags);
  }
}

}  // namespace sv
