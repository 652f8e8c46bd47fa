// sv_pair1d.cuh -- the float MUSCL-Hancock arithmetic of one lane's two cells
// (Sec. 2.3: eq. 14 reconstruction with xi = 0, the half-step predictor, eq. 13
// HLL, eq. 15 update with the source Y, and the eq. 16 bound of the result)
// carried out on both cells at once with the packed f32x2 instructions of
// sm_100+ (FFMA2 / FADD2 / FMUL2).
//
// The scalar kernel body computes the two cells of a lane with identical
// instruction sequences; here every add, multiply and fused multiply-add is
// issued once for the pair, which halves the floating-point issue slots of
// the step.  The SFU approximations (rcp, rsqrt, lg2, ex2), min/max and the
// comparisons have no packed form and stay per cell.  Each packed operation
// rounds each component exactly as the scalar one does, so the two bodies
// differ only where the scalar code leaves the fusing of a multiply and an
// add to the compiler.
//
// Component .x is the lane's even cell (or the face left of it), .y the odd
// one.
#pragma once

#include "sv_model.cuh"

namespace sv {
namespace pk {

using f2 = float2;

__device__ __forceinline__ f2 pair(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ f2 splat(float a) { return make_float2(a, a); }
__device__ __forceinline__ f2 add(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 mul(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
// a - b with one rounding (b * -1 is exact)
__device__ __forceinline__ f2 sub(f2 a, f2 b) { return __ffma2_rn(b, splat(-1.0f), a); }
__device__ __forceinline__ f2 rcp(f2 a) { return pair(Ar<float>::rcp(a.x), Ar<float>::rcp(a.y)); }
__device__ __forceinline__ f2 lg2(f2 a) { return pair(Ar<float>::lg2(a.x), Ar<float>::lg2(a.y)); }
__device__ __forceinline__ f2 ex2(f2 a) { return pair(Ar<float>::ex2(a.x), Ar<float>::ex2(a.y)); }
// sqrt of a positive argument as x * rsqrt(x), as the scalar kernels do
__device__ __forceinline__ f2 sqrt_pos(f2 a) {
  return mul(a, pair(Ar<float>::rsqrt(a.x), Ar<float>::rsqrt(a.y)));
}

// the limiter per component (minmod: three ALU instructions, sv_model.cuh)
template <int LIM>
__device__ __forceinline__ float slope(float a, float b) {
  return limit<LIM, float>(a, b);
}

// eq. 5 of two states, rho |v|^2 = kin2 given: PP = 0 in float (E - E_nu
// first, as pressure<float, 0>), PP = 2 in compensated float (the
// pressure<float, 2> policy); component by component, each packed add,
// subtract and fused multiply-add rounds as the scalar one.
template <int PP>
__device__ __forceinline__ f2 pressure(const P<float>& k, f2 kin2, f2 E, f2 Ev) {
  static_assert(PP == 0 || PP == 2, "packed pressure policies: float or compensated float");
  if constexpr (PP == 2) {
    const f2 h = mul(splat(0.5f), kin2);
    const f2 s = sub(E, Ev);
    const f2 e1 = sub(sub(E, s), Ev);
    const f2 t = sub(s, h);
    const f2 e2 = sub(sub(s, t), h);
    return fma(splat(k.g1), t, fma(splat(k.g1lo), t, mul(splat(k.g1), add(e1, e2))));
  } else {
    return mul(splat(k.g1), fma(kin2, splat(-0.5f), sub(E, Ev)));
  }
}

// Primitive recovery (eq. 5, eq. 7) of two states: 1/rho, v, rho v^2, p.
struct Prim {
  f2 ir, v, kin2, p;
};
template <int PP>
__device__ __forceinline__ Prim prim(const P<float>& k, const f2 (&u)[4]) {
  Prim q;
  q.ir = rcp(u[0]);
  q.v = mul(u[1], q.ir);
  q.kin2 = mul(u[1], q.v);
  q.p = pressure<PP>(k, q.kin2, u[2], u[3]);
  return q;
}

// Components E and E_nu of Y (eq. 6 closures), as Src<float, SRC>.
template <int SRC>
__device__ __forceinline__ void source(const P<float>& k, f2 rho, f2 T, f2 Ev, f2& yE, f2& yEv) {
  yE = splat(0.0f);
  if (SRC == 0) {
    yEv = splat(0.0f);
    return;
  }
  const f2 lr = lg2(rho), lT = lg2(T);
  const f2 inv_tau = ex2(fma(splat(k.ntau_rho), lr, fma(splat(k.ntau_T), lT, splat(k.l2_inv_tau0))));
  f2 Q = splat(k.Q0);
  if (SRC == 2) {
    Q = mul(splat(k.Q0), ex2(fma(splat(k.Q_rho), lr, mul(splat(k.Q_T), lT))));
    const f2 I = mul(splat(k.Q0), ex2(fma(splat(k.I_rho), lr, mul(splat(k.I_T), lT))));
    yE = mul(rho, sub(Q, I));
  }
  // (rho C_k T - E_nu) / tau + rho Q
  const f2 relax = fma(mul(rho, splat(k.Ck)), T, mul(Ev, splat(-1.0f)));
  yEv = fma(relax, inv_tau, mul(rho, Q));
}

// Slopes, positivity guard, half-step predictor and face states of the two
// cells X from their one-sided differences A (left) and B (right); as
// predict() of the scalar body.
template <int PP, int LIM, int SRC>
__device__ __forceinline__ void predict(const P<float>& k, const f2 (&X)[4], const f2 (&A)[4],
                                        const f2 (&B)[4], f2 ndt_2h, f2 dt_2, f2 (&WP)[4],
                                        f2 (&WM)[4], f2& yEh, f2& yEvh) {
  f2 d[4], a[4], b[4];
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    d[f] = pair(slope<LIM>(A[f].x, B[f].x), slope<LIM>(A[f].y, B[f].y));
    a[f] = fma(splat(0.5f), d[f], X[f]);
    b[f] = fma(splat(-0.5f), d[f], X[f]);
  }
  const Prim pa = prim<PP>(k, a), pb = prim<PP>(k, b);
  f2 dF[4];
  dF[0] = sub(a[1], b[1]);
  dF[1] = sub(add(pa.kin2, pa.p), add(pb.kin2, pb.p));
  dF[2] = sub(mul(pa.v, add(a[2], pa.p)), mul(pb.v, add(b[2], pb.p)));
  dF[3] = sub(mul(pa.v, a[3]), mul(pb.v, b[3]));
  // positivity guard: a non-physical extrapolated state drops that cell's slopes
  const bool g0 = fminf(fminf(a[0].x, pa.p.x), fminf(b[0].x, pb.p.x)) > 0.0f;
  const bool g1 = fminf(fminf(a[0].y, pa.p.y), fminf(b[0].y, pb.p.y)) > 0.0f;
  if (!(g0 && g1)) {
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      if (!g0) d[f].x = dF[f].x = 0.0f;
      if (!g1) d[f].y = dF[f].y = 0.0f;
    }
  }
  f2 yE = splat(0.0f), yEv = splat(0.0f);
  if (SRC != 0) {
    const Prim pu = prim<PP>(k, X);
    source<SRC>(k, X[0], mul(pu.p, pu.ir), X[3], yE, yEv);
  }
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
  if (SRC != 0) {
    const Prim ph = prim<PP>(k, uh);
    source<SRC>(k, uh[0], mul(ph.p, ph.ir), uh[3], yEh, yEvh);
  }
}

// eq. 13 at the two faces of a pair, with left states L and right states R;
// a face with a non-physical state uses the cell values instead: those of the
// pair's cells X and of the cell xl left of it (per field).  Written with
// -S_L >= 0 so that every weight is non-negative:
//   F = (S_R F_L + (-S_L) F_R + (-S_L) S_R (L - R)) / (S_R - S_L).
template <int PP>
__device__ __forceinline__ void hll(const P<float>& k, f2 (&L)[4], f2 (&R)[4], const float (&xl)[4],
                                    const f2 (&X)[4], f2 (&F)[4]) {
  Prim pl = prim<PP>(k, L), pr = prim<PP>(k, R);
  const bool g0 = fminf(fminf(L[0].x, pl.p.x), fminf(R[0].x, pr.p.x)) > 0.0f;
  const bool g1 = fminf(fminf(L[0].y, pl.p.y), fminf(R[0].y, pr.p.y)) > 0.0f;
  if (!(g0 && g1)) {
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      if (!g0) { L[f].x = xl[f]; R[f].x = X[f].x; }
      if (!g1) { L[f].y = X[f].x; R[f].y = X[f].y; }
    }
    pl = prim<PP>(k, L);
    pr = prim<PP>(k, R);
  }
  const f2 gam = splat(k.gamma);
  const f2 cL = sqrt_pos(mul(mul(gam, pl.p), pl.ir));
  const f2 cR = sqrt_pos(mul(mul(gam, pr.p), pr.ir));
  const f2 mL = sub(cL, pl.v), mR = sub(cR, pr.v);   // -(u - c)
  const f2 qL = add(pl.v, cL), qR = add(pr.v, cR);   // u + c
  const f2 nsl = pair(fmaxf(fmaxf(mL.x, mR.x), 0.0f), fmaxf(fmaxf(mL.y, mR.y), 0.0f));   // -min(S_L, 0)
  const f2 sr = pair(fmaxf(fmaxf(qL.x, qR.x), 0.0f), fmaxf(fmaxf(qL.y, qR.y), 0.0f));    // max(S_R, 0)
  const f2 FL[4] = {L[1], add(pl.kin2, pl.p), mul(pl.v, add(L[2], pl.p)), mul(pl.v, L[3])};
  const f2 FR[4] = {R[1], add(pr.kin2, pr.p), mul(pr.v, add(R[2], pr.p)), mul(pr.v, R[3])};
  const f2 inv = rcp(add(sr, nsl));
  const f2 wl = mul(sr, inv), wr = mul(nsl, inv), wd = mul(mul(nsl, sr), inv);
#pragma unroll
  for (int f = 0; f < 4; ++f) F[f] = fma(wd, sub(L[f], R[f]), fma(wl, FL[f], mul(wr, FR[f])));
}

// Conservative update (eq. 15) of the two cells Q with the fluxes of their
// left faces Fl and right faces Fr and the half-step source (yE, yEv).
template <int SRC>
__device__ __forceinline__ void update(const f2 (&Q)[4], const f2 (&Fl)[4], const f2 (&Fr)[4],
                                       f2 yE, f2 yEv, f2 dt, f2 ndtdx, f2 (&N)[4]) {
  N[0] = fma(ndtdx, sub(Fr[0], Fl[0]), Q[0]);
  N[1] = fma(ndtdx, sub(Fr[1], Fl[1]), Q[1]);
  N[2] = fma(ndtdx, sub(Fr[2], Fl[2]), Q[2]);
  if (SRC == 2) N[2] = fma(dt, yE, N[2]);
  N[3] = fma(ndtdx, sub(Fr[3], Fl[3]), Q[3]);
  if (SRC != 0) N[3] = fma(dt, yEv, N[3]);
}

// eq. 16 signal speed and tau key of updated states N, folded into the
// lane's maxima for the cells whose mask bit is set (bit 0: .x, bit 1: .y).
template <int PP, int SRC>
__device__ __forceinline__ void cfl(const P<float>& k, const f2 (&N)[4], int mask, float& smax,
                                    float& akey, uint32_t& flags) {
  const Prim q = prim<PP>(k, N);
  const f2 c = sqrt_pos(mul(mul(splat(k.gamma), q.p), q.ir));
  f2 key = splat(-INFINITY);
  if (SRC != 0) {
    const f2 lr = lg2(N[0]), lT = lg2(mul(q.p, q.ir));
    key = fma(splat(k.ntau_rho), lr, mul(splat(k.ntau_T), lT));   // -(tau_rho lg rho + tau_T lg T)
  }
  const float vx = fabsf(q.v.x), vy = fabsf(q.v.y);
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

}  // namespace pk
}  // namespace sv
