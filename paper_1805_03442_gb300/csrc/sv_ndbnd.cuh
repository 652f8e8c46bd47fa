// sv_ndbnd.cuh -- boundaries, medium map and driven cells of the 2D steps
// (the paper's two-dimensional active-sector problem, Sec. 3), shared by the
// scalar and the plane-pair kernels.
#pragma once

#include "sv_reduce.cuh"

namespace sv {

// Cell whose state position j of an axis of n cells holds: periodic wrap,
// wall mirror (flip: the normal momentum is reversed) or outflow copy.
// Positions further out than the two ghost layers are clamped into the grid;
// their values reach no updated cell.
// In the type of j, as wrap.
template <typename I>
__device__ __forceinline__ I map_axis(I j, typename index_of<I>::type n, int bc_lo, int bc_hi,
                                      bool& flip) {
  flip = false;
  if (j >= 0 && j < n) return j;
  const int bc = j < 0 ? bc_lo : bc_hi;
  if (bc == BC_PERIODIC) return wrap(j, n);
  if (bc == BC_REFLECT) {
    flip = true;
    const I m = j < 0 ? -1 - j : 2 * n - 1 - j;
    return m < 0 ? 0 : (m >= n ? n - 1 : m);
  }
  return j < 0 ? 0 : n - 1;
}

// The pulsating source of the 2D problem at time t (double, like its
// definition), in the kernel's type.
template <typename R, int NF>
__device__ __forceinline__ void pulse_state(const KParams& kp, double t, R (&u)[NF]) {
  const double s = kp.pul_amp * sin(kp.pul_omega * t);
  const double rho = 1.0 + s, p = 1.0 + kp.gamma * s, Ev = rho * kp.pul_ev;
#pragma unroll
  for (int f = 0; f < NF; ++f) u[f] = (R)0;
  u[0] = (R)rho;
  u[NF - 2] = (R)(p / kp.g1 + Ev);
  u[NF - 1] = (R)Ev;
}

}  // namespace sv
