// sv_tile1d.cuh -- the fused float 1D MUSCL-Hancock step (Sec. 2.3: eq. 14
// reconstruction with xi = 0, half-step predictor, eq. 13 HLL, eq. 15 update
// with the source Y, eq. 16 reduction) on block tiles, for large grids.
//
// A persistent block of NT threads walks over tiles of 2 NT cells, thread t
// owning the cell pair (b + 2t, b + 2t + 1) of the tile that starts at b, and
// writes the 2 NT - 4 cells [b + 2, b + 2 NT - 2): the two cells at each end
// are computed only to give the outermost written cells their faces (0.8%
// redundant work for 256 threads, no state carried from tile to tile).  Per
// tile:
//   1. the tile's 4 fields, cells [b - 2, b + 2 NT + 2), are in shared memory
//      (16-byte cp.async copies, issued one tile ahead into a second buffer);
//   2. slopes, guard, predictor and face states of the pair (packed f32x2,
//      sv_pair1d.cuh);
//   3. the left state of the pair's left face comes from lane - 1 by shuffle
//      (for lane 0 from the previous warp through shared memory);
//   4. the HLL fluxes of the pair's left and inner faces (one packed call);
//   5. the right face of the odd cell is lane + 1's left face (shuffle; for
//      lane 31 the next warp's lane 0 through shared memory);
//   6. update, eq. 16 bound of the new states, 8-byte stores.
// The per-cell arithmetic is that of the sliding warp body in float
// (sv_step1d.cuh, packed path), operation for operation, so both kernels give
// bitwise the same states.  The dt epilogue is the shared block fold and
// last-block finalize.
#pragma once

#include "sv_internal.h"
#include "sv_step1d.cuh"

namespace sv {

namespace {

// A tile of NPT cell pairs per thread of an NT-thread block: 2 NPT NT cells
// computed, the two at each end only for their neighbours' faces.
template <int NPT, int NT> struct Tile {
  static constexpr int CELLS = 2 * NPT * NT;    // cells computed per tile
  static constexpr int OUT = CELLS - 4;         // cells written per tile
  static constexpr int SPAN = CELLS + 4;        // cells held: [b - 2, b + CELLS + 2)
};

template <int NPT, int NT> struct TileSmem {
  float u[2][4][Tile<NPT, NT>::SPAN];    // double-buffered tile, field-major
  float wp[NT / 32][4];                  // lane 31's last right face state, per warp
  float fl[NT / 32][4];                  // lane 0's first left face flux, per warp
};

__device__ __forceinline__ void cp16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

// Fill buffer `dst` with tile b's cells [b - 2, b + SPAN - 2).  Interior tiles
// of a grid whose fields start on 16-byte boundaries use 16-byte copies; the
// others go cell by cell through the boundary mapping (periodic wrap, wall
// mirror, outflow copy, driven ghost state).  Commits one cp.async group.
// Whether tile b is copied with 16-byte chunks: its span lies inside the grid
// and the fields start on 16-byte boundaries.
template <int SPAN>
__device__ __forceinline__ bool tile_interior(int N, int b) {
  const int lo = b - 2;
  return (N & 3) == 0 && lo >= 0 && lo + SPAN <= N;
}

// The 16-byte copies of an interior tile (no boundary mapping, no time).
template <int SPAN, int NT>
__device__ __forceinline__ void copy_interior(float (*dst)[SPAN], const float* Uin, int N, int b) {
  // lo = b - 2 is a multiple of 4 (b = OUT i - 2 with OUT a multiple of 4).
  // A quarter of the block per field: thread q of it copies 16-byte chunks
  // q, q + NT/4, ... of the SPAN/4 = 1 + R NT/4 chunks, and thread 0 the
  // last one, so no thread divides an index.
  const int lo = b - 2;
  constexpr int C4 = SPAN / 4, TPF = NT / 4, R = (C4 - 1) / TPF;
  static_assert(C4 == 1 + R * TPF, "span of whole quarter-block rounds plus one chunk");
  const int f = threadIdx.x / TPF, q = threadIdx.x % TPF;
  const float* src = Uin + (f * N + lo + 4 * q);
  float* d = &dst[f][4 * q];
#pragma unroll
  for (int r = 0; r < R; ++r) cp16(d + 4 * TPF * r, src + 4 * TPF * r);
  if (q == 0) cp16(d + 4 * (C4 - 1), src + 4 * (C4 - 1));
}

template <int SPAN, int PP, int NT>
__device__ __forceinline__ void load_tile(float (*dst)[SPAN], const float* Uin, int N, int b,
                                          const P<float>& k, const KParams& kp, double t) {
  const int lo = b - 2;
  if (tile_interior<SPAN>(N, b)) {
    copy_interior<SPAN, NT>(dst, Uin, N, b);
  } else {
    for (int e = threadIdx.x; e < SPAN; e += NT) {
      const int j = lo + e;
      if (j < 0 && k.bc_lo == BC_DRIVEN) {
        double u[4];
        drive_state(kp, ((double)j + 0.5) * kp.h, t, u);
#pragma unroll
        for (int f = 0; f < 4; ++f) dst[f][e] = (float)(PP == 3 ? u[f] - kp.ref[f] : u[f]);
      } else {
        bool flip;
        const int i = bc_index(j, N, k.bc_lo, k.bc_hi, flip);
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          const float v = Uin[f * N + i];
          dst[f][e] = (f == 1 && flip) ? -v : v;
        }
      }
    }
  }
  cp_async_commit();
}

// Field offsets f N + j are ints: tile1d_launch admits N < 2^31 / 4.
template <int PP, int LIM, int SRC, int MINB, int NPT, int NT>
__global__ void __launch_bounds__(NT, MINB)
tile1d_kernel(const KParams kp, float* __restrict__ bufA, float* __restrict__ bufB,
              Ctl* __restrict__ ctl, int N) {
  using pk::f2;
  constexpr int CELLS = Tile<NPT, NT>::CELLS, OUT = Tile<NPT, NT>::OUT, SPAN = Tile<NPT, NT>::SPAN;
  constexpr int NWT = NT / 32;
  extern __shared__ __align__(16) unsigned char smem_tile[];
  TileSmem<NPT, NT>& S = *reinterpret_cast<TileSmem<NPT, NT>*>(smem_tile);
  const int ntile = (N + OUT - 1) / OUT;
  int tile = blockIdx.x;
  // An interior first tile needs nothing from the control block: its copies
  // from both state buffers go out before the control block is read (slot 0
  // from bufA, slot 1 from bufB), so that read's round trip overlaps the
  // tile's; the slot of the buffer that is not the input takes the next tile.
  const bool early = tile < ntile && tile_interior<SPAN>(N, OUT * tile - 2);
  pdl_wait();                                     // the previous step's grid has completed
  if (early) {
    copy_interior<SPAN, NT>(S.u[0], bufA, N, OUT * tile - 2);
    cp_async_commit();
    copy_interior<SPAN, NT>(S.u[1], bufB, N, OUT * tile - 2);
    cp_async_commit();
  }
  const StepCtl sc = block_step_ctl(ctl);
  if (!(sc.dt > 0.0)) {                           // stopped, or t_end reached
    cp_async_wait<0>();                           // no copy may outlive the block
    return;
  }
  const float* __restrict__ Uin = sc.cur ? bufB : bufA;
  float* __restrict__ Uout = sc.cur ? bufA : bufB;
  const double t = sc.t;

  const P<float> k(kp);
  const StepDt<float> sd(sc);
  const f2 dt2 = pk::splat(sd.dt), ndtdx2 = pk::splat(-sd.dtdx);
  const f2 ndt_2h2 = pk::splat(-sd.dt_2h), dt_22 = pk::splat(sd.dt_2);

  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int src_m = (lane + 31) & 31, src_p = (lane + 1) & 31;

  float smax = 0.0f, akey = -INFINITY;
  uint32_t flags = 0;

  const int first = early ? (int)sc.cur : 0;      // slot of the first tile
  if (!early && tile < ntile) load_tile<SPAN, PP, NT>(S.u[0], Uin, N, OUT * tile - 2, k, kp, t);
  for (int it = 0; tile < ntile; ++it, tile += gridDim.x) {
    const int buf = (it + first) & 1;
    const int b = OUT * tile - 2;
    cp_async_wait<0>();
    __syncthreads();                              // tile in place; the other buffer is free
    if (tile + (int)gridDim.x >= ntile) pdl_trigger();   // this block's last tile
    if (tile + (int)gridDim.x < ntile)
      load_tile<SPAN, PP, NT>(S.u[buf ^ 1], Uin, N, OUT * (tile + gridDim.x) - 2, k, kp, t);

    // pair p of the thread sits at span offsets 2 + 2 (NPT t + p) and the next
    f2 X[NPT][4], WP[NPT][4], WM[NPT][4], YE[NPT], YEv[NPT];
    float XL[NPT][4];                             // the cell left of each pair
#pragma unroll
    for (int p = 0; p < NPT; ++p) {
      const int pos = 2 + 2 * (NPT * (int)threadIdx.x + p);
      f2 A[4], B[4];
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const float* rf = S.u[buf][f];
        X[p][f] = *reinterpret_cast<const f2*>(rf + pos);
        XL[p][f] = rf[pos - 1];
        // one-sided differences, the inner one shared by both cells (scalar:
        // the limiter takes them component by component)
        const float c = X[p][f].y - X[p][f].x;
        A[f] = pk::pair(X[p][f].x - XL[p][f], c);
        B[f] = pk::pair(c, rf[pos + 2] - X[p][f].y);
      }
      pkx::predict<PP, LIM, SRC>(k, X[p], A, B, ndt_2h2, dt_22, WP[p], WM[p], YE[p], YEv[p]);
    }

    if (lane == 31) {
#pragma unroll
      for (int f = 0; f < 4; ++f) S.wp[w][f] = WP[NPT - 1][f].y;
    }
    __syncthreads();
    // left state of the first pair's left face: lane - 1's last pair
    float nb[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const float v = __shfl_sync(0xffffffffu, WP[NPT - 1][f].y, src_m);
      // thread 0's first left face is outside the written cells: any physical state
      nb[f] = lane ? v : (w ? S.wp[w - 1][f] : (f == 0 || f == 2 ? 1.0f : 0.0f));
    }
    f2 F[NPT][4];
#pragma unroll
    for (int p = 0; p < NPT; ++p) {
      f2 L[4];
#pragma unroll
      for (int f = 0; f < 4; ++f) L[f] = pk::pair(p ? WP[p - 1][f].y : nb[f], WP[p][f].x);
      pkx::hll<PP>(k, L, WM[p], XL[p], X[p], F[p]);  // the pair's left and inner faces
    }

    if (lane == 0) {
#pragma unroll
      for (int f = 0; f < 4; ++f) S.fl[w][f] = F[0][f].x;
    }
    __syncthreads();
    // right face of the last pair's odd cell: lane + 1's first left face
    float nf[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const float v = __shfl_sync(0xffffffffu, F[0][f].x, src_p);
      nf[f] = lane < 31 ? v : (w < NWT - 1 ? S.fl[w + 1][f] : 0.0f);
    }
#pragma unroll
    for (int p = 0; p < NPT; ++p) {
      const int j = b + 2 * (NPT * (int)threadIdx.x + p);   // global index of the even cell
      if (j >= b + 2 && j < b + CELLS - 2 && j < N) {
        f2 FR[4], Nw[4];
#pragma unroll
        for (int f = 0; f < 4; ++f) FR[f] = pk::pair(F[p][f].y, p < NPT - 1 ? F[p + 1][f].x : nf[f]);
        pk::update<SRC>(X[p], F[p], FR, YE[p], YEv[p], dt2, ndtdx2, Nw);
        const bool two = j + 1 < N;
        pkx::cfl<PP, SRC>(k, Nw, two ? 3 : 1, smax, akey, flags);
        if (two && (N & 1) == 0) {
#pragma unroll
          for (int f = 0; f < 4; ++f) *reinterpret_cast<f2*>(Uout + (f * N + j)) = Nw[f];
        } else {
#pragma unroll
          for (int f = 0; f < 4; ++f) {
            Uout[f * N + j] = Nw[f].x;
            if (two) Uout[f * N + j + 1] = Nw[f].y;
          }
        }
      }
    }
  }
  cp_async_wait<0>();
  reduce_and_finalize<float, NT>(ctl, kp, smax, akey, flags, true);
}

// Variants (tile1d_grid / tile1d_launch `var` = 10 NPT + MINB), all with
// 256-thread blocks: one cell pair per thread at a register budget of 3 blocks
// per SM (78 registers, 24 warps per SM), 4 (64 registers, 32 warps, a few
// bytes of spills) or 2 (its natural ~94 registers, 16 warps), or two pairs
// per thread (1024-cell tiles: half the barriers and exchanges per cell, two
// independent chains) at 2 blocks per SM.  (Other block sizes at the natural
// register count, 192 threads x 3, 160 threads x 4 and 320 threads x 2,
// measured 4-6% slower.)
// PP: the pressure policy (0 float, 2 compensated float) or the perturbation
// layout (3).
template <int PP, int LIM, int SRC>
struct KT {
  static constexpr auto fn13 = tile1d_kernel<PP, LIM, SRC, 3, 1, 256>;
  static constexpr auto fn14 = tile1d_kernel<PP, LIM, SRC, 4, 1, 256>;
  static constexpr auto fn12 = tile1d_kernel<PP, LIM, SRC, 2, 1, 256>;
  static constexpr auto fn22 = tile1d_kernel<PP, LIM, SRC, 2, 2, 256>;
};

template <int PP, int LIM, int SRC>
void* pick_var(int var) {
  switch (var) {
    case 12: return (void*)KT<PP, LIM, SRC>::fn12;
    case 22: return (void*)KT<PP, LIM, SRC>::fn22;
    case 14: return (void*)KT<PP, LIM, SRC>::fn14;
    default: return (void*)KT<PP, LIM, SRC>::fn13;
  }
}

template <int PP, int LIM>
void* pick_src(int src, int var) {
  switch (src) {
    case 0: return pick_var<PP, LIM, 0>(var);
    case 1: return pick_var<PP, LIM, 1>(var);
    default: return pick_var<PP, LIM, 2>(var);
  }
}

template <int PP>
void* pick_lim(const KParams& kp, int var) {
  const int src = kp.frozen ? 0 : (kp.qi_zero ? 1 : 2);
  switch (kp.limiter) {
    case 1: return pick_src<PP, 1>(src, var);
    case 2: return pick_src<PP, 2>(src, var);
    default: return pick_src<PP, 0>(src, var);
  }
}

int threads_of(int) { return 256; }

size_t smem_of(int var) {
  switch (var) {
    case 22: return sizeof(TileSmem<2, 256>);
    default: return sizeof(TileSmem<1, 256>);
  }
}

}  // namespace

// The kernel of variant `var` for the compensated-float pressure and for the
// perturbation layout (instantiated in sv_tile1d_pc.cu and sv_tile1d_ps.cu,
// so that the three pressure policies' variants compile in parallel).
void* tile1d_pick_pc(const KParams& kp, int var);
void* tile1d_pick_ps(const KParams& kp, int var);

}  // namespace sv
