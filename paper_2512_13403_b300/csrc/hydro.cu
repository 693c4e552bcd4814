// Fused finite-volume stage kernel and its small companions (step prologue, reductions).
//
// One launch of stage_kernel computes a full SSP-RK2 stage (App. A.3) for a block of cells:
// primitive recovery (Eq. 2), MC-limited MUSCL face states (App. A.1), HLLC fluxes (App. A.2)
// on every face of the block, the unsplit divergence and the stage combination.  The second
// stage also applies the operator-split sources in place — OU forcing (Sec. 3.1.1) then cooling
// (Sec. 4.3) — and reduces the CFL minimum of the new state for the next step (App. A.4).
//
// Blocking: a CTA owns a BX x BY column of cells and marches along z through a chunk of
// planes.  Primitive planes (with a two-cell x/y halo) sit in a three-plane shared-memory ring
// (k, k+1, k+2); every x and y face of plane k is evaluated exactly once per CTA, each thread
// taking its own cell's slopes and faces and a fixed tail of halo work, and the z faces come
// from a per-thread register pipeline (each z face once).  The conserved variables of the next
// plane arrive by TMA (five tensor-map boxes: the tile core and its four halo strips, wrapped
// periodically) into staging buffers while the current plane is computed, and are converted
// into the ring one plane later.
#include <math.h>
#include <string.h>
#include <cstring>

#include <mutex>
#include <vector>

#include <cudaTypedefs.h>

#include "async_copy.cuh"
#include "tc_ptx.cuh"
#include "tma.cuh"
#include "dh_kernels.h"
#include "dh_sources.cuh"
#include "ff.cuh"
#include "../../include/dh.h"

namespace dh {

constexpr int BX = 32, BY = 8, HX = BX + 4, HY = BY + 4;
constexpr int NTHREADS = BX * BY;
constexpr int NFORCE = BY * 9;       // forcing row factors: row x (n_x = 0, 1, 2) x component

// Staged conserved variables of the plane in flight, one dense buffer per TMA box: the tile
// core, the x halos (SCE cells = 16 bytes on each side, of which the two nearest the tile are
// read) and the y halos (two rows above and below).  The four corner blocks of the halo are
// never read by the stencil (x slopes read rows 0..BY-1, y slopes columns 0..BX-1) and are not
// loaded.  Every box is contiguous in global memory at any tile position: x0 and y0 are
// multiples of BX and BY, so a halo either lies inside the grid or is the whole wrapped strip
// at the other side.
template <typename real> struct Staging {
  static constexpr int SCE = 16 / (int)sizeof(real);
  static constexpr uint32_t BYTES = (uint32_t)sizeof(real) * 5u * (BX * BY + 2 * BY * SCE + 4 * BX);
};

// Four components of a primitive state or flux in one 16-byte-aligned word group, so that a
// shared-memory access moves them with one 128-bit instruction (two for float64); the fifth
// component sits in a separate array.
template <typename real> struct alignas(16) Q4 { real a, b, c, d; };

template <typename real>
__device__ __forceinline__ Prim<real> qprim(const Q4<real>& q, real p) {
  return Prim<real>{q.a, q.b, q.c, q.d, p};
}
template <typename real>
__device__ __forceinline__ void qstore(Q4<real>& q, real& s, const Prim<real>& w) {
  q = Q4<real>{w.r, w.vx, w.vy, w.vz};
  s = w.p;
}

template <typename real> struct StageSmem {
  alignas(128) real core[5][BY][BX];                 // staged plane: tile core
  alignas(128) real xl[5][BY][Staging<real>::SCE];   // x halo, x0 - SCE .. x0 - 1
  alignas(128) real xr[5][BY][Staging<real>::SCE];   // x halo, x0 + BX .. x0 + BX + SCE - 1
  alignas(128) real yt[5][2][BX];                    // y halo, y0 - 2, y0 - 1
  alignas(128) real yb[5][2][BX];                    // y halo, y0 + BY, y0 + BY + 1
  alignas(16) real tz[4];    // forcing: z twiddles of the plane in flight (staged with it)
  Q4<real> w4[3][HY][HX];    // primitive planes ring (k, k+1, k+2), two-cell x/y halo: rho, v
  Q4<real> xm4[BY][BX + 2];  // x face states W - dW/2 of cells lx = -1..BX (index lx + 1)
  Q4<real> xp4[BY][BX + 2];  //                W + dW/2
  Q4<real> ym4[BY + 2][BX];  // y face states of cells ly = -1..BY (index ly + 1)
  Q4<real> yp4[BY + 2][BX];
  Q4<real> fx4[BY][BX + 1];  // x-face fluxes of the current plane: mass and momentum
  Q4<real> fy4[BY + 1][BX];  // y-face fluxes
  real wp[3][HY][HX];        // pressure of the ring planes
  real xmp[BY][BX + 2], xpp[BY][BX + 2];   // pressure of the face states
  real ymp[BY + 2][BX], ypp[BY + 2][BX];
  real fxe[BY][BX + 1];      // energy fluxes
  real fye[BY + 1][BX];
  real ah[96];               // forcing: normalised OU table
  real tyt[BY][4];           // forcing: y twiddles of the tile's rows
  real fB[BY][3][3][2];      // forcing: B[row][n_x][component] = sum over modes with that n_x
  int xs[HX];                // wrapped global x of each ring column (prologue)
  int ys[HY];                // wrapped global y of each ring row (prologue)
  real red[NTHREADS / 32];   // CFL reduction scratch
  alignas(8) uint64_t bar;   // staging plane landed (TMA transaction bytes)
};

template <typename real>
__device__ __forceinline__ Prim<real> smem_prim(const StageSmem<real>& S, int slot, int sy,
                                                int sx) {
  return qprim(S.w4[slot][sy][sx], S.wp[slot][sy][sx]);
}

template <typename real>
__device__ __forceinline__ Prim<real> load_prim(const real* __restrict__ U, long long n3,
                                                long long idx, real gm1) {
  return cons_to_prim(__ldg(U + idx), __ldg(U + n3 + idx), __ldg(U + 2 * n3 + idx),
                      __ldg(U + 3 * n3 + idx), __ldg(U + 4 * n3 + idx), gm1);
}

// Bound on the probes of the staging mbarrier: a plane's copies land in microseconds; a wait
// that reaches it sets FLAG_TIMEOUT and the CTA stops.
constexpr uint32_t STAGE_WAIT_ITERS = 1u << 22;

// Work of a plane.  Thread (tx, ty) = (tid % BX, tid / BX) owns tile cell (tx, ty): its
// primitive conversion, x and y slopes, x face tx (its left face), y face ty (its lower face),
// z faces and update.  The halo work is a fixed tail: the y slopes of rows -1 and BY (warps 0
// and 1), the x slopes of columns -1 and BX (warp 2, lanes 0..15), the conversion of the 160
// used halo cells (warps 3..7), the x face BX of each row (warp 6, lanes 0..7) and the y face
// BY of each column (warp 7).  Every address is fixed for the whole march.
// float32: three CTAs per SM (shared memory allows three; registers are capped to match)
template <typename real, int STAGE, int LIM>
__global__ void __launch_bounds__(NTHREADS, sizeof(real) == 4 ? 3 : 1)
stage_kernel(const StageArgs<real> p, const int zchunk, const __grid_constant__ StageTma tma,
             const int use_tma) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  StageSmem<real>& S = *reinterpret_cast<StageSmem<real>*>(smem_raw);
  const int tid = threadIdx.x;
  // Skip the stage after a fatal failure.  One thread reads the flag and the CTA follows it, so
  // a flag raised by another CTA mid-launch cannot split this CTA across a barrier.
  __shared__ unsigned s_skip;
  __shared__ int s_abort;
  if (tid == 0) {
    s_skip = *((volatile unsigned*)&p.rec->flags) & FATAL_FLAGS;
    s_abort = 0;
  }
  __syncthreads();
  if (s_skip) return;

  const int tx = tid & (BX - 1), ty = tid / BX, warp = tid >> 5;
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  const long long plane = (long long)nx * ny;
  const long long n3 = plane * nz;
  const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
  const int z0 = blockIdx.z * zchunk;
  const int z1 = min(z0 + zchunk, nz);
  const real dt = (real)*p.dtp;
  const real gamma = p.gamma, gm1 = p.gm1;
  const int gx = x0 + tx, gy = y0 + ty;
  const bool active = gx < nx && gy < ny;
  const int gxw = gx % nx, gyw = gy % ny;
  // STAGE 1: out = U + dt L(U).  STAGE 2: RK2's final stage, out = (U0 + U + dt L(U)) / 2 with
  // the epilogue.  STAGE 3: out = w0 U0 + w1 (U + dt L(U)), with the epilogue if final_stage
  // (SSPRK3's second and third stages).
  constexpr bool COMB = STAGE >= 2;
  const bool final = STAGE == 2 || (STAGE == 3 && p.final_stage);
  const real w0 = STAGE == 2 ? real(0.5) : p.w0, w1 = STAGE == 2 ? real(0.5) : p.w1;
  const bool forcing = final && p.forcing;

  using ST = Staging<real>;
  constexpr int SCE = ST::SCE;
  const uint32_t bar = tc::smem_u32(&S.bar);
  // box destinations must start on 128 bytes; the buffers are 128-byte multiples from S
  const bool via_tma = use_tma != 0 && (tc::smem_u32(&S.core[0][0][0]) & 127u) == 0u;
  if (tid < HX) S.xs[tid] = ((x0 + tid - 2) % nx + nx) % nx;
  if (tid >= 64 && tid < 64 + HY) S.ys[tid - 64] = ((y0 + tid - 64 - 2) % ny + ny) % ny;
  if (tid == 96) {
    tc::mbar_init(&S.bar, 1u);
    tc::mbar_fence_init();
  }
  if (forcing) {
    if (tid < 96) S.ah[tid] = __ldg(p.ahat_norm + tid);
    if (tid >= 128 && tid < 128 + 4 * BY) {
      const int ly = (tid - 128) >> 2, i = (tid - 128) & 3;
      S.tyt[ly][i] = __ldg(p.tw[1] + 4 * ((y0 + ly) % ny) + i);
    }
  }
  // wrapped start coordinates of the halo boxes (TMA path: nx % BX == 0 and ny % BY == 0)
  const int xl0 = x0 >= SCE ? x0 - SCE : nx - SCE, xr0 = x0 + BX < nx ? x0 + BX : 0;
  const int yt0 = y0 >= 2 ? y0 - 2 : ny - 2, yb0 = y0 + BY < ny ? y0 + BY : 0;
  __syncthreads();

  // The conserved variables of plane k into the staging buffers, with the forcing's z twiddles
  // of plane k - 2 (the plane whose row factors the next iteration builds).  TMA: one thread
  // issues five box loads (and the twiddles' bulk copy) on the staging barrier.  Otherwise
  // every thread issues element copies of its share (wrapped coordinates of every position).
  auto stage_plane = [&](int k) {
    const int kz = wrap(k, nz);
    if (via_tma) {
      if (tid == 0) {
        tc::mbar_arrive_expect_tx(&S.bar, ST::BYTES + (forcing ? 4u * (uint32_t)sizeof(real) : 0u));
        tma_load_4d(tc::smem_u32(&S.core[0][0][0]), &tma.core, x0, y0, kz, 0, bar);
        tma_load_4d(tc::smem_u32(&S.xl[0][0][0]), &tma.xh, xl0, y0, kz, 0, bar);
        tma_load_4d(tc::smem_u32(&S.xr[0][0][0]), &tma.xh, xr0, y0, kz, 0, bar);
        tma_load_4d(tc::smem_u32(&S.yt[0][0][0]), &tma.yh, x0, yt0, kz, 0, bar);
        tma_load_4d(tc::smem_u32(&S.yb[0][0][0]), &tma.yh, x0, yb0, kz, 0, bar);
        if (forcing)
          tc::bulk_g2s(tc::smem_u32(&S.tz[0]), p.tw[2] + 4 * wrap(k - 2, nz),
                       4u * (uint32_t)sizeof(real), &S.bar);
      }
      return;
    }
    const long long zoff = (long long)kz * plane;
    if (forcing && tid == NTHREADS - 1) {
      const real* t = p.tw[2] + 4 * wrap(k - 2, nz);
#pragma unroll
      for (int i = 0; i < 4; i += SCE) cp_async16(&S.tz[i], t + i);
    }
    constexpr int NC = BX * BY, NXH = BY * SCE, NYH = 2 * BX;
    for (int c = tid; c < NC + 2 * NXH + 2 * NYH; c += NTHREADS) {
      int lx, ly, fs;
      real* dst;
      if (c < NC) {
        lx = c % BX; ly = c / BX; dst = &S.core[0][ly][lx]; fs = BY * BX;
      } else if (c < NC + 2 * NXH) {
        const int e = c - NC, side = e / NXH, r = e - side * NXH;
        ly = r / SCE;
        const int col = r - ly * SCE;
        lx = side == 0 ? col - SCE : BX + col;
        dst = side == 0 ? &S.xl[0][ly][col] : &S.xr[0][ly][col];
        fs = BY * SCE;
      } else {
        const int e = c - NC - 2 * NXH, side = e / NYH, r = e - side * NYH;
        const int row = r / BX;
        lx = r - row * BX;
        ly = side == 0 ? row - 2 : BY + row;
        dst = side == 0 ? &S.yt[0][row][lx] : &S.yb[0][row][lx];
        fs = 2 * BX;
      }
      const int gxc = ((x0 + lx) % nx + nx) % nx, gyc = ((y0 + ly) % ny + ny) % ny;
      const real* g = p.U + zoff + (long long)gyc * nx + gxc;
#pragma unroll
      for (int f = 0; f < 5; ++f) {
        if constexpr (sizeof(real) == 4) cp_async4(dst + f * fs, g + f * n3);
        else cp_async8(dst + f * fs, g + f * n3);
      }
    }
    cp_async_commit();
  };

  // ---- fixed per-thread tasks -------------------------------------------------------------
  // conversion: own cell from the core, and (warps 3..7) one halo cell
  const int ring_own = (ty + 2) * HX + tx + 2;
  const real* ext_src = nullptr;   // halo cell of the conversion tail, field stride ext_fs
  int ext_fs = 0, ext_ring = -1;
  if (tid >= 96) {
    const int e = tid - 96;   // 0 .. 159
    if (e < 64) {
      const int row = e >> 5, lx = e & 31;
      ext_src = &S.yt[0][row][lx]; ext_fs = 2 * BX; ext_ring = row * HX + lx + 2;
    } else if (e < 128) {
      const int row = (e - 64) >> 5, lx = e & 31;
      ext_src = &S.yb[0][row][lx]; ext_fs = 2 * BX; ext_ring = (BY + 2 + row) * HX + lx + 2;
    } else if (e < 144) {
      const int ly = (e - 128) & 7, c = (e - 128) >> 3;
      ext_src = &S.xl[0][ly][SCE - 2 + c]; ext_fs = BY * SCE; ext_ring = (ly + 2) * HX + c;
    } else {
      const int ly = (e - 144) & 7, c = (e - 144) >> 3;
      ext_src = &S.xr[0][ly][c]; ext_fs = BY * SCE; ext_ring = (ly + 2) * HX + BX + 2 + c;
    }
  }
  // slope tail: y slopes of rows -1 (warp 0) and BY (warp 1), x slopes of columns -1 and BX
  // (warp 2, lanes 0..15): the cell's ring position, its neighbour step and output slot
  int sl_ring = -1, sl_step = 0, sl_out = 0;
  bool sl_y = false;
  if (tid < 64) {
    const int ly = tid < 32 ? -1 : BY;
    sl_ring = (ly + 2) * HX + tx + 2; sl_step = HX; sl_out = (ly + 1) * BX + tx; sl_y = true;
  } else if (tid < 80) {
    const int lx = tid - 64 < 8 ? -1 : BX, ly = (tid - 64) & 7;
    sl_ring = (ly + 2) * HX + lx + 2; sl_step = 1; sl_out = ly * (BX + 2) + lx + 1;
  }
  // face tail: x face BX of row lane (warp 6, lanes 0..7), y face BY of column lane (warp 7)
  const bool fx_tail = warp == 6 && (tid & 31) < BY, fy_tail = warp == 7;

  // the conversion of a staged plane into ring slot `slot`
  auto convert_plane = [&](int slot) {
    const real* c0 = &S.core[0][ty][tx];
    qstore(S.w4[slot][ty + 2][tx + 2], S.wp[slot][ty + 2][tx + 2],
           cons_to_prim(c0[0], c0[BY * BX], c0[2 * BY * BX], c0[3 * BY * BX], c0[4 * BY * BX], gm1));
    if (ext_ring >= 0) {
      Q4<real>* q = &S.w4[slot][0][0] + ext_ring;
      qstore(*q, (&S.wp[slot][0][0])[ext_ring],
             cons_to_prim(ext_src[0], ext_src[ext_fs], ext_src[2 * ext_fs], ext_src[3 * ext_fs],
                          ext_src[4 * ext_fs], gm1));
    }
  };
  auto ring_prim = [&](int slot, int off) {
    return qprim((&S.w4[slot][0][0])[off], (&S.wp[slot][0][0])[off]);
  };

  auto load_plane = [&](int k, int slot) {
    const long long zoff = (long long)wrap(k, nz) * plane;
    for (int c = tid; c < HX * HY; c += NTHREADS) {
      const int sy = c / HX, sx = c - sy * HX;
      const long long idx = zoff + (long long)S.ys[sy] * nx + S.xs[sx];
      qstore(S.w4[slot][sy][sx], S.wp[slot][sy][sx], load_prim(p.U, n3, idx, gm1));
    }
  };

  // x twiddles of the own column (forcing synthesis), fixed for the whole march
  real twx[4] = {real(0), real(0), real(0), real(0)};
  if (forcing) {
#pragma unroll
    for (int q = 0; q < 4; ++q) twx[q] = __ldg(p.tw[0] + 4 * gxw + q);
  }

  // Prologue: planes z0, z0+1 in the ring; the own column's z0-2, z0-1 in registers.
  load_plane(z0, 0);
  load_plane(z0 + 1, 1);
  const long long col = (long long)gyw * nx + gxw;
  const Prim<real> wm2 = load_prim(p.U, n3, (long long)wrap(z0 - 2, nz) * plane + col, gm1);
  const Prim<real> wm1 = load_prim(p.U, n3, (long long)wrap(z0 - 1, nz) * plane + col, gm1);
  __syncthreads();
  Prim<real> dk;          // z slope of the own cell at plane k
  real fz_lo[5];          // z flux on face k - 1/2
  int nfb = 0;            // positivity fallbacks of the own cell's slopes (x, y, z per plane)
  {
    const Prim<real> w0 = smem_prim(S, 0, ty + 2, tx + 2);
    const Prim<real> w1 = smem_prim(S, 1, ty + 2, tx + 2);
    const Prim<real> dm1 = limited_slope<LIM>(wm2, wm1, w0);
    dk = limited_slope<LIM>(wm1, w0, w1, nfb);
    face_flux(2, add_half(wm1, dm1, real(1)), add_half(w0, dk, real(-1)), gamma, gm1, fz_lo);
  }
  stage_plane(z0 + 2);

  real tmin = real(INFINITY);
  unsigned flags = 0;
  int nsub_seen = 0;   // largest cooling substep count of this thread's cells

  for (int k = z0; k < z1; ++k) {
    const int s0 = (k - z0) % 3, s1 = (k - z0 + 1) % 3, s2 = (k - z0 + 2) % 3;
    if (via_tma) {
      if (!tc::mbar_wait(&S.bar, (uint32_t)(k - z0) & 1u, STAGE_WAIT_ITERS)) s_abort = 1;
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();  // ---- plane k+2 staged; the update of plane k-1 is done
    if (s_abort) break;

    convert_plane(s2);
    // limited slopes and face states of plane k: own cell on both axes, then the tail
    {
      const Prim<real> w1 = ring_prim(s0, ring_own);
      const Prim<real> dx = limited_slope<LIM>(ring_prim(s0, ring_own - 1), w1, ring_prim(s0, ring_own + 1), nfb);
      qstore(S.xm4[ty][tx + 1], S.xmp[ty][tx + 1], add_half(w1, dx, real(-1)));
      qstore(S.xp4[ty][tx + 1], S.xpp[ty][tx + 1], add_half(w1, dx, real(1)));
      const Prim<real> dy = limited_slope<LIM>(ring_prim(s0, ring_own - HX), w1, ring_prim(s0, ring_own + HX), nfb);
      qstore(S.ym4[ty + 1][tx], S.ymp[ty + 1][tx], add_half(w1, dy, real(-1)));
      qstore(S.yp4[ty + 1][tx], S.ypp[ty + 1][tx], add_half(w1, dy, real(1)));
    }
    if (sl_ring >= 0) {
      const Prim<real> w1 = ring_prim(s0, sl_ring);
      const Prim<real> d = limited_slope<LIM>(ring_prim(s0, sl_ring - sl_step), w1, ring_prim(s0, sl_ring + sl_step));
      if (sl_y) {
        qstore((&S.ym4[0][0])[sl_out], (&S.ymp[0][0])[sl_out], add_half(w1, d, real(-1)));
        qstore((&S.yp4[0][0])[sl_out], (&S.ypp[0][0])[sl_out], add_half(w1, d, real(1)));
      } else {
        qstore((&S.xm4[0][0])[sl_out], (&S.xmp[0][0])[sl_out], add_half(w1, d, real(-1)));
        qstore((&S.xp4[0][0])[sl_out], (&S.xpp[0][0])[sl_out], add_half(w1, d, real(1)));
      }
    }
    if (forcing && tid >= NTHREADS - NFORCE) {
      const int q = tid - (NTHREADS - NFORCE);
      const int ly = q / 9, rem = q - 9 * ly;
      const int nxsel = rem / 3, c = rem - 3 * nxsel;
      real tyv[4], tzv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        tyv[i] = S.tyt[ly][i];
        tzv[i] = S.tz[i];
      }
      real bre = real(0), bim = real(0);
      row_factor<real, 0>(S.ah, nxsel, c, tyv, tzv, bre, bim);
      S.fB[ly][nxsel][c][0] = bre;
      S.fB[ly][nxsel][c][1] = bim;
    }
    __syncthreads();  // ---- plane k+2 in the ring, face states ready, staging buffers free

    if (k + 1 < z1) stage_plane(k + 3);
    // the own cell's values for the update, loaded now and used after the face loop: U in
    // stage 1, U0 in the combination stages (which load U there: holding both measured
    // slower, from more live registers)
    const long long idx = (long long)k * plane + col;
    real uin[5], un[5];
    if (!COMB && active) {
#pragma unroll
      for (int c = 0; c < 5; ++c) uin[c] = __ldg(p.U + c * n3 + idx);
    }
    if (COMB && active) {
#pragma unroll
      for (int c = 0; c < 5; ++c) un[c] = __ldg(p.U0 + c * n3 + idx);
    }
    // z face k+1/2 of the own column
    real fz_hi[5];
    Prim<real> dk1;
    {
      const Prim<real> w0 = smem_prim(S, s0, ty + 2, tx + 2);
      const Prim<real> w1 = smem_prim(S, s1, ty + 2, tx + 2);
      const Prim<real> w2 = smem_prim(S, s2, ty + 2, tx + 2);
      int nfz = 0;  // plane k+1 is the own cell's only below the chunk's end (else the next chunk's)
      dk1 = limited_slope<LIM>(w0, w1, w2, nfz);
      if (k + 1 < z1) nfb += nfz;
      face_flux(2, add_half(w0, dk, real(1)), add_half(w1, dk1, real(-1)), gamma, gm1, fz_hi);
    }

    // x face tx and y face ty of the own cell, then the tail faces
    {
      real F[5];
      face_flux(0, qprim(S.xp4[ty][tx], S.xpp[ty][tx]), qprim(S.xm4[ty][tx + 1], S.xmp[ty][tx + 1]),
                gamma, gm1, F);
      S.fx4[ty][tx] = Q4<real>{F[0], F[1], F[2], F[3]};
      S.fxe[ty][tx] = F[4];
      face_flux(1, qprim(S.yp4[ty][tx], S.ypp[ty][tx]), qprim(S.ym4[ty + 1][tx], S.ymp[ty + 1][tx]),
                gamma, gm1, F);
      S.fy4[ty][tx] = Q4<real>{F[0], F[1], F[2], F[3]};
      S.fye[ty][tx] = F[4];
    }
    if (fx_tail) {
      const int ly = tid & 31;
      real F[5];
      face_flux(0, qprim(S.xp4[ly][BX], S.xpp[ly][BX]), qprim(S.xm4[ly][BX + 1], S.xmp[ly][BX + 1]),
                gamma, gm1, F);
      S.fx4[ly][BX] = Q4<real>{F[0], F[1], F[2], F[3]};
      S.fxe[ly][BX] = F[4];
    }
    if (fy_tail) {
      real F[5];
      face_flux(1, qprim(S.yp4[BY][tx], S.ypp[BY][tx]), qprim(S.ym4[BY + 1][tx], S.ymp[BY + 1][tx]),
                gamma, gm1, F);
      S.fy4[BY][tx] = Q4<real>{F[0], F[1], F[2], F[3]};
      S.fye[BY][tx] = F[4];
    }
    __syncthreads();  // ---- fluxes ready

    if (active) {
      real u[5];
      if (COMB) {
#pragma unroll
        for (int c = 0; c < 5; ++c) uin[c] = __ldg(p.U + c * n3 + idx);
      }
      const Q4<real> fxr = S.fx4[ty][tx + 1], fxl = S.fx4[ty][tx];
      const Q4<real> fyr = S.fy4[ty + 1][tx], fyl = S.fy4[ty][tx];
      const real fxh[4] = {fxr.a, fxr.b, fxr.c, fxr.d}, fxo[4] = {fxl.a, fxl.b, fxl.c, fxl.d};
      const real fyh[4] = {fyr.a, fyr.b, fyr.c, fyr.d}, fyo[4] = {fyl.a, fyl.b, fyl.c, fyl.d};
      if constexpr (std::is_same<real, float>::value) {
        // components (0,1) and (2,3) as packed pairs, 4 alone
#pragma unroll
        for (int c = 0; c < 4; c += 2) {
          const float2 dfx = p_sub(f2(fxh[c], fxh[c + 1]), f2(fxo[c], fxo[c + 1]));
          const float2 dfy = p_sub(f2(fyh[c], fyh[c + 1]), f2(fyo[c], fyo[c + 1]));
          const float2 dfz = p_sub(f2(fz_hi[c], fz_hi[c + 1]), f2(fz_lo[c], fz_lo[c + 1]));
          float2 L = p_mul(dfx, f2s(-p.idx));
          L = p_fma(dfy, f2s(-p.idy), L);
          L = p_fma(dfz, f2s(-p.idz), L);
          float2 v = p_fma(f2s(dt), L, f2(uin[c], uin[c + 1]));
          if (COMB) v = p_fma(f2s(w0), f2(un[c], un[c + 1]), p_mul(f2s(w1), v));
          u[c] = v.x;
          u[c + 1] = v.y;
        }
        {
          float L = -((S.fxe[ty][tx + 1] - S.fxe[ty][tx]) * p.idx);
          L -= (S.fye[ty + 1][tx] - S.fye[ty][tx]) * p.idy;
          L -= (fz_hi[4] - fz_lo[4]) * p.idz;
          u[4] = STAGE == 1 ? uin[4] + dt * L : w0 * un[4] + w1 * (uin[4] + dt * L);
        }
      } else {
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          const real fxd = c < 4 ? fxh[c < 4 ? c : 0] - fxo[c < 4 ? c : 0] : S.fxe[ty][tx + 1] - S.fxe[ty][tx];
          const real fyd = c < 4 ? fyh[c < 4 ? c : 0] - fyo[c < 4 ? c : 0] : S.fye[ty + 1][tx] - S.fye[ty][tx];
          real L = -(fxd * p.idx);
          L -= fyd * p.idy;
          L -= (fz_hi[c] - fz_lo[c]) * p.idz;
          if (STAGE == 1) u[c] = uin[c] + dt * L;
          else u[c] = w0 * un[c] + w1 * (uin[c] + dt * L);
        }
      }
      if (COMB && final) {
        if (p.pre_src) {
#pragma unroll
          for (int c = 0; c < 5; ++c) p.pre_src[c * n3 + idx] = u[c];
        }
        if (forcing) {
          // a = 2 Re sum_{n_x} B_{n_x} exp(2 pi i n_x x~)  (Sec. 3.1.1)
          real a[3];
#pragma unroll
          for (int c = 0; c < 3; ++c)
            a[c] = real(2) * (S.fB[ty][0][c][0] +
                              (S.fB[ty][1][c][0] * twx[0] - S.fB[ty][1][c][1] * twx[1]) +
                              (S.fB[ty][2][c][0] * twx[2] - S.fB[ty][2][c][1] * twx[3]));
          const real e = (u[1] * a[0] + u[2] * a[1] + u[3] * a[2]) * dt;
          u[1] = u[1] + u[0] * a[0] * dt;
          u[2] = u[2] + u[0] * a[1] * dt;
          u[3] = u[3] + u[0] * a[2] * dt;
          u[4] = u[4] + e;
        }
        if (p.cooling)
          u[4] = cooling_energy(u[0], u[1], u[2], u[3], u[4], dt, gm1, p.t_floor, p.cool_frac,
                                p.nsub_max, flags, nsub_seen);
        bool finite = true;
#pragma unroll
        for (int c = 0; c < 5; ++c) finite = finite && isfinite(u[c]);
        if (!finite) {
          flags |= FLAG_NONFINITE;
        } else {
          const real pr = gm1 * (u[4] - real(0.5) * q_div(u[1] * u[1] + u[2] * u[2] + u[3] * u[3], u[0]));
          if (!(u[0] > real(0)) || !(pr > real(0))) flags |= FLAG_POSITIVITY;
          if (p.reduce_cfl) {
            tmin = fmin(tmin, cfl_time(u[0], u[1], u[2], u[3], u[4], gamma, gm1, p.dx, p.dy, p.dz));
            if (p.cool_ratio > real(0))
              tmin = fmin(tmin, p.cool_ratio * cooling_time(u[0], u[1], u[2], u[3], u[4], gm1, p.t_floor));
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 5; ++c) p.out[c * n3 + idx] = u[c];
    }
    dk = dk1;
#pragma unroll
    for (int c = 0; c < 5; ++c) fz_lo[c] = fz_hi[c];
  }

  if (s_abort) {
    // a staging wait gave up: nothing this CTA would write is valid; the step fails
    if (tid == 0) {
      atomicOr(&p.rec->flags, FLAG_TIMEOUT);
      atomicCAS(&p.rec->fail_step, -1, (int)(p.rec->nstep - 1));
    }
    return;
  }

  if (p.count_fallbacks) {
    unsigned long long n = active ? (unsigned long long)nfb : 0ull;
    if (__any_sync(0xffffffffu, n != 0ull)) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
      if ((tid & 31) == 0) atomicAdd(&p.rec->slope_fallbacks, n);
    }
  }

  if (COMB) {
    if (flags) {
      atomicOr(&p.rec->flags, flags);
      if (flags & FATAL_FLAGS) atomicCAS(&p.rec->fail_step, -1, (int)(p.rec->nstep - 1));
    }
    if (nsub_seen > 1) atomicMax(&p.rec->cool_nsub_max, nsub_seen);
    if (p.reduce_cfl) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) tmin = fmin(tmin, __shfl_xor_sync(0xffffffffu, tmin, o));
      __syncthreads();
      if ((tid & 31) == 0) S.red[tid >> 5] = tmin;
      __syncthreads();
      if (tid == 0) {
        real m = S.red[0];
        for (int w = 1; w < NTHREADS / 32; ++w) m = fmin(m, S.red[w]);
        if (m < real(INFINITY)) atomicMin(&p.rec->cfl_min_bits, ordered_bits(m));
      }
    }
  }
}

int sm_count() {
  static int n = 0;
  if (n <= 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = 148;
  }
  return n;
}

int wave_zchunk(long long tiles, int nz, int resident_per_sm, double prologue, int min_planes) {
  const long long slots = (long long)sm_count() * (resident_per_sm > 0 ? resident_per_sm : 1);
  int best = nz;
  double bestv = -1.0;
  const int mp = min_planes > 0 ? min_planes : 1;
  const int cmax = nz / mp > 1 ? nz / mp : 1;
  for (int c = 1; c <= cmax; ++c) {
    const int zc = (nz + c - 1) / c;
    const int chunks = (nz + zc - 1) / zc;
    const long long waves = (tiles * chunks + slots - 1) / slots;
    const double fill = (double)tiles * nz / ((double)waves * slots * zc);
    const double v = fill * zc / (zc + prologue);
    if (v > bestv + 1e-9) {
      bestv = v;
      best = zc;
    }
  }
  return best;
}

// ---- tensor maps of state buffers (cached per base address and shape) ----------------------
namespace {
struct TmaEntry {
  const void* base;
  int nx, ny, nz, esize, bx, by, xw, yh;
  StageTma maps;
};
std::mutex g_tma_mutex;
std::vector<TmaEntry> g_tma_cache;
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
bool g_encode_failed = false;

bool encode_box(CUtensorMap* m, const void* base, int nx, int ny, int nz, int esize, int bx, int by) {
  const cuuint64_t dims[4] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz, 5};
  const cuuint64_t strides[3] = {(cuuint64_t)nx * esize, (cuuint64_t)nx * ny * esize,
                                 (cuuint64_t)nx * ny * nz * esize};
  const cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, 1, 5};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return g_encode(m, esize == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                  4, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace

bool stage_tma_maps(const void* base, int nx, int ny, int nz, int esize, int bx, int by, int xw,
                    int yh, StageTma* out) {
  std::lock_guard<std::mutex> lock(g_tma_mutex);
  for (const TmaEntry& e : g_tma_cache)
    if (e.base == base && e.nx == nx && e.ny == ny && e.nz == nz && e.esize == esize && e.bx == bx &&
        e.by == by && e.xw == xw && e.yh == yh) {
      *out = e.maps;
      return true;
    }
  if (g_encode_failed) return false;
  if (!g_encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      g_encode_failed = true;
      return false;
    }
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  TmaEntry e{base, nx, ny, nz, esize, bx, by, xw, yh, {}};
  if (!encode_box(&e.maps.core, base, nx, ny, nz, esize, bx, by) ||
      !encode_box(&e.maps.xh, base, nx, ny, nz, esize, xw, by) ||
      !encode_box(&e.maps.yh, base, nx, ny, nz, esize, bx, yh))
    return false;
  if (g_tma_cache.size() >= 64) g_tma_cache.erase(g_tma_cache.begin());
  g_tma_cache.push_back(e);
  *out = e.maps;
  return true;
}

template <typename real, int STAGE, int LIM>
static cudaError_t launch_stage_t(const StageArgs<real>& a, cudaStream_t s) {
  auto kernel = stage_kernel<real, STAGE, LIM>;
  const size_t smem = sizeof(StageSmem<real>);
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  static int resident = 0;   // CTAs per SM of this instance
  if (resident <= 0) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, kernel, NTHREADS, smem);
    if (e != cudaSuccess) return e;
    if (resident <= 0) resident = 1;
  }
  const long long tiles = (long long)((a.nx + BX - 1) / BX) * ((a.ny + BY - 1) / BY);
  const int zc = wave_zchunk(tiles, a.nz, resident, 1.0);
  dim3 grid((a.nx + BX - 1) / BX, (a.ny + BY - 1) / BY, (a.nz + zc - 1) / zc);
  // TMA boxes need whole tiles (so that every halo strip is contiguous), a 16-byte aligned base
  // and rows of a multiple of 16 bytes
  StageTma maps;
  std::memset(&maps, 0, sizeof(maps));
  const bool tma_ok = a.nx % BX == 0 && a.ny % BY == 0 && a.ny >= 2 &&
                      ((unsigned long long)a.U & 15ull) == 0 &&
                      stage_tma_maps(a.U, a.nx, a.ny, a.nz, (int)sizeof(real), BX, BY,
                                     Staging<real>::SCE, 2, &maps);
  kernel<<<grid, NTHREADS, smem, s>>>(a, zc, maps, tma_ok ? 1 : 0);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_stage(int stage, const StageArgs<real>& a, cudaStream_t s, int* launched) {
  cudaError_t pe = cudaSuccess;
  int n = 0;
  if (launch_stage_pair<real>(stage, a, s, pe, n)) {
    if (launched) *launched = n;
    return pe;
  }
  if (launched) *launched = 1;
  if (a.limiter == LIM_VL) {
    if (stage == 1) return launch_stage_t<real, 1, LIM_VL>(a, s);
    if (stage == 2) return launch_stage_t<real, 2, LIM_VL>(a, s);
    return launch_stage_t<real, 3, LIM_VL>(a, s);
  }
  if (stage == 1) return launch_stage_t<real, 1, LIM_MC>(a, s);
  if (stage == 2) return launch_stage_t<real, 2, LIM_MC>(a, s);
  return launch_stage_t<real, 3, LIM_MC>(a, s);
}
template cudaError_t launch_stage<float>(int, const StageArgs<float>&, cudaStream_t, int*);
template cudaError_t launch_stage<double>(int, const StageArgs<double>&, cudaStream_t, int*);

// ---------------------------------------------------------------------------------------------
// OU forcing draws (Sec. 3.1.1): counter-based SplitMix64 stream, Box-Muller pairs.
// key = splitmix64(seed); word i = splitmix64(key + i * golden); draw d, mode m, component c
// uses words 2*((16 d + m) * 3 + c) and the next one.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  unsigned long long z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double unit_uniform(unsigned long long w) {
  return ((double)(w >> 11) + 0.5) * 0x1.0p-53;
}

// Projected Gaussian draw eta (re, im) for lane (m, c) of draw d.  Every thread of the block
// calls this (it synchronises); lanes >= 48 only take part in the barrier.
__device__ void projected_draw(unsigned long long seed, long long d, int lane_in, double* sre,
                               double* sim, double& ere, double& eim) {
  const bool writer = lane_in < 48;
  const int lane = writer ? lane_in : 47;
  const int m = lane / 3, c = lane - 3 * m;
  const unsigned long long key = splitmix64(seed);
  const unsigned long long i0 = 2ull * (unsigned long long)((d * 16 + m) * 3 + c);
  const double u1 = unit_uniform(splitmix64(key + i0 * 0x9E3779B97F4A7C15ull));
  const double u2 = unit_uniform(splitmix64(key + (i0 + 1) * 0x9E3779B97F4A7C15ull));
  const double r = sqrt(-2.0 * log(u1));
  double sn, cs;
  sincospi(2.0 * u2, &sn, &cs);
  if (writer) {
    sre[lane] = r * cs;
    sim[lane] = r * sn;
  }
  __syncthreads();
  int nv[3];
  // mode vector of m (runtime lookup of the compile-time enumeration)
  nv[0] = nv[1] = nv[2] = 0;
#pragma unroll
  for (int q = 0; q < 16; ++q)
    if (q == m) {
      nv[0] = forced_mode_component(q, 0);
      nv[1] = forced_mode_component(q, 1);
      nv[2] = forced_mode_component(q, 2);
    }
  const double k2 = (double)(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
  double pre = 0.0, pim = 0.0;
  for (int j = 0; j < 3; ++j) {
    const double P = (c == j ? 1.0 : 0.0) - (double)nv[c] * (double)nv[j] / k2;
    pre += P * sre[3 * m + j];
    pim += P * sim[3 * m + j];
  }
  ere = pre;
  eim = pim;
}

__global__ void forcing_init_kernel(double* ahat, unsigned long long seed) {
  __shared__ double sre[48], sim[48];
  const int lane = threadIdx.x;
  double ere, eim;
  projected_draw(seed, 0, lane, sre, sim, ere, eim);
  if (lane < 48) {
    ahat[2 * lane] = ere;
    ahat[2 * lane + 1] = eim;
  }
}

cudaError_t launch_forcing_init(double* ahat, unsigned long long seed, cudaStream_t s) {
  forcing_init_kernel<<<1, 64, 0, s>>>(ahat, seed);
  return cudaGetLastError();
}

// The draws of a run of steps ahead of time: the float64 Box-Muller transform of one step is a
// latency chain on one warp, so computing many steps' draws side by side takes it off the
// steps' critical path.  Block b holds draw first + b; the values are those projected_draw
// gives inside step_begin_kernel.
__global__ void ou_draws_kernel(unsigned long long seed, long long first, double* out) {
  __shared__ double sre[48], sim[48];
  const int lane = threadIdx.x;
  double ere, eim;
  projected_draw(seed, first + blockIdx.x, lane, sre, sim, ere, eim);
  if (lane < 48) {
    out[96LL * blockIdx.x + 2 * lane] = ere;
    out[96LL * blockIdx.x + 2 * lane + 1] = eim;
  }
}

cudaError_t launch_ou_draws(unsigned long long seed, long long first, int count, double* out,
                            cudaStream_t s) {
  if (count < 1) return cudaSuccess;
  ou_draws_kernel<<<count, 64, 0, s>>>(seed, first, out);
  return cudaGetLastError();
}

template <typename real>
__device__ void store_norm(void* out, int i, double v) {
  reinterpret_cast<real*>(out)[i] = (real)v;
}

// Step prologue: choose dt (App. A.4 or the caller's), reset the CFL accumulator, advance the
// OU table (Sec. 3.1.1) and its normalisation, then advance t and the step count.
__global__ void step_begin_kernel(BeginArgs a) {
  __shared__ double sre[48], sim[48], sq[64];
  __shared__ double s_dt;
  __shared__ unsigned s_skip;
  StepRecord* rec = a.rec;
  const int lane = threadIdx.x;
  if (lane == 0) s_skip = *((volatile unsigned*)&rec->flags) & FATAL_FLAGS;
  __syncthreads();
  if (s_skip) return;
  if (lane == 0) {
    double dt = a.dt_fixed;
    if (!(dt > 0.0)) {
      const unsigned long long b = rec->cfl_min_bits;
      const double m = a.precision == 0 ? (double)__uint_as_float((unsigned)b)
                                        : __longlong_as_double((long long)b);
      dt = fmin(a.cfl * m, a.dt_max);
    }
    s_dt = dt;
  }
  __syncthreads();
  const double dt = s_dt;
  if (a.forcing) {
    double ere = 0.0, eim = 0.0;
    if (!a.hold) {
      const long long d = rec->nstep + 1;   // block-uniform: either branch is taken by all
      if (a.draws && d >= a.draw_first && d < a.draw_first + a.draw_count) {
        if (lane < 48) {
          ere = a.draws[96 * (d - a.draw_first) + 2 * lane];
          eim = a.draws[96 * (d - a.draw_first) + 2 * lane + 1];
        }
      } else {
        projected_draw(a.seed, d, lane, sre, sim, ere, eim);
      }
    }
    const double f = a.hold ? 1.0 : exp(-dt / a.tau);
    const double g = a.hold ? 0.0 : sqrt(1.0 - f * f);
    double nre = 0.0, nim = 0.0;
    if (lane < 48) {
      const double ore = a.ahat[2 * lane], oim = a.ahat[2 * lane + 1];
      a.ahat_prev[2 * lane] = ore;
      a.ahat_prev[2 * lane + 1] = oim;
      nre = a.hold ? ore : f * ore + g * ere;
      nim = a.hold ? oim : f * oim + g * eim;
      a.ahat[2 * lane] = nre;
      a.ahat[2 * lane + 1] = nim;
    }
    sq[lane] = nre * nre + nim * nim;
    __syncthreads();
    if (lane == 0) {
      double s = 0.0;
      for (int q = 0; q < 48; ++q) s += sq[q];
      sq[0] = a.arms / sqrt(2.0 * s);
      rec->ou_norm = sq[0];
    }
    __syncthreads();
    const double scale = sq[0];
    if (lane < 48) {
      if (a.precision == 0) {
        store_norm<float>(a.ahat_norm, 2 * lane, scale * nre);
        store_norm<float>(a.ahat_norm, 2 * lane + 1, scale * nim);
      } else {
        store_norm<double>(a.ahat_norm, 2 * lane, scale * nre);
        store_norm<double>(a.ahat_norm, 2 * lane + 1, scale * nim);
      }
    }
  }
  if (lane == 0) {
    rec->dt = dt;
    rec->cfl_min_bits = a.precision == 0 ? (unsigned long long)__float_as_uint(INFINITY)
                                         : (unsigned long long)__double_as_longlong(INFINITY);
    rec->t += dt;
    rec->nstep += 1;
  }
}

cudaError_t launch_step_begin(const BeginArgs& a, cudaStream_t s) {
  step_begin_kernel<<<1, 64, 0, s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// CFL minimum of a state (App. A.4), used for the first step after init_state.
template <typename real>
__global__ void cfl_reduce_kernel(const real* __restrict__ U, long long n3, int nx, int ny,
                                  real gamma, real gm1, real dx, real dy, real dz,
                                  real cool_ratio, real t_floor, StepRecord* rec) {
  __shared__ real red[8];
  real m = real(INFINITY);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n3;
       i += (long long)gridDim.x * blockDim.x) {
    const real r = __ldg(U + i), mx = __ldg(U + n3 + i), my = __ldg(U + 2 * n3 + i);
    const real mz = __ldg(U + 3 * n3 + i), E = __ldg(U + 4 * n3 + i);
    m = fmin(m, cfl_time(r, mx, my, mz, E, gamma, gm1, dx, dy, dz));
    if (cool_ratio > real(0)) m = fmin(m, cool_ratio * cooling_time(r, mx, my, mz, E, gm1, t_floor));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x / 32); ++w) m = fmin(m, red[w]);
    if (m < real(INFINITY)) atomicMin(&rec->cfl_min_bits, ordered_bits(m));
  }
}

template <typename real>
cudaError_t launch_cfl_reduce(const real* U, int nx, int ny, int nz, real gamma, real dx, real dy,
                              real dz, real cool_ratio, real t_floor, StepRecord* rec,
                              cudaStream_t s) {
  const long long n3 = (long long)nx * ny * nz;
  long long blocks = (n3 + 255) / 256;
  if (blocks > 148 * 8) blocks = 148 * 8;
  cfl_reduce_kernel<real><<<(int)blocks, 256, 0, s>>>(U, n3, nx, ny, gamma, gamma - real(1), dx,
                                                      dy, dz, cool_ratio, t_floor, rec);
  return cudaGetLastError();
}
template cudaError_t launch_cfl_reduce<float>(const float*, int, int, int, float, float, float,
                                              float, float, float, StepRecord*, cudaStream_t);
template cudaError_t launch_cfl_reduce<double>(const double*, int, int, int, double, double,
                                               double, double, double, double, StepRecord*,
                                               cudaStream_t);

// ---------------------------------------------------------------------------------------------
// Conserved totals in float64 with a fixed reduction order (two passes, no atomics).
// Conserved totals: a fixed grid of 6 CTAs per SM on 148 SMs, each CTA summing its own
// contiguous range of every field, then fixed-order reductions, so the result is the same on
// every call.
constexpr int TOTALS_BLOCKS = 148 * 6, TOTALS_THREADS = 256;
int totals_blocks() { return TOTALS_BLOCKS; }

// Sum over the CTA of five doubles per thread (warp shuffles, then the warps in order);
// thread 0 writes them to partials[blockIdx.x * 5 + f].
__device__ __forceinline__ void totals_block_store(double s[5], double* __restrict__ partials) {
  __shared__ double red[TOTALS_THREADS / 32][5];
#pragma unroll
  for (int f = 0; f < 5; ++f)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s[f] += __shfl_xor_sync(0xffffffffu, s[f], o);
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int f = 0; f < 5; ++f) red[threadIdx.x >> 5][f] = s[f];
  __syncthreads();
  if (threadIdx.x < 5) {
    double t = 0.0;
    for (int w = 0; w < TOTALS_THREADS / 32; ++w) t += red[w][threadIdx.x];
    partials[blockIdx.x * 5 + threadIdx.x] = t;
  }
}

template <typename real>
__global__ void __launch_bounds__(TOTALS_THREADS, TOTALS_BLOCKS / 148)
totals_partial_kernel(const real* __restrict__ U, long long n3, double* __restrict__ partials) {
  double s[5] = {0, 0, 0, 0, 0};
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if constexpr (std::is_same<real, float>::value) {
    // float32 state: 16-byte loads (when every field starts 16-byte aligned); each thread adds
    // 8 values per field in compensated float32 (TwoSum: the chunk's sum to a few eps32^2 of
    // its magnitude) and the chunks into a float-float running sum (accurate double-word
    // addition, relative error a few eps32^2 per chunk); float64 only at the end, since
    // float64 operations are scarce on this part
    const bool vec = (n3 % 4 == 0) && (((unsigned long long)U & 15ull) == 0);
    long long done = 0;   // elements covered by the vector loop
    ff2 tot[5];
#pragma unroll
    for (int f = 0; f < 5; ++f) tot[f] = ff2{0.0f, 0.0f};
    if (vec) {
      // each CTA streams its own contiguous range of every field, one field after the other
      const long long n4 = n3 / 4;
      const float4* __restrict__ U4 = reinterpret_cast<const float4*>(U);
      const long long per = (n4 + gridDim.x - 1) / gridDim.x;
      const long long b0 = (long long)blockIdx.x * per, b1 = b0 + per < n4 ? b0 + per : n4;
      const int bs = blockDim.x;
#pragma unroll 1
      for (int f = 0; f < 5; ++f) {
        const float4* __restrict__ Uf = U4 + f * n4;
        ff2 tf{0.0f, 0.0f};
        for (long long i = b0 + threadIdx.x; i < b1; i += 4 * bs) {
          float4 a[4];
#pragma unroll
          for (int u = 0; u < 4; ++u)
            a[u] = i + u * bs < b1 ? __ldg(Uf + i + u * bs) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            ff2 acc{0.0f, 0.0f};
            ff_acc(acc, a[2 * h].x); ff_acc(acc, a[2 * h].y);
            ff_acc(acc, a[2 * h].z); ff_acc(acc, a[2 * h].w);
            ff_acc(acc, a[2 * h + 1].x); ff_acc(acc, a[2 * h + 1].y);
            ff_acc(acc, a[2 * h + 1].z); ff_acc(acc, a[2 * h + 1].w);
            tf = ff_add(tf, ff_two_sum(acc.hi, acc.lo));
          }
        }
#pragma unroll
        for (int q = 0; q < 5; ++q)
          if (q == f) tot[q] = tf;
      }
      done = n3;
    }
    constexpr int CH = 8;
    for (long long i = done + t0; i < n3; i += (long long)CH * stride) {
      ff2 acc[5];
#pragma unroll
      for (int f = 0; f < 5; ++f) acc[f] = ff2{0.0f, 0.0f};
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const long long idx = i + (long long)u * stride;
        if (idx < n3) {
#pragma unroll
          for (int f = 0; f < 5; ++f) ff_acc(acc[f], __ldg(U + f * n3 + idx));
        }
      }
#pragma unroll
      for (int f = 0; f < 5; ++f) tot[f] = ff_add(tot[f], ff_two_sum(acc[f].hi, acc[f].lo));
    }
#pragma unroll
    for (int f = 0; f < 5; ++f) s[f] = (double)tot[f].hi + (double)tot[f].lo;
  } else {
    for (long long i = t0; i < n3; i += stride) {
#pragma unroll
      for (int f = 0; f < 5; ++f) s[f] += (double)__ldg(U + f * n3 + i);
    }
  }
  totals_block_store(s, partials);
}

// One warp per field adds the CTA partials in a fixed order.
__global__ void totals_final_kernel(const double* __restrict__ partials, int nblocks,
                                    double* __restrict__ out) {
  const int f = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (f >= 5) return;
  double t = 0.0;
  for (int b = lane; b < nblocks; b += 32) t += partials[b * 5 + f];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (lane == 0) out[f] = t;
}

template <typename real>
cudaError_t launch_totals(const real* U, long long n3, double* partials, int nblocks, double* out5,
                          cudaStream_t s) {
  totals_partial_kernel<real><<<nblocks, TOTALS_THREADS, 0, s>>>(U, n3, partials);
  totals_final_kernel<<<1, 5 * 32, 0, s>>>(partials, nblocks, out5);
  return cudaGetLastError();
}
// Minima over cells of rho and P = (gamma - 1)(E - |m|^2 / (2 rho)) (the step diagnostics):
// per-block minima into partials[2 b], [2 b + 1], then out2 = the minima over the blocks.
template <typename real>
__global__ void __launch_bounds__(TOTALS_THREADS)
minima_partial_kernel(const real* __restrict__ U, long long n3, double gm1,
                      double* __restrict__ partials) {
  __shared__ double red[2][TOTALS_THREADS / 32];
  double mr = INFINITY, mp = INFINITY;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n3;
       q += (long long)gridDim.x * blockDim.x) {
    const double r = U[q], mx = U[n3 + q], my = U[2 * n3 + q], mz = U[3 * n3 + q], E = U[4 * n3 + q];
    mr = fmin(mr, r);
    mp = fmin(mp, gm1 * (E - 0.5 * (mx * mx + my * my + mz * mz) / r));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mr = fmin(mr, __shfl_xor_sync(0xffffffffu, mr, o));
    mp = fmin(mp, __shfl_xor_sync(0xffffffffu, mp, o));
  }
  if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = mr; red[1][threadIdx.x >> 5] = mp; }
  __syncthreads();
  if (threadIdx.x < 2) {
    double m = INFINITY;
    for (int w = 0; w < TOTALS_THREADS / 32; ++w) m = fmin(m, red[threadIdx.x][w]);
    partials[2 * blockIdx.x + threadIdx.x] = m;
  }
}

__global__ void minima_final_kernel(const double* __restrict__ partials, int nblocks,
                                    double* __restrict__ out2) {
  const int f = threadIdx.x;
  if (f < 2) {
    double m = INFINITY;
    for (int b = 0; b < nblocks; ++b) m = fmin(m, partials[2 * b + f]);
    out2[f] = m;
  }
}

template <typename real>
cudaError_t launch_minima(const real* U, long long n3, double gamma, double* partials, int nblocks,
                          double* out2, cudaStream_t s) {
  minima_partial_kernel<real><<<nblocks, TOTALS_THREADS, 0, s>>>(U, n3, gamma - 1.0, partials);
  minima_final_kernel<<<1, 32, 0, s>>>(partials, nblocks, out2);
  return cudaGetLastError();
}
template cudaError_t launch_minima<float>(const float*, long long, double, double*, int, double*,
                                          cudaStream_t);
template cudaError_t launch_minima<double>(const double*, long long, double, double*, int, double*,
                                           cudaStream_t);

template cudaError_t launch_totals<float>(const float*, long long, double*, int, double*,
                                          cudaStream_t);
template cudaError_t launch_totals<double>(const double*, long long, double*, int, double*,
                                           cudaStream_t);

// ---------------------------------------------------------------------------------------------
template <typename real>
__global__ void forcing_field_kernel(const real* __restrict__ ah, const real* tw0,
                                     const real* tw1, const real* tw2, int nx, int ny, int nz,
                                     real* __restrict__ out) {
  const long long n3 = (long long)nx * ny * nz;
  const real* tw[3] = {tw0, tw1, tw2};
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n3;
       q += (long long)gridDim.x * blockDim.x) {
    const unsigned t = (unsigned)q / (unsigned)nx;   // grids below 2^31 cells
    const int i = (int)((unsigned)q - t * (unsigned)nx);
    const int j = (int)(t % (unsigned)ny);
    const int k = (int)(t / (unsigned)ny);
    real a[3];
    forcing_accel(ah, tw, i, j, k, a);
    out[q] = a[0];
    out[n3 + q] = a[1];
    out[2 * n3 + q] = a[2];
  }
}

template <typename real>
cudaError_t launch_forcing_field(const real* ahat_norm, const real* const tw[3], int nx, int ny,
                                 int nz, real* a_out, cudaStream_t s) {
  const long long n3 = (long long)nx * ny * nz;
  long long blocks = (n3 + 255) / 256;
  if (blocks > 148 * 8) blocks = 148 * 8;
  forcing_field_kernel<real><<<(int)blocks, 256, 0, s>>>(ahat_norm, tw[0], tw[1], tw[2], nx, ny,
                                                         nz, a_out);
  return cudaGetLastError();
}
template cudaError_t launch_forcing_field<float>(const float*, const float* const[3], int, int,
                                                 int, float*, cudaStream_t);
template cudaError_t launch_forcing_field<double>(const double*, const double* const[3], int,
                                                  int, int, double*, cudaStream_t);

// ---------------------------------------------------------------------------------------------
// Block mean of a float32 state over factor^3 fine cells (conservative restriction of the
// conserved fields onto a coarser grid).
__global__ void downsample_kernel(const float* __restrict__ Uf, int nx, int ny, int nz, int r,
                                  float* __restrict__ Uc) {
  const int cx = nx / r, cy = ny / r, cz = nz / r;
  const long long nc = (long long)cx * cy * cz, nf = (long long)nx * ny * nz;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nc * 5;
       q += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(q / nc);
    const long long c = q - (long long)f * nc;
    const int I = (int)(c % cx);
    const long long t = c / cx;
    const int J = (int)(t % cy), K = (int)(t / cy);
    double s = 0.0;
    for (int dk = 0; dk < r; ++dk)
      for (int dj = 0; dj < r; ++dj)
        for (int di = 0; di < r; ++di)
          s += (double)Uf[(long long)f * nf + ((long long)(K * r + dk) * ny + (J * r + dj)) * nx + (I * r + di)];
    Uc[q] = (float)(s / (double)(r * r * r));
  }
}

}  // namespace dh

extern "C" dh_status dh_downsample(const float* Uf, int nx, int ny, int nz, int factor, float* Uc,
                                   void* stream) {
  if (!Uf || !Uc || factor < 1 || nx % factor || ny % factor || nz % factor) return DH_ERR_ARG;
  const long long nc = (long long)(nx / factor) * (ny / factor) * (nz / factor) * 5;
  long long b = (nc + 255) / 256;
  if (b > 148 * 8) b = 148 * 8;
  dh::downsample_kernel<<<(int)b, 256, 0, (cudaStream_t)stream>>>(Uf, nx, ny, nz, factor, Uc);
  return cudaGetLastError() == cudaSuccess ? DH_OK : DH_ERR_CUDA;
}
