// Hand-written adjoint of the RK2 step (reverse of App. A.1-A.3, dt frozen per App. A.4) and
// the checkpointed driver behind dh_adjoint_advance (Sec. 2.3: sparse stored states, segments
// recomputed during the backward sweep).
//
// stage_adjoint_kernel computes, for one RK2 stage out = alpha U0 + beta (U + dt L(U)),
//   lam_in = c1 lam_out + c2 extra + (dL/dU)^T mu,   mu = beta dt lam_out,
// as a gather per cell.  Per plane of a CTA tile: the limited slopes and face states of every
// cell the tile's faces touch are computed once (x and y in shared memory, z in a per-thread
// register pipeline); every face VJP of HLLC is evaluated once on those states; the limiter's
// transposed stencil (slope VJPs) is evaluated once per cell and axis and gathered from the
// neighbouring cells; the primitive-recovery Jacobian is applied last.  No atomics; each output
// cell is written by one thread.  The conserved variables of the plane three ahead and the
// plane's lam_out arrive by cp.async while the previous phases compute.
//
// Kink convention: the derivative of the branch the forward took; exact ties of min/max split
// the derivative evenly between the tied arguments (the MC limiter and the Davis speeds).
#include <math.h>
#include <vector>

#include <string.h>

#include "async_copy.cuh"
#include "dh_internal.h"
#include "tc_ptx.cuh"
#include "tma.cuh"
#include "dh_adjoint.cuh"
#include "dh_sources.cuh"

namespace dh {

constexpr int ABX = 32, ABY = 8;
constexpr int ANT = ABX * ABY;
constexpr int WX = ABX + 6, WY = ABY + 6;   // primitive planes, halo 3
constexpr int MXH = ABX + 4, MYH = ABY + 4; // mu plane, halo 2
constexpr int NSXA = ABX + 4;               // x slopes per row: cells -2 .. BX+1
constexpr int NSYA = ABY + 4;               // y slopes per column: cells -2 .. BY+1
constexpr int NFXA = ABX + 3;               // x faces per row: -3/2 .. BX+1/2
constexpr int NFYA = ABY + 3;               // y faces per column
constexpr int NCXA = ABX + 2;               // x cells per row for the slope terms: -1 .. BX
constexpr int NCYA = ABY + 2;
constexpr int NSX = NSXA * ABY, NSY = NSYA * ABX;   // x and y slopes of a plane tile
constexpr int NFX = NFXA * ABY, NFY = NFYA * ABX;   // x and y faces of a plane tile
constexpr int NCX = NCXA * ABY, NCY = NCYA * ABX;   // cells with x and y slope terms
// the y items of each per-plane loop start on a warp boundary, so no warp takes both branches
constexpr int warp_up(int n) { return (n + 31) / 32 * 32; }
constexpr int NSXP = warp_up(NSX), NFXP = warp_up(NFX), NCXP = warp_up(NCX);

// Staged conserved variables of the plane in flight, one dense buffer per TMA box: the tile
// core, x halos of 4 cells on each side (3 are read) and y halos of 3 rows.  The corner blocks
// are never read by the stencil (x slopes and terms read rows 0..ABY-1, y slopes and terms
// columns 0..ABX-1).  Each box is contiguous in global memory at any tile position (x0, y0 are
// multiples of ABX, ABY), so the periodic wrap is a start coordinate.
constexpr int AXH = 4, AYH = 3;
template <typename real> struct AdjStaging {
  static constexpr uint32_t BYTES = (uint32_t)sizeof(real) * 5u * (ABX * ABY + 2 * ABY * AXH + 2 * AYH * ABX);
};

template <typename real> struct AdjSmem {
  alignas(128) real core[5][ABY][ABX];   // staged plane: tile core
  alignas(128) real xl[5][ABY][AXH];     // x0 - 4 .. x0 - 1
  alignas(128) real xr[5][ABY][AXH];     // x0 + ABX .. x0 + ABX + 3
  alignas(128) real yt[5][AYH][ABX];     // y0 - 3 .. y0 - 1
  alignas(128) real yb[5][AYH][ABX];     // y0 + ABY .. y0 + ABY + 2
  real w[4][5][WY][WX];
  real mu[5][MYH][MXH];           // lam_out of plane k (the stage's beta dt is applied at use)
  real face[10][NFXP + NFY];      // (gL[5], gR[5]) per face: x faces, then y faces
  union {
    real st[10][NSXP + NSY];      // (W - dW/2, W + dW/2) per cell and axis: x, then y
    real cell[10][NCXP + NCY];    // (A[5], B[5]) per cell: x terms, then y terms
  } u;
  unsigned char zero[NSXP + NSY];  // 1: the limited slope of slope item t is all zero
  int xs[WX], ys[WY];
  alignas(8) uint64_t bar;         // staging plane landed (TMA transaction bytes)
};
// two CTAs per SM for the float32 instance: 2 x (size + 1 KB reserved) within 228 KB
static_assert(2 * (sizeof(AdjSmem<float>) + 1024) <= 228 * 1024, "adjoint shared memory");

template <typename real>
__device__ __forceinline__ Prim<real> ring_prim(const AdjSmem<real>& S, int slot, int sy, int sx) {
  return Prim<real>{S.w[slot][0][sy][sx], S.w[slot][1][sy][sx], S.w[slot][2][sy][sx],
                    S.w[slot][3][sy][sx], S.w[slot][4][sy][sx]};
}
// the same by flat ring offset (sy WX + sx)
template <typename real>
__device__ __forceinline__ Prim<real> ring_prim_at(const AdjSmem<real>& S, int slot, int off) {
  const real* b = &S.w[slot][0][0][0] + off;
  constexpr int FS = WX * WY;
  return Prim<real>{b[0], b[FS], b[2 * FS], b[3 * FS], b[4 * FS]};
}

template <typename real>
__device__ __forceinline__ bool zero_bit(const AdjSmem<real>& S, int i) {
  return S.zero[i] != 0;
}

template <typename real>
__device__ __forceinline__ Prim<real> st_prim(const AdjSmem<real>& S, int half, int i) {
  return Prim<real>{S.u.st[half][i], S.u.st[half + 1][i], S.u.st[half + 2][i],
                    S.u.st[half + 3][i], S.u.st[half + 4][i]};
}

template <typename real>
__device__ __forceinline__ Prim<real> gload_prim(const real* __restrict__ U, long long n3,
                                                 long long idx, real gm1) {
  return cons_to_prim(__ldg(U + idx), __ldg(U + n3 + idx), __ldg(U + 2 * n3 + idx),
                      __ldg(U + 3 * n3 + idx), __ldg(U + 4 * n3 + idx), gm1);
}

template <typename real>
__device__ __forceinline__ void gload5(const real* __restrict__ p, long long n3, long long idx,
                                       real out[5]) {
#pragma unroll
  for (int c = 0; c < 5; ++c) out[c] = __ldg(p + c * n3 + idx);
}

__device__ __forceinline__ void cp_async_elem(float* s, const float* g) { cp_async4(s, g); }
__device__ __forceinline__ void cp_async_elem(double* s, const double* g) { cp_async8(s, g); }

// Bound on the probes of the staging mbarrier (a plane's copies land in microseconds); a wait
// that reaches it sets FLAG_TIMEOUT and the CTA stops.
constexpr uint32_t ADJ_WAIT_ITERS = 1u << 22;

// Work of a plane.  Thread (tx, ty) owns tile cell (tx, ty): its x and y slopes, the x face
// between cells tx - 1 and tx and the y face between ty - 1 and ty, its x and y slope terms,
// its primitive conversion and its lam_out copy.  The halo work is a fixed tail per thread with
// offsets computed once: slopes of cells -2, -1, ABX, ABX + 1 (x) and -2, -1, ABY, ABY + 1 (y)
// (threads 96..255), the conversion of the 240 used halo cells (threads 0..239), the faces
// -3/2, ABX + 1/2, ABX + 3/2 (x) and the like in y (threads 136..255), the slope terms of cells
// -1 and ABX (x), -1 and ABY (y) (threads 0..79), and the 160 halo cells of lam_out (threads
// 96..255).
// float32: two CTAs per SM (its registers and shared memory are sized for it); float64: one
template <typename real, int LIM>
__global__ void __launch_bounds__(ANT, sizeof(real) == 4 ? 2 : 1)
stage_adjoint_kernel(const AdjointArgs<real> p, const int zchunk,
                     const __grid_constant__ StageTma tma, const int use_tma) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  AdjSmem<real>& S = *reinterpret_cast<AdjSmem<real>*>(smem_raw);
  __shared__ int s_abort;
  const int tid = threadIdx.x;
  const int tx = tid & (ABX - 1), ty = tid / ABX;
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  const long long plane = (long long)nx * ny;
  const long long n3 = plane * nz;
  const int x0 = blockIdx.x * ABX, y0 = blockIdx.y * ABY;
  const int z0 = blockIdx.z * zchunk;
  const int z1 = min(z0 + zchunk, nz);
  const real gamma = p.gamma, gm1 = p.gm1;
  const real dt = (real)*p.dtp;
  const real sdt = p.beta * dt;
  // flux gradients are beta dt times differences of lam_out
  const real gfx = sdt * p.idx, gfy = sdt * p.idy, gfz = sdt * p.idz;
  const int gx = x0 + tx, gy = y0 + ty;
  const bool active = gx < nx && gy < ny;
  const long long col = (long long)(gy % ny) * nx + (gx % nx);

  if (tid < WX) S.xs[tid] = ((x0 + tid - 3) % nx + nx) % nx;
  if (tid >= 64 && tid < 64 + WY) S.ys[tid - 64] = ((y0 + tid - 64 - 3) % ny + ny) % ny;
  if (tid == 96) {
    tc::mbar_init(&S.bar, 1u);
    tc::mbar_fence_init();
    s_abort = 0;
  }
  // box destinations must start on 128 bytes; the buffers are 128-byte multiples from S
  const bool via_tma = use_tma != 0 && (tc::smem_u32(&S.core[0][0][0]) & 127u) == 0u;
  const uint32_t bar = tc::smem_u32(&S.bar);
  const int xl0 = x0 >= AXH ? x0 - AXH : nx - AXH, xr0 = x0 + ABX < nx ? x0 + ABX : 0;
  const int yt0 = y0 >= AYH ? y0 - AYH : ny - AYH, yb0 = y0 + ABY < ny ? y0 + ABY : 0;
  __syncthreads();

  auto load_w = [&](int k, int slot) {
    const long long zoff = (long long)wrap(k, nz) * plane;
    for (int c = tid; c < WX * WY; c += ANT) {
      const int sy = c / WX, sx = c - sy * WX;
      const Prim<real> w = gload_prim(p.U, n3, zoff + (long long)S.ys[sy] * nx + S.xs[sx], gm1);
      S.w[slot][0][sy][sx] = w.r;
      S.w[slot][1][sy][sx] = w.vx;
      S.w[slot][2][sy][sx] = w.vy;
      S.w[slot][3][sy][sx] = w.vz;
      S.w[slot][4][sy][sx] = w.p;
    }
  };
  // The conserved variables of plane k into the staging buffers: TMA (one thread, five boxes
  // on the staging barrier), or element copies of every position (wrapped coordinates).
  auto stage_plane = [&](int k) {
    const int kz = wrap(k, nz);
    if (via_tma) {
      if (tid == 0) {
        tc::mbar_arrive_expect_tx(&S.bar, AdjStaging<real>::BYTES);
        tma_load_4d(tc::smem_u32(&S.core[0][0][0]), &tma.core, x0, y0, kz, 0, bar);
        tma_load_4d(tc::smem_u32(&S.xl[0][0][0]), &tma.xh, xl0, y0, kz, 0, bar);
        tma_load_4d(tc::smem_u32(&S.xr[0][0][0]), &tma.xh, xr0, y0, kz, 0, bar);
        tma_load_4d(tc::smem_u32(&S.yt[0][0][0]), &tma.yh, x0, yt0, kz, 0, bar);
        tma_load_4d(tc::smem_u32(&S.yb[0][0][0]), &tma.yh, x0, yb0, kz, 0, bar);
      }
      return;
    }
    const long long zoff = (long long)kz * plane;
    constexpr int NC = ABX * ABY, NXH = ABY * AXH, NYH = AYH * ABX;
    for (int c = tid; c < NC + 2 * NXH + 2 * NYH; c += ANT) {
      int lx, ly, fs;
      real* dst;
      if (c < NC) {
        lx = c % ABX; ly = c / ABX; dst = &S.core[0][ly][lx]; fs = ABY * ABX;
      } else if (c < NC + 2 * NXH) {
        const int e = c - NC, side = e / NXH, r = e - side * NXH;
        ly = r / AXH;
        const int cl = r - ly * AXH;
        lx = side == 0 ? cl - AXH : ABX + cl;
        dst = side == 0 ? &S.xl[0][ly][cl] : &S.xr[0][ly][cl];
        fs = ABY * AXH;
      } else {
        const int e = c - NC - 2 * NXH, side = e / NYH, r = e - side * NYH;
        const int row = r / ABX;
        lx = r - row * ABX;
        ly = side == 0 ? row - AYH : ABY + row;
        dst = side == 0 ? &S.yt[0][row][lx] : &S.yb[0][row][lx];
        fs = AYH * ABX;
      }
      const int gxc = ((x0 + lx) % nx + nx) % nx, gyc = ((y0 + ly) % ny + ny) % ny;
      const real* g = p.U + zoff + (long long)gyc * nx + gxc;
#pragma unroll
      for (int f = 0; f < 5; ++f) cp_async_elem(dst + f * fs, g + f * n3);
    }
    cp_async_commit();
  };
  auto wait_staged = [&](int j) {   // the j-th staged plane of this CTA (0-based)
    if (via_tma) {
      if (!tc::mbar_wait(&S.bar, (uint32_t)j & 1u, ADJ_WAIT_ITERS)) s_abort = 1;
    } else {
      cp_async_wait<0>();
    }
  };

  // ---- fixed per-thread tasks -------------------------------------------------------------
  constexpr int RFS = WX * WY;                    // ring field stride
  const int ring_own = (ty + 3) * WX + tx + 3;
  // conversion tail: rows 3..10 x columns {0,1,2,35,36,37} (48), rows 0..2 and 11..13 x
  // columns 3..34 (192)
  // (packed to keep the march's live registers few: source offset from S.core and its field
  // stride, ring offset)
  int cv_src = -1, cv_ring_fs = 0;
  if (tid < 240) {
    const real* base = &S.core[0][0][0];
    const int e = tid;
    const real* src;
    int ring, fs;
    if (e < 48) {
      const int ly = e % ABY, c = e / ABY;          // c 0..5: sx = 0,1,2,35,36,37
      if (c < 3) { src = &S.xl[0][ly][1 + c]; ring = (ly + 3) * WX + c; }
      else { src = &S.xr[0][ly][c - 3]; ring = (ly + 3) * WX + ABX + 3 + (c - 3); }
      fs = ABY * AXH;
    } else {
      const int r = (e - 48) / ABX, lx = (e - 48) % ABX;   // r 0..5: sy = 0,1,2,11,12,13
      if (r < 3) { src = &S.yt[0][r][lx]; ring = r * WX + lx + 3; }
      else { src = &S.yb[0][r - 3][lx]; ring = (ABY + 3 + (r - 3)) * WX + lx + 3; }
      fs = AYH * ABX;
    }
    cv_src = (int)(src - base);
    cv_ring_fs = ring | (fs << 16);
  }
  // slope tail (threads 96..255): x slopes of cells -2, -1, ABX, ABX + 1 in each row (32),
  // y slopes of cells -2, -1, ABY, ABY + 1 in each column (128)
  // (packed: ring offset | item << 10 | y axis << 20; -1 none)
  int sl_pack = -1;
  if (tid >= 96) {
    const int e = tid - 96;
    if (e < 32) {
      const int ly = e % ABY, c = e / ABY;
      const int lx = c < 2 ? c - 2 : ABX + (c - 2);
      sl_pack = ((ly + 3) * WX + lx + 3) | ((ly * NSXA + lx + 2) << 10);
    } else {
      const int r = (e - 32) / ABX, lx = (e - 32) % ABX;
      const int ly = r < 2 ? r - 2 : ABY + (r - 2);
      sl_pack = ((ly + 3) * WX + lx + 3) | ((NSXP + (ly + 2) * ABX + lx) << 10) | (1 << 20);
    }
  }
  // face tail (threads 136..255): x faces q = 0, 33, 34 of each row (24), y faces q = 0, 9, 10
  // of each column (96)
  // (packed: q | l << 8 | y axis << 16; -1 none)
  int fc_pack = -1;
  if (tid >= 136) {
    const int e = tid - 136;
    if (e < 24) {
      const int c = e / ABY;
      fc_pack = (c == 0 ? 0 : ABX + c) | ((e % ABY) << 8);
    } else {
      const int c = (e - 24) / ABX;
      fc_pack = (c == 0 ? 0 : ABY + c) | (((e - 24) % ABX) << 8) | (1 << 16);
    }
  }
  // slope-term tail (threads 0..79): x terms of cells -1 and ABX in each row (16), y terms of
  // cells -1 and ABY in each column (64)
  // (packed: r | l << 8 | y axis << 16; -1 none)
  int tm_pack = -1;
  if (tid < 80) {
    if (tid < 16) tm_pack = ((tid / ABY) == 0 ? 0 : ABX + 1) | ((tid % ABY) << 8);
    else tm_pack = (((tid - 16) / ABX) == 0 ? 0 : ABY + 1) | (((tid - 16) % ABX) << 8) | (1 << 16);
  }
  // lam_out copy tail (threads 96..255): mu rows 2..9 x columns {0,1,34,35} (32), rows
  // {0,1,10,11} x columns 2..33 (128); in-plane source offset and mu offset
  int mu_goff = -1, mu_soff = 0;   // in-plane offsets (planes below 2^31 cells)
  if (tid >= 96) {
    const int e = tid - 96;
    int my, mx;
    if (e < 32) { my = 2 + e % ABY; const int c = e / ABY; mx = c < 2 ? c : ABX + c; }
    else { const int r = (e - 32) / ABX; mx = 2 + (e - 32) % ABX; my = r < 2 ? r : ABY + r; }
    mu_soff = my * MXH + mx;
    mu_goff = S.ys[my + 1] * nx + S.xs[mx + 1];
  }
  const int mu_gown = S.ys[ty + 3] * nx + S.xs[tx + 3];
  const int mu_sown = (ty + 2) * MXH + tx + 2;

  // (returns the own cell's primitives, which the z pipeline uses as well)
  auto convert_plane = [&](int slot) {
    const real* c0 = &S.core[0][ty][tx];
    const Prim<real> own = cons_to_prim(c0[0], c0[ABY * ABX], c0[2 * ABY * ABX], c0[3 * ABY * ABX],
                                        c0[4 * ABY * ABX], gm1);
    {
      real* d = &S.w[slot][0][0][0] + ring_own;
      d[0] = own.r; d[RFS] = own.vx; d[2 * RFS] = own.vy; d[3 * RFS] = own.vz; d[4 * RFS] = own.p;
    }
    if (cv_src >= 0) {
      const real* src = &S.core[0][0][0] + cv_src;
      const int fs = cv_ring_fs >> 16;
      const Prim<real> w = cons_to_prim(src[0], src[fs], src[2 * fs], src[3 * fs], src[4 * fs], gm1);
      real* d = &S.w[slot][0][0][0] + (cv_ring_fs & 0xffff);
      d[0] = w.r; d[RFS] = w.vx; d[2 * RFS] = w.vy; d[3 * RFS] = w.vz; d[4 * RFS] = w.p;
    }
    return own;
  };
  // cp.async of lam_out of plane k (x/y halo 2) into mu (one commit group)
  auto load_mu = [&](int k) {
    const long long zoff = (long long)wrap(k, nz) * plane;
#pragma unroll
    for (int f = 0; f < 5; ++f)
      cp_async_elem(&S.mu[f][0][0] + mu_sown, p.lam_out + f * n3 + zoff + mu_gown);
    if (mu_goff >= 0) {
#pragma unroll
      for (int f = 0; f < 5; ++f)
        cp_async_elem(&S.mu[f][0][0] + mu_soff, p.lam_out + f * n3 + zoff + mu_goff);
    }
    cp_async_commit();
  };
  // one slope item: the limited slope of the ring cell at `ring` along `step`, its face states
  // into slot `item` of the st arrays, and its all-zero byte
  auto slope_item = [&](int slot, int ring, int step, int item) {
    const Prim<real> w0 = ring_prim_at(S, slot, ring);
    const Prim<real> d = limited_slope<LIM>(ring_prim_at(S, slot, ring - step), w0,
                                            ring_prim_at(S, slot, ring + step));
    const Prim<real> lo = add_half(w0, d, real(-1)), hi = add_half(w0, d, real(1));
    S.u.st[0][item] = lo.r; S.u.st[1][item] = lo.vx; S.u.st[2][item] = lo.vy; S.u.st[3][item] = lo.vz;
    S.u.st[4][item] = lo.p;
    S.u.st[5][item] = hi.r; S.u.st[6][item] = hi.vx; S.u.st[7][item] = hi.vy; S.u.st[8][item] = hi.vz;
    S.u.st[9][item] = hi.p;
    S.zero[item] = slope_is_zero(d) ? 1 : 0;
  };
  // x face q of row ly (between cells lx = q - 2 and q - 1) or y face q of column lx
  auto face_item = [&](bool yaxis, int q, int l) {
    real g[5], gL[5], gR[5];
    if (!yaxis) {
      const int ly = l;
#pragma unroll
      for (int c = 0; c < 5; ++c) g[c] = (S.mu[c][ly + 2][q + 1] - S.mu[c][ly + 2][q]) * gfx;
      const int i = ly * NSXA + q;
      face_vjp(0, st_prim(S, 5, i), st_prim(S, 0, i + 1), g, gamma, gm1, gL, gR);
      const int f = ly * NFXA + q;
#pragma unroll
      for (int c = 0; c < 5; ++c) { S.face[c][f] = gL[c]; S.face[5 + c][f] = gR[c]; }
    } else {
      const int lx = l;
#pragma unroll
      for (int c = 0; c < 5; ++c) g[c] = (S.mu[c][q + 1][lx + 2] - S.mu[c][q][lx + 2]) * gfy;
      const int i = NSXP + q * ABX + lx;
      face_vjp(1, st_prim(S, 5, i), st_prim(S, 0, i + ABX), g, gamma, gm1, gL, gR);
      const int f = NFXP + q * ABX + lx;
#pragma unroll
      for (int c = 0; c < 5; ++c) { S.face[c][f] = gL[c]; S.face[5 + c][f] = gR[c]; }
    }
  };
  // slope terms (A, B) of cell lx = r - 1 in row ly (x) or ly = r - 1 in column lx (y)
  auto term_item = [&](int slot, bool yaxis, int r, int l) {
    real D[5], A[5], B[5];
    int e;
    if (!yaxis) {
      const int ly = l, sy = ly + 3;
#pragma unroll
      for (int c = 0; c < 5; ++c)
        D[c] = real(0.5) * S.face[c][ly * NFXA + r + 1] - real(0.5) * S.face[5 + c][ly * NFXA + r];
      slope_vjp<LIM>(ring_prim(S, slot, sy, r + 1), ring_prim(S, slot, sy, r + 2),
                     ring_prim(S, slot, sy, r + 3), zero_bit(S, ly * NSXA + r + 1), D, A, B);
      e = ly * NCXA + r;
    } else {
      const int lx = l, sx = lx + 3;
#pragma unroll
      for (int c = 0; c < 5; ++c)
        D[c] = real(0.5) * S.face[c][NFXP + (r + 1) * ABX + lx] -
               real(0.5) * S.face[5 + c][NFXP + r * ABX + lx];
      slope_vjp<LIM>(ring_prim(S, slot, r + 1, sx), ring_prim(S, slot, r + 2, sx),
                     ring_prim(S, slot, r + 3, sx), zero_bit(S, NSXP + (r + 1) * ABX + lx), D, A, B);
      e = NCXP + r * ABX + lx;
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) { S.u.cell[c][e] = A[c]; S.u.cell[5 + c][e] = B[c]; }
  };

  // ---- prologue: ring planes z0..z0+2, own-column history below z0 -------------------------
  load_w(z0, 0);
  load_w(z0 + 1, 1);
  load_w(z0 + 2, 2);
  const Prim<real> wm3 = gload_prim(p.U, n3, (long long)wrap(z0 - 3, nz) * plane + col, gm1);
  const Prim<real> wm2 = gload_prim(p.U, n3, (long long)wrap(z0 - 2, nz) * plane + col, gm1);
  const Prim<real> wm1 = gload_prim(p.U, n3, (long long)wrap(z0 - 1, nz) * plane + col, gm1);
  real mum2[5], mum1[5], mu0[5], mun[5];
  gload5(p.lam_out, n3, (long long)wrap(z0 - 2, nz) * plane + col, mum2);
  gload5(p.lam_out, n3, (long long)wrap(z0 - 1, nz) * plane + col, mum1);
  gload5(p.lam_out, n3, (long long)wrap(z0, nz) * plane + col, mu0);
  gload5(p.lam_out, n3, (long long)wrap(z0 + 1, nz) * plane + col, mun);
  __syncthreads();

  // z pipeline of the own column at the top of iteration k: the limited slope dz1 of cell k+1,
  // the face gradients gLn, gRn of face k+1/2 and gRc of face k-1/2, and the slope terms
  // A_{k-1}, A_k, B_k.
  real gLn[5], gRc[5], gRn[5], Ap[5], Ac[5], Bc[5];
  Prim<real> dz1;
  {
    const Prim<real> w0 = ring_prim(S, 0, ty + 3, tx + 3);
    const Prim<real> w1 = ring_prim(S, 1, ty + 3, tx + 3);
    const Prim<real> w2 = ring_prim(S, 2, ty + 3, tx + 3);
    const Prim<real> dm2 = limited_slope<LIM>(wm3, wm2, wm1);
    const Prim<real> dm1 = limited_slope<LIM>(wm2, wm1, w0);
    const Prim<real> d0 = limited_slope<LIM>(wm1, w0, w1);
    dz1 = limited_slope<LIM>(w0, w1, w2);
    real g[5], gLa[5], gRa[5], gLb[5], gRb[5], D[5], Bt[5];
    // face z0-3/2
    for (int c = 0; c < 5; ++c) g[c] = (mum1[c] - mum2[c]) * gfz;
    face_vjp(2, add_half(wm2, dm2, real(1)), add_half(wm1, dm1, real(-1)), g, gamma, gm1, gLa, gRa);
    // face z0-1/2
    for (int c = 0; c < 5; ++c) g[c] = (mu0[c] - mum1[c]) * gfz;
    face_vjp(2, add_half(wm1, dm1, real(1)), add_half(w0, d0, real(-1)), g, gamma, gm1, gLb, gRb);
    // A_{z0-1} from D = gL(z0-1/2)/2 - gR(z0-3/2)/2
    for (int c = 0; c < 5; ++c) D[c] = real(0.5) * gLb[c] - real(0.5) * gRa[c];
    slope_vjp<LIM>(wm2, wm1, w0, slope_is_zero(dm1), D, Ap, Bt);
    // face z0+1/2
    for (int c = 0; c < 5; ++c) g[c] = (mun[c] - mu0[c]) * gfz;
    face_vjp(2, add_half(w0, d0, real(1)), add_half(w1, dz1, real(-1)), g, gamma, gm1, gLn, gRn);
    for (int c = 0; c < 5; ++c) D[c] = real(0.5) * gLn[c] - real(0.5) * gRb[c];
    slope_vjp<LIM>(wm1, w0, w1, slope_is_zero(d0), D, Ac, Bc);
    for (int c = 0; c < 5; ++c) gRc[c] = gRb[c];
  }
  stage_plane(z0 + 3);

  for (int k = z0; k < z1; ++k) {
    const int s0 = (k - z0) & 3, s1 = (k - z0 + 1) & 3, s2 = (k - z0 + 2) & 3, s3 = (k - z0 + 3) & 3;
    wait_staged(k - z0);
    __syncthreads();  // ---- plane k+3 staged; the gather of plane k-1 is done
    if (s_abort) break;

    load_mu(k);
    real mun2[5];
    gload5(p.lam_out, n3, (long long)wrap(k + 2, nz) * plane + col, mun2);

    // ---- limited slopes and face states of plane k along x and y: own cell, then the tail ----
    // (one call site: every item, own or tail, runs the same instructions, so a cell's result
    // does not depend on where it falls in its tile)
#pragma unroll 1
    for (int it = 0; it < (sl_pack >= 0 ? 3 : 2); ++it) {
      const int ring = it < 2 ? ring_own : sl_pack & 0x3ff;
      const int step = it == 0 ? 1 : (it == 1 ? WX : ((sl_pack >> 20) ? WX : 1));
      const int item = it == 0 ? ty * NSXA + tx + 2
                               : (it == 1 ? NSXP + (ty + 2) * ABX + tx : (sl_pack >> 10) & 0x3ff);
      slope_item(s0, ring, step, item);
    }
    const Prim<real> w3 = convert_plane(s3);   // own cell of plane k+3

    real gW[5];
    Prim<real> wk;   // own cell of plane k, kept for the primitive-recovery step
    // ---- z: slope of k+2, face k+3/2, slope terms of k+1, gather for k ------------------------
    {
      wk = ring_prim(S, s0, ty + 3, tx + 3);
      const Prim<real> w1 = ring_prim(S, s1, ty + 3, tx + 3);
      const Prim<real> w2 = ring_prim(S, s2, ty + 3, tx + 3);
      const Prim<real> dz2 = limited_slope<LIM>(w1, w2, w3);
      real g[5], gL2[5], gR2[5], D[5], An[5], Bn[5];
      for (int c = 0; c < 5; ++c) g[c] = (mun2[c] - mun[c]) * gfz;
      face_vjp(2, add_half(w1, dz1, real(1)), add_half(w2, dz2, real(-1)), g, gamma, gm1, gL2, gR2);
      for (int c = 0; c < 5; ++c) D[c] = real(0.5) * gL2[c] - real(0.5) * gRn[c];
      slope_vjp<LIM>(wk, w1, w2, slope_is_zero(dz1), D, An, Bn);
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        gW[c] = (gLn[c] + gRc[c]) + Ap[c] - Ac[c] + Bc[c] - Bn[c];
        gRc[c] = gRn[c];
        gLn[c] = gL2[c];
        gRn[c] = gR2[c];
        Ap[c] = Ac[c];
        Ac[c] = An[c];
        Bc[c] = Bn[c];
        mun[c] = mun2[c];
      }
      dz1 = dz2;
    }
    cp_async_wait<0>();
    __syncthreads();  // ---- face states, mu of plane k and ring slot of plane k+3 ready

    if (k + 1 < z1) stage_plane(k + 4);
    // ---- x and y face VJPs of plane k: own faces, then the tail ------------------------------
#pragma unroll 1
    for (int it = 0; it < (fc_pack >= 0 ? 3 : 2); ++it) {
      const int pk = it == 0 ? (tx + 1) | (ty << 8) : (it == 1 ? (ty + 1) | (tx << 8) | (1 << 16) : fc_pack);
      face_item((pk >> 16) != 0, pk & 0xff, (pk >> 8) & 0xff);
    }
    __syncthreads();  // ---- face gradients ready; the face states are dead from here

    // ---- slope terms (A, B) of the x and y slopes; they overwrite the face states --------------
#pragma unroll 1
    for (int it = 0; it < (tm_pack >= 0 ? 3 : 2); ++it) {
      const int pk = it == 0 ? (tx + 1) | (ty << 8) : (it == 1 ? (ty + 1) | (tx << 8) | (1 << 16) : tm_pack);
      term_item(s0, (pk >> 16) != 0, pk & 0xff, (pk >> 8) & 0xff);
    }
    __syncthreads();  // ---- slope terms ready
    {
      const int fb = ty * NFXA, cb = ty * NCXA;
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        gW[c] += (S.face[c][fb + tx + 2] + S.face[5 + c][fb + tx + 1]) + S.u.cell[c][cb + tx] -
                 S.u.cell[c][cb + tx + 1] + S.u.cell[5 + c][cb + tx + 1] - S.u.cell[5 + c][cb + tx + 2];
        gW[c] += (S.face[c][NFXP + (ty + 2) * ABX + tx] + S.face[5 + c][NFXP + (ty + 1) * ABX + tx]) +
                 S.u.cell[c][NCXP + ty * ABX + tx] - S.u.cell[c][NCXP + (ty + 1) * ABX + tx] +
                 S.u.cell[5 + c][NCXP + (ty + 1) * ABX + tx] - S.u.cell[5 + c][NCXP + (ty + 2) * ABX + tx];
      }
    }

    // ---- primitive recovery transposed, stage combination, store ------------------------------
    // (from registers only: the next plane's loads may already overwrite the ring slot of k)
    if (active) {
      const Prim<real> w = wk;
      const real ir = q_div(real(1), w.r);
      const real v2 = w.vx * w.vx + w.vy * w.vy + w.vz * w.vz;
      real gU[5];
      gU[0] = gW[0] - (gW[1] * w.vx + gW[2] * w.vy + gW[3] * w.vz) * ir + gW[4] * gm1 * real(0.5) * v2;
      gU[1] = gW[1] * ir - gW[4] * gm1 * w.vx;
      gU[2] = gW[2] * ir - gW[4] * gm1 * w.vy;
      gU[3] = gW[3] * ir - gW[4] * gm1 * w.vz;
      gU[4] = gW[4] * gm1;
      const long long idx = (long long)k * plane + col;
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        real v = p.c1 * S.mu[c][ty + 2][tx + 2] + gU[c];
        if (p.extra) v += p.c2 * __ldg(p.extra + c * n3 + idx);
        if (p.extra2) v += p.c3 * __ldg(p.extra2 + c * n3 + idx);
        p.lam_in[c * n3 + idx] = v;
      }
    }
  }
  if (s_abort && tid == 0) atomicOr(p.flags, FLAG_TIMEOUT);   // a staging wait gave up
}

template <typename real>
cudaError_t launch_stage_adjoint(const AdjointArgs<real>& a, cudaStream_t s) {
  const size_t smem = sizeof(AdjSmem<real>);
  auto run = [&](auto kernel, int& resident) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (resident <= 0) {
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, kernel, ANT, smem);
      if (e != cudaSuccess) return e;
      if (resident <= 0) resident = 1;
    }
    const long long tiles = (long long)((a.nx + ABX - 1) / ABX) * ((a.ny + ABY - 1) / ABY);
    const int zc = wave_zchunk(tiles, a.nz, resident, 1.0);
    dim3 grid((a.nx + ABX - 1) / ABX, (a.ny + ABY - 1) / ABY, (a.nz + zc - 1) / zc);
    StageTma maps;
    memset(&maps, 0, sizeof(maps));
    const bool tma_ok = a.nx % ABX == 0 && a.ny % ABY == 0 && a.nx >= AXH && a.ny >= AYH &&
                        ((unsigned long long)a.U & 15ull) == 0 &&
                        stage_tma_maps(a.U, a.nx, a.ny, a.nz, (int)sizeof(real), ABX, ABY, AXH, AYH, &maps);
    kernel<<<grid, ANT, smem, s>>>(a, zc, maps, tma_ok ? 1 : 0);
    return cudaGetLastError();
  };
  static int res_vl = 0, res_mc = 0;   // CTAs per SM of each instance
  return a.limiter == LIM_VL ? run(stage_adjoint_kernel<real, LIM_VL>, res_vl)
                             : run(stage_adjoint_kernel<real, LIM_MC>, res_mc);
}
template cudaError_t launch_stage_adjoint<float>(const AdjointArgs<float>&, cudaStream_t);
template cudaError_t launch_stage_adjoint<double>(const AdjointArgs<double>&, cudaStream_t);

// Pointwise adjoint of the sources of one step (Sec. 3.1.1 kick, then Sec. 4.3 cooling): the
// forward is recomputed from UH (kick with the step's field a(x), then the cooling tangents), and
//   cooling^T:  lam_rho += lam_E (cR - (1 - cE) K / rho),  lam_m += lam_E (1 - cE) v,
//               lam_E *= cE    (K = |m|^2 / (2 rho), v = m / rho of the kicked state),
//   kick^T:     lam_rho += dt a . lam_m,  lam_m += dt a lam_E.
template <typename real>
__global__ void source_adjoint_kernel(const SourceAdjArgs<real> p) {
  const long long n3 = (long long)p.nx * p.ny * p.nz;
  const real dt = (real)*p.dtp;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n3;
       q += (long long)gridDim.x * blockDim.x) {
    const unsigned t1 = (unsigned)q / (unsigned)p.nx;
    const int i = (int)((unsigned)q - t1 * (unsigned)p.nx);
    const int j = (int)(t1 % (unsigned)p.ny), k = (int)(t1 / (unsigned)p.ny);
    real u[5], l[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      u[c] = p.UH[c * n3 + q];
      l[c] = p.lam[c * n3 + q];
    }
    real a[3] = {real(0), real(0), real(0)};
    if (p.tab) {
      forcing_accel(p.tab, p.tw, i, j, k, a);
      // the kick as the forward applies it (momentum before the kick in the energy)
      const real e = (u[1] * a[0] + u[2] * a[1] + u[3] * a[2]) * dt;
      u[1] = u[1] + u[0] * a[0] * dt;
      u[2] = u[2] + u[0] * a[1] * dt;
      u[3] = u[3] + u[0] * a[2] * dt;
      u[4] = u[4] + e;
    }
    real gv[3] = {real(0), real(0), real(0)}, mF[3] = {u[1], u[2], u[3]};
    if (p.phi) {
      // g = -grad phi (central differences) and the gravity kick, as gravity_sources_kernel
      potential_gradient(p.phi, p.nx, p.ny, p.nz, i, j, k, (real)p.i2h, gv[0], gv[1], gv[2]);
      const real e = (u[1] * gv[0] + u[2] * gv[1] + u[3] * gv[2]) * dt;
      u[1] = u[1] + u[0] * gv[0] * dt;
      u[2] = u[2] + u[0] * gv[1] * dt;
      u[3] = u[3] + u[0] * gv[2] * dt;
      u[4] = u[4] + e;
    }
    if (p.cooling) {
      real cR, cE;
      cooling_tangents(u[0], u[1], u[2], u[3], u[4], dt, p.gm1, p.t_floor, p.cool_frac,
                       p.nsub_max, cR, cE);
      const real ir = q_div(real(1), u[0]);
      const real v0 = u[1] * ir, v1 = u[2] * ir, v2 = u[3] * ir;
      const real K = real(0.5) * (u[1] * v0 + u[2] * v1 + u[3] * v2);
      const real w = (real(1) - cE) * l[4];
      l[0] += l[4] * cR - w * K * ir;
      l[1] += w * v0;
      l[2] += w * v1;
      l[3] += w * v2;
      l[4] *= cE;
    }
    if (p.phi) {
      // gravity kick^T, and dL/dg = dt (rho lam_m + m lam_E) with m before the kick
#pragma unroll
      for (int d = 0; d < 3; ++d)
        p.h[d * n3 + q] = (double)dt * ((double)u[0] * (double)l[1 + d] + (double)mF[d] * (double)l[4]);
      l[0] += dt * (gv[0] * l[1] + gv[1] * l[2] + gv[2] * l[3]);
      l[1] += dt * gv[0] * l[4];
      l[2] += dt * gv[1] * l[4];
      l[3] += dt * gv[2] * l[4];
    }
    if (p.tab) {
      l[0] += dt * (a[0] * l[1] + a[1] * l[2] + a[2] * l[3]);
      l[1] += dt * a[0] * l[4];
      l[2] += dt * a[1] * l[4];
      l[3] += dt * a[2] * l[4];
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) p.lamH[c * n3 + q] = l[c];
  }
}

template <typename real>
cudaError_t launch_source_adjoint(const SourceAdjArgs<real>& a, cudaStream_t s) {
  const long long n3 = (long long)a.nx * a.ny * a.nz;
  long long blocks = (n3 + 255) / 256;
  if (blocks > 148 * 8) blocks = 148 * 8;
  source_adjoint_kernel<real><<<(int)blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}
template cudaError_t launch_source_adjoint<float>(const SourceAdjArgs<float>&, cudaStream_t);
template cudaError_t launch_source_adjoint<double>(const SourceAdjArgs<double>&, cudaStream_t);

// psi = dL/dphi = sum_a (h_a(i + e_a) - h_a(i - e_a)) / (2 dx): the transpose of g = -grad phi.
__global__ void gravity_psi_kernel(const double* __restrict__ h, int nx, int ny, int nz, double i2h,
                                   double* __restrict__ psi) {
  const long long n3 = (long long)nx * ny * nz;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n3;
       q += (long long)gridDim.x * blockDim.x) {
    const unsigned t1 = (unsigned)q / (unsigned)nx;
    const int i = (int)((unsigned)q - t1 * (unsigned)nx);
    const int j = (int)(t1 % (unsigned)ny), k = (int)(t1 / (unsigned)ny);
    const long long row = (long long)k * ny;
    const double hx = h[(row + j) * nx + wrap(i + 1, nx)] - h[(row + j) * nx + wrap(i - 1, nx)];
    const double hy = h[n3 + (row + wrap(j + 1, ny)) * nx + i] - h[n3 + (row + wrap(j - 1, ny)) * nx + i];
    const double hz = h[2 * n3 + ((long long)wrap(k + 1, nz) * ny + j) * nx + i] -
                      h[2 * n3 + ((long long)wrap(k - 1, nz) * ny + j) * nx + i];
    psi[q] = (hx + hy + hz) * i2h;
  }
}

// lam_rho += 4 pi G w: the density's share through the Poisson source F = 4 pi G (rho - <rho>)
// (w = dL/dF has zero mean, so the mean subtraction adds nothing).
// w is float-float (planar).
template <typename real>
__global__ void add_density_adjoint_kernel(real* __restrict__ lam, const float* __restrict__ w,
                                           long long n3, real four_pi_G) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n3;
       q += (long long)gridDim.x * blockDim.x)
    lam[q] = lam[q] + four_pi_G * ((real)w[q] + (real)w[n3 + q]);
}

}  // namespace dh

// =============================================================================================
// Checkpointed driver.
struct AdjointSpace {
  std::vector<void*> ckpt;   // U at steps 0, k, 2k, ...
  std::vector<void*> seg;    // segment inputs U^{m0+1..m0+k-1}
  std::vector<void*> seg1;   // segment stage-1 outputs U1^{m0..m0+k-1}
  std::vector<void*> seg2;   // SSPRK3: segment stage-2 outputs U2^{m0..m0+k-1}
  std::vector<void*> segH;   // segment stage-2 states before the sources (forcing / cooling on)
  void* scratch = nullptr;   // replayed output nobody reads
  // lambda of: the step output, the step input, U1, the pre-source state, U2 (SSPRK3)
  void* lam[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  double* dts = nullptr;
  void* tabs = nullptr;      // normalised OU table of every step (96 reals each)
  // gravity: the potential at every checkpoint (warm start of the replay), of every segment
  // step, dL/dg, dL/dphi, dL/dF, and the forward's final potential
  std::vector<float*> ckPhi, segPhi;   // float-float potentials, 8 B per cell
  double *hbuf = nullptr, *psi = nullptr;
  float *wsol = nullptr, *phi_keep = nullptr;   // float-float, planar
  int nck = 0, k = 0, nsteps = 0;
  bool sources = false, gravity = false, rk3 = false;
};

namespace dh {
void adjoint_free(dh_ctx* c) {
  if (!c->adj) return;
  AdjointSpace* a = c->adj;
  for (void* p : a->ckpt) cudaFree(p);
  for (void* p : a->seg) cudaFree(p);
  for (void* p : a->seg1) cudaFree(p);
  for (void* p : a->seg2) cudaFree(p);
  for (void* p : a->segH) cudaFree(p);
  for (void* p : a->lam) cudaFree(p);
  cudaFree(a->scratch);
  cudaFree(a->dts);
  cudaFree(a->tabs);
  for (float* p : a->ckPhi) cudaFree(p);
  for (float* p : a->segPhi) cudaFree(p);
  cudaFree(a->hbuf);
  cudaFree(a->psi);
  cudaFree(a->wsol);
  cudaFree(a->phi_keep);
  delete a;
  c->adj = nullptr;
}
}  // namespace dh

using namespace dh;

static cudaError_t adjoint_reserve(dh_ctx* c, int n, int k) {
  const int nck = (n + k - 1) / k;
  const bool gravity = c->cfg.gravity;
  const bool sources = c->cfg.forcing || c->cfg.cooling || gravity;
  const bool rk3 = c->cfg.integrator == 3;
  AdjointSpace* a = c->adj;
  if (a && a->nck >= nck && a->k == k && a->nsteps >= n && a->sources == sources &&
      a->gravity == gravity && a->rk3 == rk3)
    return cudaSuccess;
  adjoint_free(c);
  a = new AdjointSpace();
  c->adj = a;
  a->nck = nck;
  a->k = k;
  a->nsteps = n;
  a->sources = sources;
  a->gravity = gravity;
  a->rk3 = rk3;
  cudaError_t e = cudaSuccess;
  if (gravity) {
    const size_t pb = (size_t)c->n3 * sizeof(double);
    a->ckPhi.assign(nck, nullptr);
    a->segPhi.assign(k, nullptr);
    for (auto& p : a->ckPhi) if (e == cudaSuccess) e = cudaMalloc((void**)&p, pb);
    for (auto& p : a->segPhi) if (e == cudaSuccess) e = cudaMalloc((void**)&p, pb);
    if (e == cudaSuccess) e = cudaMalloc((void**)&a->hbuf, 3 * pb);
    if (e == cudaSuccess) e = cudaMalloc((void**)&a->psi, pb);
    if (e == cudaSuccess) e = cudaMalloc((void**)&a->wsol, pb);
    if (e == cudaSuccess) e = cudaMalloc((void**)&a->phi_keep, pb);
  }
  a->ckpt.assign(nck, nullptr);
  a->seg.assign(k > 1 ? k - 1 : 0, nullptr);
  a->seg1.assign(k, nullptr);
  a->seg2.assign(rk3 ? k : 0, nullptr);
  a->segH.assign(sources ? k : 0, nullptr);
  for (auto& p : a->ckpt) if (e == cudaSuccess) e = cudaMalloc(&p, c->state_bytes);
  for (auto& p : a->seg) if (e == cudaSuccess) e = cudaMalloc(&p, c->state_bytes);
  for (auto& p : a->seg1) if (e == cudaSuccess) e = cudaMalloc(&p, c->state_bytes);
  for (auto& p : a->seg2) if (e == cudaSuccess) e = cudaMalloc(&p, c->state_bytes);
  for (auto& p : a->segH) if (e == cudaSuccess) e = cudaMalloc(&p, c->state_bytes);
  for (int q = 0; q < (rk3 ? 5 : 4); ++q)
    if (e == cudaSuccess) e = cudaMalloc(&a->lam[q], c->state_bytes);
  if (e == cudaSuccess && sources) e = cudaMalloc(&a->scratch, c->state_bytes);
  if (e == cudaSuccess && sources)
    e = cudaMalloc(&a->tabs, (size_t)(n > 0 ? n : 1) * 96 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&a->dts, (size_t)(n > 0 ? n : 1) * sizeof(double));
  if (e != cudaSuccess) adjoint_free(c);
  return e;
}

// Re-runs one stage as the forward ran it: stage 1, or a combination stage
// out = w0 U0 + w1 (U + dt L(U)), the step's final one (final) or SSPRK3's middle one.  The final
// stage with sources applies the step's forcing table `tab` and cooling exactly as the fused
// forward kernel did, and stores the state before the sources into pre_src.
template <typename real>
static cudaError_t replay_stage(dh_ctx* c, int stage, const void* U, const void* U0, void* out,
                                const double* dtp, real w0, real w1, bool final,
                                const void* tab = nullptr, void* pre_src = nullptr) {
  const dh_config& g = c->cfg;
  StageArgs<real> a;
  memset(&a, 0, sizeof(a));
  a.U = (const real*)U; a.U0 = (const real*)U0; a.out = (real*)out;
  a.nx = g.nx; a.ny = g.ny; a.nz = g.nz;
  a.gamma = (real)g.gamma; a.gm1 = (real)(g.gamma - 1.0);
  a.idx = (real)(1.0 / g.dx); a.idy = (real)(1.0 / g.dy); a.idz = (real)(1.0 / g.dz);
  a.dx = (real)g.dx; a.dy = (real)g.dy; a.dz = (real)g.dz;
  a.rec = c->rec; a.dtp = dtp;
  a.limiter = g.limiter;
  a.w0 = w0; a.w1 = w1;
  a.final_stage = final ? 1 : 0;
  if (stage == 2 && final && pre_src) {
    a.pre_src = (real*)pre_src;
    a.forcing = g.forcing && tab;
    a.ahat_norm = (const real*)tab;
    for (int q = 0; q < 3; ++q) a.tw[q] = (const real*)c->tw[q];
    a.frow = (real*)c->frow;
    a.cooling = g.cooling;
    a.t_floor = (real)g.t_floor; a.cool_frac = (real)g.cool_frac; a.nsub_max = g.nsub_max;
  }
  prof_begin(c, stage == 2 && final ? DH_KERNEL_STAGE2 : DH_KERNEL_STAGE1);
  // RK2's final stage is kernel stage 2; SSPRK3's weighted stages are kernel stage 3
  const bool rk2_final = stage == 2 && final && w0 == real(0.5) && w1 == real(0.5);
  int nl = 1;
  cudaError_t e = launch_stage<real>(stage == 1 ? 1 : (rk2_final ? 2 : 3), a, c->stream, &nl);
  prof_end(c, nl);
  return e;
}

template <typename real>
static cudaError_t adjoint_stage(dh_ctx* c, const void* U, const void* lam_out, const void* extra,
                                 void* lam_in, real c1, real c2, real beta, const double* dtp,
                                 const void* extra2 = nullptr, real c3 = real(0)) {
  const dh_config& g = c->cfg;
  AdjointArgs<real> a;
  a.U = (const real*)U; a.lam_out = (const real*)lam_out; a.extra = (const real*)extra;
  a.lam_in = (real*)lam_in;
  a.nx = g.nx; a.ny = g.ny; a.nz = g.nz;
  a.gamma = (real)g.gamma; a.gm1 = (real)(g.gamma - 1.0);
  a.idx = (real)(1.0 / g.dx); a.idy = (real)(1.0 / g.dy); a.idz = (real)(1.0 / g.dz);
  a.c1 = c1; a.c2 = c2; a.beta = beta; a.dtp = dtp;
  a.extra2 = (const real*)extra2; a.c3 = c3;
  a.limiter = g.limiter;
  a.flags = &c->rec->flags;
  prof_begin(c, DH_KERNEL_ADJOINT);
  cudaError_t e = launch_stage_adjoint<real>(a, c->stream);
  prof_end(c, 1);
  return e;
}

template <typename real>
static cudaError_t adjoint_backward(dh_ctx* c, int n, int k, void* lam_final_dev, bool last_kept) {
  AdjointSpace* a = c->adj;
  cudaError_t e;
  void* lam = a->lam[0];
  void* lam_new = a->lam[1];
  void* lam_u1 = a->lam[2];
  e = cudaMemcpyAsync(lam, lam_final_dev, c->state_bytes, cudaMemcpyDeviceToDevice, c->stream);
  if (e != cudaSuccess) return e;
  for (int sgi = (n + k - 1) / k - 1; sgi >= 0; --sgi) {
    const int m0 = sgi * k;
    const int len = (m0 + k <= n ? k : n - m0);
    // recompute the segment: inputs U^{m0+j} and stage-1 outputs U1^{m0+j}
    auto in = [&](int j) -> void* { return j == 0 ? a->ckpt[sgi] : a->seg[j - 1]; };
    const bool src = a->sources;
    auto tab = [&](int m) -> const void* {
      return c->cfg.forcing ? (const void*)((const real*)a->tabs + (size_t)m * 96) : nullptr;
    };
    const size_t pb = (size_t)c->n3 * sizeof(double);
    if (a->gravity) {
      // the potential the forward started this segment from (warm start of its first solve)
      e = cudaMemcpyAsync(mg_phi(c), a->ckPhi[sgi], pb, cudaMemcpyDeviceToDevice, c->stream);
      if (e != cudaSuccess) return e;
    }
    // final-stage weights: RK2 (1/2, 1/2); SSPRK3 (1/3, 2/3) after the middle stage (3/4, 1/4)
    const real fw0 = a->rk3 ? real(1.0 / 3.0) : real(0.5), fw1 = a->rk3 ? real(2.0 / 3.0) : real(0.5);
    // the last segment was kept by the forward sweep
    const bool kept = last_kept && m0 + k >= n;
    for (int j = 0; j < len && !kept; ++j) {
      const double* dtp = a->dts + m0 + j;
      e = replay_stage<real>(c, 1, in(j), nullptr, a->seg1[j], dtp, real(1), real(1), false);
      if (e != cudaSuccess) return e;
      const void* last = a->seg1[j];   // input of the final stage
      if (a->rk3) {
        e = replay_stage<real>(c, 2, a->seg1[j], in(j), a->seg2[j], dtp, real(0.75), real(0.25), false);
        if (e != cudaSuccess) return e;
        last = a->seg2[j];
      }
      if (a->gravity) {
        // the final stage without fused sources, then the Poisson solve and forcing -> gravity
        // -> cooling exactly as the forward step took them
        void* out = j + 1 < len ? in(j + 1) : a->scratch;
        e = replay_stage<real>(c, 2, last, in(j), out, dtp, fw0, fw1, true);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(a->segH[j], out, c->state_bytes, cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess) e = gravity_sources<real>(c, out, tab(m0 + j), dtp, false);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(a->segPhi[j], mg_phi(c), pb, cudaMemcpyDeviceToDevice, c->stream);
        if (e != cudaSuccess) return e;
      } else if (src) {
        // with sources the last final stage is replayed too: its pre-source state is needed
        e = replay_stage<real>(c, 2, last, in(j), j + 1 < len ? in(j + 1) : a->scratch, dtp, fw0,
                               fw1, true, tab(m0 + j), a->segH[j]);
        if (e != cudaSuccess) return e;
      } else if (j + 1 < len) {
        e = replay_stage<real>(c, 2, last, in(j), in(j + 1), dtp, fw0, fw1, true);
        if (e != cudaSuccess) return e;
      }
    }
    for (int j = len - 1; j >= 0; --j) {
      const double* dtp = a->dts + m0 + j;
      // sources: U^{n+1} = C(F(U_H)) -> lambda of U_H
      void* lam_h = lam;
      if (src) {
        SourceAdjArgs<real> sa;
        memset(&sa, 0, sizeof(sa));
        sa.lam = (const real*)lam; sa.UH = (const real*)a->segH[j]; sa.lamH = (real*)a->lam[3];
        sa.tab = (const real*)tab(m0 + j);
        for (int q = 0; q < 3; ++q) sa.tw[q] = (const real*)c->tw[q];
        sa.nx = c->cfg.nx; sa.ny = c->cfg.ny; sa.nz = c->cfg.nz;
        sa.cooling = c->cfg.cooling;
        sa.gm1 = (real)(c->cfg.gamma - 1.0); sa.t_floor = (real)c->cfg.t_floor;
        sa.cool_frac = (real)c->cfg.cool_frac; sa.nsub_max = c->cfg.nsub_max;
        sa.dtp = dtp;
        sa.phi = a->gravity ? a->segPhi[j] : nullptr;
        sa.h = a->hbuf;
        sa.i2h = 1.0 / (2.0 * c->cfg.dx);
        e = launch_source_adjoint<real>(sa, c->stream);
        if (e != cudaSuccess) return e;
        lam_h = a->lam[3];
        if (a->gravity) {
          // the potential's share: psi = dL/dphi, A w = psi - <psi>, lam_rho += 4 pi G w
          const long long n3 = c->n3;
          const int blocks = (int)((n3 + 255) / 256 < 148 * 8 ? (n3 + 255) / 256 : 148 * 8);
          gravity_psi_kernel<<<blocks, 256, 0, c->stream>>>(a->hbuf, c->cfg.nx, c->cfg.ny, c->cfg.nz,
                                                            1.0 / (2.0 * c->cfg.dx), a->psi);
          e = cudaGetLastError();
          if (e == cudaSuccess) e = mg_solve_rhs(c, a->psi, a->wsol);
          if (e != cudaSuccess) return e;
          add_density_adjoint_kernel<real><<<blocks, 256, 0, c->stream>>>((real*)lam_h, a->wsol, n3,
                                                                          (real)c->cfg.four_pi_G);
          e = cudaGetLastError();
          if (e != cudaSuccess) return e;
        }
      }
      if (!a->rk3) {
        // stage 2: U_H = U^n/2 + (U1 + dt L(U1))/2
        e = adjoint_stage<real>(c, a->seg1[j], lam_h, nullptr, lam_u1, real(0.5), real(0), real(0.5), dtp);
        if (e != cudaSuccess) return e;
        // stage 1: U1 = U^n + dt L(U^n); lambda^n also receives lambda_H/2 from stage 2
        e = adjoint_stage<real>(c, in(j), lam_u1, lam_h, lam_new, real(1), real(0.5), real(1), dtp);
        if (e != cudaSuccess) return e;
      } else {
        void* lam_u2 = a->lam[4];
        // stage 3: U_H = U^n/3 + 2/3 (U2 + dt L(U2))
        e = adjoint_stage<real>(c, a->seg2[j], lam_h, nullptr, lam_u2, real(2.0 / 3.0), real(0),
                                real(2.0 / 3.0), dtp);
        if (e != cudaSuccess) return e;
        // stage 2: U2 = 3/4 U^n + 1/4 (U1 + dt L(U1))
        e = adjoint_stage<real>(c, a->seg1[j], lam_u2, nullptr, lam_u1, real(0.25), real(0),
                                real(0.25), dtp);
        if (e != cudaSuccess) return e;
        // stage 1: U1 = U^n + dt L(U^n); lambda^n also receives lambda_H/3 and 3/4 lambda_U2
        e = adjoint_stage<real>(c, in(j), lam_u1, lam_h, lam_new, real(1), real(1.0 / 3.0), real(1),
                                dtp, lam_u2, real(0.75));
        if (e != cudaSuccess) return e;
      }
      void* t = lam; lam = lam_new; lam_new = t;
    }
  }
  a->lam[0] = lam;
  a->lam[1] = lam_new;
  return cudaSuccess;
}

extern "C" dh_status dh_adjoint_advance_dt(dh_ctx* c, int n, int k, double dt,
                                           const void* dLdU_final, void* dLdU0, int on_device) {
  if (!c || !dLdU_final || !dLdU0) return DH_ERR_ARG;
  if (!(dt >= 0.0)) { c->err = "dt must be >= 0 (0: the CFL time step)"; return DH_ERR_ARG; }
  if (!c->initialized) { c->err = "state not initialised"; return DH_ERR_STATE; }
  if (c->correct_each_step) {
    c->err = "the adjoint covers the solver step only: turn the per-step corrector off";
    return DH_ERR_STATE;
  }
  if (n < 0 || k < 1) { c->err = "need n_steps >= 0 and ckpt_every >= 1"; return DH_ERR_ARG; }
  const cudaMemcpyKind h2d = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const cudaMemcpyKind d2h = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (n == 0) {
    cudaError_t e = cudaMemcpyAsync(dLdU0, dLdU_final, c->state_bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) { c->err = cudaGetErrorString(e); return DH_ERR_CUDA; }
    return DH_OK;
  }
  if (k > n) k = n;   // one segment: a larger interval would only allocate unused buffers
  cudaError_t e = adjoint_reserve(c, n, k);
  if (e != cudaSuccess) { c->err = std::string("adjoint allocation: ") + cudaGetErrorString(e); return DH_ERR_CUDA; }
  AdjointSpace* a = c->adj;
  // forward sweep with checkpoints; the dt of every step is recorded on the device.  Without
  // gravity the steps of the last segment also keep their inputs and intermediate states (the
  // segment buffers the backward sweep would otherwise fill by replaying them).
  const bool keep_last = !a->gravity;
  const int m_last = (n - 1) / k * k;
  for (int m = 0; m < n && e == cudaSuccess; ++m) {
    if (m % k == 0) {
      e = cudaMemcpyAsync(a->ckpt[m / k], c->U[c->cur], c->state_bytes, cudaMemcpyDeviceToDevice, c->stream);
      if (e == cudaSuccess && a->gravity)
        e = cudaMemcpyAsync(a->ckPhi[m / k], mg_phi(c), (size_t)c->n3 * sizeof(double),
                            cudaMemcpyDeviceToDevice, c->stream);
    }
    StepCapture cap;
    const bool keep = keep_last && m >= m_last;
    if (keep) {
      const int j = m - m_last;
      if (j > 0 && e == cudaSuccess)
        e = cudaMemcpyAsync(a->seg[j - 1], c->U[c->cur], c->state_bytes, cudaMemcpyDeviceToDevice,
                            c->stream);
      cap.u1 = a->seg1[j];
      cap.u2 = a->rk3 ? a->seg2[j] : nullptr;
      cap.pre_src = a->sources ? a->segH[j] : nullptr;
    }
    if (e == cudaSuccess)
      e = c->prec == DH_F64 ? dh_enqueue_step_f64(c, dt, keep ? &cap : nullptr)
                            : dh_enqueue_step_f32(c, dt, keep ? &cap : nullptr);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(a->dts + m, &c->rec->dt, sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess && c->cfg.forcing) {
      const size_t tb = 96 * (c->prec == DH_F64 ? sizeof(double) : sizeof(float));
      e = cudaMemcpyAsync((char*)a->tabs + (size_t)m * tb, c->ahat_norm, tb, cudaMemcpyDeviceToDevice,
                          c->stream);
    }
  }
  if (e != cudaSuccess) { c->err = std::string("adjoint forward: ") + cudaGetErrorString(e); return DH_ERR_CUDA; }
  dh_status st = dh_finish_steps(c);
  if (st != DH_OK) return st;
  const size_t pb = (size_t)c->n3 * sizeof(double);
  if (a->gravity) {
    // keep the forward's final potential (the next step's warm start); start dL/dF at zero
    e = cudaMemcpyAsync(a->phi_keep, mg_phi(c), pb, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(a->wsol, 0, pb, c->stream);
  }
  // backward sweep
  if (e == cudaSuccess) e = cudaMemcpyAsync(a->lam[1], dLdU_final, c->state_bytes, h2d, c->stream);
  if (e == cudaSuccess)
    e = c->prec == DH_F64 ? adjoint_backward<double>(c, n, k, a->lam[1], keep_last)
                          : adjoint_backward<float>(c, n, k, a->lam[1], keep_last);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dLdU0, a->lam[0], c->state_bytes, d2h, c->stream);
  if (e == cudaSuccess && a->gravity)
    e = cudaMemcpyAsync(mg_phi(c), a->phi_keep, pb, cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) { c->err = std::string("adjoint backward: ") + cudaGetErrorString(e); return DH_ERR_CUDA; }
  {
    // a kernel whose bounded wait for its own copies gave up raised the flag in the step record
    StepRecord r;
    e = cudaMemcpy(&r, c->rec, sizeof(r), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) { c->err = cudaGetErrorString(e); return DH_ERR_CUDA; }
    if (r.flags & FLAG_TIMEOUT) {
      r.flags &= ~FLAG_TIMEOUT;
      r.fail_step = -1;
      cudaMemcpy(c->rec, &r, sizeof(r), cudaMemcpyHostToDevice);
      c->err = "adjoint: a kernel's bounded wait for its own copies gave up";
      return DH_ERR_CUDA;
    }
  }
  if (a->gravity) {
    // an adjoint Poisson solve that missed mg_tol raised the flag in the step record
    StepRecord r;
    e = cudaMemcpy(&r, c->rec, sizeof(r), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) { c->err = cudaGetErrorString(e); return DH_ERR_CUDA; }
    if (r.flags & FLAG_MG_NOCONV) {
      r.flags &= ~FLAG_MG_NOCONV;
      r.fail_step = -1;
      cudaMemcpy(c->rec, &r, sizeof(r), cudaMemcpyHostToDevice);
      c->err = "a multigrid solve of the adjoint did not reach mg_tol within mg_max_cycles";
      return DH_ERR_MG_NOCONV;
    }
  }
  return DH_OK;
}

extern "C" dh_status dh_adjoint_advance(dh_ctx* c, int n, int k, const void* dLdU_final,
                                        void* dLdU0, int on_device) {
  return dh_adjoint_advance_dt(c, n, k, 0.0, dLdU_final, dLdU0, on_device);
}
