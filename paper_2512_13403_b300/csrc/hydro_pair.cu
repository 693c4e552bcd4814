// Paired stage kernel: one launch computes a full SSP-RK2 (or SSPRK3) stage (App. A.3) of a
// tile of cells — primitive recovery (Eq. 2), limited MUSCL face states (App. A.1), HLLC fluxes
// (App. A.2), the unsplit divergence and the stage combination, and in the final stage the
// operator-split sources (OU forcing, Sec. 3.1.1; cooling, Sec. 4.3) and the CFL minimum of the
// new state (App. A.4).  It computes what stage_kernel (hydro.cu) computes, on grids whose x
// extent is a multiple of 64 and y extent a multiple of 8.
//
// Pairs: a CTA owns a 64 x 8 column of cells and each of its 256 threads owns two cells of one
// row, 32 apart in x (lane A at x0 + tx, lane B at x0 + 32 + tx).  Every stencil neighbour of
// the two cells is again a pair at the same offset, so the whole update runs on two-lane values
// (dh_pair.cuh): packed FP32x2 arithmetic that needs no register shuffling, the compares and
// selects of the limiter and of HLLC once per lane.
//
// March along z with the update one plane behind: iteration k converts the staged plane k+1 to
// primitives, computes the x and y half slopes of plane k and its x and y face fluxes (shared
// memory), and the z slope of plane k and the z face k - 1/2 of the own column (registers).
// With the z face k - 1/2 known, plane k - 1 is complete: its x/y divergence (from the fluxes
// of iteration k - 1), the z difference and the stage combination are applied and stored.  The
// lag keeps only planes k and k+1 in shared memory.  The conserved variables arrive by TMA (five
// tensor-map boxes: the 64 x 8 core and its four halo strips, periodic wrap in the start
// coordinates) into two staging slots with a barrier each: plane k+3 is requested during
// iteration k, as soon as plane k+1's slot has been converted, so every plane has two
// iterations to land.  The waits are bounded and a timeout fails the step.  Two CTA barriers
// per plane.
#include <math.h>
#include <string.h>

#include <cstring>
#include <type_traits>

#include "tc_ptx.cuh"
#include "tma.cuh"
#include "dh_kernels.h"
#include "dh_pair.cuh"
#include "dh_pair_sources.cuh"
#include "dh_sources.cuh"
#include "../../include/dh.h"

namespace dh {

constexpr int QX = 32;              // threads along x (one warp per row)
constexpr int QY = 8;               // rows of the tile (warps)
constexpr int QNT = QX * QY;        // threads per CTA
constexpr int QCX = 2 * QX;         // cells along x per tile
constexpr int QRW = QX + 4;         // ring positions per row: -2 .. 33
constexpr int QRH = QY + 4;         // ring rows: -2 .. 9

template <typename real> struct PairStaging {
  static constexpr int SCE = 16 / (int)sizeof(real);   // x-halo box width: 16 bytes
  static constexpr uint32_t BYTES = (uint32_t)sizeof(real) * 5u * (QCX * QY + 2 * QY * SCE + 4 * QCX);
};

template <typename real> struct PairSmem {
  using P = pair_t<real>;
  using Q = Quad<real>;
  static constexpr int SCE = PairStaging<real>::SCE;
  // staged conserved variables of the planes in flight (TMA destinations, slot = plane & 1)
  alignas(128) real core[2][5][QY][QCX];   // cells x0 .. x0 + 63, rows y0 .. y0 + 7
  alignas(128) real xl[2][5][QY][SCE];     // x0 - SCE .. x0 - 1
  alignas(128) real xr[2][5][QY][SCE];     // x0 + 64 .. x0 + 63 + SCE
  alignas(128) real yt[2][5][2][QCX];      // rows y0 - 2, y0 - 1
  alignas(128) real yb[2][5][2][QCX];      // rows y0 + 8, y0 + 9
  // primitive pairs of planes k and k + 1 (slot = plane & 1) at rows -2..9, positions -2..33:
  // (rho, vx), (vy, vz), p.  Corner positions are never written or read.
  Q w01[2][QRH][QRW];
  Q w23[2][QRH][QRW];
  P wp[2][QRH][QRW];
  // half slopes dW/2 of plane k: x at rows 0..7, positions -1..32; y at rows -1..8, positions 0..31
  Q hx01[QY][QX + 2], hx23[QY][QX + 2];
  P hxp[QY][QX + 2];
  Q hy01[QY + 2][QX], hy23[QY + 2][QX];
  P hyp[QY + 2][QX];
  // face fluxes of plane k: x face p (between positions p - 1 and p) of rows 0..7, p = 0..32;
  // y face r (between rows r - 1 and r), r = 0..8
  Q fx01[QY][QX + 1], fx23[QY][QX + 1];
  P fxe[QY][QX + 1];
  Q fy01[QY + 1][QX], fy23[QY + 1][QX];
  P fye[QY + 1][QX];
  // forcing row factors B[row][n_x][component] (re, im) of plane j - 2, staged with plane j
  alignas(16) real fB[2][QY][3][3][2];
  real red[QNT / 32];           // CFL reduction scratch
  alignas(8) uint64_t bar[2];   // staging slot landed (TMA transaction bytes; slot = plane & 1)
};
static_assert(2 * (sizeof(PairSmem<float>) + 1024) <= 228 * 1024, "two float32 CTAs per SM");
static_assert(sizeof(PairSmem<float>::core[0]) == 5 * QY * QCX * sizeof(float) &&
              sizeof(PairSmem<float>::xl[0]) == 5 * QY * PairStaging<float>::SCE * sizeof(float) &&
              sizeof(PairSmem<float>::yt[0]) == 5 * 2 * QCX * sizeof(float), "staging slot strides");
static_assert(sizeof(PairSmem<double>) + 1024 <= 228 * 1024, "one float64 CTA per SM");

// Bound on the probes of the staging mbarrier (a plane's copies land in microseconds); a wait
// that reaches it sets FLAG_TIMEOUT and the CTA stops.
constexpr uint32_t PAIR_WAIT_ITERS = 1u << 22;

template <typename real>
__device__ __forceinline__ Prim2<real> qload(const Quad<real>& a, const Quad<real>& b, const pair_t<real>& p) {
  const Quad<real> x = a, y = b;
  return Prim2<real>{x.a, x.b, y.a, y.b, p};
}
template <typename real>
__device__ __forceinline__ void qstore(Quad<real>& a, Quad<real>& b, pair_t<real>& p, const Prim2<real>& w) {
  a = Quad<real>{w.r, w.vx};
  b = Quad<real>{w.vy, w.vz};
  p = w.p;
}

// Conserved pair (cells A and B) from shared or global memory: field f of A at pa[f * sa],
// of B at pb[f * sb].
template <typename real>
__device__ __forceinline__ Prim2<real> convert_pair(const real* pa, int sa, const real* pb, int sb, real gm1) {
  return cons_to_prim2<real>(pmk(pa[0], pb[0]), pmk(pa[sa], pb[sb]), pmk(pa[2 * sa], pb[2 * sb]),
                             pmk(pa[3 * sa], pb[3 * sb]), pmk(pa[4 * sa], pb[4 * sb]), gm1);
}
template <typename real>
__device__ __forceinline__ Prim2<real> gload_pair(const real* __restrict__ U, long long n3, long long ia,
                                                  long long ib, real gm1) {
  return cons_to_prim2<real>(pmk(__ldg(U + ia), __ldg(U + ib)), pmk(__ldg(U + n3 + ia), __ldg(U + n3 + ib)),
                             pmk(__ldg(U + 2 * n3 + ia), __ldg(U + 2 * n3 + ib)),
                             pmk(__ldg(U + 3 * n3 + ia), __ldg(U + 3 * n3 + ib)),
                             pmk(__ldg(U + 4 * n3 + ia), __ldg(U + 4 * n3 + ib)), gm1);
}

// Work of a plane.  Thread (tx, ty) owns the pair at row ty, position tx: its conversion, x and
// y half slopes, x face tx (its left face), y face ty (its lower face), z slope, z faces and
// update.  Fixed tails: the conversion of the 160 halo pairs (threads 96..255), the y slopes of
// rows -1 and 8 (warps 0 and 1), the x slopes of positions -1 and 32 (warp 2, lanes 0..15), the
// x face 32 of each row (warp 6, lanes 0..7) and the y face 8 of each position (warp 7).
// float32: two CTAs per SM (shared memory and 128 registers); float64: one.
// Per-field base pointers of the stage's state buffers, read from the parameter bank, so that a
// cell's address is one 32-bit index scaled onto a constant base (grids below 2^31 cells per field).
template <typename real> struct FieldPtrs {
  const real* U[5];
  const real* U0[5];
  real* out[5];
  real* pre[5];
};

template <typename real, int STAGE, int LIM>
__global__ void __launch_bounds__(QNT, sizeof(real) == 4 ? 2 : 1)
stage_pair_kernel(const StageArgs<real> p, const int zchunk, const __grid_constant__ StageTma tma,
                  const __grid_constant__ FieldPtrs<real> fp) {
  using P = pair_t<real>;
  using Q = Quad<real>;
  using ST = PairStaging<real>;
  constexpr int SCE = ST::SCE;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  PairSmem<real>& S = *reinterpret_cast<PairSmem<real>*>(smem_raw);
  const int tid = threadIdx.x;
  // Skip the stage after a fatal failure (one thread reads the flag; the CTA follows it).
  __shared__ unsigned s_skip;
  __shared__ int s_abort;
  if (tid == 0) {
    s_skip = *((volatile unsigned*)&p.rec->flags) & FATAL_FLAGS;
    s_abort = 0;
  }
  __syncthreads();
  if (s_skip) return;

  const int tx = tid & (QX - 1), ty = tid / QX;
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  const long long plane = (long long)nx * ny;
  const long long n3 = plane * nz;
  const int x0 = blockIdx.x * QCX, y0 = blockIdx.y * QY;
  const int z0 = blockIdx.z * zchunk;
  const int z1 = min(z0 + zchunk, nz);
  const real dt = (real)*p.dtp;
  const real gamma = p.gamma, gm1 = p.gm1, igm1 = real(1) / p.gm1;
  // STAGE 1: out = U + dt L(U).  STAGE 2: RK2's final stage (U0 + U + dt L(U)) / 2.  STAGE 3:
  // out = w0 U0 + w1 (U + dt L(U)) (SSPRK3); the final stage takes the epilogue.
  constexpr bool COMB = STAGE >= 2;
  const bool final = STAGE == 2 || (STAGE == 3 && p.final_stage);
  const real w0c = STAGE == 2 ? real(0.5) : p.w0, w1c = STAGE == 2 ? real(0.5) : p.w1;
  const bool forcing = final && p.forcing;
  if (tid == 32) {
    tc::mbar_init(&S.bar[0], 1u);
    tc::mbar_init(&S.bar[1], 1u);
    tc::mbar_fence_init();
  }
  // wrapped start coordinates of the halo boxes
  const int xl0 = x0 >= SCE ? x0 - SCE : nx - SCE, xr0 = x0 + QCX < nx ? x0 + QCX : 0;
  const int yt0 = y0 >= 2 ? y0 - 2 : ny - 2, yb0 = y0 + QY < ny ? y0 + QY : 0;
  __syncthreads();

  // thread 0: the five boxes of plane k on the staging barrier, and with forcing the row factors
  // of plane k - 2 (the plane whose update runs when plane k is converted)
  constexpr uint32_t FB_BYTES = (uint32_t)sizeof(real) * QY * 18;
  auto stage_plane = [&](int k) {
    const int kz = wrap(k, nz), b = k & 1;
    const uint32_t bar = tc::smem_u32(&S.bar[b]);
    tc::mbar_arrive_expect_tx(&S.bar[b], ST::BYTES + (forcing ? FB_BYTES : 0u));
    if (forcing)
      tc::bulk_g2s(tc::smem_u32(&S.fB[b][0][0][0][0]), p.frow + ((long long)wrap(k - 2, nz) * ny + y0) * 18,
                   FB_BYTES, &S.bar[b]);
    tma_load_4d(tc::smem_u32(&S.core[b][0][0][0]), &tma.core, x0, y0, kz, 0, bar);
    tma_load_4d(tc::smem_u32(&S.xl[b][0][0][0]), &tma.xh, xl0, y0, kz, 0, bar);
    tma_load_4d(tc::smem_u32(&S.xr[b][0][0][0]), &tma.xh, xr0, y0, kz, 0, bar);
    tma_load_4d(tc::smem_u32(&S.yt[b][0][0][0]), &tma.yh, x0, yt0, kz, 0, bar);
    tma_load_4d(tc::smem_u32(&S.yb[b][0][0][0]), &tma.yh, x0, yb0, kz, 0, bar);
  };

  // ---- fixed per-thread tasks ----------------------------------------------------------------
  // halo conversion (threads 96..255): staged sources of lanes A and B with their field
  // strides, the ring position, and the global coordinates (for the prologue's direct loads)
  // (slot 1 of each staging array lies a fixed number of elements after slot 0)
  constexpr int CORE_SLOT = 5 * QY * QCX, XH_SLOT = 5 * QY * SCE, YH_SLOT = 5 * 2 * QCX;
  const int hbase = 96;
  const bool halo = tid >= hbase;
  const real* hsa = nullptr;
  const real* hsb = nullptr;
  int hfa = 0, hfb = 0, hoa = 0, hob = 0, hr = 0, hp = 0, hgxa = 0, hgxb = 0, hgy = 0;
  if (halo) {
    const int e = tid - hbase;   // 0 .. 159
    if (e < 128) {            // y halo rows -2, -1 (e < 64) and 8, 9
      const bool top = e < 64;
      const int row = (e >> 5) & 1, q = e & 31;
      const real* base = top ? &S.yt[0][0][row][0] : &S.yb[0][0][row][0];
      hsa = base + q; hsb = base + q + QX; hfa = hfb = 2 * QCX; hoa = hob = YH_SLOT;
      hr = top ? row - 2 : QY + row; hp = q;
      hgy = top ? wrap(y0 - 2 + row, ny) : wrap(y0 + QY + row, ny);
      hgxa = x0 + q; hgxb = x0 + QX + q;
    } else {                  // x halo positions -2, -1 (e < 144) and 32, 33
      const int q = (e - 128) & 15, ly = q & 7, c = q >> 3;
      if (e < 144) {
        hsa = &S.xl[0][0][ly][SCE - 2 + c]; hfa = QY * SCE; hoa = XH_SLOT;
        hsb = &S.core[0][0][ly][QX - 2 + c]; hfb = QY * QCX; hob = CORE_SLOT;
        hp = c - 2; hgxa = wrap(x0 - 2 + c, nx); hgxb = x0 + QX - 2 + c;
      } else {
        hsa = &S.core[0][0][ly][QX + c]; hfa = QY * QCX; hoa = CORE_SLOT;
        hsb = &S.xr[0][0][ly][c]; hfb = QY * SCE; hob = XH_SLOT;
        hp = QX + c; hgxa = x0 + QX + c; hgxb = wrap(x0 + QCX + c, nx);
      }
      hr = ly; hgy = y0 + ly;
    }
  }
  // slope tail: y slopes of rows -1 (warp 0) and 8 (warp 1), x slopes of positions -1 and 32
  // (warp 2, lanes 0..15): the ring row and position of the cell
  int sr = -100, sp = 0;
  bool sy = false;
  if (tid < 64) {
    sr = tid < 32 ? -1 : QY; sp = tx; sy = true;
  } else if (tid < 80) {
    const int q = tid - 64;
    sr = q & 7; sp = q < 8 ? -1 : QX;
  }
  // face tail: x face 32 of row lane (warp 6, lanes 0..7), y face 8 of position lane (warp 7)
  const bool fx_tail = ty == 6 && tx < QY, fy_tail = ty == 7;

  auto ring = [&](int slot, int r, int q) {
    return qload<real>(S.w01[slot][r + 2][q + 2], S.w23[slot][r + 2][q + 2], S.wp[slot][r + 2][q + 2]);
  };
  auto ring_put = [&](int slot, int r, int q, const Prim2<real>& w) {
    qstore<real>(S.w01[slot][r + 2][q + 2], S.w23[slot][r + 2][q + 2], S.wp[slot][r + 2][q + 2], w);
  };
  auto hx_get = [&](int r, int q) { return qload<real>(S.hx01[r][q + 1], S.hx23[r][q + 1], S.hxp[r][q + 1]); };
  auto hy_get = [&](int r, int q) { return qload<real>(S.hy01[r + 1][q], S.hy23[r + 1][q], S.hyp[r + 1][q]); };

  // x twiddles of the own pair (forcing synthesis), fixed for the whole march
  P twx[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) twx[q] = pset(real(0));
  if (forcing) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
      twx[q] = pmk(__ldg(p.tw[0] + 4 * (x0 + tx) + q), __ldg(p.tw[0] + 4 * (x0 + QX + tx) + q));
  }

  // ---- prologue: plane z0 into its ring slot; own column z0 - 2, z0 - 1 in registers ----------
  const long long col = (long long)(y0 + ty) * nx + (x0 + tx);
  Prim2<real> w_k, w_km1, h_km1;
  {
    const long long zo = (long long)wrap(z0, nz) * plane;
    w_k = gload_pair<real>(p.U, n3, zo + col, zo + col + QX, gm1);
    ring_put(z0 & 1, ty, tx, w_k);
    if (halo) {
      const long long hb = zo + (long long)hgy * nx;
      ring_put(z0 & 1, hr, hp, gload_pair<real>(p.U, n3, hb + hgxa, hb + hgxb, gm1));
    }
    const long long zm1 = (long long)wrap(z0 - 1, nz) * plane, zm2 = (long long)wrap(z0 - 2, nz) * plane;
    w_km1 = gload_pair<real>(p.U, n3, zm1 + col, zm1 + col + QX, gm1);
    const Prim2<real> w_km2 = gload_pair<real>(p.U, n3, zm2 + col, zm2 + col + QX, gm1);
    int ua = 0, ub = 0;
    h_km1 = limited_half2<LIM>(w_km2, w_km1, w_k, ua, ub);
  }
  if (tid == 0) {
    stage_plane(z0 + 1);
    stage_plane(z0 + 2);
  }
  __syncthreads();

  P fz_lo[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) fz_lo[c] = pset(real(0));
  int nfa = 0, nfb = 0;   // positivity fallbacks of the own cells' slopes (lanes A, B)
  real tmin = real(INFINITY);
  unsigned flags = 0;
  int nsub_seen = 0;

  for (int k = z0; k <= z1; ++k) {
    if (!tc::mbar_wait(&S.bar[(k + 1) & 1], (uint32_t)((k - z0) >> 1) & 1u, PAIR_WAIT_ITERS)) s_abort = 1;
    __syncthreads();   // ---- plane k+1 staged; the fluxes of plane k-1 are in shared memory
    if (s_abort) break;
    const bool last = k == z1;
    const int sk = k & 1, sk1 = sk ^ 1;

    // x/y divergence of plane k-1 from its face fluxes (written last iteration)
    // the own cells' U (and U0) of plane k-1, loaded early for its update below
    P uin_e[5], un_e[5];
    const int ia32 = (k - 1) * (int)plane + (int)col;
    if (k > z0) {
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        uin_e[c] = pmk(__ldg(fp.U[c] + ia32), __ldg(fp.U[c] + ia32 + QX));
        if (COMB) un_e[c] = pmk(__ldg(fp.U0[c] + ia32), __ldg(fp.U0[c] + ia32 + QX));
      }
    }
    P lxy[5];
    if (k > z0) {
      const Q ar = S.fx01[ty][tx + 1], al = S.fx01[ty][tx], br = S.fx23[ty][tx + 1], bl = S.fx23[ty][tx];
      const Q cu = S.fy01[ty + 1][tx], cd = S.fy01[ty][tx], du = S.fy23[ty + 1][tx], dd = S.fy23[ty][tx];
      const P ex = psub(S.fxe[ty][tx + 1], S.fxe[ty][tx]), ey = psub(S.fye[ty + 1][tx], S.fye[ty][tx]);
      const P mix = pset(-p.idx), miy = pset(-p.idy);
      lxy[0] = pfma(psub(cu.a, cd.a), miy, pmul(psub(ar.a, al.a), mix));
      lxy[1] = pfma(psub(cu.b, cd.b), miy, pmul(psub(ar.b, al.b), mix));
      lxy[2] = pfma(psub(du.a, dd.a), miy, pmul(psub(br.a, bl.a), mix));
      lxy[3] = pfma(psub(du.b, dd.b), miy, pmul(psub(br.b, bl.b), mix));
      lxy[4] = pfma(ey, miy, pmul(ex, mix));
    }

    // conversion of the staged plane k+1: own pair (registers and ring), halo pairs (ring)
    const int sb = (k + 1) & 1;
    const Prim2<real> w_k1 = convert_pair<real>(&S.core[sb][0][ty][tx], QY * QCX, &S.core[sb][0][ty][tx + QX], QY * QCX, gm1);
    if (!last) {
      ring_put(sk1, ty, tx, w_k1);
      if (halo) ring_put(sk1, hr, hp, convert_pair<real>(hsa + sb * hoa, hfa, hsb + sb * hob, hfb, gm1));

      // x and y half slopes of plane k: own pair, then the tail
      {
        const Prim2<real> hxo = limited_half2<LIM>(ring(sk, ty, tx - 1), w_k, ring(sk, ty, tx + 1), nfa, nfb);
        qstore<real>(S.hx01[ty][tx + 1], S.hx23[ty][tx + 1], S.hxp[ty][tx + 1], hxo);
        const Prim2<real> hyo = limited_half2<LIM>(ring(sk, ty - 1, tx), w_k, ring(sk, ty + 1, tx), nfa, nfb);
        qstore<real>(S.hy01[ty + 1][tx], S.hy23[ty + 1][tx], S.hyp[ty + 1][tx], hyo);
      }
      if (sr > -100) {
        int u0 = 0, u1 = 0;
        if (sy) {
          const Prim2<real> h = limited_half2<LIM>(ring(sk, sr - 1, sp), ring(sk, sr, sp), ring(sk, sr + 1, sp), u0, u1);
          qstore<real>(S.hy01[sr + 1][sp], S.hy23[sr + 1][sp], S.hyp[sr + 1][sp], h);
        } else {
          const Prim2<real> h = limited_half2<LIM>(ring(sk, sr, sp - 1), ring(sk, sr, sp), ring(sk, sr, sp + 1), u0, u1);
          qstore<real>(S.hx01[sr][sp + 1], S.hx23[sr][sp + 1], S.hxp[sr][sp + 1], h);
        }
      }
    }

    // z slope of plane k and the z face k - 1/2 of the own column
    Prim2<real> d_k;
    {
      int za = 0, zb = 0;
      d_k = limited_half2<LIM>(w_km1, w_k, w_k1, za, zb);
      if (!last) {
        nfa += za;
        nfb += zb;
      }
    }
    P fz_hi[5];
    face_flux2<2, real>(face_state2<real>(w_km1, h_km1, true), face_state2<real>(w_k, d_k, false), gamma, igm1, fz_hi);

    // plane k-1 is complete: stage combination, epilogue, store
    if (k > z0) {
      P u[5];
      const P miz = pset(-p.idz), pdt = pset(dt);
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        const P uin = uin_e[c];
        const P L = pfma(psub(fz_hi[c], fz_lo[c]), miz, lxy[c]);
        P v = pfma(pdt, L, uin);
        if (COMB) {
          const P un = un_e[c];
          v = pfma(pset(w0c), un, pmul(pset(w1c), v));
        }
        u[c] = v;
      }
      if (COMB && final) {
        if (p.pre_src) {
#pragma unroll
          for (int c = 0; c < 5; ++c) {
            fp.pre[c][ia32] = u[c].x;
            fp.pre[c][ia32 + QX] = u[c].y;
          }
        }
        if (forcing) {
          // a = 2 Re sum_{n_x} B_{n_x} exp(2 pi i n_x x~)  (Sec. 3.1.1)
          const real(*B)[3][2] = S.fB[(k + 1) & 1][ty];   // staged with plane k + 1
          P a[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const P t1 = pfma(pset(B[1][c][0]), twx[0], pmul(pset(-B[1][c][1]), twx[1]));
            const P t2 = pfma(pset(B[2][c][0]), twx[2], pmul(pset(-B[2][c][1]), twx[3]));
            a[c] = pmul(pset(real(2)), padd(padd(pset(B[0][c][0]), t1), t2));
          }
          const P e = pmul(pfma(u[3], a[2], pfma(u[2], a[1], pmul(u[1], a[0]))), pdt);
          u[1] = pfma(pmul(u[0], a[0]), pdt, u[1]);
          u[2] = pfma(pmul(u[0], a[1]), pdt, u[2]);
          u[3] = pfma(pmul(u[0], a[2]), pdt, u[3]);
          u[4] = padd(u[4], e);
        }
        if (p.cooling)
          u[4] = cooling_energy2<real>(u[0], u[1], u[2], u[3], u[4], dt, gm1, p.t_floor, p.cool_frac,
                                       p.nsub_max, flags, nsub_seen);
        bool fa = true, fb = true;
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          fa = fa && isfinite(u[c].x);
          fb = fb && isfinite(u[c].y);
        }
        P pres;
        const P tc = cfl_time2<real>(u, gamma, gm1, p.dx, p.dy, p.dz, pres);
        auto finish = [&](bool fin, real rho, real pr, real t, int lane) {
          if (!fin) {
            flags |= FLAG_NONFINITE;
            return;
          }
          if (!(rho > real(0)) || !(pr > real(0))) flags |= FLAG_POSITIVITY;
          if (p.reduce_cfl) {
            tmin = fmin(tmin, t);
            if (p.cool_ratio > real(0)) {
              const real v[5] = {lane ? u[0].y : u[0].x, lane ? u[1].y : u[1].x, lane ? u[2].y : u[2].x,
                                 lane ? u[3].y : u[3].x, lane ? u[4].y : u[4].x};
              tmin = fmin(tmin, p.cool_ratio * cooling_time(v[0], v[1], v[2], v[3], v[4], gm1, p.t_floor));
            }
          }
        };
        finish(fa, u[0].x, pres.x, tc.x, 0);
        finish(fb, u[0].y, pres.y, tc.y, 1);
      }
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        fp.out[c][ia32] = u[c].x;
        fp.out[c][ia32 + QX] = u[c].y;
      }
    }
    if (last) break;

    __syncthreads();   // ---- half slopes of plane k ready; the staging buffers are free

    if (tid == 0 && k + 3 <= z1 + 1) stage_plane(k + 3);
    // x face tx and y face ty of the own pair, then the tail faces
    {
      P F[5];
      const Prim2<real> hxo = hx_get(ty, tx);
      face_flux2<0, real>(face_state2<real>(ring(sk, ty, tx - 1), hx_get(ty, tx - 1), true),
                          face_state2<real>(w_k, hxo, false), gamma, igm1, F);
      S.fx01[ty][tx] = Q{F[0], F[1]};
      S.fx23[ty][tx] = Q{F[2], F[3]};
      S.fxe[ty][tx] = F[4];
      const Prim2<real> hyo = hy_get(ty, tx);
      face_flux2<1, real>(face_state2<real>(ring(sk, ty - 1, tx), hy_get(ty - 1, tx), true),
                          face_state2<real>(w_k, hyo, false), gamma, igm1, F);
      S.fy01[ty][tx] = Q{F[0], F[1]};
      S.fy23[ty][tx] = Q{F[2], F[3]};
      S.fye[ty][tx] = F[4];
    }
    if (fx_tail) {
      P F[5];
      face_flux2<0, real>(face_state2<real>(ring(sk, tx, QX - 1), hx_get(tx, QX - 1), true),
                          face_state2<real>(ring(sk, tx, QX), hx_get(tx, QX), false), gamma, igm1, F);
      S.fx01[tx][QX] = Q{F[0], F[1]};
      S.fx23[tx][QX] = Q{F[2], F[3]};
      S.fxe[tx][QX] = F[4];
    }
    if (fy_tail) {
      P F[5];
      face_flux2<1, real>(face_state2<real>(ring(sk, QY - 1, tx), hy_get(QY - 1, tx), true),
                          face_state2<real>(ring(sk, QY, tx), hy_get(QY, tx), false), gamma, igm1, F);
      S.fy01[QY][tx] = Q{F[0], F[1]};
      S.fy23[QY][tx] = Q{F[2], F[3]};
      S.fye[QY][tx] = F[4];
    }

    w_km1 = w_k;
    w_k = w_k1;
    h_km1 = d_k;
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
    unsigned long long n = (unsigned long long)(nfa + nfb);
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
        for (int w = 1; w < QNT / 32; ++w) m = fmin(m, S.red[w]);
        if (m < real(INFINITY)) atomicMin(&p.rec->cfl_min_bits, ordered_bits(m));
      }
    }
  }
}

// The forcing row factors of every (y, z) row of the step (Sec. 3.1.1): for n_x in {0, 1, 2} and
// component c, B = sum over the forced modes with that n_x of a_hat_{m,c} exp(2 pi i (n_y y~ +
// n_z z~)), stored [z][y][n_x][c][re, im].  One thread per (row, component).
template <typename real>
__global__ void forcing_rows_kernel(const real* __restrict__ ah, const real* __restrict__ tw1,
                                    const real* __restrict__ tw2, int ny, int nz, real* __restrict__ out) {
  __shared__ real s_ah[96];
  for (int i = threadIdx.x; i < 96; i += blockDim.x) s_ah[i] = ah[i];
  __syncthreads();
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3ll * ny * nz) return;
  const int c = (int)(t % 3);
  const long long row = t / 3;
  const int y = (int)(row % ny), z = (int)(row / ny);
  real tyv[4], tzv[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    tyv[i] = tw1[4 * y + i];
    tzv[i] = tw2[4 * z + i];
  }
  real bre[3] = {real(0), real(0), real(0)}, bim[3] = {real(0), real(0), real(0)};
  row_factors3<real, 0>(s_ah, c, tyv, tzv, bre, bim);
  real* o = out + row * 18;
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    o[(b * 3 + c) * 2] = bre[b];
    o[(b * 3 + c) * 2 + 1] = bim[b];
  }
}

template <typename real, int STAGE, int LIM>
static cudaError_t launch_pair_t(const StageArgs<real>& a, const StageTma& maps, cudaStream_t s) {
  auto kernel = stage_pair_kernel<real, STAGE, LIM>;
  const size_t smem = sizeof(PairSmem<real>);
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  static int resident = 0;   // CTAs per SM of this instance
  if (resident <= 0) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, kernel, QNT, smem);
    if (e != cudaSuccess) return e;
    if (resident <= 0) resident = 1;
  }
  const long long tiles = (long long)(a.nx / QCX) * (a.ny / QY);
  // small grids fill the GPU with short chunks (down to two planes); a chunk's start costs
  // about two planes (three planes loaded and converted, and the trailing half iteration)
  const int zc = wave_zchunk(tiles, a.nz, resident, 2.0, 2);
  dim3 grid(a.nx / QCX, a.ny / QY, (a.nz + zc - 1) / zc);
  FieldPtrs<real> fp;
  for (int c = 0; c < 5; ++c) {
    const long long off = (long long)c * a.nx * a.ny * a.nz;
    fp.U[c] = a.U + off;
    fp.U0[c] = a.U0 ? a.U0 + off : nullptr;
    fp.out[c] = a.out + off;
    fp.pre[c] = a.pre_src ? a.pre_src + off : nullptr;
  }
  kernel<<<grid, QNT, smem, s>>>(a, zc, maps, fp);
  return cudaGetLastError();
}

template <typename real>
bool launch_stage_pair(int stage, const StageArgs<real>& a, cudaStream_t s, cudaError_t& err, int& launched) {
  launched = 0;
  // whole 64 x 8 tiles (every halo box contiguous), at least four planes, a 16-byte aligned base
  if (a.nx % QCX != 0 || a.ny % QY != 0 || a.nz < 4 || ((unsigned long long)a.U & 15ull) != 0 ||
      (long long)a.nx * a.ny * a.nz >= (1ll << 31))
    return false;
  const bool final = stage == 2 || (stage == 3 && a.final_stage);
  if (final && a.forcing && (!a.frow || ((unsigned long long)a.frow & 15ull) != 0)) return false;
  StageTma maps;
  std::memset(&maps, 0, sizeof(maps));
  if (!stage_tma_maps(a.U, a.nx, a.ny, a.nz, (int)sizeof(real), QCX, QY, PairStaging<real>::SCE, 2, &maps))
    return false;
  if (final && a.forcing) {
    const long long nt = 3ll * a.ny * a.nz;
    forcing_rows_kernel<real><<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(a.ahat_norm, a.tw[1], a.tw[2],
                                                                           a.ny, a.nz, a.frow);
    err = cudaGetLastError();
    launched = 1;
    if (err != cudaSuccess) return true;
  }
  ++launched;
  if (a.limiter == LIM_VL) {
    if (stage == 1) err = launch_pair_t<real, 1, LIM_VL>(a, maps, s);
    else if (stage == 2) err = launch_pair_t<real, 2, LIM_VL>(a, maps, s);
    else err = launch_pair_t<real, 3, LIM_VL>(a, maps, s);
  } else {
    if (stage == 1) err = launch_pair_t<real, 1, LIM_MC>(a, maps, s);
    else if (stage == 2) err = launch_pair_t<real, 2, LIM_MC>(a, maps, s);
    else err = launch_pair_t<real, 3, LIM_MC>(a, maps, s);
  }
  return true;
}
template bool launch_stage_pair<float>(int, const StageArgs<float>&, cudaStream_t, cudaError_t&, int&);
template bool launch_stage_pair<double>(int, const StageArgs<double>&, cudaStream_t, cudaError_t&, int&);

}  // namespace dh
