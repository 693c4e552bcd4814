// Multigrid self-gravity (Sec. 5.2; App. C) and the operator-split source kernel of steps that
// use it.
//
// Solve A phi = F, F = 4 pi G (rho - <rho>), A the seven-point periodic Laplacian.  The fine
// level keeps phi and F in float-float (a pair of float32 words, ~48 significant bits, ff.cuh)
// and iterates defect correction: r = F - A phi (float-float), then one float32 V-cycle for
// A e = r (red-black Gauss-Seidel, mg_pre / mg_post sweeps, 8-child mean restriction,
// cell-centred trilinear prolongation, exact coarsest solve), then phi += e.  For a linear
// smoother this is the V-cycle applied to phi itself, so the iterates are those of Sec. 5.2's
// cycle; keeping phi and the residual in extended precision lets the relative residual reach
// 1e-6 at large N, which float32 phi cannot (its rounding alone leaves ~eps_32 * |phi| / h^2 in
// A phi).  Float-float runs on the float32 pipes: on this part float64 arithmetic is scarce
// enough that a float64 residual is bound by it.  Norms and means are accumulated per thread
// in compensated float32 and across threads in float64, in a fixed order; the residual norm is
// taken relative to the RMS of F, so the working range is that of float32.
//
// The coarsest grid (<= 1024 cells) is solved with the pseudo-inverse of its operator, a
// circulant: A^+ e_p = sum_q G[(p - q) mod n] r_q with G[d] = (1/N) sum_{k != 0}
// cos(2 pi k.d / n) / lambda_k and lambda_k = -(4/h^2) sum_a sin^2(pi k_a / n_a), the discrete
// eigenvalues; it also removes the mean (the constant null space).
#include <math.h>
#include <string.h>
#include <utility>
#include <vector>

#include "async_copy.cuh"
#include "dh_internal.h"
#include "dh_pair_sources.cuh"
#include "dh_sources.cuh"
#include "ff.cuh"

namespace dh {
constexpr int MG_LMAX = 16;
// State of one solve on the device.  The residual of each iterate is judged by
// mg_decide_kernel, so the host enqueues several cycles between reads of this block; once stop
// is set, the kernels enqueued after it return at once.
struct MGCtl {
  int stop;      // the solve has finished (first word: the kernels' guard)
  int cycles;    // cycles run
  int ok;        // the residual reached mg_tol (or the source is zero)
  int zero;      // zero source: phi = 0
  int skipped;   // a fatal failure earlier in the step: nothing solved
  int pad;
  double rel;    // ||F - A phi||_2 / ||F||_2 of the last iterate
};
// reductions: 8 CTAs per SM over 148 SMs (enough warps to cover the stencil loads), then one
// warp adds the per-block partials in a fixed order
constexpr int RED_BLOCKS = 148 * 8, RED_THREADS = 256;
// the residual's z-march: 32 x 8 columns of RZ_ZC planes (one partial sum per CTA)
constexpr int RZ_TX = 32, RZ_TY = 8, RZ_ZC = 64;
constexpr int RZ_HX = RZ_TX + 2, RZ_HY = RZ_TY + 2, RZ_H = RZ_HX * RZ_HY;
constexpr int RZ_D = 2, RZ_RING = 4 + RZ_D;
inline long long residual_zm_blocks(int nx, int ny, int nz) {
  return (long long)((nx + RZ_TX - 1) / RZ_TX) * ((ny + RZ_TY - 1) / RZ_TY) * ((nz + RZ_ZC - 1) / RZ_ZC);
}
}

struct MG {
  int L = 0;
  int n[dh::MG_LMAX][3];
  double h[dh::MG_LMAX];
  long long cells[dh::MG_LMAX];
  // potential and source in float-float, planar: n hi floats then n lo floats (ff.cuh)
  float* phi = nullptr;
  float* phi2 = nullptr;         // the other buffer of the residual's fused update
  float* F = nullptr;
  float* e[dh::MG_LMAX] = {nullptr};
  float* e2[dh::MG_LMAX] = {nullptr};   // the sweep's other buffer (a sweep writes e2, then swaps)
  float* r[dh::MG_LMAX] = {nullptr};
  // float64 correction hierarchy of a float64 context (instead of e / e2 / r): its cycles are
  // the oracle's float64 cycles, so its iterates match them to rounding
  bool f64 = false;
  double* de[dh::MG_LMAX] = {nullptr};
  double* de2[dh::MG_LMAX] = {nullptr};  // Jacobi's other buffer
  double* dr[dh::MG_LMAX] = {nullptr};
  double* G = nullptr;           // coarsest circulant pseudo-inverse
  double* partials = nullptr;    // max(RED_BLOCKS, residual CTAs) doubles
  double* scal = nullptr;        // [0] mean rho, [1] |F|^2, [2] |r|^2, [3] mean phi
  // the solve's control block on the device (dh::MGCtl); stop points at its first word, which
  // every kernel of a cycle and of the residual reads first
  void* ctl = nullptr;
  int* stop = nullptr;
  int last_cycles = 0;
  double last_res = 0.0;
  // One cycle as a CUDA graph (captured on first use): its hundreds of small launches at the
  // coarse levels (a W-cycle visits level l 2^l times) replay without per-launch host work.
  // Valid while the e / e2 buffers are where they were at capture, which holds when every
  // level swaps them an even number of times per cycle.
  cudaGraphExec_t cycle_exec = nullptr;
  float* cycle_e[dh::MG_LMAX] = {nullptr};
  float* cycle_e2[dh::MG_LMAX] = {nullptr};
  long long cycle_launches = 0;
  bool cycle_graph_failed = false;
};

namespace dh {

static void level_dims(const dh_config& c, MG* m) {
  int d[3] = {c.nx, c.ny, c.nz};
  double h = c.dx;
  m->L = 0;
  while (true) {
    const int l = m->L++;
    for (int a = 0; a < 3; ++a) m->n[l][a] = d[a];
    m->h[l] = h;
    m->cells[l] = (long long)d[0] * d[1] * d[2];
    const bool halve = d[0] % 2 == 0 && d[1] % 2 == 0 && d[2] % 2 == 0 && d[0] >= 8 &&
                       d[1] >= 8 && d[2] >= 8 && m->L < MG_LMAX;
    if (!halve) break;
    for (int a = 0; a < 3; ++a) d[a] /= 2;
    h *= 2.0;
  }
}

std::string mg_validate(const dh_config& c) {
  if (std::fabs(c.dx - c.dy) > 1e-12 * c.dx || std::fabs(c.dx - c.dz) > 1e-12 * c.dx)
    return "gravity needs cubic cells (dx == dy == dz)";
  if (c.mg_max_cycles < 1 || c.mg_pre < 0 || c.mg_post < 0) return "bad multigrid cycle settings";
  if (!(c.mg_tol > 0.0)) return "mg_tol must be positive";
  if (c.mg_smoother != 0 && c.mg_smoother != 1) return "mg_smoother must be 0 (RBGS) or 1 (Jacobi)";
  if (!(c.mg_omega > 0.0 && c.mg_omega <= 1.0)) return "mg_omega must lie in (0, 1]";
  if (c.mg_cycle != 1 && c.mg_cycle != 2) return "mg_cycle must be 1 (V) or 2 (W)";
  MG m;
  level_dims(c, &m);
  if (m.cells[m.L - 1] > 1024) return "coarsest multigrid level exceeds 1024 cells";
  return "";
}

cudaError_t mg_allocate(dh_ctx* c) {
  MG* m = new MG();
  c->mg = m;
  level_dims(c->cfg, m);
  cudaError_t e = cudaMalloc(&m->phi, 2 * m->cells[0] * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->phi2, 2 * m->cells[0] * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->F, 2 * m->cells[0] * sizeof(float));
  m->f64 = c->prec == DH_F64;
  for (int l = 0; l < m->L && e == cudaSuccess; ++l) {
    if (m->f64) {
      e = cudaMalloc(&m->de[l], m->cells[l] * sizeof(double));
      if (e == cudaSuccess) e = cudaMalloc(&m->de2[l], m->cells[l] * sizeof(double));
      if (e == cudaSuccess) e = cudaMalloc(&m->dr[l], m->cells[l] * sizeof(double));
      continue;
    }
    e = cudaMalloc(&m->e[l], m->cells[l] * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&m->e2[l], m->cells[l] * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&m->r[l], m->cells[l] * sizeof(float));
  }
  if (e == cudaSuccess) e = cudaMalloc(&m->G, m->cells[m->L - 1] * sizeof(double));
  {
    const long long rb = residual_zm_blocks(m->n[0][0], m->n[0][1], m->n[0][2]);
    if (e == cudaSuccess)
      e = cudaMalloc(&m->partials, (rb > RED_BLOCKS ? rb : RED_BLOCKS) * sizeof(double));
  }
  if (e == cudaSuccess) e = cudaMalloc(&m->scal, 8 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&m->ctl, sizeof(MGCtl));
  if (e == cudaSuccess) e = cudaMemset(m->ctl, 0, sizeof(MGCtl));
  m->stop = (int*)m->ctl;
  // the potential is the warm start of the first solve: zero, not whatever the allocator held
  if (e == cudaSuccess) e = cudaMemset(m->phi, 0, 2 * m->cells[0] * sizeof(float));
  return e;
}

void mg_setup_host(dh_ctx* c) {
  MG* m = c->mg;
  const int l = m->L - 1;
  const int n0 = m->n[l][0], n1 = m->n[l][1], n2 = m->n[l][2];
  const double h = m->h[l];
  const long long N = m->cells[l];
  std::vector<double> G(N, 0.0);
  for (int d2 = 0; d2 < n2; ++d2)
    for (int d1 = 0; d1 < n1; ++d1)
      for (int d0 = 0; d0 < n0; ++d0) {
        double s = 0.0;
        for (int k2 = 0; k2 < n2; ++k2)
          for (int k1 = 0; k1 < n1; ++k1)
            for (int k0 = 0; k0 < n0; ++k0) {
              if (k0 == 0 && k1 == 0 && k2 == 0) continue;
              const double s0 = std::sin(M_PI * k0 / n0), s1 = std::sin(M_PI * k1 / n1),
                           s2 = std::sin(M_PI * k2 / n2);
              const double lam = -(4.0 / (h * h)) * (s0 * s0 + s1 * s1 + s2 * s2);
              const double ph = 2.0 * M_PI * ((double)k0 * d0 / n0 + (double)k1 * d1 / n1 +
                                              (double)k2 * d2 / n2);
              s += std::cos(ph) / lam;
            }
        G[((long long)d2 * n1 + d1) * n0 + d0] = s / (double)N;
      }
  cudaMemcpy(m->G, G.data(), N * sizeof(double), cudaMemcpyHostToDevice);
}

cudaError_t mg_reset(dh_ctx* c) {
  MG* m = c->mg;
  m->last_cycles = 0;
  m->last_res = 0.0;
  return cudaMemsetAsync(m->phi, 0, 2 * m->cells[0] * sizeof(float), c->stream);
}

void* mg_phi(dh_ctx* c) { return c->mg ? c->mg->phi : nullptr; }

void mg_last(const dh_ctx* c, int* cycles, double* rel_residual) {
  *cycles = c->mg ? c->mg->last_cycles : 0;
  *rel_residual = c->mg ? c->mg->last_res : 0.0;
}

void mg_free(dh_ctx* c) {
  MG* m = c->mg;
  if (!m) return;
  cudaFree(m->phi);
  cudaFree(m->phi2);
  cudaFree(m->F);
  for (int l = 0; l < MG_LMAX; ++l) {
    cudaFree(m->e[l]); cudaFree(m->e2[l]); cudaFree(m->r[l]);
    cudaFree(m->de[l]); cudaFree(m->de2[l]); cudaFree(m->dr[l]);
  }
  cudaFree(m->G);
  cudaFree(m->partials);
  cudaFree(m->scal);
  cudaFree(m->ctl);
  if (m->cycle_exec) cudaGraphExecDestroy(m->cycle_exec);
  delete m;
  c->mg = nullptr;
}

// ---------------------------------------------------------------------------------------------
// Deterministic float64 reductions: per-block partials in a fixed order, then one block.
__device__ __forceinline__ double block_sum(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  return red[0];
}

__device__ __forceinline__ void block_range(long long n, long long& b0, long long& b1) {
  const long long per = (n + gridDim.x - 1) / gridDim.x;
  b0 = blockIdx.x * per;
  b1 = b0 + per < n ? b0 + per : n;
}

// out = scale * sum(partials), launched as one block of FIN_THREADS: thread t adds entries
// t, t + FIN_THREADS, ..., then a fixed shuffle tree per warp and a fixed sum of the warps (the
// order, and so the result, does not depend on scheduling)
constexpr int FIN_THREADS = 1024;
__global__ void __launch_bounds__(FIN_THREADS)
finalize_kernel(const double* partials, int nb, double* out, double scale, const int* stop = nullptr) {
  if (stop && *stop) return;
  __shared__ double wsum[FIN_THREADS / 32];
  const int t = threadIdx.x;
  double s = 0.0;
  for (int b = t; b < nb; b += FIN_THREADS) s += partials[b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((t & 31) == 0) wsum[t >> 5] = s;
  __syncthreads();
  if (t == 0) {
    double a = 0.0;
    for (int w = 0; w < FIN_THREADS / 32; ++w) a += wsum[w];
    *out = scale * a;
  }
}

template <typename T>
__global__ void sum_partial_kernel(const T* __restrict__ x, long long n, double* partials);

// float32 data: compensated float32 per thread (no float64 arithmetic per cell)
template <>
__global__ void sum_partial_kernel<float>(const float* __restrict__ x, long long n, double* partials) {
  __shared__ double red[RED_THREADS];
  long long b0, b1;
  block_range(n, b0, b1);
  ff2 acc{0.0f, 0.0f};
  for (long long i = b0 + threadIdx.x; i < b1; i += blockDim.x) ff_acc(acc, x[i]);
  const double s = block_sum(ff_to_double(acc), red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

template <>
__global__ void sum_partial_kernel<double>(const double* __restrict__ x, long long n, double* partials) {
  __shared__ double red[RED_THREADS];
  long long b0, b1;
  block_range(n, b0, b1);
  double s = 0.0;
  for (long long i = b0 + threadIdx.x; i < b1; i += blockDim.x) s += x[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// F = four_pi_G (rho - <rho>) in float-float, the mean and the factor carried as float-float;
// partials of |F|^2.
template <typename T>
__global__ void poisson_source_kernel(const T* __restrict__ rho, long long n, const double* mean,
                                      double four_pi_G, float* __restrict__ F, double* partials) {
  __shared__ double red[RED_THREADS];
  const ff2 mneg = ff_neg(ff_from_double(*mean));
  const ff2 fpg = ff_from_double(four_pi_G);
  ff2 acc{0.0f, 0.0f};
  // cells q0 + u * stride, u < 4, per pass: four independent loads in flight per thread
  const long long stride = (long long)gridDim.x * RED_THREADS;
  for (long long q0 = blockIdx.x * (long long)RED_THREADS + threadIdx.x; q0 < n; q0 += 4 * stride) {
    T v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = q0 + u * stride < n ? rho[q0 + u * stride] : T(0);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const long long q = q0 + u * stride;
      if (q < n) {
        const ff2 f = ff_mul(ff_add(ff_from(v[u]), mneg), fpg);
        ff_store(F, n, q, f);
        ff_acc(acc, f.hi * f.hi);
      }
    }
  }
  const double s = block_sum(ff_to_double(acc), red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}



// One red-black Gauss-Seidel sweep on A e = r in one pass, from e_old into e_new: first every
// red cell (i + j + k even), then every black cell, each e_i = (sum of 6 neighbours - h^2 r_i)/6.
// Every neighbour of a cell has the other colour, so the red update reads only old black values
// and the black update only new red values: the result is that of two colour passes in place,
// value for value.  A CTA owns a 32 x 8 column of cells and a run of planes [z0, z1); it marches
// p = z0-1 .. z1, computing red on plane p over the tile and a one-cell halo (from old values on
// the tile and a two-cell halo, planes p-1..p+1), then black on plane p-1 over the tile from the
// red planes p-2..p, and writes plane p-1 (both colours).  The halo's red values are recomputed
// by each CTA that needs them, so CTAs never wait on one another; the periodic wrap in z is just
// the march's first and last red planes.  Old e and r arrive by cp.async SW_D planes ahead.
constexpr int SW_TX = 32, SW_TY = 8;                  // tile (one thread per cell of a plane)
constexpr int SW_EX = SW_TX + 4, SW_EY = SW_TY + 4;   // old e: tile + 2-cell halo
constexpr int SW_RX = SW_TX + 2, SW_RY = SW_TY + 2;   // new red e and r: tile + 1-cell halo
constexpr int SW_E = SW_EX * SW_EY, SW_R = SW_RX * SW_RY;
constexpr int SW_ZC = 64;                              // planes per CTA
constexpr int SW_D = 3;                                // copy groups in flight
constexpr int SW_RING = 6;                             // >= 3 + SW_D old-e and 2 + SW_D r slots

template <bool ZERO>   // ZERO: e_old = 0 (the first sweep of a V-cycle level; e_old unread)
__global__ void __launch_bounds__(256, 8)
rbgs_sweep_kernel(const float* __restrict__ eo, float* __restrict__ en, const float* __restrict__ r,
                  int nx, int ny, int nz, float h2, const int* __restrict__ stop) {
  if (*stop) return;  // the solve has finished: the rest of its batch does nothing
  __shared__ float s_eo[ZERO ? 1 : SW_RING][SW_E];
  __shared__ float s_r[SW_RING][SW_R];
  __shared__ float s_red[3][SW_R];
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * SW_TX, y0 = blockIdx.y * SW_TY;   // both even
  const int z0 = blockIdx.z * SW_ZC;
  const int z1 = z0 + SW_ZC < nz ? z0 + SW_ZC : nz;
  const int nit = z1 - z0 + 2;   // iterations ip = 0 .. nit - 1 (p = z0 - 1 + ip)
  const long long plane = (long long)nx * ny;
  // Global offsets within a plane of this thread's (up to) two halo positions; positions past
  // the halo of the grid's last cells (tiles larger than the grid) read cell 0 and are unused.
  int eoff[2], roff[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int pe = tid + 256 * u;
    const int ex = x0 - 2 + pe % SW_EX, ey = y0 - 2 + pe / SW_EX;
    eoff[u] = (pe < SW_E && ex < nx + 2 && ey < ny + 2) ? wrap(ey, ny) * nx + wrap(ex, nx) : 0;
    const int rx = x0 - 1 + pe % SW_RX, ry = y0 - 1 + pe / SW_RX;
    roff[u] = (pe < SW_R && rx < nx + 1 && ry < ny + 1) ? wrap(ry, ny) * nx + wrap(rx, nx) : 0;
  }
  const bool e2nd = tid + 256 < SW_E, r2nd = tid + 256 < SW_R;
  // Old-e plane z0 - 2 + m lives in s_eo[m % SW_RING]; r plane z0 - 1 + m in s_r[m % SW_RING].
  auto copy_eo = [&](int m) {
    const float* b = eo + (long long)wrap(z0 - 2 + m, nz) * plane;
    float* d = s_eo[ZERO ? 0 : m % SW_RING];
    cp_async4(d + tid, b + eoff[0]);
    if (e2nd) cp_async4(d + tid + 256, b + eoff[1]);
  };
  // group m (m = 0 .. nit - 1): old-e plane z0 + m and r plane z0 - 1 + m
  auto issue_group = [&](int m) {
    if (m < nit) {
      if (!ZERO) copy_eo(m + 2);
      const float* b = r + (long long)wrap(z0 - 1 + m, nz) * plane;
      float* d = s_r[m % SW_RING];
      cp_async4(d + tid, b + roff[0]);
      if (r2nd) cp_async4(d + tid + 256, b + roff[1]);
    }
    cp_async_commit();   // empty groups keep the count uniform
  };
  // Red cells of the tile + 1 halo: SW_RY rows of SW_RX / 2; thread t < SW_R / 2 takes one.  The
  // cell (x0 - 1 + rx, y0 - 1 + ry, p) is red when rx + ry + p is even (x0, y0 even, n even).
  const bool has_red = tid < SW_R / 2;
  const int ry = has_red ? tid / (SW_RX / 2) : 0, kk = has_red ? tid % (SW_RX / 2) : 0;
  const int rx_even = 2 * kk + (ry & 1), rx_odd = 2 * kk + ((ry + 1) & 1);
  // this thread's cell of the tile
  const int tx = tid & (SW_TX - 1), ty = tid / SW_TX;
  const int cb = (ty + 1) * SW_RX + tx + 1;
  const bool writes = x0 + tx < nx && y0 + ty < ny;
  float* out = en + (long long)(y0 + ty) * nx + (x0 + tx);

  if (!ZERO) {
    copy_eo(0);
    copy_eo(1);
  }
#pragma unroll
  for (int m = 0; m < SW_D; ++m) issue_group(m);   // the first group also carries e planes 0, 1
  int s3 = 0;   // ip % 3: slot of the red plane p
  for (int ip = 0; ip < nit; ++ip) {
    const int p = z0 - 1 + ip;
    issue_group(ip + SW_D);
    cp_async_wait<SW_D>();   // groups 0 .. ip have landed (this thread's copies)
    __syncthreads();
    const int s3p = s3 == 2 ? 0 : s3 + 1, s3m = s3 == 0 ? 2 : s3 - 1;
    // red on plane p over the tile + 1 halo
    if (has_red) {
      const int rx = (p & 1) ? rx_odd : rx_even;
      const int c = ry * SW_RX + rx;
      float nb = 0.f;
      if (!ZERO) {
        const float* em = s_eo[ip % SW_RING];
        const float* ec = s_eo[(ip + 1) % SW_RING];
        const float* ep = s_eo[(ip + 2) % SW_RING];
        const int e = (ry + 1) * SW_EX + rx + 1;
        nb = em[e] + ep[e] + ec[e - SW_EX] + ec[e + SW_EX] + ec[e - 1] + ec[e + 1];
      }
      s_red[s3][c] = (nb - h2 * s_r[ip % SW_RING][c]) * (1.0f / 6.0f);
    }
    __syncthreads();
    // black on plane p - 1 over the tile, and the write of plane p - 1
    if (ip >= 2) {
      const float* rm = s_red[s3p];   // plane p - 2 (the slot p + 1 will take)
      const float* rc = s_red[s3m];   // plane p - 1
      const float* rp = s_red[s3];    // plane p
      float v;
      if ((tx + ty + p - 1) & 1) {
        const float nb = rm[cb] + rp[cb] + rc[cb - SW_RX] + rc[cb + SW_RX] + rc[cb - 1] + rc[cb + 1];
        v = (nb - h2 * s_r[(ip - 1) % SW_RING][cb]) * (1.0f / 6.0f);
      } else {
        v = rc[cb];
      }
      if (writes) out[(long long)(p - 1) * plane] = v;
    }
    s3 = s3p;
  }
  cp_async_wait<0>();
}


// The same sweep for rows of a multiple of 4 cells, two cells per thread: a CTA owns a 64 x 8
// column; thread (t, y) takes the pair x0 + 2t, x0 + 2t + 1 of row y, which holds one red and
// one black cell.  Planes arrive as aligned float4 chunks covering x0 - 4 .. x0 + 67 (the red
// cells of x0 - 2 .. x0 + 65 and their black neighbours; with n_x a multiple of 4 no chunk
// straddles the periodic wrap), old e on rows y0 - 2 .. y0 + 9 and r on y0 - 1 .. y0 + 8.
constexpr int S4_TX = 64, S4_TY = 8, S4_W = 72;       // tile, smem row width (floats)
constexpr int S4_EROWS = S4_TY + 4, S4_RROWS = S4_TY + 2;
constexpr int S4_ECH = S4_EROWS * (S4_W / 4), S4_RCH = S4_RROWS * (S4_W / 4);   // float4 chunks
constexpr int S4_NRED = S4_RROWS * (S4_W / 2 - 2);   // red tasks: pairs x0 - 2 .. x0 + 65
// rings: old e in use for planes p-1..p+1 plus S4_D in flight; r in use for p-1 (black), p (red),
// S4_D in flight, and one more so that a copy never lands in the slot a slower thread's black
// step of the previous plane may still read
constexpr int S4_D = 2, S4_ERING = 3 + S4_D, S4_RRING = 3 + S4_D;

template <bool ZERO>
__global__ void __launch_bounds__(256)
rbgs_sweep4_kernel(const float* __restrict__ eo, float* __restrict__ en, const float* __restrict__ r,
                   int nx, int ny, int nz, float h2, const int* __restrict__ stop) {
  if (*stop) return;  // the solve has finished: the rest of its batch does nothing
  __shared__ __align__(16) float s_eo[ZERO ? 1 : S4_ERING][S4_EROWS * S4_W];
  __shared__ __align__(16) float s_r[S4_RRING][S4_RROWS * S4_W];
  __shared__ float s_red[3][S4_RROWS * S4_W];
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * S4_TX, y0 = blockIdx.y * S4_TY;
  const int z0 = blockIdx.z * SW_ZC;
  const int z1 = z0 + SW_ZC < nz ? z0 + SW_ZC : nz;
  const int nit = z1 - z0 + 2;
  const long long plane = (long long)nx * ny;
  // this thread's chunk of each plane: global offset within the plane and smem offset
  int eg = 0, es = 0, rg = 0, rs = 0;
  const bool ech = tid < S4_ECH, rch = tid < S4_RCH;
  {
    const int row = tid / (S4_W / 4), cc = tid % (S4_W / 4);
    const int gx = x0 - 4 + 4 * cc;
    const int wx = gx < nx + 4 ? wrap(gx, nx) : 0;   // chunks past the needed halo: unused
    const int gye = y0 - 2 + row, gyr = y0 - 1 + row;
    eg = (gye < ny + 2 ? wrap(gye, ny) : 0) * nx + wx;
    rg = (gyr < ny + 1 ? wrap(gyr, ny) : 0) * nx + wx;
    es = row * S4_W + 4 * cc;
    rs = es;
  }
  auto issue_group = [&](int m) {   // old-e plane z0 + m and r plane z0 - 1 + m
    if (m < nit) {
      if (!ZERO && ech)
        cp_async16(&s_eo[ZERO ? 0 : (m + 2) % S4_ERING][es],
                   eo + (long long)wrap(z0 + m, nz) * plane + eg);
      if (rch) cp_async16(&s_r[m % S4_RRING][rs], r + (long long)wrap(z0 - 1 + m, nz) * plane + rg);
    }
    cp_async_commit();
  };
  // this thread's pair
  const int t2 = tid % (S4_TX / 2), ty = tid / (S4_TX / 2);
  const bool writes = x0 + 2 * t2 < nx && y0 + ty < ny;
  float* out = en + (long long)(y0 + ty) * nx + (x0 + 2 * t2);

  if (!ZERO && ech) {
    for (int m = 0; m < 2; ++m)
      cp_async16(&s_eo[ZERO ? 0 : m][es], eo + (long long)wrap(z0 - 2 + m, nz) * plane + eg);
  }
#pragma unroll
  for (int m = 0; m < S4_D; ++m) issue_group(m);
  int s3 = 0;
  for (int ip = 0; ip < nit; ++ip) {
    const int p = z0 - 1 + ip;
    issue_group(ip + S4_D);
    cp_async_wait<S4_D>();
    __syncthreads();
    const int s3p = s3 == 2 ? 0 : s3 + 1, s3m = s3 == 0 ? 2 : s3 - 1;
    // red on plane p: pairs x0 - 2 + 2 pp (pp = 0 .. 33) of rows y0 - 1 .. y0 + 8
    {
      const float* rr = s_r[ip % S4_RRING];
      float* red = s_red[s3];
      for (int t = tid; t < S4_NRED; t += 256) {
        const int ry = t / (S4_W / 2 - 2), pp = t % (S4_W / 2 - 2);
        const int c = 2 + 2 * pp + ((ry + 1 + p) & 1);   // smem column (origin x0 - 4)
        float nb = 0.f;
        if (!ZERO) {
          const float* em = s_eo[ZERO ? 0 : ip % S4_ERING];
          const float* ec = s_eo[ZERO ? 0 : (ip + 1) % S4_ERING];
          const float* ep = s_eo[ZERO ? 0 : (ip + 2) % S4_ERING];
          const int e = (ry + 1) * S4_W + c;
          nb = em[e] + ep[e] + ec[e - S4_W] + ec[e + S4_W] + ec[e - 1] + ec[e + 1];
        }
        red[ry * S4_W + c] = (nb - h2 * rr[ry * S4_W + c]) * (1.0f / 6.0f);
      }
    }
    __syncthreads();
    // black on plane p - 1 (one cell of the pair), and the write of the pair
    if (ip >= 2) {
      const float* rm = s_red[s3p];
      const float* rc = s_red[s3m];
      const float* rp = s_red[s3];
      const int q = p - 1;
      const int b = (ty + q + 1) & 1;                     // black cell's offset in the pair
      const int c = (ty + 1) * S4_W + 4 + 2 * t2 + b;
      const float nb = rm[c] + rp[c] + rc[c - S4_W] + rc[c + S4_W] + rc[c - 1] + rc[c + 1];
      const float vb = (nb - h2 * s_r[(ip - 1) % S4_RRING][c]) * (1.0f / 6.0f);
      const float vr = rc[b ? c - 1 : c + 1];
      if (writes)
        *reinterpret_cast<float2*>(out + (long long)q * plane) = b ? make_float2(vr, vb) : make_float2(vb, vr);
    }
    s3 = s3p;
  }
  cp_async_wait<0>();
}

// Weighted Jacobi (Sec. 5.2) on A e = r from e_old into e_new: e_new = e + omega D^{-1} (r - A e)
// with D = -6/h^2, i.e. e_new = (1 - omega) e + (omega / 6) (sum of 6 neighbours - h^2 r).
// Rows of a multiple of 4 cells: a CTA owns a 64 x 8 column and a run of planes; old e arrives
// by 16-byte cp.async on the tile and a one-row halo (x0 - 4 .. x0 + 67), r on the tile, two
// planes ahead; each thread updates a pair of cells and stores a float2.
constexpr int J4_EROWS = S4_TY + 2, J4_ECH = J4_EROWS * (S4_W / 4);
constexpr int J4_RCH = S4_TY * (S4_TX / 4);
constexpr int J4_D = 2, J4_ERING = 4 + J4_D, J4_RRING = 2 + J4_D;   // no slot a slower thread
                                                                    // of the last plane reads

__global__ void __launch_bounds__(256)
jacobi4_kernel(const float* __restrict__ eo, float* __restrict__ en, const float* __restrict__ r,
               int nx, int ny, int nz, float h2, float omega, const int* __restrict__ stop) {
  if (*stop) return;  // the solve has finished: the rest of its batch does nothing
  __shared__ __align__(16) float s_e[J4_ERING][J4_EROWS * S4_W];
  __shared__ __align__(16) float s_r[J4_RRING][S4_TY * S4_TX];
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * S4_TX, y0 = blockIdx.y * S4_TY;
  const int z0 = blockIdx.z * SW_ZC;
  const int z1 = z0 + SW_ZC < nz ? z0 + SW_ZC : nz;
  const int nit = z1 - z0;
  const long long plane = (long long)nx * ny;
  int eg = 0, es = 0, rg = 0, rs = 0;
  const bool ech = tid < J4_ECH, rch = tid < J4_RCH;
  {
    const int row = tid / (S4_W / 4), cc = tid % (S4_W / 4);
    const int gx = x0 - 4 + 4 * cc, gy = y0 - 1 + row;
    const int wx = gx < nx + 4 ? wrap(gx, nx) : 0;
    eg = (gy < ny + 1 ? wrap(gy, ny) : 0) * nx + wx;
    es = row * S4_W + 4 * cc;
    const int rrow = tid / (S4_TX / 4), rc4 = tid % (S4_TX / 4);
    const int rgx = x0 + 4 * rc4, rgy = y0 + rrow;
    rg = (rgx < nx && rgy < ny) ? rgy * nx + rgx : 0;
    rs = rrow * S4_TX + 4 * rc4;
  }
  // e plane z0 - 1 + m in s_e[m % J4_ERING]; r plane z0 + m in s_r[m % J4_RRING]
  auto copy_e = [&](int m) {
    if (ech) cp_async16(&s_e[m % J4_ERING][es], eo + (long long)wrap(z0 - 1 + m, nz) * plane + eg);
  };
  auto issue_group = [&](int m) {   // e plane z0 + 1 + m and r plane z0 + m
    if (m < nit) {
      copy_e(m + 2);
      if (rch) cp_async16(&s_r[m % J4_RRING][rs], r + (long long)(z0 + m) * plane + rg);
    }
    cp_async_commit();
  };
  const int t2 = tid % (S4_TX / 2), ty = tid / (S4_TX / 2);
  const bool writes = x0 + 2 * t2 < nx && y0 + ty < ny;
  float* out = en + (long long)(y0 + ty) * nx + (x0 + 2 * t2);
  const float cw = 1.0f - omega, cn = omega * (1.0f / 6.0f);
  copy_e(0);
  copy_e(1);
#pragma unroll
  for (int m = 0; m < J4_D; ++m) issue_group(m);
  for (int it = 0; it < nit; ++it) {
    issue_group(it + J4_D);
    cp_async_wait<J4_D>();
    __syncthreads();
    const float* em = s_e[it % J4_ERING];
    const float* ec = s_e[(it + 1) % J4_ERING];
    const float* ep = s_e[(it + 2) % J4_ERING];
    const float* rr = s_r[it % J4_RRING];
    const int c = (ty + 1) * S4_W + 4 + 2 * t2;   // the pair's first cell
    float v[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int cu = c + u;
      const float nb = em[cu] + ep[cu] + ec[cu - S4_W] + ec[cu + S4_W] + ec[cu - 1] + ec[cu + 1];
      v[u] = cw * ec[cu] + cn * (nb - h2 * rr[ty * S4_TX + 2 * t2 + u]);
    }
    if (writes) *reinterpret_cast<float2*>(out + (long long)(z0 + it) * plane) = make_float2(v[0], v[1]);
  }
  cp_async_wait<0>();
}

// The same for any row length, one cell per thread from global memory.
__global__ void jacobi_kernel(const float* __restrict__ eo, float* __restrict__ en,
                              const float* __restrict__ r, int nx, int ny, int nz, float h2,
                              float omega, const int* __restrict__ stop) {
  if (*stop) return;  // the solve has finished: the rest of its batch does nothing
  const long long n = (long long)nx * ny * nz;
  const float cw = 1.0f - omega, cn = omega * (1.0f / 6.0f);
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const unsigned t = (unsigned)q / (unsigned)nx;
    const int i = (int)((unsigned)q - t * (unsigned)nx);
    const int k = (int)(t / (unsigned)ny);
    const int j = (int)(t - (unsigned)k * (unsigned)ny);
    const long long row = (long long)k * ny;
    const float nb = eo[((long long)wrap(k - 1, nz) * ny + j) * nx + i] +
                     eo[((long long)wrap(k + 1, nz) * ny + j) * nx + i] +
                     eo[(row + wrap(j - 1, ny)) * nx + i] + eo[(row + wrap(j + 1, ny)) * nx + i] +
                     eo[(row + j) * nx + wrap(i - 1, nx)] + eo[(row + j) * nx + wrap(i + 1, nx)];
    en[q] = cw * eo[q] + cn * (nb - h2 * r[q]);
  }
}

// The first Jacobi sweep of a level from e = 0: e_new = -(omega h^2 / 6) r.
__global__ void jacobi_zero_kernel(float* __restrict__ en, const float* __restrict__ r,
                                   long long n, float s, const int* __restrict__ stop) {
  if (*stop) return;  // the solve has finished: the rest of its batch does nothing
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x)
    en[q] = s * r[q];
}

// r = F - A phi as a z-march, with the correction of the previous cycle applied on the way
// (UPDATE): phi' = phi + e (float-float), r = F - A phi' (stored as the float32 right-hand side
// of the next correction), and partials of |r / rms(F)|^2 with rms(F) = sqrt(fnorm2 / n); phi'
// goes to a second buffer (neighbouring CTAs still read phi).  A CTA owns a 32 x 8 column and
// RZ_ZC planes; phi (both words) and e arrive by cp.async on the tile and a one-cell halo, two
// planes ahead; each landed plane is updated in shared memory once.  h^2 A phi is the neighbour
// sum minus 6 phi: the hi words go through a TwoSum chain (exact), the lo words, the chain's
// rounding errors and the exact error of 6 phi_hi through float32, an absolute error of a few
// eps32^2 times sum |phi| -- far below what a relative residual of 1e-6 needs at any N this
// part holds.

template <bool UPDATE>
__global__ void __launch_bounds__(256)
residual_zm_kernel(const float* __restrict__ phi, float* __restrict__ phi_out,
                   const float* __restrict__ e, const float* __restrict__ F,
                   float* __restrict__ r32, int nx, int ny, int nz, ff2 h2, float ih2,
                   const double* fnorm2, double* partials, const int* __restrict__ stop) {
  if (*stop) return;  // the solve has finished: the rest of its batch does nothing
  __shared__ float s_hi[RZ_RING][RZ_H];
  __shared__ float s_lo[RZ_RING][RZ_H];
  __shared__ float s_e[UPDATE ? RZ_RING : 1][RZ_H];
  __shared__ double red[256];
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * RZ_TX, y0 = blockIdx.y * RZ_TY, z0 = blockIdx.z * RZ_ZC;
  const int z1 = z0 + RZ_ZC < nz ? z0 + RZ_ZC : nz;
  const int nit = z1 - z0;
  const long long plane = (long long)nx * ny;
  const long long n = plane * nz;
  const float* __restrict__ phl = phi + n;
  const float sF = (float)(1.0 / sqrt(*fnorm2 / (double)n));
  // this thread's (up to) two halo positions: offsets within a plane (cell 0 past the halo)
  int hoff[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int pe = tid + 256 * u;
    const int hx = x0 - 1 + pe % RZ_HX, hy = y0 - 1 + pe / RZ_HX;
    hoff[u] = (pe < RZ_H && hx < nx + 1 && hy < ny + 1) ? wrap(hy, ny) * nx + wrap(hx, nx) : 0;
  }
  const bool h2nd = tid + 256 < RZ_H;
  // plane z0 - 1 + m lives in slot m % RZ_RING
  auto copy_plane = [&](int m) {
    const long long b = (long long)wrap(z0 - 1 + m, nz) * plane;
    const int sl = m % RZ_RING;
    cp_async4(&s_hi[sl][tid], phi + b + hoff[0]);
    cp_async4(&s_lo[sl][tid], phl + b + hoff[0]);
    if (UPDATE) cp_async4(&s_e[UPDATE ? sl : 0][tid], e + b + hoff[0]);
    if (h2nd) {
      cp_async4(&s_hi[sl][tid + 256], phi + b + hoff[1]);
      cp_async4(&s_lo[sl][tid + 256], phl + b + hoff[1]);
      if (UPDATE) cp_async4(&s_e[UPDATE ? sl : 0][tid + 256], e + b + hoff[1]);
    }
  };
  auto issue_group = [&](int g) {   // group g carries plane index g + 2
    if (g < nit) copy_plane(g + 2);
    cp_async_commit();
  };
  auto update_plane = [&](int m) {  // phi' = phi + e in place, this thread's positions
    const int sl = m % RZ_RING;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int pe = tid + 256 * u;
      if (pe < RZ_H) {
        const ff2 v = ff_add_f(ff2{s_hi[sl][pe], s_lo[sl][pe]}, s_e[UPDATE ? sl : 0][pe]);
        s_hi[sl][pe] = v.hi;
        s_lo[sl][pe] = v.lo;
      }
    }
  };
  const int tx = tid % RZ_TX, ty = tid / RZ_TX;
  const int x = x0 + tx, y = y0 + ty;
  const bool active = x < nx && y < ny;
  const int c = (ty + 1) * RZ_HX + tx + 1;
  copy_plane(0);
  copy_plane(1);
#pragma unroll
  for (int g = 0; g < RZ_D; ++g) issue_group(g);
  ff2 acc{0.0f, 0.0f};
  for (int it = 0; it < nit; ++it) {
    const long long q = (long long)(z0 + it) * plane + (long long)y * nx + x;
    float fhi = 0.f, flo = 0.f;
    if (active) { fhi = F[q]; flo = F[n + q]; }
    issue_group(it + RZ_D);
    cp_async_wait<RZ_D>();
    __syncthreads();
    if (UPDATE) {
      if (it == 0) { update_plane(0); update_plane(1); }
      update_plane(it + 2);
      __syncthreads();
    }
    if (active) {
      const int sm = it % RZ_RING, sc = (it + 1) % RZ_RING, sp = (it + 2) % RZ_RING;
      const ff2 cv{s_hi[sc][c], s_lo[sc][c]};
      ff2 sum{__fmul_rn(-6.0f, cv.hi), 0.0f};
      const float err = __fmaf_rn(-6.0f, cv.hi, -sum.hi);
      float lo = __fmul_rn(-6.0f, cv.lo);
      ff_acc(sum, s_hi[sm][c]);      lo = __fadd_rn(lo, s_lo[sm][c]);
      ff_acc(sum, s_hi[sp][c]);      lo = __fadd_rn(lo, s_lo[sp][c]);
      ff_acc(sum, s_hi[sc][c - RZ_HX]); lo = __fadd_rn(lo, s_lo[sc][c - RZ_HX]);
      ff_acc(sum, s_hi[sc][c + RZ_HX]); lo = __fadd_rn(lo, s_lo[sc][c + RZ_HX]);
      ff_acc(sum, s_hi[sc][c - 1]);  lo = __fadd_rn(lo, s_lo[sc][c - 1]);
      ff_acc(sum, s_hi[sc][c + 1]);  lo = __fadd_rn(lo, s_lo[sc][c + 1]);
      const ff2 lap = ff_fast_two_sum(sum.hi, __fadd_rn(sum.lo, __fadd_rn(err, lo)));   // h^2 A phi
      const ff2 fh = ff_mul(ff2{fhi, flo}, h2);                                          // h^2 F
      const ff2 d = ff_two_sum(fh.hi, -lap.hi);
      const float rr = __fmul_rn(__fadd_rn(d.hi, __fadd_rn(d.lo, __fsub_rn(fh.lo, lap.lo))), ih2);
      r32[q] = rr;
      const float rs = rr * sF;
      ff_acc(acc, rs * rs);
      if (UPDATE) {
        phi_out[q] = cv.hi;
        phi_out[n + q] = cv.lo;
      }
    }
  }
  cp_async_wait<0>();
  red[tid] = ff_to_double(acc);
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (tid < w) red[tid] += red[tid + w];
    __syncthreads();
  }
  if (tid == 0)
    partials[((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = red[0];
}

// The same residual for two cells per thread, 32 apart in x, on rows of whole 64-cell
// multiples: a CTA owns a 64 x 8 column, and the float-float Laplacian and residual run as packed
// FP32x2 pairs with the scalar kernel's operations per lane (so r matches it cell for cell; the
// norm's partial sums are grouped per CTA of this kernel, in a fixed order).
constexpr int RP_QX = 32, RP_HX = 2 * RP_QX + 2, RP_H = RP_HX * RZ_HY;
static_assert(RP_H <= 3 * 256, "three halo positions per thread");
inline long long residual_pair_blocks(int nx, int ny, int nz) {
  return (long long)(nx / (2 * RP_QX)) * ((ny + RZ_TY - 1) / RZ_TY) * ((nz + RZ_ZC - 1) / RZ_ZC);
}

struct ffp {
  float2 hi, lo;
};
__device__ __forceinline__ ffp ffp_two_sum(float2 a, float2 b) {
  const float2 s = padd(a, b);
  const float2 bb = psub(s, a);
  return ffp{s, padd(psub(a, psub(s, bb)), psub(b, bb))};
}
__device__ __forceinline__ ffp ffp_fast_two_sum(float2 a, float2 b) {   // |a| >= |b| per lane
  const float2 s = padd(a, b);
  return ffp{s, psub(b, psub(s, a))};
}
__device__ __forceinline__ void ffp_acc(ffp& acc, float2 x) {
  const ffp t = ffp_two_sum(acc.hi, x);
  acc.hi = t.hi;
  acc.lo = padd(acc.lo, t.lo);
}

template <bool UPDATE>
__global__ void __launch_bounds__(256)
residual_zm_pair_kernel(const float* __restrict__ phi, float* __restrict__ phi_out,
                        const float* __restrict__ e, const float* __restrict__ F,
                        float* __restrict__ r32, int nx, int ny, int nz, ff2 h2, float ih2,
                        const double* fnorm2, double* partials, const int* __restrict__ stop) {
  if (*stop) return;  // the solve has finished: the rest of its batch does nothing
  __shared__ float s_hi[RZ_RING][RP_H];
  __shared__ float s_lo[RZ_RING][RP_H];
  __shared__ float s_e[UPDATE ? RZ_RING : 1][RP_H];
  __shared__ double red[8];
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * (2 * RP_QX), y0 = blockIdx.y * RZ_TY, z0 = blockIdx.z * RZ_ZC;
  const int z1 = z0 + RZ_ZC < nz ? z0 + RZ_ZC : nz;
  const int nit = z1 - z0;
  const long long plane = (long long)nx * ny;
  const long long n = plane * nz;
  const float* __restrict__ phl = phi + n;
  const float sF = (float)(1.0 / sqrt(*fnorm2 / (double)n));
  // this thread's (up to) three halo positions: offsets within a plane
  int hoff[3];
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    const int pe = tid + 256 * u;
    const int hx = x0 - 1 + pe % RP_HX, hy = y0 - 1 + pe / RP_HX;
    hoff[u] = (pe < RP_H && hy < ny + 1) ? wrap(hy, ny) * nx + wrap(hx, nx) : 0;
  }
  // plane z0 - 1 + m lives in slot m % RZ_RING
  auto copy_plane = [&](int m) {
    const long long b = (long long)wrap(z0 - 1 + m, nz) * plane;
    const int sl = m % RZ_RING;
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const int pe = tid + 256 * u;
      if (pe < RP_H) {
        cp_async4(&s_hi[sl][pe], phi + b + hoff[u]);
        cp_async4(&s_lo[sl][pe], phl + b + hoff[u]);
        if (UPDATE) cp_async4(&s_e[UPDATE ? sl : 0][pe], e + b + hoff[u]);
      }
    }
  };
  auto issue_group = [&](int g) {   // group g carries plane index g + 2
    if (g < nit) copy_plane(g + 2);
    cp_async_commit();
  };
  auto update_plane = [&](int m) {  // phi' = phi + e in place, this thread's positions
    const int sl = m % RZ_RING;
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const int pe = tid + 256 * u;
      if (pe < RP_H) {
        const ff2 v = ff_add_f(ff2{s_hi[sl][pe], s_lo[sl][pe]}, s_e[UPDATE ? sl : 0][pe]);
        s_hi[sl][pe] = v.hi;
        s_lo[sl][pe] = v.lo;
      }
    }
  };
  const int tx = tid % RP_QX, ty = tid / RP_QX;
  const int x = x0 + tx, y = y0 + ty;
  const bool active = y < ny;
  const int c = (ty + 1) * RP_HX + tx + 1, cb = c + RP_QX;
  const float2 m6 = pset(-6.0f), h2hi = pset(h2.hi), h2lo = pset(h2.lo), pih2 = pset(ih2);
  copy_plane(0);
  copy_plane(1);
#pragma unroll
  for (int g = 0; g < RZ_D; ++g) issue_group(g);
  ff2 acc{0.0f, 0.0f};
  for (int it = 0; it < nit; ++it) {
    const long long q = (long long)(z0 + it) * plane + (long long)y * nx + x;
    float2 fhi = pset(0.f), flo = pset(0.f);
    if (active) {
      fhi = pmk(F[q], F[q + RP_QX]);
      flo = pmk(F[n + q], F[n + q + RP_QX]);
    }
    issue_group(it + RZ_D);
    cp_async_wait<RZ_D>();
    __syncthreads();
    if (UPDATE) {
      if (it == 0) { update_plane(0); update_plane(1); }
      update_plane(it + 2);
      __syncthreads();
    }
    if (active) {
      const int sm = it % RZ_RING, sc = (it + 1) % RZ_RING, sp = (it + 2) % RZ_RING;
      auto hi2 = [&](int sl, int o) { return pmk(s_hi[sl][c + o], s_hi[sl][cb + o]); };
      auto lo2 = [&](int sl, int o) { return pmk(s_lo[sl][c + o], s_lo[sl][cb + o]); };
      const float2 cvh = hi2(sc, 0), cvl = lo2(sc, 0);
      ffp sum{pmul(m6, cvh), pset(0.0f)};
      const float2 err = pfma(m6, cvh, pneg(sum.hi));
      float2 lo = pmul(m6, cvl);
      ffp_acc(sum, hi2(sm, 0));      lo = padd(lo, lo2(sm, 0));
      ffp_acc(sum, hi2(sp, 0));      lo = padd(lo, lo2(sp, 0));
      ffp_acc(sum, hi2(sc, -RP_HX)); lo = padd(lo, lo2(sc, -RP_HX));
      ffp_acc(sum, hi2(sc, RP_HX));  lo = padd(lo, lo2(sc, RP_HX));
      ffp_acc(sum, hi2(sc, -1));     lo = padd(lo, lo2(sc, -1));
      ffp_acc(sum, hi2(sc, 1));      lo = padd(lo, lo2(sc, 1));
      const ffp lap = ffp_fast_two_sum(sum.hi, padd(sum.lo, padd(err, lo)));   // h^2 A phi
      // h^2 F (ff_mul with both words)
      const float2 pr = pmul(fhi, h2hi);
      float2 pe = pfma(fhi, h2hi, pneg(pr));
      pe = pfma(fhi, h2lo, pe);
      pe = pfma(flo, h2hi, pe);
      const ffp fh = ffp_fast_two_sum(pr, pe);
      const ffp d = ffp_two_sum(fh.hi, pneg(lap.hi));
      const float2 rr = pmul(padd(d.hi, padd(d.lo, psub(fh.lo, lap.lo))), pih2);
      r32[q] = rr.x;
      r32[q + RP_QX] = rr.y;
      const float ra = rr.x * sF, rb = rr.y * sF;
      ff_acc(acc, ra * ra);
      ff_acc(acc, rb * rb);
      if (UPDATE) {
        phi_out[q] = cvh.x;
        phi_out[q + RP_QX] = cvh.y;
        phi_out[n + q] = cvl.x;
        phi_out[n + q + RP_QX] = cvl.y;
      }
    }
  }
  cp_async_wait<0>();
  // fixed-order block sum: each warp by shuffles, then the eight warp sums in order
  double v = ff_to_double(acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  if (tid == 0) {
    double t = red[0];
    for (int w = 1; w < 8; ++w) t += red[w];
    partials[((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = t;
  }
}

// rc[I] = mean over the 8 children of (r - A e), coarse dims (cx, cy, cz).  One thread per coarse
// cell.  Over a 2x2x2 block the children's Laplacians sum to the 24 faces of the block:
// sum_children h^2 (A e)_child = (sum of the 24 outside neighbours) - 3 (sum of the 8 children),
// since every interior face cancels.  Rows of the fine grid are read as float2 pairs (x even).
__global__ void resid_restrict_kernel(const float* __restrict__ e, const float* __restrict__ r,
                                      float* __restrict__ rc, int cx, int cy, int cz, float ih2, const int* __restrict__ stop) {
  if (*stop) return;  // the solve has finished: the rest of its batch does nothing
  const int nx = 2 * cx, ny = 2 * cy, nz = 2 * cz;
  const long long nc = (long long)cx * cy * cz;
  const long long plane = (long long)nx * ny;
#pragma unroll 2
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nc;
       t += (long long)gridDim.x * blockDim.x) {
    const unsigned u = (unsigned)t / (unsigned)cx;
    const int I = (int)((unsigned)t - u * (unsigned)cx);
    const int K = (int)(u / (unsigned)cy);
    const int J = (int)(u - (unsigned)K * (unsigned)cy);
    const int i0 = 2 * I, j0 = 2 * J, k0 = 2 * K;
    const int im = wrap(i0 - 1, nx), ip = wrap(i0 + 2, nx);
    const int jm = wrap(j0 - 1, ny), jp = wrap(j0 + 2, ny);
    const int km = wrap(k0 - 1, nz), kp = wrap(k0 + 2, nz);
    auto row = [&](int j, int k) { return (long long)k * plane + (long long)j * nx; };
    float inside = 0.f, outside = 0.f, rs = 0.f;
#pragma unroll
    for (int dk = 0; dk < 2; ++dk)
#pragma unroll
      for (int dj = 0; dj < 2; ++dj) {
        const long long rw = row(j0 + dj, k0 + dk);
        const float2 ev = *reinterpret_cast<const float2*>(e + rw + i0);
        const float2 rv = *reinterpret_cast<const float2*>(r + rw + i0);
        inside += ev.x + ev.y;
        rs += rv.x + rv.y;
        outside += e[rw + im] + e[rw + ip];                              // x faces
      }
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      const float2 ym = *reinterpret_cast<const float2*>(e + row(jm, k0 + d) + i0);   // y faces
      const float2 yp = *reinterpret_cast<const float2*>(e + row(jp, k0 + d) + i0);
      const float2 zm = *reinterpret_cast<const float2*>(e + row(j0 + d, km) + i0);   // z faces
      const float2 zp = *reinterpret_cast<const float2*>(e + row(j0 + d, kp) + i0);
      outside += (ym.x + ym.y) + (yp.x + yp.y) + (zm.x + zm.y) + (zp.x + zp.y);
    }
    rc[t] = 0.125f * (rs - (outside - 3.0f * inside) * ih2);
  }
}

// e_fine += P e_coarse: per axis 3/4 of the parent and 1/4 of the parent's neighbour on the
// fine cell's side (weights (27, 9, 9, 9, 3, 3, 3, 1)/64), periodic.  One thread per coarse
// cell: its 27-neighbourhood, combined axis by axis, gives its 8 children (stored as float2
// pairs along x).
__global__ void prolong_add_kernel(float* __restrict__ ef, const float* __restrict__ ec, int cx,
                                   int cy, int cz, const int* __restrict__ stop) {
  if (*stop) return;  // the solve has finished: the rest of its batch does nothing
  const int nx = 2 * cx, ny = 2 * cy;
  const long long nc = (long long)cx * cy * cz;
  const long long plane = (long long)nx * ny;
#pragma unroll 2
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nc;
       t += (long long)gridDim.x * blockDim.x) {
    const unsigned u = (unsigned)t / (unsigned)cx;
    const int I = (int)((unsigned)t - u * (unsigned)cx);
    const int K = (int)(u / (unsigned)cy);
    const int J = (int)(u - (unsigned)K * (unsigned)cy);
    const int Is[3] = {wrap(I - 1, cx), I, wrap(I + 1, cx)};
    const int Js[3] = {wrap(J - 1, cy), J, wrap(J + 1, cy)};
    const int Ks[3] = {wrap(K - 1, cz), K, wrap(K + 1, cz)};
    // along x: X[d][b][c] = 3/4 parent + 1/4 neighbour on side d (d = 0: -1, d = 1: +1)
    float X[2][3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const float* rowp = ec + ((long long)Ks[c] * cy + Js[b]) * cx;
        const float m0 = rowp[Is[0]], m1 = rowp[Is[1]], m2 = rowp[Is[2]];
        X[0][b][c] = 0.75f * m1 + 0.25f * m0;
        X[1][b][c] = 0.75f * m1 + 0.25f * m2;
      }
#pragma unroll
    for (int dk = 0; dk < 2; ++dk)
#pragma unroll
      for (int dj = 0; dj < 2; ++dj) {
        float v[2];
#pragma unroll
        for (int di = 0; di < 2; ++di) {
          float Y[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) Y[c] = 0.75f * X[di][1][c] + 0.25f * X[di][dj == 0 ? 0 : 2][c];
          v[di] = 0.75f * Y[1] + 0.25f * Y[dk == 0 ? 0 : 2];
        }
        float2* dst = reinterpret_cast<float2*>(ef + (long long)(2 * K + dk) * plane +
                                                (long long)(2 * J + dj) * nx + 2 * I);
        float2 w = *dst;
        w.x += v[0];
        w.y += v[1];
        *dst = w;
      }
  }
}

__global__ void coarse_solve_kernel(const float* __restrict__ r, float* __restrict__ e,
                                    const double* __restrict__ G, int n0, int n1, int n2, const int* __restrict__ stop) {
  if (*stop) return;  // the solve has finished: the rest of its batch does nothing
  const int N = n0 * n1 * n2;
  for (int p = threadIdx.x; p < N; p += blockDim.x) {
    const int p0 = p % n0, p1 = (p / n0) % n1, p2 = p / (n0 * n1);
    double s = 0.0;
    for (int q = 0; q < N; ++q) {
      const int q0 = q % n0, q1 = (q / n0) % n1, q2 = q / (n0 * n1);
      const int d0 = wrap(p0 - q0, n0), d1 = wrap(p1 - q1, n1), d2 = wrap(p2 - q2, n2);
      s += G[(d2 * n1 + d1) * n0 + d0] * (double)r[q];
    }
    e[p] = (float)s;
  }
}

// ---------------------------------------------------------------------------------------------
// The float64 cycle of a float64 context.  Plain one-cell-per-thread kernels that take the
// oracle's steps in its order (Sec. 5.2; App. C): a red-black sweep is a red pass then a black
// pass in place, each cell (sum of its 6 neighbours - h^2 r) / 6 with the neighbours summed as
// (z-, z+), then (y-, y+), then (x-, x+); the Jacobi sweep e + omega (-h^2/6)(r - A e); the
// restriction the mean of the 8 children of r - A e; the prolongation interpolates along z,
// then y, then x (3/4 of the parent, 1/4 of its neighbour on the fine cell's side).  Such a
// context exists for parity (float64 arithmetic is scarce on this part), so these kernels are
// written for clarity, not speed.

__device__ __forceinline__ void cell_of(long long q, int nx, int ny, int& i, int& j, int& k) {
  const long long t = q / nx;
  i = (int)(q - t * nx);
  k = (int)(t / ny);
  j = (int)(t - (long long)k * ny);
}

// the oracle's neighbour sum: (z- + z+) + (y- + y+) + (x- + x+)
__device__ __forceinline__ double nb_sum_d(const double* __restrict__ e, int i, int j, int k,
                                           int nx, int ny, int nz) {
  const long long row = (long long)k * ny;
  const double z = e[((long long)wrap(k - 1, nz) * ny + j) * nx + i] +
                   e[((long long)wrap(k + 1, nz) * ny + j) * nx + i];
  const double y = e[(row + wrap(j - 1, ny)) * nx + i] + e[(row + wrap(j + 1, ny)) * nx + i];
  const double x = e[(row + j) * nx + wrap(i - 1, nx)] + e[(row + j) * nx + wrap(i + 1, nx)];
  return ((0.0 + z) + y) + x;
}

// A e at a cell as the oracle forms it: (-6 e + (z- + z+) + (y- + y+) + (x- + x+)) / h^2
__device__ __forceinline__ double apply_A_d(const double* __restrict__ e, int i, int j, int k,
                                            int nx, int ny, int nz, double hh) {
  const long long row = (long long)k * ny;
  double s = -6.0 * e[(row + j) * nx + i];
  s = s + e[((long long)wrap(k - 1, nz) * ny + j) * nx + i] + e[((long long)wrap(k + 1, nz) * ny + j) * nx + i];
  s = s + e[(row + wrap(j - 1, ny)) * nx + i] + e[(row + wrap(j + 1, ny)) * nx + i];
  s = s + e[(row + j) * nx + wrap(i - 1, nx)] + e[(row + j) * nx + wrap(i + 1, nx)];
  return s / hh;
}

// one colour pass in place: cells with (i + j + k) % 2 == colour
__global__ void rbgs_colour_d_kernel(double* __restrict__ e, const double* __restrict__ r, int nx,
                                     int ny, int nz, double hh, int colour, const int* __restrict__ stop) {
  if (*stop) return;  // the solve has finished: the rest of its batch does nothing
  const long long n = (long long)nx * ny * nz;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    cell_of(q, nx, ny, i, j, k);
    if (((i + j + k) & 1) != colour) continue;
    e[q] = (nb_sum_d(e, i, j, k, nx, ny, nz) - hh * r[q]) / 6.0;
  }
}

__global__ void jacobi_d_kernel(const double* __restrict__ eo, double* __restrict__ en,
                                const double* __restrict__ r, int nx, int ny, int nz, double hh,
                                double omega, const int* __restrict__ stop) {
  if (*stop) return;  // the solve has finished: the rest of its batch does nothing
  const long long n = (long long)nx * ny * nz;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    cell_of(q, nx, ny, i, j, k);
    en[q] = eo[q] + omega * (-hh / 6.0) * (r[q] - apply_A_d(eo, i, j, k, nx, ny, nz, hh));
  }
}

// rc = mean over the 8 children of (r - A e); coarse dims (cx, cy, cz)
__global__ void resid_restrict_d_kernel(const double* __restrict__ e, const double* __restrict__ r,
                                        double* __restrict__ rc, int cx, int cy, int cz, double hh, const int* __restrict__ stop) {
  if (*stop) return;  // the solve has finished: the rest of its batch does nothing
  const int nx = 2 * cx, ny = 2 * cy, nz = 2 * cz;
  const long long nc = (long long)cx * cy * cz;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nc;
       t += (long long)gridDim.x * blockDim.x) {
    int I, J, K;
    cell_of(t, cx, cy, I, J, K);
    double s = 0.0;
    for (int dk = 0; dk < 2; ++dk)
      for (int dj = 0; dj < 2; ++dj)
        for (int di = 0; di < 2; ++di) {
          const int i = 2 * I + di, j = 2 * J + dj, k = 2 * K + dk;
          const long long q = ((long long)k * ny + j) * nx + i;
          s += r[q] - apply_A_d(e, i, j, k, nx, ny, nz, hh);
        }
    rc[t] = s / 8.0;
  }
}

// ef += P ec, one thread per fine cell
__global__ void prolong_add_d_kernel(double* __restrict__ ef, const double* __restrict__ ec,
                                     int cx, int cy, int cz, const int* __restrict__ stop) {
  if (*stop) return;  // the solve has finished: the rest of its batch does nothing
  const int nx = 2 * cx, ny = 2 * cy, nz = 2 * cz;
  const long long n = (long long)nx * ny * nz;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    cell_of(q, nx, ny, i, j, k);
    const int I = i >> 1, J = j >> 1, K = k >> 1;
    const int Is[2] = {I, wrap(I + ((i & 1) ? 1 : -1), cx)};
    const int Js[2] = {J, wrap(J + ((j & 1) ? 1 : -1), cy)};
    const int Ks[2] = {K, wrap(K + ((k & 1) ? 1 : -1), cz)};
    auto at = [&](int kk, int jj, int ii) { return ec[((long long)kk * cy + jj) * cx + ii]; };
    double Y[2];
    for (int b = 0; b < 2; ++b) {            // the x index of the y pass: parent, neighbour
      double Z[2];
      for (int a = 0; a < 2; ++a)            // the y index of the z pass: parent, neighbour
        Z[a] = 0.75 * at(Ks[0], Js[a], Is[b]) + 0.25 * at(Ks[1], Js[a], Is[b]);
      Y[b] = 0.75 * Z[0] + 0.25 * Z[1];
    }
    ef[q] += 0.75 * Y[0] + 0.25 * Y[1];
  }
}

__global__ void coarse_solve_d_kernel(const double* __restrict__ r, double* __restrict__ e,
                                      const double* __restrict__ G, int n0, int n1, int n2, const int* __restrict__ stop) {
  if (*stop) return;  // the solve has finished: the rest of its batch does nothing
  const int N = n0 * n1 * n2;
  for (int p = threadIdx.x; p < N; p += blockDim.x) {
    const int p0 = p % n0, p1 = (p / n0) % n1, p2 = p / (n0 * n1);
    double s = 0.0;
    for (int q = 0; q < N; ++q) {
      const int q0 = q % n0, q1 = (q / n0) % n1, q2 = q / (n0 * n1);
      const int d0 = wrap(p0 - q0, n0), d1 = wrap(p1 - q1, n1), d2 = wrap(p2 - q2, n2);
      s += G[(d2 * n1 + d1) * n0 + d0] * r[q];
    }
    e[p] = s;
  }
}

// The fine level of a float64 context: phi' = phi + e (UPDATE, float-float + float64), the
// residual r = F - A phi' in float-float, stored in float64, and per-block partials of
// |r / rms(F)|^2.  Each thread forms the updated neighbours itself (the same rounding as the
// owner's), so phi' may go to a second buffer while other blocks read phi.
template <bool UPDATE>
__global__ void __launch_bounds__(RED_THREADS)
residual_d_kernel(const float* __restrict__ phi, float* __restrict__ phi_out,
                  const double* __restrict__ e, const float* __restrict__ F,
                  double* __restrict__ r, int nx, int ny, int nz, ff2 h2, double ih2,
                  const double* fnorm2, double* partials, const int* __restrict__ stop) {
  if (*stop) return;  // the solve has finished: the rest of its batch does nothing
  __shared__ double red[RED_THREADS];
  const long long n = (long long)nx * ny * nz;
  const double sF = 1.0 / sqrt(*fnorm2 / (double)n);
  auto val = [&](long long q) {
    const ff2 v = ff_load(phi, n, q);
    return UPDATE ? ff_add(v, ff_from_double(e[q])) : v;
  };
  double acc = 0.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    cell_of(q, nx, ny, i, j, k);
    const long long row = (long long)k * ny;
    const ff2 cv = val(q);
    ff2 lap = ff_mul_f(cv, -6.0f);
    lap = ff_add(lap, val(((long long)wrap(k - 1, nz) * ny + j) * nx + i));
    lap = ff_add(lap, val(((long long)wrap(k + 1, nz) * ny + j) * nx + i));
    lap = ff_add(lap, val((row + wrap(j - 1, ny)) * nx + i));
    lap = ff_add(lap, val((row + wrap(j + 1, ny)) * nx + i));
    lap = ff_add(lap, val((row + j) * nx + wrap(i - 1, nx)));
    lap = ff_add(lap, val((row + j) * nx + wrap(i + 1, nx)));
    const ff2 d = ff_sub(ff_mul(ff_load(F, n, q), h2), lap);      // h^2 (F - A phi)
    const double rr = ff_to_double(d) * ih2;
    r[q] = rr;
    acc += (rr * sF) * (rr * sF);
    if (UPDATE) ff_store(phi_out, n, q, cv);
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// Per-block float-float sums of the potential (the gauge's mean), in float64 partials.
__global__ void sum_ff_kernel(const float* __restrict__ phi, long long n, double* partials) {
  __shared__ double red[RED_THREADS];
  long long b0, b1;
  block_range(n, b0, b1);
  ff2 acc{0.0f, 0.0f};
  for (long long i = b0 + threadIdx.x; i < b1; i += blockDim.x) acc = ff_add(acc, ff_load(phi, n, i));
  const double s = block_sum(ff_to_double(acc), red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void sub_mean_ff_kernel(float* __restrict__ phi, long long n, const double* mean) {
  const ff2 mneg = ff_neg(ff_from_double(*mean));
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x)
    ff_store(phi, n, q, ff_add(ff_load(phi, n, q), mneg));
}

// phi - <phi>, float-float -> float64 (for callers of the potential)
__global__ void ff_to_double_kernel(const float* __restrict__ phi, long long n, const double* mean,
                                    double* __restrict__ out) {
  const ff2 mneg = ff_neg(ff_from_double(*mean));
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x)
    out[q] = ff_to_double(ff_add(ff_load(phi, n, q), mneg));
}

__global__ void mark_fail_kernel(StepRecord* rec, unsigned flag) {
  if (threadIdx.x == 0) {
    rec->flags |= flag;
    if (rec->fail_step < 0) rec->fail_step = (int)(rec->nstep - 1);
  }
}

// Judges the iterate whose residual finalize_kernel just reduced (scal[1] = |F|^2,
// scal[2] = |r|^2 / |F|^2): stop at mg_tol, at a non-finite residual or after max_cycles
// cycles, else count the cycle enqueued next.  rec (nullable): a step whose earlier kernels
// failed fatally solves nothing.
__global__ void mg_decide_kernel(MGCtl* ctl, const double* scal, double tol, int max_cycles,
                                 const StepRecord* rec) {
  if (threadIdx.x != 0 || ctl->stop) return;
  if (rec && (rec->flags & FATAL_FLAGS)) {
    ctl->skipped = 1;
    ctl->stop = 1;
    return;
  }
  if (!(scal[1] > 0.0)) {
    ctl->zero = 1;
    ctl->ok = 1;
    ctl->rel = 0.0;
    ctl->stop = 1;
    return;
  }
  const double rel = sqrt(scal[2]);
  ctl->rel = rel;
  if (rel <= tol) {
    ctl->ok = 1;
    ctl->stop = 1;
  } else if (!(rel == rel) || ctl->cycles >= max_cycles) {
    ctl->stop = 1;
  } else {
    ctl->cycles += 1;
  }
}

static int grid_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 148 * 16) b = 148 * 16;
  if (b < 1) b = 1;
  return (int)b;
}

// One float32 cycle for A e_l = r_l (Sec. 5.2; App. C): pre-smoothing, restriction of the
// residual, the coarser level visited once (V-cycle) or twice (W-cycle: the second visit starts
// from the first's result; a coarsest level, solved exactly, is visited once), prolongation and
// post-smoothing.  zero_init: e_l starts at 0 (the first visit of a level), else from e_l.
static void cycle(dh_ctx* c, int l, bool zero_init) {
  MG* m = c->mg;
  const dh_config& g = c->cfg;
  cudaStream_t s = c->stream;
  const int nx = m->n[l][0], ny = m->n[l][1], nz = m->n[l][2];
  const float h2 = (float)(m->h[l] * m->h[l]);
  if (l == m->L - 1) {
    coarse_solve_kernel<<<1, 256, 0, s>>>(m->r[l], m->e[l], m->G, nx, ny, nz, m->stop);
    c->launches += 1;
    return;
  }
  // smoothing sweeps write e2 from e, then swap; a first sweep from e = 0 reads no e
  const dim3 sg((nx + SW_TX - 1) / SW_TX, (ny + SW_TY - 1) / SW_TY, (nz + SW_ZC - 1) / SW_ZC);
  const dim3 sg4((nx + S4_TX - 1) / S4_TX, (ny + S4_TY - 1) / S4_TY, (nz + SW_ZC - 1) / SW_ZC);
  const bool vec = nx % 4 == 0;
  const float omega = (float)g.mg_omega;
  auto smooth = [&](bool zero) {
    if (g.mg_smoother == 1) {
      if (zero)
        jacobi_zero_kernel<<<grid_for(m->cells[l]), 256, 0, s>>>(m->e2[l], m->r[l], m->cells[l],
                                                                 -omega * h2 * (1.0f / 6.0f), m->stop);
      else if (vec)
        jacobi4_kernel<<<sg4, 256, 0, s>>>(m->e[l], m->e2[l], m->r[l], nx, ny, nz, h2, omega, m->stop);
      else
        jacobi_kernel<<<grid_for(m->cells[l]), 256, 0, s>>>(m->e[l], m->e2[l], m->r[l], nx, ny,
                                                            nz, h2, omega, m->stop);
    } else if (vec && zero) {
      rbgs_sweep4_kernel<true><<<sg4, 256, 0, s>>>(m->e[l], m->e2[l], m->r[l], nx, ny, nz, h2, m->stop);
    } else if (vec) {
      rbgs_sweep4_kernel<false><<<sg4, 256, 0, s>>>(m->e[l], m->e2[l], m->r[l], nx, ny, nz, h2, m->stop);
    } else if (zero) {
      rbgs_sweep_kernel<true><<<sg, 256, 0, s>>>(m->e[l], m->e2[l], m->r[l], nx, ny, nz, h2, m->stop);
    } else {
      rbgs_sweep_kernel<false><<<sg, 256, 0, s>>>(m->e[l], m->e2[l], m->r[l], nx, ny, nz, h2, m->stop);
    }
    std::swap(m->e[l], m->e2[l]);
    c->launches += 1;
  };
  if (zero_init && g.mg_pre == 0) cudaMemsetAsync(m->e[l], 0, m->cells[l] * sizeof(float), s);
  for (int it = 0; it < g.mg_pre; ++it) smooth(zero_init && it == 0);
  resid_restrict_kernel<<<grid_for(m->cells[l + 1]), 256, 0, s>>>(
      m->e[l], m->r[l], m->r[l + 1], nx / 2, ny / 2, nz / 2, 1.0f / h2, m->stop);
  const int visits = (g.mg_cycle == 2 && l + 1 < m->L - 1) ? 2 : 1;
  for (int v = 0; v < visits; ++v) cycle(c, l + 1, v == 0);
  prolong_add_kernel<<<grid_for(m->cells[l]), 256, 0, s>>>(m->e[l], m->e[l + 1], nx / 2, ny / 2, nz / 2,
                                                           m->stop);
  for (int it = 0; it < g.mg_post; ++it) smooth(false);
  c->launches += 2;
}

// The float64 cycle of a float64 context for A e_l = r_l, in the oracle's order: e_l = 0 on a
// first visit, mg_pre sweeps, restriction of r - A e, the coarser level once (V) or twice (W),
// prolongation, mg_post sweeps; the coarsest level is solved exactly.
static void cycle_d(dh_ctx* c, int l, bool zero_init) {
  MG* m = c->mg;
  const dh_config& g = c->cfg;
  cudaStream_t s = c->stream;
  const int nx = m->n[l][0], ny = m->n[l][1], nz = m->n[l][2];
  const double hh = m->h[l] * m->h[l];
  const int gb = grid_for(m->cells[l]);
  if (l == m->L - 1) {
    coarse_solve_d_kernel<<<1, 256, 0, s>>>(m->dr[l], m->de[l], m->G, nx, ny, nz, m->stop);
    c->launches += 1;
    return;
  }
  auto smooth = [&]() {
    if (g.mg_smoother == 1) {
      jacobi_d_kernel<<<gb, 256, 0, s>>>(m->de[l], m->de2[l], m->dr[l], nx, ny, nz, hh, g.mg_omega, m->stop);
      std::swap(m->de[l], m->de2[l]);
      c->launches += 1;
    } else {
      rbgs_colour_d_kernel<<<gb, 256, 0, s>>>(m->de[l], m->dr[l], nx, ny, nz, hh, 0, m->stop);
      rbgs_colour_d_kernel<<<gb, 256, 0, s>>>(m->de[l], m->dr[l], nx, ny, nz, hh, 1, m->stop);
      c->launches += 2;
    }
  };
  if (zero_init) cudaMemsetAsync(m->de[l], 0, m->cells[l] * sizeof(double), s);
  for (int it = 0; it < g.mg_pre; ++it) smooth();
  resid_restrict_d_kernel<<<grid_for(m->cells[l + 1]), 256, 0, s>>>(m->de[l], m->dr[l], m->dr[l + 1],
                                                                    nx / 2, ny / 2, nz / 2, hh, m->stop);
  const int visits = (g.mg_cycle == 2 && l + 1 < m->L - 1) ? 2 : 1;
  for (int v = 0; v < visits; ++v) cycle_d(c, l + 1, v == 0);
  prolong_add_d_kernel<<<gb, 256, 0, s>>>(m->de[l], m->de[l + 1], nx / 2, ny / 2, nz / 2, m->stop);
  for (int it = 0; it < g.mg_post; ++it) smooth();
  c->launches += 2;
}

// Launches one cycle from the finest level: replays the captured graph when the buffers are
// where they were at capture, else captures it (or, if capture fails, launches directly).
static cudaError_t run_cycle(dh_ctx* c) {
  MG* m = c->mg;
  const dh_config& g = c->cfg;
  if (m->f64) {
    cycle_d(c, 0, true);
    return cudaGetLastError();
  }
  // the buffer layout returns to its start after a cycle iff every level swaps an even number
  // of times: each visit swaps (mg_pre + mg_post) times
  const bool even = (g.mg_pre + g.mg_post) % 2 == 0;
  auto same_layout = [&]() {
    for (int l = 0; l < m->L; ++l)
      if (m->cycle_e[l] != m->e[l]) return false;
    return true;
  };
  if (m->cycle_exec && even && same_layout()) {
    c->launches += m->cycle_launches;
    return cudaGraphLaunch(m->cycle_exec, c->stream);
  }
  if (!even || m->cycle_graph_failed) {
    cycle(c, 0, true);
    return cudaGetLastError();
  }
  if (m->cycle_exec) {
    cudaGraphExecDestroy(m->cycle_exec);
    m->cycle_exec = nullptr;
  }
  for (int l = 0; l < m->L; ++l) {
    m->cycle_e[l] = m->e[l];
    m->cycle_e2[l] = m->e2[l];
  }
  cudaGraph_t graph = nullptr;
  const long long before = c->launches;
  cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cycle(c, 0, true);
    e = cudaStreamEndCapture(c->stream, &graph);
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&m->cycle_exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  m->cycle_launches = c->launches - before;
  c->launches = before;
  if (e != cudaSuccess || !m->cycle_exec) {
    // no graph on this stream (for instance the caller is capturing it): direct launches, and
    // the buffers as they were before the aborted capture
    cudaGetLastError();
    m->cycle_exec = nullptr;
    m->cycle_graph_failed = true;
    for (int l = 0; l < m->L; ++l) {
      m->e[l] = m->cycle_e[l];
      m->e2[l] = m->cycle_e2[l];
    }
    cycle(c, 0, true);
    return cudaGetLastError();
  }
  // the capture swapped the buffers as the cycle does; the graph leaves them as at its start
  for (int l = 0; l < m->L; ++l) {
    m->e[l] = m->cycle_e[l];
    m->e2[l] = m->cycle_e2[l];
  }
  c->launches += m->cycle_launches;
  return cudaGraphLaunch(m->cycle_exec, c->stream);
}

// V-cycles on phi for the source in F (|F|^2 already in scal[1]) until the relative residual
// reaches mg_tol, then (gauge) <phi> = 0.  Marks FLAG_MG_NOCONV on failure.  The solves inside
// a step leave the gauge open: only differences of phi enter the step, and dh_get_potential
// removes the mean when it hands phi out (a constant is in A's null space, so the warm start and
// the iterates are unaffected by it).
//
// The host does not read the residual after every cycle.  It enqueues a batch of items (a
// cycle, the residual of the new iterate with the correction added, its reduction and
// mg_decide_kernel), as many as the previous solve took cycles, then reads the control block
// once; items after the decision to stop return at once.  A batch that ends before the
// decision is followed by batches of 1, 2, 4, ... items.  The iterates and the cycle count are
// those of a residual check after every cycle.  check_rec (nullable): the step record whose
// fatal flags make the solve a no-op.
static cudaError_t mg_iterate(dh_ctx* c, bool gauge, const StepRecord* check_rec) {
  MG* m = c->mg;
  const dh_config& g = c->cfg;
  cudaStream_t s = c->stream;
  const long long n = m->cells[0];
  const int nx = m->n[0][0], ny = m->n[0][1], nz = m->n[0][2];
  const double hh = m->h[0] * m->h[0];
  const ff2 h2 = ff_from_double(hh);
  const float ih2 = (float)(1.0 / hh);
  const dim3 rg((nx + RZ_TX - 1) / RZ_TX, (ny + RZ_TY - 1) / RZ_TY, (nz + RZ_ZC - 1) / RZ_ZC);
  // rows of whole 64-cell multiples take the two-cells-per-thread residual
  const bool pair_res = nx % (2 * RP_QX) == 0;
  const dim3 rpg(nx / (2 * RP_QX), (ny + RZ_TY - 1) / RZ_TY, (nz + RZ_ZC - 1) / RZ_ZC);
  const int rblocks = (int)(pair_res ? residual_pair_blocks(nx, ny, nz) : residual_zm_blocks(nx, ny, nz));
  MGCtl* ctl = (MGCtl*)m->ctl;
  cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(MGCtl), s);
  if (e != cudaSuccess) return e;
  // one residual evaluation: of phi (first) or of phi + e[0] into phi2 (after a cycle), which
  // then becomes phi
  int swaps = 0;
  auto evaluate = [&](bool add) {
    prof_begin(c, DH_KERNEL_MG);
    if (m->f64) {
      if (add)
        residual_d_kernel<true><<<RED_BLOCKS, RED_THREADS, 0, s>>>(
            m->phi, m->phi2, m->de[0], m->F, m->dr[0], nx, ny, nz, h2, 1.0 / hh, m->scal + 1,
            m->partials, m->stop);
      else
        residual_d_kernel<false><<<RED_BLOCKS, RED_THREADS, 0, s>>>(
            m->phi, nullptr, nullptr, m->F, m->dr[0], nx, ny, nz, h2, 1.0 / hh, m->scal + 1,
            m->partials, m->stop);
    } else if (pair_res) {
      if (add)
        residual_zm_pair_kernel<true><<<rpg, 256, 0, s>>>(m->phi, m->phi2, m->e[0], m->F, m->r[0], nx,
                                                          ny, nz, h2, ih2, m->scal + 1, m->partials,
                                                          m->stop);
      else
        residual_zm_pair_kernel<false><<<rpg, 256, 0, s>>>(m->phi, nullptr, nullptr, m->F, m->r[0], nx,
                                                           ny, nz, h2, ih2, m->scal + 1, m->partials,
                                                           m->stop);
    } else if (add) {
      residual_zm_kernel<true><<<rg, 256, 0, s>>>(m->phi, m->phi2, m->e[0], m->F, m->r[0], nx, ny,
                                                  nz, h2, ih2, m->scal + 1, m->partials, m->stop);
    } else {
      residual_zm_kernel<false><<<rg, 256, 0, s>>>(m->phi, nullptr, nullptr, m->F, m->r[0], nx, ny,
                                                   nz, h2, ih2, m->scal + 1, m->partials, m->stop);
    }
    if (add) {
      std::swap(m->phi, m->phi2);
      ++swaps;
    }
    finalize_kernel<<<1, FIN_THREADS, 0, s>>>(m->partials, m->f64 ? RED_BLOCKS : rblocks, m->scal + 2,
                                              1.0 / (double)n, m->stop);
    mg_decide_kernel<<<1, 32, 0, s>>>(ctl, m->scal, g.mg_tol, g.mg_max_cycles, check_rec);
    c->launches += 3;
    prof_end(c, 2);
  };
  const int max_items = g.mg_max_cycles + 1;   // residual evaluations of a solve at most
  int items = m->last_cycles + 1;                // the previous solve's count
  int enqueued = 0, next = 1;
  MGCtl h;
  while (true) {
    if (items > max_items - enqueued) items = max_items - enqueued;
    for (int i = 0; i < items; ++i, ++enqueued) {
      if (enqueued > 0) {
        prof_begin(c, DH_KERNEL_MG);
        e = run_cycle(c);
        prof_end(c, 0);
        if (e != cudaSuccess) return e;
      }
      evaluate(enqueued > 0);
    }
    e = cudaMemcpyAsync(&h, ctl, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    if (h.stop || enqueued >= max_items) break;
    items = next;
    next *= 2;
  }
  // every cycle that ran was followed by the evaluation that added its correction; the swaps
  // enqueued after the decision did not happen
  if ((swaps - h.cycles) & 1) std::swap(m->phi, m->phi2);
  if (h.skipped) return cudaGetLastError();
  if (h.zero) {
    e = cudaMemsetAsync(m->phi, 0, 2 * n * sizeof(float), s);
    if (e != cudaSuccess) return e;
  }
  if (gauge) {
    prof_begin(c, DH_KERNEL_MG);
    sum_ff_kernel<<<RED_BLOCKS, RED_THREADS, 0, s>>>(m->phi, n, m->partials);
    finalize_kernel<<<1, FIN_THREADS, 0, s>>>(m->partials, RED_BLOCKS, m->scal + 3, 1.0 / (double)n);
    sub_mean_ff_kernel<<<grid_for(n), 256, 0, s>>>(m->phi, n, m->scal + 3);
    prof_end(c, 3);
  }
  m->last_cycles = h.cycles;
  m->last_res = h.rel;
  if (!h.ok) {
    mark_fail_kernel<<<1, 32, 0, s>>>(c->rec, FLAG_MG_NOCONV);
    c->launches += 1;
  }
  return cudaGetLastError();
}

// Solves for phi from the density plane of U (type real).
template <typename real>
cudaError_t mg_solve(dh_ctx* c, const real* rho, bool in_step) {
  MG* m = c->mg;
  const dh_config& g = c->cfg;
  cudaStream_t s = c->stream;
  const long long n = m->cells[0];
  prof_begin(c, DH_KERNEL_MG);
  sum_partial_kernel<real><<<RED_BLOCKS, RED_THREADS, 0, s>>>(rho, n, m->partials);
  finalize_kernel<<<1, FIN_THREADS, 0, s>>>(m->partials, RED_BLOCKS, m->scal + 0, 1.0 / (double)n);
  poisson_source_kernel<real><<<RED_BLOCKS, RED_THREADS, 0, s>>>(rho, n, m->scal + 0, g.four_pi_G,
                                                                 m->F, m->partials);
  finalize_kernel<<<1, FIN_THREADS, 0, s>>>(m->partials, RED_BLOCKS, m->scal + 1, 1.0);
  prof_end(c, 4);
  // in a step, nothing is solved after a fatal failure earlier in the batch (the stages skipped)
  return mg_iterate(c, false, in_step ? c->rec : nullptr);
}

// A x = rhs - <rhs> for a float64 right-hand side; x (float-float, planar, n cells) is the warm
// start and the result, with <x> = 0.  The solve the adjoint of the gravity step needs (A is
// symmetric).
cudaError_t mg_solve_rhs(dh_ctx* c, const double* rhs, float* x) {
  MG* m = c->mg;
  cudaStream_t s = c->stream;
  const long long n = m->cells[0];
  prof_begin(c, DH_KERNEL_MG);
  sum_partial_kernel<double><<<RED_BLOCKS, RED_THREADS, 0, s>>>(rhs, n, m->partials);
  finalize_kernel<<<1, FIN_THREADS, 0, s>>>(m->partials, RED_BLOCKS, m->scal + 0, 1.0 / (double)n);
  poisson_source_kernel<double><<<RED_BLOCKS, RED_THREADS, 0, s>>>(rhs, n, m->scal + 0, 1.0,
                                                                   m->F, m->partials);
  finalize_kernel<<<1, FIN_THREADS, 0, s>>>(m->partials, RED_BLOCKS, m->scal + 1, 1.0);
  prof_end(c, 4);
  // x stands in for the context's potential; the fused update alternates between the two
  // buffers, so the result is copied into x if it ends in the other one
  float* keep = m->phi;
  float* keep2 = m->phi2;
  m->phi = x;
  cudaError_t e = mg_iterate(c, true, nullptr);
  if (e == cudaSuccess && m->phi != x)
    e = cudaMemcpyAsync(x, m->phi, 2 * n * sizeof(float), cudaMemcpyDeviceToDevice, s);
  m->phi = keep;
  m->phi2 = keep2;
  return e;
}

// ---------------------------------------------------------------------------------------------
// Sources after the hydro update when gravity is on: forcing -> gravity -> cooling (the Lie
// splitting order), then the positivity/finite checks and the CFL minimum for the next step.
// A CTA owns a 64 x 4 column of cells and marches GS_ZC planes.  The forcing is synthesised as
// in the stage kernel: per plane, 36 threads form the row factors B[row][n_x][component] (the
// forced modes summed over n_y, n_z for that row), and each cell adds its x twiddles, so the
// per-cell cost is a few FMAs instead of a sum over all forced modes.
constexpr int GS_TX = 64, GS_TY = 4, GS_ZC = 16, GS_NF = GS_TY * 9;

template <typename real>
__global__ void __launch_bounds__(256)
gravity_sources_kernel(real* __restrict__ U, const float* __restrict__ phi, int nx, int ny,
                       int nz, real i2h, StepRecord* rec, const double* dtp, int in_step,
                       int forcing,
                       const real* __restrict__ ah, const real* tw0, const real* tw1,
                       const real* tw2, int cooling, real gamma, real gm1, real t_floor,
                       real frac, int nsub_max, real dx, real dy, real dz, real cool_ratio) {
  __shared__ unsigned s_skip;
  __shared__ real red[8];
  __shared__ real fB[2][GS_TY][3][3][2];   // double-buffered by plane parity
  // forcing tables of the CTA: the OU table, the y twiddles of its rows and the z twiddles of
  // its planes, loaded once so that the per-plane row factors wait on no global load
  __shared__ real s_ah[96], s_ty[GS_TY][4], s_tz[GS_ZC][4];
  const int tid = threadIdx.x;
  const int z0 = blockIdx.z * GS_ZC, z1 = z0 + GS_ZC < nz ? z0 + GS_ZC : nz;
  if (tid == 0) s_skip = *((volatile unsigned*)&rec->flags) & FATAL_FLAGS;
  if (forcing) {
    if (tid < 96) s_ah[tid] = __ldg(ah + tid);
    if (tid >= 96 && tid < 96 + 4 * GS_TY) {
      const int ly = (tid - 96) >> 2, q = (tid - 96) & 3;
      s_ty[ly][q] = __ldg(tw1 + 4 * ((blockIdx.y * GS_TY + ly) % ny) + q);
    }
    if (tid >= 128 && tid < 128 + 4 * GS_ZC) {
      const int lz = (tid - 128) >> 2, q = (tid - 128) & 3;
      if (z0 + lz < nz) s_tz[lz][q] = __ldg(tw2 + 4 * (z0 + lz) + q);
    }
  }
  __syncthreads();
  if (s_skip) return;
  const real dt = (real)*dtp;
  const long long plane = (long long)nx * ny;
  const long long n3 = plane * nz;
  const int tx = tid % GS_TX, ty = tid / GS_TX;
  const int i = blockIdx.x * GS_TX + tx, j = blockIdx.y * GS_TY + ty;
  const bool active = i < nx && j < ny;
  real twx[4] = {real(0), real(0), real(0), real(0)};
  if (forcing && active) {
#pragma unroll
    for (int q = 0; q < 4; ++q) twx[q] = __ldg(tw0 + 4 * i + q);
  }
  real tmin = real(INFINITY);
  unsigned flags = 0;
  int nsub_seen = 0;
  // the state and potential words of the next plane are loaded a plane ahead
  real un[5];
  float pv[12];
  if (active) {
    const long long q = (long long)z0 * plane + (long long)j * nx + i;
#pragma unroll
    for (int c = 0; c < 5; ++c) un[c] = U[c * n3 + q];
    potential_gradient_load(phi, nx, ny, nz, i, j, z0, pv);
  }
  for (int k = z0; k < z1; ++k) {
    const int buf = (k - z0) & 1;
    if (forcing) {
      if (tid < GS_NF) {
        const int ly = tid / 9, rem = tid - 9 * ly;
        const int nxsel = rem / 3, c = rem - 3 * nxsel;
        real tyv[4], tzv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          tyv[q] = s_ty[ly][q];
          tzv[q] = s_tz[k - z0][q];
        }
        real bre = real(0), bim = real(0);
        row_factor<real, 0>(s_ah, nxsel, c, tyv, tzv, bre, bim);
        fB[buf][ly][nxsel][c][0] = bre;
        fB[buf][ly][nxsel][c][1] = bim;
      }
      __syncthreads();   // one barrier per plane: the other buffer is rewritten a plane later
    }
    if (!active) continue;
    const long long q = (long long)k * plane + (long long)j * nx + i;
    real u[5];
    float pw[12];
#pragma unroll
    for (int c = 0; c < 5; ++c) u[c] = un[c];
#pragma unroll
    for (int c = 0; c < 12; ++c) pw[c] = pv[c];
    if (k + 1 < z1) {
#pragma unroll
      for (int c = 0; c < 5; ++c) un[c] = U[c * n3 + q + plane];
      potential_gradient_load(phi, nx, ny, nz, i, j, k + 1, pv);
    }
    if (forcing) {
      // a = 2 Re sum_{n_x} B_{n_x} exp(2 pi i n_x x~)  (Sec. 3.1.1)
      real a[3];
#pragma unroll
      for (int c = 0; c < 3; ++c)
        a[c] = real(2) * (fB[buf][ty][0][c][0] +
                          (fB[buf][ty][1][c][0] * twx[0] - fB[buf][ty][1][c][1] * twx[1]) +
                          (fB[buf][ty][2][c][0] * twx[2] - fB[buf][ty][2][c][1] * twx[3]));
      const real e = (u[1] * a[0] + u[2] * a[1] + u[3] * a[2]) * dt;
      u[1] = u[1] + u[0] * a[0] * dt;
      u[2] = u[2] + u[0] * a[1] * dt;
      u[3] = u[3] + u[0] * a[2] * dt;
      u[4] = u[4] + e;
    }
    {
      // g = -grad phi by central differences (Sec. 5), momentum taken before the kick
      real g0, g1, g2;
      potential_gradient_eval(pw, i2h, g0, g1, g2);
      const real e = (u[1] * g0 + u[2] * g1 + u[3] * g2) * dt;
      u[1] = u[1] + u[0] * g0 * dt;
      u[2] = u[2] + u[0] * g1 * dt;
      u[3] = u[3] + u[0] * g2 * dt;
      u[4] = u[4] + e;
    }
    if (cooling)
      u[4] = cooling_energy(u[0], u[1], u[2], u[3], u[4], dt, gm1, t_floor, frac, nsub_max, flags,
                            nsub_seen);
    bool finite = true;
#pragma unroll
    for (int c = 0; c < 5; ++c) finite = finite && isfinite(u[c]);
    if (!finite) {
      flags |= FLAG_NONFINITE;
    } else {
      const real pr = gm1 * (u[4] - real(0.5) * q_div(u[1] * u[1] + u[2] * u[2] + u[3] * u[3], u[0]));
      if (!(u[0] > real(0)) || !(pr > real(0))) flags |= FLAG_POSITIVITY;
      tmin = fmin(tmin, cfl_time(u[0], u[1], u[2], u[3], u[4], gamma, gm1, dx, dy, dz));
      if (cool_ratio > real(0))
        tmin = fmin(tmin, cool_ratio * cooling_time(u[0], u[1], u[2], u[3], u[4], gm1, t_floor));
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) U[c * n3 + q] = u[c];
  }
  if (!in_step) return;   // a replay (adjoint) leaves the step record alone
  if (flags) {
    atomicOr(&rec->flags, flags);
    if (flags & FATAL_FLAGS) atomicCAS(&rec->fail_step, -1, (int)(rec->nstep - 1));
  }
  if (nsub_seen > 1) atomicMax(&rec->cool_nsub_max, nsub_seen);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tmin = fmin(tmin, __shfl_xor_sync(0xffffffffu, tmin, o));
  if ((tid & 31) == 0) red[tid >> 5] = tmin;
  __syncthreads();
  if (tid == 0) {
    real m = red[0];
    for (int w = 1; w < 8; ++w) m = fmin(m, red[w]);
    if (m < real(INFINITY)) atomicMin(&rec->cfl_min_bits, ordered_bits(m));
  }
}

// The same sources for two cells per thread, 32 apart in x (grids whose rows are whole multiples
// of 64 cells): a CTA owns a 64 x 8 column and marches GS_ZC planes, and every quantity is a
// two-lane pair, so the forcing and gravity kicks, the cooling and the CFL time run as packed
// FP32x2 arithmetic.  The cooling and CFL time have the scalar functions' roundings per lane;
// the checks are those of the paired stage kernel.  The potential gradient of the plane is
// evaluated before the next plane's words are requested, so that only one plane of words is
// held in registers.
constexpr int GP_QX = 32, GP_TY = 8, GP_NF = GP_TY * 9;

template <typename real>
__global__ void __launch_bounds__(256)
gravity_sources_pair_kernel(real* __restrict__ U, const float* __restrict__ phi, int nx, int ny,
                            int nz, real i2h, StepRecord* rec, const double* dtp, int in_step,
                            int forcing, const real* __restrict__ ah, const real* tw0,
                            const real* tw1, const real* tw2, int cooling, real gamma, real gm1,
                            real t_floor, real frac, int nsub_max, real dx, real dy, real dz,
                            real cool_ratio) {
  using P = pair_t<real>;
  __shared__ unsigned s_skip;
  __shared__ real red[8];
  __shared__ real fB[2][GP_TY][3][3][2];   // double-buffered by plane parity
  __shared__ real s_ah[96], s_ty[GP_TY][4], s_tz[GS_ZC][4];
  const int tid = threadIdx.x;
  const int z0 = blockIdx.z * GS_ZC, z1 = z0 + GS_ZC < nz ? z0 + GS_ZC : nz;
  if (tid == 0) s_skip = *((volatile unsigned*)&rec->flags) & FATAL_FLAGS;
  if (forcing) {
    if (tid < 96) s_ah[tid] = __ldg(ah + tid);
    if (tid >= 96 && tid < 96 + 4 * GP_TY) {
      const int ly = (tid - 96) >> 2, q = (tid - 96) & 3;
      s_ty[ly][q] = __ldg(tw1 + 4 * ((blockIdx.y * GP_TY + ly) % ny) + q);
    }
    if (tid >= 128 && tid < 128 + 4 * GS_ZC) {
      const int lz = (tid - 128) >> 2, q = (tid - 128) & 3;
      if (z0 + lz < nz) s_tz[lz][q] = __ldg(tw2 + 4 * (z0 + lz) + q);
    }
  }
  __syncthreads();
  if (s_skip) return;
  const real dt = (real)*dtp;
  const long long plane = (long long)nx * ny;
  const long long n3 = plane * nz;
  const int tx = tid % GP_QX, ty = tid / GP_QX;
  const int ia = blockIdx.x * (2 * GP_QX) + tx, ib = ia + GP_QX;
  const int j = blockIdx.y * GP_TY + ty;
  const bool active = j < ny;
  P twx[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) twx[q] = pset(real(0));
  if (forcing && active) {
#pragma unroll
    for (int q = 0; q < 4; ++q) twx[q] = pmk(__ldg(tw0 + 4 * ia + q), __ldg(tw0 + 4 * ib + q));
  }
  real tmin = real(INFINITY);
  unsigned flags = 0;
  int nsub_seen = 0;
  const P pdt = pset(dt);
  // the state and potential words of the next plane are loaded a plane ahead
  P un[5];
  float pva[12], pvb[12];
  if (active) {
    const long long q = (long long)z0 * plane + (long long)j * nx + ia;
#pragma unroll
    for (int c = 0; c < 5; ++c) un[c] = pmk(U[c * n3 + q], U[c * n3 + q + GP_QX]);
    potential_gradient_load(phi, nx, ny, nz, ia, j, z0, pva);
    potential_gradient_load(phi, nx, ny, nz, ib, j, z0, pvb);
  }
  for (int k = z0; k < z1; ++k) {
    const int buf = (k - z0) & 1;
    if (forcing) {
      if (tid < GP_NF) {
        const int ly = tid / 9, rem = tid - 9 * ly;
        const int nxsel = rem / 3, c = rem - 3 * nxsel;
        real tyv[4], tzv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          tyv[q] = s_ty[ly][q];
          tzv[q] = s_tz[k - z0][q];
        }
        real bre = real(0), bim = real(0);
        row_factor<real, 0>(s_ah, nxsel, c, tyv, tzv, bre, bim);
        fB[buf][ly][nxsel][c][0] = bre;
        fB[buf][ly][nxsel][c][1] = bim;
      }
      __syncthreads();   // one barrier per plane: the other buffer is rewritten a plane later
    }
    if (!active) continue;
    const long long q = (long long)k * plane + (long long)j * nx + ia;
    // g = -grad phi by central differences (Sec. 5) of this plane, then the next plane's loads
    real ga0, ga1, ga2, gb0, gb1, gb2;
    potential_gradient_eval(pva, i2h, ga0, ga1, ga2);
    potential_gradient_eval(pvb, i2h, gb0, gb1, gb2);
    P u[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) u[c] = un[c];
    if (k + 1 < z1) {
#pragma unroll
      for (int c = 0; c < 5; ++c) un[c] = pmk(U[c * n3 + q + plane], U[c * n3 + q + plane + GP_QX]);
      potential_gradient_load(phi, nx, ny, nz, ia, j, k + 1, pva);
      potential_gradient_load(phi, nx, ny, nz, ib, j, k + 1, pvb);
    }
    if (forcing) {
      // a = 2 Re sum_{n_x} B_{n_x} exp(2 pi i n_x x~)  (Sec. 3.1.1)
      const real(*B)[3][2] = fB[buf][ty];
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
    {
      // the gravity kick, momentum taken before the kick
      const P g0 = pmk(ga0, gb0), g1 = pmk(ga1, gb1), g2 = pmk(ga2, gb2);
      const P e = pmul(pfma(u[3], g2, pfma(u[2], g1, pmul(u[1], g0))), pdt);
      u[1] = pfma(pmul(u[0], g0), pdt, u[1]);
      u[2] = pfma(pmul(u[0], g1), pdt, u[2]);
      u[3] = pfma(pmul(u[0], g2), pdt, u[3]);
      u[4] = padd(u[4], e);
    }
    if (cooling)
      u[4] = cooling_energy2<real>(u[0], u[1], u[2], u[3], u[4], dt, gm1, t_floor, frac, nsub_max,
                                   flags, nsub_seen);
    bool fa = true, fb = true;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      fa = fa && isfinite(u[c].x);
      fb = fb && isfinite(u[c].y);
    }
    P pres;
    const P tc = cfl_time2<real>(u, gamma, gm1, dx, dy, dz, pres);
    auto finish = [&](bool fin, real rho, real pr, real t, int lane) {
      if (!fin) {
        flags |= FLAG_NONFINITE;
        return;
      }
      if (!(rho > real(0)) || !(pr > real(0))) flags |= FLAG_POSITIVITY;
      tmin = fmin(tmin, t);
      if (cool_ratio > real(0)) {
        const real v[5] = {lane ? u[0].y : u[0].x, lane ? u[1].y : u[1].x, lane ? u[2].y : u[2].x,
                           lane ? u[3].y : u[3].x, lane ? u[4].y : u[4].x};
        tmin = fmin(tmin, cool_ratio * cooling_time(v[0], v[1], v[2], v[3], v[4], gm1, t_floor));
      }
    };
    finish(fa, u[0].x, pres.x, tc.x, 0);
    finish(fb, u[0].y, pres.y, tc.y, 1);
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      U[c * n3 + q] = u[c].x;
      U[c * n3 + q + GP_QX] = u[c].y;
    }
  }
  if (!in_step) return;   // a replay (adjoint) leaves the step record alone
  if (flags) {
    atomicOr(&rec->flags, flags);
    if (flags & FATAL_FLAGS) atomicCAS(&rec->fail_step, -1, (int)(rec->nstep - 1));
  }
  if (nsub_seen > 1) atomicMax(&rec->cool_nsub_max, nsub_seen);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tmin = fmin(tmin, __shfl_xor_sync(0xffffffffu, tmin, o));
  if ((tid & 31) == 0) red[tid >> 5] = tmin;
  __syncthreads();
  if (tid == 0) {
    real m = red[0];
    for (int w = 1; w < 8; ++w) m = fmin(m, red[w]);
    if (m < real(INFINITY)) atomicMin(&rec->cfl_min_bits, ordered_bits(m));
  }
}

template <typename real>
cudaError_t gravity_sources(dh_ctx* c, void* Ustar, const void* tab, const double* dtp,
                            bool in_step) {
  const dh_config& g = c->cfg;
  real* U = (real*)Ustar;
  // in a step, skip when an earlier failure is pending (the stage kernels already skipped)
  cudaError_t e = mg_solve<real>(c, U, in_step);
  if (e != cudaSuccess) return e;
  prof_begin(c, DH_KERNEL_SOURCES);
  const real cool_ratio = g.cooling && std::isfinite(g.c_cool) ? (real)(g.c_cool / g.cfl) : real(0);
  if (std::is_same<real, float>::value && g.nx % (2 * GP_QX) == 0) {
    // two cells per thread (float32, rows of whole 64-cell multiples)
    const dim3 grid(g.nx / (2 * GP_QX), (g.ny + GP_TY - 1) / GP_TY, (g.nz + GS_ZC - 1) / GS_ZC);
    gravity_sources_pair_kernel<real><<<grid, 256, 0, c->stream>>>(
        U, c->mg->phi, g.nx, g.ny, g.nz, (real)(1.0 / (2.0 * g.dx)), c->rec, dtp, in_step ? 1 : 0,
        g.forcing, (const real*)(tab ? tab : c->ahat_norm), (const real*)c->tw[0],
        (const real*)c->tw[1], (const real*)c->tw[2], g.cooling, (real)g.gamma,
        (real)(g.gamma - 1.0), (real)g.t_floor, (real)g.cool_frac, g.nsub_max, (real)g.dx,
        (real)g.dy, (real)g.dz, cool_ratio);
    prof_end(c, 1);
    return cudaGetLastError();
  }
  const dim3 grid((g.nx + GS_TX - 1) / GS_TX, (g.ny + GS_TY - 1) / GS_TY, (g.nz + GS_ZC - 1) / GS_ZC);
  gravity_sources_kernel<real><<<grid, 256, 0, c->stream>>>(
      U, c->mg->phi, g.nx, g.ny, g.nz, (real)(1.0 / (2.0 * g.dx)), c->rec, dtp, in_step ? 1 : 0,
      g.forcing, (const real*)(tab ? tab : c->ahat_norm), (const real*)c->tw[0],
      (const real*)c->tw[1], (const real*)c->tw[2], g.cooling, (real)g.gamma,
      (real)(g.gamma - 1.0), (real)g.t_floor, (real)g.cool_frac, g.nsub_max, (real)g.dx,
      (real)g.dy, (real)g.dz, cool_ratio);
  prof_end(c, 1);
  return cudaGetLastError();
}
template cudaError_t gravity_sources<float>(dh_ctx*, void*, const void*, const double*, bool);
template cudaError_t gravity_sources<double>(dh_ctx*, void*, const void*, const double*, bool);

}  // namespace dh

extern "C" dh_status dh_get_potential(dh_ctx* c, double* phi_out, int on_device, int* cycles,
                                      double* rel_residual) {
  if (!c) return DH_ERR_ARG;
  if (!c->cfg.gravity || !c->mg) { c->err = "gravity is off"; return DH_ERR_STATE; }
  if (phi_out) {
    // float-float -> float64 in the source buffer F (free between solves), then copied out
    MG* m = c->mg;
    const long long n = m->cells[0];
    double* tmp = on_device ? phi_out : (double*)m->F;
    dh::sum_ff_kernel<<<dh::RED_BLOCKS, dh::RED_THREADS, 0, c->stream>>>(m->phi, n, m->partials);
    dh::finalize_kernel<<<1, dh::FIN_THREADS, 0, c->stream>>>(m->partials, dh::RED_BLOCKS, m->scal + 3,
                                                 1.0 / (double)n);
    dh::ff_to_double_kernel<<<dh::grid_for(n), 256, 0, c->stream>>>(m->phi, n, m->scal + 3, tmp);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && !on_device)
      e = cudaMemcpyAsync(phi_out, tmp, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) { c->err = cudaGetErrorString(e); return DH_ERR_CUDA; }
  }
  if (cycles) *cycles = c->mg->last_cycles;
  if (rel_residual) *rel_residual = c->mg->last_res;
  return DH_OK;
}

extern "C" dh_status dh_reset_potential(dh_ctx* c) {
  if (!c) return DH_ERR_ARG;
  if (!c->cfg.gravity || !c->mg) { c->err = "gravity is off"; return DH_ERR_STATE; }
  const cudaError_t e = dh::mg_reset(c);
  if (e != cudaSuccess) { c->err = cudaGetErrorString(e); return DH_ERR_CUDA; }
  return DH_OK;
}

extern "C" dh_status dh_solve_poisson(dh_ctx* c, const void* rho, int on_device) {
  if (!c || !rho) return DH_ERR_ARG;
  if (!c->cfg.gravity || !c->mg) { c->err = "gravity is off"; return DH_ERR_STATE; }
  const size_t es = c->prec == DH_F64 ? 8 : 4;
  const size_t bytes = (size_t)c->n3 * es;
  // the RK2 intermediate buffer is free between steps: stage the density there
  cudaError_t e = cudaMemcpyAsync(c->U1, rho, bytes,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  c->stream);
  if (e == cudaSuccess)
    e = c->prec == DH_F64 ? dh::mg_solve<double>(c, (const double*)c->U1, false)
                          : dh::mg_solve<float>(c, (const float*)c->U1, false);
  unsigned fl = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&fl, &c->rec->flags, sizeof(fl), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) { c->err = cudaGetErrorString(e); return DH_ERR_CUDA; }
  if (fl & dh::FLAG_MG_NOCONV) {
    // a standalone solve leaves no failed step behind: clear the flag it raised
    dh::StepRecord r;
    cudaMemcpy(&r, c->rec, sizeof(r), cudaMemcpyDeviceToHost);
    r.flags &= ~dh::FLAG_MG_NOCONV;
    r.fail_step = -1;
    cudaMemcpy(c->rec, &r, sizeof(r), cudaMemcpyHostToDevice);
    c->err = "multigrid did not reach mg_tol within mg_max_cycles";
    return DH_ERR_MG_NOCONV;
  }
  return DH_OK;
}

// =============================================================================================
// Exact periodic Poisson solve by the discrete Fourier transform (Sec. 2.3 and 5 name the FFT
// solver beside the multigrid one): the DFT diagonalises the seven-point operator A, with
// eigenvalue lambda(k) = -(4/h^2) sum_a sin^2(pi k_a / n_a), so phi_hat = F_hat / lambda for
// k != 0 and 0 for k = 0 (<phi> = 0).  Float64 complex, power-of-two dimensions.  Each 1D
// transform is an iterative radix-2 Cooley-Tukey pass of one CTA over one line in shared memory
// (bit-reversed load, log2 n butterfly stages, twiddles from a per-axis table).
namespace dh {

constexpr int FFT_MAX = 1024;

// F = four_pi_G (rho - <rho>) as complex float64
template <typename T>
__global__ void fft_load_kernel(const T* __restrict__ rho, long long n, const double* mean,
                                double four_pi_G, double2* __restrict__ buf) {
  const double m = *mean;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x)
    buf[q] = make_double2(four_pi_G * ((double)rho[q] - m), 0.0);
}

// One line per CTA: lines `line` = 0 .. count-1 start at line_base(line) and step `stride`.
// Axis layout: x lines (stride 1) are rows; y lines (stride nx) are indexed by (x, z); z lines
// (stride nx ny) by (x, y).  tw[j] = exp(-2 pi i j / n), j < n/2; inverse uses the conjugate.
__global__ void fft_lines_kernel(double2* __restrict__ buf, const double2* __restrict__ tw, int n,
                                 int logn, int axis, int nx, int ny, int nz, int inverse) {
  extern __shared__ double2 s_fft[];   // n values, then n/2 twiddles
  double2* v = s_fft;
  double2* w = s_fft + n;
  const long long plane = (long long)nx * ny;
  const long long count = axis == 0 ? (long long)ny * nz : (axis == 1 ? (long long)nx * nz : plane);
  const long long stride = axis == 0 ? 1 : (axis == 1 ? nx : plane);
  for (int j = threadIdx.x; j < n / 2; j += blockDim.x)
    w[j] = inverse ? make_double2(tw[j].x, -tw[j].y) : tw[j];
  for (long long line = blockIdx.x; line < count; line += gridDim.x) {
    long long base;
    if (axis == 0) base = line * nx;
    else if (axis == 1) base = (line / nx) * plane + (line % nx);     // (x, z) -> z plane + x
    else base = line;                                                  // (x, y) -> y row + x
    __syncthreads();   // the previous line's values are no longer read
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int r = (int)(__brev((unsigned)i) >> (32 - logn));
      v[r] = buf[base + (long long)i * stride];
    }
    __syncthreads();
    for (int len = 2, s = 1; len <= n; len <<= 1, ++s) {
      const int half = len >> 1, step = n >> s;   // twiddle index step for this stage
      for (int b = threadIdx.x; b < n / 2; b += blockDim.x) {
        const int grp = b / half, k = b - grp * half;
        const int i0 = grp * len + k, i1 = i0 + half;
        const double2 t = w[k * step];
        const double2 a = v[i0], c = v[i1];
        const double2 tc = make_double2(t.x * c.x - t.y * c.y, t.x * c.y + t.y * c.x);
        v[i0] = make_double2(a.x + tc.x, a.y + tc.y);
        v[i1] = make_double2(a.x - tc.x, a.y - tc.y);
      }
      __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) buf[base + (long long)i * stride] = v[i];
  }
}

// phi_hat = F_hat / lambda(k), 0 at k = 0; s2x[k] = sin^2(pi k / nx) etc.
__global__ void fft_divide_kernel(double2* __restrict__ buf, const double* __restrict__ s2x,
                                  const double* __restrict__ s2y, const double* __restrict__ s2z,
                                  int nx, int ny, int nz, double m4ih2) {
  const long long n = (long long)nx * ny * nz;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const long long t = q / nx;
    const int i = (int)(q - t * nx), j = (int)(t % ny), k = (int)(t / ny);
    if (q == 0) {
      buf[q] = make_double2(0.0, 0.0);
    } else {
      const double il = 1.0 / (m4ih2 * (s2x[i] + s2y[j] + s2z[k]));
      buf[q] = make_double2(buf[q].x * il, buf[q].y * il);
    }
  }
}

__global__ void fft_store_kernel(const double2* __restrict__ buf, long long n, double scale,
                                 double* __restrict__ phi) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x)
    phi[q] = buf[q].x * scale;
}

}  // namespace dh

namespace {
int log2_exact(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return (1 << l) == n ? l : -1;
}
}  // namespace

extern "C" dh_status dh_fft_poisson(dh_ctx* c, const void* rho, int on_device, double* phi_out,
                                    int out_on_device) {
  if (!c || !rho || !phi_out) return DH_ERR_ARG;
  if (!c->cfg.gravity || !c->mg) { c->err = "gravity is off"; return DH_ERR_STATE; }
  const int dims[3] = {c->cfg.nx, c->cfg.ny, c->cfg.nz};
  int logs[3];
  for (int a = 0; a < 3; ++a) {
    logs[a] = log2_exact(dims[a]);
    if (logs[a] < 1 || dims[a] > dh::FFT_MAX) {
      c->err = "dh_fft_poisson: every dimension must be a power of two between 2 and 1024";
      return DH_ERR_ARG;
    }
  }
  MG* m = c->mg;
  cudaStream_t s = c->stream;
  const long long n = c->n3;
  const size_t es = c->prec == DH_F64 ? 8 : 4;
  // buffers: the complex field, twiddles and sin^2 tables of the three axes
  double2* buf = nullptr;
  double2* tw = nullptr;
  double* s2 = nullptr;
  cudaError_t e = cudaMallocAsync(&buf, n * sizeof(double2), s);
  if (e == cudaSuccess) e = cudaMallocAsync(&tw, 3 * (dh::FFT_MAX / 2) * sizeof(double2), s);
  if (e == cudaSuccess) e = cudaMallocAsync(&s2, 3 * dh::FFT_MAX * sizeof(double), s);
  std::vector<double2> htw(3 * (dh::FFT_MAX / 2));
  std::vector<double> hs2(3 * dh::FFT_MAX);
  for (int a = 0; a < 3; ++a) {
    for (int j = 0; j < dims[a] / 2; ++j) {
      const double ang = -2.0 * M_PI * j / dims[a];
      htw[a * (dh::FFT_MAX / 2) + j] = make_double2(std::cos(ang), std::sin(ang));
    }
    for (int k = 0; k < dims[a]; ++k) {
      const double sn = std::sin(M_PI * k / dims[a]);
      hs2[a * dh::FFT_MAX + k] = sn * sn;
    }
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(tw, htw.data(), htw.size() * sizeof(double2), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s2, hs2.data(), hs2.size() * sizeof(double), cudaMemcpyHostToDevice, s);
  // the density in the stage scratch (free between steps), its mean, then F
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->U1, rho, (size_t)n * es,
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    if (c->prec == DH_F64) {
      dh::sum_partial_kernel<double><<<dh::RED_BLOCKS, dh::RED_THREADS, 0, s>>>((const double*)c->U1, n, m->partials);
      dh::finalize_kernel<<<1, dh::FIN_THREADS, 0, s>>>(m->partials, dh::RED_BLOCKS, m->scal + 0, 1.0 / (double)n);
      dh::fft_load_kernel<double><<<dh::grid_for(n), 256, 0, s>>>((const double*)c->U1, n, m->scal + 0, c->cfg.four_pi_G, buf);
    } else {
      dh::sum_partial_kernel<float><<<dh::RED_BLOCKS, dh::RED_THREADS, 0, s>>>((const float*)c->U1, n, m->partials);
      dh::finalize_kernel<<<1, dh::FIN_THREADS, 0, s>>>(m->partials, dh::RED_BLOCKS, m->scal + 0, 1.0 / (double)n);
      dh::fft_load_kernel<float><<<dh::grid_for(n), 256, 0, s>>>((const float*)c->U1, n, m->scal + 0, c->cfg.four_pi_G, buf);
    }
    e = cudaGetLastError();
  }
  auto pass = [&](int inverse) {
    for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
      const int len = dims[a];
      const long long lines = n / len;
      const int threads = len / 2 < 32 ? 32 : (len / 2 > 512 ? 512 : len / 2);
      const size_t smem = (size_t)(len + len / 2) * sizeof(double2);
      const int blocks = (int)(lines < 148LL * 16 ? lines : 148LL * 16);
      if (smem > 48 * 1024)
        e = cudaFuncSetAttribute(dh::fft_lines_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) break;
      dh::fft_lines_kernel<<<blocks, threads, smem, s>>>(buf, tw + a * (dh::FFT_MAX / 2), len, logs[a], a,
                                                         dims[0], dims[1], dims[2], inverse);
      e = cudaGetLastError();
    }
  };
  dh::prof_begin(c, DH_KERNEL_MG);
  pass(0);
  if (e == cudaSuccess) {
    const double h = c->cfg.dx;
    dh::fft_divide_kernel<<<dh::grid_for(n), 256, 0, s>>>(buf, s2, s2 + dh::FFT_MAX, s2 + 2 * dh::FFT_MAX,
                                                          dims[0], dims[1], dims[2], -4.0 / (h * h));
    e = cudaGetLastError();
  }
  pass(1);
  // a host result is staged in the stage scratch (5 planes: at least 20 bytes per cell)
  double* out = out_on_device ? phi_out : (double*)c->U1;
  if (e == cudaSuccess) {
    dh::fft_store_kernel<<<dh::grid_for(n), 256, 0, s>>>(buf, n, 1.0 / (double)n, out);
    e = cudaGetLastError();
  }
  dh::prof_end(c, 11);
  if (e == cudaSuccess && !out_on_device)
    e = cudaMemcpyAsync(phi_out, out, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(buf, s);
  cudaFreeAsync(tw, s);
  cudaFreeAsync(s2, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { c->err = cudaGetErrorString(e); return DH_ERR_CUDA; }
  return DH_OK;
}
