// Multigrid self-gravity (Sec. 5.2; App. C) and the operator-split source kernel of steps that
// use it.
//
// Solve A phi = F, F = 4 pi G (rho - <rho>), A the seven-point periodic Laplacian.  The fine
// level keeps phi and F in float64 and iterates defect correction: r = F - A phi (float64),
// then one float32 V-cycle for A e = r (red-black Gauss-Seidel, mg_pre / mg_post sweeps,
// 8-child mean restriction, cell-centred trilinear prolongation, exact coarsest solve), then
// phi += e.  For a linear smoother this is the V-cycle applied to phi itself, so the iterates
// are those of Sec. 5.2's cycle; keeping phi and the residual in float64 lets the relative
// residual reach 1e-6 at large N, which float32 phi cannot (its rounding alone leaves
// ~eps_32 * |phi| / h^2 in A phi).  Norms and means are float64 with a fixed reduction order.
//
// The coarsest grid (<= 1024 cells) is solved with the pseudo-inverse of its operator, a
// circulant: A^+ e_p = sum_q G[(p - q) mod n] r_q with G[d] = (1/N) sum_{k != 0}
// cos(2 pi k.d / n) / lambda_k and lambda_k = -(4/h^2) sum_a sin^2(pi k_a / n_a), the discrete
// eigenvalues; it also removes the mean (the constant null space).
#include <math.h>
#include <string.h>
#include <vector>

#include "dh_internal.h"
#include "dh_sources.cuh"

namespace dh {
constexpr int MG_LMAX = 16;
constexpr int RED_BLOCKS = 296, RED_THREADS = 256;
}

struct MG {
  int L = 0;
  int n[dh::MG_LMAX][3];
  double h[dh::MG_LMAX];
  long long cells[dh::MG_LMAX];
  double* phi64 = nullptr;
  double* F64 = nullptr;
  float* e[dh::MG_LMAX] = {nullptr};
  float* r[dh::MG_LMAX] = {nullptr};
  double* G = nullptr;           // coarsest circulant pseudo-inverse
  double* partials = nullptr;    // RED_BLOCKS doubles
  double* scal = nullptr;        // [0] mean rho, [1] |F|^2, [2] |r|^2, [3] mean phi
  int last_cycles = 0;
  double last_res = 0.0;
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
  MG m;
  level_dims(c, &m);
  if (m.cells[m.L - 1] > 1024) return "coarsest multigrid level exceeds 1024 cells";
  return "";
}

cudaError_t mg_allocate(dh_ctx* c) {
  MG* m = new MG();
  c->mg = m;
  level_dims(c->cfg, m);
  cudaError_t e = cudaMalloc(&m->phi64, m->cells[0] * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&m->F64, m->cells[0] * sizeof(double));
  for (int l = 0; l < m->L && e == cudaSuccess; ++l) {
    e = cudaMalloc(&m->e[l], m->cells[l] * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&m->r[l], m->cells[l] * sizeof(float));
  }
  if (e == cudaSuccess) e = cudaMalloc(&m->G, m->cells[m->L - 1] * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&m->partials, RED_BLOCKS * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&m->scal, 8 * sizeof(double));
  // the potential is the warm start of the first solve: zero, not whatever the allocator held
  if (e == cudaSuccess) e = cudaMemset(m->phi64, 0, m->cells[0] * sizeof(double));
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
  return cudaMemsetAsync(m->phi64, 0, m->cells[0] * sizeof(double), c->stream);
}

double* mg_phi64(dh_ctx* c) { return c->mg ? c->mg->phi64 : nullptr; }

void mg_free(dh_ctx* c) {
  MG* m = c->mg;
  if (!m) return;
  cudaFree(m->phi64);
  cudaFree(m->F64);
  for (int l = 0; l < MG_LMAX; ++l) { cudaFree(m->e[l]); cudaFree(m->r[l]); }
  cudaFree(m->G);
  cudaFree(m->partials);
  cudaFree(m->scal);
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

template <typename T>
__global__ void sum_partial_kernel(const T* __restrict__ x, long long n, double* partials) {
  __shared__ double red[RED_THREADS];
  long long b0, b1;
  block_range(n, b0, b1);
  double s = 0.0;
  for (long long i = b0 + threadIdx.x; i < b1; i += blockDim.x) s += (double)x[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// out = scale * sum(partials)
__global__ void finalize_kernel(const double* partials, int nb, double* out, double scale) {
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += partials[b];
    *out = scale * s;
  }
}

template <typename T>
__global__ void poisson_source_kernel(const T* __restrict__ rho, long long n, const double* mean,
                                      double four_pi_G, double* __restrict__ F, double* partials) {
  __shared__ double red[RED_THREADS];
  long long b0, b1;
  block_range(n, b0, b1);
  const double m = *mean;
  double s = 0.0;
  for (long long i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
    const double f = four_pi_G * ((double)rho[i] - m);
    F[i] = f;
    s += f * f;
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// r = F - A phi in float64; stores r as the float32 right-hand side of the correction.
__global__ void residual64_kernel(const double* __restrict__ phi, const double* __restrict__ F,
                                  float* __restrict__ r32, int nx, int ny, int nz, double ih2,
                                  double* partials) {
  __shared__ double red[RED_THREADS];
  const long long n = (long long)nx * ny * nz;
  long long b0, b1;
  block_range(n, b0, b1);
  double s = 0.0;
  for (long long q = b0 + threadIdx.x; q < b1; q += blockDim.x) {
    const int i = (int)(q % nx);
    const long long t = q / nx;
    const int j = (int)(t % ny);
    const int k = (int)(t / ny);
    const long long row = (long long)k * ny;
    const double c = phi[q];
    const double nb = phi[((long long)wrap(k - 1, nz) * ny + j) * nx + i] +
                      phi[((long long)wrap(k + 1, nz) * ny + j) * nx + i] +
                      phi[(row + wrap(j - 1, ny)) * nx + i] + phi[(row + wrap(j + 1, ny)) * nx + i] +
                      phi[(row + j) * nx + wrap(i - 1, nx)] + phi[(row + j) * nx + wrap(i + 1, nx)];
    const double rr = F[q] - (nb - 6.0 * c) * ih2;
    r32[q] = (float)rr;
    s += rr * rr;
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// One colour of red-black Gauss-Seidel on A e = r: e_i = (sum of 6 neighbours - h^2 r_i) / 6.
__global__ void rbgs_kernel(float* __restrict__ e, const float* __restrict__ r, int nx, int ny,
                            int nz, float h2, int color) {
  const long long half = (long long)(nx / 2) * ny * nz;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < half;
       t += (long long)gridDim.x * blockDim.x) {
    const int ih = (int)(t % (nx / 2));
    const long long u = t / (nx / 2);
    const int j = (int)(u % ny);
    const int k = (int)(u / ny);
    const int i = 2 * ih + ((j + k + color) & 1);
    const long long row = (long long)k * ny;
    const long long q = (row + j) * nx + i;
    const float nb = e[((long long)wrap(k - 1, nz) * ny + j) * nx + i] +
                     e[((long long)wrap(k + 1, nz) * ny + j) * nx + i] +
                     e[(row + wrap(j - 1, ny)) * nx + i] + e[(row + wrap(j + 1, ny)) * nx + i] +
                     e[(row + j) * nx + wrap(i - 1, nx)] + e[(row + j) * nx + wrap(i + 1, nx)];
    e[q] = (nb - h2 * r[q]) * (1.0f / 6.0f);
  }
}

// rc[I] = mean over the 8 children of (r - A e), coarse dims (cx, cy, cz).
__global__ void resid_restrict_kernel(const float* __restrict__ e, const float* __restrict__ r,
                                      float* __restrict__ rc, int cx, int cy, int cz, float ih2) {
  const int nx = 2 * cx, ny = 2 * cy, nz = 2 * cz;
  const long long nc = (long long)cx * cy * cz;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nc;
       t += (long long)gridDim.x * blockDim.x) {
    const int I = (int)(t % cx);
    const long long u = t / cx;
    const int J = (int)(u % cy);
    const int K = (int)(u / cy);
    float s = 0.f;
    for (int dk = 0; dk < 2; ++dk)
      for (int dj = 0; dj < 2; ++dj)
        for (int di = 0; di < 2; ++di) {
          const int i = 2 * I + di, j = 2 * J + dj, k = 2 * K + dk;
          const long long row = (long long)k * ny;
          const long long q = (row + j) * nx + i;
          const float nb = e[((long long)wrap(k - 1, nz) * ny + j) * nx + i] +
                           e[((long long)wrap(k + 1, nz) * ny + j) * nx + i] +
                           e[(row + wrap(j - 1, ny)) * nx + i] + e[(row + wrap(j + 1, ny)) * nx + i] +
                           e[(row + j) * nx + wrap(i - 1, nx)] + e[(row + j) * nx + wrap(i + 1, nx)];
          s += r[q] - (nb - 6.0f * e[q]) * ih2;
        }
    rc[t] = 0.125f * s;
  }
}

// e_fine += P e_coarse: per axis 3/4 of the parent and 1/4 of the parent's neighbour on the
// fine cell's side (weights (27, 9, 9, 9, 3, 3, 3, 1)/64), periodic.
__global__ void prolong_add_kernel(float* __restrict__ ef, const float* __restrict__ ec, int cx,
                                   int cy, int cz) {
  const int nx = 2 * cx, ny = 2 * cy, nz = 2 * cz;
  const long long nf = (long long)nx * ny * nz;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nf;
       q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % nx);
    const long long u = q / nx;
    const int j = (int)(u % ny);
    const int k = (int)(u / ny);
    const int I = i >> 1, J = j >> 1, K = k >> 1;
    const int I2 = wrap(I + ((i & 1) ? 1 : -1), cx);
    const int J2 = wrap(J + ((j & 1) ? 1 : -1), cy);
    const int K2 = wrap(K + ((k & 1) ? 1 : -1), cz);
    const int Is[2] = {I, I2}, Js[2] = {J, J2}, Ks[2] = {K, K2};
    const float w[2] = {0.75f, 0.25f};
    float s = 0.f;
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b)
        for (int c = 0; c < 2; ++c)
          s += w[a] * w[b] * w[c] * ec[((long long)Ks[a] * cy + Js[b]) * cx + Is[c]];
    ef[q] += s;
  }
}

__global__ void coarse_solve_kernel(const float* __restrict__ r, float* __restrict__ e,
                                    const double* __restrict__ G, int n0, int n1, int n2) {
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

__global__ void update64_kernel(double* __restrict__ phi, const float* __restrict__ e, long long n) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x)
    phi[q] += (double)e[q];
}

__global__ void sub_mean_kernel(double* __restrict__ phi, long long n, const double* mean) {
  const double m = *mean;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x)
    phi[q] -= m;
}

__global__ void zero64_kernel(double* __restrict__ phi, long long n) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x)
    phi[q] = 0.0;
}

__global__ void mark_fail_kernel(StepRecord* rec, unsigned flag) {
  if (threadIdx.x == 0) {
    rec->flags |= flag;
    if (rec->fail_step < 0) rec->fail_step = (int)(rec->nstep - 1);
  }
}

static int grid_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 148 * 16) b = 148 * 16;
  if (b < 1) b = 1;
  return (int)b;
}

// One float32 V-cycle for A e_l = r_l starting from e_l = 0.
static void vcycle(dh_ctx* c, int l) {
  MG* m = c->mg;
  const dh_config& g = c->cfg;
  cudaStream_t s = c->stream;
  const int nx = m->n[l][0], ny = m->n[l][1], nz = m->n[l][2];
  const float h2 = (float)(m->h[l] * m->h[l]);
  if (l == m->L - 1) {
    coarse_solve_kernel<<<1, 256, 0, s>>>(m->r[l], m->e[l], m->G, nx, ny, nz);
    c->launches += 1;
    return;
  }
  cudaMemsetAsync(m->e[l], 0, m->cells[l] * sizeof(float), s);
  const int gb = grid_for(m->cells[l] / 2);
  for (int it = 0; it < g.mg_pre; ++it) {
    rbgs_kernel<<<gb, 256, 0, s>>>(m->e[l], m->r[l], nx, ny, nz, h2, 0);
    rbgs_kernel<<<gb, 256, 0, s>>>(m->e[l], m->r[l], nx, ny, nz, h2, 1);
  }
  resid_restrict_kernel<<<grid_for(m->cells[l + 1]), 256, 0, s>>>(
      m->e[l], m->r[l], m->r[l + 1], nx / 2, ny / 2, nz / 2, 1.0f / h2);
  vcycle(c, l + 1);
  prolong_add_kernel<<<grid_for(m->cells[l]), 256, 0, s>>>(m->e[l], m->e[l + 1], nx / 2, ny / 2, nz / 2);
  for (int it = 0; it < g.mg_post; ++it) {
    rbgs_kernel<<<gb, 256, 0, s>>>(m->e[l], m->r[l], nx, ny, nz, h2, 0);
    rbgs_kernel<<<gb, 256, 0, s>>>(m->e[l], m->r[l], nx, ny, nz, h2, 1);
  }
  c->launches += 2 * (g.mg_pre + g.mg_post) + 2;
}

// V-cycles on phi64 for the source in F64 (|F|^2 already in scal[1]) until the relative
// residual reaches mg_tol, then the gauge <phi> = 0.  Marks FLAG_MG_NOCONV on failure.
static cudaError_t mg_iterate(dh_ctx* c) {
  MG* m = c->mg;
  const dh_config& g = c->cfg;
  cudaStream_t s = c->stream;
  const long long n = m->cells[0];
  const int nx = m->n[0][0], ny = m->n[0][1], nz = m->n[0][2];
  const double ih2 = 1.0 / (m->h[0] * m->h[0]);
  int cycles = 0;
  double rel = 0.0;
  bool ok = false;
  while (true) {
    prof_begin(c, DH_KERNEL_MG);
    residual64_kernel<<<RED_BLOCKS, RED_THREADS, 0, s>>>(m->phi64, m->F64, m->r[0], nx, ny, nz,
                                                         ih2, m->partials);
    finalize_kernel<<<1, 32, 0, s>>>(m->partials, RED_BLOCKS, m->scal + 2, 1.0);
    prof_end(c, 2);
    double h[3];
    cudaError_t e = cudaMemcpyAsync(h, m->scal, 3 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    if (!(h[1] > 0.0)) {  // zero source: phi = 0
      zero64_kernel<<<grid_for(n), 256, 0, s>>>(m->phi64, n);
      c->launches += 1;
      ok = true;
      rel = 0.0;
      break;
    }
    rel = std::sqrt(h[2] / h[1]);
    if (rel <= g.mg_tol) { ok = true; break; }
    if (!(rel == rel)) break;                 // non-finite residual
    if (cycles >= g.mg_max_cycles) break;
    prof_begin(c, DH_KERNEL_MG);
    vcycle(c, 0);
    update64_kernel<<<grid_for(n), 256, 0, s>>>(m->phi64, m->e[0], n);
    prof_end(c, 1);
    ++cycles;
  }
  // gauge <phi> = 0
  prof_begin(c, DH_KERNEL_MG);
  sum_partial_kernel<double><<<RED_BLOCKS, RED_THREADS, 0, s>>>(m->phi64, n, m->partials);
  finalize_kernel<<<1, 32, 0, s>>>(m->partials, RED_BLOCKS, m->scal + 3, 1.0 / (double)n);
  sub_mean_kernel<<<grid_for(n), 256, 0, s>>>(m->phi64, n, m->scal + 3);
  prof_end(c, 3);
  m->last_cycles = cycles;
  m->last_res = rel;
  if (!ok) {
    mark_fail_kernel<<<1, 32, 0, s>>>(c->rec, FLAG_MG_NOCONV);
    c->launches += 1;
  }
  return cudaGetLastError();
}

// Solves for phi64 from the density plane of U (type real).
template <typename real>
cudaError_t mg_solve(dh_ctx* c, const real* rho, bool in_step) {
  MG* m = c->mg;
  const dh_config& g = c->cfg;
  cudaStream_t s = c->stream;
  const long long n = m->cells[0];
  if (in_step) {
    // nothing to solve after a fatal failure earlier in this batch (the stages skipped)
    unsigned fl = 0;
    cudaError_t e = cudaMemcpyAsync(&fl, &c->rec->flags, sizeof(fl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    if (fl & FATAL_FLAGS) return cudaSuccess;
  }
  prof_begin(c, DH_KERNEL_MG);
  sum_partial_kernel<real><<<RED_BLOCKS, RED_THREADS, 0, s>>>(rho, n, m->partials);
  finalize_kernel<<<1, 32, 0, s>>>(m->partials, RED_BLOCKS, m->scal + 0, 1.0 / (double)n);
  poisson_source_kernel<real><<<RED_BLOCKS, RED_THREADS, 0, s>>>(rho, n, m->scal + 0, g.four_pi_G,
                                                                 m->F64, m->partials);
  finalize_kernel<<<1, 32, 0, s>>>(m->partials, RED_BLOCKS, m->scal + 1, 1.0);
  prof_end(c, 4);
  return mg_iterate(c);
}

// A x = rhs - <rhs> for a float64 right-hand side; x (float64, n cells) is the warm start and
// the result, with <x> = 0.  The solve the adjoint of the gravity step needs (A is symmetric).
cudaError_t mg_solve_rhs(dh_ctx* c, const double* rhs, double* x) {
  MG* m = c->mg;
  cudaStream_t s = c->stream;
  const long long n = m->cells[0];
  prof_begin(c, DH_KERNEL_MG);
  sum_partial_kernel<double><<<RED_BLOCKS, RED_THREADS, 0, s>>>(rhs, n, m->partials);
  finalize_kernel<<<1, 32, 0, s>>>(m->partials, RED_BLOCKS, m->scal + 0, 1.0 / (double)n);
  poisson_source_kernel<double><<<RED_BLOCKS, RED_THREADS, 0, s>>>(rhs, n, m->scal + 0, 1.0,
                                                                   m->F64, m->partials);
  finalize_kernel<<<1, 32, 0, s>>>(m->partials, RED_BLOCKS, m->scal + 1, 1.0);
  prof_end(c, 4);
  double* keep = m->phi64;
  m->phi64 = x;
  cudaError_t e = mg_iterate(c);
  m->phi64 = keep;
  return e;
}

// ---------------------------------------------------------------------------------------------
// Sources after the hydro update when gravity is on: forcing -> gravity -> cooling (the Lie
// splitting order), then the positivity/finite checks and the CFL minimum for the next step.
template <typename real>
__global__ void __launch_bounds__(256)
gravity_sources_kernel(real* __restrict__ U, const double* __restrict__ phi, int nx, int ny,
                       int nz, double i2h, StepRecord* rec, const double* dtp, int in_step,
                       int forcing,
                       const real* __restrict__ ah, const real* tw0, const real* tw1,
                       const real* tw2, int cooling, real gamma, real gm1, real t_floor,
                       real frac, int nsub_max, real dx, real dy, real dz) {
  __shared__ unsigned s_skip;
  __shared__ real red[8];
  if (threadIdx.x == 0) s_skip = *((volatile unsigned*)&rec->flags) & FATAL_FLAGS;
  __syncthreads();
  if (s_skip) return;
  const real dt = (real)*dtp;
  const long long plane = (long long)nx * ny;
  const long long n3 = plane * nz;
  const real* tw[3] = {tw0, tw1, tw2};
  real tmin = real(INFINITY);
  unsigned flags = 0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n3;
       q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % nx);
    const long long t = q / nx;
    const int j = (int)(t % ny);
    const int k = (int)(t / ny);
    real u[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) u[c] = U[c * n3 + q];
    if (forcing) {
      real a[3];
      forcing_accel(ah, tw, i, j, k, a);
      const real e = (u[1] * a[0] + u[2] * a[1] + u[3] * a[2]) * dt;
      u[1] = u[1] + u[0] * a[0] * dt;
      u[2] = u[2] + u[0] * a[1] * dt;
      u[3] = u[3] + u[0] * a[2] * dt;
      u[4] = u[4] + e;
    }
    {
      // g = -grad phi by central differences (Sec. 5), momentum taken before the kick
      const long long row = (long long)k * ny;
      const real g0 = (real)(-(phi[(row + j) * nx + wrap(i + 1, nx)] - phi[(row + j) * nx + wrap(i - 1, nx)]) * i2h);
      const real g1 = (real)(-(phi[(row + wrap(j + 1, ny)) * nx + i] - phi[(row + wrap(j - 1, ny)) * nx + i]) * i2h);
      const real g2 = (real)(-(phi[((long long)wrap(k + 1, nz) * ny + j) * nx + i] -
                               phi[((long long)wrap(k - 1, nz) * ny + j) * nx + i]) * i2h);
      const real e = (u[1] * g0 + u[2] * g1 + u[3] * g2) * dt;
      u[1] = u[1] + u[0] * g0 * dt;
      u[2] = u[2] + u[0] * g1 * dt;
      u[3] = u[3] + u[0] * g2 * dt;
      u[4] = u[4] + e;
    }
    if (cooling)
      u[4] = cooling_energy(u[0], u[1], u[2], u[3], u[4], dt, gm1, t_floor, frac, nsub_max, flags);
    bool finite = true;
#pragma unroll
    for (int c = 0; c < 5; ++c) finite = finite && isfinite(u[c]);
    if (!finite) {
      flags |= FLAG_NONFINITE;
    } else {
      const real pr = gm1 * (u[4] - real(0.5) * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) / u[0]);
      if (!(u[0] > real(0)) || !(pr > real(0))) flags |= FLAG_POSITIVITY;
      tmin = fmin(tmin, cfl_time(u[0], u[1], u[2], u[3], u[4], gamma, gm1, dx, dy, dz));
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) U[c * n3 + q] = u[c];
  }
  if (!in_step) return;   // a replay (adjoint) leaves the step record alone
  if (flags) {
    atomicOr(&rec->flags, flags);
    if (flags & FATAL_FLAGS) atomicCAS(&rec->fail_step, -1, (int)(rec->nstep - 1));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tmin = fmin(tmin, __shfl_xor_sync(0xffffffffu, tmin, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = tmin;
  __syncthreads();
  if (threadIdx.x == 0) {
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
  const long long n = c->n3;
  prof_begin(c, DH_KERNEL_SOURCES);
  gravity_sources_kernel<real><<<grid_for(n), 256, 0, c->stream>>>(
      U, c->mg->phi64, g.nx, g.ny, g.nz, 1.0 / (2.0 * g.dx), c->rec, dtp, in_step ? 1 : 0,
      g.forcing, (const real*)(tab ? tab : c->ahat_norm), (const real*)c->tw[0],
      (const real*)c->tw[1], (const real*)c->tw[2], g.cooling, (real)g.gamma,
      (real)(g.gamma - 1.0), (real)g.t_floor, (real)g.cool_frac, g.nsub_max, (real)g.dx,
      (real)g.dy, (real)g.dz);
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
    cudaError_t e = cudaMemcpyAsync(phi_out, c->mg->phi64, c->mg->cells[0] * sizeof(double),
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                    c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) { c->err = cudaGetErrorString(e); return DH_ERR_CUDA; }
  }
  if (cycles) *cycles = c->mg->last_cycles;
  if (rel_residual) *rel_residual = c->mg->last_res;
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
