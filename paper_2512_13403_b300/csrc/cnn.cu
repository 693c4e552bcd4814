// The corrector network around the tensor-core convolutions: normalisation, the three layers,
// the residual correction with its floors, the mean-squared-error gradient, back-propagation
// (data and weight gradients on the tensor cores, bias gradients by reduction) and Adam.
//
// Network: x0 = bf16((U - mu)/sigma) (5 channels, padded to 8); z1 = conv(x0, W1) + b1,
// h1 = bf16(gelu(z1)); z2 = conv(h1, W2) + b2, h2 = bf16(gelu(z2)); y = conv(h2, W3) + b3.
// Two forms of the correction dU, then rho >= rho_floor and E raised so that the thermal energy
// is at least rho T_floor / (gamma - 1):
//   state form (5 outputs): dU_c = s_c y_c (s the per-channel output scale);
//   flux form (15 outputs, y[5 a + c] the flux of field c through face i + 1/2 along axis a):
//   dU_c(i) = -s_c sum_a (y_{a,c}(i) - y_{a,c}(i - e_a)), a divergence, so that every conserved
//   total is unchanged (Sec. 7's flux corrector, applied after the step).
// Parameters, flat fp32: W1[32][5][27], b1[32], W2[32][32][27], b2[32], W3[nout][32][27],
// b3[nout] (36357 values for 5 outputs, 45007 for 15).
#include <cuda_bf16.h>
#include <math.h>

#include <string>

#include "conv_layout.cuh"
#include "dh_internal.h"

namespace {
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + 32 * 5 * 27, OFF_W2 = OFF_B1 + 32,
              OFF_B2 = OFF_W2 + 32 * 32 * 27, OFF_W3 = OFF_B2 + 32;
constexpr int off_b3(int nout) { return OFF_W3 + nout * 32 * 27; }
constexpr int nparam(int nout) { return off_b3(nout) + nout; }
constexpr int NPARAM = nparam(5);
static_assert(NPARAM == 36357 && nparam(15) == 45007, "parameter layout");
constexpr int RBLOCKS = 256;
}  // namespace

extern "C" dh_status dh_pack_conv_weights(const float*, int, int, int, void*, void*);
extern "C" dh_status dh_conv3d_bf16(const void*, int, const void*, int, const float*, int,
                                    const float*, void*, float*, int, int, int, int, unsigned*,
                                    void*);
extern "C" dh_status dh_conv3d_wgrad_bf16(const void*, int, int, const void*, int, int, int, int,
                                          int, float*, int, float*, unsigned*, void*);

struct dh_cnn {
  int nx = 0, ny = 0, nz = 0;
  long long ncell = 0;
  int form = 0;                             // 0 state, 1 flux
  int nout = 5;                             // network outputs: 5 or 15
  int dyc = 8;                              // channels of the padded output gradient: 8 or 32
  cudaStream_t stream = nullptr;
  float* params = nullptr;                  // device copy of the parameters
  float norm[15] = {0};                     // mu[5], sigma[5], output scale[5]
  float* norm_dev = nullptr;
  __nv_bfloat16 *pk_w1 = nullptr, *pk_w2 = nullptr, *pk_w3 = nullptr;   // forward operands
  __nv_bfloat16 *pk_w2t = nullptr, *pk_w3t = nullptr, *pk_w1t = nullptr;   // data-gradient operands
  // activations and their gradients, padded layout (conv_layout.cuh): 1 or 4 channel groups
  __nv_bfloat16 *x0 = nullptr, *h1 = nullptr, *h2 = nullptr;
  float *z1 = nullptr, *z2 = nullptr, *y = nullptr;                     // [cell][32], [nout][cell]
  float* g5 = nullptr;                      // [5][cell]: gradient of the correction / input
  __nv_bfloat16 *dy = nullptr, *dz2 = nullptr, *dz1 = nullptr;
  float* partial = nullptr;                 // weight-gradient partials
  int nctas = 148;
  double* red = nullptr;                    // reduction scratch
  double* bpart = nullptr;                  // bias-gradient partial sums [32][BG_BLOCKS]
  unsigned* err = nullptr;
  bool have_params = false;
  bool have_forward = false;
  std::string msg;
};

namespace dh {

// Cell coordinates of linear index q (grids below 2^31 cells: 32-bit arithmetic).
__device__ __forceinline__ void cell_xyz(long long q, const ConvGeom& g, int& x, int& y, int& z) {
  const unsigned t = (unsigned)q / (unsigned)g.nx;
  x = (int)((unsigned)q - t * (unsigned)g.nx);
  const unsigned w = t / (unsigned)g.ny;
  y = (int)(t - w * (unsigned)g.ny);
  z = (int)w;
}

__global__ void normalize_kernel(const float* __restrict__ U, ConvGeom g,
                                 const float* __restrict__ norm, __nv_bfloat16* __restrict__ x0) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    __align__(16) __nv_bfloat16 v[8];
#pragma unroll
    for (int c = 0; c < 5; ++c) v[c] = __float2bfloat16_rn((U[c * n + q] - norm[c]) / norm[5 + c]);
    v[5] = v[6] = v[7] = __float2bfloat16_rn(0.0f);
    int x, y, z;
    cell_xyz(q, g, x, y, z);
    store_with_images(reinterpret_cast<uint4*>(x0), g, x, y, z, *reinterpret_cast<const uint4*>(v));
  }
}

// Residual target t = (U_target - U_in) / s per channel; loss = mean over 5 channels and cells of
// (y - t)^2; dy = d loss / d y as bf16 [cell][8].
__global__ void mse_grad_kernel(const float* __restrict__ y, const float* __restrict__ Uin,
                                const float* __restrict__ Utgt, const float* __restrict__ norm,
                                ConvGeom g, __nv_bfloat16* __restrict__ dy,
                                double* __restrict__ partial) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  __shared__ double red[256];
  double s = 0.0;
  const double scale = 2.0 / (5.0 * (double)n);
  const long long per = (n + gridDim.x - 1) / gridDim.x;
  const long long b0 = blockIdx.x * per, b1 = b0 + per < n ? b0 + per : n;
  for (long long q = b0 + threadIdx.x; q < b1; q += blockDim.x) {
    __align__(16) __nv_bfloat16 v[8];
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const float t = (Utgt[c * n + q] - Uin[c * n + q]) / norm[10 + c];
      const float d = y[c * n + q] - t;
      s += (double)d * (double)d;
      v[c] = __float2bfloat16_rn((float)scale * d);
    }
    v[5] = v[6] = v[7] = __float2bfloat16_rn(0.0f);
    int x, yy, z;
    cell_xyz(q, g, x, yy, z);
    store_with_images(reinterpret_cast<uint4*>(dy), g, x, yy, z, *reinterpret_cast<const uint4*>(v));
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// Periodic neighbour cell index along axis a (0 x, 1 y, 2 z), offset d = +-1.
__device__ __forceinline__ long long nb_cell(const ConvGeom& g, int x, int y, int z, int a, int d) {
  if (a == 0) x = x + d < 0 ? g.nx - 1 : (x + d >= g.nx ? 0 : x + d);
  else if (a == 1) y = y + d < 0 ? g.ny - 1 : (y + d >= g.ny ? 0 : y + d);
  else z = z + d < 0 ? g.nz - 1 : (z + d >= g.nz ? 0 : z + d);
  return ((long long)z * g.ny + y) * g.nx + x;
}

// Flux form: p_c(i) = -sum_a (y_{a,c}(i) - y_{a,c}(i - e_a)), the divergence of the 15 outputs.
__device__ __forceinline__ float flux_div(const float* __restrict__ y, long long n, const ConvGeom& g,
                                          long long q, int x, int yy, int z, int c) {
  float p = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float* ya = y + (long long)(5 * a + c) * n;
    p -= ya[q] - ya[nb_cell(g, x, yy, z, a, -1)];
  }
  return p;
}

// Flux form, one-step loss: t = (U_target - U_in) / s, loss = mean over 5 channels and cells of
// (p - t)^2 with p the divergence above; g = d loss / d p (float [5][cell]) and loss partials.
__global__ void flux_mse_kernel(const float* __restrict__ y, const float* __restrict__ Uin,
                                const float* __restrict__ Utgt, const float* __restrict__ norm,
                                ConvGeom geo, float* __restrict__ g, double* __restrict__ partial) {
  const long long n = (long long)geo.nx * geo.ny * geo.nz;
  __shared__ double red[256];
  double s = 0.0;
  const double scale = 2.0 / (5.0 * (double)n);
  const long long per = (n + gridDim.x - 1) / gridDim.x;
  const long long b0 = blockIdx.x * per, b1 = b0 + per < n ? b0 + per : n;
  for (long long q = b0 + threadIdx.x; q < b1; q += blockDim.x) {
    int x, yy, z;
    cell_xyz(q, geo, x, yy, z);
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const float t = (Utgt[c * n + q] - Uin[c * n + q]) / norm[10 + c];
      const float d = flux_div(y, n, geo, q, x, yy, z, c) - t;
      s += (double)d * (double)d;
      g[c * n + q] = (float)scale * d;
    }
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// Output gradient dy (bf16, padded layout) from g = d L / d p (state form: p = y; flux form:
// p = the divergence of y), each channel c of g scaled by sc[c] (nullable: 1).
//   state form: dy_c = sc_c g_c (8 channels);
//   flux form:  dy_{a,c}(i) = sc_c (g_c(i + e_a) - g_c(i)), the transposed divergence (32 channels).
__global__ void output_grad_kernel(const float* __restrict__ g, const float* __restrict__ sc,
                                   int form, ConvGeom geo, __nv_bfloat16* __restrict__ dy) {
  const long long n = (long long)geo.nx * geo.ny * geo.nz;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    int x, yy, z;
    cell_xyz(q, geo, x, yy, z);
    float f[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) f[k] = 0.f;
    if (form == 0) {
#pragma unroll
      for (int c = 0; c < 5; ++c) f[c] = (sc ? sc[c] : 1.f) * g[c * n + q];
    } else {
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        const float gc = g[c * n + q];
#pragma unroll
        for (int a = 0; a < 3; ++a)
          f[5 * a + c] = (sc ? sc[c] : 1.f) * (g[c * n + nb_cell(geo, x, yy, z, a, +1)] - gc);
      }
    }
    const int groups = form == 0 ? 1 : 4;
    for (int gr = 0; gr < groups; ++gr) {
      __align__(16) __nv_bfloat16 v[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = __float2bfloat16_rn(f[8 * gr + e]);
      store_with_images(reinterpret_cast<uint4*>(dy) + (long long)gr * geo.rows, geo, x, yy, z,
                        *reinterpret_cast<const uint4*>(v));
    }
  }
}

// dL/dU = dL/dx0 / sigma per channel (the input normalisation transposed), in place.
__global__ void input_grad_kernel(float* __restrict__ g, const float* __restrict__ norm, long long n) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < 5 * n;
       q += (long long)gridDim.x * blockDim.x)
    g[q] = g[q] / norm[5 + (int)(q / n)];
}

// *out = scale * sum of partial[0..nb) in a fixed order: lane l sums entries l, l+32, ...,
// then a fixed shuffle tree (one warp).
__global__ void sum_blocks_kernel(const double* partial, int nb, double scale, double* out) {
  const int l = threadIdx.x;
  double s = 0.0;
  for (int b = l; b < nb; b += 32) s += partial[b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (l == 0) *out = scale * s;
}

// Bias gradient db[c] = sum over cells of channel c of a padded gradient.  Block (b, group)
// sums a contiguous cell range of one 8-channel group (each thread reads whole 16-byte rows);
// part[c][b] is then added in block order by bias_grad_final_kernel.
constexpr int BG_BLOCKS = 64;
__global__ void bias_grad_partial_kernel(const __nv_bfloat16* __restrict__ grad, ConvGeom g,
                                         double* __restrict__ part) {
  __shared__ double red[8][256];
  const int grp = blockIdx.y;
  const long long n = (long long)g.nx * g.ny * g.nz;
  const long long per = (n + gridDim.x - 1) / gridDim.x;
  const long long q0 = blockIdx.x * per, q1 = q0 + per < n ? q0 + per : n;
  const uint4* rows = reinterpret_cast<const uint4*>(grad) + (long long)grp * g.rows;
  float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  // (unrolled so that several rows are in flight; the sums keep their order)
#pragma unroll 4
  for (long long q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
    int x, y, z;
    cell_xyz(q, g, x, y, z);
    const uint4 v = __ldg(rows + pad_row(g, x, y, z));
    const __nv_bfloat16* h = reinterpret_cast<const __nv_bfloat16*>(&v);
#pragma unroll
    for (int e = 0; e < 8; ++e) acc[e] += __bfloat162float(h[e]);
  }
#pragma unroll
  for (int e = 0; e < 8; ++e) red[e][threadIdx.x] = (double)acc[e];
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
#pragma unroll
      for (int e = 0; e < 8; ++e) red[e][threadIdx.x] += red[e][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 8) part[(long long)(grp * 8 + threadIdx.x) * gridDim.x + blockIdx.x] = red[threadIdx.x][0];
}

__global__ void bias_grad_final_kernel(const double* __restrict__ part, int nb, int nch,
                                       float* __restrict__ db) {
  const int c = threadIdx.x;
  if (c < nch) {
    double s = 0.0;
#pragma unroll 8
    for (int b = 0; b < nb; ++b) s += part[(long long)c * nb + b];
    db[c] = (float)s;
  }
}

static void bias_grad(const __nv_bfloat16* grad, int groups, int nch, const ConvGeom& g,
                      double* part, float* db, cudaStream_t s) {
  bias_grad_partial_kernel<<<dim3(BG_BLOCKS, groups), 256, 0, s>>>(grad, g, part);
  bias_grad_final_kernel<<<1, 32, 0, s>>>(part, BG_BLOCKS, nch, db);
}

// Uout = floors(Uin + s * y) (Uout may be Uin).  rho_floor is rho_floor_c, or
// floor_per_mass * totals[0] when `totals` (the FP64 conserved totals of Uin, on the device) is
// given.  A non-finite result sets bit 2 of *err.
constexpr unsigned CNN_ERR_WAIT = 1u, CNN_ERR_NONFINITE = 2u;
//
// Inside a step (rec not null) the kernel writes nothing after a fatal failure earlier in the
// batch or after a convolution's bounded wait gave up (which fails the step), and a non-finite
// result fails the step instead of setting *err.
__global__ void correct_kernel(const float* Uin, float* Uout, const float* __restrict__ y,
                               long long n, const float* __restrict__ norm, float rho_floor_c,
                               const double* __restrict__ totals, double floor_per_mass,
                               float T_floor, float gm1, unsigned* err, int form, ConvGeom geo,
                               StepRecord* rec) {
  if (rec) {
    if (*(volatile unsigned*)&rec->flags & FATAL_FLAGS) return;
    if (*(volatile unsigned*)err & CNN_ERR_WAIT) {
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        atomicOr(&rec->flags, FLAG_TIMEOUT);
        atomicCAS(&rec->fail_step, -1, (int)(rec->nstep - 1));
      }
      return;
    }
  }
  const float rho_floor = totals ? (float)(floor_per_mass * totals[0]) : rho_floor_c;
  bool finite = true;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    float v[5];
    if (form == 0) {
#pragma unroll
      for (int c = 0; c < 5; ++c) v[c] = Uin[c * n + q] + norm[10 + c] * y[c * n + q];
    } else {
      int x, yy, z;
      cell_xyz(q, geo, x, yy, z);
#pragma unroll
      for (int c = 0; c < 5; ++c) v[c] = Uin[c * n + q] + norm[10 + c] * flux_div(y, n, geo, q, x, yy, z, c);
    }
    const float rho = fmaxf(v[0], rho_floor);
    const float kin = 0.5f * (v[1] * v[1] + v[2] * v[2] + v[3] * v[3]) / rho;
    const float Emin = kin + rho * T_floor / gm1;
    const float E = fmaxf(v[4], Emin);
    finite = finite && isfinite(rho) && isfinite(v[1]) && isfinite(v[2]) && isfinite(v[3]) &&
             isfinite(E) && isfinite(kin);
    Uout[q] = rho;
    Uout[n + q] = v[1];
    Uout[2 * n + q] = v[2];
    Uout[3 * n + q] = v[3];
    Uout[4 * n + q] = E;
  }
  if (!__all_sync(0xffffffffu, finite) && (threadIdx.x & 31) == 0) {
    if (rec) {
      atomicOr(&rec->flags, FLAG_NONFINITE);
      atomicCAS(&rec->fail_step, -1, (int)(rec->nstep - 1));
    } else {
      atomicOr(err, CNN_ERR_NONFINITE);
    }
  }
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long long n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

static int grid_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 148 * 8) b = 148 * 8;
  return (int)(b < 1 ? 1 : b);
}

// ---- solver-in-the-loop rollout training (Sec. 7) ---------------------------------------------
struct Weights5 {
  float iw2[5];   // 1 / w_c^2
};

// One term of the rollout loss, coef * sum over fields c and cells of ((U - T) / w_c)^2, as
// per-block partials; with lam, also its gradient 2 coef (U - T) / w_c^2, written or added.
__global__ void misfit_kernel(const float* __restrict__ U, const float* __restrict__ T, long long n,
                              Weights5 w, double coef, float* __restrict__ lam, int accumulate,
                              double* __restrict__ partial) {
  __shared__ double red[256];
  double s = 0.0;
  const long long per = (n + gridDim.x - 1) / gridDim.x;
  const long long b0 = blockIdx.x * per, b1 = b0 + per < n ? b0 + per : n;
  for (long long q = b0 + threadIdx.x; q < b1; q += blockDim.x) {
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const float d = U[c * n + q] - T[c * n + q];
      s += (double)d * (double)d * (double)w.iw2[c];
      if (lam) {
        const float g = (float)(2.0 * coef * (double)w.iw2[c]) * d;
        lam[c * n + q] = accumulate ? lam[c * n + q] + g : g;
      }
    }
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = coef * red[0];
}

// *acc += sum of partial[0..nb) in a fixed order (one warp)
__global__ void add_blocks_kernel(const double* partial, int nb, double* acc) {
  const int l = threadIdx.x;
  double s = 0.0;
  for (int b = l; b < nb; b += 32) s += partial[b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (l == 0) *acc += s;
}

// The floors of the correction transposed: lam holds dL/dU' for U' = floors(Y), Y = V + dU(V)
// (recomputed from the network output y of the forward on V exactly as correct_kernel forms
// it), and becomes dL/dY.  rho' = max(Y_rho, rho_floor) passes the gradient where
// Y_rho >= rho_floor; E' = max(Y_E, E_min), E_min = |m|^2 / (2 rho') + rho' T_floor / (gamma - 1),
// gives it to the larger argument and splits an exact tie evenly; the share of E_min flows to
// m (m / rho') and to rho' (-|m|^2 / (2 rho'^2) + T_floor / (gamma - 1)).
__global__ void floor_vjp_kernel(const float* __restrict__ V, const float* __restrict__ y,
                                 float* __restrict__ lam, long long n, const float* __restrict__ norm,
                                 float rho_floor, float T_floor, float gm1, int form, ConvGeom geo) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    float v[5];
    if (form == 0) {
#pragma unroll
      for (int c = 0; c < 5; ++c) v[c] = V[c * n + q] + norm[10 + c] * y[c * n + q];
    } else {
      int x, yy, z;
      cell_xyz(q, geo, x, yy, z);
#pragma unroll
      for (int c = 0; c < 5; ++c) v[c] = V[c * n + q] + norm[10 + c] * flux_div(y, n, geo, q, x, yy, z, c);
    }
    const float rho = fmaxf(v[0], rho_floor);
    const float kin = 0.5f * (v[1] * v[1] + v[2] * v[2] + v[3] * v[3]) / rho;
    const float Emin = kin + rho * T_floor / gm1;
    const float gE = lam[4 * n + q];
    const float gEmin = v[4] > Emin ? 0.0f : (v[4] < Emin ? gE : 0.5f * gE);
    const float grho = lam[q] + gEmin * (T_floor / gm1 - kin / rho);
    lam[q] = v[0] >= rho_floor ? grho : 0.0f;
#pragma unroll
    for (int a = 1; a <= 3; ++a) lam[a * n + q] += gEmin * v[a] / rho;
    lam[4 * n + q] = gE - gEmin;
  }
}

// Per-channel sums over `count` samples of 5 planes of n cells of A - B (B nullable): pass 1
// (mean == nullptr) sums the values, pass 2 the squared deviations from mean[c].  Block
// partials; blockIdx.y is the channel.
__global__ void moments_kernel(const float* __restrict__ A, const float* __restrict__ B,
                               long long count, long long n, const double* __restrict__ mean,
                               double* __restrict__ partial) {
  __shared__ double red[256];
  const int c = blockIdx.y;
  const long long total = count * n;
  const long long per = (total + gridDim.x - 1) / gridDim.x;
  const long long b0 = blockIdx.x * per, b1 = b0 + per < total ? b0 + per : total;
  const double m = mean ? mean[c] : 0.0;
  double s = 0.0;
  for (long long t = b0 + threadIdx.x; t < b1; t += blockDim.x) {
    const long long p = t / n, q = t - p * n;
    const long long i = (p * 5 + c) * n + q;
    const double x = (double)A[i] - (B ? (double)B[i] : 0.0);
    s += mean ? (x - m) * (x - m) : x;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[(long long)c * gridDim.x + blockIdx.x] = red[0];
}

// out[c] = scale * sum of partial[c][0..nb), one warp per channel
__global__ void channel_sums_kernel(const double* partial, int nb, double scale, double* out) {
  const int c = threadIdx.x >> 5, l = threadIdx.x & 31;
  double s = 0.0;
  for (int b = l; b < nb; b += 32) s += partial[(long long)c * nb + b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (l == 0) out[c] = scale * s;
}

__global__ void axpy_kernel(long long n, float a, const float* __restrict__ x, float* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = fmaf(a, x[i], y[i]);
}

}  // namespace dh

using namespace dh;

#define CNN_TRY(call)                                   \
  do {                                                  \
    dh_status s__ = (call);                             \
    if (s__ != DH_OK) return s__;                       \
  } while (0)

static dh_status cnn_cuda(dh_cnn* c, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return DH_OK;
  c->msg = std::string(where) + ": " + cudaGetErrorString(e);
  dh_set_global_error(c->msg);
  return DH_ERR_CUDA;
}

extern "C" void dh_cnn_destroy(dh_cnn* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream); else cudaDeviceSynchronize();
  void* ps[] = {c->params, c->norm_dev, c->pk_w1, c->pk_w2, c->pk_w3, c->pk_w2t, c->pk_w3t,
                c->pk_w1t, c->x0, c->h1, c->h2, c->z1, c->z2, c->y, c->g5, c->dy, c->dz2, c->dz1,
                c->partial, c->red, c->bpart, c->err};
  for (void* p : ps) cudaFree(p);
  delete c;
}

extern "C" dh_status dh_cnn_create_form(int nx, int ny, int nz, int form, void* stream,
                                        dh_cnn** out) {
  if (!out) return DH_ERR_ARG;
  *out = nullptr;
  if (form != 0 && form != 1) {
    dh_set_global_error("dh_cnn_create_form: form must be 0 (state) or 1 (flux)");
    return DH_ERR_ARG;
  }
  const long long n = (long long)nx * ny * nz;
  if (nx < 3 || ny < 3 || nz < 3 || n >= (1LL << 31)) {
    dh_set_global_error("dh_cnn_create: every dimension must be >= 3 and the grid below 2^31 cells");
    return DH_ERR_ARG;
  }
  const long long prow = conv_geom(nx, ny, nz).rows;   // 16-byte rows per channel group
  dh_cnn* c = new dh_cnn();
  c->nx = nx; c->ny = ny; c->nz = nz; c->ncell = n;
  c->form = form;
  c->nout = form == 0 ? 5 : 15;
  c->dyc = form == 0 ? 8 : 32;
  c->stream = (cudaStream_t)stream;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&c->nctas, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t b) { if (e == cudaSuccess) e = cudaMalloc(p, b); };
  A((void**)&c->params, nparam(c->nout) * sizeof(float));
  A((void**)&c->norm_dev, 15 * sizeof(float));
  A((void**)&c->pk_w1, 32 * 224 * 2);
  A((void**)&c->pk_w2, 32 * 864 * 2);
  A((void**)&c->pk_w3, 16 * 864 * 2);
  A((void**)&c->pk_w2t, 32 * 864 * 2);
  A((void**)&c->pk_w3t, 32 * (c->nout > 8 ? 864 : 224) * 2);
  A((void**)&c->pk_w1t, 16 * 864 * 2);
  A((void**)&c->x0, prow * 16);
  A((void**)&c->h1, prow * 4 * 16);
  A((void**)&c->h2, prow * 4 * 16);
  A((void**)&c->z1, n * 32 * 4);
  A((void**)&c->z2, n * 32 * 4);
  A((void**)&c->y, n * c->nout * 4);
  A((void**)&c->g5, n * 5 * 4);
  A((void**)&c->dy, prow * (c->dyc / 8) * 16);
  A((void**)&c->dz2, prow * 4 * 16);
  A((void**)&c->dz1, prow * 4 * 16);
  A((void**)&c->partial, (size_t)c->nctas * 7 * 128 * 32 * sizeof(float));
  A((void**)&c->red, (5 * RBLOCKS + 16) * sizeof(double));
  A((void**)&c->bpart, 32 * BG_BLOCKS * sizeof(double));
  A((void**)&c->err, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(c->err, 0, sizeof(unsigned));
  // the guard rows of the padded buffers must read as zero; every other row is rewritten by
  // the producer of the buffer (cell rows and their halo images)
  if (e == cudaSuccess) e = cudaMemset(c->x0, 0, prow * 16);
  if (e == cudaSuccess) e = cudaMemset(c->dy, 0, prow * (c->dyc / 8) * 16);
  for (__nv_bfloat16* b : {c->h1, c->h2, c->dz2, c->dz1})
    if (e == cudaSuccess) e = cudaMemset(b, 0, prow * 4 * 16);
  if (e != cudaSuccess) {
    dh_set_global_error(std::string("dh_cnn_create: ") + cudaGetErrorString(e));
    dh_cnn_destroy(c);
    return DH_ERR_CUDA;
  }
  *out = c;
  return DH_OK;
}

extern "C" dh_status dh_cnn_create(int nx, int ny, int nz, void* stream, dh_cnn** out) {
  return dh_cnn_create_form(nx, ny, nz, 0, stream, out);
}

extern "C" dh_status dh_cnn_set_params(dh_cnn* c, const float* params_dev, const float* norm15) {
  if (!c || !params_dev || !norm15) return DH_ERR_ARG;
  for (int k = 0; k < 5; ++k)
    if (!(norm15[5 + k] > 0.0f)) { dh_set_global_error("dh_cnn_set_params: sigma must be > 0"); return DH_ERR_ARG; }
  for (int k = 0; k < 15; ++k) c->norm[k] = norm15[k];
  cudaStream_t s = c->stream;
  CNN_TRY(cnn_cuda(c, cudaMemcpyAsync(c->params, params_dev, nparam(c->nout) * sizeof(float), cudaMemcpyDeviceToDevice, s), "params"));
  CNN_TRY(cnn_cuda(c, cudaMemcpyAsync(c->norm_dev, c->norm, 15 * sizeof(float), cudaMemcpyHostToDevice, s), "norm"));
  CNN_TRY(dh_pack_conv_weights(c->params + OFF_W1, 32, 5, 0, c->pk_w1, s));
  CNN_TRY(dh_pack_conv_weights(c->params + OFF_W2, 32, 32, 0, c->pk_w2, s));
  CNN_TRY(dh_pack_conv_weights(c->params + OFF_W3, c->nout, 32, 0, c->pk_w3, s));
  CNN_TRY(dh_pack_conv_weights(c->params + OFF_W2, 32, 32, 1, c->pk_w2t, s));
  CNN_TRY(dh_pack_conv_weights(c->params + OFF_W3, c->nout, 32, 1, c->pk_w3t, s));
  CNN_TRY(dh_pack_conv_weights(c->params + OFF_W1, 32, 5, 1, c->pk_w1t, s));
  CNN_TRY(cnn_cuda(c, cudaStreamSynchronize(s), "set_params"));
  c->have_params = true;
  return DH_OK;
}

static dh_status check_err(dh_cnn* c) {
  unsigned h = 0;
  CNN_TRY(cnn_cuda(c, cudaMemcpyAsync(&h, c->err, sizeof(h), cudaMemcpyDeviceToHost, c->stream), "err"));
  CNN_TRY(cnn_cuda(c, cudaStreamSynchronize(c->stream), "sync"));
  if (h) {
    cudaMemsetAsync(c->err, 0, sizeof(unsigned), c->stream);
    if (h & CNN_ERR_WAIT) {
      dh_set_global_error("corrector: a bounded tensor-core wait gave up");
      return DH_ERR_CUDA;
    }
    dh_set_global_error("corrector: the corrected state is not finite");
    return DH_ERR_NONFINITE;
  }
  return DH_OK;
}

// The forward pass; keep_z stores the pre-activations z1, z2 that back-propagation needs
// (an inference pass skips those 256 bytes per cell of writes).
static dh_status cnn_forward(dh_cnn* c, const float* U, float* y_out, bool keep_z) {
  if (!c || !U) return DH_ERR_ARG;
  if (!c->have_params) { dh_set_global_error("dh_cnn_forward: parameters not set"); return DH_ERR_STATE; }
  const long long n = c->ncell;
  cudaStream_t s = c->stream;
  c->have_forward = false;
  normalize_kernel<<<grid_for(n), 256, 0, s>>>(U, conv_geom(c->nx, c->ny, c->nz), c->norm_dev, c->x0);
  CNN_TRY(cnn_cuda(c, cudaGetLastError(), "normalize"));
  CNN_TRY(dh_conv3d_bf16(c->x0, 8, c->pk_w1, 32, c->params + OFF_B1, 0, nullptr, c->h1, keep_z ? c->z1 : nullptr, 32, c->nx, c->ny, c->nz, c->err, s));
  CNN_TRY(dh_conv3d_bf16(c->h1, 32, c->pk_w2, 32, c->params + OFF_B2, 0, nullptr, c->h2, keep_z ? c->z2 : nullptr, 32, c->nx, c->ny, c->nz, c->err, s));
  CNN_TRY(dh_conv3d_bf16(c->h2, 32, c->pk_w3, 16, c->params + off_b3(c->nout), 1, nullptr, c->y, nullptr, c->nout, c->nx, c->ny, c->nz, c->err, s));
  if (y_out) CNN_TRY(cnn_cuda(c, cudaMemcpyAsync(y_out, c->y, n * c->nout * sizeof(float), cudaMemcpyDeviceToDevice, s), "y"));
  c->have_forward = keep_z;
  return DH_OK;
}

extern "C" dh_status dh_cnn_forward(dh_cnn* c, const float* U, float* y_out) {
  return cnn_forward(c, U, y_out, true);
}

// Back-propagation from the output gradient already in c->dy, for the last forward: parameter
// gradients into grads; with dLdU (nullable) also the gradient of the network input U.
static dh_status backprop(dh_cnn* c, float* grads, float* dLdU) {
  cudaStream_t s = c->stream;
  const ConvGeom geo = conv_geom(c->nx, c->ny, c->nz);
  const int nb3 = off_b3(c->nout);
  // output layer
  CNN_TRY(dh_conv3d_wgrad_bf16(c->h2, 32, 32, c->dy, c->dyc, c->nout, c->nx, c->ny, c->nz, c->partial, c->nctas, grads + OFF_W3, c->err, s));
  if (c->form == 0) {
    bias_grad(c->dy, c->dyc / 8, c->nout, geo, c->bpart, grads + nb3, s);
  } else {
    // a constant flux has no divergence: b3 does not enter the flux-form correction (its exact
    // gradient is zero; summing the bf16 output gradient would only add rounding noise)
    CNN_TRY(cnn_cuda(c, cudaMemsetAsync(grads + nb3, 0, c->nout * sizeof(float), s), "b3 grad"));
  }
  CNN_TRY(dh_conv3d_bf16(c->dy, c->dyc, c->pk_w3t, 32, nullptr, 2, c->z2, c->dz2, nullptr, 32, c->nx, c->ny, c->nz, c->err, s));
  // hidden layer
  CNN_TRY(dh_conv3d_wgrad_bf16(c->h1, 32, 32, c->dz2, 32, 32, c->nx, c->ny, c->nz, c->partial, c->nctas, grads + OFF_W2, c->err, s));
  bias_grad(c->dz2, 4, 32, geo, c->bpart, grads + OFF_B2, s);
  CNN_TRY(dh_conv3d_bf16(c->dz2, 32, c->pk_w2t, 32, nullptr, 2, c->z1, c->dz1, nullptr, 32, c->nx, c->ny, c->nz, c->err, s));
  // first layer
  CNN_TRY(dh_conv3d_wgrad_bf16(c->x0, 8, 5, c->dz1, 32, 32, c->nx, c->ny, c->nz, c->partial, c->nctas, grads + OFF_W1, c->err, s));
  bias_grad(c->dz1, 4, 32, geo, c->bpart, grads + OFF_B1, s);
  if (dLdU) {
    // input: dL/dx0 = conv(dz1, W1 transposed), then the normalisation transposed
    CNN_TRY(dh_conv3d_bf16(c->dz1, 32, c->pk_w1t, 16, nullptr, 1, nullptr, dLdU, nullptr, 5, c->nx, c->ny, c->nz, c->err, s));
    input_grad_kernel<<<grid_for(5 * c->ncell), 256, 0, s>>>(dLdU, c->norm_dev, c->ncell);
  }
  return cnn_cuda(c, cudaGetLastError(), "backward");
}

extern "C" dh_status dh_cnn_backward(dh_cnn* c, const float* U_in, const float* U_target,
                                     float* grads, double* loss) {
  if (!c || !U_in || !U_target || !grads) return DH_ERR_ARG;
  if (!c->have_forward) { dh_set_global_error("dh_cnn_backward: run dh_cnn_forward first"); return DH_ERR_STATE; }
  const long long n = c->ncell;
  cudaStream_t s = c->stream;
  const ConvGeom geo = conv_geom(c->nx, c->ny, c->nz);
  if (c->form == 0) {
    mse_grad_kernel<<<RBLOCKS, 256, 0, s>>>(c->y, U_in, U_target, c->norm_dev, geo, c->dy, c->red);
  } else {
    flux_mse_kernel<<<RBLOCKS, 256, 0, s>>>(c->y, U_in, U_target, c->norm_dev, geo, c->g5, c->red);
    output_grad_kernel<<<grid_for(n), 256, 0, s>>>(c->g5, nullptr, 1, geo, c->dy);
  }
  sum_blocks_kernel<<<1, 32, 0, s>>>(c->red, RBLOCKS, 1.0 / (5.0 * (double)n), c->red + RBLOCKS);
  CNN_TRY(backprop(c, grads, nullptr));
  if (loss) CNN_TRY(cnn_cuda(c, cudaMemcpyAsync(loss, c->red + RBLOCKS, sizeof(double), cudaMemcpyDeviceToHost, s), "loss"));
  return check_err(c);
}

extern "C" dh_status dh_cnn_vjp(dh_cnn* c, const float* dL_dcorr, float* grads, float* dL_dU) {
  if (!c || !dL_dcorr || !grads) return DH_ERR_ARG;
  if (!c->have_forward) { dh_set_global_error("dh_cnn_vjp: run dh_cnn_forward first"); return DH_ERR_STATE; }
  const ConvGeom geo = conv_geom(c->nx, c->ny, c->nz);
  output_grad_kernel<<<grid_for(c->ncell), 256, 0, c->stream>>>(dL_dcorr, c->norm_dev + 10, c->form,
                                                                geo, c->dy);
  CNN_TRY(backprop(c, grads, dL_dU));
  return check_err(c);
}

static dh_status cnn_correct(dh_cnn* c, const float* Uin, float* Uout, double rho_floor,
                             const double* totals, double floor_per_mass, double T_floor,
                             double gamma) {
  if (!c || !Uin || !Uout) return DH_ERR_ARG;
  CNN_TRY(cnn_forward(c, Uin, nullptr, false));
  correct_kernel<<<grid_for(c->ncell), 256, 0, c->stream>>>(Uin, Uout, c->y, c->ncell, c->norm_dev,
                                                            (float)rho_floor, totals,
                                                            floor_per_mass, (float)T_floor,
                                                            (float)(gamma - 1.0), c->err, c->form,
                                                            conv_geom(c->nx, c->ny, c->nz), nullptr);
  CNN_TRY(cnn_cuda(c, cudaGetLastError(), "correct"));
  return check_err(c);
}

namespace dh {
cudaError_t correct_in_step(dh_ctx* ctx, float* U) {
  dh_cnn* c = ctx->cnn;
  // rho floor: 1e-6 of the mean density of the uncorrected state (FP64 totals on the device)
  cudaError_t e = launch_totals<float>(U, ctx->n3, ctx->partials, totals_blocks(), ctx->totals,
                                       ctx->stream);
  if (e != cudaSuccess) return e;
  if (cnn_forward(c, U, nullptr, false) != DH_OK) return cudaErrorLaunchFailure;
  correct_kernel<<<grid_for(c->ncell), 256, 0, c->stream>>>(
      U, U, c->y, c->ncell, c->norm_dev, 0.0f, ctx->totals, 1e-6 / (double)ctx->n3,
      (float)ctx->cfg.t_floor, (float)(ctx->cfg.gamma - 1.0), c->err, c->form,
      conv_geom(c->nx, c->ny, c->nz), ctx->rec);
  ctx->launches += 7;   // totals (2), normalise, three convolutions, correction
  return cudaGetLastError();
}
}  // namespace dh

extern "C" dh_status dh_set_correct_every_step(dh_ctx* ctx, int on) {
  if (!ctx) return DH_ERR_ARG;
  if (on && (!ctx->cnn || !ctx->cnn->have_params)) { ctx->err = "no corrector set"; return DH_ERR_STATE; }
  ctx->correct_each_step = on != 0;
  return DH_OK;
}

extern "C" dh_status dh_cnn_correct_state(dh_cnn* c, float* U, double rho_floor, double T_floor,
                                          double gamma) {
  return cnn_correct(c, U, U, rho_floor, nullptr, 0.0, T_floor, gamma);
}

extern "C" dh_status dh_adam_step(float* params, const float* grads, float* m, float* v, long long n,
                                  double lr, double beta1, double beta2, double eps, int step,
                                  void* stream) {
  if (!params || !grads || !m || !v || n < 1 || step < 1) return DH_ERR_ARG;
  const float c1 = (float)(1.0 - pow(beta1, step)), c2 = (float)(1.0 - pow(beta2, step));
  adam_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(params, grads, m, v, n, (float)lr,
                                                             (float)beta1, (float)beta2,
                                                             (float)eps, c1, c2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { dh_set_global_error(cudaGetErrorString(e)); return DH_ERR_CUDA; }
  return DH_OK;
}

extern "C" dh_status dh_cnn_rollout_misfit(dh_cnn* c, const float* U, const float* T,
                                           const float* w5, double coef, float* lam,
                                           int accumulate, double* loss_acc) {
  if (!c || !U || !T || !w5) return DH_ERR_ARG;
  Weights5 w;
  for (int k = 0; k < 5; ++k) {
    if (!(w5[k] > 0.0f)) { dh_set_global_error("dh_cnn_rollout_misfit: weights must be positive"); return DH_ERR_ARG; }
    w.iw2[k] = 1.0f / (w5[k] * w5[k]);
  }
  misfit_kernel<<<RBLOCKS, 256, 0, c->stream>>>(U, T, c->ncell, w, coef, lam, accumulate, c->red);
  if (loss_acc) add_blocks_kernel<<<1, 32, 0, c->stream>>>(c->red, RBLOCKS, loss_acc);
  return cnn_cuda(c, cudaGetLastError(), "rollout misfit");
}

extern "C" dh_status dh_cnn_floor_vjp(dh_cnn* c, const float* V, float* lam, double rho_floor,
                                      double T_floor, double gamma) {
  if (!c || !V || !lam) return DH_ERR_ARG;
  if (!c->have_forward) { dh_set_global_error("dh_cnn_floor_vjp: run dh_cnn_forward on V first"); return DH_ERR_STATE; }
  floor_vjp_kernel<<<grid_for(c->ncell), 256, 0, c->stream>>>(
      V, c->y, lam, c->ncell, c->norm_dev, (float)rho_floor, (float)T_floor, (float)(gamma - 1.0),
      c->form, conv_geom(c->nx, c->ny, c->nz));
  return cnn_cuda(c, cudaGetLastError(), "floor vjp");
}

extern "C" dh_status dh_cnn_field_moments(dh_cnn* c, const float* A, const float* B, long long count,
                                          double* out10) {
  if (!c || !A || !out10 || count < 1) return DH_ERR_ARG;
  const long long N = count * c->ncell;
  if (N < 2) { dh_set_global_error("dh_cnn_field_moments: need at least two values per channel"); return DH_ERR_ARG; }
  double* res = c->red + 5 * RBLOCKS;   // 5 means, then 5 standard deviations
  cudaStream_t s = c->stream;
  moments_kernel<<<dim3(RBLOCKS, 5), 256, 0, s>>>(A, B, count, c->ncell, nullptr, c->red);
  channel_sums_kernel<<<1, 160, 0, s>>>(c->red, RBLOCKS, 1.0 / (double)N, res);
  moments_kernel<<<dim3(RBLOCKS, 5), 256, 0, s>>>(A, B, count, c->ncell, res, c->red);
  channel_sums_kernel<<<1, 160, 0, s>>>(c->red, RBLOCKS, 1.0 / (double)(N - 1), res + 5);
  CNN_TRY(cnn_cuda(c, cudaMemcpyAsync(out10, res, 10 * sizeof(double), cudaMemcpyDeviceToHost, s), "moments"));
  CNN_TRY(cnn_cuda(c, cudaStreamSynchronize(s), "moments"));
  for (int k = 5; k < 10; ++k) out10[k] = sqrt(out10[k]);
  return DH_OK;
}

extern "C" dh_status dh_axpy(long long n, double a, const float* x, float* y, void* stream) {
  if (!x || !y || n < 0) return DH_ERR_ARG;
  if (n == 0) return DH_OK;
  axpy_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(n, (float)a, x, y);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { dh_set_global_error(cudaGetErrorString(e)); return DH_ERR_CUDA; }
  return DH_OK;
}

extern "C" long long dh_cnn_param_count(void) { return NPARAM; }
extern "C" long long dh_cnn_param_count_form(int form) { return form == 1 ? nparam(15) : nparam(5); }

// ---- the context's corrector -------------------------------------------------------------------
extern "C" dh_status dh_set_corrector_form(dh_ctx* ctx, int form, const float* params_dev,
                                           const float* norm15) {
  if (!ctx || !params_dev || !norm15) return DH_ERR_ARG;
  if (ctx->prec != DH_F32) { ctx->err = "the corrector runs on float32 states"; return DH_ERR_ARG; }
  if (form != 0 && form != 1) { ctx->err = "form must be 0 (state) or 1 (flux)"; return DH_ERR_ARG; }
  if (ctx->cnn && ctx->cnn->form != form) {
    dh_cnn_destroy(ctx->cnn);
    ctx->cnn = nullptr;
  }
  if (!ctx->cnn) {
    dh_status st = dh_cnn_create_form(ctx->cfg.nx, ctx->cfg.ny, ctx->cfg.nz, form, ctx->stream, &ctx->cnn);
    if (st != DH_OK) { ctx->err = dh_last_error(nullptr); return st; }
  }
  dh_status st = dh_cnn_set_params(ctx->cnn, params_dev, norm15);
  if (st != DH_OK) ctx->err = dh_last_error(nullptr);
  return st;
}

extern "C" dh_status dh_set_corrector(dh_ctx* ctx, const float* params_dev, const float* norm15) {
  return dh_set_corrector_form(ctx, 0, params_dev, norm15);
}

extern "C" dh_status dh_correct(dh_ctx* ctx) {
  if (!ctx) return DH_ERR_ARG;
  if (!ctx->cnn || !ctx->cnn->have_params) { ctx->err = "no corrector set"; return DH_ERR_STATE; }
  if (!ctx->initialized) { ctx->err = "state not initialised"; return DH_ERR_STATE; }
  // settle enqueued steps: their rollback bookkeeping assumes no other buffer swap
  if (ctx->pending_steps > 0) {
    dh_status s0 = dh_finish_steps(ctx);
    if (s0 != DH_OK) return s0;
  }
  // rho floor: 1e-6 of the mean density, from FP64 totals that stay on the device
  const float* U = (const float*)ctx->U[ctx->cur];
  float* V = (float*)ctx->U[1 - ctx->cur];
  cudaError_t e = launch_totals<float>(U, ctx->n3, ctx->partials, totals_blocks(), ctx->totals,
                                       ctx->stream);
  if (e != cudaSuccess) { ctx->err = cudaGetErrorString(e); return DH_ERR_CUDA; }
  // the corrected state goes to the other buffer and becomes current only if it is finite
  dh_status st = cnn_correct(ctx->cnn, U, V, 0.0, ctx->totals, 1e-6 / (double)ctx->n3,
                             ctx->cfg.t_floor, ctx->cfg.gamma);
  if (st != DH_OK) { ctx->err = dh_last_error(nullptr); return st; }
  ctx->cur = 1 - ctx->cur;
  // the state changed: the next CFL step must see it
  return dh_refresh_cfl(ctx);
}
