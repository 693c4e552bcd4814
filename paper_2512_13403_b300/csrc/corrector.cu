// Residual 3D convolutional corrector on the tensor cores (BF16 operands, FP32 accumulation).
//
// Every 3x3x3 periodic convolution is an implicit GEMM: D[cell, n] = sum_k A[cell, k] B[n, k]
// with k = (tap, input channel), A gathered from the 27 neighbours of each cell and B the packed
// weights.  A persistent CTA of 128 threads walks 128-cell tiles (M = 128); for each 16-wide
// K step the threads gather A into a 4-stage shared-memory ring (no-swizzle K-major core
// matrices), one elected thread issues tcgen05.mma into a TMEM accumulator (128 lanes x N FP32
// columns) and commits to the stage's mbarrier; B (all taps) stays resident in shared memory.
// The epilogue reads TMEM with tcgen05.ld (one row per thread) and fuses bias + GELU, the
// GELU derivative (backward), or the linear output.  The same kernel computes the backward
// data gradient with tap-flipped, channel-transposed weights.
//
// Channel-last activations: bf16 [cell][C], C = 8 (5 state channels padded) or 32.
// K layout: k = tap * C + c, tap = (dz+1)*9 + (dy+1)*3 + (dx+1); for C = 8 a 16-wide K step
// holds two taps (tap 27 is a zero pad), for C = 32 half a tap.
#include <cuda_bf16.h>
#include <math.h>

#include "dh_internal.h"
#include "tc_ptx.cuh"

namespace dh {

constexpr int CV_THREADS = 128;
constexpr int CV_STAGES = 4;
constexpr int CV_STAGE_BYTES = 128 * 16 * 2;   // 128 rows x 16 bf16
constexpr uint32_t CV_WAIT_ITERS = 1u << 22;   // bounded mbarrier waits

enum ConvMode : int {
  CONV_GELU = 0,        // out_bf16 = bf16(gelu(acc + bias)); z_out = acc + bias (fp32)
  CONV_LINEAR = 1,      // out_f32 planar [c][cell] = acc + bias for c < n_real
  CONV_GELU_GRAD = 2,   // out_bf16 = bf16(acc * gelu'(z_in))
};

__device__ __forceinline__ float gelu_exact(float z) {
  return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad(float z) {
  // d/dz [z Phi(z)] = Phi(z) + z phi(z)
  const float Phi = 0.5f * (1.0f + erff(z * 0.70710678118654752f));
  const float phi = 0.39894228040143268f * expf(-0.5f * z * z);
  return Phi + z * phi;
}

struct ConvArgs {
  const __nv_bfloat16* act;   // [cells][CIN]
  const __nv_bfloat16* wpk;   // packed B, [NOUT/8][K/8][8][8] bf16
  const float* bias;          // [NOUT] (nullable: zero)
  const float* z_in;          // [cells][32] fp32, CONV_GELU_GRAD
  __nv_bfloat16* out_bf16;    // [cells][NOUT] for GELU modes
  float* out_f32;             // planar [n_real][cells] for CONV_LINEAR
  float* z_out;               // [cells][NOUT] fp32 (nullable) for CONV_GELU
  int n_real;                 // real output channels (CONV_LINEAR)
  int nx, ny, nz;
  unsigned* err;              // set to 1 if a bounded wait gave up
};

template <int CIN, int NOUT, int MODE>
__global__ void __launch_bounds__(CV_THREADS)
conv3d_tc_kernel(const ConvArgs p) {
  constexpr int K = CIN == 32 ? 27 * 32 : 28 * 8;      // padded reduction length
  constexpr int KSTEPS = K / 16;
  constexpr int B_BYTES = NOUT * K * 2;
  constexpr uint32_t TMEM_COLS = 32;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sB = smem;                              // resident weights
  unsigned char* sA = smem + B_BYTES;                    // stage ring
  uint64_t* bars = reinterpret_cast<uint64_t*>(sA + CV_STAGES * CV_STAGE_BYTES);
  uint64_t* bar_done = bars + CV_STAGES;
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bar_done + 1);
  __shared__ int s_abort;

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const long long ncell = (long long)p.nx * p.ny * p.nz;
  const int ntiles = (int)(ncell / 128);

  // weights -> shared memory (same packed layout)
  {
    const uint4* src = reinterpret_cast<const uint4*>(p.wpk);
    uint4* dst = reinterpret_cast<uint4*>(sB);
    for (int i = tid; i < B_BYTES / 16; i += CV_THREADS) dst[i] = __ldg(src + i);
  }
  if (tid == 0) {
    for (int b = 0; b < CV_STAGES; ++b) tc::mbar_init(&bars[b], 1);
    tc::mbar_init(bar_done, 1);
    tc::mbar_fence_init();
    s_abort = 0;
  }
  if (warp == 0) {
    tc::tmem_alloc(s_tmem, TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::fence_async_smem();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *s_tmem;
  const uint32_t idesc = tc::idesc_bf16_f32(128, NOUT);
  const uint32_t sA_addr = tc::smem_u32(sA);
  const uint32_t sB_addr = tc::smem_u32(sB);

  uint32_t phase_bits = 0;   // parity of the next wait, per stage
  uint32_t done_phase = 0;
  long long it = 0;          // running K-step counter across tiles

  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    // the cell of this thread's A row
    const long long q = (long long)tile * 128 + tid;
    const int i = (int)(q % p.nx);
    const long long t1 = q / p.nx;
    const int j = (int)(t1 % p.ny);
    const int k = (int)(t1 / p.ny);

    for (int s = 0; s < KSTEPS; ++s, ++it) {
      const int b = (int)(it % CV_STAGES);
      if (it >= CV_STAGES) {
        if (!tc::mbar_wait(&bars[b], (phase_bits >> b) & 1u, CV_WAIT_ITERS)) s_abort = 1;
        phase_bits ^= 1u << b;
      }
      // gather the two 16-byte core-matrix rows of this thread (kg = 0, 1)
      unsigned char* stage = sA + b * CV_STAGE_BYTES;
#pragma unroll
      for (int kg = 0; kg < 2; ++kg) {
        int tap, c0;
        if (CIN == 32) { tap = s >> 1; c0 = (s & 1) * 16 + kg * 8; }
        else { tap = 2 * s + kg; c0 = 0; }
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (tap < 27) {
          const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
          const int ii = wrap(i + dx, p.nx), jj = wrap(j + dy, p.ny), kk = wrap(k + dz, p.nz);
          const long long nq = ((long long)kk * p.ny + jj) * p.nx + ii;
          v = __ldg(reinterpret_cast<const uint4*>(p.act + nq * CIN + c0));
        }
        const int off = (((tid >> 3) * 2 + kg) * 8 + (tid & 7)) * 16;
        *reinterpret_cast<uint4*>(stage + off) = v;
      }
      tc::fence_async_smem();
      __syncthreads();
      if (s_abort) break;
      if (tid == 0) {
        tc::tc_fence_after();
        const uint64_t adesc = tc::smem_desc(sA_addr + b * CV_STAGE_BYTES, 128, 256);
        const uint64_t bdesc = tc::smem_desc(sB_addr + s * 256, 128, (K / 8) * 128);
        tc::mma_bf16(tmem, adesc, bdesc, idesc, s > 0 ? 1u : 0u);
        tc::mma_commit(&bars[b]);
        if (s == KSTEPS - 1) tc::mma_commit(bar_done);
      }
    }
    if (s_abort) break;
    if (!tc::mbar_wait(bar_done, done_phase, CV_WAIT_ITERS)) s_abort = 1;
    done_phase ^= 1u;
    __syncthreads();
    if (s_abort) break;
    tc::tc_fence_after();

    // epilogue: this thread owns TMEM lane `tid` (warp w reads lanes 32w..32w+31)
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
    if (NOUT == 32) {
      float acc[32];
      tc::tmem_ld_32x32b_x32(taddr, acc);
      tc::tmem_ld_wait();
      if (MODE == CONV_GELU) {
        __align__(16) __nv_bfloat16 hv[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          const float z = acc[c] + (p.bias ? __ldg(p.bias + c) : 0.0f);
          if (p.z_out) p.z_out[q * 32 + c] = z;
          hv[c] = __float2bfloat16_rn(gelu_exact(z));
        }
        uint4* dst = reinterpret_cast<uint4*>(p.out_bf16 + q * 32);
#pragma unroll
        for (int v4 = 0; v4 < 4; ++v4) dst[v4] = reinterpret_cast<const uint4*>(hv)[v4];
      } else if (MODE == CONV_GELU_GRAD) {
        __align__(16) __nv_bfloat16 hv[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) hv[c] = __float2bfloat16_rn(acc[c] * gelu_grad(__ldg(p.z_in + q * 32 + c)));
        uint4* dst = reinterpret_cast<uint4*>(p.out_bf16 + q * 32);
#pragma unroll
        for (int v4 = 0; v4 < 4; ++v4) dst[v4] = reinterpret_cast<const uint4*>(hv)[v4];
      } else {
        for (int c = 0; c < p.n_real; ++c)
          p.out_f32[(long long)c * ncell + q] = acc[c] + (p.bias ? __ldg(p.bias + c) : 0.0f);
      }
    } else {
      float acc[16];
      tc::tmem_ld_32x32b_x16(taddr, acc);
      tc::tmem_ld_wait();
      for (int c = 0; c < p.n_real && c < 16; ++c)
        p.out_f32[(long long)c * ncell + q] = acc[c] + (p.bias ? __ldg(p.bias + c) : 0.0f);
    }
    tc::tc_fence_before();
    __syncthreads();
  }

  // drain: every MMA issued must be complete before the accumulator is released.  Normally
  // the last tile's completion was awaited above; after an abort, commit once more and give the
  // tensor cores a bounded wait before freeing TMEM.
  if (s_abort) {
    if (tid == 0) {
      atomicOr(p.err, 1u);
      tc::mma_commit(bar_done);
    }
    tc::mbar_wait(bar_done, done_phase, CV_WAIT_ITERS);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, TMEM_COLS);
  }
}

template <int CIN, int NOUT, int MODE>
static cudaError_t launch_conv(const ConvArgs& a, int max_ctas, cudaStream_t s) {
  constexpr int K = CIN == 32 ? 27 * 32 : 28 * 8;
  const size_t smem = (size_t)NOUT * K * 2 + CV_STAGES * CV_STAGE_BYTES + 8 * (CV_STAGES + 1) + 16;
  cudaError_t e = cudaFuncSetAttribute(conv3d_tc_kernel<CIN, NOUT, MODE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long ncell = (long long)a.nx * a.ny * a.nz;
  int ntiles = (int)(ncell / 128);
  int grid = ntiles < max_ctas ? ntiles : max_ctas;
  if (grid < 1) grid = 1;
  conv3d_tc_kernel<CIN, NOUT, MODE><<<grid, CV_THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Weight packing: master fp32 W[cout][cin][27] (torch conv3d order [o][i][kz][ky][kx]) into the
// K-major core-matrix layout of B.  forward: n = cout, k = tap * cin_pad + cin.
// data gradient: n = cin, k = tap' * cout_pad + cout with tap' = 26 - tap (mirrored offsets).
__global__ void pack_conv_weights_kernel(const float* __restrict__ W, int cout, int cin,
                                         int transpose_flip, int n_pad, int c_pad, int k_pad,
                                         __nv_bfloat16* __restrict__ out) {
  const long long total = (long long)n_pad * k_pad;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int n = (int)(idx / k_pad), kk = (int)(idx % k_pad);
    const int tap = kk / c_pad, c = kk % c_pad;
    float v = 0.0f;
    if (tap < 27) {
      if (!transpose_flip) {
        if (n < cout && c < cin) v = W[((long long)n * cin + c) * 27 + tap];
      } else {
        // n = input channel of the forward layer, c = its output channel
        if (n < cin && c < cout) v = W[((long long)c * cin + n) * 27 + (26 - tap)];
      }
    }
    const long long o = ((((long long)(n >> 3) * (k_pad >> 3) + (kk >> 3)) * 8 + (n & 7)) * 8) + (kk & 7);
    out[o] = __float2bfloat16_rn(v);
  }
}

}  // namespace dh

using namespace dh;

extern "C" dh_status dh_pack_conv_weights(const float* W, int cout, int cin, int transpose_flip,
                                          void* packed, void* stream) {
  if (!W || !packed) return DH_ERR_ARG;
  const int n_real = transpose_flip ? cin : cout;
  const int c_real = transpose_flip ? cout : cin;
  if (!(n_real == 32 || n_real <= 16) || c_real > 32 || n_real < 1 || c_real < 1) {
    dh_set_global_error("dh_pack_conv_weights: output channels must be 32 or <= 16, inputs <= 32");
    return DH_ERR_ARG;
  }
  const int n_pad = n_real == 32 ? 32 : 16;
  const int c_pad = c_real > 8 ? 32 : 8;
  const int k_pad = c_pad == 32 ? 27 * 32 : 28 * 8;
  pack_conv_weights_kernel<<<64, 256, 0, (cudaStream_t)stream>>>(W, cout, cin, transpose_flip,
                                                                  n_pad, c_pad, k_pad,
                                                                  (__nv_bfloat16*)packed);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { dh_set_global_error(cudaGetErrorString(e)); return DH_ERR_CUDA; }
  return DH_OK;
}

extern "C" dh_status dh_conv3d_bf16(const void* act, int cin_pad, const void* packed, int nout_pad,
                                    const float* bias, int mode, const float* z_in, void* out,
                                    float* z_out, int n_real, int nx, int ny, int nz,
                                    unsigned* err_flag, void* stream) {
  if (!act || !packed || !out || !err_flag) return DH_ERR_ARG;
  const long long ncell = (long long)nx * ny * nz;
  if (nx < 3 || ny < 3 || nz < 3 || ncell % 128 != 0) {
    dh_set_global_error("dh_conv3d_bf16: needs every dimension >= 3 and nx*ny*nz divisible by 128");
    return DH_ERR_ARG;
  }
  ConvArgs a;
  a.act = (const __nv_bfloat16*)act;
  a.wpk = (const __nv_bfloat16*)packed;
  a.bias = bias;
  a.z_in = z_in;
  a.out_bf16 = (__nv_bfloat16*)out;
  a.out_f32 = (float*)out;
  a.z_out = z_out;
  a.n_real = n_real;
  a.nx = nx; a.ny = ny; a.nz = nz;
  a.err = err_flag;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int max_ctas = 2 * sms;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaErrorInvalidValue;
  if (cin_pad == 8 && nout_pad == 32 && mode == CONV_GELU) e = launch_conv<8, 32, CONV_GELU>(a, max_ctas, s);
  else if (cin_pad == 8 && nout_pad == 32 && mode == CONV_GELU_GRAD) e = launch_conv<8, 32, CONV_GELU_GRAD>(a, max_ctas, s);
  else if (cin_pad == 32 && nout_pad == 32 && mode == CONV_GELU) e = launch_conv<32, 32, CONV_GELU>(a, max_ctas, s);
  else if (cin_pad == 32 && nout_pad == 32 && mode == CONV_GELU_GRAD) e = launch_conv<32, 32, CONV_GELU_GRAD>(a, max_ctas, s);
  else if (cin_pad == 32 && nout_pad == 16 && mode == CONV_LINEAR) e = launch_conv<32, 16, CONV_LINEAR>(a, max_ctas, s);
  else if (cin_pad == 32 && nout_pad == 32 && mode == CONV_LINEAR) e = launch_conv<32, 32, CONV_LINEAR>(a, max_ctas, s);
  else {
    dh_set_global_error("dh_conv3d_bf16: unsupported (cin_pad, nout_pad, mode) combination");
    return DH_ERR_ARG;
  }
  if (e != cudaSuccess) { dh_set_global_error(cudaGetErrorString(e)); return DH_ERR_CUDA; }
  return DH_OK;
}

// =============================================================================================
// Weight gradient: dW[n][c][tap] = sum_cells g[cell][n] * act[cell + offset(tap)][c], a GEMM
// with M = (tap, c) rows (27 * CIN, in tiles of 128), N = n, K = cells.  Each CTA reduces a
// contiguous range of cells in 16-cell K steps: the threads gather, for every tap, the 16
// neighbour rows and transpose them into K-major core matrices (a row holds one (tap, c) over
// 16 consecutive cells), the gradient rows likewise; one thread issues one MMA per M tile into
// its own TMEM accumulator.  Per-CTA partial sums go to global memory and a second kernel adds
// them in a fixed order.
namespace dh {

constexpr int WG_THREADS = 128;
constexpr int WG_STAGES = 2;

template <int CIN, int NOUT>
__global__ void __launch_bounds__(WG_THREADS)
conv3d_wgrad_tc_kernel(const __nv_bfloat16* __restrict__ act, const __nv_bfloat16* __restrict__ g,
                       int g_stride, int nx, int ny, int nz, long long cells_per_cta,
                       float* __restrict__ partial, unsigned* err) {
  constexpr int MROWS = 27 * CIN;
  constexpr int MT = (MROWS + 127) / 128;           // M tiles
  constexpr int A_TILE = 128 * 16 * 2;              // bytes per M tile per stage
  constexpr int B_TILE = NOUT * 16 * 2;
  constexpr int STAGE = MT * A_TILE + B_TILE;
  constexpr uint32_t TMEM_COLS = MT * NOUT <= 32 ? 32 : (MT * NOUT <= 64 ? 64 : (MT * NOUT <= 128 ? 128 : 256));
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + WG_STAGES * STAGE);
  uint64_t* bar_done = bars + WG_STAGES;
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bar_done + 1);
  __shared__ int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5;
  const long long ncell = (long long)nx * ny * nz;
  const long long c0 = (long long)blockIdx.x * cells_per_cta;
  const long long c1 = c0 + cells_per_cta < ncell ? c0 + cells_per_cta : ncell;
  const int ksteps = c1 > c0 ? (int)((c1 - c0 + 15) / 16) : 0;

  // zero both stages once: padding rows (beyond 27 * CIN) and tail cells stay zero
  for (int i = tid; i < WG_STAGES * STAGE / 16; i += WG_THREADS)
    reinterpret_cast<uint4*>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    for (int b = 0; b < WG_STAGES; ++b) tc::mbar_init(&bars[b], 1);
    tc::mbar_init(bar_done, 1);
    tc::mbar_fence_init();
    s_abort = 0;
  }
  if (warp == 0) {
    tc::tmem_alloc(s_tmem, TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::fence_async_smem();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *s_tmem;
  const uint32_t idesc = tc::idesc_bf16_f32(128, NOUT);
  const uint32_t s_addr = tc::smem_u32(smem);
  uint32_t phase_bits = 0;

  for (int s = 0; s < ksteps; ++s) {
    const int b = s % WG_STAGES;
    if (s >= WG_STAGES) {
      if (!tc::mbar_wait(&bars[b], (phase_bits >> b) & 1u, CV_WAIT_ITERS)) s_abort = 1;
      phase_bits ^= 1u << b;
    }
    unsigned char* st = smem + b * STAGE;
    const long long x0 = c0 + 16LL * s;
    // A: items (tap, channel group of 8, cell k); each loads 8 channels and scatters them
    for (int it = tid; it < 27 * (CIN / 8) * 16; it += WG_THREADS) {
      const int k = it & 15;
      const int rest = it >> 4;
      const int cg = rest % (CIN / 8), tap = rest / (CIN / 8);
      const long long x = x0 + k;
      __align__(16) __nv_bfloat16 v[8];
      if (x < c1) {
        const int i = (int)(x % nx);
        const long long t1 = x / nx;
        const int j = (int)(t1 % ny), kz = (int)(t1 / ny);
        const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
        const long long nq = ((long long)wrap(kz + dz, nz) * ny + wrap(j + dy, ny)) * nx + wrap(i + dx, nx);
        *reinterpret_cast<uint4*>(v) = __ldg(reinterpret_cast<const uint4*>(act + nq * CIN + cg * 8));
      } else {
        *reinterpret_cast<uint4*>(v) = make_uint4(0u, 0u, 0u, 0u);
      }
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int m = tap * CIN + cg * 8 + e;       // A row
        const int t = m >> 7, mr = m & 127;
        const int off = t * A_TILE + (((mr >> 3) * 2 + (k >> 3)) * 8 + (mr & 7)) * 16 + (k & 7) * 2;
        *reinterpret_cast<__nv_bfloat16*>(st + off) = v[e];
      }
    }
    // B: items (channel group of 8, cell k)
    for (int it = tid; it < (NOUT / 8) * 16; it += WG_THREADS) {
      const int k = it & 15, ng = it >> 4;
      const long long x = x0 + k;
      __align__(16) __nv_bfloat16 v[8];
      if (x < c1 && ng * 8 < g_stride)
        *reinterpret_cast<uint4*>(v) = __ldg(reinterpret_cast<const uint4*>(g + x * g_stride + ng * 8));
      else
        *reinterpret_cast<uint4*>(v) = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int n = ng * 8 + e;
        const int off = MT * A_TILE + (((n >> 3) * 2 + (k >> 3)) * 8 + (n & 7)) * 16 + (k & 7) * 2;
        *reinterpret_cast<__nv_bfloat16*>(st + off) = v[e];
      }
    }
    tc::fence_async_smem();
    __syncthreads();
    if (s_abort) break;
    if (tid == 0) {
      tc::tc_fence_after();
      const uint32_t base = s_addr + b * STAGE;
      const uint64_t bdesc = tc::smem_desc(base + MT * A_TILE, 128, 256);
#pragma unroll
      for (int t = 0; t < MT; ++t) {
        const uint64_t adesc = tc::smem_desc(base + t * A_TILE, 128, 256);
        tc::mma_bf16(tmem + t * NOUT, adesc, bdesc, idesc, s > 0 ? 1u : 0u);
      }
      tc::mma_commit(&bars[b]);
      if (s == ksteps - 1) tc::mma_commit(bar_done);
    }
  }
  bool have = ksteps > 0 && !s_abort;
  if (have) {
    if (!tc::mbar_wait(bar_done, 0, CV_WAIT_ITERS)) { s_abort = 1; have = false; }
  }
  __syncthreads();
  if (s_abort) have = false;
  tc::tc_fence_after();
  // epilogue: partial[cta][m][n]
  float* out = partial + (long long)blockIdx.x * MT * 128 * NOUT;
  for (int t = 0; t < MT; ++t) {
    const int m = t * 128 + warp * 32 + (tid & 31);
    if (have) {
      const uint32_t taddr = tmem + t * NOUT + ((uint32_t)(warp * 32) << 16);
      if (NOUT == 32) {
        float acc[32];
        tc::tmem_ld_32x32b_x32(taddr, acc);
        tc::tmem_ld_wait();
        for (int n = 0; n < 32; ++n) out[(long long)m * NOUT + n] = acc[n];
      } else {
        float acc[16];
        tc::tmem_ld_32x32b_x16(taddr, acc);
        tc::tmem_ld_wait();
        for (int n = 0; n < 16; ++n) out[(long long)m * NOUT + n] = acc[n];
      }
    } else {
      for (int n = 0; n < NOUT; ++n) out[(long long)m * NOUT + n] = 0.0f;
    }
  }
  if (s_abort) {
    if (tid == 0) {
      atomicOr(err, 1u);
      tc::mma_commit(bar_done);
    }
    tc::mbar_wait(bar_done, ksteps > 0 ? 1u : 0u, CV_WAIT_ITERS);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, TMEM_COLS);
  }
}

// dW[n][c][tap] (master layout) = sum over CTAs of partial[cta][tap * cin_pad + c][n]
__global__ void wgrad_reduce_kernel(const float* __restrict__ partial, int nctas, int mt, int nout_pad,
                                    int cin_pad, int cout, int cin, float* __restrict__ dW) {
  const int total = cout * cin * 27;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const int tap = idx % 27, c = (idx / 27) % cin, n = idx / (27 * cin);
    const int m = tap * cin_pad + c;
    double s = 0.0;
    for (int b = 0; b < nctas; ++b) s += (double)partial[((long long)b * mt * 128 + m) * nout_pad + n];
    dW[idx] = (float)s;
  }
}

template <int CIN, int NOUT>
static cudaError_t launch_wgrad(const __nv_bfloat16* act, const __nv_bfloat16* g, int g_stride,
                                int nx, int ny, int nz, int nctas, float* partial, unsigned* err,
                                cudaStream_t s) {
  constexpr int MT = (27 * CIN + 127) / 128;
  constexpr int STAGE = MT * 128 * 16 * 2 + NOUT * 16 * 2;
  const size_t smem = (size_t)WG_STAGES * STAGE + 8 * (WG_STAGES + 1) + 16;
  cudaError_t e = cudaFuncSetAttribute(conv3d_wgrad_tc_kernel<CIN, NOUT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long ncell = (long long)nx * ny * nz;
  long long per = (ncell + nctas - 1) / nctas;
  per = (per + 15) / 16 * 16;
  conv3d_wgrad_tc_kernel<CIN, NOUT><<<nctas, WG_THREADS, smem, s>>>(act, g, g_stride, nx, ny, nz,
                                                                   per, partial, err);
  return cudaGetLastError();
}

}  // namespace dh

extern "C" dh_status dh_conv3d_wgrad_bf16(const void* act, int cin_pad, int cin, const void* grad,
                                          int grad_stride, int cout, int nx, int ny, int nz,
                                          float* partial, int nctas, float* dW, unsigned* err_flag,
                                          void* stream) {
  if (!act || !grad || !partial || !dW || !err_flag || nctas < 1) return DH_ERR_ARG;
  if ((cin_pad != 8 && cin_pad != 32) || cin > cin_pad || cout > 32 || cout < 1 ||
      (grad_stride != 8 && grad_stride != 32) || cout > grad_stride) {
    dh_set_global_error("dh_conv3d_wgrad_bf16: cin_pad 8 or 32, cout <= grad_stride in {8, 32}");
    return DH_ERR_ARG;
  }
  const int nout_pad = cout > 16 ? 32 : 16;
  const int mt = (27 * cin_pad + 127) / 128;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  const __nv_bfloat16* a = (const __nv_bfloat16*)act;
  const __nv_bfloat16* gg = (const __nv_bfloat16*)grad;
  if (cin_pad == 8 && nout_pad == 32) e = launch_wgrad<8, 32>(a, gg, grad_stride, nx, ny, nz, nctas, partial, err_flag, s);
  else if (cin_pad == 32 && nout_pad == 32) e = launch_wgrad<32, 32>(a, gg, grad_stride, nx, ny, nz, nctas, partial, err_flag, s);
  else if (cin_pad == 32 && nout_pad == 16) e = launch_wgrad<32, 16>(a, gg, grad_stride, nx, ny, nz, nctas, partial, err_flag, s);
  else if (cin_pad == 8 && nout_pad == 16) e = launch_wgrad<8, 16>(a, gg, grad_stride, nx, ny, nz, nctas, partial, err_flag, s);
  else return DH_ERR_ARG;
  if (e != cudaSuccess) { dh_set_global_error(cudaGetErrorString(e)); return DH_ERR_CUDA; }
  wgrad_reduce_kernel<<<64, 256, 0, s>>>(partial, nctas, mt, nout_pad, cin_pad, cout, cin, dW);
  e = cudaGetLastError();
  if (e != cudaSuccess) { dh_set_global_error(cudaGetErrorString(e)); return DH_ERR_CUDA; }
  return DH_OK;
}
