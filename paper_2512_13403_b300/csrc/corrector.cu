// Residual 3D convolutional corrector on the tensor cores (BF16 operands, FP32 accumulation).
//
// Every 3x3x3 periodic convolution is an implicit GEMM: D[cell, n] = sum_k A[cell, k] B[n, k]
// with k = (tap, input channel), A the 27 neighbours of each cell and B the packed weights.
// Activations are kept in the padded channel-group-major layout of conv_layout.cuh, in which a
// tap is a constant row shift.  A persistent CTA walks 128-row tiles of the padded volume
// (M = 128); for each tile one thread copies three windows (the tile's rows in planes dz = -1,
// 0, +1, widened by the in-plane reach of the taps) into a shared-memory ring with 1D bulk
// copies (TMA engine, mbarrier transaction counts), then issues one tcgen05.mma per 16-wide K
// step whose A descriptor is the window shifted by the tap's row offset — no gather, no
// per-step barrier.  B (all taps) stays resident in shared memory.  Two TMEM accumulators
// alternate, so the epilogue of tile j-1 (tcgen05.ld, bias + GELU, the GELU derivative, or the
// linear output; padded writes with halo images) runs while the tensor cores work on tile j.
// Rows of a tile that are halo positions are computed and dropped.  The same kernel computes
// the backward data gradient with tap-flipped, channel-transposed weights.
//
// K layout: k = tap * C + c, tap = (dz+1)*9 + (dy+1)*3 + (dx+1).  C = 32: a K step is half a
// tap (two channel groups, LBO = one window).  C = 8: a K step holds taps 2s and 2s+1 (LBO =
// the distance between their two shifted windows; tap 27 points at a zero block).
#include <cuda_bf16.h>
#include <math.h>

#include "conv_layout.cuh"
#include "dh_internal.h"
#include "tc_ptx.cuh"

namespace dh {

constexpr int CV_THREADS = 320;   // 10 warps: TMA, MMA, 8 x epilogue
constexpr int CV_MAX_STAGES = 3;
constexpr uint32_t CV_WAIT_ITERS = 1u << 22;   // bounded mbarrier waits
constexpr int CV_SMEM_MAX = 226 * 1024;   // dynamic; the kernel's static part is below 1 KB

enum ConvMode : int {
  CONV_GELU = 0,        // out_bf16 = bf16(gelu(acc + bias)) (padded); z_out = acc + bias (fp32)
  CONV_LINEAR = 1,      // out_f32 planar [c][cell] = acc + bias for c < n_real
  CONV_GELU_GRAD = 2,   // out_bf16 = bf16(acc * gelu'(z_in)) (padded)
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

// Two floats rounded to bf16 (nearest even), element 0 in the low half (lower address).
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  uint32_t u;
  memcpy(&u, &h, sizeof(u));
  return u;
}

struct ConvArgs {
  const __nv_bfloat16* act;   // padded layout, CIN / 8 groups
  const __nv_bfloat16* wpk;   // packed B, [NOUT/8][K/8][8][8] bf16
  const float* bias;          // [NOUT] (nullable: zero)
  const float* z_in;          // [cells][32] fp32, CONV_GELU_GRAD
  __nv_bfloat16* out_bf16;    // padded layout, 4 groups, for the GELU modes
  float* out_f32;             // planar [n_real][cells] for CONV_LINEAR
  float* z_out;               // [cells][NOUT] fp32 (nullable) for CONV_GELU
  int n_real;                 // real output channels (CONV_LINEAR)
  unsigned* err;              // set to 1 if a bounded wait gave up
};

template <int CIN, int NOUT>
struct ConvShape {
  static constexpr int G = CIN / 8;
  static constexpr int K = CIN == 32 ? 27 * 32 : 28 * 8;   // padded reduction length
  static constexpr int KSTEPS = K / 16;
  static constexpr int B_BYTES = NOUT * K * 2;
  static constexpr int ZERO_BYTES = CIN == 8 ? 128 * 16 : 0;
  static constexpr uint32_t TMEM_COLS = 2 * NOUT <= 32 ? 32 : 64;   // two accumulators
  static size_t stage_bytes(const ConvGeom& g) { return (size_t)3 * G * g.win * 16; }
  static size_t smem_bytes(const ConvGeom& g, int stages) {
    return (size_t)B_BYTES + stages * stage_bytes(g) + ZERO_BYTES + 12 * 8 + 16;
  }
};

// Bounded wait on an mbarrier phase that also gives up when another role has aborted.
__device__ __forceinline__ bool cv_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  for (uint32_t i = 0; i < CV_WAIT_ITERS; ++i) {
    if (tc::mbar_try_wait(bar, parity)) return true;
    if ((i & 63u) == 63u && *abort_flag) return false;
  }
  *abort_flag = 1;
  return false;
}

// Warp roles: warp 0 lane 0 copies windows (TMA), warp 1 issues the MMAs (converged, one
// elected lane), warps 2..9 run the epilogue (warp w reads TMEM lanes 32 (w % 4) .. and 16
// of the accumulator's columns).
template <int CIN, int NOUT, int MODE>
__global__ void __launch_bounds__(CV_THREADS)
conv3d_tc_kernel(const ConvArgs p, const ConvGeom g, const int stages) {
  using S = ConvShape<CIN, NOUT>;
  constexpr int G = S::G, KSTEPS = S::KSTEPS, K = S::K;
  extern __shared__ __align__(1024) unsigned char smem[];
  const uint32_t win_bytes = (uint32_t)g.win * 16;
  const uint32_t stage_bytes = 3u * G * win_bytes;
  unsigned char* sB = smem;                                        // resident weights
  unsigned char* sA = smem + S::B_BYTES;                           // window ring
  unsigned char* sZero = sA + (size_t)stages * stage_bytes;        // zero tap (C = 8)
  uint64_t* bars = reinterpret_cast<uint64_t*>(sZero + S::ZERO_BYTES);
  uint64_t* full = bars;          // [3] windows of a tile landed (TMA -> MMA)
  uint64_t* empty = bars + 3;     // [3] MMAs reading a slot completed (MMA -> TMA)
  uint64_t* accf = bars + 6;      // [2] accumulator holds a finished tile (MMA -> epilogue)
  uint64_t* acce = bars + 8;      // [2] accumulator read out (epilogue -> MMA), 8 arrivals
  uint64_t* bbar = bars + 10;     // weights landed
  uint64_t* drain = bars + 11;    // abort path: all issued MMAs completed
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bars + 12);
  __shared__ int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long ncell = (long long)g.nx * g.ny * g.nz;
  const int nt = (int)((g.ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x);   // own tiles

  if (S::ZERO_BYTES)
    for (int i = tid; i < S::ZERO_BYTES / 16; i += CV_THREADS)
      reinterpret_cast<uint4*>(sZero)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    for (int b = 0; b < 12; ++b) tc::mbar_init(&bars[b], (b == 8 || b == 9) ? 8u : 1u);
    tc::mbar_fence_init();
    s_abort = 0;
  }
  if (warp == 1) {
    tc::tmem_alloc(s_tmem, S::TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::fence_async_smem();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *s_tmem;
  volatile int* abort_flag = &s_abort;
  int tma_issued = 0;            // warp 0 lane 0
  bool b_waited = false;         // warp 1

  if (warp == 0) {
    if (lane == 0) {
      const uint32_t sA_addr = tc::smem_u32(sA);
      tc::mbar_arrive_expect_tx(bbar, S::B_BYTES);
      tc::bulk_g2s(tc::smem_u32(sB), p.wpk, S::B_BYTES, bbar);
      for (int j = 0; j < nt; ++j) {
        const int slot = j % stages;
        if (j >= stages && !cv_wait(&empty[slot], (uint32_t)(j / stages - 1) & 1u, abort_flag)) break;
        const long long R0 = g.PXY + 128 * (blockIdx.x + (long long)j * gridDim.x);
        tc::mbar_arrive_expect_tx(&full[slot], stage_bytes);
        for (int dzi = 0; dzi < 3; ++dzi) {
          const long long row = g.guard + R0 + (long long)(dzi - 1) * g.PXY - (g.PX + 1);
#pragma unroll
          for (int cg = 0; cg < G; ++cg)
            tc::bulk_g2s(sA_addr + slot * stage_bytes + (dzi * G + cg) * win_bytes,
                         p.act + ((long long)cg * g.rows + row) * 8, win_bytes, &full[slot]);
        }
        ++tma_issued;
      }
    }
  } else if (warp == 1) {
    // converged warp: every lane waits and computes the (uniform) descriptors; one lane issues
    const uint32_t idesc = tc::idesc_bf16_f32(128, NOUT);
    const uint32_t sA_addr = tc::smem_u32(sA), sB_addr = tc::smem_u32(sB);
    const uint32_t win16 = (uint32_t)g.win;          // window length in 16-byte units
    const int px16 = g.PX;                           // one padded row of a plane, in 16-byte units
    const uint64_t bdesc0 = tc::smem_desc(sB_addr, 128, (K / 8) * 128);
    // zero block relative to a slot's window origin (C = 8 pairs tap 26 with it), 16-byte units
    uint32_t zero16_slot[CV_MAX_STAGES];
#pragma unroll
    for (int sl = 0; sl < CV_MAX_STAGES; ++sl)
      zero16_slot[sl] = (tc::smem_u32(sZero) - (sA_addr + sl * stage_bytes + (uint32_t)(g.PX + 1) * 16u)) >> 4;
    bool ok = __all_sync(0xffffffffu, cv_wait(bbar, 0, abort_flag));
    b_waited = ok;
    for (int j = 0; ok && j < nt; ++j) {
      const int slot = j % stages, a = j & 1;
      ok = __all_sync(0xffffffffu, cv_wait(&full[slot], (uint32_t)(j / stages) & 1u, abort_flag));
      if (ok && j >= 2)
        ok = __all_sync(0xffffffffu, cv_wait(&acce[a], (uint32_t)((j >> 1) - 1) & 1u, abort_flag));
      if (!ok) break;
      __syncwarp();
      tc::tc_fence_after();
      const uint32_t acc = tmem + (uint32_t)a * NOUT;
      const uint32_t zero16 = zero16_slot[slot == 0 ? 0 : (slot == 1 ? 1 : 2)];
      // Descriptor of the slot's window origin (output row 0 of plane dz = 0, PX + 1 rows in);
      // every K step adds its tap's offset (and, for C = 8, its LBO) to the low word, in 16-byte
      // units: start-address field bits 0..13, LBO field bits 16..29, both without carry.
      const uint64_t d0 = tc::smem_desc(sA_addr + slot * stage_bytes + (uint32_t)(g.PX + 1) * 16u,
                                        CIN == 32 ? win_bytes : 0u, 128);
      const uint32_t d0_lo = (uint32_t)d0, d0_hi = (uint32_t)(d0 >> 32);
      const uint32_t b0_lo = (uint32_t)bdesc0, b0_hi = (uint32_t)(bdesc0 >> 32);
#pragma unroll
      for (int s = 0; s < KSTEPS; ++s) {
        const int t = CIN == 32 ? (s >> 1) : 2 * s;
        uint32_t off = (uint32_t)((t / 9) * G) * win16 + (uint32_t)(((t / 3) % 3 - 1) * px16 + (t % 3 - 1));
        if (CIN == 32) {
          off += (uint32_t)((s & 1) * 2) * win16;
        } else {
          const int t1 = t + 1;
          uint32_t lbo16;
          if (t1 < 27) {
            lbo16 = (uint32_t)((t1 / 9) * G) * win16 +
                    (uint32_t)(((t1 / 3) % 3 - 1) * px16 + (t1 % 3 - 1)) - off;
          } else {
            lbo16 = zero16 - off;
          }
          off += lbo16 << 16;
        }
        const uint64_t adesc = ((uint64_t)d0_hi << 32) | (uint64_t)(d0_lo + off);
        const uint64_t bdesc = ((uint64_t)b0_hi << 32) | (uint64_t)(b0_lo + (uint32_t)(s * 16));
        tc::mma_bf16_elect(acc, adesc, bdesc, idesc, s > 0 ? 1u : 0u);
      }
      tc::mma_commit_elect(&empty[slot]);
      tc::mma_commit_elect(&accf[a]);
    }
  } else {
    // epilogue: warp w reads TMEM lane quarter w % 4 and output columns [16 h, 16 h + 16)
    const int q = warp & 3;
    const int hcol = (warp - 2) >> 2;
    const int trow = q * 32 + lane;        // tile row = TMEM lane
    const bool cols = 16 * hcol < NOUT;    // this warp has columns to read
    for (int j = 0; j < nt; ++j) {
      const int a = j & 1;
      if (!__all_sync(0xffffffffu, cv_wait(&accf[a], (uint32_t)(j >> 1) & 1u, abort_flag))) break;
      __syncwarp();   // tcgen05.ld below is warp-collective
      tc::tc_fence_after();
      float acc[16];
      if (cols) {
        tc::tmem_ld_32x32b_x16(tmem + (uint32_t)(a * NOUT + 16 * hcol) + ((uint32_t)(q * 32) << 16), acc);
        tc::tmem_ld_wait();
      }
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&acce[a]);   // the accumulator may be overwritten now
      if (!cols) continue;

      // padded row of this thread (fits 32 bits: the launcher rejects larger volumes)
      const uint32_t rho = (uint32_t)g.PXY + 128u * (blockIdx.x + (uint32_t)j * gridDim.x) + trow;
      const uint32_t pz = rho / (uint32_t)g.PXY;
      const uint32_t rem = rho - pz * (uint32_t)g.PXY;
      const int py = (int)(rem / (uint32_t)g.PX), px = (int)(rem - (uint32_t)py * (uint32_t)g.PX);
      if (!(px >= 1 && px <= g.nx && py >= 1 && py <= g.ny && (int)pz <= g.nz)) continue;   // halo row
      const int x = px - 1, y = py - 1, z = (int)pz - 1;
      const long long qc = ((long long)z * g.ny + y) * g.nx + x;
      const int c0 = 16 * hcol;
      if (MODE == CONV_LINEAR) {
        for (int c = 0; c < 16 && c0 + c < p.n_real; ++c)
          p.out_f32[(long long)(c0 + c) * ncell + qc] = acc[c] + (p.bias ? __ldg(p.bias + c0 + c) : 0.0f);
      } else {
        float hv[16];   // values to round to bf16
        if (MODE == CONV_GELU) {
#pragma unroll
          for (int c = 0; c < 16; ++c) {
            const float zv = acc[c] + (p.bias ? __ldg(p.bias + c0 + c) : 0.0f);
            acc[c] = zv;
            hv[c] = gelu_exact(zv);
          }
          if (p.z_out) {
            float4* zo = reinterpret_cast<float4*>(p.z_out + qc * 32 + c0);
#pragma unroll
            for (int v4 = 0; v4 < 4; ++v4)
              zo[v4] = make_float4(acc[4 * v4], acc[4 * v4 + 1], acc[4 * v4 + 2], acc[4 * v4 + 3]);
          }
        } else {
          const float4* zi = reinterpret_cast<const float4*>(p.z_in + qc * 32 + c0);
#pragma unroll
          for (int v4 = 0; v4 < 4; ++v4) {
            const float4 zz = __ldg(zi + v4);
            hv[4 * v4] = acc[4 * v4] * gelu_grad(zz.x);
            hv[4 * v4 + 1] = acc[4 * v4 + 1] * gelu_grad(zz.y);
            hv[4 * v4 + 2] = acc[4 * v4 + 2] * gelu_grad(zz.z);
            hv[4 * v4 + 3] = acc[4 * v4 + 3] * gelu_grad(zz.w);
          }
        }
        uint4* out = reinterpret_cast<uint4*>(p.out_bf16);
#pragma unroll
        for (int cg = 0; cg < 2; ++cg)
          store_with_images(out + (long long)(2 * hcol + cg) * g.rows, g, x, y, z,
                            make_uint4(pack_bf16x2(hv[8 * cg], hv[8 * cg + 1]),
                                       pack_bf16x2(hv[8 * cg + 2], hv[8 * cg + 3]),
                                       pack_bf16x2(hv[8 * cg + 4], hv[8 * cg + 5]),
                                       pack_bf16x2(hv[8 * cg + 6], hv[8 * cg + 7])));
      }
    }
  }

  // All roles are done.  After an abort, every MMA issued and every copy in flight must land
  // before TMEM and shared memory are released; the waits stay bounded.
  tc::tc_fence_before();
  __syncthreads();
  const bool aborted = s_abort != 0;
  if (aborted) {
    if (tid == 0) atomicOr(p.err, 1u);
    if (warp == 1) {
      tc::mma_commit_elect(drain);
      tc::mbar_wait(drain, 0, CV_WAIT_ITERS);
    }
    if (warp == 0 && lane == 0) {
      const int first = tma_issued > stages ? tma_issued - stages : 0;
      for (int jj = first; jj < tma_issued; ++jj)
        tc::mbar_wait(&full[jj % stages], (uint32_t)(jj / stages) & 1u, CV_WAIT_ITERS);
      tc::mbar_wait(bbar, 0, CV_WAIT_ITERS);
    }
  }
  (void)b_waited;
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, S::TMEM_COLS);
  }
}

template <int CIN, int NOUT, int MODE>
static cudaError_t launch_conv(const ConvArgs& a, const ConvGeom& g, cudaStream_t s) {
  using S = ConvShape<CIN, NOUT>;
  if (g.rows >= (1LL << 31)) return cudaErrorInvalidValue;   // padded rows are 32-bit indices
  // as many window stages as fit (one stage: each tile's windows load after the previous
  // tile's MMAs, without overlap, for long rows)
  int stages = CV_MAX_STAGES;
  while (stages >= 2 && S::smem_bytes(g, stages) > (size_t)CV_SMEM_MAX) --stages;
  if (S::smem_bytes(g, stages) > (size_t)CV_SMEM_MAX) return cudaErrorInvalidValue;
  const size_t smem = S::smem_bytes(g, stages);
  auto kern = conv3d_tc_kernel<CIN, NOUT, MODE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 148, occ = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, CV_THREADS, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) occ = 1;
  if (occ * (int)S::TMEM_COLS > 512) occ = 512 / (int)S::TMEM_COLS;   // TMEM per SM
  long long grid = (long long)sms * occ;
  if (grid > g.ntiles) grid = g.ntiles;
  kern<<<(unsigned)grid, CV_THREADS, smem, s>>>(a, g, stages);
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

namespace dh {

// ---------------------------------------------------------------------------------------------
// Layout conversion between channel-last [cell][C] bf16 and the padded layout.
__global__ void pad_kernel(const __nv_bfloat16* __restrict__ src, int C, ConvGeom g,
                           __nv_bfloat16* __restrict__ dst) {
  const long long ncell = (long long)g.nx * g.ny * g.nz;
  const int G = C / 8;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ncell * G;
       i += (long long)gridDim.x * blockDim.x) {
    const long long q = i / G;
    const int cg = (int)(i - q * G);
    const unsigned t = (unsigned)q / (unsigned)g.nx;
    const int x = (int)((unsigned)q - t * (unsigned)g.nx);
    const int y = (int)(t % (unsigned)g.ny), z = (int)(t / (unsigned)g.ny);
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(src + q * C + cg * 8));
    store_with_images(reinterpret_cast<uint4*>(dst) + (long long)cg * g.rows, g, x, y, z, v);
  }
}

__global__ void unpad_kernel(const __nv_bfloat16* __restrict__ src, int C, ConvGeom g,
                             __nv_bfloat16* __restrict__ dst) {
  const long long ncell = (long long)g.nx * g.ny * g.nz;
  const int G = C / 8;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ncell * G;
       i += (long long)gridDim.x * blockDim.x) {
    const long long q = i / G;
    const int cg = (int)(i - q * G);
    const unsigned t = (unsigned)q / (unsigned)g.nx;
    const int x = (int)((unsigned)q - t * (unsigned)g.nx);
    const int y = (int)(t % (unsigned)g.ny), z = (int)(t / (unsigned)g.ny);
    reinterpret_cast<uint4*>(dst + q * C)[cg] =
        __ldg(reinterpret_cast<const uint4*>(src) + (long long)cg * g.rows + pad_row(g, x, y, z));
  }
}

static bool conv_dims_ok(int nx, int ny, int nz) {
  return nx >= 3 && ny >= 3 && nz >= 3 && (long long)nx * ny * nz < (1LL << 31);
}

}  // namespace dh

using namespace dh;

extern "C" long long dh_conv_padded_rows(int nx, int ny, int nz) {
  if (!conv_dims_ok(nx, ny, nz)) return -1;
  return conv_geom(nx, ny, nz).rows;
}

extern "C" dh_status dh_conv_pad(const void* src, int channels, int nx, int ny, int nz, void* dst,
                                 void* stream) {
  if (!src || !dst || (channels != 8 && channels != 32) || !conv_dims_ok(nx, ny, nz)) return DH_ERR_ARG;
  pad_kernel<<<148 * 4, 256, 0, (cudaStream_t)stream>>>((const __nv_bfloat16*)src, channels,
                                                       conv_geom(nx, ny, nz), (__nv_bfloat16*)dst);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { dh_set_global_error(cudaGetErrorString(e)); return DH_ERR_CUDA; }
  return DH_OK;
}

extern "C" dh_status dh_conv_unpad(const void* src, int channels, int nx, int ny, int nz, void* dst,
                                   void* stream) {
  if (!src || !dst || (channels != 8 && channels != 32) || !conv_dims_ok(nx, ny, nz)) return DH_ERR_ARG;
  unpad_kernel<<<148 * 4, 256, 0, (cudaStream_t)stream>>>((const __nv_bfloat16*)src, channels,
                                                         conv_geom(nx, ny, nz), (__nv_bfloat16*)dst);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { dh_set_global_error(cudaGetErrorString(e)); return DH_ERR_CUDA; }
  return DH_OK;
}

extern "C" dh_status dh_conv3d_bf16(const void* act, int cin_pad, const void* packed, int nout_pad,
                                    const float* bias, int mode, const float* z_in, void* out,
                                    float* z_out, int n_real, int nx, int ny, int nz,
                                    unsigned* err_flag, void* stream) {
  if (!act || !packed || !out || !err_flag) return DH_ERR_ARG;
  if (!conv_dims_ok(nx, ny, nz)) {
    dh_set_global_error("dh_conv3d_bf16: every dimension must be >= 3");
    return DH_ERR_ARG;
  }
  if (mode == CONV_GELU_GRAD && !z_in) return DH_ERR_ARG;
  const ConvGeom g = conv_geom(nx, ny, nz);
  ConvArgs a;
  a.act = (const __nv_bfloat16*)act;
  a.wpk = (const __nv_bfloat16*)packed;
  a.bias = bias;
  a.z_in = z_in;
  a.out_bf16 = (__nv_bfloat16*)out;
  a.out_f32 = (float*)out;
  a.z_out = z_out;
  a.n_real = n_real;
  a.err = err_flag;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaErrorNotSupported;
  if (cin_pad == 8 && nout_pad == 32 && mode == CONV_GELU) e = launch_conv<8, 32, CONV_GELU>(a, g, s);
  else if (cin_pad == 8 && nout_pad == 32 && mode == CONV_GELU_GRAD) e = launch_conv<8, 32, CONV_GELU_GRAD>(a, g, s);
  else if (cin_pad == 32 && nout_pad == 32 && mode == CONV_GELU) e = launch_conv<32, 32, CONV_GELU>(a, g, s);
  else if (cin_pad == 32 && nout_pad == 32 && mode == CONV_GELU_GRAD) e = launch_conv<32, 32, CONV_GELU_GRAD>(a, g, s);
  else if (cin_pad == 32 && nout_pad == 16 && mode == CONV_LINEAR && n_real >= 1 && n_real <= 16) e = launch_conv<32, 16, CONV_LINEAR>(a, g, s);
  else if (cin_pad == 32 && nout_pad == 32 && mode == CONV_LINEAR && n_real >= 1 && n_real <= 32) e = launch_conv<32, 32, CONV_LINEAR>(a, g, s);
  else {
    dh_set_global_error("dh_conv3d_bf16: unsupported (cin_pad, nout_pad, mode, n_real) combination");
    return DH_ERR_ARG;
  }
  if (e == cudaErrorInvalidValue) {
    dh_set_global_error("dh_conv3d_bf16: the x extent is too large for two shared-memory windows");
    return DH_ERR_ARG;
  }
  if (e != cudaSuccess) { dh_set_global_error(cudaGetErrorString(e)); return DH_ERR_CUDA; }
  return DH_OK;
}

// =============================================================================================
// Weight gradient: dW[n][c][tap] = sum_cells g[cell][n] * act[cell + offset(tap)][c], a GEMM
// with M = (tap, c) rows (27 * CIN, in tiles of 128), N = n, K = cells.  Each CTA reduces a
// contiguous range of cells in 32-cell K steps.  An 8-cell x 8-channel block of either operand
// (act shifted by a tap, or the gradient) is transposed into a K-major core matrix (a row = one
// channel over 8 consecutive cells) by one quarter of an stmatrix.trans: lane t loads the 4
// bytes of cell t/4, channels 2(t%4)..+1 of the padded layout (where a tap is a row offset).
// A converged warp issues the MMAs of a step (one per M tile and 16-cell half) into per-tile TMEM
// accumulators while the threads build the next step.  Per-CTA partial sums go to global memory
// and a second kernel adds them in a fixed order.
namespace dh {

constexpr int WG_THREADS = 256;
constexpr int WG_STAGES = 2;
constexpr int WG_KG = 4;                 // 8-cell groups per K step
constexpr int WG_KCELLS = 8 * WG_KG;     // cells per K step

template <int CIN, int NOUT>
struct WgShape {
  static constexpr int G = CIN / 8;                    // activation channel groups
  static constexpr int GN = NOUT / 8;                  // gradient channel groups (B rows / 8)
  static constexpr int MT = (27 * CIN + 127) / 128;    // M tiles
  static constexpr int A_TILE = 16 * WG_KG * 128;      // 16 M groups x WG_KG K groups x 128 B
  static constexpr int B_BYTES = GN * WG_KG * 128;
  static constexpr int STAGE = MT * A_TILE + B_BYTES;
  static constexpr uint32_t TMEM_COLS =
      MT * NOUT <= 32 ? 32 : (MT * NOUT <= 64 ? 64 : (MT * NOUT <= 128 ? 128 : 256));
  static constexpr size_t SMEM = (size_t)WG_STAGES * STAGE + 8 * 4 + 16;
};

template <int CIN, int NOUT>
__global__ void __launch_bounds__(WG_THREADS)
conv3d_wgrad_tc_kernel(const __nv_bfloat16* __restrict__ act, const __nv_bfloat16* __restrict__ g,
                       int g_stride, int nx, int ny, int nz, long long cells_per_cta,
                       float* __restrict__ partial, unsigned* err) {
  using W = WgShape<CIN, NOUT>;
  constexpr int G = W::G, GN = W::GN, MT = W::MT;
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + WG_STAGES * W::STAGE);
  uint64_t* bar_done = bars + WG_STAGES;
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bar_done + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const ConvGeom geo = conv_geom(nx, ny, nz);
  const long long ncell = (long long)nx * ny * nz;
  const long long c0 = (long long)blockIdx.x * cells_per_cta;
  const long long c1 = c0 + cells_per_cta < ncell ? c0 + cells_per_cta : ncell;
  const int ksteps = c1 > c0 ? (int)((c1 - c0 + WG_KCELLS - 1) / WG_KCELLS) : 0;

  // zero both stages once: M rows past 27 * CIN stay zero
  for (int i = tid; i < WG_STAGES * W::STAGE / 16; i += WG_THREADS)
    reinterpret_cast<uint4*>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
  // row offset of each tap in the padded layout
  __shared__ long long s_shift[27];
  if (tid < 27)
    s_shift[tid] = (long long)(tid / 9 - 1) * geo.PXY + (long long)((tid / 3) % 3 - 1) * geo.PX + (tid % 3 - 1);
  if (tid == 0) {
    for (int b = 0; b < WG_STAGES; ++b) tc::mbar_init(&bars[b], 1);
    tc::mbar_init(bar_done, 1);
    tc::mbar_fence_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(s_tmem, W::TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::fence_async_smem();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *s_tmem;
  const uint32_t idesc = tc::idesc_bf16_f32(128, NOUT);
  const uint32_t s_addr = tc::smem_u32(smem);
  const unsigned char* act_b = reinterpret_cast<const unsigned char*>(act);
  const unsigned char* g_b = reinterpret_cast<const unsigned char*>(g);
  const int g_groups = g_stride / 8;
  uint32_t phase_bits = 0;
  int my_abort = 0;
  bool aborted = false;

  for (int s = 0; s < ksteps; ++s) {
    const int b = s % WG_STAGES;
    if (s >= WG_STAGES) {
      if (!tc::mbar_wait(&bars[b], (phase_bits >> b) & 1u, CV_WAIT_ITERS)) my_abort = 1;
      phase_bits ^= 1u << b;
    }
    const uint32_t st = s_addr + b * W::STAGE;
    const long long k0 = c0 + (long long)WG_KCELLS * s;
    // padded rows of this lane's cells (cell k0 + 8 kg + lane/4), -1 past the range
    // (32-bit index arithmetic: the launcher rejects grids of 2^31 cells or more)
    long long prow[WG_KG];
#pragma unroll
    for (int kg = 0; kg < WG_KG; ++kg) {
      const long long q = k0 + 8 * kg + (lane >> 2);
      if (q < c1) {
        const unsigned uq = (unsigned)q;
        const unsigned t1 = uq / (unsigned)nx;
        const int x = (int)(uq - t1 * (unsigned)nx);
        const unsigned z = t1 / (unsigned)ny;
        prow[kg] = pad_row(geo, x, (int)(t1 - z * (unsigned)ny), (int)z);
      } else {
        prow[kg] = -1;
      }
    }
    // Quad q transposes the four K groups of one operand row group: q < 27 G is activation
    // group (tap, cg) = (q / G, q % G), then the GN gradient groups.  All of this warp's loads
    // are issued first (their latencies overlap), then the transposing stores.
    constexpr int NWARP = WG_THREADS / 32;
    constexpr int NQA = 27 * G, NQ = NQA + GN;
    constexpr int QPW = (NQ + NWARP - 1) / NWARP;   // quads per warp
    uint32_t r[QPW][4];
#pragma unroll
    for (int j = 0; j < QPW; ++j) {
      const int quad = warp + NWARP * j;
      // row offset of this quad's operand row group (a tap shift may be negative)
      long long base = 0;
      bool valid = false;
      if (quad < NQA) {
        base = (long long)(quad % G) * geo.rows + s_shift[quad / G];
        valid = true;
      } else if (quad < NQ && quad - NQA < g_groups) {
        base = (long long)(quad - NQA) * geo.rows;
        valid = true;
      }
      const unsigned char* src = quad < NQA ? act_b : g_b;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        uint32_t v = 0u;
        if (valid && prow[i] >= 0)
          v = __ldg(reinterpret_cast<const uint32_t*>(src + (base + prow[i]) * 16 + (lane & 3) * 4));
        r[j][i] = v;
      }
    }
#pragma unroll
    for (int j = 0; j < QPW; ++j) {
      const int quad = warp + NWARP * j;
      if (quad >= NQ) break;   // warp-uniform
      // lane 8i + jj gives the address of row jj of K group i of this quad's row group
      const uint32_t grp = quad < NQA ? (uint32_t)((quad >> 4) * W::A_TILE + (quad & 15) * WG_KG * 128)
                                      : (uint32_t)(MT * W::A_TILE + (quad - NQA) * WG_KG * 128);
      const uint32_t dst = st + grp + (uint32_t)(lane >> 3) * 128u + (uint32_t)(lane & 7) * 16u;
      tc::stmatrix_x4_trans(dst, r[j][0], r[j][1], r[j][2], r[j][3]);
    }
    tc::fence_async_smem();
    if (__syncthreads_or(my_abort)) { aborted = true; break; }
    if (warp == 0) {
      __syncwarp();
      tc::tc_fence_after();
#pragma unroll
      for (int t = 0; t < MT; ++t) {
#pragma unroll
        for (int h = 0; h < WG_KG / 2; ++h) {
          const uint64_t adesc = tc::smem_desc(st + t * W::A_TILE + h * 256, 128, WG_KG * 128);
          const uint64_t bdesc = tc::smem_desc(st + MT * W::A_TILE + h * 256, 128, WG_KG * 128);
          tc::mma_bf16_elect(tmem + t * NOUT, adesc, bdesc, idesc, (s > 0 || h > 0) ? 1u : 0u);
        }
      }
      tc::mma_commit_elect(&bars[b]);
      if (s == ksteps - 1) tc::mma_commit_elect(bar_done);
    }
  }
  int done_fail = 0;
  if (ksteps > 0 && !aborted && !tc::mbar_wait(bar_done, 0, CV_WAIT_ITERS)) done_fail = 1;
  if (__syncthreads_or(done_fail)) aborted = true;
  const bool have = ksteps > 0 && !aborted;
  tc::tc_fence_after();
  // epilogue (warps 0..3, one TMEM lane quarter each): partial[cta][m][n]
  float* out = partial + (long long)blockIdx.x * MT * 128 * NOUT;
  if (warp < 4) {
    for (int t = 0; t < MT; ++t) {
      const int m = t * 128 + warp * 32 + lane;
      if (have) {
        const uint32_t taddr = tmem + t * NOUT + ((uint32_t)(warp * 32) << 16);
        if (NOUT == 32) {
          float acc[32];
          tc::tmem_ld_32x32b_x32(taddr, acc);
          tc::tmem_ld_wait();
          float4* o4 = reinterpret_cast<float4*>(out + (long long)m * NOUT);
#pragma unroll
          for (int v = 0; v < 8; ++v) o4[v] = make_float4(acc[4 * v], acc[4 * v + 1], acc[4 * v + 2], acc[4 * v + 3]);
        } else {
          float acc[16];
          tc::tmem_ld_32x32b_x16(taddr, acc);
          tc::tmem_ld_wait();
          float4* o4 = reinterpret_cast<float4*>(out + (long long)m * NOUT);
#pragma unroll
          for (int v = 0; v < 4; ++v) o4[v] = make_float4(acc[4 * v], acc[4 * v + 1], acc[4 * v + 2], acc[4 * v + 3]);
        }
      } else {
        for (int n = 0; n < NOUT; ++n) out[(long long)m * NOUT + n] = 0.0f;
      }
    }
  }
  if (aborted) {
    // phase 0 of bar_done completes once every MMA issued so far has completed
    if (tid == 0) atomicOr(err, 1u);
    if (warp == 0) {
      tc::mma_commit_elect(bar_done);
      tc::mbar_wait(bar_done, 0, CV_WAIT_ITERS);
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, W::TMEM_COLS);
  }
}

// dW[n][c][tap] (master layout) = sum over the CTAs b of partial[b][tap * cin_pad + c][n], in a
// fixed order: warp w of the block adds b = w, w + 8, w + 16, ... in increasing b (float64), and
// the eight warp sums are combined as ((s0 + s1) + (s2 + s3)) + ((s4 + s5) + (s6 + s7)).  One
// block per (c, tap); lane n reads element n of each CTA's row, so a warp's loads are contiguous,
// and the CTAs' rows are read by eight warps at once.
constexpr int WR_WARPS = 8;
__global__ void __launch_bounds__(32 * WR_WARPS)
wgrad_reduce_kernel(const float* __restrict__ partial, int nctas, long long stride, int nout_pad,
                    int cin_pad, int cout, int cin, float* __restrict__ dW) {
  __shared__ double red[WR_WARPS][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = blockIdx.x % cin, tap = blockIdx.x / cin;
  double s = 0.0;
  if (lane < cout) {
    const float* p = partial + (long long)(tap * cin_pad + c) * nout_pad + lane;
#pragma unroll 4
    for (int b = warp; b < nctas; b += WR_WARPS) s += (double)__ldg(p + b * stride);
  }
  red[warp][lane] = s;
  __syncthreads();
  if (warp == 0 && lane < cout) {
    const double r = ((red[0][lane] + red[1][lane]) + (red[2][lane] + red[3][lane])) +
                     ((red[4][lane] + red[5][lane]) + (red[6][lane] + red[7][lane]));
    dW[((long long)lane * cin + c) * 27 + tap] = (float)r;
  }
}

template <int CIN, int NOUT>
static cudaError_t launch_wgrad(const __nv_bfloat16* act, const __nv_bfloat16* g, int g_stride,
                                int nx, int ny, int nz, int nctas, float* partial, unsigned* err,
                                cudaStream_t s) {
  using W = WgShape<CIN, NOUT>;
  if ((long long)nx * ny * nz >= (1LL << 31)) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(conv3d_wgrad_tc_kernel<CIN, NOUT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)W::SMEM);
  if (e != cudaSuccess) return e;
  const long long ncell = (long long)nx * ny * nz;
  long long per = (ncell + nctas - 1) / nctas;
  per = (per + WG_KCELLS - 1) / WG_KCELLS * WG_KCELLS;
  conv3d_wgrad_tc_kernel<CIN, NOUT><<<nctas, WG_THREADS, W::SMEM, s>>>(act, g, g_stride, nx, ny, nz,
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
  wgrad_reduce_kernel<<<cin * 27, 32 * WR_WARPS, 0, s>>>(partial, nctas, (long long)mt * 128 * nout_pad,
                                                         nout_pad, cin_pad, cout, cin, dW);
  e = cudaGetLastError();
  if (e != cudaSuccess) { dh_set_global_error(cudaGetErrorString(e)); return DH_ERR_CUDA; }
  return DH_OK;
}
