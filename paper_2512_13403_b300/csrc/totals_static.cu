// dh_conserved_totals_static: the conserved-totals reduction for callers that cannot allocate
// device memory.  The paper has no counterpart; this exists for integration only.
//
// The regular dh_conserved_totals keeps its per-block partial sums in a buffer that dh_create
// allocates with cudaMalloc.  Some callers cannot allocate: a host framework whose allocator
// owns the whole device-memory budget, or a time-critical loop that must not pay for the
// implicit device-wide synchronisation of cudaMalloc/cudaFree.  This variant keeps its partial
// sums in a fixed file-scope device array instead and allocates nothing; the caller passes the
// state and a device buffer for the five results.
//
// The array lives on every device that loads the library until the process exits.  All calls
// share it and it keeps the last call's contents; each call writes every slot it reads before
// reading it, so nothing needs clearing.  Two calls whose kernels overlap on the GPU (for
// example on two streams at once) race on the array and may return wrong sums.
#include <mutex>
#include <string>

#include "../../include/dh.h"
#include "dh_internal.h"

namespace {

constexpr int kStaticBlocks = 4096;            // partial-sum slots
constexpr long long kCellsPerBlock = 65536;    // cells summed by one block (fixed order)
constexpr long long kMaxCells = (long long)kStaticBlocks * kCellsPerBlock;  // 2^28 cells
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_totals_scratch[kStaticBlocks * 5];  // 160 KiB

std::mutex g_setup_mutex;
double* g_scratch_on_device[kMaxDevices] = {nullptr};

template <typename real>
__global__ void static_totals_partial(const real* __restrict__ U, long long n3,
                                      double* __restrict__ scratch) {
  __shared__ double red[5][kThreads];
  const long long b0 = (long long)blockIdx.x * kCellsPerBlock;
  const long long b1 = b0 + kCellsPerBlock < n3 ? b0 + kCellsPerBlock : n3;
  double s[5] = {0, 0, 0, 0, 0};
  for (long long i = b0 + threadIdx.x; i < b1; i += kThreads) {
#pragma unroll
    for (int f = 0; f < 5; ++f) s[f] += (double)__ldg(U + f * n3 + i);
  }
#pragma unroll
  for (int f = 0; f < 5; ++f) red[f][threadIdx.x] = s[f];
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
#pragma unroll
      for (int f = 0; f < 5; ++f) red[f][threadIdx.x] += red[f][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x < 5) scratch[blockIdx.x * 5 + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void static_totals_final(const double* __restrict__ scratch, int nblocks,
                                    double* __restrict__ out) {
  const int f = threadIdx.x;
  if (f < 5) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += scratch[b * 5 + f];
    out[f] = s;
  }
}

// Device address of the file-scope array on the current device.  In host code the array's
// name is only a host-side stand-in, never a device address.  Outside stream capture the
// address is looked up on every call (so a cudaDeviceReset and a fresh context cannot leave a
// stale address behind); while the stream is being captured the address cached by an earlier
// call on this device is used.
cudaError_t scratch_address(cudaStream_t s, double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
    cudaGetLastError();                  // treat an undeterminable status as capturing
    cap = cudaStreamCaptureStatusActive;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_on_device[dev] || cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_totals_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_on_device[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_on_device[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" dh_status dh_conserved_totals_static(const void* U, int precision, long long n_cells,
                                                double* totals_out, void* cuda_stream) {
  if (!U || !totals_out) {
    dh_set_global_error("dh_conserved_totals_static: null pointer");
    return DH_ERR_ARG;
  }
  if (precision != DH_F32 && precision != DH_F64) {
    dh_set_global_error("dh_conserved_totals_static: precision must be DH_F32 or DH_F64");
    return DH_ERR_ARG;
  }
  if (n_cells < 1 || n_cells > kMaxCells) {
    dh_set_global_error("dh_conserved_totals_static: n_cells must be in [1, 268435456] "
                        "(the fixed scratch holds 4096 blocks of 65536 cells)");
    return DH_ERR_ARG;
  }
  double* scratch = nullptr;
  cudaError_t e = scratch_address((cudaStream_t)cuda_stream, &scratch);
  if (e != cudaSuccess) {
    dh_set_global_error(std::string("dh_conserved_totals_static: cudaGetSymbolAddress: ") +
                        cudaGetErrorString(e));
    return DH_ERR_CUDA;
  }
  const int nblocks = (int)((n_cells + kCellsPerBlock - 1) / kCellsPerBlock);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (precision == DH_F64)
    static_totals_partial<double><<<nblocks, kThreads, 0, s>>>((const double*)U, n_cells, scratch);
  else
    static_totals_partial<float><<<nblocks, kThreads, 0, s>>>((const float*)U, n_cells, scratch);
  static_totals_final<<<1, 32, 0, s>>>(scratch, nblocks, totals_out);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    dh_set_global_error(std::string("dh_conserved_totals_static: launch: ") + cudaGetErrorString(e));
    return DH_ERR_CUDA;
  }
  return DH_OK;
}
