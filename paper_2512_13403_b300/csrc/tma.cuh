// Tensor-map (TMA) copies of state planes: the host encodes a 4D tiled tensor map over a
// planar state (x, y, z, field), and one thread of a CTA loads a box of it into shared memory
// with cp.async.bulk.tensor, completion counted in transaction bytes on an mbarrier.  The
// encoder comes from the driver through the runtime's entry-point query, so the library needs
// no link-time driver dependency.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace dh {

// Box loads of a state plane used by the stage kernels: the tile core, the x halos on each side
// and the y halos above and below, all five fields at once (the fourth dimension).
struct StageTma {
  CUtensorMap core, xh, yh;
};

// Encodes the three maps for a state of nx * ny * nz cells of `esize` bytes (4 or 8) at `base`:
// core boxes of bx x by cells, x-halo boxes of xw x by, y-halo boxes of bx x yh (cached per base
// address, shape and box sizes).  False if the driver refuses, in which case callers use plain
// asynchronous copies.
bool stage_tma_maps(const void* base, int nx, int ny, int nz, int esize, int bx, int by, int xw,
                    int yh, StageTma* out);

#if defined(__CUDACC__)
// Loads the box at coordinates (x, y, z, f) of `map` into shared memory at dst (128-byte
// aligned); the box's bytes complete on `bar`.
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            int z, int f, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(f), "r"(bar)
      : "memory");
}
#endif

}  // namespace dh
