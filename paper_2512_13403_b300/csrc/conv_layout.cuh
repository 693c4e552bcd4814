// Padded, channel-group-major activation layout of the corrector's convolutions.
//
// An activation with C channels (C = 8 or 32) is stored as C/8 channel groups; group g is an
// array of `rows` 16-byte rows (8 bf16 channels each).  Row `guard + rho` holds padded cell rho
// of the (nx+2) x (ny+2) x (nz+2) volume, x fastest: padded coordinate p = cell coordinate + 1,
// and the one-cell halo around the grid holds periodic images of the opposite faces, edges and
// corners.  `guard` zero rows sit before and after the padded volume.
//
// Why: in this layout a 3x3x3 tap (dz, dy, dx) is a constant row shift
// dz (nx+2)(ny+2) + dy (nx+2) + dx, so 128 consecutive padded rows shifted by one tap are again
// 128 consecutive rows.  Rows are 16 bytes apart, which is exactly the no-swizzle K-major
// core-matrix layout with 128-byte stride between 8-row groups; the tensor-core operand of every
// tap is then a descriptor into the same shared-memory window, offset by 16 bytes per row.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace dh {

struct ConvGeom {
  int nx, ny, nz;
  int PX, PY;        // padded row and plane extents: nx + 2, ny + 2
  long long PXY;     // PX * PY
  long long rows;    // rows per channel group, guards included
  int guard;         // zero rows before (and at least as many after) the padded volume
  int win;           // rows of one shared-memory window: a 128-row tile and its +-(PX+1) reach
  long long ntiles;  // 128-row output tiles over the interior planes
};

__host__ __device__ inline ConvGeom conv_geom(int nx, int ny, int nz) {
  ConvGeom g;
  g.nx = nx; g.ny = ny; g.nz = nz;
  g.PX = nx + 2;
  g.PY = ny + 2;
  g.PXY = (long long)g.PX * g.PY;
  g.win = (130 + 2 * g.PX + 7) / 8 * 8;
  // a window of tile T for offset dz spans padded rows
  // [PXY (1 + dz) + 128 T - PX - 1, ... + win); the guards cover both ends
  g.guard = (g.PX + 136 + 7) / 8 * 8;
  g.rows = g.PXY * (nz + 2) + 2LL * g.guard;
  g.ntiles = ((long long)nz * g.PXY + 127) / 128;
  return g;
}

// Buffer row of cell coordinate (x, y, z), each in [-1, n].
__host__ __device__ inline long long pad_row(const ConvGeom& g, int x, int y, int z) {
  return g.guard + ((long long)(z + 1) * g.PY + (y + 1)) * g.PX + (x + 1);
}

// Writes 16 bytes (one channel group of cell (x, y, z)) to the cell's row and to every halo
// image of it.  `grp` points at the group's first row.
__device__ inline void store_with_images(uint4* __restrict__ grp, const ConvGeom& g, int x, int y,
                                         int z, uint4 v) {
  const long long r = pad_row(g, x, y, z);
  // row offset of the image across each axis (0: the cell is not on that face)
  const long long ox = x == 0 ? g.nx : (x == g.nx - 1 ? -g.nx : 0);
  const long long oy = y == 0 ? (long long)g.ny * g.PX : (y == g.ny - 1 ? -(long long)g.ny * g.PX : 0);
  const long long oz = z == 0 ? (long long)g.nz * g.PXY : (z == g.nz - 1 ? -(long long)g.nz * g.PXY : 0);
  grp[r] = v;
  if (ox) grp[r + ox] = v;
  if (oy) {
    grp[r + oy] = v;
    if (ox) grp[r + oy + ox] = v;
  }
  if (oz) {
    grp[r + oz] = v;
    if (ox) grp[r + oz + ox] = v;
    if (oy) {
      grp[r + oz + oy] = v;
      if (ox) grp[r + oz + oy + ox] = v;
    }
  }
}

}  // namespace dh
