// Binning helpers shared by the set-up kernels: the spread tile of a point,
// its cell inside a tile, and a block-wide exclusive scan.
#pragma once

#include <cuda_runtime.h>

#include "kernels.h"

namespace efgp {

// ---------------------------------------------------------------- tile map
// Tile of a point from its coordinates xa[0..D-1]; q receives the
// tile-local footprint start plus sub-cell offset per axis.
template <int D, typename TC, typename TR>
__device__ __forceinline__ int tile_of_coords(const TC* xa_in, const SortGeom& sg, TR (&q)[3], bool& bad) {
  constexpr int TB = tile_edge(D);
  int tc[3] = {0, 0, 0};
#pragma unroll
  for (int a = 0; a < D; ++a) {
    TC xa = xa_in[a];
    if (!(xa >= TC(0) && xa <= TC(1))) {  // also catches NaN
      bad = true;
      xa = TC(0);
    }
    int l0;
    TR f;
    GridPos<TC, TR>::get(xa, sg.gs, l0, f);
    int e0 = l0 + sg.off;
    e0 = max(0, min(e0, sg.nt[a] * TB - 1));
    tc[a] = e0 / TB;
    q[a] = (TR)(e0 - tc[a] * TB) + f;   // tile-local footprint start + offset
  }
  int t = tc[0];
  if (D > 1) t = t * sg.nt[1] + tc[1];
  if (D > 2) t = t * sg.nt[2] + tc[2];
  return t;
}

template <int D> struct RegTile;
template <> struct RegTile<1> { static constexpr int TB = 256; };
template <> struct RegTile<2> { static constexpr int TB = 16; };

template <int D>
__device__ __forceinline__ int reg_cell(const float* q, float* f) {
  constexpr int TB = RegTile<D>::TB;
  int c = 0;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    int l = (int)floorf(q[a]);
    l = max(0, min(l, TB - 1));
    f[a] = q[a] - (float)l;
    c = c * TB + l;
  }
  return c;
}

// exclusive scan of one int per thread over an NT-thread block
template <int NT>
__device__ __forceinline__ int block_excl_scan_n(int v, int* warp_tot) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int w = lane < NW ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < NW; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < NW) warp_tot[lane] = w;
  }
  __syncthreads();
  const int before = wid > 0 ? warp_tot[wid - 1] : 0;
  __syncthreads();
  return before + x - v;
}

}  // namespace efgp
