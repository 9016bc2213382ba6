// Setup kernels (Algorithm steps 2-3): bin sort of the points by spread
// tile, type-1 spreading with the exponential-of-semicircle kernel into
// shared-memory tiles flushed once per tile visit, folding of the extended
// grid onto the periodic fine grid, and deconvolution that splits the packed
// strengths (1 + i y) into the Toeplitz generating vector w (eq. 88, as
// w = conj v) and the right-hand side D F^* y (eq. rhs).
#include <cmath>
#include <cstdio>
#include <string>
#include <type_traits>

#include "binning.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace efgp {

constexpr int kSortThreads = 256;
constexpr int kScatterPPT = 8;        // points per thread per scatter chunk
constexpr int kSmemBins = 8192;       // tiles handled with shared-memory histograms

template <int D, typename TC, typename TR>
__device__ __forceinline__ int tile_of(const TC* __restrict__ x, int soa, long long N, long long n, const SortGeom& sg,
                                       TR (&q)[3], bool& bad) {
  TC xa[3];
  if (!soa && D == 2 && sizeof(TC) == 4 && sg.x_vec) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(x) + n);
    xa[0] = (TC)v.x;
    xa[1] = (TC)v.y;
  } else {
#pragma unroll
    for (int a = 0; a < D; ++a) xa[a] = soa ? x[(long long)a * N + n] : x[n * D + a];
  }
  return tile_of_coords<D, TC, TR>(xa, sg, q, bad);
}

template <int D, typename TC, typename TR>
__global__ void __launch_bounds__(kSortThreads) bin_count_kernel(const TC* __restrict__ x, int soa, long long N,
                                                                 SortGeom sg, unsigned int* __restrict__ counts,
                                                                 int* range_flag) {
  extern __shared__ unsigned int hist[];
  constexpr int U = 8;   // points per thread per step: keeps several loads in flight
  const bool sm = sg.ntiles <= kSmemBins;
  if (sm) {
    for (int i = threadIdx.x; i < sg.ntiles; i += blockDim.x) hist[i] = 0u;
    __syncthreads();
  }
  bool bad = false;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long n0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; n0 < N; n0 += U * stride) {
    int t[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long n = n0 + u * stride;
      TR q[3];
      t[u] = n < N ? tile_of<D, TC, TR>(x, soa, N, n, sg, q, bad) : -1;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (t[u] < 0) continue;
      if (sm) atomicAdd(&hist[t[u]], 1u);
      else atomicAdd(&counts[t[u]], 1u);
    }
  }
  if (bad) atomicOr(range_flag, 1);
  if (sm) {
    __syncthreads();
    for (int i = threadIdx.x; i < sg.ntiles; i += blockDim.x)
      if (hist[i]) atomicAdd(&counts[i], hist[i]);
  }
}

// exclusive scan of tile counts (one block; tile counts are small)
__global__ void __launch_bounds__(1024) scan_tiles_kernel(const unsigned int* __restrict__ counts, int ntiles,
                                                          long long* __restrict__ tile_off,
                                                          long long* __restrict__ cursor) {
  __shared__ long long part[1024];
  const int per = (ntiles + blockDim.x - 1) / blockDim.x;
  const int a = threadIdx.x * per, b = min(ntiles, a + per);
  long long s = 0;
  for (int i = a; i < b; ++i) s += counts[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long run = 0;
    for (int i = 0; i < (int)blockDim.x; ++i) {
      const long long v = part[i];
      part[i] = run;
      run += v;
    }
    tile_off[ntiles] = run;
  }
  __syncthreads();
  long long run = part[threadIdx.x];
  for (int i = a; i < b; ++i) {
    tile_off[i] = run;
    cursor[i] = run;
    run += counts[i];
  }
}

template <int D, typename TC, typename TV, typename TR>
__global__ void __launch_bounds__(kSortThreads) bin_scatter_kernel(const TC* __restrict__ x, const TV* __restrict__ y,
                                                                   int soa, long long N, SortGeom sg,
                                                                   long long* __restrict__ cursor,
                                                                   TR* __restrict__ rec) {
  extern __shared__ __align__(128) unsigned char smraw[];
  const bool sm = sg.ntiles <= kSmemBins;
  long long* base = reinterpret_cast<long long*>(smraw);
  unsigned int* hist = reinterpret_cast<unsigned int*>(base + (sm ? sg.ntiles : 0));
  const long long chunk = (long long)blockDim.x * kScatterPPT;
  for (long long c0 = blockIdx.x * chunk; c0 < N; c0 += (long long)gridDim.x * chunk) {
    int tt[kScatterPPT];
    unsigned int rk[kScatterPPT];
    TR qq[kScatterPPT][D];
    TR yy[kScatterPPT];
    if (sm) {
      for (int i = threadIdx.x; i < sg.ntiles; i += blockDim.x) hist[i] = 0u;
      __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < kScatterPPT; ++p) {
      const long long n = c0 + (long long)p * blockDim.x + threadIdx.x;
      tt[p] = -1;
      if (n < N) {
        bool bad = false;
        TR q[3];
        tt[p] = tile_of<D, TC, TR>(x, soa, N, n, sg, q, bad);
#pragma unroll
        for (int a = 0; a < D; ++a) qq[p][a] = q[a];
        yy[p] = (TR)y[n];
        if (sm) rk[p] = atomicAdd(&hist[tt[p]], 1u);
      }
      if (!sm) {
        // warp-aggregated reservation directly in the global cursors
        const unsigned int act = __ballot_sync(0xffffffffu, tt[p] >= 0);
        if (tt[p] >= 0) {
          const unsigned int peers = __match_any_sync(act, tt[p]);
          const int leader = __ffs(peers) - 1;
          const int lane = threadIdx.x & 31;
          unsigned long long b0 = 0;
          if (lane == leader) b0 = atomicAdd(reinterpret_cast<unsigned long long*>(&cursor[tt[p]]),
                                             (unsigned long long)__popc(peers));
          b0 = __shfl_sync(peers, b0, leader);
          const long long pos = (long long)b0 + __popc(peers & ((1u << lane) - 1u));
#pragma unroll
          for (int a = 0; a < D; ++a) rec[(long long)a * sg.rstride + pos] = qq[p][a];
          rec[(long long)D * sg.rstride + pos] = yy[p];
        }
      }
    }
    if (sm) {
      __syncthreads();
      for (int i = threadIdx.x; i < sg.ntiles; i += blockDim.x) {
        const unsigned int h = hist[i];
        if (h) base[i] = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(&cursor[i]), (unsigned long long)h);
      }
      __syncthreads();
#pragma unroll
      for (int p = 0; p < kScatterPPT; ++p) {
        if (tt[p] >= 0) {
          const long long pos = base[tt[p]] + rk[p];
#pragma unroll
          for (int a = 0; a < D; ++a) rec[(long long)a * sg.rstride + pos] = qq[p][a];
          rec[(long long)D * sg.rstride + pos] = yy[p];
        }
      }
      __syncthreads();
    }
  }
}


// exclusive scan of one int per thread over a 256-thread block
__device__ __forceinline__ int block_excl_scan256(int v, int* warp_tot) {
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
    int w = lane < 8 ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < 8) warp_tot[lane] = w;   // inclusive warp prefix
  }
  __syncthreads();
  const int before = wid > 0 ? warp_tot[wid - 1] : 0;
  __syncthreads();
  return before + x - v;
}

// Sorting scatter: each block takes chunks of 256*PPT points, sorts a chunk
// by tile in shared memory (counting sort), reserves one range per tile in
// the global output with a single atomic per non-empty tile, and writes the
// chunk out tile run by tile run, so that consecutive threads store
// consecutive addresses.
constexpr int kSortedScatterMaxTiles = 4096;

template <int D, typename TC, typename TV, typename TR, int PPT>
__global__ void __launch_bounds__(256) bin_scatter_sorted_kernel(const TC* __restrict__ x, const TV* __restrict__ y,
                                                                 int soa, long long N, long long n_begin, SortGeom sg,
                                                                 long long* __restrict__ cursor,
                                                                 TR* __restrict__ rec) {
  constexpr int P = 256 * PPT;
  extern __shared__ __align__(128) unsigned char smraw[];
  const int T = sg.ntiles;
  TR* sq = reinterpret_cast<TR*>(smraw);                                   // (D+1) x P
  long long* base = reinterpret_cast<long long*>(sq + (size_t)(D + 1) * P);  // T
  int* stile = reinterpret_cast<int*>(base + T);                           // P
  unsigned int* hist = reinterpret_cast<unsigned int*>(stile + P);         // T
  int* lstart = reinterpret_cast<int*>(hist + T);                          // T
  __shared__ int wtot[8];
  const int slice = (T + 255) / 256;
  for (long long c0 = n_begin + blockIdx.x * (long long)P; c0 < N; c0 += (long long)gridDim.x * P) {
    for (int i = threadIdx.x; i < T; i += 256) hist[i] = 0u;
    __syncthreads();
    int tt[PPT];
    unsigned int rk[PPT];
    TR qq[PPT][D];
    TR yy[PPT];
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
      const long long n = c0 + (long long)p * 256 + threadIdx.x;
      tt[p] = -1;
      if (n < N) {
        bool bad = false;
        TR q[3];
        tt[p] = tile_of<D, TC, TR>(x, soa, N, n, sg, q, bad);
#pragma unroll
        for (int a = 0; a < D; ++a) qq[p][a] = q[a];
        yy[p] = (TR)y[n];
        rk[p] = atomicAdd(&hist[tt[p]], 1u);
      }
    }
    __syncthreads();
    // exclusive scan of the chunk's tile histogram; reserve global ranges
    {
      const int a = threadIdx.x * slice, b = min(T, a + slice);
      int sum = 0;
      for (int i = a; i < b; ++i) sum += (int)hist[i];
      int run = block_excl_scan256(sum, wtot);
      for (int i = a; i < b; ++i) {
        lstart[i] = run;
        const unsigned int h = hist[i];
        run += (int)h;
        if (h) base[i] = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(&cursor[i]),
                                              (unsigned long long)h);
      }
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
      if (tt[p] >= 0) {
        const int pos = lstart[tt[p]] + (int)rk[p];
#pragma unroll
        for (int a = 0; a < D; ++a) sq[(size_t)a * P + pos] = qq[p][a];
        sq[(size_t)D * P + pos] = yy[p];
        stile[pos] = tt[p];
      }
    }
    __syncthreads();
    const int nvalid = (int)min((long long)P, N - c0);
    for (int i = threadIdx.x; i < nvalid; i += 256) {
      const int t = stile[i];
      const long long g = base[t] + (i - lstart[t]);
#pragma unroll
      for (int a = 0; a <= D; ++a) rec[(long long)a * sg.rstride + g] = sq[(size_t)a * P + i];
    }
    __syncthreads();
  }
}


// Sorting scatter fed by bulk asynchronous copies (FP32 row-major
// coordinates and values): full chunks of 4096 points are copied into a
// double-buffered shared staging area while the previous chunk is binned,
// counting-sorted by tile and written out tile run by tile run.  The last
// partial chunk is left to bin_scatter_sorted_kernel.
constexpr int kTmaScatterThreads = 512;
constexpr int kTmaScatterPPT = 8;
constexpr int kTmaScatterChunk = kTmaScatterThreads * kTmaScatterPPT;
constexpr int kTmaScatterMaxSlice = (kSortedScatterMaxTiles + kTmaScatterThreads - 1) / kTmaScatterThreads;

template <int D>
__global__ void __launch_bounds__(kTmaScatterThreads, 1)
    bin_scatter_tma_kernel(const float* __restrict__ x, const float* __restrict__ y, long long nfull, long long N,
                           SortGeom sg, long long* __restrict__ cursor, float* __restrict__ rec, int* err) {
  constexpr int NT = kTmaScatterThreads, PPT = kTmaScatterPPT, P = kTmaScatterChunk;
  constexpr int SB = (D + 1) * P;
  extern __shared__ __align__(128) unsigned char smraw[];
  const int T = sg.ntiles;
  float* stage = reinterpret_cast<float*>(smraw);
  float* sq = stage + 2 * SB;
  int* stile = reinterpret_cast<int*>(sq + SB);
  long long* base = reinterpret_cast<long long*>(stile + P);
  unsigned int* hist = reinterpret_cast<unsigned int*>(base + T);
  int* lstart = reinterpret_cast<int*>(hist + T);
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int wtot[NT / 32];
  __shared__ int abort_flag;
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_barrier_init();
    abort_flag = 0;
  }
  __syncthreads();
  const uint32_t bytes_x = D * P * 4, bytes_y = P * 4;
  long long c = blockIdx.x;
  if (tid == 0 && c < nfull) {
    mbar_arrive_expect_tx(&bar[0], bytes_x + bytes_y);
    bulk_g2s(stage, x + c * (long long)P * D, bytes_x, &bar[0]);
    bulk_g2s(stage + D * P, y + c * (long long)P, bytes_y, &bar[0]);
  }
  const int slice = (T + NT - 1) / NT;
  int it = 0;
  bool pending_other = false;
  for (; c < nfull; c += gridDim.x, ++it) {
    const int b = it & 1;
    const long long cn = c + gridDim.x;
    pending_other = cn < nfull;
    if (tid == 0 && pending_other) {
      float* dst = stage + (b ^ 1) * SB;
      mbar_arrive_expect_tx(&bar[b ^ 1], bytes_x + bytes_y);
      bulk_g2s(dst, x + cn * (long long)P * D, bytes_x, &bar[b ^ 1]);
      bulk_g2s(dst + D * P, y + cn * (long long)P, bytes_y, &bar[b ^ 1]);
    }
    if (!mbar_wait_bounded(&bar[b], (uint32_t)((it >> 1) & 1), err)) abort_flag = 1;
    for (int i = tid; i < T; i += NT) hist[i] = 0u;
    __syncthreads();
    if (abort_flag) break;
    const float* sx = stage + b * SB;
    int tt[PPT];
    unsigned int rk[PPT];
    float qk[PPT][D];   // tile-local coordinates, kept for the write-out
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
      const int k = p * NT + tid;
      float xa[3];
#pragma unroll
      for (int a = 0; a < D; ++a) xa[a] = sx[k * D + a];
      bool bad = false;
      float q[3];
      tt[p] = tile_of_coords<D, float, float>(xa, sg, q, bad);
#pragma unroll
      for (int a = 0; a < D; ++a) qk[p][a] = q[a];
      rk[p] = atomicAdd(&hist[tt[p]], 1u);
    }
    __syncthreads();
    // output runs: reserve each tile's run with a global fetch-add whose
    // result is only stored after the shared-memory scatter below, so the
    // atomics' round trip overlaps the barrier and the scatter
    const int a0 = tid * slice, a1 = min(T, a0 + slice);
    unsigned long long got[kTmaScatterMaxSlice];
    {
      int sum = 0;
      for (int i = a0; i < a1; ++i) sum += (int)hist[i];
      int run = block_excl_scan_n<NT>(sum, wtot);
#pragma unroll
      for (int u = 0; u < kTmaScatterMaxSlice; ++u) {
        const int i = a0 + u;
        got[u] = 0ull;
        if (i < a1) {
          lstart[i] = run;
          const unsigned int h = hist[i];
          run += (int)h;
          if (h) got[u] = atomicAdd(reinterpret_cast<unsigned long long*>(&cursor[i]), (unsigned long long)h);
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
      const int k = p * NT + tid;
      const int pos = lstart[tt[p]] + (int)rk[p];
#pragma unroll
      for (int a = 0; a < D; ++a) sq[a * P + pos] = qk[p][a];
      sq[D * P + pos] = sx[D * P + k];
      stile[pos] = tt[p];
    }
#pragma unroll
    for (int u = 0; u < kTmaScatterMaxSlice; ++u)
      if (a0 + u < a1) base[a0 + u] = (long long)got[u];
    __syncthreads();
    for (int i = tid; i < P; i += NT) {
      const int t = stile[i];
      const long long g = base[t] + (i - lstart[t]);
#pragma unroll
      for (int a = 0; a <= D; ++a) rec[(long long)a * sg.rstride + g] = sq[a * P + i];
    }
    __syncthreads();
  }
  // after an abandoned wait, let the copy already issued into the other
  // buffer land (bounded) before the block's shared memory is released
  if (abort_flag && tid == 0 && pending_other) mbar_wait_bounded(&bar[(it & 1) ^ 1], (uint32_t)(((it + 1) >> 1) & 1), err);
}

// Sorting scatter over 8192-point chunks (at most 1024 tiles): twice the
// points of a chunk per tile run (longer write runs, half the cursor
// reservations per point).  One staging buffer: each point's tile-local
// coordinates overwrite its coordinates in place, the chunk is reordered into
// a second buffer, and the next chunk's bulk copy is issued into the staging
// buffer then, so it lands while the reordered chunk is written out.
constexpr int kBigScatterPPT = 16;
constexpr int kBigScatterChunk = kTmaScatterThreads * kBigScatterPPT;
constexpr int kBigScatterMaxTiles = 1024;
constexpr int kBigScatterMaxSlice = (kBigScatterMaxTiles + kTmaScatterThreads - 1) / kTmaScatterThreads;

template <int D>
__global__ void __launch_bounds__(kTmaScatterThreads, 1)
    bin_scatter_big_kernel(const float* __restrict__ x, const float* __restrict__ y, long long nfull, SortGeom sg,
                           long long* __restrict__ cursor, float* __restrict__ rec, int* err) {
  constexpr int NT = kTmaScatterThreads, PPT = kBigScatterPPT, P = kBigScatterChunk;
  extern __shared__ __align__(128) unsigned char smraw[];
  const int T = sg.ntiles;
  float* stage = reinterpret_cast<float*>(smraw);                                  // (D+1) x P: x then y
  float* sq = stage + (D + 1) * P;                                                  // (D+1) x P, sorted
  unsigned short* stile = reinterpret_cast<unsigned short*>(sq + (D + 1) * P);     // P
  long long* base = reinterpret_cast<long long*>(stile + P);                       // T
  unsigned int* hist = reinterpret_cast<unsigned int*>(base + T);                  // T
  int* lstart = reinterpret_cast<int*>(hist + T);                                  // T
  __shared__ __align__(8) uint64_t bar;
  __shared__ int wtot[NT / 32];
  __shared__ int abort_flag;
  const int tid = threadIdx.x;
  const uint32_t bytes_x = D * P * 4, bytes_y = P * 4;
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
    abort_flag = 0;
  }
  __syncthreads();
  long long c = blockIdx.x;
  if (tid == 0 && c < nfull) {
    mbar_arrive_expect_tx(&bar, bytes_x + bytes_y);
    bulk_g2s(stage, x + c * (long long)P * D, bytes_x, &bar);
    bulk_g2s(stage + D * P, y + c * (long long)P, bytes_y, &bar);
  }
  const int slice = (T + NT - 1) / NT;
  uint32_t ph = 0u;
  bool pending = c < nfull;
  for (; c < nfull; c += gridDim.x) {
    for (int i = tid; i < T; i += NT) hist[i] = 0u;
    if (mbar_wait_bounded(&bar, ph, err)) {
      ph ^= 1u;
      pending = false;
    } else {
      abort_flag = 1;   // (the copy waited for is still in flight: pending)
    }
    __syncthreads();
    if (abort_flag) break;
    int tt[PPT];
    unsigned int rk[PPT];
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
      const int k = p * NT + tid;
      float xa[3];
#pragma unroll
      for (int a = 0; a < D; ++a) xa[a] = stage[k * D + a];
      bool bad = false;
      float q[3];
      tt[p] = tile_of_coords<D, float, float>(xa, sg, q, bad);
#pragma unroll
      for (int a = 0; a < D; ++a) stage[k * D + a] = q[a];   // same thread, same slot
      rk[p] = atomicAdd(&hist[tt[p]], 1u);
    }
    __syncthreads();
    const int a0 = tid * slice, a1 = min(T, a0 + slice);
    unsigned long long got[kBigScatterMaxSlice];
    {
      int sum = 0;
      for (int i = a0; i < a1; ++i) sum += (int)hist[i];
      int run = block_excl_scan_n<NT>(sum, wtot);
#pragma unroll
      for (int u = 0; u < kBigScatterMaxSlice; ++u) {
        const int i = a0 + u;
        got[u] = 0ull;
        if (i < a1) {
          lstart[i] = run;
          const unsigned int h = hist[i];
          run += (int)h;
          if (h) got[u] = atomicAdd(reinterpret_cast<unsigned long long*>(&cursor[i]), (unsigned long long)h);
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
      const int k = p * NT + tid;
      const int pos = lstart[tt[p]] + (int)rk[p];
#pragma unroll
      for (int a = 0; a < D; ++a) sq[a * P + pos] = stage[k * D + a];
      sq[D * P + pos] = stage[D * P + k];
      stile[pos] = (unsigned short)tt[p];
    }
#pragma unroll
    for (int u = 0; u < kBigScatterMaxSlice; ++u)
      if (a0 + u < a1) base[a0 + u] = (long long)got[u];
    __syncthreads();
    // the staging buffer is free: the next chunk's copy lands during the write-out
    const long long cn = c + gridDim.x;
    if (cn < nfull) {
      pending = true;
      if (tid == 0) {
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&bar, bytes_x + bytes_y);
        bulk_g2s(stage, x + cn * (long long)P * D, bytes_x, &bar);
        bulk_g2s(stage + D * P, y + cn * (long long)P, bytes_y, &bar);
      }
    }
    for (int i = tid; i < P; i += NT) {
      const int t = stile[i];
      const long long g = base[t] + (i - lstart[t]);
#pragma unroll
      for (int a = 0; a <= D; ++a) rec[(long long)a * sg.rstride + g] = sq[a * P + i];
    }
    __syncthreads();
  }
  // after an abandoned wait, let a copy already issued land (bounded) before
  // the block's shared memory is released
  if (abort_flag && tid == 0 && pending) mbar_wait_bounded(&bar, ph, err);
}

size_t scatter_big_smem(int d, int ntiles) {
  const size_t P = kBigScatterChunk;
  return sizeof(float) * (2 * (size_t)(d + 1) * P) + sizeof(unsigned short) * P +
         (sizeof(long long) + 2 * sizeof(int)) * ntiles;
}

size_t scatter_tma_smem(int d, int ntiles) {
  const size_t P = kTmaScatterChunk;
  return sizeof(float) * (3 * (size_t)(d + 1) * P) + sizeof(int) * P + (sizeof(long long) + 2 * sizeof(int)) * ntiles;
}

// ---------------------------------------------------------------- spread
// One block per segment of the sorted records; for every tile the segment
// overlaps, accumulate that tile's points into a shared-memory tile (with
// halo) in TR precision, then add the tile into the FP64 extended grid.
template <int D, int W, typename TR>
__global__ void __launch_bounds__(256) spread_kernel(const TR* __restrict__ rec, long long N, SortGeom sg,
                                                     const long long* __restrict__ tile_off, long long seg_len,
                                                     EsCoef<TR> cf, double2* __restrict__ E) {
  extern __shared__ __align__(128) unsigned char smraw[];
  TR* acc = reinterpret_cast<TR*>(smraw);
  __shared__ int t_first;
  const int TB = sg.TB;
  const int S = TB + W - 1;
  int cells = S;
  if (D > 1) cells *= S;
  if (D > 2) cells *= S;
  const long long s0 = blockIdx.x * seg_len;
  const long long s1 = min(N, s0 + seg_len);
  if (s0 >= s1) return;
  if (threadIdx.x == 0) {
    // largest t < ntiles with tile_off[t] <= s0
    int lo = 0, hi = sg.ntiles - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tile_off[mid] <= s0) lo = mid; else hi = mid - 1;
    }
    t_first = lo;
  }
  __syncthreads();
  for (int t = t_first; t < sg.ntiles; ++t) {
    const long long ta = tile_off[t], tb = tile_off[t + 1];
    if (ta >= s1) break;
    const long long a = max(s0, ta), b = min(s1, tb);
    if (a >= b) continue;
    for (int c = threadIdx.x; c < 2 * cells; c += blockDim.x) acc[c] = TR(0);
    __syncthreads();
    for (long long i = a + threadIdx.x; i < b; i += blockDim.x) {
      TR wt[D][W];
      int lb[D];
#pragma unroll
      for (int dd = 0; dd < D; ++dd) {
        const TR qv = rec[(long long)dd * sg.rstride + i];
        int l = (int)floor(qv);
        l = max(0, min(l, TB - 1));
        lb[dd] = l;
        es_weights<TR, W>(qv - (TR)l, cf, wt[dd]);
      }
      const TR yv = rec[(long long)D * sg.rstride + i];
      if (D == 1) {
#pragma unroll
        for (int u = 0; u < W; ++u) {
          TR* c = acc + 2 * (lb[0] + u);
          atomicAdd(c, wt[0][u]);
          atomicAdd(c + 1, wt[0][u] * yv);
        }
      } else if (D == 2) {
#pragma unroll
        for (int u = 0; u < W; ++u) {
          const TR wa = wt[0][u], wy = wa * yv;
          TR* row = acc + 2 * ((lb[0] + u) * S + lb[1]);
#pragma unroll
          for (int v = 0; v < W; ++v) {
            atomicAdd(row + 2 * v, wa * wt[D - 1][v]);
            atomicAdd(row + 2 * v + 1, wy * wt[D - 1][v]);
          }
        }
      } else {
        for (int u = 0; u < W; ++u) {
#pragma unroll
          for (int v = 0; v < W; ++v) {
            const TR wa = wt[0][u] * wt[1 % D][v], wy = wa * yv;
            TR* row = acc + 2 * (((lb[0] + u) * S + lb[1 % D] + v) * S + lb[D - 1]);
#pragma unroll
            for (int z = 0; z < W; ++z) {
              atomicAdd(row + 2 * z, wa * wt[D - 1][z]);
              atomicAdd(row + 2 * z + 1, wy * wt[D - 1][z]);
            }
          }
        }
      }
    }
    __syncthreads();
    // flush the tile into the FP64 extended grid
    int tcv[3];
    {
      int r = t;
      for (int dd = D - 1; dd >= 0; --dd) {
        tcv[dd] = r % sg.nt[dd];
        r /= sg.nt[dd];
      }
    }
    for (int c = threadIdx.x; c < cells; c += blockDim.x) {
      const TR re = acc[2 * c], im = acc[2 * c + 1];
      if (re == TR(0) && im == TR(0)) continue;
      int rem = c;
      long long gi = 0;
      bool inside = true;
      int loc[3];
      for (int dd = D - 1; dd >= 0; --dd) {
        loc[dd] = rem % S;
        rem /= S;
      }
      for (int dd = 0; dd < D; ++dd) {
        const int e = tcv[dd] * TB + loc[dd];
        inside = inside && (e < sg.nEx);
        gi = gi * sg.nEx + e;
      }
      if (inside) {
        atomicAdd(&E[gi].x, (double)re);
        atomicAdd(&E[gi].y, (double)im);
      }
    }
    __syncthreads();
  }
}

// Register-accumulating spread (FP32 records, d = 1 or 2, W <= 8).  The
// points of a tile are processed in batches: a counting sort in shared
// memory groups each batch by fine-grid cell, then thread t, which owns
// cell t of the tile, adds the weights of every point of its cell into a
// W^d footprint held in registers.  The registers are added into the
// shared-memory tile in W^d phases in which all threads write distinct
// cells (no atomics), and the tile is flushed to the FP64 extended grid
// once per tile visit.
constexpr int kRegThreads = 256;
constexpr int kRegBatch = 8192;
constexpr int kRegBatchPad = kRegBatch + kRegBatch / 32;

__device__ __forceinline__ int pad32(int p) { return p + (p >> 5); }

// exclusive block scan of one int per thread (blockDim.x == kRegThreads)
__device__ __forceinline__ int block_excl_scan(int v, int* warp_tot) {
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
    int w = lane < kRegThreads / 32 ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kRegThreads / 32) warp_tot[lane] = w;   // inclusive warp prefix
  }
  __syncthreads();
  const int before = wid > 0 ? warp_tot[wid - 1] : 0;
  return before + x - v;
}

template <int D, int W>
__global__ void __launch_bounds__(kRegThreads, 2) spread_reg_kernel(const float* __restrict__ rec, long long N,
                                                                     SortGeom sg, const long long* __restrict__ tile_off,
                                                                     long long seg_len, EsCoef<float> cf,
                                                                     double2* __restrict__ E) {
  constexpr int TB = RegTile<D>::TB;
  constexpr int S = TB + W - 1;
  constexpr int CELLS = (D == 1) ? S : S * S;
  constexpr int FP = (D == 1) ? W : W * W;
  extern __shared__ __align__(128) unsigned char smraw[];
  float* sf = reinterpret_cast<float*>(smraw);            // D x kRegBatchPad fractional offsets
  float* sy = sf + D * kRegBatchPad;                        // kRegBatchPad values
  float* tile = sy + kRegBatchPad;                          // 2*CELLS
  int* cnt = reinterpret_cast<int*>(tile + 2 * CELLS);      // kRegThreads
  int* cur = cnt + kRegThreads;                             // kRegThreads
  int* wtot = cur + kRegThreads;                            // 32
  __shared__ int t_first;
  const int t = threadIdx.x;
  const long long s0 = blockIdx.x * seg_len;
  const long long s1 = min(N, s0 + seg_len);
  if (s0 >= s1) return;
  if (t == 0) {
    int lo = 0, hi = sg.ntiles - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tile_off[mid] <= s0) lo = mid; else hi = mid - 1;
    }
    t_first = lo;
  }
  __syncthreads();
  // cell owned by this thread
  int own[D];
  {
    int r = t;
#pragma unroll
    for (int a = D - 1; a >= 0; --a) {
      own[a] = r % TB;
      r /= TB;
    }
  }
  for (int tt = t_first; tt < sg.ntiles; ++tt) {
    const long long ta = tile_off[tt], tb = tile_off[tt + 1];
    if (ta >= s1) break;
    const long long a0 = max(s0, ta), b0 = min(s1, tb);
    if (a0 >= b0) continue;
    float are[FP], aim[FP];
#pragma unroll
    for (int i = 0; i < FP; ++i) are[i] = aim[i] = 0.f;
    for (long long p0 = a0; p0 < b0; p0 += kRegBatch) {
      const int nbat = (int)min((long long)kRegBatch, b0 - p0);
      cnt[t] = 0;
      __syncthreads();
#pragma unroll 4
      for (int k = t; k < nbat; k += kRegThreads) {
        float q[D], f[D];
#pragma unroll
        for (int a = 0; a < D; ++a) q[a] = rec[(long long)a * sg.rstride + p0 + k];
        atomicAdd(&cnt[reg_cell<D>(q, f)], 1);
      }
      __syncthreads();
      const int mine = cnt[t];
      const int st = block_excl_scan(mine, wtot);
      cur[t] = st;
      __syncthreads();
#pragma unroll 4
      for (int k = t; k < nbat; k += kRegThreads) {
        float q[D], f[D];
#pragma unroll
        for (int a = 0; a < D; ++a) q[a] = rec[(long long)a * sg.rstride + p0 + k];
        const float yv = rec[(long long)D * sg.rstride + p0 + k];
        const int pos = pad32(atomicAdd(&cur[reg_cell<D>(q, f)], 1));
#pragma unroll
        for (int a = 0; a < D; ++a) sf[a * kRegBatchPad + pos] = f[a];
        sy[pos] = yv;
      }
      __syncthreads();
      for (int k = 0; k < mine; ++k) {
        const int pos = pad32(st + k);
        float w0[W], w1[W];
        es_weights<float, W>(sf[pos], cf, w0);
        const float yv = sy[pos];
        if (D == 1) {
#pragma unroll
          for (int u = 0; u < W; ++u) {
            are[u] += w0[u];
            aim[u] = fmaf(w0[u], yv, aim[u]);
          }
        } else {
          es_weights<float, W>(sf[(D - 1) * kRegBatchPad + pos], cf, w1);
#pragma unroll
          for (int u = 0; u < W; ++u) {
            const float wa = w0[u], wy = w0[u] * yv;
#pragma unroll
            for (int v = 0; v < W; ++v) {
              are[u * W + v] = fmaf(wa, w1[v], are[u * W + v]);
              aim[u * W + v] = fmaf(wy, w1[v], aim[u * W + v]);
            }
          }
        }
      }
      __syncthreads();
    }
    // registers -> shared tile, one footprint offset per phase
    for (int c = t; c < 2 * CELLS; c += kRegThreads) tile[c] = 0.f;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < FP; ++i) {
      int cell;
      if (D == 1) cell = own[0] + i;
      else cell = (own[0] + i / W) * S + own[D - 1] + i % W;
      tile[2 * cell] += are[i];
      tile[2 * cell + 1] += aim[i];
      __syncthreads();
    }
    // shared tile -> FP64 extended grid
    int tcv[3] = {0, 0, 0};
    {
      int r = tt;
      for (int dd = D - 1; dd >= 0; --dd) {
        tcv[dd] = r % sg.nt[dd];
        r /= sg.nt[dd];
      }
    }
    for (int c = t; c < CELLS; c += kRegThreads) {
      const float re = tile[2 * c], im = tile[2 * c + 1];
      if (re == 0.f && im == 0.f) continue;
      int loc[2];
      if (D == 1) loc[0] = c;
      else { loc[0] = c / S; loc[1] = c % S; }
      long long gi = 0;
      bool inside = true;
      for (int dd = 0; dd < D; ++dd) {
        const int e = tcv[dd] * TB + loc[dd];
        inside = inside && (e < sg.nEx);
        gi = gi * sg.nEx + e;
      }
      if (inside) {
        atomicAdd(&E[gi].x, (double)re);
        atomicAdd(&E[gi].y, (double)im);
      }
    }
    __syncthreads();
  }
}


constexpr int kSpreadUnroll = 2;   // points of a cell whose weights are evaluated together (4: no gain)

// Register-accumulating spread with two resident blocks per SM (FP32
// records, d = 1 or 2).  One thread owns each of the 256 cells of a tile.
// A batch of the tile-sorted records is copied into a staging buffer by one
// bulk asynchronous copy per array, counted by fine cell, and reordered by
// cell into a second buffer (coordinates, value); the staging buffer
// is then free, so the copy of the next batch lands while the threads walk
// their cells' runs from contiguous shared memory.  The two blocks of an SM
// interleave: the sorting phases and barrier waits of one overlap the
// multiply-adds of the other.
constexpr int kPairThreads = 256;
constexpr int kPairBatch = 4096;
constexpr int kPairSlot = kPairBatch + 8;   // floats per staged array

template <int D, int W>
__global__ void __launch_bounds__(kPairThreads, 2)
    spread_pair_kernel(const float* __restrict__ rec, long long N, long long rstride, SortGeom sg,
                       const long long* __restrict__ tile_off, long long seg_len, EsCoef<float> cf,
                       double2* __restrict__ E, int* err) {
  constexpr int TB = RegTile<D>::TB;
  constexpr int S = TB + W - 1;
  constexpr int CELLS = (D == 1) ? S : S * S;
  constexpr int FP = (D == 1) ? W : W * W;
  constexpr int NT = kPairThreads;
  constexpr int B = kPairBatch;
  constexpr int SLOT = kPairSlot;
  constexpr int NA = D + 1;   // arrays per record: D coordinates, one value
  static_assert(NT == 256, "one thread per cell of a 256-cell tile");
  extern __shared__ __align__(128) unsigned char smraw[];
  float* stage = reinterpret_cast<float*>(smraw);                  // NA * SLOT
  float* sorted = stage + NA * SLOT;                                // NA * B
  float* tile = sorted + NA * B;                                    // 2 * CELLS
  int* cnt = reinterpret_cast<int*>(tile + 2 * CELLS);              // 256
  int* cur = cnt + 256;                                             // 256
  unsigned char* ucell = reinterpret_cast<unsigned char*>(cur + 256);   // B
  __shared__ __align__(8) uint64_t bar;
  __shared__ int wtot[32];
  __shared__ int it_tile[2], it_n[2];
  __shared__ long long it_p0[2];
  __shared__ int it_off;
  __shared__ int abort_flag;
  const int t = threadIdx.x;
  const long long s0 = blockIdx.x * seg_len;
  const long long s1 = min(N, s0 + seg_len);
  if (s0 >= s1) return;

  // next batch after (tile tt, start p0, count n): false at the segment end
  auto next_item = [&](int& tt, long long& p0, int& n) -> bool {
    const long long b = min(s1, tile_off[tt + 1]);
    p0 += n;
    if (p0 < b) {
      n = (int)min((long long)B, b - p0);
      return true;
    }
    for (++tt; tt < sg.ntiles; ++tt) {
      const long long ta = tile_off[tt];
      if (ta >= s1) return false;
      const long long a = max(s0, ta), bb = min(s1, tile_off[tt + 1]);
      if (a < bb) {
        p0 = a;
        n = (int)min((long long)B, bb - a);
        return true;
      }
    }
    return false;
  };
  // copy the batch's arrays into the staging buffer: a window of whole
  // 16-byte groups, (p0 + n + 3) & ~3 <= rstride - 4 keeps it in bounds
  auto issue = [&](long long p0, int n) {
    const long long pa = p0 & ~3ll;
    const long long pe = (p0 + n + 3) & ~3ll;
    const uint32_t bytes = (uint32_t)((pe - pa) * 4);
    mbar_arrive_expect_tx(&bar, bytes * NA);
    for (int a = 0; a < NA; ++a) bulk_g2s(stage + a * SLOT, rec + a * rstride + pa, bytes, &bar);
    it_off = (int)(p0 - pa);
  };

  if (t == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
    abort_flag = 0;
    int lo = 0, hi = sg.ntiles - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tile_off[mid] <= s0) lo = mid; else hi = mid - 1;
    }
    int tt = lo;
    long long p0 = s0;
    int n = 0;
    bool ok;
    const long long b = min(s1, tile_off[tt + 1]);
    if (p0 < b) {
      n = (int)min((long long)B, b - p0);
      ok = true;
    } else {
      ok = next_item(tt, p0, n);
    }
    it_tile[0] = ok ? tt : -1;
    it_p0[0] = p0;
    it_n[0] = n;
    if (ok) issue(p0, n);
  }
  __syncthreads();

  int own[D];
  {
    int r = t;
#pragma unroll
    for (int a = D - 1; a >= 0; --a) {
      own[a] = r % TB;
      r /= TB;
    }
  }
  float2 acc[FP];   // (strength 1, strength y) per footprint cell
#pragma unroll
  for (int i = 0; i < FP; ++i) acc[i] = make_float2(0.f, 0.f);
  // by cell: the coordinates (a float2 per point in 2D) and the values
  float* q1s = sorted;                                      // d = 1
  float2* q2s = reinterpret_cast<float2*>(sorted);          // d = 2
  float* ys = sorted + D * B;
  float ownf[D];
#pragma unroll
  for (int a = 0; a < D; ++a) ownf[a] = (float)own[a];

  int abort_it = -1;
  for (int it = 0;; ++it) {
    const int b = it & 1;
    const int tt = it_tile[b];
    if (tt < 0) break;
    const int n = it_n[b];
    if (!mbar_wait_bounded(&bar, (uint32_t)(it & 1), err)) abort_flag = 1;
    cnt[t] = 0;
    __syncthreads();
    if (abort_flag) {
      abort_it = it;
      break;
    }
    const int off = it_off;
    const float* sq0 = stage + off;
    const float* sq1 = stage + (D - 1) * SLOT + off;
    const float* sy = stage + D * SLOT + off;
    // count by cell (the cell is kept for the reorder)
    for (int k = t; k < n; k += NT) {
      float q[D], f[D];
      q[0] = sq0[k];
      if (D == 2) q[D - 1] = sq1[k];
      const int c = reg_cell<D>(q, f);
      ucell[k] = (unsigned char)c;
      atomicAdd(&cnt[c], 1);
    }
    __syncthreads();
    const int mine = cnt[t];
    const int start = block_excl_scan_n<NT>(mine, wtot);
    cur[t] = start;
    __syncthreads();
    // reorder by cell
    for (int k = t; k < n; k += NT) {
      const int pos = atomicAdd(&cur[ucell[k]], 1);
      if (D == 2) q2s[pos] = make_float2(sq0[k], sq1[k]);
      else q1s[pos] = sq0[k];
      ys[pos] = sy[k];
    }
    __syncthreads();
    // the staging buffer is free: start the copy of the next batch
    if (t == 0) {
      int nt = tt;
      long long np0 = it_p0[b];
      int nn = n;
      const bool ok = next_item(nt, np0, nn);
      it_tile[b ^ 1] = ok ? nt : -1;
      it_p0[b ^ 1] = np0;
      it_n[b ^ 1] = nn;
      if (ok) issue(np0, nn);
    }
    // the run of my cell, two points per step (independent weight chains)
    {
      auto add_point = [&](const float (&w0)[W], const float (&w1)[W], float yv) {
        const float2 c2 = make_float2(1.f, yv);
        if (D == 1) {
#pragma unroll
          for (int u = 0; u < W; ++u) acc[u] = __ffma2_rn(make_float2(w0[u], w0[u]), c2, acc[u]);
        } else {
#pragma unroll
          for (int u = 0; u < W; ++u) {
            const float2 wa = __fmul2_rn(make_float2(w0[u], w0[u]), c2);
#pragma unroll
            for (int v = 0; v < W; ++v) acc[u * W + v] = __ffma2_rn(wa, make_float2(w1[v], w1[v]), acc[u * W + v]);
          }
        }
      };
      // in-cell offsets f = q - (cell corner), as the cell binning takes them
      auto weights = [&](int j, float (&w0)[W], float (&w1)[W]) {
        if (D == 2) {
          const float2 qq = q2s[start + j];
          es_weights_x2<W>(qq.x - ownf[0], cf, w0);
          es_weights_x2<W>(qq.y - ownf[D - 1], cf, w1);
        } else {
          es_weights_x2<W>(q1s[start + j] - ownf[0], cf, w0);
        }
      };
      const float* pys = ys + start;
      constexpr int UP = kSpreadUnroll;
      int j = 0;
      for (; j + UP - 1 < mine; j += UP) {
        float w0[UP][W], w1[UP][W], yv[UP];
#pragma unroll
        for (int e = 0; e < UP; ++e) {
          weights(j + e, w0[e], w1[e]);
          yv[e] = pys[j + e];
        }
#pragma unroll
        for (int e = 0; e < UP; ++e) add_point(w0[e], w1[e], yv[e]);
      }
      for (; j < mine; ++j) {
        float w0[W], w1[W];
        weights(j, w0, w1);
        add_point(w0, w1, pys[j]);
      }
    }
    __syncthreads();
    // last batch of this tile visit: registers -> shared tile -> FP64 grid
    if (it_tile[b ^ 1] != tt) {
      for (int c = t; c < 2 * CELLS; c += NT) tile[c] = 0.f;
      __syncthreads();
#pragma unroll
      for (int i = 0; i < FP; ++i) {
        int cc;
        if (D == 1) cc = own[0] + i;
        else cc = (own[0] + i / W) * S + own[D - 1] + i % W;
        tile[2 * cc] += acc[i].x;
        tile[2 * cc + 1] += acc[i].y;
        acc[i] = make_float2(0.f, 0.f);
        __syncthreads();
      }
      int tcv[2] = {0, 0};
      {
        int r = tt;
        for (int dd = D - 1; dd >= 0; --dd) {
          tcv[dd] = r % sg.nt[dd];
          r /= sg.nt[dd];
        }
      }
      for (int c = t; c < CELLS; c += NT) {
        const float re = tile[2 * c], im = tile[2 * c + 1];
        if (re == 0.f && im == 0.f) continue;
        int loc[2];
        if (D == 1) loc[0] = c;
        else { loc[0] = c / S; loc[1] = c % S; }
        long long gi = 0;
        bool inside = true;
        for (int dd = 0; dd < D; ++dd) {
          const int e = tcv[dd] * TB + loc[dd];
          inside = inside && (e < sg.nEx);
          gi = gi * sg.nEx + e;
        }
        if (inside) {
          atomicAdd(&E[gi].x, (double)re);
          atomicAdd(&E[gi].y, (double)im);
        }
      }
      __syncthreads();
    }
  }
  // after an abandoned wait, let the copy already issued land (bounded)
  // before the block's shared memory is released
  if (abort_it >= 0 && t == 0) mbar_wait_bounded(&bar, (uint32_t)(abort_it & 1), nullptr);
}

size_t spread_pair_smem(int d, int W) {
  const int TB = d == 1 ? RegTile<1>::TB : RegTile<2>::TB;
  const int S = TB + W - 1;
  const int cells = d == 1 ? S : S * S;
  return sizeof(float) * ((size_t)(d + 1) * (kPairSlot + kPairBatch) + 2 * cells) + sizeof(int) * 512 +
         sizeof(unsigned char) * kPairBatch;
}

size_t spread_reg_smem(int d, int W) {
  const int TB = d == 1 ? RegTile<1>::TB : RegTile<2>::TB;
  const int S = TB + W - 1;
  const int cells = d == 1 ? S : S * S;
  return sizeof(float) * ((size_t)(d + 1) * kRegBatchPad + 2 * cells) + sizeof(int) * (2 * kRegThreads + 32);
}

// ---------------------------------------------------------------- fold / deconvolve
// P[p] = sum of E[e] over extended indices e = (p + off) mod nf + j*nf < nEx
template <int D, typename T>
__global__ void fold_kernel(const double2* __restrict__ E, int nEx, int off, int nf, cplx<T>* __restrict__ P) {
  long long total = nf;
  if (D > 1) total *= nf;
  if (D > 2) total *= nf;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    int p[3] = {0, 0, 0};
    long long r = idx;
    for (int a = D - 1; a >= 0; --a) {
      p[a] = (int)(r % nf);
      r /= nf;
    }
    int e0[3];
    for (int a = 0; a < D; ++a) e0[a] = (p[a] + off) % nf;
    double sx = 0.0, sy = 0.0;
    for (int i0 = e0[0]; i0 < nEx; i0 += nf) {
      if constexpr (D == 1) {
        const double2 v = E[i0];
        sx += v.x;
        sy += v.y;
      } else {
        for (int i1 = e0[1 % D]; i1 < nEx; i1 += nf) {
          if constexpr (D == 2) {
            const double2 v = E[(long long)i0 * nEx + i1];
            sx += v.x;
            sy += v.y;
          } else {
            for (int i2 = e0[D - 1]; i2 < nEx; i2 += nf) {
              const double2 v = E[((long long)i0 * nEx + i1) * nEx + i2];
              sx += v.x;
              sy += v.y;
            }
          }
        }
      }
    }
    P[idx] = mk<T>((T)sx, (T)sy);
  }
}

// Modes k in J_{2m}: G = FFT of the packed grid.  With G1 and Gy the
// transforms of the real grids of strengths 1 and y:
//   G1(k) = (G(k) + conj G(-k))/2,  Gy(k) = (G(k) - conj G(-k))/(2i).
// w_k = G1(k)/prod psihat, b_j = D_j Gy(j)/prod psihat for j in J_m.
template <int D, typename T>
__global__ void deconv_split_kernel(const cplx<T>* __restrict__ G, int nf, int m, const double* __restrict__ corr,
                                    const double* __restrict__ Dw, double2* __restrict__ w, double2* __restrict__ b) {
  const int K = 4 * m + 1, n1 = 2 * m + 1;
  long long total = K;
  if (D > 1) total *= K;
  if (D > 2) total *= K;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    int k[3] = {0, 0, 0};
    long long r = idx;
    for (int a = D - 1; a >= 0; --a) {
      k[a] = (int)(r % K) - 2 * m;
      r /= K;
    }
    long long ip = 0, im = 0;
    double c = 1.0;
    bool inner = true;
    long long jflat = 0;
    for (int a = 0; a < D; ++a) {
      const int kp = ((k[a] % nf) + nf) % nf;
      const int km = ((-k[a] % nf) + nf) % nf;
      ip = ip * nf + kp;
      im = im * nf + km;
      c *= corr[k[a] + 2 * m];
      inner = inner && (k[a] >= -m && k[a] <= m);
      jflat = jflat * n1 + (k[a] + m);
    }
    const cplx<T> gp = G[ip], gm = G[im];
    const double gpx = gp.x, gpy = gp.y, gmx = gm.x, gmy = gm.y;
    w[idx] = make_double2(0.5 * c * (gpx + gmx), 0.5 * c * (gpy - gmy));
    if (inner) {
      const double dc = Dw[jflat] * c;
      b[jflat] = make_double2(0.5 * dc * (gpy + gmy), -0.5 * dc * (gpx - gmx));
    }
  }
}

// grid (L^d, complex FP64): w_k at k mod L for k in J_{2m}, zero elsewhere
template <int D>
__global__ void place_w_kernel(const double2* __restrict__ w, int m, int L, double2* __restrict__ grid) {
  const int K = 4 * m + 1;
  long long total = L;
  if (D > 1) total *= L;
  if (D > 2) total *= L;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    long long r = idx;
    long long src = 0;
    bool ok = true;
    int g[3];
    for (int a = D - 1; a >= 0; --a) {
      g[a] = (int)(r % L);
      r /= L;
    }
    for (int a = 0; a < D; ++a) {
      int k;
      if (g[a] <= 2 * m) k = g[a];
      else if (g[a] >= L - 2 * m) k = g[a] - L;
      else { ok = false; k = 0; }
      src = src * K + (k + 2 * m);
    }
    grid[idx] = ok ? w[src] : make_double2(0.0, 0.0);
  }
}

template <typename T>
__global__ void extract_what_kernel(const double2* __restrict__ grid, long long n, double scale, T* __restrict__ what) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    what[i] = (T)(grid[i].x * scale);
}

// D_j = sqrt(h^d khat(h |j|)) on J_m (eq. 117), row-major, FP64.
// SE: khat = c exp(-b xi^2); Matern: khat = c (a + b xi^2)^(-e).
__global__ void spectral_weights_kernel(double* __restrict__ Dw, int m, int d, double h, int matern, double c,
                                        double a, double b, double e) {
  const int n1 = 2 * m + 1;
  long long total = n1;
  for (int i = 1; i < d; ++i) total *= n1;
  const double hd = d == 1 ? h : (d == 2 ? h * h : h * h * h);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    long long r = idx;
    double j2 = 0.0;
    for (int i = 0; i < d; ++i) {
      const double j = (double)(r % n1) - m;
      r /= n1;
      j2 += j * j;
    }
    const double xi2 = h * h * j2;
    const double kh = matern ? c * pow(a + b * xi2, -e) : c * exp(-b * xi2);
    Dw[idx] = sqrt(hd * kh);
  }
}

// ---------------------------------------------------------------- launchers
static int grid_for(long long n, int threads, int cap = 4096) {
  long long b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

// Opt the kernel in to `bytes` of dynamic shared memory (needed above the
// 48 KB default; static shared memory counts against that default too).
template <typename K>
static cudaError_t allow_smem(K kern, size_t bytes) {
  if (bytes <= 32 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int D, typename TC, typename TR>
static cudaError_t count_d(const void* x, int soa, long long N, const SortGeom& sg, unsigned int* counts, int* flag,
                           cudaStream_t s) {
  const size_t sm = sg.ntiles <= kSmemBins ? sg.ntiles * sizeof(unsigned int) : 0;
  auto k = bin_count_kernel<D, TC, TR>;
  cudaError_t e = allow_smem(k, sm);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = grid_for(N, kSortThreads, nsm * 8);
  k<<<blocks, kSortThreads, sm, s>>>(reinterpret_cast<const TC*>(x), soa, N, sg, counts, flag);
  return cudaGetLastError();
}

cudaError_t launch_bin_count(const void* x, int coord_f64, int rec_f64, int soa, long long N, const SortGeom& sg,
                             unsigned int* counts, int* range_flag, cudaStream_t s) {
  if (N == 0) return cudaSuccess;
  // the tile map uses the same arithmetic (record precision) as the scatter
#define EFGP_CNT(DD)                                                                                        \
  if (sg.d == DD) {                                                                                         \
    if (coord_f64) return rec_f64 ? count_d<DD, double, double>(x, soa, N, sg, counts, range_flag, s)      \
                                  : count_d<DD, double, float>(x, soa, N, sg, counts, range_flag, s);      \
    return rec_f64 ? count_d<DD, float, double>(x, soa, N, sg, counts, range_flag, s)                      \
                   : count_d<DD, float, float>(x, soa, N, sg, counts, range_flag, s);                      \
  }
  EFGP_CNT(1) EFGP_CNT(2) EFGP_CNT(3)
#undef EFGP_CNT
  return cudaErrorInvalidValue;
}

cudaError_t launch_scan_tiles(const unsigned int* counts, int ntiles, long long* tile_off, long long* cursor,
                              cudaStream_t s) {
  scan_tiles_kernel<<<1, 1024, 0, s>>>(counts, ntiles, tile_off, cursor);
  return cudaGetLastError();
}

template <int D, typename TC, typename TV, typename TR>
static cudaError_t scatter_sorted(const void* x, const void* y, int soa, long long N, long long n_begin,
                                  const SortGeom& sg, long long* cursor, void* rec, int nsm, cudaStream_t s) {
  constexpr int PPT = (sizeof(TR) == 8 || D == 3) ? 8 : 16;
  constexpr int P = 256 * PPT;
  const size_t sm = sizeof(TR) * (size_t)(D + 1) * P + sizeof(long long) * sg.ntiles + sizeof(int) * P +
                    2 * sizeof(int) * sg.ntiles;
  auto k = bin_scatter_sorted_kernel<D, TC, TV, TR, PPT>;
  cudaError_t e = allow_smem(k, sm);
  if (e != cudaSuccess) {
    set_error("sorting scatter: shared-memory opt-in of " + std::to_string(sm) + " bytes failed");
    return e;
  }
  const int blocks = grid_for(N - n_begin, P, nsm * 4);
  k<<<blocks, 256, sm, s>>>(reinterpret_cast<const TC*>(x), reinterpret_cast<const TV*>(y), soa, N, n_begin, sg,
                            cursor, reinterpret_cast<TR*>(rec));
  e = cudaGetLastError();
  if (e != cudaSuccess)
    set_error("sorting scatter launch (" + std::to_string(blocks) + " blocks, " + std::to_string(sm) +
              " bytes): " + cudaGetErrorString(e));
  return e;
}

template <int D, typename TC, typename TV, typename TR>
static cudaError_t scatter_d(const void* x, const void* y, int soa, long long N, const SortGeom& sg, long long* cursor,
                             void* rec, int* err, cudaStream_t s) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (sg.ntiles <= kSortedScatterMaxTiles) {
    if constexpr (std::is_same<TC, float>::value && std::is_same<TV, float>::value &&
                  std::is_same<TR, float>::value) {
      const bool aligned = (reinterpret_cast<uintptr_t>(x) % 16 == 0) && (reinterpret_cast<uintptr_t>(y) % 16 == 0);
      const size_t smb = scatter_big_smem(D, sg.ntiles);
      const long long nbig = N / kBigScatterChunk;
      if (!soa && aligned && sg.ntiles <= kBigScatterMaxTiles && smb <= 226 * 1024 && nbig > 0) {
        auto k = bin_scatter_big_kernel<D>;
        cudaError_t e = allow_smem(k, smb);
        if (e != cudaSuccess) {
          set_error("bulk-copy scatter: shared-memory opt-in of " + std::to_string(smb) + " bytes failed: " +
                    cudaGetErrorString(e));
          return e;
        }
        const int blocks = (int)std::min<long long>(nbig, nsm);
        k<<<blocks, kTmaScatterThreads, smb, s>>>(reinterpret_cast<const float*>(x), reinterpret_cast<const float*>(y),
                                                  nbig, sg, cursor, reinterpret_cast<float*>(rec), err);
        e = cudaGetLastError();
        if (e != cudaSuccess) {
          set_error("bulk-copy scatter launch (" + std::to_string(blocks) + " blocks, " + std::to_string(smb) +
                    " bytes): " + cudaGetErrorString(e));
          return e;
        }
        const long long done = nbig * kBigScatterChunk;
        if (done < N) return scatter_sorted<D, TC, TV, TR>(x, y, soa, N, done, sg, cursor, rec, nsm, s);
        return cudaSuccess;
      }
      const size_t sm = scatter_tma_smem(D, sg.ntiles);
      const long long nfull = N / kTmaScatterChunk;
      if (!soa && aligned && sm <= 226 * 1024 && nfull > 0) {
        auto k = bin_scatter_tma_kernel<D>;
        cudaError_t e = allow_smem(k, sm);
        if (e != cudaSuccess) {
          set_error("bulk-copy scatter: shared-memory opt-in of " + std::to_string(sm) + " bytes failed: " +
                    cudaGetErrorString(e));
          return e;
        }
        const int blocks = (int)std::min<long long>(nfull, nsm);
        k<<<blocks, kTmaScatterThreads, sm, s>>>(reinterpret_cast<const float*>(x), reinterpret_cast<const float*>(y),
                                                 nfull, N, sg, cursor, reinterpret_cast<float*>(rec), err);
        e = cudaGetLastError();
        if (e != cudaSuccess) {
          set_error("bulk-copy scatter launch (" + std::to_string(blocks) + " blocks, " + std::to_string(sm) +
                    " bytes): " + cudaGetErrorString(e));
          return e;
        }
        const long long done = nfull * kTmaScatterChunk;
        if (done < N) return scatter_sorted<D, TC, TV, TR>(x, y, soa, N, done, sg, cursor, rec, nsm, s);
        return cudaSuccess;
      }
    }
    return scatter_sorted<D, TC, TV, TR>(x, y, soa, N, 0, sg, cursor, rec, nsm, s);
  }
  const size_t sm = sg.ntiles <= kSmemBins ? sg.ntiles * (sizeof(long long) + sizeof(unsigned int)) : 0;
  auto k = bin_scatter_kernel<D, TC, TV, TR>;
  cudaError_t e = allow_smem(k, sm);
  if (e != cudaSuccess) return e;
  const int blocks = grid_for(N, kSortThreads * kScatterPPT, nsm * 8);
  k<<<blocks, kSortThreads, sm, s>>>(reinterpret_cast<const TC*>(x), reinterpret_cast<const TV*>(y), soa, N, sg, cursor,
                                     reinterpret_cast<TR*>(rec));
  return cudaGetLastError();
}

cudaError_t launch_bin_scatter(const void* x, int coord_f64, const void* y, int value_f64, int soa, long long N,
                               const SortGeom& sg, int rec_f64, long long* cursor, void* rec, int* err,
                               cudaStream_t s) {
  if (N == 0) return cudaSuccess;
  const SortGeom& g = sg;
#define EFGP_SC(DD, TC, TV)                                                                  \
  return rec_f64 ? scatter_d<DD, TC, TV, double>(x, y, soa, N, g, cursor, rec, err, s)      \
                 : scatter_d<DD, TC, TV, float>(x, y, soa, N, g, cursor, rec, err, s);
#define EFGP_SCD(DD)                                                \
  if (sg.d == DD) {                                                 \
    if (coord_f64 && value_f64) { EFGP_SC(DD, double, double) }     \
    if (coord_f64 && !value_f64) { EFGP_SC(DD, double, float) }     \
    if (!coord_f64 && value_f64) { EFGP_SC(DD, float, double) }     \
    EFGP_SC(DD, float, float)                                       \
  }
  EFGP_SCD(1) EFGP_SCD(2) EFGP_SCD(3)
#undef EFGP_SCD
#undef EFGP_SC
  return cudaErrorInvalidValue;
}

template <int D, int W, typename TR>
static cudaError_t spread_dw(const void* rec, long long N, const SortGeom& sg, const long long* tile_off,
                             const void* coef, double2* E, int* err, cudaStream_t s) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  constexpr bool use_tma = std::is_same<TR, float>::value && (D == 1 || (D == 2 && W <= 6));
  if constexpr (use_tma) {
    const size_t smp = spread_pair_smem(D, W);
    if (sg.TB == RegTile<(D == 1 ? 1 : 2)>::TB && smp <= 110 * 1024 && sg.rstride % 4 == 0 &&
        reinterpret_cast<uintptr_t>(rec) % 16 == 0) {
      auto k = spread_pair_kernel<(D == 1 ? 1 : 2), W>;
      cudaError_t e = allow_smem(k, smp);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
      if (e != cudaSuccess) return e;
      // two resident blocks per SM, about four waves of equal segments
      long long nseg = (long long)nsm * 2 * 4;
      long long seg = (N + nseg - 1) / nseg;
      if (seg < kPairBatch) seg = kPairBatch;
      nseg = (N + seg - 1) / seg;
      k<<<(unsigned)nseg, kPairThreads, smp, s>>>(reinterpret_cast<const float*>(rec), N, sg.rstride, sg, tile_off,
                                                  seg, *reinterpret_cast<const EsCoef<float>*>(coef), E, err);
      return cudaGetLastError();
    }
  }
  constexpr bool use_reg = std::is_same<TR, float>::value && (D == 1 || (D == 2 && W <= 7));
  if constexpr (use_reg) {
    if (sg.TB == RegTile<(D == 1 ? 1 : 2)>::TB) {
      const size_t sm = spread_reg_smem(D, W);
      auto k = spread_reg_kernel<(D == 1 ? 1 : 2), W>;
      cudaError_t e = allow_smem(k, sm);
      if (e != cudaSuccess) return e;
      // equal-size segments, about four resident waves
      long long nseg = (long long)nsm * 2 * 4;
      long long seg = (N + nseg - 1) / nseg;
      if (seg < 2048) seg = 2048;
      nseg = (N + seg - 1) / seg;
      k<<<(unsigned)nseg, kRegThreads, sm, s>>>(reinterpret_cast<const float*>(rec), N, sg, tile_off, seg,
                                                *reinterpret_cast<const EsCoef<float>*>(coef), E);
      return cudaGetLastError();
    }
  }
  const int S = sg.TB + W - 1;
  size_t cells = S;
  if (D > 1) cells *= S;
  if (D > 2) cells *= S;
  const size_t sm = 2 * cells * sizeof(TR);
  auto k = spread_kernel<D, W, TR>;
  cudaError_t e = allow_smem(k, sm);
  if (e != cudaSuccess) return e;
  // equal-size segments: enough blocks for several waves, each visiting
  // few tiles
  long long nseg = (long long)nsm * 8;
  long long seg = (N + nseg - 1) / nseg;
  if (seg < 1024) seg = 1024;
  nseg = (N + seg - 1) / seg;
  k<<<(unsigned)nseg, 256, sm, s>>>(reinterpret_cast<const TR*>(rec), N, sg, tile_off, seg,
                                    *reinterpret_cast<const EsCoef<TR>*>(coef), E);
  return cudaGetLastError();
}

template <int D, typename TR>
static cudaError_t spread_d(const void* rec, long long N, const SortGeom& sg, const long long* tile_off,
                            const void* coef, double2* E, int* err, cudaStream_t s) {
  switch (sg.W) {
    case 3: return spread_dw<D, 3, TR>(rec, N, sg, tile_off, coef, E, err, s);
    case 4: return spread_dw<D, 4, TR>(rec, N, sg, tile_off, coef, E, err, s);
    case 5: return spread_dw<D, 5, TR>(rec, N, sg, tile_off, coef, E, err, s);
    case 6: return spread_dw<D, 6, TR>(rec, N, sg, tile_off, coef, E, err, s);
    case 7: return spread_dw<D, 7, TR>(rec, N, sg, tile_off, coef, E, err, s);
    case 8: return spread_dw<D, 8, TR>(rec, N, sg, tile_off, coef, E, err, s);
    case 10: return spread_dw<D, 10, TR>(rec, N, sg, tile_off, coef, E, err, s);
    case 12: return spread_dw<D, 12, TR>(rec, N, sg, tile_off, coef, E, err, s);
    case 14: return spread_dw<D, 14, TR>(rec, N, sg, tile_off, coef, E, err, s);
    case 16: return spread_dw<D, 16, TR>(rec, N, sg, tile_off, coef, E, err, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_spread(const void* rec, int rec_f64, long long N, const SortGeom& sg, const long long* tile_off,
                          const void* coef, double2* E, int* err, cudaStream_t s) {
  if (N == 0) return cudaSuccess;
  if (sg.d == 1) return rec_f64 ? spread_d<1, double>(rec, N, sg, tile_off, coef, E, err, s)
                                : spread_d<1, float>(rec, N, sg, tile_off, coef, E, err, s);
  if (sg.d == 2) return rec_f64 ? spread_d<2, double>(rec, N, sg, tile_off, coef, E, err, s)
                                : spread_d<2, float>(rec, N, sg, tile_off, coef, E, err, s);
  if (sg.d == 3) return rec_f64 ? spread_d<3, double>(rec, N, sg, tile_off, coef, E, err, s)
                                : spread_d<3, float>(rec, N, sg, tile_off, coef, E, err, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_spectral_weights(double* Dw, int m, int d, double h, const efgp_kernel& k, cudaStream_t s) {
  const double pi = 3.14159265358979323846;
  const double var = k.variance > 0 ? k.variance : 1.0;
  const double ell = k.lengthscale;
  double c, a = 0.0, b, e = 0.0;
  int matern = k.family == EFGP_KERNEL_MATERN;
  if (!matern) {
    c = var * std::pow(2.0 * pi * ell * ell, 0.5 * d);
    b = 2.0 * pi * pi * ell * ell;
  } else {
    const double nu = k.nu;
    c = var * std::pow(2.0, d) * std::pow(pi, 0.5 * d) * std::tgamma(nu + 0.5 * d) * std::pow(2.0 * nu, nu) /
        (std::tgamma(nu) * std::pow(ell, 2.0 * nu));
    a = 2.0 * nu / (ell * ell);
    b = 4.0 * pi * pi;
    e = nu + 0.5 * d;
  }
  long long total = 2 * m + 1;
  for (int i = 1; i < d; ++i) total *= 2 * m + 1;
  spectral_weights_kernel<<<grid_for(total, 256), 256, 0, s>>>(Dw, m, d, h, matern, c, a, b, e);
  return cudaGetLastError();
}

cudaError_t launch_fold(const double2* E, int nEx, int off, int nf, int d, void* P, int p_f64, cudaStream_t s) {
  long long total = nf;
  for (int a = 1; a < d; ++a) total *= nf;
  const int blocks = grid_for(total, 256);
#define EFGP_FOLD(DD)                                                                                            \
  if (d == DD) {                                                                                                 \
    if (p_f64) fold_kernel<DD, double><<<blocks, 256, 0, s>>>(E, nEx, off, nf, reinterpret_cast<double2*>(P)); \
    else fold_kernel<DD, float><<<blocks, 256, 0, s>>>(E, nEx, off, nf, reinterpret_cast<float2*>(P));         \
    return cudaGetLastError();                                                                                   \
  }
  EFGP_FOLD(1) EFGP_FOLD(2) EFGP_FOLD(3)
#undef EFGP_FOLD
  return cudaErrorInvalidValue;
}

cudaError_t launch_deconv_split(const void* Phat, int p_f64, int nf, int d, int m, const double* corr1,
                                const double* Dw, double2* w, double2* b, cudaStream_t s) {
  long long total = 4 * m + 1;
  for (int a = 1; a < d; ++a) total *= 4 * m + 1;
  const int blocks = grid_for(total, 256);
#define EFGP_DC(DD)                                                                                          \
  if (d == DD) {                                                                                             \
    if (p_f64)                                                                                               \
      deconv_split_kernel<DD, double><<<blocks, 256, 0, s>>>(reinterpret_cast<const double2*>(Phat), nf, m, \
                                                             corr1, Dw, w, b);                               \
    else                                                                                                     \
      deconv_split_kernel<DD, float><<<blocks, 256, 0, s>>>(reinterpret_cast<const float2*>(Phat), nf, m,   \
                                                            corr1, Dw, w, b);                                \
    return cudaGetLastError();                                                                               \
  }
  EFGP_DC(1) EFGP_DC(2) EFGP_DC(3)
#undef EFGP_DC
  return cudaErrorInvalidValue;
}

cudaError_t launch_place_w(const double2* w, int m, int d, int L, double2* grid, cudaStream_t s) {
  long long total = L;
  for (int a = 1; a < d; ++a) total *= L;
  const int blocks = grid_for(total, 256);
  if (d == 1) place_w_kernel<1><<<blocks, 256, 0, s>>>(w, m, L, grid);
  else if (d == 2) place_w_kernel<2><<<blocks, 256, 0, s>>>(w, m, L, grid);
  else place_w_kernel<3><<<blocks, 256, 0, s>>>(w, m, L, grid);
  return cudaGetLastError();
}

cudaError_t launch_extract_what(const double2* grid, long long n, double scale, void* what, int what_f64,
                                cudaStream_t s) {
  const int blocks = grid_for(n, 256);
  if (what_f64) extract_what_kernel<double><<<blocks, 256, 0, s>>>(grid, n, scale, reinterpret_cast<double*>(what));
  else extract_what_kernel<float><<<blocks, 256, 0, s>>>(grid, n, scale, reinterpret_cast<float*>(what));
  return cudaGetLastError();
}

}  // namespace efgp
