// Fused, chunked set-up for 2D points in FP32 (Algorithm steps 2-3): the
// points are read from HBM twice in all (once to count, once to sort and
// spread) instead of four times, and the result is bitwise reproducible.
//
// 1. fused_count_kernel: the points are cut into chunks of G x S points (G =
//    blocks of the persistent kernel, one per SM; S = one block's share of a
//    chunk); every share gets its own histogram of spread tiles.
// 2. fused_scan_kernel: per chunk, the histograms become output offsets: the
//    chunk is ordered by tile, then by share, then by position in the share.
// 3. setup_fused_kernel (one cooperative launch, every block resident) loops
//    over the chunks.  Scatter: every block sorts its share of chunk k by tile
//    in shared memory (a stable counting sort) and writes it into chunk
//    buffer k mod 2, which is small enough to stay in L2.  Grid barrier.
//    Spread: every block takes an equal segment of that buffer and spreads it
//    with register-tiled accumulation (thread per fine-grid cell, W x W
//    footprint in registers); at the end of each tile visit the FP32 tile is
//    written to a slot of its own (no atomics).  After the next barrier the
//    owner block of each tile adds that chunk's slots for the tile, in block
//    order, into an FP64 halo'd tile with a compensated (Neumaier) sum.
// 4. fused_fold_kernel: the halo'd FP64 tiles are summed, in a fixed order,
//    onto the periodic fine grid.
//
// Every sum is taken in an order fixed by the input alone (counting sorts
// rank equal keys by position, reductions run in block order), so reruns
// give bitwise-identical w and b.  Waits (bulk copies, grid barriers) are
// bounded; a block that gives up records an error and every block leaves.
#include <cuda_runtime.h>

#include <cstdint>

#include "binning.cuh"
#include "grid_sync.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace efgp {

constexpr int kFThreads = 512;
constexpr int kFWarps = kFThreads / 32;
constexpr int kFSub = 4096;                 // points per scatter sub-chunk (8 per thread)
constexpr int kFSubPerWarp = kFSub / kFWarps;
constexpr int kFBatch = 4096;               // points per spread batch
constexpr int kFBatchPerWarp = kFBatch / kFWarps;
constexpr int kFSlot = kFBatch + 8;         // floats per staged record array
constexpr int kFTB = 16;                    // tile edge (2D)
constexpr int kFCells = kFTB * kFTB;        // cells of a tile (two threads each)

static_assert(kFSub % (32 * kFWarps) == 0 && kFBatch % (32 * kFWarps) == 0, "warp-strided sorts");

// ---------------------------------------------------------------- count
// Block per share (chunk k, block c): tile histogram of points
// [k*chunk + c*share, +share) clipped to N, written to cnt[(k*G + c)*T ..].
__global__ void __launch_bounds__(kFThreads) fused_count_kernel(const float* __restrict__ x, long long N, SortGeom sg,
                                                                long long share, long long chunk, int G,
                                                                unsigned int* __restrict__ cnt, int* range_flag,
                                                                int add_totals) {
  extern __shared__ unsigned int hist[];
  const int T = sg.ntiles;
  const long long sh = blockIdx.x;
  const long long k = sh / G, c = sh - k * G;
  const long long p0 = k * chunk + c * share;
  const long long p1 = p0 + share < N ? p0 + share : N;
  for (int i = threadIdx.x; i < T; i += kFThreads) hist[i] = 0u;
  __syncthreads();
  bool bad = false;
  if (p0 < p1) {
    // two points per 16-byte load (p0 is a multiple of the share, hence even)
    const long long npair = (p1 - p0) >> 1;
    const float4* x4 = reinterpret_cast<const float4*>(x + 2 * p0);
    constexpr int U = 4;
    for (long long i0 = threadIdx.x; i0 < npair; i0 += U * kFThreads) {
      float4 v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const long long i = i0 + (long long)u * kFThreads;
        v[u] = i < npair ? __ldcs(x4 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const long long i = i0 + (long long)u * kFThreads;
        if (i >= npair) continue;
        float q[3];
        const float a[2] = {v[u].x, v[u].y}, b[2] = {v[u].z, v[u].w};
        atomicAdd(&hist[tile_of_coords<2, float, float>(a, sg, q, bad)], 1u);
        atomicAdd(&hist[tile_of_coords<2, float, float>(b, sg, q, bad)], 1u);
      }
    }
    if (((p1 - p0) & 1) && threadIdx.x == 0) {
      float q[3];
      const float a[2] = {x[2 * (p1 - 1)], x[2 * (p1 - 1) + 1]};
      atomicAdd(&hist[tile_of_coords<2, float, float>(a, sg, q, bad)], 1u);
    }
  }
  if (bad) atomicOr(range_flag, 1);
  __syncthreads();
  if (add_totals) {
    // tile totals only (the three-pass set-up): integer sums, any order
    for (int i = threadIdx.x; i < T; i += kFThreads)
      if (hist[i]) atomicAdd(&cnt[i], hist[i]);
    return;
  }
  unsigned int* out = cnt + sh * T;
  for (int i = threadIdx.x; i < T; i += kFThreads) out[i] = hist[i];
}

// ---------------------------------------------------------------- scan
// Block per chunk: cnt[k][c][t] becomes the chunk position of share c's first
// point of tile t (tile-major, then share-major); toff[k][t] = first position
// of tile t in the chunk, toff[k][T] = points in the chunk.
constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kScanThreads) fused_scan_kernel(unsigned int* __restrict__ cnt, int G, int T,
                                                                  unsigned int* __restrict__ toff) {
  __shared__ unsigned int tot[kFusedMaxTiles];
  __shared__ unsigned int wsum[kScanThreads / 32];
  unsigned int* base = cnt + (long long)blockIdx.x * G * T;
  for (int t = threadIdx.x; t < T; t += kScanThreads) {
    unsigned int run = 0u;
    for (int c = 0; c < G; ++c) {
      const unsigned int v = base[(long long)c * T + t];
      base[(long long)c * T + t] = run;
      run += v;
    }
    tot[t] = run;
  }
  __syncthreads();
  // exclusive scan of tot over the tiles (T <= kScanThreads: one per thread)
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const unsigned int v = t < T ? tot[t] : 0u;
  unsigned int xs = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned int y = __shfl_up_sync(0xffffffffu, xs, o);
    if (lane >= o) xs += y;
  }
  if (lane == 31) wsum[wid] = xs;
  __syncthreads();
  if (wid == 0) {
    unsigned int w = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    wsum[lane] = w;
  }
  __syncthreads();
  const unsigned int excl = (wid > 0 ? wsum[wid - 1] : 0u) + xs - v;
  unsigned int* to = toff + (long long)blockIdx.x * (T + 1);
  if (t < T) {
    to[t] = excl;
    tot[t] = excl;
  }
  if (t == T - 1) to[T] = excl + v;
  __syncthreads();
  for (int tt = threadIdx.x; tt < T; tt += kScanThreads) {
    const unsigned int b = tot[tt];
    for (int c = 0; c < G; ++c) base[(long long)c * T + tt] += b;
  }
}

// ---------------------------------------------------------------- persistent kernel
// Shared memory, scatter view: staging 2 x (x pairs, y) of a sub-chunk, the
// sorted sub-chunk (q0, q1, y, tile), per-warp tile counts, cursors.
__host__ __device__ constexpr int fused_tiles_pad(int T) { return (T + 1) & ~1; }

__host__ __device__ inline size_t fused_scatter_smem(int T) {
  return sizeof(float) * (6 * (size_t)kFSub + 3 * (size_t)kFSub) + sizeof(unsigned short) * (size_t)kFSub +
         sizeof(unsigned short) * (size_t)kFWarps * fused_tiles_pad(T) + sizeof(int) * 3 * (size_t)T;
}

// Scatter of block c's share of chunk k into buffer k mod 2.  Positions: the
// share's first point of tile t goes to off[k][c][t]; inside a share points
// keep their input order within a tile (ranks from per-warp counts of the
// earlier points: warp w handles sub-chunk points [w*256, (w+1)*256) in
// order).  Returns false if a bounded wait for a bulk copy ran out.
__device__ bool fused_scatter(const FusedArgs& A, int k, unsigned char* smraw, uint64_t* sbar, uint32_t (&sph)[2],
                              int* err) {
  const int T = A.sg.ntiles, Tp = fused_tiles_pad(T), G = gridDim.x;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  float* stage = reinterpret_cast<float*>(smraw);                       // 2 x 3 x kFSub
  float* sq = stage + 6 * kFSub;                                         // 3 x kFSub
  unsigned short* stile = reinterpret_cast<unsigned short*>(sq + 3 * kFSub);   // kFSub
  unsigned short* whist = stile + kFSub;                                 // kFWarps x Tp
  int* cur = reinterpret_cast<int*>(whist + kFWarps * Tp);               // T
  int* lstart = cur + T;                                                 // T
  int* tcnt = lstart + T;                                                // T
  __shared__ int wtot[kFWarps];
  __shared__ int abort_s;
  const long long p0 = (long long)k * A.chunk + (long long)blockIdx.x * A.share;
  const long long p1 = p0 + A.share < A.N ? p0 + A.share : A.N;
  const unsigned int* offp = A.off + ((long long)k * G + blockIdx.x) * T;
  for (int t = tid; t < T; t += kFThreads) cur[t] = (int)offp[t];
  for (int i = tid; i < kFWarps * Tp / 2; i += kFThreads) reinterpret_cast<unsigned int*>(whist)[i] = 0u;
  if (tid == 0) abort_s = 0;
  __syncthreads();
  if (p0 >= p1) return true;
  const int nsub = (int)((p1 - p0 + kFSub - 1) / kFSub);
  float* Bk = A.B[k & 1];
  const long long bs = A.bstride;
  auto full = [&](int j) { return p0 + (long long)(j + 1) * kFSub <= p1; };
  auto issue = [&](int j, int b) {   // thread 0
    const long long q0 = p0 + (long long)j * kFSub;
    float* dst = stage + b * 3 * kFSub;
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&sbar[b], 12u * kFSub);
    bulk_g2s(dst, A.x + 2 * q0, 8u * kFSub, &sbar[b]);
    bulk_g2s(dst + 2 * kFSub, A.y + q0, 4u * kFSub, &sbar[b]);
  };
  if (tid == 0 && full(0)) issue(0, 0);
  int pending = -1;   // buffer of a copy issued and not yet waited for
  if (full(0)) pending = 0;
  for (int j = 0; j < nsub; ++j) {
    const int b = j & 1;
    float* sx = stage + b * 3 * kFSub;
    const long long q0 = p0 + (long long)j * kFSub;
    const int n = (int)(p1 - q0 < kFSub ? p1 - q0 : kFSub);
    const bool next_full = j + 1 < nsub && full(j + 1);
    if (tid == 0 && next_full) issue(j + 1, b ^ 1);
    if (n == kFSub) {
      if (!mbar_wait_bounded(&sbar[b], sph[b], err)) abort_s = 1;
      sph[b] ^= 1u;
    } else {
      // the partial last sub-chunk of the data: plain loads
      for (int i = tid; i < n; i += kFThreads) {
        sx[2 * i] = A.x[2 * (q0 + i)];
        sx[2 * i + 1] = A.x[2 * (q0 + i) + 1];
        sx[2 * kFSub + i] = A.y[q0 + i];
      }
    }
    pending = next_full ? (b ^ 1) : -1;
    __syncthreads();
    if (abort_s) break;
    // pass 1: tile and stable rank of each point among its warp's earlier points
    int tt[kFSubPerWarp / 32];
    unsigned short rk[kFSubPerWarp / 32];
    float qa[kFSubPerWarp / 32], qb[kFSubPerWarp / 32];
#pragma unroll
    for (int it = 0; it < kFSubPerWarp / 32; ++it) {
      const int kk = wid * kFSubPerWarp + it * 32 + lane;
      const bool valid = kk < n;
      int t = 0;
      float q[3] = {0.f, 0.f, 0.f};
      if (valid) {
        bool bad = false;
        const float2 xv = reinterpret_cast<const float2*>(sx)[kk];
        const float xa[2] = {xv.x, xv.y};
        t = tile_of_coords<2, float, float>(xa, A.sg, q, bad);
      }
      const unsigned int key = valid ? (unsigned int)t : 0x10000u + lane;
      const unsigned int peers = __match_any_sync(0xffffffffu, key);
      const unsigned int below = peers & ((1u << lane) - 1u);
      unsigned short old = 0;
      if (valid) old = whist[wid * Tp + t];
      __syncwarp();
      if (valid && below == 0u) whist[wid * Tp + t] = (unsigned short)(old + __popc(peers));
      __syncwarp();
      tt[it] = valid ? t : -1;
      rk[it] = (unsigned short)(old + __popc(below));
      qa[it] = q[0];
      qb[it] = q[1];
    }
    __syncthreads();
    // pass 2: per tile, exclusive prefix over warps; tile counts; local starts
    int sum = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int t = 2 * tid + h;
      if (t < T) {
        int run = 0;
#pragma unroll
        for (int w = 0; w < kFWarps; ++w) {
          const int c = whist[w * Tp + t];
          whist[w * Tp + t] = (unsigned short)run;
          run += c;
        }
        tcnt[t] = run;
        sum += run;
      }
    }
    const int ex = block_excl_scan_n<kFThreads>(sum, wtot);
    if (2 * tid < T) lstart[2 * tid] = ex;
    if (2 * tid + 1 < T) lstart[2 * tid + 1] = ex + tcnt[2 * tid];
    __syncthreads();
    // pass 3: the sub-chunk sorted by tile in shared memory
#pragma unroll
    for (int it = 0; it < kFSubPerWarp / 32; ++it) {
      const int t = tt[it];
      if (t < 0) continue;
      const int kk = wid * kFSubPerWarp + it * 32 + lane;
      const int pos = lstart[t] + whist[wid * Tp + t] + rk[it];
      sq[pos] = qa[it];
      sq[kFSub + pos] = qb[it];
      sq[2 * kFSub + pos] = sx[2 * kFSub + kk];
      stile[pos] = (unsigned short)t;
    }
    __syncthreads();
    // write-out, tile run by tile run (consecutive threads, consecutive addresses)
    for (int i = tid; i < n; i += kFThreads) {
      const int t = stile[i];
      const long long g = (long long)cur[t] + (i - lstart[t]);
      __stcg(Bk + g, sq[i]);
      __stcg(Bk + bs + g, sq[kFSub + i]);
      __stcg(Bk + 2 * bs + g, sq[2 * kFSub + i]);
    }
    __syncthreads();
    for (int t = tid; t < T; t += kFThreads) cur[t] += tcnt[t];
    for (int i = tid; i < kFWarps * Tp / 2; i += kFThreads) reinterpret_cast<unsigned int*>(whist)[i] = 0u;
    __syncthreads();
  }
  // after an abandoned wait, let a copy already issued land before the
  // shared memory is reused or released
  if (abort_s && tid == 0 && pending >= 0) mbar_wait_bounded(&sbar[pending], sph[pending], nullptr);
  if (abort_s && pending >= 0) sph[pending] ^= 1u;
  fence_proxy_async_global();
  return abort_s == 0;
}

// Shared memory, spread view: staging 2 x (q0, q1, y) of a batch, the FP32
// tile, the batch's cell sort (index, per-point rank and cell, per-warp cell
// counts), cell counts and starts.
template <int W>
__host__ __device__ constexpr size_t fused_spread_smem() {
  return sizeof(float) * (6 * (size_t)kFSlot + 2 * (size_t)(kFTB + W - 1) * (kFTB + W - 1)) +
         sizeof(unsigned short) * 2 * (size_t)kFBatch + sizeof(unsigned char) * (size_t)kFBatch +
         sizeof(unsigned short) * (size_t)kFWarps * kFCells + sizeof(int) * 2 * (size_t)kFCells;
}

// Spread of block c's equal segment of chunk k's sorted buffer.  The segment
// is walked as batches (tile, first point, count) of at most kFBatch points,
// each copied into shared memory while the previous one is processed.  A
// batch is sorted by cell (stable: per-warp ranks, warps in order); thread
// pairs own the tile's 256 cells and add their cell's points (even and odd
// positions) into W x W float2 footprints in registers.  At the end of a tile
// visit the footprints are added into the shared tile in a fixed phase order
// and the tile is written to slot (c + tile) of the chunk's slot array.
template <int W>
__device__ bool fused_spread(const FusedArgs& A, int k, const EsCoef<float>& cf, unsigned char* smraw,
                             uint64_t* pbar, uint32_t (&pph)[2], int* err) {
  constexpr int TB = kFTB, S = TB + W - 1, CELLS = S * S, FP = W * W, NA = 3;
  const int T = A.sg.ntiles, G = gridDim.x;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int cell = tid & (kFCells - 1), half = tid >> 8;
  float* stg = reinterpret_cast<float*>(smraw);                                   // 2 x NA x kFSlot
  float* tile = stg + 2 * NA * kFSlot;                                             // 2 x CELLS
  unsigned short* idx = reinterpret_cast<unsigned short*>(tile + 2 * CELLS);      // kFBatch
  unsigned short* urank = idx + kFBatch;                                           // kFBatch
  unsigned char* ucell = reinterpret_cast<unsigned char*>(urank + kFBatch);        // kFBatch
  unsigned short* wh2 = reinterpret_cast<unsigned short*>(ucell + kFBatch);        // kFWarps x kFCells
  int* ccnt = reinterpret_cast<int*>(wh2 + kFWarps * kFCells);                     // kFCells
  int* cst = ccnt + kFCells;                                                       // kFCells
  __shared__ int wtot[kFWarps];
  __shared__ int it_tile[2], it_off[2], it_n[2];
  __shared__ long long it_p0[2];
  __shared__ int abort_s;
  const long long rest = A.N - (long long)k * A.chunk;
  const long long Ck = rest < A.chunk ? rest : A.chunk;
  const long long seg = (Ck + G - 1) / G;
  const long long s0 = (long long)blockIdx.x * seg;
  const long long s1 = s0 + seg < Ck ? s0 + seg : Ck;
  if (s0 >= s1) return true;
  const unsigned int* tof = A.toff + (long long)k * (T + 1);
  const float* rec = A.B[k & 1];
  const long long rs = A.bstride;
  float2* slot = A.slots[k & 1];

  auto next_item = [&](int& tt, long long& p0, int& n) -> bool {
    long long b = tof[tt + 1];
    if (b > s1) b = s1;
    p0 += n;
    if (p0 < b) {
      n = (int)(b - p0 < kFBatch ? b - p0 : kFBatch);
      return true;
    }
    for (++tt; tt < T; ++tt) {
      const long long ta = tof[tt];
      if (ta >= s1) return false;
      long long bb = tof[tt + 1];
      if (bb > s1) bb = s1;
      const long long a = ta > s0 ? ta : s0;
      if (a < bb) {
        p0 = a;
        n = (int)(bb - a < kFBatch ? bb - a : kFBatch);
        return true;
      }
    }
    return false;
  };
  auto issue = [&](int sl, long long p0, int n) {   // thread 0
    const long long pa = p0 & ~3ll;
    const long long pe = (p0 + n + 3) & ~3ll;
    const uint32_t bytes = (uint32_t)((pe - pa) * 4);
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&pbar[sl], bytes * NA);
    for (int a = 0; a < NA; ++a) bulk_g2s(stg + (sl * NA + a) * kFSlot, rec + a * rs + pa, bytes, &pbar[sl]);
    it_off[sl] = (int)(p0 - pa);
  };

  for (int i = tid; i < kFWarps * kFCells / 2; i += kFThreads) reinterpret_cast<unsigned int*>(wh2)[i] = 0u;
  if (tid == 0) {
    abort_s = 0;
    int lo = 0, hi = T - 1;   // largest tile with tof[t] <= s0
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if ((long long)tof[mid] <= s0) lo = mid; else hi = mid - 1;
    }
    int tt = lo;
    long long p0 = s0;
    int n = 0;
    bool ok;
    long long b = tof[tt + 1];
    if (b > s1) b = s1;
    if (p0 < b) {
      n = (int)(b - p0 < kFBatch ? b - p0 : kFBatch);
      ok = true;
    } else {
      ok = next_item(tt, p0, n);
    }
    it_tile[0] = ok ? tt : -1;
    it_p0[0] = p0;
    it_n[0] = n;
    if (ok) issue(0, p0, n);
  }
  __syncthreads();

  const int own0 = cell / TB, own1 = cell % TB;
  float2 acc[FP];
#pragma unroll
  for (int i = 0; i < FP; ++i) acc[i] = make_float2(0.f, 0.f);
  int abort_it = -1;
  for (int it = 0;; ++it) {
    const int b = it & 1;
    const int tt = it_tile[b];
    if (tt < 0) break;
    const int n = it_n[b];
    if (tid == 0) {
      int nt = tt;
      long long np0 = it_p0[b];
      int nn = n;
      const bool ok = next_item(nt, np0, nn);
      it_tile[b ^ 1] = ok ? nt : -1;
      it_p0[b ^ 1] = np0;
      it_n[b ^ 1] = nn;
      if (ok) issue(b ^ 1, np0, nn);
    }
    if (!mbar_wait_bounded(&pbar[b], pph[b], err)) abort_s = 1;
    pph[b] ^= 1u;
    __syncthreads();
    if (abort_s) {
      abort_it = it;
      break;
    }
    const int off = it_off[b];
    const float* sq0 = stg + (b * NA) * kFSlot + off;
    const float* sq1 = sq0 + kFSlot;
    const float* sy = sq0 + 2 * kFSlot;
    // cell sort, pass 1: per-warp stable ranks
#pragma unroll
    for (int r = 0; r < kFBatchPerWarp / 32; ++r) {
      const int kk = wid * kFBatchPerWarp + r * 32 + lane;
      const bool valid = kk < n;
      int c = 0;
      if (valid) {
        float q[2] = {sq0[kk], sq1[kk]}, f[2];
        c = reg_cell<2>(q, f);
      }
      const unsigned int key = valid ? (unsigned int)c : 0x100u + lane;
      const unsigned int peers = __match_any_sync(0xffffffffu, key);
      const unsigned int below = peers & ((1u << lane) - 1u);
      unsigned short old = 0;
      if (valid) old = wh2[wid * kFCells + c];
      __syncwarp();
      if (valid && below == 0u) wh2[wid * kFCells + c] = (unsigned short)(old + __popc(peers));
      __syncwarp();
      if (valid) {
        ucell[kk] = (unsigned char)c;
        urank[kk] = (unsigned short)(old + __popc(below));
      }
    }
    __syncthreads();
    // pass 2: per cell, prefix over warps, counts; starts by a block scan
    int mine = 0;
    if (tid < kFCells) {
      int run = 0;
#pragma unroll
      for (int w = 0; w < kFWarps; ++w) {
        const int v = wh2[w * kFCells + tid];
        wh2[w * kFCells + tid] = (unsigned short)run;
        run += v;
      }
      ccnt[tid] = run;
      mine = run;
    }
    const int st = block_excl_scan_n<kFThreads>(mine, wtot);
    if (tid < kFCells) cst[tid] = st;
    __syncthreads();
    // pass 3: batch indices in cell order
    for (int kk = tid; kk < n; kk += kFThreads) {
      const int c = ucell[kk];
      idx[cst[c] + wh2[(kk / kFBatchPerWarp) * kFCells + c] + urank[kk]] = (unsigned short)kk;
    }
    __syncthreads();
    for (int i = tid; i < kFWarps * kFCells / 2; i += kFThreads) reinterpret_cast<unsigned int*>(wh2)[i] = 0u;
    {
      const int c_n = ccnt[cell];
      const int c_s = cst[cell];
      auto add_point = [&](const float (&w0)[W], const float (&w1)[W], float yv) {
        const float2 c2 = make_float2(1.f, yv);
#pragma unroll
        for (int u = 0; u < W; ++u) {
          const float2 wa = __fmul2_rn(make_float2(w0[u], w0[u]), c2);
#pragma unroll
          for (int v = 0; v < W; ++v) acc[u * W + v] = __ffma2_rn(wa, make_float2(w1[v], w1[v]), acc[u * W + v]);
        }
      };
      int j = half;
      for (; j + 2 < c_n; j += 4) {
        const int k0 = idx[c_s + j], k1 = idx[c_s + j + 2];
        float a0[W], b0[W], a1[W], b1[W];
        es_weights_x2<W>(sq0[k0] - (float)own0, cf, a0);
        es_weights_x2<W>(sq1[k0] - (float)own1, cf, b0);
        es_weights_x2<W>(sq0[k1] - (float)own0, cf, a1);
        es_weights_x2<W>(sq1[k1] - (float)own1, cf, b1);
        add_point(a0, b0, sy[k0]);
        add_point(a1, b1, sy[k1]);
      }
      for (; j < c_n; j += 2) {
        const int k0 = idx[c_s + j];
        float a0[W], b0[W];
        es_weights_x2<W>(sq0[k0] - (float)own0, cf, a0);
        es_weights_x2<W>(sq1[k0] - (float)own1, cf, b0);
        add_point(a0, b0, sy[k0]);
      }
    }
    __syncthreads();
    if (it_tile[b ^ 1] != tt) {
      // end of the tile visit: registers -> shared tile (fixed order) -> slot
      for (int c = tid; c < 2 * CELLS; c += kFThreads) tile[c] = 0.f;
      __syncthreads();
      for (int h = 0; h < 2; ++h) {
#pragma unroll
        for (int i = 0; i < FP; ++i) {
          if (half == h) {
            const int cc = (own0 + i / W) * S + own1 + i % W;
            tile[2 * cc] += acc[i].x;
            tile[2 * cc + 1] += acc[i].y;
          }
          __syncthreads();
        }
      }
#pragma unroll
      for (int i = 0; i < FP; ++i) acc[i] = make_float2(0.f, 0.f);
      float2* dst = slot + ((long long)blockIdx.x + tt) * CELLS;
      for (int c = tid; c < CELLS; c += kFThreads) __stcg(dst + c, make_float2(tile[2 * c], tile[2 * c + 1]));
      __syncthreads();
    }
  }
  if (abort_s && tid == 0 && abort_it >= 0 && it_tile[(abort_it & 1) ^ 1] >= 0)
    mbar_wait_bounded(&pbar[(abort_it & 1) ^ 1], pph[(abort_it & 1) ^ 1], nullptr);
  return abort_s == 0;
}

__device__ __forceinline__ void neumaier_add(double& s, double& c, double v) {
  const double t = s + v;
  if (fabs(s) >= fabs(v)) c += (s - t) + v;
  else c += (v - t) + s;
  s = t;
}

// Owner reduction of chunk k: block b adds, for each tile t = b, b + G, ...,
// the slots of the segments that overlap the tile (segments c_lo..c_hi, in
// order) into the tile's FP64 accumulator.
template <int W>
__device__ void fused_reduce(const FusedArgs& A, int k) {
  constexpr int S = kFTB + W - 1, CELLS = S * S;
  const int T = A.sg.ntiles, G = gridDim.x;
  const long long rest = A.N - (long long)k * A.chunk;
  const long long Ck = rest < A.chunk ? rest : A.chunk;
  const long long seg = (Ck + G - 1) / G;
  const unsigned int* tof = A.toff + (long long)k * (T + 1);
  const float2* slot = A.slots[k & 1];
  for (int t = blockIdx.x; t < T; t += G) {
    const long long a = tof[t], b = tof[t + 1];
    if (a >= b) continue;
    const long long clo = a / seg, chi = (b - 1) / seg;
    for (int c = threadIdx.x; c < CELLS; c += kFThreads) {
      TileAcc e = A.Et[(long long)t * CELLS + c];
      for (long long sgi = clo; sgi <= chi; ++sgi) {
        const float2 v = __ldcg(slot + (sgi + t) * CELLS + c);
        neumaier_add(e.sx, e.cx, (double)v.x);
        neumaier_add(e.sy, e.cy, (double)v.y);
      }
      A.Et[(long long)t * CELLS + c] = e;
    }
  }
}

template <int W>
__global__ void __launch_bounds__(kFThreads, 1)
    setup_fused_kernel(FusedArgs A, EsCoef<float> cf, GridBarrier* gb, long long limit, int* err) {
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ __align__(8) uint64_t bars[4];   // scatter staging 0, 1; spread staging 2, 3
  if (threadIdx.x == 0) {
    for (int i = 0; i < 4; ++i) mbar_init(&bars[i], 1);
    fence_barrier_init();
  }
  __syncthreads();
  uint32_t sph[2] = {0u, 0u}, pph[2] = {0u, 0u};
  unsigned int gen = 0u;
  const unsigned int G = gridDim.x;
  bool ok = true;
  for (int k = 0; k < A.nchunks; ++k) {
    if (!fused_scatter(A, k, smraw, bars, sph, err)) {
      ok = false;
      if (threadIdx.x == 0) atomicOr(&gb->err, 2);
      break;
    }
    if (!grid_barrier(gb, G, gen, limit)) {
      ok = false;
      break;
    }
    fence_proxy_async_global();
    if (k > 0) fused_reduce<W>(A, k - 1);
    if (!fused_spread<W>(A, k, cf, smraw, bars + 2, pph, err)) {
      ok = false;
      if (threadIdx.x == 0) atomicOr(&gb->err, 2);
      break;
    }
  }
  if (ok && grid_barrier(gb, G, gen, limit)) fused_reduce<W>(A, A.nchunks - 1);
}

// Periodic fine grid from the halo'd FP64 tiles: P[p] = sum over extended
// cells e = p + off (mod nf), e < nEx, of every tile cell covering e, in tile
// order (deterministic).
template <int W>
__global__ void fused_fold_kernel(const TileAcc* __restrict__ Et, SortGeom sg, int nf, int off, float2* __restrict__ P) {
  constexpr int TB = kFTB, S = TB + W - 1, CELLS = S * S;
  const long long total = (long long)nf * nf;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int p0 = (int)(idx / nf), p1 = (int)(idx - (long long)p0 * nf);
    double sx = 0.0, sy = 0.0;
    for (int e0 = (p0 + off) % nf; e0 < sg.nEx; e0 += nf) {
      for (int e1 = (p1 + off) % nf; e1 < sg.nEx; e1 += nf) {
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          const int t0 = e0 / TB - a;
          if (t0 < 0 || t0 >= sg.nt[0]) continue;
          const int l0 = e0 - t0 * TB;
          if (l0 >= S) continue;
#pragma unroll
          for (int bb = 0; bb < 2; ++bb) {
            const int t1 = e1 / TB - bb;
            if (t1 < 0 || t1 >= sg.nt[1]) continue;
            const int l1 = e1 - t1 * TB;
            if (l1 >= S) continue;
            const TileAcc v = Et[(long long)(t0 * sg.nt[1] + t1) * CELLS + l0 * S + l1];
            sx += v.sx + v.cx;
            sy += v.sy + v.cy;
          }
        }
      }
    }
    P[idx] = make_float2((float)sx, (float)sy);
  }
}

// ---------------------------------------------------------------- launchers
template <int W>
static size_t smem_w(int T) {
  const size_t a = fused_scatter_smem(T), b = fused_spread_smem<W>();
  return a > b ? a : b;
}

size_t fused_smem_bytes(int ntiles, int W) {
  switch (W) {
    case 3: return smem_w<3>(ntiles);
    case 4: return smem_w<4>(ntiles);
    case 5: return smem_w<5>(ntiles);
    case 6: return smem_w<6>(ntiles);
  }
  return 0;
}

template <int W>
static int blocks_w(size_t smem) {
  int dev = 0, nsm = 0, coop = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop) return 0;
  if (cudaFuncSetAttribute(setup_fused_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, setup_fused_kernel<W>, kFThreads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per >= 1 ? nsm : 0;
}

int fused_blocks(int W, size_t smem) {
  switch (W) {
    case 3: return blocks_w<3>(smem);
    case 4: return blocks_w<4>(smem);
    case 5: return blocks_w<5>(smem);
    case 6: return blocks_w<6>(smem);
  }
  return 0;
}

cudaError_t launch_fused_count(const float* x, long long N, const SortGeom& sg, long long share, long long chunk,
                               int blocks, int nchunks, unsigned int* cnt, int* range_flag, cudaStream_t s) {
  const size_t sm = sizeof(unsigned int) * (size_t)sg.ntiles;
  const long long grid = (long long)nchunks * blocks;
  fused_count_kernel<<<(unsigned)grid, kFThreads, sm, s>>>(x, N, sg, share, chunk, blocks, cnt, range_flag, 0);
  return cudaGetLastError();
}

// Tile totals of all N points (2D, FP32 row-major, 16-byte aligned x) added
// into counts, by the share-per-block kernel above.
cudaError_t launch_tile_totals_2d(const float* x, long long N, const SortGeom& sg, unsigned int* counts,
                                  int* range_flag, cudaStream_t s) {
  const size_t sm = sizeof(unsigned int) * (size_t)sg.ntiles;
  const long long share = 8192;
  const long long grid = (N + share - 1) / share;
  fused_count_kernel<<<(unsigned)grid, kFThreads, sm, s>>>(x, N, sg, share, share, 1, counts, range_flag, 1);
  return cudaGetLastError();
}

cudaError_t launch_fused_scan(unsigned int* cnt, int blocks, int ntiles, int nchunks, unsigned int* toff,
                              cudaStream_t s) {
  fused_scan_kernel<<<(unsigned)nchunks, kScanThreads, 0, s>>>(cnt, blocks, ntiles, toff);
  return cudaGetLastError();
}

template <int W>
static cudaError_t launch_w(const FusedArgs& a, const void* coef, int blocks, size_t smem, GridBarrier* gb,
                            long long limit, int* err, cudaStream_t s) {
  auto kern = setup_fused_kernel<W>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)blocks, 1, 1);
  cfg.blockDim = dim3(kFThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const EsCoef<float> cf = *reinterpret_cast<const EsCoef<float>*>(coef);
  return cudaLaunchKernelEx(&cfg, kern, a, cf, gb, limit, err);
}

cudaError_t launch_setup_fused(const FusedArgs& a, const void* coef, int blocks, size_t smem, GridBarrier* gb,
                               long long limit, int* err, cudaStream_t s) {
  switch (a.sg.W) {
    case 3: return launch_w<3>(a, coef, blocks, smem, gb, limit, err, s);
    case 4: return launch_w<4>(a, coef, blocks, smem, gb, limit, err, s);
    case 5: return launch_w<5>(a, coef, blocks, smem, gb, limit, err, s);
    case 6: return launch_w<6>(a, coef, blocks, smem, gb, limit, err, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_fused_fold(const TileAcc* Et, const SortGeom& sg, int nf, int off, float2* P, cudaStream_t s) {
  const long long total = (long long)nf * nf;
  long long blocks = (total + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  switch (sg.W) {
    case 3: fused_fold_kernel<3><<<(unsigned)blocks, 256, 0, s>>>(Et, sg, nf, off, P); break;
    case 4: fused_fold_kernel<4><<<(unsigned)blocks, 256, 0, s>>>(Et, sg, nf, off, P); break;
    case 5: fused_fold_kernel<5><<<(unsigned)blocks, 256, 0, s>>>(Et, sg, nf, off, P); break;
    case 6: fused_fold_kernel<6><<<(unsigned)blocks, 256, 0, s>>>(Et, sg, nf, off, P); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace efgp
