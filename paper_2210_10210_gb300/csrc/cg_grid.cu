// Conjugate gradients (Algorithm 2, step 4) for one problem in one
// cooperative launch over the whole GPU.
//
// Every block of the grid is resident (cooperative launch), so the blocks can
// wait for one another: each pass of the Toeplitz product (Algorithm 1 steps
// 3-6; the first pass also forms p = r + beta p, the last one adds sigma^2 p
// and reduces p^H A p) deals its line blocks round-robin to the grid's blocks
// and ends at a grid barrier; the vector update (x += alpha p, r -= alpha A p,
// r^H r) ends at one more.  An iteration therefore costs (passes + 1) grid
// barriers instead of (passes + 1) kernel boundaries.
//
// The two inner products of an iteration are reduced per block; after the
// barrier every block reads all blocks' partial sums in block order, so all
// blocks hold bitwise-identical alpha, beta and convergence decisions and
// leave the loop together.
//
// Every barrier wait is bounded: a block that polls past the limit records an
// error for the host, and every block that sees the error leaves the loop at
// its next barrier, so the launch always ends (the host reports ETIMEOUT).
#include <cuda_runtime.h>

#include "kernels.h"
#include "grid_sync.cuh"
#include "line_fft.cuh"

namespace efgp {

// Sum of one double per block (written before the barrier that precedes the
// call), read by every block in block order: identical in every block.
__device__ __forceinline__ double grid_sum(const double* partials, int nblocks, double* red) {
  double v = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) v += __ldcg(partials + i);
  v = block_sum(v, red);
  __shared__ double out;
  if (threadIdx.x == 0) out = v;
  __syncthreads();
  const double r = out;
  __syncthreads();
  return r;
}

template <typename T>
__global__ void __launch_bounds__(kGridCgThreads) cg_grid_kernel(const PersistentProblem* __restrict__ probs,
                                                                  GridBarrier* gb, double* __restrict__ part,
                                                                  long long limit) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  const PersistentProblem& P = probs[0];
  const int tid = threadIdx.x, bid = blockIdx.x, G = gridDim.x;
  const long long M = P.M;
  unsigned int gen = 0u;
  double* part_a = part;        // p^H A p partials
  double* part_b = part + G;    // r^H r partials
  const long long e0 = (long long)bid * blockDim.x + tid;
  const long long es = (long long)G * blockDim.x;

  double s = 0.0;
  for (long long i = e0; i < M; i += es) {
    const double2 v = P.b[i];
    P.x[i] = make_double2(0.0, 0.0);
    P.r[i] = v;
    P.p[i] = v;
    s += v.x * v.x + v.y * v.y;
  }
  {
    const double bs = block_sum(s, red);
    if (tid == 0) part_b[bid] = bs;
  }
  int done = 0;
  if (!grid_barrier(gb, G, gen, limit)) done = 4;
  const double bnorm2 = done ? 0.0 : grid_sum(part_b, G, red);
  const double tol2 = P.rho * P.rho * bnorm2;
  double rr = bnorm2, beta = 0.0, alpha = 0.0, pAp = 0.0;
  if (!done) done = bnorm2 == 0.0 ? 1 : (P.max_iter <= 0 ? 2 : 0);
  long long it = 0;
  CgArgs cga{};
  cga.src = P.p;
  cga.r = P.r;
  cga.Dw = P.Dw;
  cga.dst = P.Ap;
  cga.sigma2 = P.sigma2;
  // first iteration: p = r already (beta = 0 gives p = r + 0 p as well)
  cga.update_p = 1;
  while (!done) {
    double dot = 0.0;
    for (int q = 0; q < P.npass && !done; ++q) {
      const LineGeom& g = P.pass[q];
      const long long nblk = (g.outer * g.inner + g.nb - 1) / g.nb;
      for (long long blk = bid; blk < nblk; blk += G) dot += run_pass<T>(P, q, blk, cga, beta, smem_raw);
      if (q + 1 == P.npass) {
        const double bs = block_sum(dot, red);
        if (tid == 0) part_a[bid] = bs;
      }
      if (!grid_barrier(gb, G, gen, limit)) done = 4;
    }
    if (done) break;
    pAp = grid_sum(part_a, G, red);
    if (!(pAp > 0.0) || !isfinite(pAp)) {
      done = 3;
      break;
    }
    alpha = rr / pAp;
    double s2 = 0.0;
    for (long long i = e0; i < M; i += es) {
      const double2 pv = __ldcg(P.p + i), av = __ldcg(P.Ap + i);
      double2 xv = P.x[i], rv = __ldcg(P.r + i);
      xv.x += alpha * pv.x;
      xv.y += alpha * pv.y;
      rv.x -= alpha * av.x;
      rv.y -= alpha * av.y;
      P.x[i] = xv;
      P.r[i] = rv;
      s2 += rv.x * rv.x + rv.y * rv.y;
    }
    {
      const double bs = block_sum(s2, red);
      if (tid == 0) part_b[bid] = bs;
    }
    if (!grid_barrier(gb, G, gen, limit)) {
      done = 4;
      break;
    }
    const double rr_new = grid_sum(part_b, G, red);
    ++it;
    beta = rr_new / rr;
    rr = rr_new;
    if (!isfinite(rr)) done = 3;
    else if (rr <= tol2) done = 1;
    else if (it >= P.max_iter) done = 2;
  }
  if (bid == 0 && tid == 0) {
    CgState* st = P.st;
    st->bnorm2 = bnorm2;
    st->rr = rr;
    st->rr_new = rr;
    st->tol2 = tol2;
    st->iter = it;
    st->max_iter = P.max_iter;
    st->alpha = alpha;
    st->beta = beta;
    st->pAp = pAp;
    st->done = done == 4 ? 0 : done;
  }
}

template <typename T>
static cudaError_t launch_t(const PersistentProblem* d_prob, GridBarrier* gb, double* part, int blocks, size_t smem,
                            long long limit, cudaStream_t s) {
  auto kern = cg_grid_kernel<T>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)blocks, 1, 1);
  cfg.blockDim = dim3(kGridCgThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, d_prob, gb, part, limit);
}

cudaError_t launch_cg_grid(const PersistentProblem* d_prob, GridBarrier* gb, double* part, int blocks, size_t smem,
                           int f64, long long limit, cudaStream_t s) {
  return f64 ? launch_t<double>(d_prob, gb, part, blocks, smem, limit, s)
             : launch_t<float>(d_prob, gb, part, blocks, smem, limit, s);
}

// Blocks of a cooperative launch with this shared memory: one per SM (the
// passes are latency-bound; more blocks only lengthen every barrier), or 0 if
// a block does not fit or the device cannot launch cooperatively.
int cg_grid_blocks(int f64, size_t smem) {
  int dev = 0, nsm = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop || nsm <= 0) return 0;
  int per = 0;
  cudaError_t e;
  if (f64) {
    cudaFuncSetAttribute(cg_grid_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, cg_grid_kernel<double>, kGridCgThreads, smem);
  } else {
    cudaFuncSetAttribute(cg_grid_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, cg_grid_kernel<float>, kGridCgThreads, smem);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per >= 1 ? nsm : 0;
}

}  // namespace efgp
