// Persistent conjugate gradients (Algorithm 2, step 4) on one thread-block
// cluster per problem.
//
// The whole CG loop runs in one launch.  Every pass of the Toeplitz product
// (Algorithm 1 steps 3-6, see fft.cu) is a phase whose line blocks are dealt
// round-robin to the cluster's blocks, separated by hardware cluster barriers
// (release/acquire at cluster scope, so the pass outputs the blocks leave in
// global memory are visible to the next phase).  The two inner products of an
// iteration are reduced per block and combined through distributed shared
// memory: every block reads all blocks' partial sums in the same order, so
// all blocks hold bitwise-identical alpha, beta and the convergence decision,
// and leave the loop together.  The loop is bounded by max_iter.
//
// Several problems can share a launch (one cluster each), which is how a
// batch of small problems is solved without a launch per iteration.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "kernels.h"
#include "line_fft.cuh"

namespace cg = cooperative_groups;

namespace efgp {

template <typename T>
__global__ void __launch_bounds__(kPersistentThreads) cg_cluster_kernel(const PersistentProblem* __restrict__ probs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  __shared__ double slots[2];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int CL = (int)cl.num_blocks();
  const PersistentProblem& P = probs[blockIdx.x / CL];
  const int tid = threadIdx.x;
  const long long M = P.M;
  int slot = 0;
  // sum of v over the cluster, identical in every thread of every block
  auto cluster_sum = [&](double v) -> double {
    const double bs = block_sum(v, red);
    if (tid == 0) slots[slot] = bs;
    cl.sync();
    double tot = 0.0;
    for (int q = 0; q < CL; ++q) tot += *cl.map_shared_rank(&slots[slot], q);
    slot ^= 1;
    return tot;
  };

  const long long e0 = (long long)rank * blockDim.x + tid;
  const long long es = (long long)CL * blockDim.x;
  double s = 0.0;
  for (long long i = e0; i < M; i += es) {
    const double2 v = P.b[i];
    P.x[i] = make_double2(0.0, 0.0);
    P.r[i] = v;
    P.p[i] = v;
    s += v.x * v.x + v.y * v.y;
  }
  const double bnorm2 = cluster_sum(s);
  const double tol2 = P.rho * P.rho * bnorm2;
  double rr = bnorm2, beta = 0.0, alpha = 0.0, pAp = 0.0;
  int done = bnorm2 == 0.0 ? 1 : 0;
  long long it = 0;
  CgArgs cga{};
  cga.src = P.p;
  cga.r = P.r;
  cga.Dw = P.Dw;
  cga.dst = P.Ap;
  cga.sigma2 = P.sigma2;
  cga.update_p = 1;
  while (!done && it < P.max_iter) {
    double dot = 0.0;
    for (int q = 0; q < P.npass; ++q) {
      const LineGeom& g = P.pass[q];
      const long long nblk = (g.outer * g.inner + g.nb - 1) / g.nb;
      for (long long blk = rank; blk < nblk; blk += CL) dot += run_pass<T>(P, q, blk, cga, beta, smem_raw);
      if (q + 1 < P.npass) cl.sync();
    }
    pAp = cluster_sum(dot);
    if (!(pAp > 0.0) || !isfinite(pAp)) {
      done = 3;
      break;
    }
    alpha = rr / pAp;
    double s2 = 0.0;
    for (long long i = e0; i < M; i += es) {
      const double2 pv = P.p[i], av = P.Ap[i];
      double2 xv = P.x[i], rv = P.r[i];
      xv.x += alpha * pv.x;
      xv.y += alpha * pv.y;
      rv.x -= alpha * av.x;
      rv.y -= alpha * av.y;
      P.x[i] = xv;
      P.r[i] = rv;
      s2 += rv.x * rv.x + rv.y * rv.y;
    }
    const double rr_new = cluster_sum(s2);
    ++it;
    beta = rr_new / rr;
    rr = rr_new;
    if (!isfinite(rr)) done = 3;
    else if (rr <= tol2) done = 1;
  }
  if (!done) done = 2;
  if (rank == 0 && tid == 0) {
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
    st->done = done;
  }
}

template <typename T>
static cudaError_t launch_t(const PersistentProblem* d_probs, int nprob, int cluster, size_t smem, cudaStream_t s) {
  auto kern = cg_cluster_kernel<T>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (cluster > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(cluster * nprob), 1, 1);
  cfg.blockDim = dim3(kPersistentThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, d_probs);
}

cudaError_t launch_cg_persistent(const PersistentProblem* d_probs, int nprob, int cluster, size_t smem, int f64,
                                 cudaStream_t s) {
  return f64 ? launch_t<double>(d_probs, nprob, cluster, smem, s) : launch_t<float>(d_probs, nprob, cluster, smem, s);
}

// Largest cluster (16, else 8) whose blocks fit with this shared memory.
int persistent_cluster_size(int f64, size_t smem) {
  for (int cluster : {16, 8}) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)cluster, 1, 1);
    cfg.blockDim = dim3(kPersistentThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    cudaError_t e;
    if (f64) {
      cudaFuncSetAttribute(cg_cluster_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (cluster > 8) cudaFuncSetAttribute(cg_cluster_kernel<double>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      e = cudaOccupancyMaxActiveClusters(&n, cg_cluster_kernel<double>, &cfg);
    } else {
      cudaFuncSetAttribute(cg_cluster_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (cluster > 8) cudaFuncSetAttribute(cg_cluster_kernel<float>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      e = cudaOccupancyMaxActiveClusters(&n, cg_cluster_kernel<float>, &cfg);
    }
    if (e == cudaSuccess && n > 0) return cluster;
    cudaGetLastError();
  }
  return 0;
}

}  // namespace efgp
