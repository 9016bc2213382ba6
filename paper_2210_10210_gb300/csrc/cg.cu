// Conjugate-gradient vector kernels (Algorithm step 4): initialisation,
// the x/r update with the r^H r reduction and convergence test, and a
// residual norm.  Scalars live in a device CgState so that a whole group of
// iterations can be captured in one CUDA graph; every kernel returns at once
// when the state says the solve has finished.  Reductions are two-level and
// deterministic: per-block partials, summed in a fixed order by the block
// that arrives last.
#include "kernels.h"

namespace efgp {

constexpr int kCgThreads = 256;

// One element per thread up to 1024 blocks: the FP64 vector arithmetic is
// spread over as many SMs as the vector allows (FP64 throughput per SM is low).
int cg_blocks(long long M) {
  long long b = (M + kCgThreads - 1) / kCgThreads;
  if (b < 1) b = 1;
  if (b > 1024) b = 1024;
  return (int)b;
}

// Sums of two values over the block (results valid in thread 0).
__device__ __forceinline__ void block_sum2(double& a, double& b, double* red) {
  a = block_sum(a, red);
  __syncthreads();
  b = block_sum(b, red);
}

// x = 0, r = b, p = z = M^-1 r (z = r without a preconditioner); ||b||^2 and
// r^H z reduced in block order by the last block.
__global__ void __launch_bounds__(kCgThreads) cg_init_kernel(const double2* __restrict__ b, double2* __restrict__ x,
                                                             double2* __restrict__ r, double2* __restrict__ p,
                                                             long long M, double rho, long long max_iter, CgState* st,
                                                             double* partials, const double* __restrict__ Minv) {
  __shared__ double red[32];
  double s = 0.0, sz = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
    const double2 v = b[i];
    const double mi = Minv ? Minv[i] : 1.0;
    x[i] = make_double2(0.0, 0.0);
    r[i] = v;
    p[i] = make_double2(mi * v.x, mi * v.y);
    const double n2 = v.x * v.x + v.y * v.y;
    s += n2;
    sz += mi * n2;
  }
  block_sum2(s, sz, red);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = s;
    partials[gridDim.x + blockIdx.x] = sz;
    __threadfence();
    last = (atomicAdd(&st->ticket_b, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    const double tot = block_sum_partials(partials, gridDim.x, red);
    __syncthreads();
    const double totz = block_sum_partials(partials + gridDim.x, gridDim.x, red);
    if (threadIdx.x == 0) {
      st->bnorm2 = tot;
      st->rr = tot;
      st->rz = Minv ? totz : tot;
      st->rr_new = tot;
      st->tol2 = rho * rho * tot;
      st->iter = 0;
      st->max_iter = max_iter;
      st->alpha = 0.0;
      st->beta = 0.0;
      st->pAp = 0.0;
      st->done = (tot == 0.0) ? 1 : (max_iter <= 0 ? 2 : 0);
      st->ticket_b = 0u;
    }
  }
}

// x += alpha p, r -= alpha A p; r^H r (the stopping rule) and r^H M^-1 r (for
// beta = (r^H z)_new / (r^H z)) reduced in block order by the last block.
__global__ void __launch_bounds__(kCgThreads) cg_update_kernel(double2* __restrict__ x, double2* __restrict__ r,
                                                               const double2* __restrict__ p,
                                                               const double2* __restrict__ Ap, long long M,
                                                               CgState* st, double* partials,
                                                               const double* __restrict__ Minv) {
  __shared__ double red[32];
  grid_dependency_wait();
  if (st->done) return;
  const double alpha = st->alpha;
  double s = 0.0, sz = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
    const double2 pv = p[i], av = Ap[i];
    double2 xv = x[i], rv = r[i];
    xv.x += alpha * pv.x;
    xv.y += alpha * pv.y;
    rv.x -= alpha * av.x;
    rv.y -= alpha * av.y;
    x[i] = xv;
    r[i] = rv;
    const double n2 = rv.x * rv.x + rv.y * rv.y;
    s += n2;
    if (Minv) sz += Minv[i] * n2;
  }
  if (Minv) block_sum2(s, sz, red);
  else s = block_sum(s, red);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = s;
    if (Minv) partials[gridDim.x + blockIdx.x] = sz;
    __threadfence();
    last = (atomicAdd(&st->ticket_b, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    const double tot = block_sum_partials(partials, gridDim.x, red);
    double totz = tot;
    if (Minv) {
      __syncthreads();
      totz = block_sum_partials(partials + gridDim.x, gridDim.x, red);
    }
    if (threadIdx.x == 0) {
      st->rr_new = tot;
      st->iter += 1;
      st->beta = totz / st->rz;
      st->rr = tot;
      st->rz = totz;
      if (!isfinite(tot)) st->done = 3;
      else if (tot <= st->tol2) st->done = 1;
      else if (st->iter >= st->max_iter) st->done = 2;
      st->ticket_b = 0u;
    }
  }
}

__global__ void jacobi_kernel(const double* __restrict__ Dw, const double2* __restrict__ wc, double sigma2,
                              long long M, double* __restrict__ Minv) {
  const double w0 = wc->x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x)
    Minv[i] = 1.0 / (Dw[i] * Dw[i] * w0 + sigma2);
}

// out_sum[0] = ||b - Ax||^2 (single value, deterministic)
__global__ void __launch_bounds__(kCgThreads) residual_kernel(const double2* __restrict__ b,
                                                              const double2* __restrict__ Ax, long long M,
                                                              double* out_sum, double* partials,
                                                              unsigned int* ticket) {
  __shared__ double red[32];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
    const double2 u = b[i], v = Ax[i];
    const double dx = u.x - v.x, dy = u.y - v.y;
    s += dx * dx + dy * dy;
  }
  const double bs = block_sum(s, red);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = bs;
    __threadfence();
    last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    const double tot = block_sum_partials(partials, gridDim.x, red);
    if (threadIdx.x == 0) {
      out_sum[0] = tot;
      *ticket = 0u;
    }
  }
}

cudaError_t launch_cg_init(const double2* b, double2* x, double2* r, double2* p, long long M, double rho,
                           long long max_iter, CgState* st, double* partials, const double* Minv, cudaStream_t s) {
  cg_init_kernel<<<cg_blocks(M), kCgThreads, 0, s>>>(b, x, r, p, M, rho, max_iter, st, partials, Minv);
  return cudaGetLastError();
}

cudaError_t launch_cg_update(double2* x, double2* r, const double2* p, const double2* Ap, long long M, CgState* st,
                             double* partials, const double* Minv, cudaStream_t s) {
  return launch_pdl(cg_update_kernel, dim3(cg_blocks(M)), dim3(kCgThreads), 0, s, x, r, p, Ap, M, st, partials, Minv);
}

cudaError_t launch_jacobi(const double* Dw, const double2* w_center, double sigma2, long long M, double* Minv,
                          cudaStream_t s) {
  jacobi_kernel<<<cg_blocks(M), kCgThreads, 0, s>>>(Dw, w_center, sigma2, M, Minv);
  return cudaGetLastError();
}

cudaError_t launch_residual_norm(const double2* b, const double2* Ax, long long M, double* out_sum, double* partials,
                                 unsigned int* ticket, cudaStream_t s) {
  residual_kernel<<<cg_blocks(M), kCgThreads, 0, s>>>(b, Ax, M, out_sum, partials, ticket);
  return cudaGetLastError();
}

}  // namespace efgp
