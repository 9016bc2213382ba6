// Batched mixed-radix Stockham FFTs along one axis of a strided array, held
// in shared memory one block of lines at a time.
//
// Used for the Toeplitz product of Algorithm "Fast product of Toeplitz
// matrix F^*F with a vector" (zero-pad, FFT, multiply by the transformed
// generating vector, inverse FFT, crop) and for the fine-grid FFTs of the
// type-1 and type-2 nonuniform FFTs.  Pads and crops are folded into the
// loads and stores (n_in < L entries read, n_out < L entries written), the
// pointwise product sits between the forward and inverse passes of the
// outermost axis, and the first/last pass of a matrix-vector product can
// apply the spectral-weight diagonal D, the CG direction update and the
// sigma^2 shift plus the p^H A p reduction (eq. 97).
//
// Stockham autosort (decimation in time): with Ns the product of the radices
// already applied, butterfly j of a radix-R pass reads x[j + r L/R], scales
// element r by exp(dir 2 pi i r (j mod Ns) / (Ns R)), takes a length-R DFT and
// writes y[(j/Ns) Ns R + (j mod Ns) + q Ns]; after all passes y holds the DFT
// in natural order.
#include <cstdio>

#include "kernels.h"
#include "line_fft.cuh"

namespace efgp {

// p^H A p over the grid from each thread's part: per-block partials, summed in
// block order by the block that arrives last, which sets alpha = r^H r / p^H A p.
__device__ void pap_reduce(double dot, const CgArgs& cga, double* red) {
  const double bs = block_sum(dot, red);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    cga.partials[blockIdx.x] = bs;
    __threadfence();
    const unsigned int t = atomicAdd(&cga.st->ticket_a, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    const double tot = block_sum_partials(cga.partials, gridDim.x, red);
    if (threadIdx.x == 0) {
      CgState* st = cga.st;
      st->pAp = tot;
      if (!(tot > 0.0) || !isfinite(tot)) {
        st->alpha = 0.0;
        st->done = 3;   // breakdown: p^H A p not positive
      } else {
        st->alpha = st->rz / tot;
      }
      st->ticket_a = 0u;
    }
  }
}

template <typename T, int INM, int OUTM, bool CONV>
__global__ void __launch_bounds__(kLineFftMaxThreads) line_fft_kernel(LineGeom g, const void* __restrict__ in_v, void* out_v, int dir,
                                                       const cplx<T>* __restrict__ tw, const T* __restrict__ what,
                                                       CgArgs cga) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  grid_dependency_wait();
  // (plain passes skip the state read: one dependent load on every
  // iteration's critical path costs more than the few passes run after
  // convergence inside a captured group)
  if (INM == IN_CG || OUTM == OUT_CG) {
    if (cga.check_done && cga.st->done) return;
  }
  double cg_beta = 0.0;
  if (INM == IN_CG && cga.update_p) cg_beta = cga.st->beta;
  const double dot = line_block<T, INM, OUTM, CONV>(g, blockIdx.x, in_v, out_v, dir, tw, what, cga, cg_beta, smem_raw);
  if (OUTM == OUT_CG && cga.do_dot) pap_reduce(dot, cga, red);
}

size_t line_fft_smem_bytes(int L, int nb, size_t elem_bytes) { return 2 * (size_t)nb * (L + 1) * elem_bytes; }

// ---- 3D Toeplitz product, inner two axes of one slab per block.
// The CG vector is [j0][j1][j2] (n1^3); the scratch S holds [j0][k1][k2]
// (n1 x L x L) between the forward plane pass, the axis-0 pass with the
// w-hat product, and the inverse plane pass.  A block takes slab j0: its
// n1 x n1 values are FFT'd along axis 2 (n1 rows, padded to L), transposed in
// shared memory and FFT'd along axis 1 (L rows); the inverse pass mirrors it
// and keeps the first n1 entries of each axis.

// forward: CG prologue (p = r + beta p, times D) -> S
template <typename T>
__global__ void __launch_bounds__(kPlaneThreads) plane_fwd_kernel(LineGeom g, int n1, cplx<T>* __restrict__ S,
                                                                  const cplx<T>* __restrict__ tw, CgArgs cga) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  grid_dependency_wait();
  if (cga.check_done && cga.st->done) return;
  const double beta = cga.update_p ? cga.st->beta : 0.0;
  const int L = g.L, LP = L + 1;
  cplx<T>* b0 = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* b1 = b0 + (size_t)L * LP;
  const long long j0 = blockIdx.x;
  const long long base = j0 * n1 * n1;
  const float rL = 1.0f / (float)L;
  for (int e = threadIdx.x; e < n1 * L; e += blockDim.x) {
    const int j1 = quick_div(e, L, rL), k = e - j1 * L;
    cplx<T> v = mk<T>(0, 0);
    if (k < n1) {
      const long long j = base + (long long)j1 * n1 + k;
      double2 pv = __ldcg(cga.src + j);
      if (cga.update_p) {
        double2 rv = __ldcg(cga.r + j);
        if (cga.Minv) {
          const double mi = cga.Minv[j];
          rv.x *= mi;
          rv.y *= mi;
        }
        pv.x = rv.x + beta * pv.x;
        pv.y = rv.y + beta * pv.y;
        cga.src[j] = pv;
      }
      const double dj = cga.Dw[j];
      v = mk<T>((T)(dj * pv.x), (T)(dj * pv.y));
    }
    b0[j1 * LP + k] = v;
  }
  __syncthreads();
  cplx<T>* r = stockham_all<T>(b0, b1, g, LP, n1, -1, tw);   // axis 2, rows j1 < n1
  cplx<T>* o = (r == b0) ? b1 : b0;
  for (int e = threadIdx.x; e < L * L; e += blockDim.x) {
    const int k2 = quick_div(e, L, rL), j1 = e - k2 * L;
    o[k2 * LP + j1] = j1 < n1 ? r[j1 * LP + k2] : mk<T>(0, 0);
  }
  __syncthreads();
  cplx<T>* r2 = stockham_all<T>(o, r, g, LP, L, -1, tw);     // axis 1, rows k2 < L
  cplx<T>* out = S + j0 * L * L;
  for (int e = threadIdx.x; e < L * L; e += blockDim.x) {
    const int k1 = quick_div(e, L, rL), k2 = e - k1 * L;
    out[e] = r2[k2 * LP + k1];
  }
}

// inverse: S -> CG epilogue (A p = D v + sigma^2 p) and the p^H A p reduction
template <typename T>
__global__ void __launch_bounds__(kPlaneThreads) plane_inv_kernel(LineGeom g, int n1, const cplx<T>* __restrict__ S,
                                                                  const cplx<T>* __restrict__ tw, CgArgs cga) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  grid_dependency_wait();
  if (cga.check_done && cga.st->done) return;
  const int L = g.L, LP = L + 1;
  cplx<T>* b0 = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* b1 = b0 + (size_t)L * LP;
  const long long j0 = blockIdx.x;
  const float rL = 1.0f / (float)L, rn1 = 1.0f / (float)n1;
  const cplx<T>* in = S + j0 * L * L;
  for (int e = threadIdx.x; e < L * L; e += blockDim.x) {
    const int k1 = quick_div(e, L, rL), k2 = e - k1 * L;
    b0[k1 * LP + k2] = __ldcg(in + e);
  }
  __syncthreads();
  cplx<T>* r = stockham_all<T>(b0, b1, g, LP, L, +1, tw);    // axis 2, rows k1 < L
  cplx<T>* o = (r == b0) ? b1 : b0;
  for (int e = threadIdx.x; e < n1 * L; e += blockDim.x) {
    const int j2 = quick_div(e, L, rL), k1 = e - j2 * L;
    o[j2 * LP + k1] = r[k1 * LP + j2];
  }
  __syncthreads();
  cplx<T>* r2 = stockham_all<T>(o, r, g, LP, n1, +1, tw);    // axis 1, rows j2 < n1
  double dot = 0.0;
  const long long base = j0 * n1 * n1;
  for (int e = threadIdx.x; e < n1 * n1; e += blockDim.x) {
    const int j1 = quick_div(e, n1, rn1), j2 = e - j1 * n1;
    const cplx<T> v = r2[j2 * LP + j1];
    const long long j = base + e;
    const double dj = cga.Dw[j];
    const double2 sv = __ldcg(cga.src + j);
    double2 a;
    a.x = dj * (double)v.x + cga.sigma2 * sv.x;
    a.y = dj * (double)v.y + cga.sigma2 * sv.y;
    cga.dst[j] = a;
    dot += sv.x * a.x + sv.y * a.y;
  }
  __syncthreads();
  if (cga.do_dot) pap_reduce(dot, cga, red);
}

size_t plane_fft_smem_bytes(int L, size_t elem_bytes) { return 2 * (size_t)L * (L + 1) * elem_bytes; }

template <typename T>
cudaError_t launch_plane_fft(const LineGeom& g, int n1, int inverse, void* S, const cplx<T>* tw, const CgArgs& cga,
                             cudaStream_t s) {
  const size_t smem = plane_fft_smem_bytes(g.L, sizeof(cplx<T>));
  if (inverse)
    return launch_pdl(plane_inv_kernel<T>, dim3((unsigned)n1), dim3(kPlaneThreads), smem, s, g, n1,
                      reinterpret_cast<const cplx<T>*>(S), tw, cga);
  return launch_pdl(plane_fwd_kernel<T>, dim3((unsigned)n1), dim3(kPlaneThreads), smem, s, g, n1,
                    reinterpret_cast<cplx<T>*>(S), tw, cga);
}
template cudaError_t launch_plane_fft<float>(const LineGeom&, int, int, void*, const float2*, const CgArgs&,
                                             cudaStream_t);
template cudaError_t launch_plane_fft<double>(const LineGeom&, int, int, void*, const double2*, const CgArgs&,
                                              cudaStream_t);

template <typename T>
cudaError_t prepare_plane_fft() {
  cudaError_t e = cudaFuncSetAttribute(plane_fwd_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kLineFftBlockSmem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(plane_inv_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kLineFftBlockSmem);
}
template cudaError_t prepare_plane_fft<float>();
template cudaError_t prepare_plane_fft<double>();

template <typename T, int INM, int OUTM, bool CONV>
static cudaError_t launch_one(const LineGeom& g, const void* in, void* out, int dir, const cplx<T>* tw, const T* what,
                              const CgArgs& cga, int threads, cudaStream_t s) {
  auto kern = line_fft_kernel<T, INM, OUTM, CONV>;
  const long long nlines = g.outer * g.inner;
  const long long blocks = (nlines + g.nb - 1) / g.nb;
  const size_t smem = line_fft_smem_bytes(g.L, g.nb, sizeof(cplx<T>));
  return launch_pdl(kern, dim3((unsigned)blocks), dim3(threads), smem, s, g, in, out, dir, tw, what, cga);
}

// Opt every instantiation in to the large dynamic shared-memory carve-out
// (done once, outside any stream capture).
template <typename T>
cudaError_t prepare_line_fft() {
  const int bytes = kLineFftMaxSmem;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(line_fft_kernel<T, IN_PLAIN, OUT_PLAIN, false>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(line_fft_kernel<T, IN_PLAIN, OUT_PLAIN, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(line_fft_kernel<T, IN_CG, OUT_PLAIN, false>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(line_fft_kernel<T, IN_PLAIN, OUT_CG, false>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess) return e;
  return cudaFuncSetAttribute(line_fft_kernel<T, IN_CG, OUT_CG, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              bytes);
}
template cudaError_t prepare_line_fft<float>();
template cudaError_t prepare_line_fft<double>();

template <typename T>
cudaError_t launch_line_fft(const LineGeom& g, const void* in, void* out, int dir, const cplx<T>* tw, const T* what,
                            int inm, int outm, const CgArgs* cgap, int threads, cudaStream_t s) {
  CgArgs cga{};
  if (cgap) cga = *cgap;
  const bool conv = what != nullptr;
  if (inm == IN_PLAIN && outm == OUT_PLAIN && !conv)
    return launch_one<T, IN_PLAIN, OUT_PLAIN, false>(g, in, out, dir, tw, what, cga, threads, s);
  if (inm == IN_PLAIN && outm == OUT_PLAIN && conv)
    return launch_one<T, IN_PLAIN, OUT_PLAIN, true>(g, in, out, dir, tw, what, cga, threads, s);
  if (inm == IN_CG && outm == OUT_PLAIN && !conv)
    return launch_one<T, IN_CG, OUT_PLAIN, false>(g, in, out, dir, tw, what, cga, threads, s);
  if (inm == IN_PLAIN && outm == OUT_CG && !conv)
    return launch_one<T, IN_PLAIN, OUT_CG, false>(g, in, out, dir, tw, what, cga, threads, s);
  if (inm == IN_CG && outm == OUT_CG && conv)
    return launch_one<T, IN_CG, OUT_CG, true>(g, in, out, dir, tw, what, cga, threads, s);
  return cudaErrorInvalidValue;
}

template cudaError_t launch_line_fft<float>(const LineGeom&, const void*, void*, int, const float2*, const float*, int,
                                            int, const CgArgs*, int, cudaStream_t);
template cudaError_t launch_line_fft<double>(const LineGeom&, const void*, void*, int, const double2*, const double*,
                                             int, int, const CgArgs*, int, cudaStream_t);

}  // namespace efgp
