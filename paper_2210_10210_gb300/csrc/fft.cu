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

template <typename T, int INM, int OUTM, bool CONV>
__global__ void __launch_bounds__(kLineFftMaxThreads) line_fft_kernel(LineGeom g, const void* __restrict__ in_v, void* out_v, int dir,
                                                       const cplx<T>* __restrict__ tw, const T* __restrict__ what,
                                                       CgArgs cga) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  grid_dependency_wait();
  if (INM == IN_CG || OUTM == OUT_CG) {
    if (cga.check_done && cga.st->done) return;
  }
  double cg_beta = 0.0;
  if (INM == IN_CG && cga.update_p) cg_beta = cga.st->beta;
  const double dot = line_block<T, INM, OUTM, CONV>(g, blockIdx.x, in_v, out_v, dir, tw, what, cga, cg_beta, smem_raw);
  if (OUTM == OUT_CG && cga.do_dot) {
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
          st->alpha = st->rr / tot;
        }
        st->ticket_a = 0u;
      }
    }
  }
}

size_t line_fft_smem_bytes(int L, int nb, size_t elem_bytes) { return 2 * (size_t)nb * (L + 1) * elem_bytes; }

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
