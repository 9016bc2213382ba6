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

namespace efgp {

// ------------------------------------------------------------ small DFTs
template <typename T, int R> struct Roots;
template <typename T> struct Roots<T, 3> {
  static __device__ __forceinline__ T c(int k) { return k == 0 ? T(1) : T(-0.5); }
  static __device__ __forceinline__ T s(int k) {
    return k == 0 ? T(0) : (k == 1 ? T(0.86602540378443864676) : T(-0.86602540378443864676));
  }
};
template <typename T> struct Roots<T, 5> {
  static __device__ __forceinline__ T c(int k) {
    const T t[5] = {T(1), T(0.30901699437494742410), T(-0.80901699437494742410), T(-0.80901699437494742410),
                    T(0.30901699437494742410)};
    return t[k];
  }
  static __device__ __forceinline__ T s(int k) {
    const T t[5] = {T(0), T(0.95105651629515357212), T(0.58778525229247312917), T(-0.58778525229247312917),
                    T(-0.95105651629515357212)};
    return t[k];
  }
};
template <typename T> struct Roots<T, 7> {
  static __device__ __forceinline__ T c(int k) {
    const T t[7] = {T(1),
                    T(0.62348980185873353053),
                    T(-0.22252093395631440429),
                    T(-0.90096886790241912624),
                    T(-0.90096886790241912624),
                    T(-0.22252093395631440429),
                    T(0.62348980185873353053)};
    return t[k];
  }
  static __device__ __forceinline__ T s(int k) {
    const T t[7] = {T(0),
                    T(0.78183148246802980871),
                    T(0.97492791218182360702),
                    T(0.43388373911755812048),
                    T(-0.43388373911755812048),
                    T(-0.97492791218182360702),
                    T(-0.78183148246802980871)};
    return t[k];
  }
};

// out[q] = sum_r v[r] exp(dir 2 pi i r q / R), in place.
template <typename T, int R>
__device__ __forceinline__ void dft_generic(cplx<T>* v, int dir) {
  cplx<T> o[R];
#pragma unroll
  for (int q = 0; q < R; ++q) {
    T re = 0, im = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int k = (r * q) % R;
      const T c = Roots<T, R>::c(k), s = dir * Roots<T, R>::s(k);
      re += v[r].x * c - v[r].y * s;
      im += v[r].x * s + v[r].y * c;
    }
    o[q] = mk<T>(re, im);
  }
#pragma unroll
  for (int q = 0; q < R; ++q) v[q] = o[q];
}

template <typename T>
__device__ __forceinline__ void dft2(cplx<T>& a, cplx<T>& b) {
  cplx<T> t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <typename T>
__device__ __forceinline__ void dft4(cplx<T>* v, int dir) {
  cplx<T> a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
  cplx<T> c = cadd(v[1], v[3]), d = cmul_si(csub(v[1], v[3]), dir);
  v[0] = cadd(a, c);
  v[2] = csub(a, c);
  v[1] = cadd(b, d);
  v[3] = csub(b, d);
}

template <typename T>
__device__ __forceinline__ void dft8(cplx<T>* v, int dir) {
  cplx<T> e[4] = {v[0], v[2], v[4], v[6]};
  cplx<T> o[4] = {v[1], v[3], v[5], v[7]};
  dft4<T>(e, dir);
  dft4<T>(o, dir);
  const T h = T(0.70710678118654752440);
  // o[q] *= exp(dir 2 pi i q / 8)
  o[1] = mk<T>(h * (o[1].x - dir * o[1].y), h * (o[1].y + dir * o[1].x));
  o[2] = cmul_si(o[2], dir);
  o[3] = mk<T>(h * (-o[3].x - dir * o[3].y), h * (-o[3].y + dir * o[3].x));
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    v[q] = cadd(e[q], o[q]);
    v[q + 4] = csub(e[q], o[q]);
  }
}

template <typename T, int R>
__device__ __forceinline__ void dft(cplx<T>* v, int dir) {
  if constexpr (R == 2) dft2<T>(v[0], v[1]);
  else if constexpr (R == 4) dft4<T>(v, dir);
  else if constexpr (R == 8) dft8<T>(v, dir);
  else dft_generic<T, R>(v, dir);
}

// One radix-R Stockham pass over nb lines in shared memory.
template <typename T, int R>
__device__ __forceinline__ void stockham_pass(const cplx<T>* __restrict__ src, cplx<T>* __restrict__ dst, int L,
                                              int LP, int nb, int Ns, int dir, const cplx<T>* __restrict__ tw) {
  const int nbf = L / R;
  const int tstride = L / (Ns * R);
  for (int bidx = threadIdx.x; bidx < nb * nbf; bidx += blockDim.x) {
    const int li = bidx / nbf;
    const int j = bidx - li * nbf;
    const int k = j % Ns;
    const cplx<T>* s = src + li * LP;
    cplx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = s[j + r * nbf];
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        cplx<T> t = __ldg(tw + k * r * tstride);
        if (dir > 0) t.y = -t.y;
        v[r] = cmul(v[r], t);
      }
    }
    dft<T, R>(v, dir);
    cplx<T>* d = dst + li * LP + (j / Ns) * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) d[r * Ns] = v[r];
  }
}

// Full transform of nb lines; returns the buffer holding the result.
template <typename T>
__device__ cplx<T>* stockham_all(cplx<T>* b0, cplx<T>* b1, const LineGeom& g, int LP, int nb, int dir,
                                 const cplx<T>* tw) {
  int Ns = 1;
  cplx<T>* src = b0;
  cplx<T>* dst = b1;
  for (int p = 0; p < g.npass; ++p) {
    const int R = g.radix[p];
    switch (R) {
      case 2: stockham_pass<T, 2>(src, dst, g.L, LP, nb, Ns, dir, tw); break;
      case 3: stockham_pass<T, 3>(src, dst, g.L, LP, nb, Ns, dir, tw); break;
      case 4: stockham_pass<T, 4>(src, dst, g.L, LP, nb, Ns, dir, tw); break;
      case 5: stockham_pass<T, 5>(src, dst, g.L, LP, nb, Ns, dir, tw); break;
      case 7: stockham_pass<T, 7>(src, dst, g.L, LP, nb, Ns, dir, tw); break;
      default: stockham_pass<T, 8>(src, dst, g.L, LP, nb, Ns, dir, tw); break;
    }
    __syncthreads();
    cplx<T>* t = src;
    src = dst;
    dst = t;
    Ns *= R;
  }
  return src;
}

template <typename T, int INM, int OUTM, bool CONV>
__global__ void __launch_bounds__(256) line_fft_kernel(LineGeom g, const void* __restrict__ in_v, void* out_v, int dir,
                                                       const cplx<T>* __restrict__ tw, const T* __restrict__ what,
                                                       CgArgs cga) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  if (INM == IN_CG || OUTM == OUT_CG) {
    if (cga.check_done && cga.st->done) return;
  }
  const int L = g.L, nb = g.nb;
  const int LP = L + 1;
  cplx<T>* b0 = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* b1 = b0 + (size_t)nb * LP;
  const long long nlines = g.outer * g.inner;
  const long long line0 = (long long)blockIdx.x * nb;
  const bool strided = g.inner > 1;

  // ---- load (zero-padded to L)
  double cg_beta = 0.0;
  if (INM == IN_CG && cga.update_p) cg_beta = cga.st->beta;
  for (int e = threadIdx.x; e < nb * L; e += blockDim.x) {
    int li, k;
    if (strided) { li = e % nb; k = e / nb; } else { li = e / L; k = e - li * L; }
    const long long line = line0 + li;
    cplx<T> v = mk<T>(0, 0);
    if (line < nlines && k < g.n_in) {
      const long long o = line / g.inner, i = line - o * g.inner;
      if (INM == IN_PLAIN) {
        v = reinterpret_cast<const cplx<T>*>(in_v)[o * g.in_so + (long long)k * g.in_sk + i * g.in_si];
      } else {
        const long long j = o * g.n_in + k;   // flat index into the M-vector
        double2 pv = cga.src[j];
        if (cga.update_p) {
          const double2 rv = cga.r[j];
          pv.x = rv.x + cg_beta * pv.x;
          pv.y = rv.y + cg_beta * pv.y;
          cga.src[j] = pv;
        }
        const double dj = cga.Dw[j];
        v = mk<T>((T)(dj * pv.x), (T)(dj * pv.y));
      }
    }
    b0[li * LP + k] = v;
  }
  __syncthreads();

  cplx<T>* res;
  if (CONV) {
    res = stockham_all<T>(b0, b1, g, LP, nb, -1, tw);
    // pointwise product with the (real) transformed generating vector
    for (int e = threadIdx.x; e < nb * L; e += blockDim.x) {
      int li, k;
      if (strided) { li = e % nb; k = e / nb; } else { li = e / L; k = e - li * L; }
      const long long line = line0 + li;
      if (line < nlines) {
        const long long o = line / g.inner, i = line - o * g.inner;
        const T wv = __ldg(what + (o * L + k) * g.inner + i);
        cplx<T> t = res[li * LP + k];
        res[li * LP + k] = mk<T>(t.x * wv, t.y * wv);
      }
    }
    __syncthreads();
    cplx<T>* other = (res == b0) ? b1 : b0;
    res = stockham_all<T>(res, other, g, LP, nb, +1, tw);
  } else {
    res = stockham_all<T>(b0, b1, g, LP, nb, dir, tw);
  }

  // ---- store the first n_out entries
  double dot = 0.0;
  for (int e = threadIdx.x; e < nb * g.n_out; e += blockDim.x) {
    int li, k;
    if (strided) { li = e % nb; k = e / nb; } else { li = e / g.n_out; k = e - li * g.n_out; }
    const long long line = line0 + li;
    if (line >= nlines) continue;
    const long long o = line / g.inner, i = line - o * g.inner;
    const cplx<T> v = res[li * LP + k];
    if (OUTM == OUT_PLAIN) {
      reinterpret_cast<cplx<T>*>(out_v)[o * g.out_so + (long long)k * g.out_sk + i * g.out_si] = v;
    } else {
      const long long j = o * g.n_out + k;
      const double dj = cga.Dw[j];
      const double2 sv = cga.src[j];
      double2 a;
      a.x = dj * (double)v.x + cga.sigma2 * sv.x;
      a.y = dj * (double)v.y + cga.sigma2 * sv.y;
      cga.dst[j] = a;
      dot += sv.x * a.x + sv.y * a.y;   // Re(conj(src) * a)
    }
  }

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
  kern<<<(unsigned)blocks, threads, smem, s>>>(g, in, out, dir, tw, what, cga);
  return cudaGetLastError();
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
