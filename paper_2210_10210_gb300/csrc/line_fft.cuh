// Device functions of the batched Stockham line FFT (see fft.cu), shared
// by the per-pass kernels and the two single-launch CG kernels.  Inputs that
// another block of the same launch may have written are read with L2-only
// loads (__ldcg), so that no stale L1 line is ever used.
#pragma once

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

// Odd R: with a_r = v_r + v_{R-r} and b_r = v_r - v_{R-r} (r = 1..(R-1)/2),
// out[q] = v_0 + sum_r a_r cos(2 pi r q / R) + i dir sum_r b_r sin(2 pi r q / R)
// and out[R-q] the same with the sine sum negated (the pairs' exponentials are
// complex conjugates), about a third of the multiply-adds of the plain sum.
template <typename T, int R>
__device__ __forceinline__ void dft_odd(cplx<T>* v, int dir) {
  constexpr int H = (R - 1) / 2;
  cplx<T> a[H], b[H];
  cplx<T> y0 = v[0];
#pragma unroll
  for (int r = 1; r <= H; ++r) {
    a[r - 1] = cadd(v[r], v[R - r]);
    b[r - 1] = csub(v[r], v[R - r]);
    y0 = cadd(y0, a[r - 1]);
  }
  const T fd = (T)dir;
  cplx<T> o[R];
  o[0] = y0;
#pragma unroll
  for (int q = 1; q <= H; ++q) {
    T ax = v[0].x, ay = v[0].y, bx = T(0), by = T(0);
#pragma unroll
    for (int r = 1; r <= H; ++r) {
      const int k = (r * q) % R;
      const T c = Roots<T, R>::c(k), sn = Roots<T, R>::s(k);
      ax = fma(a[r - 1].x, c, ax);
      ay = fma(a[r - 1].y, c, ay);
      bx = fma(b[r - 1].x, sn, bx);
      by = fma(b[r - 1].y, sn, by);
    }
    const T ix = -fd * by, iy = fd * bx;   // i dir (bx + i by)
    o[q] = mk<T>(ax + ix, ay + iy);
    o[R - q] = mk<T>(ax - ix, ay - iy);
  }
#pragma unroll
  for (int q = 0; q < R; ++q) v[q] = o[q];
}

// a / b for 0 <= a < 2^24, 0 < b, with rb ~ 1/b: a float estimate corrected by one step
__device__ __forceinline__ int quick_div(int a, int b, float rb) {
  int q = __float2int_rz(__int2float_rn(a) * rb);
  const int r = a - q * b;
  if (r < 0) --q;
  else if (r >= b) ++q;
  return q;
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
  else dft_odd<T, R>(v, dir);
}

// One radix-R Stockham pass over nb lines in shared memory.
template <typename T, int R>
__device__ __forceinline__ void stockham_pass(const cplx<T>* __restrict__ src, cplx<T>* __restrict__ dst, int L,
                                              int LP, int nb, int Ns, int dir, const cplx<T>* __restrict__ tw) {
  const int nbf = L / R;
  const int tstride = L / (Ns * R);
  const float rnbf = 1.0f / (float)nbf, rns = 1.0f / (float)Ns;
  for (int bidx = threadIdx.x; bidx < nb * nbf; bidx += blockDim.x) {
    const int li = nb == 1 ? 0 : quick_div(bidx, nbf, rnbf);
    const int j = bidx - li * nbf;
    const int k = j - quick_div(j, Ns, rns) * Ns;   // j mod Ns
    const cplx<T>* s = src + li * LP;
    cplx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = s[j + r * nbf];
    if (Ns > 1) {
      const int kt = k * tstride;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        cplx<T> t = __ldg(tw + r * kt);
        if (dir > 0) t.y = -t.y;
        v[r] = cmul(v[r], t);
      }
    }
    dft<T, R>(v, dir);
    cplx<T>* d = dst + li * LP + (j - k) * R + k;
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

// One block of nb lines of a pass: load (zero-padded, optionally the CG
// prologue), transform (optionally forward, product, inverse), store the
// first n_out entries (optionally the CG epilogue).  Returns this thread's
// part of Re(src^H dst) for the epilogue.  Ends with the block synchronised.
template <typename T, int INM, int OUTM, bool CONV>
__device__ double line_block(const LineGeom& g, long long blk, const void* __restrict__ in_v, void* out_v, int dir,
                             const cplx<T>* __restrict__ tw, const T* __restrict__ what, const CgArgs& cga,
                             double cg_beta, unsigned char* smem_raw) {
  // per-line element offsets, computed once per line (a line's elements then
  // cost one multiply-add each); -1 marks lines past the end
  __shared__ long long t_in[kMaxLineBatch], t_out[kMaxLineBatch], t_w[kMaxLineBatch];
  const int L = g.L, nb = g.nb;
  const int LP = L + 1;
  cplx<T>* b0 = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* b1 = b0 + (size_t)nb * LP;
  const long long nlines = g.outer * g.inner;
  const long long line0 = blk * nb;
  const bool strided = g.inner > 1;
  if (threadIdx.x < nb) {
    const long long line = line0 + threadIdx.x;
    long long bi = -1, bo = -1, bw = -1;
    if (line < nlines) {
      const long long o = line / g.inner, i = line - o * g.inner;
      bi = INM == IN_PLAIN ? o * g.in_so + i * g.in_si : o * g.n_in;
      bo = OUTM == OUT_PLAIN ? o * g.out_so + i * g.out_si : o * g.n_out;
      bw = o * L * g.inner + i;
    }
    t_in[threadIdx.x] = bi;
    t_out[threadIdx.x] = bo;
    t_w[threadIdx.x] = bw;
  }
  __syncthreads();
  const float rnb = 1.0f / (float)nb, rL = 1.0f / (float)L, rno = 1.0f / (float)g.n_out;

  // ---- load (zero-padded to L)
  for (int e = threadIdx.x; e < nb * L; e += blockDim.x) {
    int li, k;
    if (strided) { k = quick_div(e, nb, rnb); li = e - k * nb; } else { li = quick_div(e, L, rL); k = e - li * L; }
    const long long base = t_in[li];
    cplx<T> v = mk<T>(0, 0);
    if (base >= 0 && k < g.n_in) {
      if (INM == IN_PLAIN) {
        v = __ldcg(reinterpret_cast<const cplx<T>*>(in_v) + (base + (long long)k * g.in_sk));
      } else {
        const long long j = base + k;   // flat index into the M-vector
        double2 pv = __ldcg(cga.src + j);
        if (cga.update_p) {
          double2 rv = __ldcg(cga.r + j);
          if (cga.Minv) {   // preconditioned residual z = M^-1 r
            const double mi = cga.Minv[j];
            rv.x *= mi;
            rv.y *= mi;
          }
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
      if (strided) { k = quick_div(e, nb, rnb); li = e - k * nb; } else { li = quick_div(e, L, rL); k = e - li * L; }
      const long long bw = t_w[li];
      if (bw >= 0) {
        const T wv = __ldg(what + (bw + (long long)k * g.inner));
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
    if (strided) { k = quick_div(e, nb, rnb); li = e - k * nb; } else { li = quick_div(e, g.n_out, rno); k = e - li * g.n_out; }
    const long long base = t_out[li];
    if (base < 0) continue;
    const cplx<T> v = res[li * LP + k];
    if (OUTM == OUT_PLAIN) {
      reinterpret_cast<cplx<T>*>(out_v)[base + (long long)k * g.out_sk] = v;
    } else {
      const long long j = base + k;
      const double dj = cga.Dw[j];
      const double2 sv = __ldcg(cga.src + j);
      double2 a;
      a.x = dj * (double)v.x + cga.sigma2 * sv.x;
      a.y = dj * (double)v.y + cga.sigma2 * sv.y;
      cga.dst[j] = a;
      dot += sv.x * a.x + sv.y * a.y;   // Re(conj(src) * a)
    }
  }

  __syncthreads();
  return dot;
}

// Line block blk of pass q of a problem descriptor (the CG variants of the
// product: prologue on the first pass, epilogue on the last).
template <typename T>
__device__ __forceinline__ double run_pass(const PersistentProblem& P, int q, long long blk, const CgArgs& cga,
                                           double beta, unsigned char* smem) {
  const LineGeom& g = P.pass[q];
  const void* in = P.buf[P.inb[q]];
  void* out = P.buf[P.outb[q]];
  const cplx<T>* tw = reinterpret_cast<const cplx<T>*>(P.tw);
  const T* what = reinterpret_cast<const T*>(P.what);
  const int dir = P.dir[q];
  const int inm = P.inm[q], outm = P.outm[q];
  if (P.conv[q]) {
    if (inm == IN_CG) return line_block<T, IN_CG, OUT_CG, true>(g, blk, in, out, dir, tw, what, cga, beta, smem);
    return line_block<T, IN_PLAIN, OUT_PLAIN, true>(g, blk, in, out, dir, tw, what, cga, beta, smem);
  }
  if (inm == IN_CG) return line_block<T, IN_CG, OUT_PLAIN, false>(g, blk, in, out, dir, tw, what, cga, beta, smem);
  if (outm == OUT_CG) return line_block<T, IN_PLAIN, OUT_CG, false>(g, blk, in, out, dir, tw, what, cga, beta, smem);
  return line_block<T, IN_PLAIN, OUT_PLAIN, false>(g, blk, in, out, dir, tw, what, cga, beta, smem);
}

}  // namespace efgp
