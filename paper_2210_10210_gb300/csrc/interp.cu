// Prediction kernels (Algorithm step 6): the posterior mean
// mu(z) = sum_{j in J_m} D_j beta_j exp(+2 pi i h j.z) (eq. muws) at q
// targets by a type-2 nonuniform FFT: divide the coefficients by the ES
// kernel's Fourier transform, place them on the fine grid, inverse FFT,
// unfold the periodic grid into an extended real grid (the coefficients are
// conjugate-symmetric, so the grid is real), and interpolate with the same
// exponential-of-semicircle weights as the spread.
#include <algorithm>
#include <cstdint>

#include "kernels.h"

namespace efgp {

// g[j mod nf] = D_j beta_j / prod psihat(j_a); the grid is zeroed first
template <int D, typename T>
__global__ void precorrect_kernel(const double2* __restrict__ beta, const double* __restrict__ Dw,
                                  const double* __restrict__ corr, int m, int nf, cplx<T>* __restrict__ g) {
  const int n1 = 2 * m + 1;
  long long total = n1;
  if (D > 1) total *= n1;
  if (D > 2) total *= n1;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    long long r = idx;
    int j[3];
    for (int a = D - 1; a >= 0; --a) {
      j[a] = (int)(r % n1) - m;
      r /= n1;
    }
    double c = Dw[idx];
    long long gi = 0;
    for (int a = 0; a < D; ++a) {
      c *= corr[j[a] + m];
      gi = gi * nf + (((j[a] % nf) + nf) % nf);
    }
    const double2 bv = beta[idx];
    g[gi] = mk<T>((T)(c * bv.x), (T)(c * bv.y));
  }
}

// E2[e] = Re g[(e - off) mod nf] on the extended grid nE^d
template <int D, typename T>
__global__ void unfold_kernel(const cplx<T>* __restrict__ g, int nf, int off, int nE, T* __restrict__ E2) {
  long long total = nE;
  if (D > 1) total *= nE;
  if (D > 2) total *= nE;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    long long r = idx, gi = 0;
    int e[3];
    for (int a = D - 1; a >= 0; --a) {
      e[a] = (int)(r % nE);
      r /= nE;
    }
    for (int a = 0; a < D; ++a) gi = gi * nf + (((e[a] - off) % nf + nf) % nf);
    E2[idx] = g[gi].x;
  }
}

template <int D, int W, typename TC, typename TV, typename TR>
__global__ void __launch_bounds__(256) interp_kernel(const TC* __restrict__ z, int soa, long long q, GridScale gs,
                                                     int off, int nE, const TR* __restrict__ E2, EsCoef<TR> cf,
                                                     TV* __restrict__ mu, int* range_flag) {
  bool bad = false;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < q; i += (long long)gridDim.x * blockDim.x) {
    TR wt[D][W];
    int e0[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      TC za = soa ? z[(long long)a * q + i] : z[i * D + a];
      if (!(za >= TC(0) && za <= TC(1))) {
        bad = true;
        za = TC(0);
      }
      int l0;
      TR f;
      GridPos<TC, TR>::get(za, gs, l0, f);
      int e = l0 + off;
      e = max(0, min(e, nE - W));
      e0[a] = e;
      if constexpr (sizeof(TR) == 4) es_weights_x2<W>(f, cf, wt[a]);
      else es_weights<TR, W>(f, cf, wt[a]);
    }
    TR acc = 0;
    if (D == 1) {
#pragma unroll
      for (int u = 0; u < W; ++u) acc += wt[0][u] * __ldg(E2 + e0[0] + u);
    } else if (D == 2) {
#pragma unroll
      for (int u = 0; u < W; ++u) {
        const TR* row = E2 + (long long)(e0[0] + u) * nE + e0[D - 1];
        TR s = 0;
#pragma unroll
        for (int v = 0; v < W; ++v) s += wt[D - 1][v] * __ldg(row + v);
        acc += wt[0][u] * s;
      }
    } else {
      for (int u = 0; u < W; ++u) {
        TR s1 = 0;
#pragma unroll
        for (int v = 0; v < W; ++v) {
          const TR* row = E2 + ((long long)(e0[0] + u) * nE + e0[1 % D] + v) * nE + e0[D - 1];
          TR s = 0;
#pragma unroll
          for (int x = 0; x < W; ++x) s += wt[D - 1][x] * __ldg(row + x);
          s1 += wt[1 % D][v] * s;
        }
        acc += wt[0][u] * s1;
      }
    }
    mu[i] = (TV)acc;
  }
  if (bad) atomicOr(range_flag, 1);
}

// The same interpolation with the whole real extended grid staged in shared
// memory once per block (grids up to kInterpSmemGrid bytes, d <= 2, FP32):
// for many unsorted targets the W^d reads per target then hit shared memory
// instead of one L1 line per lane per row.  One persistent block per SM.
constexpr int kInterpSmemThreads = 1024;
constexpr size_t kInterpSmemGrid = 200 * 1024;
constexpr long long kInterpSmemMinTargets = 1ll << 22;

template <int D, int W, typename TC, typename TV>
__global__ void __launch_bounds__(kInterpSmemThreads, 1)
    interp_smem_kernel(const TC* __restrict__ z, int soa, long long q, GridScale gs, int off, int nE,
                       const float* __restrict__ E2, EsCoef<float> cf, TV* __restrict__ mu, int* range_flag) {
  extern __shared__ __align__(16) float sgrid[];
  const long long total = D == 1 ? (long long)nE : (long long)nE * nE;
  long long done = 0;
  if ((reinterpret_cast<uintptr_t>(E2) & 15) == 0) {
    const long long n4 = total / 4;
    for (long long i = threadIdx.x; i < n4; i += blockDim.x)
      reinterpret_cast<float4*>(sgrid)[i] = __ldg(reinterpret_cast<const float4*>(E2) + i);
    done = n4 * 4;
  }
  for (long long i = done + threadIdx.x; i < total; i += blockDim.x) sgrid[i] = __ldg(E2 + i);
  __syncthreads();
  bool bad = false;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < q; i += (long long)gridDim.x * blockDim.x) {
    float wt[D][W];
    int e0[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      TC za = soa ? z[(long long)a * q + i] : z[i * D + a];
      if (!(za >= TC(0) && za <= TC(1))) {
        bad = true;
        za = TC(0);
      }
      int l0;
      float f;
      GridPos<TC, float>::get(za, gs, l0, f);
      int e = l0 + off;
      e = max(0, min(e, nE - W));
      e0[a] = e;
      es_weights_x2<W>(f, cf, wt[a]);
    }
    float acc = 0.f;
    if (D == 1) {
#pragma unroll
      for (int u = 0; u < W; ++u) acc = fmaf(wt[0][u], sgrid[e0[0] + u], acc);
    } else {
#pragma unroll
      for (int u = 0; u < W; ++u) {
        const float* row = sgrid + (e0[0] + u) * nE + e0[D - 1];
        float s = 0.f;
#pragma unroll
        for (int v = 0; v < W; ++v) s = fmaf(wt[D - 1][v], row[v], s);
        acc = fmaf(wt[0][u], s, acc);
      }
    }
    mu[i] = (TV)acc;
  }
  if (bad) atomicOr(range_flag, 1);
}

static int grid_for(long long n, int threads, int cap = 4096) {
  long long b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

cudaError_t launch_precorrect(const double2* beta, const double* Dw, const double* corr2, int m, int d, int nf,
                              void* g, int g_f64, cudaStream_t s) {
  long long total = 2 * m + 1;
  for (int a = 1; a < d; ++a) total *= 2 * m + 1;
  const int blocks = grid_for(total, 256);
#define EFGP_PC(DD)                                                                                               \
  if (d == DD) {                                                                                                  \
    if (g_f64) precorrect_kernel<DD, double><<<blocks, 256, 0, s>>>(beta, Dw, corr2, m, nf,                      \
                                                                    reinterpret_cast<double2*>(g));               \
    else precorrect_kernel<DD, float><<<blocks, 256, 0, s>>>(beta, Dw, corr2, m, nf, reinterpret_cast<float2*>(g)); \
    return cudaGetLastError();                                                                                    \
  }
  EFGP_PC(1) EFGP_PC(2) EFGP_PC(3)
#undef EFGP_PC
  return cudaErrorInvalidValue;
}

cudaError_t launch_unfold(const void* g, int g_f64, int nf, int d, int off, int nE, void* E2, cudaStream_t s) {
  long long total = nE;
  for (int a = 1; a < d; ++a) total *= nE;
  const int blocks = grid_for(total, 256);
#define EFGP_UF(DD)                                                                                        \
  if (d == DD) {                                                                                           \
    if (g_f64) unfold_kernel<DD, double><<<blocks, 256, 0, s>>>(reinterpret_cast<const double2*>(g), nf, off, nE, \
                                                                reinterpret_cast<double*>(E2));            \
    else unfold_kernel<DD, float><<<blocks, 256, 0, s>>>(reinterpret_cast<const float2*>(g), nf, off, nE,   \
                                                         reinterpret_cast<float*>(E2));                    \
    return cudaGetLastError();                                                                             \
  }
  EFGP_UF(1) EFGP_UF(2) EFGP_UF(3)
#undef EFGP_UF
  return cudaErrorInvalidValue;
}

template <int D, int W, typename TC, typename TV, typename TR>
static cudaError_t interp_dw(const void* z, int soa, long long q, const GridScale& gs, int off, int nE, const void* E2,
                             const void* coef, void* mu, int* flag, cudaStream_t s) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if constexpr (sizeof(TR) == 4 && D <= 2) {
    const size_t bytes = sizeof(float) * (D == 1 ? (size_t)nE : (size_t)nE * nE);
    if (q >= kInterpSmemMinTargets && bytes <= kInterpSmemGrid) {
      auto k = interp_smem_kernel<D, W, TC, TV>;
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
      if (e != cudaSuccess) return e;
      const int blocks = (int)std::min<long long>(nsm, (q + kInterpSmemThreads - 1) / kInterpSmemThreads);
      k<<<blocks, kInterpSmemThreads, bytes, s>>>(reinterpret_cast<const TC*>(z), soa, q, gs, off, nE,
                                                  reinterpret_cast<const float*>(E2),
                                                  *reinterpret_cast<const EsCoef<float>*>(coef),
                                                  reinterpret_cast<TV*>(mu), flag);
      return cudaGetLastError();
    }
  }
  const int blocks = grid_for(q, 256, nsm * 16);
  interp_kernel<D, W, TC, TV, TR><<<blocks, 256, 0, s>>>(reinterpret_cast<const TC*>(z), soa, q, gs, off, nE,
                                                         reinterpret_cast<const TR*>(E2),
                                                         *reinterpret_cast<const EsCoef<TR>*>(coef),
                                                         reinterpret_cast<TV*>(mu), flag);
  return cudaGetLastError();
}

template <int D, typename TC, typename TV, typename TR>
static cudaError_t interp_d(int W, const void* z, int soa, long long q, const GridScale& gs, int off, int nE,
                            const void* E2, const void* coef, void* mu, int* flag, cudaStream_t s) {
  switch (W) {
    case 3: return interp_dw<D, 3, TC, TV, TR>(z, soa, q, gs, off, nE, E2, coef, mu, flag, s);
    case 4: return interp_dw<D, 4, TC, TV, TR>(z, soa, q, gs, off, nE, E2, coef, mu, flag, s);
    case 5: return interp_dw<D, 5, TC, TV, TR>(z, soa, q, gs, off, nE, E2, coef, mu, flag, s);
    case 6: return interp_dw<D, 6, TC, TV, TR>(z, soa, q, gs, off, nE, E2, coef, mu, flag, s);
    case 7: return interp_dw<D, 7, TC, TV, TR>(z, soa, q, gs, off, nE, E2, coef, mu, flag, s);
    case 8: return interp_dw<D, 8, TC, TV, TR>(z, soa, q, gs, off, nE, E2, coef, mu, flag, s);
    case 10: return interp_dw<D, 10, TC, TV, TR>(z, soa, q, gs, off, nE, E2, coef, mu, flag, s);
    case 12: return interp_dw<D, 12, TC, TV, TR>(z, soa, q, gs, off, nE, E2, coef, mu, flag, s);
    case 14: return interp_dw<D, 14, TC, TV, TR>(z, soa, q, gs, off, nE, E2, coef, mu, flag, s);
    case 16: return interp_dw<D, 16, TC, TV, TR>(z, soa, q, gs, off, nE, E2, coef, mu, flag, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_interp(const void* targets, int coord_f64, int soa, long long q, int d, int W, const GridScale& gs,
                          int off, int nE, const void* E2, int g_f64, const void* coef, void* mu, int value_f64,
                          int* range_flag, cudaStream_t s) {
  if (q == 0) return cudaSuccess;
  // coordinate and value dtypes follow the inputs; the grid precision
  // follows the handle (FP32 mixed, FP64 plain)
#define EFGP_I(DD, TC, TV, TR) return interp_d<DD, TC, TV, TR>(W, targets, soa, q, gs, off, nE, E2, coef, mu, range_flag, s);
#define EFGP_ID(DD)                                                     \
  if (d == DD) {                                                        \
    if (g_f64) {                                                        \
      if (coord_f64 && value_f64) { EFGP_I(DD, double, double, double) } \
      if (coord_f64) { EFGP_I(DD, double, float, double) }              \
      if (value_f64) { EFGP_I(DD, float, double, double) }              \
      EFGP_I(DD, float, float, double)                                  \
    } else {                                                            \
      if (coord_f64 && value_f64) { EFGP_I(DD, double, double, float) } \
      if (coord_f64) { EFGP_I(DD, double, float, float) }               \
      if (value_f64) { EFGP_I(DD, float, double, float) }               \
      EFGP_I(DD, float, float, float)                                   \
    }                                                                   \
  }
  EFGP_ID(1) EFGP_ID(2) EFGP_ID(3)
#undef EFGP_ID
#undef EFGP_I
  return cudaErrorInvalidValue;
}

}  // namespace efgp
