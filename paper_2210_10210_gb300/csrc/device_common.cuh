// Device helpers shared by the CUDA translation units of libefgp.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "efgp_internal.h"

namespace efgp {

// ---------------------------------------------------------------- complex
template <typename T> struct CplxOf;
template <> struct CplxOf<float> { using type = float2; };
template <> struct CplxOf<double> { using type = double2; };
template <typename T> using cplx = typename CplxOf<T>::type;

template <typename T>
__host__ __device__ __forceinline__ cplx<T> mk(T re, T im) {
  cplx<T> c;
  c.x = re;
  c.y = im;
  return c;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  C c;
  c.x = a.x * b.x - a.y * b.y;
  c.y = a.x * b.y + a.y * b.x;
  return c;
}
template <typename C, typename T> __device__ __forceinline__ C cscale(C a, T s) { a.x *= s; a.y *= s; return a; }
// multiply by s*i (s = +1 or -1)
template <typename C> __device__ __forceinline__ C cmul_si(C a, int s) {
  C c;
  if (s > 0) { c.x = -a.y; c.y = a.x; } else { c.x = a.y; c.y = -a.x; }
  return c;
}

// ---------------------------------------------------------------- ES kernel
// Weights of the W grid points l0..l0+W-1 for sub-cell offset f in [0,1]:
// piece j is a polynomial P_j in t = 2f-1.  psi is even, so P_{W-1-j}(t) =
// P_j(-t): with P_j(t) = E_j(t^2) + t O_j(t^2) one Horner pass in t^2 over the
// coefficient pairs gives both pieces of a pair (the host fit is exactly
// mirror-symmetric).
template <typename T, int W>
__device__ __forceinline__ void es_weights(T f, const EsCoef<T>& cf, T (&wt)[W]) {
  constexpr int NPR = es_pairs(W);
  const T t = T(2) * f - T(1);
  const T s = t * t;
#pragma unroll
  for (int j = 0; j < (W + 1) / 2; ++j) {
    const T* c = cf.sp + 2 * j * NPR;
    T e = c[2 * (NPR - 1)], o = c[2 * (NPR - 1) + 1];
#pragma unroll
    for (int i = NPR - 2; i >= 0; --i) {
      e = fma(e, s, c[2 * i]);
      o = fma(o, s, c[2 * i + 1]);
    }
    if (2 * j == W - 1) {
      wt[j] = e;
    } else {
      wt[j] = fma(t, o, e);
      wt[W - 1 - j] = fma(-t, o, e);
    }
  }
}

// The same weights with each (even, odd) Horner pair and each mirrored pair
// of pieces computed by packed two-lane FP32 FMAs.
template <int W>
__device__ __forceinline__ void es_weights_x2(float f, const EsCoef<float>& cf, float (&wt)[W]) {
  constexpr int NPR = es_pairs(W);
  const float t = 2.f * f - 1.f;
  const float s = t * t;
  const float2 ss = make_float2(s, s), tm = make_float2(t, -t);
  const float2* c2 = reinterpret_cast<const float2*>(cf.sp);
#pragma unroll
  for (int j = 0; j < (W + 1) / 2; ++j) {
    float2 eo = c2[j * NPR + NPR - 1];
#pragma unroll
    for (int i = NPR - 2; i >= 0; --i) eo = __ffma2_rn(eo, ss, c2[j * NPR + i]);
    if (2 * j == W - 1) {
      wt[j] = eo.x;
    } else {
      const float2 r = __ffma2_rn(tm, make_float2(eo.y, eo.y), make_float2(eo.x, eo.x));
      wt[j] = r.x;
      wt[W - 1 - j] = r.y;
    }
  }
}

// Fine-grid position of a coordinate x in [0,1]: u = x * s, footprint start
// l0 = ceil(u - W/2), offset f = l0 - (u - W/2) in [0,1).
struct GridScale {
  double s;        // nf * h
  float s_hi, s_lo;  // s split so that s_hi + s_lo carries ~48 bits
  float halfw_f;
  double halfw_d;
};

__device__ __forceinline__ void grid_pos_f(float x, const GridScale& g, int& l0, float& f) {
  // u = x*s evaluated as a + lo with a = fl(x*s_hi) and lo the product's
  // rounding error plus x*s_lo, so f keeps ~1e-7 cell accuracy even for
  // fine grids of thousands of cells.
  // (explicitly rounded operations: no call site may contract them into a
  // different FMA, so every kernel that bins a point computes the same cell)
  const float a = __fmul_rn(x, g.s_hi);
  const float r = fmaf(x, g.s_hi, -a);
  const float lo = fmaf(x, g.s_lo, r);
  const float v = __fsub_rn(a, g.halfw_f);
  float l = ceilf(__fadd_rn(v, lo));
  float ff = __fsub_rn(__fsub_rn(l, v), lo);
  if (ff < 0.f) { l += 1.f; ff += 1.f; }
  else if (ff >= 1.f) { l -= 1.f; ff -= 1.f; }
  l0 = (int)l;
  f = ff;
}
__device__ __forceinline__ void grid_pos_d(double x, const GridScale& g, int& l0, double& f) {
  const double v = x * g.s - g.halfw_d;
  const double l = ceil(v);
  l0 = (int)l;
  f = l - v;
}
template <typename TC, typename TR> struct GridPos;
template <> struct GridPos<float, float> {
  static __device__ __forceinline__ void get(float x, const GridScale& g, int& l0, float& f) { grid_pos_f(x, g, l0, f); }
};
template <> struct GridPos<double, float> {
  static __device__ __forceinline__ void get(double x, const GridScale& g, int& l0, float& f) {
    double fd;
    grid_pos_d(x, g, l0, fd);
    f = (float)fd;
  }
};
template <typename TC> struct GridPos<TC, double> {
  static __device__ __forceinline__ void get(TC x, const GridScale& g, int& l0, double& f) {
    grid_pos_d((double)x, g, l0, f);
  }
};

// ---------------------------------------------------------------- launch order
// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may start while its predecessor is still running; it must
// wait here before touching anything the predecessor writes.  Without the
// launch attribute this returns at once.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ---------------------------------------------------------------- reductions
// Sum of v over the block (blockDim.x a multiple of 32, <= 1024).  Result
// valid in thread 0.  Uses 32 doubles of shared scratch.
__device__ __forceinline__ double block_sum(double v, double* scratch) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? scratch[threadIdx.x] : 0.0;
  if (wid == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;
}

// Deterministic sum of n partials by one block (fixed order for fixed n).
__device__ __forceinline__ double block_sum_partials(const double* partials, int n, double* scratch) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += __ldcg(partials + i);
  return block_sum(v, scratch);
}

}  // namespace efgp
