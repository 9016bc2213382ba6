// Internal declarations shared by the translation units of libefgp.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/efgp.h"

#ifdef __CUDACC__
#include <cuda_runtime.h>
#endif

namespace efgp {

// ---------------------------------------------------------------------------
// Compile-time limits of the library.
// ---------------------------------------------------------------------------
constexpr int kMaxWidth = 16;   // largest ES kernel width (grid points per dim)
constexpr int kMaxDeg = 20;     // largest degree of the piecewise ES polynomial
constexpr int kMaxRadixPasses = 16;
// ES widths with compiled spread/interp kernels; a requested width is rounded
// up to the next one (a wider kernel is only more accurate).
constexpr int kWidths[] = {3, 4, 5, 6, 7, 8, 10, 12, 14, 16};
// Degree of the polynomial that replaces each piece of the ES kernel: fixed
// per width so device code evaluates it fully unrolled with the coefficients
// as constant operands (W+2 is at the accuracy plateau of the fit for the
// upsampling factors used, set by the kernel's square-root edge).
constexpr int es_degree(int w) { return w + 2; }
// coefficient rows are padded to an even length, so that the pair of pieces
// (2j, 2j+1) of every degree is one aligned 8-byte operand
constexpr int es_stride(int w) { return w + (w & 1); }
// Edge (fine-grid cells) of the spread tiles by which points are binned; the
// register spread kernel gives one thread per cell of a 256-cell tile.
constexpr int tile_edge(int d) { return d == 1 ? 256 : (d == 2 ? 16 : 8); }

void set_error(const std::string& msg);
void clear_error();
bool error_empty();

// ---------------------------------------------------------------------------
// Host-side planning (host_params.cpp).  All FP64.
// ---------------------------------------------------------------------------
double kernel_value(const efgp_kernel& k, double r);
double kernel_spectral_density(const efgp_kernel& k, int d, double xi);
double kernel_l2_norm_cube(const efgp_kernel& k, int d);
// (h, m) of Sec. 4.2; returns the L2 norm used (0 for SE)
double choose_h_m(const efgp_kernel& k, int d, double eps, double* h, int* m);
int next_smooth(int n);            // smallest 2^a 3^b 5^c 7^e >= n
int factor_radices(int n, int* radices);  // radices from {8,7,5,4,3,2}; returns count (0 if not smooth)
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);

// One nonuniform FFT plan: fine grid, ES kernel and its polynomial form.
struct NufftPlan {
  int K = 0;          // modes -K..K per dim are produced / consumed
  int nf = 0;         // fine grid per dim
  int w = 0;          // ES width
  double beta = 0;    // ES shape
  double upsamp = 0;  // nf / (2K+1)
  int deg = 0;        // polynomial degree
  double err = 0;     // estimated sup-norm relative error
  double s = 0;       // nf * h : fine-grid coordinate of x = 1
  int off = 0;        // extended-grid offset (extended index = footprint start + off)
  int nE = 0;         // extended grid per dim
  std::vector<double> coef;   // (deg+1) x w, coefficient k of piece j at [k*w + j]
  std::vector<double> corr;   // 2K+1 per-dim deconvolution factors, index k+K
};

// Plans the NUFFT producing modes -K..K from points scaled by h, to
// relative accuracy tol.  cost_points weights the spreading cost.
int plan_nufft(int d, int K, double h, double tol, double cost_points,
               double upsamp_override, int width_override, NufftPlan* out);

// ES kernel exp(beta(sqrt(1-z^2)-1)) on |z|<=1
double es_kernel(double z, double beta);

// ---------------------------------------------------------------------------
// Device-side parameter blocks passed by value to kernels.
// ---------------------------------------------------------------------------
constexpr int es_pairs(int w) { return es_degree(w) / 2 + 1; }   // (even, odd) coefficient pairs per piece
template <typename T>
struct alignas(16) EsCoef {
  T c[(kMaxDeg + 1) * kMaxWidth];  // coefficient k of piece j at c[k*es_stride(W) + j]
  // pieces j < (W+1)/2 as pairs (c_{j,2i}, c_{j,2i+1}) at sp[2*(j*es_pairs(W) + i)]:
  // piece j is E_j(t^2) + t O_j(t^2) and piece W-1-j is E_j(t^2) - t O_j(t^2)
  T sp[2 * (kMaxWidth / 2) * (kMaxDeg / 2 + 1)];
  int deg;
};

struct CgState {
  double rr;          // r^H r
  double rz;          // r^H M^-1 r (= rr without a preconditioner)
  double rr_new;
  double pAp;
  double alpha;
  double beta;
  double bnorm2;      // ||b||^2
  double tol2;        // rho^2 ||b||^2
  long long iter;
  long long max_iter;
  int done;           // 0 running, 1 converged, 2 iteration cap, 3 breakdown
  unsigned int ticket_a;   // last-block tickets of the two reductions
  unsigned int ticket_b;
  int pad;
};

// Line FFT descriptor: lines (o, i), o < outer, i < inner; element k of line
// (o,i) at base + o*s_o + k*s_k + i*s_i (element units).
struct LineGeom {
  long long outer, inner;
  long long in_so, in_sk, in_si;
  long long out_so, out_sk, out_si;
  int L;        // transform length
  int n_in;     // input entries present (rest are zero)
  int n_out;    // output entries written (the first n_out)
  int nb;       // lines per block
  int npass;
  int radix[kMaxRadixPasses];
};

}  // namespace efgp
