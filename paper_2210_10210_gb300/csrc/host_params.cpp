// Host-side planning for EFGP: kernels and spectral densities, the (h, m)
// choice of Sec. 4.2, FFT sizes, and the exponential-of-semicircle (ES)
// nonuniform-FFT plans (kernel width, shape, piecewise polynomial form and
// deconvolution factors).  Everything here is FP64 and runs without a GPU.
#include <algorithm>
#include <cmath>
#include <complex>
#include <limits>
#include <mutex>
#include <vector>

#include "efgp_internal.h"

namespace efgp {

static const double kPi = 3.14159265358979323846264338327950288;

// ---------------------------------------------------------------------------
// Gauss-Legendre nodes and weights on [-1, 1] (Newton on the Legendre
// three-term recurrence).
// ---------------------------------------------------------------------------
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double pn = (n == 1) ? z : p1;
      double pnm1 = (n == 1) ? 1.0 : p0;
      dp = n * (z * pn - pnm1) / (z * z - 1.0);
      double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    // recompute derivative at the converged node
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    double pn = (n == 1) ? z : p1;
    double pnm1 = (n == 1) ? 1.0 : p0;
    dp = n * (z * pn - pnm1) / (z * z - 1.0);
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// ---------------------------------------------------------------------------
// Kernels (eqs. Gker, Cker) and their spectral densities under the Fourier
// convention khat(xi) = int k(x) exp(-2 pi i xi.x) dx (Sec. 3.1).  The
// densities are the standard closed forms; the paper defines only k.
// ---------------------------------------------------------------------------
static bool near(double a, double b) { return std::fabs(a - b) < 1e-12; }

double kernel_value(const efgp_kernel& k, double r) {
  const double var = k.variance > 0 ? k.variance : 1.0;
  const double ell = k.lengthscale;
  r = std::fabs(r);
  if (k.family == EFGP_KERNEL_SE) return var * std::exp(-r * r / (2.0 * ell * ell));
  const double nu = k.nu;
  const double s = std::sqrt(2.0 * nu) * r / ell;
  if (s == 0.0) return var;
  if (near(nu, 0.5)) return var * std::exp(-s);
  if (near(nu, 1.5)) return var * (1.0 + s) * std::exp(-s);
  if (near(nu, 2.5)) return var * (1.0 + s + s * s / 3.0) * std::exp(-s);
  return var * std::pow(2.0, 1.0 - nu) / std::tgamma(nu) * std::pow(s, nu) * std::cyl_bessel_k(nu, s);
}

double kernel_spectral_density(const efgp_kernel& k, int d, double xi) {
  const double var = k.variance > 0 ? k.variance : 1.0;
  const double ell = k.lengthscale;
  if (k.family == EFGP_KERNEL_SE)
    return var * std::pow(2.0 * kPi * ell * ell, 0.5 * d) * std::exp(-2.0 * kPi * kPi * ell * ell * xi * xi);
  const double nu = k.nu;
  const double c = std::pow(2.0, d) * std::pow(kPi, 0.5 * d) * std::tgamma(nu + 0.5 * d) *
                   std::pow(2.0 * nu, nu) / (std::tgamma(nu) * std::pow(ell, 2.0 * nu));
  return var * c * std::pow(2.0 * nu / (ell * ell) + 4.0 * kPi * kPi * xi * xi, -(nu + 0.5 * d));
}

// ||k||_{L2[-1,1]^d}: the integrand is even in each coordinate, so integrate
// over [0,1]^d with composite Gauss-Legendre panels graded toward 0.
double kernel_l2_norm_cube(const efgp_kernel& kin, int d) {
  efgp_kernel k = kin;
  k.variance = 1.0;
  const int npan = d < 3 ? 48 : 24, order = d < 3 ? 24 : 12;
  std::vector<double> xg, wg;
  gauss_legendre(order, xg, wg);
  std::vector<double> x, w;
  double a = 0.0;
  for (int p = 0; p < npan; ++p) {
    // geometric edges 1e-7 .. 1
    double b = std::pow(10.0, -7.0 + 7.0 * p / (npan - 1));
    for (int i = 0; i < order; ++i) {
      x.push_back(0.5 * (b - a) * xg[i] + 0.5 * (a + b));
      w.push_back(0.5 * (b - a) * wg[i]);
    }
    a = b;
  }
  const size_t n = x.size();
  double s = 0.0;
  if (d == 1) {
    for (size_t i = 0; i < n; ++i) {
      double v = kernel_value(k, x[i]);
      s += w[i] * v * v;
    }
  } else if (d == 2) {
    for (size_t i = 0; i < n; ++i)
      for (size_t j = 0; j < n; ++j) {
        double v = kernel_value(k, std::sqrt(x[i] * x[i] + x[j] * x[j]));
        s += w[i] * w[j] * v * v;
      }
  } else {
    for (size_t i = 0; i < n; ++i)
      for (size_t j = 0; j < n; ++j) {
        double r2 = x[i] * x[i] + x[j] * x[j];
        double acc = 0.0;
        for (size_t l = 0; l < n; ++l) {
          double v = kernel_value(k, std::sqrt(r2 + x[l] * x[l]));
          acc += w[l] * v * v;
        }
        s += w[i] * w[j] * acc;
      }
  }
  return std::sqrt(std::pow(2.0, d) * s);
}

// Sec. 4.2.  Natural logarithms.
double choose_h_m(const efgp_kernel& k, int d, double eps, double* h_out, int* m_out) {
  const double ell = k.lengthscale;
  if (k.family == EFGP_KERNEL_SE) {
    double h = 1.0 / (1.0 + ell * std::sqrt(2.0 * std::log(4.0 * d * std::pow(3.0, d) / eps)));
    double m = std::ceil(std::sqrt(0.5 * std::log(std::pow(4.0, d + 1) * d / eps)) / (kPi * ell * h));
    *h_out = h;
    *m_out = (int)m;
    return 0.0;
  }
  const double nu = k.nu;
  if (nu <= 2.5) {
    // L2 heuristic, eq. maternheur, with eps~ = eps ||k||_{L2[-1,1]^d}
    double l2 = kernel_l2_norm_cube(k, d);
    double et = eps * l2;
    double h = 1.0 / (1.0 + 0.85 * (ell / std::sqrt(nu)) * std::log(1.0 / et));
    double m = std::ceil((1.0 / h) * std::pow(std::pow(kPi, nu + 0.5 * d) * std::pow(ell, 2.0 * nu) * et / 0.15,
                                              -1.0 / (2.0 * nu + 0.5 * d)));
    *h_out = h;
    *m_out = (int)m;
    return l2;
  }
  // uniform bound, eq. maternhm
  double h = 1.0 / (1.0 + ell * std::sqrt(2.0 * d / nu) * std::log(d * std::pow(3.0, d) / eps));
  double m = std::ceil(std::pow(d * std::pow(5.0, d - 1) / (std::pow(kPi, 0.5 * d) * eps), 1.0 / (2.0 * nu)) * 1.6 *
                       std::sqrt(nu) / (kPi * h * ell));
  *h_out = h;
  *m_out = (int)m;
  return 0.0;
}

int next_smooth(int n) {
  if (n < 1) n = 1;
  for (int c = n;; ++c) {
    int v = c;
    for (int p : {2, 3, 5, 7})
      while (v % p == 0) v /= p;
    if (v == 1) return c;
  }
}

int factor_radices(int n, int* radices) {
  int cnt = 0;
  int v = n;
  for (int r : {8, 7, 5, 4, 3, 2}) {
    while (v % r == 0 && cnt < kMaxRadixPasses) {
      radices[cnt++] = r;
      v /= r;
    }
  }
  return v == 1 ? cnt : 0;
}

// ---------------------------------------------------------------------------
// Exponential-of-semicircle kernel and the NUFFT plan.
//
// A point at fine-grid coordinate u is spread onto the w grid points
// l0..l0+w-1 with l0 = ceil(u - w/2); with f = l0 - (u - w/2) in [0,1) the
// weight of point l0+j is psi((j + f - w/2)/(w/2)).  Each piece j is
// replaced by a polynomial P_j(t) in t = 2f - 1 (Chebyshev interpolation,
// evaluated by Horner on the device).  Spreading, an FFT of the fine grid
// and division by the kernel's Fourier transform give the modes
// sum_n c_n exp(-i k 2 pi u_n / nf) (the standard type-1 NUFFT).
// ---------------------------------------------------------------------------
double es_kernel(double z, double beta) {
  if (std::fabs(z) > 1.0) return 0.0;
  return std::exp(beta * (std::sqrt(std::max(0.0, 1.0 - z * z)) - 1.0));
}

// 2 int_0^1 psi(z) cos(omega z) dz, with z = sin(theta) to remove the
// square-root endpoint behaviour.
static double es_ft(double omega, double beta, const std::vector<double>& qx, const std::vector<double>& qw) {
  double s = 0.0;
  for (size_t i = 0; i < qx.size(); ++i) {
    double th = 0.25 * kPi * (qx[i] + 1.0);  // [0, pi/2]
    double z = std::sin(th), c = std::cos(th);
    s += qw[i] * std::exp(beta * (c - 1.0)) * std::cos(omega * z) * c;
  }
  return 2.0 * 0.25 * kPi * s;
}

static bool solve_dense(std::vector<double>& A, std::vector<double>& b, int n) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0.0) return false;
    if (piv != c) {
      for (int k = 0; k < n; ++k) std::swap(A[c * n + k], A[piv * n + k]);
      std::swap(b[c], b[piv]);
    }
    for (int r = c + 1; r < n; ++r) {
      double f = A[r * n + c] / A[c * n + c];
      for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
      b[r] -= f * b[c];
    }
  }
  for (int c = n - 1; c >= 0; --c) {
    double s = b[c];
    for (int k = c + 1; k < n; ++k) s -= A[c * n + k] * b[k];
    b[c] = s / A[c * n + c];
  }
  return true;
}

// Fit all w pieces with degree deg; returns max abs error on a fine sample.
static double fit_pieces(int w, double beta, int deg, std::vector<double>& coef) {
  const int np = deg + 1;
  coef.assign((size_t)np * w, 0.0);
  std::vector<double> nodes(np);
  for (int i = 0; i < np; ++i) nodes[i] = std::cos(kPi * (i + 0.5) / np);
  double err = 0.0;
  // psi is even, so piece w-1-j at t is piece j at -t: the first half of the
  // pieces is fitted, the rest mirrored (coefficient k times (-1)^k), and the
  // odd coefficients of a middle piece are zero -- exactly, so that the device
  // may evaluate the pieces pairwise from their even and odd parts.
  for (int j = 0; j < (w + 1) / 2; ++j) {
    std::vector<double> A((size_t)np * np), b(np);
    for (int i = 0; i < np; ++i) {
      double t = nodes[i], tp = 1.0;
      for (int k = 0; k < np; ++k) {
        A[i * np + k] = tp;
        tp *= t;
      }
      double f = 0.5 * (t + 1.0);
      b[i] = es_kernel((j + f - 0.5 * w) / (0.5 * w), beta);
    }
    solve_dense(A, b, np);
    const int jm = w - 1 - j;
    if (jm == j)
      for (int k = 1; k < np; k += 2) b[k] = 0.0;
    for (int k = 0; k < np; ++k) {
      coef[(size_t)k * w + j] = b[k];
      coef[(size_t)k * w + jm] = (k & 1) ? -b[k] : b[k];
    }
  }
  for (int j = 0; j < w; ++j) {
    for (int s = 0; s <= 400; ++s) {
      double t = -1.0 + 2.0 * s / 400.0;
      double p = 0.0;
      for (int k = np - 1; k >= 0; --k) p = p * t + coef[(size_t)k * w + j];
      double f = 0.5 * (t + 1.0);
      err = std::max(err, std::fabs(p - es_kernel((j + f - 0.5 * w) / (0.5 * w), beta)));
    }
  }
  return err;
}

// Worst relative error over sample modes and sub-cell offsets of spreading
// one unit point with the polynomial weights and deconvolving.
static double point_error(int nf, int K, int w, const std::vector<double>& corr, const std::vector<double>& coef,
                          int deg) {
  std::vector<int> ks;
  if (2 * K + 1 <= 129) {
    for (int k = -K; k <= K; ++k) ks.push_back(k);
  } else {
    for (int i = 0; i <= 128; ++i) ks.push_back(-K + (int)std::llround((2.0 * K) * i / 128.0));
  }
  double err = 0.0;
  for (int s = 0; s < 16; ++s) {
    double f = (s + 0.37) / 16.0;  // sub-cell offset
    double t = 2.0 * f - 1.0;
    double wt[kMaxWidth];
    for (int j = 0; j < w; ++j) {
      double p = 0.0;
      for (int k = deg; k >= 0; --k) p = p * t + coef[(size_t)k * w + j];
      wt[j] = p;
    }
    for (int k : ks) {
      std::complex<double> acc(0.0, 0.0);
      for (int j = 0; j < w; ++j) {
        // grid point l0+j sits at offset (j + f - w/2) from the point
        double ph = -2.0 * kPi * k * (j + f - 0.5 * w) / nf;
        acc += wt[j] * std::complex<double>(std::cos(ph), std::sin(ph));
      }
      acc *= corr[k + K];
      err = std::max(err, std::abs(acc - 1.0));
    }
  }
  return err;
}

int plan_nufft(int d, int K, double h, double tol, double cost_points, double upsamp_override, int width_override,
               NufftPlan* out) {
  std::vector<double> qx, qw;
  gauss_legendre(96, qx, qw);
  std::vector<double> sigmas = {1.5, 2.0, 2.5, 3.0, 4.0};
  if (upsamp_override > 0) sigmas = {upsamp_override};
  double best = std::numeric_limits<double>::infinity();
  bool found = false;
  NufftPlan bestp;
  for (double sg : sigmas) {
    int nf = next_smooth(std::max((int)std::ceil(sg * (2 * K + 1)), 2 * kMaxWidth));
    double sig_eff = (double)nf / (2 * K + 1);
    for (int w : kWidths) {
      if (width_override > 0 && w < width_override) continue;
      if (w > nf / 2) continue;
      double beta = 0.97 * kPi * w * (1.0 - 1.0 / (2.0 * sig_eff));
      // polynomial degree fixed per width (see es_degree)
      std::vector<double> cbest;
      const int dbest = es_degree(w);
      fit_pieces(w, beta, dbest, cbest);
      std::vector<double> corr(2 * K + 1);
      for (int k = -K; k <= K; ++k) corr[k + K] = 1.0 / (0.5 * w * es_ft(kPi * w * k / (double)nf, beta, qx, qw));
      double err = point_error(nf, K, w, corr, cbest, dbest);
      bool ok = err <= tol || (width_override > 0);
      if (!ok) continue;
      double fft = 10.0 * std::pow((double)nf, d) * std::log2(std::pow((double)nf, d));
      double cost = cost_points * (d * w * (dbest + 1) + 2.0 * std::pow((double)w, d)) + fft;
      if (cost < best) {
        best = cost;
        found = true;
        bestp.K = K;
        bestp.nf = nf;
        bestp.w = w;
        bestp.beta = beta;
        bestp.upsamp = sig_eff;
        bestp.deg = dbest;
        bestp.err = err;
        bestp.coef = cbest;
        bestp.corr = corr;
      }
      break;  // wider kernels at this upsampling only cost more
    }
  }
  if (!found) return EFGP_EUNSUPPORTED;
  bestp.s = bestp.nf * h;
  bestp.off = (bestp.w + 1) / 2 + 1;
  bestp.nE = (int)std::ceil(bestp.s) + bestp.w + 4;
  *out = bestp;
  return EFGP_OK;
}

}  // namespace efgp
