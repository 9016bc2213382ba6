"""FP64 CPU oracle for equispaced-Fourier GP regression (EFGP).

TEST INFRASTRUCTURE, NOT PART OF THE LIBRARY.  Only the test suite,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this module.  It shares no code with the CUDA path: it never touches a
nonuniform FFT, an FFT or an iterative solver.  Every quantity is the plain
definition written out in float64:

* the kernel k and its spectral density k-hat            (eqs. Gker, Cker; Sec. 3.1 convention)
* the grid spacing h and half-width m                    (Sec. 4.2, eq. maternheur, eq. maternhm)
* spectral weights D_j = sqrt(h^d khat(h j))             (eq. 117)
* Toeplitz generating vector by direct sums              (eq. 88, sign reading below)
* right-hand side Phi^* y by direct sums                 (eq. rhs)
* dense system matrix D (F^*F) D + sigma^2 I             (eqs. 97, 223)
* its solution by a Cholesky factorisation              (eq. be; Lemma 1)
* the posterior mean as a direct Fourier sum             (eq. muws)

Sign reading (the paper prints +i in both eq. 88 and eq. 205, which would not
make eq. 223 equal to F^*F): F_{nj} = exp(+2 pi i h j.x_n), so the Toeplitz
entries are w_k = sum_n exp(-2 pi i h k.x_n) (the complex conjugate of the
printed v) and (F^* y)_j = sum_n y_n exp(-2 pi i h j.x_n).  The posterior mean
uses exp(+2 pi i h j.z).  Because khat is even, the mirror labelling j -> -j
gives the same real mean.

Matrix products (BLAS) serve only to evaluate the separable direct sums
sum_n prod_l e^{..x_n^(l)} and dense products; no blocking or reordering of
the method's own steps is done.

Parity pins for every function live in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy import linalg, special

# ----------------------------------------------------------------------------
# Kernels (eq. Gker, eq. Cker) and spectral densities (Fourier convention of
# Sec. 3.1: khat(xi) = int k(x) exp(-2 pi i xi.x) dx).  The densities are the
# textbook closed forms of the cited GP reference; the paper prints only k.
# ----------------------------------------------------------------------------


def k_se(r, ell):
    """Squared-exponential kernel exp(-r^2 / (2 ell^2)) (eq. Gker)."""
    r = np.asarray(r, dtype=np.float64)
    return np.exp(-(r * r) / (2.0 * ell * ell))


def k_matern(r, nu, ell):
    """Matern kernel (eq. Cker), value 1 at r = 0."""
    r = np.abs(np.asarray(r, dtype=np.float64))
    s = math.sqrt(2.0 * nu) * r / ell
    out = np.ones_like(s)
    nz = s > 0
    out[nz] = (2.0 ** (1.0 - nu) / math.gamma(nu)) * s[nz] ** nu * special.kv(nu, s[nz])
    return out


def khat_se(xi, ell, d):
    """Spectral density of the SE kernel at frequency magnitude |xi|."""
    xi = np.asarray(xi, dtype=np.float64)
    return (2.0 * math.pi * ell * ell) ** (d / 2.0) * np.exp(-2.0 * math.pi ** 2 * ell * ell * xi * xi)


def khat_matern(xi, nu, ell, d):
    """Spectral density of the Matern kernel at frequency magnitude |xi|."""
    xi = np.asarray(xi, dtype=np.float64)
    c = (2.0 ** d * math.pi ** (d / 2.0) * math.gamma(nu + d / 2.0) * (2.0 * nu) ** nu
         / (math.gamma(nu) * ell ** (2.0 * nu)))
    return c * (2.0 * nu / (ell * ell) + 4.0 * math.pi ** 2 * xi * xi) ** (-(nu + d / 2.0))


@dataclass(frozen=True)
class Kernel:
    family: str          # "se" | "matern"
    nu: float            # Matern smoothness (ignored for SE)
    ell: float           # length scale
    variance: float = 1.0

    def k(self, r):
        base = k_se(r, self.ell) if self.family == "se" else k_matern(r, self.nu, self.ell)
        return self.variance * base

    def khat(self, xi, d):
        base = khat_se(xi, self.ell, d) if self.family == "se" else khat_matern(xi, self.nu, self.ell, d)
        return self.variance * base


# ----------------------------------------------------------------------------
# ||k||_{L^2[-1,1]^d} (needed by eq. maternheur) by tensor Gauss-Legendre
# quadrature on [0,1]^d (the integrand is even in every coordinate), with
# panels graded geometrically toward the origin where the Matern-1/2 kernel
# has its kink.
# ----------------------------------------------------------------------------


def _panels(npan=48, order=24):
    xg, wg = np.polynomial.legendre.leggauss(order)
    edges = np.concatenate([[0.0], np.geomspace(1e-7, 1.0, npan)])
    xs, ws = [], []
    for a, b in zip(edges[:-1], edges[1:]):
        xs.append(0.5 * (b - a) * xg + 0.5 * (a + b))
        ws.append(0.5 * (b - a) * wg)
    return np.concatenate(xs), np.concatenate(ws)


def kernel_l2_norm_cube(kern: Kernel, d: int) -> float:
    x, w = _panels() if d < 3 else _panels(24, 12)
    if d == 1:
        s = np.sum(w * kern.k(x) ** 2)
    elif d == 2:
        r = np.sqrt(x[:, None] ** 2 + x[None, :] ** 2)
        s = np.sum(np.outer(w, w) * kern.k(r) ** 2)
    elif d == 3:
        s = 0.0
        ww = np.outer(w, w)
        r2 = x[:, None] ** 2 + x[None, :] ** 2
        for i in range(len(x)):
            s += w[i] * np.sum(ww * kern.k(np.sqrt(r2 + x[i] ** 2)) ** 2)
    else:
        raise ValueError("d must be 1, 2 or 3")
    return math.sqrt((2.0 ** d) * s)


# ----------------------------------------------------------------------------
# Parameter choice (Sec. 4.2).  Natural logarithms throughout.
# ----------------------------------------------------------------------------


def choose_h_m(kern: Kernel, d: int, eps: float):
    """Returns (h, m) for tolerance eps.

    SE: h = 1/(1 + ell sqrt(2 log(4 d 3^d / eps))),
        m = ceil( sqrt(log(4^{d+1} d / eps) / 2) / (pi ell h) ).
    Matern, 1/2 <= nu <= 5/2: the L2 heuristic eq. maternheur with
        eps~ = eps ||k||_{L2[-1,1]^d}.
    Matern, nu > 5/2: the uniform bound eq. maternhm (smallest h, m allowed).
    """
    ell = kern.ell
    if kern.family == "se":
        h = 1.0 / (1.0 + ell * math.sqrt(2.0 * math.log(4.0 * d * 3.0 ** d / eps)))
        m = math.ceil(math.sqrt(0.5 * math.log(4.0 ** (d + 1) * d / eps)) / (math.pi * ell * h))
        return h, int(m)
    nu = kern.nu
    if nu <= 2.5:
        et = eps * kernel_l2_norm_cube(Kernel(kern.family, nu, ell), d)
        h = 1.0 / (1.0 + 0.85 * (ell / math.sqrt(nu)) * math.log(1.0 / et))
        m = math.ceil((1.0 / h) * (math.pi ** (nu + d / 2.0) * ell ** (2.0 * nu) * et / 0.15)
                      ** (-1.0 / (2.0 * nu + d / 2.0)))
        return h, int(m)
    h = 1.0 / (1.0 + ell * math.sqrt(2.0 * d / nu) * math.log(d * 3.0 ** d / eps))
    m = math.ceil((d * 5.0 ** (d - 1) / (math.pi ** (d / 2.0) * eps)) ** (1.0 / (2.0 * nu))
                  * 1.6 * math.sqrt(nu) / (math.pi * h * ell))
    return h, int(m)


# ----------------------------------------------------------------------------
# Frequency grids and spectral weights (Sec. 3.1-3.2, eqs. 110, basis, 117).
# Multi-indices j in J_m = {-m..m}^d are enumerated row-major with the first
# coordinate slowest; entry j sits at flat index sum_l (j_l + m)(2m+1)^{d-1-l}.
# ----------------------------------------------------------------------------


def freq_grid(m: int, d: int) -> np.ndarray:
    """All j in J_m as an (M, d) integer array, row-major order."""
    g = np.arange(-m, m + 1)
    mesh = np.meshgrid(*([g] * d), indexing="ij")
    return np.stack([a.ravel() for a in mesh], 1)


def spectral_weights(kern: Kernel, d: int, h: float, m: int) -> np.ndarray:
    """D_j = sqrt(h^d khat(h j)), j in J_m (eq. 117), flat row-major."""
    j = freq_grid(m, d).astype(np.float64)
    return np.sqrt(h ** d * kern.khat(h * np.sqrt((j * j).sum(1)), d))


def ktilde(r_vec: np.ndarray, kern: Kernel, h: float, m: int) -> np.ndarray:
    """Discretised kernel eq. 110 at displacements r (n, d):
    sum_{j in J_m} h^d khat(h j) exp(2 pi i h j.r), which is real."""
    r_vec = np.atleast_2d(np.asarray(r_vec, np.float64))
    d = r_vec.shape[1]
    j = freq_grid(m, d).astype(np.float64)
    wts = h ** d * kern.khat(h * np.sqrt((j * j).sum(1)), d)
    ph = 2.0 * math.pi * h * (r_vec @ j.T)
    return (np.cos(ph) * wts[None, :]).sum(1)


# ----------------------------------------------------------------------------
# Direct sums for the Toeplitz vector (eq. 88) and Phi^* y (eq. rhs).
# For points x_n the sum over n of prod_l exp(-2 pi i h k_l x_n^(l)) is a
# product of per-dimension factor matrices contracted over n.
# ----------------------------------------------------------------------------


def _factor(k: np.ndarray, xcol: np.ndarray, h: float, sign: float) -> np.ndarray:
    return np.exp(sign * 2j * math.pi * h * np.outer(k, xcol))


def direct_type1(x: np.ndarray, c: np.ndarray, h: float, K: int, chunk: int = 200_000) -> np.ndarray:
    """sum_n c_n exp(-2 pi i h k.x_n) for all k in J_K; shape (2K+1,)*d."""
    x = np.asarray(x, np.float64)
    if x.ndim == 1:
        x = x[:, None]
    n, d = x.shape
    k = np.arange(-K, K + 1)
    out = np.zeros((2 * K + 1,) * d, dtype=np.complex128)
    c = np.asarray(c, np.complex128)
    for s in range(0, n, chunk):
        xs = x[s:s + chunk]
        cs = c[s:s + chunk]
        e = [_factor(k, xs[:, a], h, -1.0) for a in range(d)]
        if d == 1:
            out += e[0] @ cs
        elif d == 2:
            out += (e[0] * cs[None, :]) @ e[1].T
        else:
            for i in range(2 * K + 1):
                out[i] += (e[1] * (e[0][i] * cs)[None, :]) @ e[2].T
    return out


def direct_modes(x, c, h: float, ks, chunk: int = 4_000_000, threads: int = 0) -> np.ndarray:
    """sum_n c_n exp(-2 pi i h k.x_n) for each listed multi-index k (rows of ks).

    The same direct sum as direct_type1, for a few modes over very many points:
    the points are visited in chunks (numpy releases the interpreter lock in
    its array loops, so chunks run on several threads); each chunk's sums are
    added in chunk order, so the result does not depend on the thread count.
    """
    import concurrent.futures as cf
    import os
    x = np.asarray(x)
    if x.ndim == 1:
        x = x[:, None]
    ks = np.atleast_2d(np.asarray(ks, np.float64))
    n = x.shape[0]
    scalar_c = np.isscalar(c)

    def part(s):
        xs = x[s:s + chunk].astype(np.float64)
        cs = 1.0 if scalar_c else np.asarray(c[s:s + chunk], np.float64)
        ph = -2.0 * math.pi * h * (xs @ ks.T)          # (chunk, nk)
        cr = np.cos(ph)
        ci = np.sin(ph)
        if scalar_c:
            return cr.sum(0) + 1j * ci.sum(0)
        return cs @ cr + 1j * (cs @ ci)
    starts = list(range(0, n, chunk))
    nthreads = threads or min(16, os.cpu_count() or 1)
    with cf.ThreadPoolExecutor(nthreads) as ex:
        parts = list(ex.map(part, starts))
    out = np.zeros(ks.shape[0], np.complex128)
    for p_ in parts:
        out += p_ * (c if scalar_c else 1.0)
    return out


def toeplitz_vector(x, h: float, m: int) -> np.ndarray:
    """w_k = sum_n exp(-2 pi i h k.x_n), k in J_{2m} (eq. 88, sign reading above)."""
    x = np.asarray(x, np.float64)
    return direct_type1(x, np.ones(x.shape[0]), h, 2 * m)


def rhs(x, y, h: float, m: int, D: np.ndarray) -> np.ndarray:
    """b = D F^* y, flat over J_m (eq. rhs times eq. 117)."""
    return D * direct_type1(x, y, h, m).ravel()


# ----------------------------------------------------------------------------
# Dense system (eqs. 97, 223) and its Cholesky solution (eq. be).
# ----------------------------------------------------------------------------


def toeplitz_dense(w: np.ndarray, m: int, d: int) -> np.ndarray:
    """(F^*F)_{pl} = w_{j_p - j_l} assembled densely from the J_{2m} array."""
    j = freq_grid(m, d)
    diff = j[:, None, :] - j[None, :, :] + 2 * m          # index into J_{2m}
    return w[tuple(diff[..., a] for a in range(d))]


def system_matrix(w, D, sigma: float, m: int, d: int) -> np.ndarray:
    T = toeplitz_dense(w, m, d)
    A = D[:, None] * T * D[None, :]
    A[np.diag_indices_from(A)] += sigma * sigma
    return A


def solve_weights(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    """beta = A^{-1} b by Cholesky (A is Hermitian positive definite)."""
    cf = linalg.cho_factor(A, lower=True, check_finite=False)
    return linalg.cho_solve(cf, b, check_finite=False)


def design_matrix(x, h: float, m: int, D: np.ndarray) -> np.ndarray:
    """Phi = F D with F_{nj} = exp(+2 pi i h j.x_n) (eq. 205); tiny N only."""
    x = np.asarray(x, np.float64)
    if x.ndim == 1:
        x = x[:, None]
    j = freq_grid(m, x.shape[1]).astype(np.float64)
    return np.exp(2j * math.pi * h * (x @ j.T)) * D[None, :]


def mean_at(z, beta: np.ndarray, D: np.ndarray, h: float, m: int, chunk: int = 100_000) -> np.ndarray:
    """mu(z) = sum_j D_j beta_j exp(+2 pi i h j.z) (eq. muws); complex."""
    z = np.asarray(z, np.float64)
    if z.ndim == 1:
        z = z[:, None]
    q, d = z.shape
    f = (D * beta).reshape((2 * m + 1,) * d)
    k = np.arange(-m, m + 1)
    out = np.empty(q, np.complex128)
    for s in range(0, q, chunk):
        zs = z[s:s + chunk]
        e = [_factor(k, zs[:, a], h, +1.0) for a in range(d)]   # (2m+1, q)
        if d == 1:
            out[s:s + chunk] = f @ e[0]
        elif d == 2:
            out[s:s + chunk] = ((f @ e[1]) * e[0]).sum(0)
        else:
            t = np.einsum("abc,cq->abq", f, e[2])
            t = (t * e[1][None, :, :]).sum(1)
            out[s:s + chunk] = (t * e[0]).sum(0)
    return out


# ----------------------------------------------------------------------------
# The whole method, and the function-space references it is checked against.
# ----------------------------------------------------------------------------


@dataclass
class OracleResult:
    h: float
    m: int
    D: np.ndarray        # (M,)
    w: np.ndarray        # (4m+1,)*d Toeplitz generating vector
    b: np.ndarray        # (M,) right-hand side
    beta: np.ndarray     # (M,) weights
    mu: np.ndarray       # (q,) real posterior mean at targets
    mu_imag_max: float   # max |Im mu| (zero up to rounding)


def efgp(x, y, z, kern: Kernel, sigma: float, eps: float, h: float | None = None,
         m: int | None = None) -> OracleResult:
    """Posterior mean at z by the weight-space method with exact linear algebra."""
    x = np.asarray(x, np.float64)
    if x.ndim == 1:
        x = x[:, None]
    d = x.shape[1]
    hh, mm = choose_h_m(kern, d, eps)
    h = hh if h is None else h
    m = mm if m is None else m
    D = spectral_weights(kern, d, h, m)
    w = toeplitz_vector(x, h, m)
    b = rhs(x, np.asarray(y, np.float64), h, m, D)
    A = system_matrix(w, D, sigma, m, d)
    beta = solve_weights(A, b)
    muc = mean_at(z, beta, D, h, m)
    return OracleResult(h=h, m=m, D=D, w=w, b=b, beta=beta, mu=muc.real,
                        mu_imag_max=float(np.abs(muc.imag).max()) if muc.size else 0.0)


def exact_gp_mean(x, y, z, kern: Kernel, sigma: float) -> np.ndarray:
    """Function-space mean k_z^T (K + sigma^2 I)^{-1} y (eqs. mu, 362)."""
    x = np.asarray(x, np.float64)
    z = np.asarray(z, np.float64)
    if x.ndim == 1:
        x = x[:, None]
    if z.ndim == 1:
        z = z[:, None]
    dist = lambda a, b: np.sqrt(((a[:, None, :] - b[None, :, :]) ** 2).sum(-1))
    K = kern.k(dist(x, x))
    K[np.diag_indices_from(K)] += sigma * sigma
    alpha = linalg.solve(K, np.asarray(y, np.float64), assume_a="pos")
    return kern.k(dist(z, x)) @ alpha


def ktilde_gp_mean(x, y, z, kern: Kernel, sigma: float, h: float, m: int) -> np.ndarray:
    """Function-space mean with the discretised kernel of eq. 110 in place of k."""
    x = np.asarray(x, np.float64)
    z = np.asarray(z, np.float64)
    if x.ndim == 1:
        x = x[:, None]
    if z.ndim == 1:
        z = z[:, None]
    n = x.shape[0]
    diff = (x[:, None, :] - x[None, :, :]).reshape(-1, x.shape[1])
    Kt = ktilde(diff, kern, h, m).reshape(n, n)
    Kt[np.diag_indices_from(Kt)] += sigma * sigma
    alpha = linalg.solve(Kt, np.asarray(y, np.float64), assume_a="pos")
    dz = (z[:, None, :] - x[None, :, :]).reshape(-1, x.shape[1])
    return ktilde(dz, kern, h, m).reshape(z.shape[0], n) @ alpha


def matvec(w, D, sigma, beta, m, d):
    """(D F^*F D + sigma^2 I) beta with the dense Toeplitz matrix (for checks)."""
    return system_matrix(w, D, sigma, m, d) @ beta


# ----------------------------------------------------------------------------
# Error metrics of Sec. 5 (EEPM, RMSE).
# ----------------------------------------------------------------------------


def rms(a, b) -> float:
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.sqrt(np.mean((a - b) ** 2))) if a.size else 0.0
