"""Multithreaded FP64 CPU EFGP: the CPU baseline the GPU path is timed beside.

TEST AND BENCHMARK INFRASTRUCTURE, NOT PART OF THE LIBRARY.  Only the test
suite and the CPU-baseline leg of ``bench.py`` may import this package.  It is
not the oracle (``oracle.efgp_oracle``, which uses direct sums and a dense
solve): it runs the method the fast way, on the host, in float64, from the
same plain definitions (it takes (h, m) and D from the oracle's parameter
functions), and is pinned against the oracle in ``tests/test_cpu_efgp.py``.

Steps (Algorithm 2 of the paper, with the nonuniform FFTs of Sec. 4.1):

* (h, m) and D_j = sqrt(h^d khat(h j))                 (Sec. 4.2, eq. 117; the oracle's functions)
* type-1 NUFFTs for the Toeplitz vector w on J_2m and b = D F^* y on J_m
  (eqs. 88 and rhs, exponents exp(-2 pi i h k.x)), by spreading with the
  exponential-of-semicircle kernel psi(z) = exp(beta (sqrt(1 - z^2) - 1))
  of width W on a grid upsampled by 2, an FFT, and division by psi's
  Fourier transform (Gauss-Legendre quadrature)
* conjugate gradients on (D T D + sigma^2 I) beta = b with the Toeplitz
  product by zero padding to an FFT length L >= 4m + 1 (Algorithm 1), beta_0 = 0,
  stopping at ||r|| <= rho ||b||, rho = eps / 10
* type-2 NUFFT for mu(z) = Re sum_j D_j beta_j exp(+2 pi i h j.z) (eq. muws):
  division by the transform of psi, an inverse FFT, interpolation with psi.

Parallelism: FFTs on all host cores (scipy.fft workers); spreading and
interpolation vectorised over chunks of points, chunks on a thread pool.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import scipy.fft as sfft

from oracle import efgp_oracle as O

WORKERS = os.cpu_count() or 1


def _chunk(W, d):
    """Points per vectorised chunk: about 4M footprint entries."""
    return max(4096, (1 << 22) // W ** d)


def es_params(tol: float):
    """Width W (grid points per dimension) and shape beta for accuracy tol with
    upsampling 2: W = ceil(log10(1/tol)) + 1, beta = 2.30 W."""
    W = max(2, int(math.ceil(math.log10(1.0 / tol))) + 1)
    return W, 2.30 * W


def es_kernel(z, beta):
    z = np.asarray(z, np.float64)
    out = np.zeros_like(z)
    inside = np.abs(z) < 1.0
    out[inside] = np.exp(beta * (np.sqrt(1.0 - z[inside] ** 2) - 1.0))
    return out


def es_transform(k, nf, W, beta, nodes=400):
    """phi-hat(k) = sum over the grid of phi(s) exp(-2 pi i k s / nf), phi(s) =
    psi(2 s / W), taken as the integral (W/2) int psi(z) exp(-i pi k W z / nf) dz
    = W int_0^1 psi(z) cos(pi k W z / nf) dz (psi is even)."""
    zq, wq = np.polynomial.legendre.leggauss(nodes)
    zq = 0.5 * (zq + 1.0)
    wq = 0.5 * wq
    psi = es_kernel(zq, beta)
    k = np.asarray(k, np.float64)
    return W * (np.cos(np.pi * W * np.outer(k, zq) / nf) @ (wq * psi))


def fine_grid(K: int) -> int:
    """Upsampled grid for modes |k| <= K: at least 2 (2K + 1), FFT-friendly."""
    return sfft.next_fast_len(2 * (2 * K + 1))


def _footprint(x, h, nf, W, beta):
    """Grid start l0 (N,) and weights (N, W) of points x in [0,1] at grid
    coordinate u = h x nf: point n touches l0_n .. l0_n + W - 1 (mod nf)."""
    u = h * x * nf
    l0 = np.ceil(u - 0.5 * W).astype(np.int64)
    offs = np.arange(W)
    wts = es_kernel((l0[:, None] + offs[None, :] - u[:, None]) / (0.5 * W), beta)
    return l0, wts


def _spread_chunk(xc, cc, h, nf, W, beta, d):
    grid = np.zeros((nf,) * d, np.complex128)
    l0, wt = zip(*[_footprint(xc[:, a], h, nf, W, beta) for a in range(d)])
    offs = np.arange(W)
    idx = [(l0[a][:, None] + offs[None, :]) % nf for a in range(d)]
    if d == 1:
        flat = idx[0]
        val = wt[0] * cc[:, None]
    elif d == 2:
        flat = idx[0][:, :, None] * nf + idx[1][:, None, :]
        val = wt[0][:, :, None] * wt[1][:, None, :] * cc[:, None, None]
    else:
        flat = (idx[0][:, :, None, None] * nf + idx[1][:, None, :, None]) * nf + idx[2][:, None, None, :]
        val = wt[0][:, :, None, None] * wt[1][:, None, :, None] * wt[2][:, None, None, :] * cc[:, None, None, None]
    flat = flat.ravel()
    val = val.ravel()
    g = grid.reshape(-1)
    g.real += np.bincount(flat, weights=val.real, minlength=nf ** d)
    g.imag += np.bincount(flat, weights=val.imag, minlength=nf ** d)
    return grid


def type1(x, c, h, K, tol):
    """sum_n c_n exp(-2 pi i h k.x_n) for k in {-K..K}^d (row-major)."""
    x = np.asarray(x, np.float64)
    if x.ndim == 1:
        x = x[:, None]
    d = x.shape[1]
    W, beta = es_params(tol)
    nf = fine_grid(K)
    c = np.asarray(c, np.complex128)
    ch = _chunk(W, d)
    chunks = [(s, min(len(x), s + ch)) for s in range(0, len(x), ch)]
    grid = np.zeros((nf,) * d, np.complex128)
    if chunks:
        with ThreadPoolExecutor(WORKERS) as ex:
            for part in ex.map(lambda ab: _spread_chunk(x[ab[0]:ab[1]], c[ab[0]:ab[1]], h, nf, W, beta, d), chunks):
                grid += part
    G = sfft.fftn(grid, workers=WORKERS)
    ks = np.arange(-K, K + 1)
    corr = 1.0 / es_transform(ks, nf, W, beta)
    sel = np.ix_(*([ks % nf] * d))
    out = G[sel]
    for a in range(d):
        shape = [1] * d
        shape[a] = len(ks)
        out = out * corr.reshape(shape)
    return out.reshape(-1)


def type2_real(z, f, h, K, tol):
    """Re sum_{k in {-K..K}^d} f_k exp(+2 pi i h k.z) at points z."""
    z = np.asarray(z, np.float64)
    if z.ndim == 1:
        z = z[:, None]
    q, d = z.shape
    W, beta = es_params(tol)
    nf = fine_grid(K)
    ks = np.arange(-K, K + 1)
    corr = 1.0 / es_transform(ks, nf, W, beta)
    g = np.asarray(f, np.complex128).reshape((2 * K + 1,) * d)
    for a in range(d):
        shape = [1] * d
        shape[a] = len(ks)
        g = g * corr.reshape(shape)
    grid = np.zeros((nf,) * d, np.complex128)
    grid[np.ix_(*([ks % nf] * d))] = g
    # sum_k g_k exp(+2 pi i k l / nf) on the grid (unnormalised inverse FFT)
    gr = sfft.ifftn(grid, workers=WORKERS, norm="forward").real.reshape(-1)
    out = np.empty(q)
    offs = np.arange(W)

    def chunk(ab):
        a0, a1 = ab
        zc = z[a0:a1]
        l0, wt = zip(*[_footprint(zc[:, a], h, nf, W, beta) for a in range(d)])
        idx = [(l0[a][:, None] + offs[None, :]) % nf for a in range(d)]
        if d == 1:
            out[a0:a1] = (gr[idx[0]] * wt[0]).sum(1)
        elif d == 2:
            vals = gr[idx[0][:, :, None] * nf + idx[1][:, None, :]]
            out[a0:a1] = np.einsum("nu,nv,nuv->n", wt[0], wt[1], vals)
        else:
            vals = gr[(idx[0][:, :, None, None] * nf + idx[1][:, None, :, None]) * nf + idx[2][:, None, None, :]]
            out[a0:a1] = np.einsum("nu,nv,nw,nuvw->n", wt[0], wt[1], wt[2], vals)

    ch = _chunk(W, d)
    with ThreadPoolExecutor(WORKERS) as ex:
        list(ex.map(chunk, [(s, min(q, s + ch)) for s in range(0, q, ch)]))
    return out


class ToeplitzOperator:
    """v -> D T D v + sigma^2 v with T_{jl} = w_{j-l} (Algorithm 1): w placed
    at k mod L, v at j + m, product in Fourier space, output read at j + m."""

    def __init__(self, w, D, sigma, m, d):
        self.m, self.d, self.D, self.s2 = m, d, D, sigma * sigma
        self.L = sfft.next_fast_len(4 * m + 1)
        n4 = 4 * m + 1
        grid = np.zeros((self.L,) * d, np.complex128)
        k = np.arange(-2 * m, 2 * m + 1) % self.L
        grid[np.ix_(*([k] * d))] = np.asarray(w).reshape((n4,) * d)
        self.what = sfft.fftn(grid, workers=WORKERS)

    def __call__(self, v):
        n1 = 2 * self.m + 1
        u = np.zeros((self.L,) * self.d, np.complex128)
        u[(slice(0, n1),) * self.d] = (self.D * v).reshape((n1,) * self.d)
        y = sfft.ifftn(self.what * sfft.fftn(u, workers=WORKERS), workers=WORKERS)
        return self.D * y[(slice(0, n1),) * self.d].reshape(-1) + self.s2 * v


def conjugate_gradients(A, b, rho, max_iter=100000):
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(np.vdot(r, r).real)
    tol2 = rho * rho * rr
    it = 0
    while rr > tol2 and it < max_iter:
        Ap = A(p)
        alpha = rr / float(np.vdot(p, Ap).real)
        x += alpha * p
        r -= alpha * Ap
        rr_new = float(np.vdot(r, r).real)
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it


def efgp(x, y, z, kern: "O.Kernel", sigma: float, eps: float, cg_tol: float | None = None):
    """Posterior mean at z; returns (mu, info dict)."""
    x = np.asarray(x, np.float64)
    if x.ndim == 1:
        x = x[:, None]
    d = x.shape[1]
    h, m = O.choose_h_m(kern, d, eps)
    D = O.spectral_weights(kern, d, h, m)
    tol = eps / 10
    w = type1(x, np.ones(len(x)), h, 2 * m, tol)
    b = D * type1(x, np.asarray(y, np.float64), h, m, tol)
    A = ToeplitzOperator(w, D, sigma, m, d)
    beta, iters = conjugate_gradients(A, b, eps / 10 if cg_tol is None else cg_tol)
    mu = type2_real(z, D * beta, h, m, tol)
    return mu, {"h": h, "m": m, "iters": iters, "threads": WORKERS}
