"""The multithreaded CPU EFGP (the CPU baseline of the benchmark) against the
FP64 oracle: its NUFFTs against direct sums, and its posterior mean against
the oracle's exact solve of the same discretised problem."""
import numpy as np
import pytest

import synthdata
import cpu_efgp as C
from oracle import efgp_oracle as O


@pytest.mark.parametrize("d,K", [(1, 40), (2, 12), (3, 5)])
def test_type1_and_type2_against_direct_sums(d, K):
    rng = np.random.default_rng(d)
    x = rng.random((3000, d))
    c = rng.standard_normal(3000) + 1j * rng.standard_normal(3000)
    h, tol = 0.7, 1e-7
    got = C.type1(x, c, h, K, tol)
    ks = O.freq_grid(K, d)
    want = np.exp(-2j * np.pi * h * (ks @ x.T)) @ c
    assert np.abs(got - want).max() <= 10 * tol * np.abs(c).sum()
    f = rng.standard_normal(len(ks)) + 1j * rng.standard_normal(len(ks))
    z = rng.random((500, d))
    got2 = C.type2_real(z, f, h, K, tol)
    want2 = (np.exp(2j * np.pi * h * (z @ ks.T)) @ f).real
    assert np.abs(got2 - want2).max() <= 10 * tol * np.abs(f).sum()


@pytest.mark.parametrize("name,n,ntar", [("se1d", 3000, 300), ("matern2d", 5000, 500), ("se3d", 3000, 300)])
def test_cpu_efgp_mean_matches_oracle(name, n, ntar):
    rec = synthdata.config(name, n=n)
    x, y, z = synthdata.make_np(rec)
    z = z[:ntar]
    fam, nu, ell, sigma, eps = synthdata.MODELS[name]
    kern = O.Kernel(fam, nu, ell)
    mu, info = C.efgp(x, y, z, kern, sigma, eps)
    ref = O.efgp(x, y, z, kern, sigma, eps)
    assert info["m"] == ref.m
    assert np.abs(mu - ref.mu).max() <= 10 * eps * np.abs(y).max(), np.abs(mu - ref.mu).max()


@pytest.mark.parametrize("d,m", [(1, 9), (2, 5), (3, 2)])
def test_fft_toeplitz_operator_matches_dense_assembly(d, m):
    """The CPU FFT Toeplitz product (Algorithm 1 with zero padding to a fast
    length) against the oracle's dense D W D + sigma^2 I, entry by entry; it
    then serves as the solver of the reference at shapes whose M is beyond a
    dense solve (the paper's Table 4/5 half-width m = 94)."""
    rng = np.random.default_rng(d)
    x = rng.random((400, d))
    kern = O.Kernel("matern", 1.5, 0.3)
    h = 0.45
    D = O.spectral_weights(kern, d, h, m)
    w = O.toeplitz_vector(x, h, m)
    v = rng.standard_normal(D.size) + 1j * rng.standard_normal(D.size)
    got = C.ToeplitzOperator(w, D, 0.7, m, d)(v)
    want = O.matvec(w, D, 0.7, v, m, d)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    A = C.ToeplitzOperator(w, D, 0.7, m, d)
    b = D * O.toeplitz_vector(x, h, m).reshape(-1)[: D.size]
    beta, it = C.conjugate_gradients(A, b, 1e-13)
    assert np.abs(O.matvec(w, D, 0.7, beta, m, d) - b).max() <= 1e-11 * np.abs(b).max()
