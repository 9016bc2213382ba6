"""GP prior draws in the Fourier basis (Sec. 6): the host-drawn weights give
a real field whose covariance is the discretised kernel ktilde (eq. 110)."""
import numpy as np
import pytest

from oracle import efgp_oracle as O


def _weights():
    from paper_2210_10210_gb300 import prior_weights
    return prior_weights


@pytest.mark.parametrize("m,d", [(7, 1), (3, 2), (2, 3)])
def test_prior_weights_conjugate_symmetric(m, d):
    pw = _weights()
    M = (2 * m + 1) ** d
    b = pw(M, np.random.default_rng(3))
    j = O.freq_grid(m, d)
    # flat index of -j is M-1-flat(j) in row-major order
    neg = {tuple(v): i for i, v in enumerate(-j)}
    for i, v in enumerate(j):
        assert b[neg[tuple(v)]] == np.conj(b[i])
    assert b[M // 2].imag == 0.0 and not np.any(j[M // 2])


def test_prior_draws_are_real():
    pw = _weights()
    kern = O.Kernel("matern", 1.5, 0.2)
    h, m = O.choose_h_m(kern, 2, 1e-3)
    D = O.spectral_weights(kern, 2, h, m)
    z = np.random.default_rng(0).uniform(-0.5, 0.5, (50, 2))
    f = O.mean_at(z, pw(D.size, np.random.default_rng(1)), D, h, m)
    assert np.abs(f.imag).max() <= 1e-12 * np.abs(f.real).max()


def test_prior_covariance_is_ktilde():
    """Sample covariance over 40000 draws at 6 points against ktilde(z - z'):
    each entry is a mean of 40000 products with variance <= 2 k(0)^2, so 6
    standard errors bound it at 6 sqrt(2/40000) k(0)."""
    pw = _weights()
    kern = O.Kernel("matern", 0.5, 0.3)
    h, m = O.choose_h_m(kern, 1, 1e-3)
    D = O.spectral_weights(kern, 1, h, m)
    z = np.array([-0.45, -0.3, -0.05, 0.0, 0.2, 0.48])
    Phi = O.design_matrix(z, h, m, D)                      # (6, M)
    rng = np.random.default_rng(11)
    draws = 40000
    B = np.stack([pw(D.size, rng) for _ in range(draws)], 1)
    F = (Phi @ B).real                                      # (6, draws)
    C = F @ F.T / draws
    K = O.ktilde((z[:, None] - z[None, :]).reshape(-1, 1), kern, h, m).reshape(6, 6)
    k0 = O.ktilde(np.zeros((1, 1)), kern, h, m)[0]
    assert abs(k0 - 1.0) <= 1e-2                           # ktilde(0) ~ k(0) = 1
    assert np.abs(C - K).max() <= 6 * np.sqrt(2.0 / draws) * k0
