"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: values the
paper prints, closed forms, numerical transforms, brute force and identities.
No test here needs a GPU.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, special

from oracle import efgp_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- spectral densities
def _numerical_khat(kern, d, xi):
    """Radial Fourier transform of k by adaptive quadrature (Sec. 3.1 convention)."""
    R = 60.0 * kern.ell
    if d == 1:
        f = lambda r: 2.0 * kern.k(np.array([r]))[0] * math.cos(2 * math.pi * xi * r)
    elif d == 2:
        f = lambda r: 2.0 * math.pi * kern.k(np.array([r]))[0] * special.j0(2 * math.pi * xi * r) * r
    else:
        def f(r):
            a = 2 * math.pi * xi * r
            s = 1.0 if a == 0 else math.sin(a) / a
            return 4.0 * math.pi * kern.k(np.array([r]))[0] * s * r * r
    pts = np.linspace(0, R, 41)
    return sum(integrate.quad(f, a, b, limit=400, epsabs=1e-15, epsrel=1e-12)[0]
               for a, b in zip(pts[:-1], pts[1:]))


@pytest.mark.parametrize("family,nu", [("se", 0.0), ("matern", 0.5), ("matern", 1.5), ("matern", 2.5),
                                       ("matern", 3.5)])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_khat_is_fourier_transform_of_k(family, nu, d):
    kern = O.Kernel(family, nu, 0.1)
    for xi in [0.0, 0.7, 2.3, 6.1]:
        num = _numerical_khat(kern, d, xi)
        cf = float(kern.khat(np.array(xi), d))
        assert abs(num - cf) <= 1e-8 * max(abs(cf), 1e-6), (family, nu, d, xi, num, cf)


@pytest.mark.parametrize("family,nu", [("se", 0.0), ("matern", 1.5)])
def test_trapezoid_sum_of_khat_is_k0(family, nu):
    # ||phi_z||^2 = sum_j h^d khat(h j) ~ khat integral = k(0) = 1 (proof of Theorem 6)
    kern = O.Kernel(family, nu, 0.1)
    for d in (1, 2):
        eps = 1e-6 if family == "se" else 1e-4
        h, m = O.choose_h_m(kern, d, eps)
        D = O.spectral_weights(kern, d, h, m)
        tol = eps if family == "se" else 3e-2
        assert abs((D * D).sum() - 1.0) <= tol


# ---------------------------------------------------------------- parameter choice
def _golden_m():
    rows = []
    with open(os.path.join(GOLDEN, "paper_m_values.txt")) as f:
        for line in f:
            line = line.split("#")[0].split()
            if line:
                fam, nu, ell, d, eps, m = line
                rows.append((fam, float(nu), float(ell), int(d), float(eps), int(m)))
    return rows


@pytest.mark.parametrize("row", _golden_m())
def test_matern_m_matches_paper_tables(row):
    fam, nu, ell, d, eps, m = row
    _, mm = O.choose_h_m(O.Kernel(fam, nu, ell), d, eps)
    assert mm == m


def test_l2_norm_closed_form_matern_half_1d():
    # int_{-1}^{1} exp(-2|x|/l) dx = l (1 - exp(-2/l))
    for ell in (0.05, 0.1, 0.3):
        want = math.sqrt(ell * (1.0 - math.exp(-2.0 / ell)))
        got = O.kernel_l2_norm_cube(O.Kernel("matern", 0.5, ell), 1)
        assert abs(got - want) <= 1e-12 * want


@pytest.mark.parametrize("d", [1, 2, 3])
def test_l2_norm_closed_form_se(d):
    # int_{[-1,1]^d} exp(-|x|^2/l^2) = (sqrt(pi) l erf(1/l))^d
    for ell in (0.1, 0.5):
        want = math.sqrt((math.sqrt(math.pi) * ell * math.erf(1.0 / ell)) ** d)
        got = O.kernel_l2_norm_cube(O.Kernel("se", 0.0, ell), d)
        assert abs(got - want) <= 1e-12 * want


def test_l2_norm_matern_3d_quadrature_converged():
    # the coarser 3D rule agrees with a much finer one (Matern-1/2 kink at 0)
    kern = O.Kernel("matern", 0.5, 0.1)
    x, w = O._panels(40, 20)
    r2 = x[:, None] ** 2 + x[None, :] ** 2
    # Matern-1/2 is exp(-r/l): the fine rule uses that closed form
    fine = sum(w[i] * np.sum(np.outer(w, w) * np.exp(-2.0 * np.sqrt(r2 + x[i] ** 2) / 0.1)) for i in range(len(x)))
    fine = math.sqrt(8.0 * fine)
    assert abs(O.kernel_l2_norm_cube(kern, 3) - fine) <= 1e-10 * fine


@pytest.mark.parametrize("d,ell,eps", [(1, 0.1, 1e-6), (1, 0.3, 1e-4), (2, 0.1, 1e-4), (2, 0.2, 1e-6)])
def test_se_choice_meets_uniform_bound(d, ell, eps):
    # Sec. 4.2: the SE choice bounds |ktilde - k| by eps uniformly on [-1,1]^d
    kern = O.Kernel("se", 0.0, ell)
    h, m = O.choose_h_m(kern, d, eps)
    g = np.linspace(-1, 1, 401 if d == 1 else 61)
    pts = np.stack([a.ravel() for a in np.meshgrid(*([g] * d), indexing="ij")], 1)
    err = np.abs(O.ktilde(pts, kern, h, m) - kern.k(np.sqrt((pts ** 2).sum(1))))
    assert err.max() <= eps


@pytest.mark.parametrize("d,eps,h_hand,m_hand", [(1, 1e-4, 0.6740, 12), (2, 1e-4, 0.6582, 13), (3, 1e-3, 0.6650, 13)])
def test_se_printed_formula_at_table2_configs(d, eps, h_hand, m_hand):
    """The printed SE choice (Sec. 4.2) at Table 2's SE configurations
    (l = 0.1), worked by hand.  Table 2 itself prints m = 13/16/17, which
    this formula does not give (the uniform-bound pin above is the
    one-sided check; the table's values are not reproduced).
      d = 1, eps = 1e-4: log(4*1*3/eps) = log(1.2e5) = 11.695, sqrt(2*11.695)
        = 4.836, h = 1/1.4836 = 0.6740; log(4^2*1/eps) = log(1.6e5) = 11.983,
        sqrt(11.983/2) = 2.4478, / (pi*0.1*0.6740 = 0.21174) = 11.56 -> m = 12
      d = 2, eps = 1e-4: log(72/eps) = 13.487, sqrt(26.975) = 5.1937,
        h = 1/1.51937 = 0.6582; log(4^3*2/eps) = 14.062, sqrt(7.031) = 2.6516,
        / (pi*0.1*0.6582 = 0.20677) = 12.82 -> m = 13
      d = 3, eps = 1e-3: log(324/eps) = 12.688, sqrt(25.376) = 5.0374,
        h = 1/1.50374 = 0.6650; log(4^4*3/eps) = 13.552, sqrt(6.776) = 2.6031,
        / (pi*0.1*0.6650 = 0.20892) = 12.46 -> m = 13"""
    h, m = O.choose_h_m(O.Kernel("se", 0.0, 0.1), d, eps)
    assert abs(h - h_hand) < 5e-5 and m == m_hand


@pytest.mark.parametrize("nu,d,ell,eps", [(3.5, 1, 0.1, 1e-6), (3.5, 2, 0.2, 1e-4), (4.5, 2, 0.1, 1e-3),
                                          (3.5, 3, 0.4, 1e-2)])
def test_matern_high_nu_choice_meets_uniform_bound(nu, d, ell, eps):
    # Sec. 4.2, eq. maternhm: for nu > 5/2 the (h, m) choice is the one that
    # guarantees |ktilde - k| <= eps uniformly on [-1,1]^d (the heuristic
    # L2 choice is only for nu <= 5/2)
    kern = O.Kernel("matern", nu, ell)
    h, m = O.choose_h_m(kern, d, eps)
    h2, m2 = O.choose_h_m(O.Kernel("matern", 2.5, ell), d, eps)
    assert (h, m) != (h2, m2)
    g = np.linspace(-1, 1, {1: 801, 2: 61, 3: 17}[d])
    pts = np.stack([a.ravel() for a in np.meshgrid(*([g] * d), indexing="ij")], 1)
    err = np.abs(O.ktilde(pts, kern, h, m) - kern.k(np.sqrt((pts ** 2).sum(1))))
    assert err.max() <= eps, err.max()


def test_pointwise_error_split_prop3():
    # Prop. 3 (derived from the Poisson summation formula it cites): ktilde - k
    # equals the sum over nonzero aliasing images minus h^d times the truncated
    # spectral tail.  The printed statement carries the opposite sign on both
    # terms; subtracting ktilde from the Poisson identity gives the signs used here.
    kern = O.Kernel("se", 0.0, 0.15)
    h, m = 1.5, 1
    x = np.linspace(-1, 1, 9)
    lhs = O.ktilde(x[:, None], kern, h, m) - kern.k(x)
    n = np.arange(-40, 41)
    n = n[n != 0]
    alias = kern.k(x[:, None] + n[None, :] / h).sum(1)
    j = np.arange(-400, 401)
    j = j[np.abs(j) > m]
    trunc = h * (kern.khat(np.abs(j) * h, 1)[None, :] * np.cos(2 * math.pi * h * np.outer(x, j))).sum(1)
    assert np.abs(alias).max() > 1e-3 and np.abs(trunc).max() > 1e-3   # both terms matter
    assert np.abs(lhs - (alias - trunc)).max() <= 1e-13


# ---------------------------------------------------------------- direct sums
def test_type1_lattice_closed_form_1d():
    # x_n = n/N on a lattice: sum_n exp(-2 pi i h k n / N) is a geometric sum
    N, h, K = 37, 0.63, 9
    x = np.arange(N) / N
    got = O.direct_type1(x, np.ones(N), h, K)
    k = np.arange(-K, K + 1)
    q = np.exp(-2j * math.pi * h * k / N)
    want = np.where(np.abs(1 - q) < 1e-15, N, (1 - q ** N) / (1 - q + (np.abs(1 - q) < 1e-15)))
    assert np.abs(got - want).max() <= 1e-12 * N


def test_type1_tensor_lattice_with_strengths_2d():
    # strengths c_n = exp(2 pi i (a.x_n)) on a tensor lattice: product of two geometric sums
    N1, N2, h, K = 11, 7, 0.55, 5
    a = np.array([1.7, -2.13])
    g1, g2 = np.meshgrid(np.arange(N1) / N1, np.arange(N2) / N2, indexing="ij")
    x = np.stack([g1.ravel(), g2.ravel()], 1)
    c = np.exp(2j * math.pi * (x @ a))
    got = O.direct_type1(x, c, h, K)
    k = np.arange(-K, K + 1)

    def geo(Nn, aa):
        q = np.exp(2j * math.pi * (aa - h * k) / Nn)
        return (1 - q ** Nn) / (1 - q)
    want = np.outer(geo(N1, a[0]), geo(N2, a[1]))
    assert np.abs(got - want).max() <= 1e-12 * x.shape[0]


def test_toeplitz_vector_symmetries():
    rng = np.random.default_rng(1)
    x = rng.random((300, 2))
    w = O.toeplitz_vector(x, 0.7, 4)
    assert abs(w[8, 8] - 300) <= 1e-12 * 300                      # w_0 = N
    assert np.abs(w - np.conj(w[::-1, ::-1])).max() <= 1e-12 * 300  # w_{-k} = conj w_k
    assert np.abs(w).max() <= 300 * (1 + 1e-12)


def test_type1_brute_force_3d():
    rng = np.random.default_rng(2)
    x = rng.random((50, 3))
    c = rng.standard_normal(50)
    h, K = 0.8, 2
    got = O.direct_type1(x, c, h, K)
    k = np.arange(-K, K + 1)
    for i, j, l in [(0, 0, 0), (1, 4, 2), (4, 0, 3), (2, 2, 2)]:
        kk = np.array([k[i], k[j], k[l]])
        want = sum(c[n] * np.exp(-2j * math.pi * h * kk @ x[n]) for n in range(50))
        assert abs(got[i, j, l] - want) <= 1e-12 * np.abs(c).sum()


def test_direct_modes_agree_with_direct_type1():
    # the few-mode, many-point direct sum against the lattice-pinned full sum
    rng = np.random.default_rng(9)
    x = rng.random((5000, 2)).astype(np.float32)
    y = rng.standard_normal(5000).astype(np.float32)
    h, K = 0.7, 6
    full_w = O.direct_type1(x, np.ones(5000), h, K)
    full_b = O.direct_type1(x, y, h, K)
    ks = np.array([[0, 0], [3, -2], [-6, 6], [1, 5]])
    got_w = O.direct_modes(x, 1.0, h, ks, chunk=777, threads=3)
    got_b = O.direct_modes(x, y, h, ks, chunk=1000, threads=2)
    for i, (a, b) in enumerate(ks):
        assert abs(got_w[i] - full_w[a + K, b + K]) <= 1e-10 * 5000
        assert abs(got_b[i] - full_b[a + K, b + K]) <= 1e-10 * np.abs(y).sum()


# ---------------------------------------------------------------- structure and solve
@pytest.mark.parametrize("d", [1, 2, 3])
def test_dense_PhiStarPhi_equals_toeplitz_assembly(d):
    rng = np.random.default_rng(3 + d)
    m = {1: 6, 2: 3, 3: 2}[d]
    kern = O.Kernel("matern", 1.5, 0.2)
    x = rng.random((40, d))
    h = 0.6
    D = O.spectral_weights(kern, d, h, m)
    Phi = O.design_matrix(x, h, m, D)
    w = O.toeplitz_vector(x, h, m)
    A = O.system_matrix(w, D, 0.3, m, d)
    ref = Phi.conj().T @ Phi + 0.09 * np.eye(Phi.shape[1])
    assert np.abs(A - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.abs(A - A.conj().T).max() <= 1e-13 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() >= 0.09 * (1 - 1e-9)
    # right-hand side: b = Phi^* y
    y = rng.standard_normal(40)
    assert np.abs(O.rhs(x, y, h, m, D) - Phi.conj().T @ y).max() <= 1e-12 * np.abs(y).sum()


def _small_problem(d, family="matern", nu=1.5, ell=0.15, n=150, seed=7):
    rng = np.random.default_rng(seed)
    x = rng.random((n, d))
    y = np.cos(2 * math.pi * x.sum(1)) + 0.3 * rng.standard_normal(n)
    z = rng.random((40, d))
    return x, y, z, O.Kernel(family, nu, ell)


@pytest.mark.parametrize("d", [1, 2])
def test_solve_residual_and_conjugate_symmetry(d):
    x, y, z, kern = _small_problem(d)
    r = O.efgp(x, y, z, kern, 0.3, 1e-4)
    A = O.system_matrix(r.w, r.D, 0.3, r.m, d)
    assert np.linalg.norm(A @ r.beta - r.b) <= 1e-12 * np.linalg.norm(r.b)
    assert np.abs(r.beta - np.conj(r.beta[::-1])).max() <= 1e-10 * np.abs(r.beta).max()
    assert r.mu_imag_max <= 1e-12 * np.abs(y).max()


@pytest.mark.parametrize("d", [1, 2, 3])
def test_weight_space_equals_function_space_with_ktilde(d):
    # Lemma 1: sum_j beta_j phi_j(z) = ktilde_z^T (Ktilde + sigma^2 I)^{-1} y
    x, y, z, kern = _small_problem(d, n=120, ell=0.2)
    h, m = O.choose_h_m(kern, d, 1e-3)
    m = min(m, {1: 40, 2: 12, 3: 5}[d])
    r = O.efgp(x, y, z, kern, 0.3, 1e-3, h=h, m=m)
    fs = O.ktilde_gp_mean(x, y, z, kern, 0.3, h, m)
    assert np.abs(r.mu - fs).max() <= 1e-9 * np.abs(y).max()


def test_proposition2_identities():
    # beta = Phi^* alpha and alpha = (y - Phi beta)/sigma^2 for the discretised kernel
    x, y, z, kern = _small_problem(2, n=80, ell=0.25)
    h, m = 0.55, 6
    r = O.efgp(x, y, z, kern, 0.4, 1e-3, h=h, m=m)
    Phi = O.design_matrix(x, h, m, r.D)
    Kt = (Phi @ Phi.conj().T).real
    alpha = np.linalg.solve(Kt + 0.16 * np.eye(80), y)
    assert np.abs(Phi.conj().T @ alpha - r.beta).max() <= 1e-9 * np.abs(r.beta).max()
    assert np.abs((y - Phi @ r.beta) / 0.16 - alpha).max() <= 1e-8 * np.abs(alpha).max()


@pytest.mark.parametrize("d,ell,eps", [(1, 0.1, 1e-10), (2, 0.2, 1e-9)])
def test_against_exact_gp_within_theorem6(d, ell, eps):
    x, y, z, _ = _small_problem(d, n=200 if d == 1 else 120, seed=11)
    kern = O.Kernel("se", 0.0, ell)
    sigma = 0.3
    r = O.efgp(x, y, z, kern, sigma, eps)
    ex = O.exact_gp_mean(x, y, z, kern, sigma)
    n = x.shape[0]
    rho = 1e-12
    bound = (n * n / sigma ** 4 * eps + n / sigma ** 2 * (eps + rho + eps * rho)) * np.linalg.norm(y) / math.sqrt(n)
    err = np.abs(r.mu - ex).max()
    assert err <= bound
    assert err <= 1e3 * eps * np.abs(y).max()     # far inside the (loose) bound in practice


def test_planted_sign_error_is_caught(monkeypatch):
    # Plant a plausible mistake in the oracle (type-2 sign flipped relative to
    # type-1, on a kernel whose weights are not conjugate-symmetric) and check
    # that the Lemma-1 pin fails.
    x, y, z, kern = _small_problem(1, n=60, ell=0.2)
    h, m = 0.6, 20
    fs = O.ktilde_gp_mean(x, y, z, kern, 0.3, h, m)
    orig = O._factor

    def flipped(k, xcol, hh, sign):
        return orig(k, xcol, hh, -sign)
    good = O.efgp(x, y, z, kern, 0.3, 1e-3, h=h, m=m).mu
    assert np.abs(good - fs).max() <= 1e-9
    monkeypatch.setattr(O, "_factor", flipped)
    # flipping every exponential is the harmless relabelling j -> -j ...
    assert np.abs(O.efgp(x, y, z, kern, 0.3, 1e-3, h=h, m=m).mu - fs).max() <= 1e-9
    # ... but dropping D from the right-hand side is not
    monkeypatch.setattr(O, "_factor", orig)
    bad_rhs = lambda xx, yy, hh, mm, D: O.direct_type1(xx, yy, hh, mm).ravel()
    monkeypatch.setattr(O, "rhs", bad_rhs)
    assert np.abs(O.efgp(x, y, z, kern, 0.3, 1e-3, h=h, m=m).mu - fs).max() > 1e-3
