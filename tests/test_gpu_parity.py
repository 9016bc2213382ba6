"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Inputs are the seeded synthetic workloads of ``synthdata`` at sizes the
oracle finishes in seconds (N-reduced twins of the large workloads, with the
same kernel, length scale, noise and tolerance, hence the same h and m).
Criterion for the posterior mean: max |mu_gpu - mu_oracle| <= 10 eps max|y|.
"""
import math

import numpy as np
import pytest

import synthdata
from oracle import efgp_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_10210_gb300 as E
    from paper_2210_10210_gb300 import build
    build.build()
    return E


def _kernel(E, model):
    fam, nu, ell, sigma, eps = model
    return E.Kernel(fam, nu, ell), O.Kernel(fam, nu, ell), sigma, eps


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


_ORACLE_CACHE = {}


def _oracle(key, x, y, z, okern, sigma, eps):
    if key not in _ORACLE_CACHE:
        _ORACLE_CACHE[key] = O.efgp(x, y, z, okern, sigma, eps)
    return _ORACLE_CACHE[key]


def _run_case(E, name, n, precision, n_targets=None, max_targets=20000, **opts):
    rec = synthdata.config(name, n=n)
    if n_targets is not None:
        rec.targets, rec.n_targets = "iid", n_targets
    x, y, z = synthdata.make_np(rec)
    z = z[:max_targets]
    ek, ok, sigma, eps = _kernel(E, synthdata.MODELS[name])
    h = E.setup(_dev(x), _dev(y), ek, sigma, eps, precision=precision, **opts)
    info = h.solve()
    mu = h.predict(_dev(z)).double().cpu().numpy()
    w, b = h.system()
    beta = h.beta()
    par = h.params()
    ref = _oracle((name, n, n_targets, max_targets), x, y, z, ok, sigma, eps)
    return dict(h=h, info=info, mu=mu, w=w, b=b, beta=beta, par=par, ref=ref, x=x, y=y, z=z, eps=eps, sigma=sigma)


def _check(r, mu_factor=10.0, nufft_slack=3.0):
    ref, par, eps = r["ref"], r["par"], r["eps"]
    assert par["m"] == ref.m and abs(par["h"] - ref.h) < 1e-12
    n = r["x"].shape[0]
    tol = eps / 10
    # Toeplitz vector (eq. 88) and right-hand side: NUFFT error relative to sum |c_n|
    if n:
        ew = np.abs(r["w"] - ref.w).max() / n
        eb = (np.abs(r["b"] - ref.b) / ref.D).max() / np.abs(r["y"]).sum()
        assert ew <= nufft_slack * tol, ew
        assert eb <= nufft_slack * tol, eb
    # CG reached its tolerance
    assert r["info"]["converged"], r["info"]
    assert r["info"]["true_rel_residual"] <= 10 * eps
    # posterior mean
    err = np.abs(r["mu"] - ref.mu).max()
    assert err <= mu_factor * eps * np.abs(r["y"]).max(), (err, eps * np.abs(r["y"]).max())
    return err


def test_se1d_fp64_full_size(E):
    r = _run_case(E, "se1d", 10_000, "fp64", max_targets=500)
    _check(r)


def test_se1d_mixed_at_fp32_reach(E):
    # the 1D SE workload is specified in FP64 (eps = 1e-6 is at the FP32
    # floor of the mixed path); the mixed path is checked at eps = 1e-5
    rec = synthdata.config("se1d", n=10_000)
    x, y, z = synthdata.make_np(rec)
    kern = O.Kernel("se", 0.0, 0.1)
    h = E.setup(_dev(x), _dev(y), E.Kernel("se", 0.0, 0.1), 0.3, 1e-5, precision="mixed")
    info = h.solve()
    mu = h.predict(_dev(z)).double().cpu().numpy()
    ref = O.efgp(x, y, z, kern, 0.3, 1e-5)
    assert info["converged"]
    assert np.abs(mu - ref.mu).max() <= 10 * 1e-5 * np.abs(y).max()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_matern2d_twin(E, precision):
    r = _run_case(E, "matern2d", 100_000, precision, max_targets=20_000)
    _check(r)


def test_matern2d_full_size_mixed(E):
    r = _run_case(E, "matern2d", 1_000_000, "mixed", max_targets=20_000)
    _check(r)


def test_se3d_clustered_twin(E):
    r = _run_case(E, "se3d", 100_000, "mixed", max_targets=5_000)
    _check(r)


def test_matern2d_1e9_shape_twin(E):
    # the billion-point workload's kernel, noise and tolerance at N = 1e6
    r = _run_case(E, "matern2d_1e9", 1_000_000, "mixed", max_targets=20_000)
    _check(r)


def test_toeplitz_apply_matches_dense(E):
    # the FFT Toeplitz product against the dense oracle matrix built from the
    # GPU's own w (isolates Algorithm "Fast product of Toeplitz matrix")
    for name, n, prec, tol in [("matern2d", 20_000, "mixed", 2e-5), ("matern2d", 20_000, "fp64", 1e-12),
                               ("se3d", 20_000, "mixed", 2e-5), ("se3d", 5_000, "fp64", 1e-12),
                               ("se1d", 2_000, "fp64", 1e-12)]:
        rec = synthdata.config(name, n=n)
        x, y, _ = synthdata.make_np(rec)
        ek, ok, sigma, eps = _kernel(E, synthdata.MODELS[name])
        h = E.setup(_dev(x), _dev(y), ek, sigma, eps, precision=prec)
        w, _ = h.system()
        par = h.params()
        D = O.spectral_weights(ok, rec.d, par["h"], par["m"])
        rng = np.random.default_rng(0)
        v = rng.standard_normal(par["M"]) + 1j * rng.standard_normal(par["M"])
        got = h.apply_system(v)
        want = O.matvec(w, D, sigma, v, par["m"], rec.d)
        # entry by entry, relative to the largest entry of the product
        err = np.abs(got - want).max() / np.abs(want).max()
        assert err <= tol, (name, prec, err)
        h.close()


@pytest.mark.parametrize("name,n,prec", [("matern2d", 100_000, "mixed"), ("se3d", 50_000, "mixed"),
                                         ("se1d", 10_000, "fp64"), ("matern2d", 20_000, "fp64")])
def test_single_launch_cg_matches_graph_cg(E, name, n, prec):
    # one persistent launch on a thread-block cluster (mode 2), one launch of
    # the work-claiming scheduled kernel (mode 3) and one cooperative launch
    # over the whole GPU with grid barriers (mode 4) vs graph-captured per-pass
    # kernels (mode 1): same iterations up to rounding, same mean
    rec = synthdata.config(name, n=n)
    x, y, z = synthdata.make_np(rec)
    z = z[:5000]
    ek, ok, sigma, eps = _kernel(E, synthdata.MODELS[name])
    out = {}
    for mode in (1, 2, 3, 4):
        h = E.setup(_dev(x), _dev(y), ek, sigma, eps, precision=prec, cg_mode=mode)
        info = h.solve()
        assert info["converged"], (mode, info)
        out[mode] = (info, h.predict(_dev(z)).double().cpu().numpy())
        h.close()
    i1, m1 = out[1]
    for mode in (2, 3, 4):
        i2, m2 = out[mode]
        assert abs(i1["iters"] - i2["iters"]) <= max(5, 0.1 * i1["iters"]), mode
        # other line batches, other FP32 rounding, another CG path: two
        # iterates that stop at the same residual agree to half the criterion
        assert np.abs(m1 - m2).max() <= 0.5 * 10 * eps * np.abs(y).max(), mode
        assert i2["true_rel_residual"] <= 10 * eps, mode


def test_ragged_tiny_and_edge_points(E):
    ek, ok, sigma, eps = _kernel(E, synthdata.MODELS["matern2d"])
    rng = np.random.default_rng(5)
    for n in (1, 7, 33, 1001):
        x = rng.random((n, 2)).astype(np.float32)
        x[0] = [0.0, 1.0]
        if n > 1:
            x[1] = [1.0, 1.0]
        y = rng.standard_normal(n).astype(np.float32)
        z = np.array([[0, 0], [1, 1], [0.5, 0.25], [1, 0]], np.float32)
        h = E.setup(_dev(x), _dev(y), ek, sigma, eps)
        h.solve()
        mu = h.predict(_dev(z)).double().cpu().numpy()
        ref = O.efgp(x, y, z, ok, sigma, eps)
        assert np.abs(mu - ref.mu).max() <= 10 * eps * np.abs(y).max(), n
        h.close()


def test_empty_data_gives_zero_mean(E):
    ek, _, sigma, eps = _kernel(E, synthdata.MODELS["matern2d"])
    x = torch.empty((0, 2), dtype=torch.float32, device="cuda")
    y = torch.empty((0,), dtype=torch.float32, device="cuda")
    h = E.setup(x, y, ek, sigma, eps)
    info = h.solve()
    assert info["iters"] == 0
    mu = h.predict(torch.rand(10, 2, device="cuda"))
    assert torch.all(mu == 0)


def test_out_of_range_points_rejected(E):
    ek, _, sigma, eps = _kernel(E, synthdata.MODELS["matern2d"])
    x = torch.rand(100, 2, device="cuda")
    x[17, 1] = 1.5
    y = torch.rand(100, device="cuda")
    with pytest.raises(E.EfgpError) as ei:
        E.setup(x, y, ek, sigma, eps)
    assert ei.value.status == 2
    x[17, 1] = float("nan")
    with pytest.raises(E.EfgpError):
        E.setup(x, y, ek, sigma, eps)
    x[17, 1] = 0.5
    h = E.setup(x, y, ek, sigma, eps)
    h.solve()
    with pytest.raises(E.EfgpError) as ei:
        h.predict(torch.tensor([[0.5, -0.1]], device="cuda"))
    assert ei.value.status == 2


def test_predict_before_solve_is_state_error(E):
    ek, _, sigma, eps = _kernel(E, synthdata.MODELS["matern2d"])
    h = E.setup(torch.rand(50, 2, device="cuda"), torch.rand(50, device="cuda"), ek, sigma, eps)
    with pytest.raises(E.EfgpError) as ei:
        h.predict(torch.rand(3, 2, device="cuda"))
    assert ei.value.status == 7


def test_host_io_and_soa_layouts_agree(E):
    rec = synthdata.config("matern2d", n=50_000)
    x, y, z = synthdata.make_np(rec)
    z = z[:5000]
    ek, _, sigma, eps = _kernel(E, synthdata.MODELS["matern2d"])
    h1 = E.setup(_dev(x), _dev(y), ek, sigma, eps)
    h1.solve()
    mu1 = h1.predict(_dev(z)).cpu().numpy()
    h2 = E.setup(x, y, ek, sigma, eps)            # host arrays: the library copies
    h2.solve()
    mu2 = h2.predict(z)
    h3 = E.setup(_dev(x.T.copy()), _dev(y), ek, sigma, eps, soa=True)
    h3.solve()
    mu3 = h3.predict(_dev(z.T.copy()))            # targets in the same d x q layout
    scale = 10 * eps * np.abs(y).max()
    assert np.abs(mu1 - mu2).max() <= 0.2 * scale
    assert np.abs(mu1 - mu3.cpu().numpy()).max() <= 0.2 * scale


def test_cg_iteration_cap_reports_not_converged(E):
    rec = synthdata.config("matern2d", n=20_000)
    x, y, _ = synthdata.make_np(rec)
    ek, _, sigma, eps = _kernel(E, synthdata.MODELS["matern2d"])
    h = E.setup(_dev(x), _dev(y), ek, sigma, eps, max_iter=3)
    info = h.solve()
    assert not info["converged"] and info["iters"] == 3 and info["status"] == 4
    mu = h.predict(torch.rand(10, 2, device="cuda"))     # beta is still usable
    assert torch.isfinite(mu).all()


# The fused set-up applies to ES widths <= 6: the planner picks them for the
# billion-point workload (sigma_up = 2.5, W = 5), at small N it prefers wider
# kernels on smaller grids; the fused-path tests fix that plan.
_FUSED_PLAN = dict(upsampfac=2.5, es_width=5)


def test_deterministic_rerun(E):
    """The fused set-up sums in an order fixed by the input alone (stable
    counting sorts, slot reductions in block order) and the CG reduces in
    block order: two runs give bitwise-identical w, b, beta and mean."""
    rec = synthdata.config("matern2d_1e9", n=300_000)
    x, y, z = synthdata.make_np(rec)
    ek, _, sigma, eps = _kernel(E, synthdata.MODELS["matern2d_1e9"])
    outs = []
    for _ in range(2):
        h = E.setup(_dev(x), _dev(y), ek, sigma, eps, setup_path=2, **_FUSED_PLAN)
        assert h.phase_times()["setups_fused"] == 1
        h.solve()
        w, b = h.system()
        outs.append((w, b, h.beta(), h.predict(_dev(z[:2000])).cpu().numpy()))
        h.close()
    for a, c in zip(outs[0], outs[1]):
        assert np.array_equal(a, c)


@pytest.mark.parametrize("n", [1, 7, 4097, 300_001, 9_000_003])
def test_fused_setup_matches_three_pass(E, n):
    """The fused chunked set-up (count, scan, one persistent sort-and-spread
    launch) against the three-pass form (count, sorting scatter, spread) on
    the same points: w and b agree to FP32 rounding of the in-tile sums, far
    inside the NUFFT tolerance.  9e6 points span three chunks of the
    persistent kernel, the last one partial, with a partial sub-chunk and an
    odd count; 4097 leaves one point past the first sub-chunk."""
    rec = synthdata.config("matern2d_1e9", n=n)
    x, y, _ = synthdata.make_np(rec)
    ek, _, sigma, eps = _kernel(E, synthdata.MODELS["matern2d_1e9"])
    got = {}
    for path in (1, 2):
        h = E.setup(_dev(x), _dev(y), ek, sigma, eps, setup_path=path, **_FUSED_PLAN)
        assert h.phase_times()["setups_fused"] == (1 if path == 2 and n > 0 else 0)
        got[path] = h.system()
        h.close()
    tol = eps / 10
    scale_w = max(n, 1)
    scale_b = max(np.abs(y).sum(), 1e-30)
    (w1, b1), (w2, b2) = got[1], got[2]
    assert np.abs(w1 - w2).max() / scale_w <= 1e-2 * tol
    assert np.abs(b1 - b2).max() / scale_b <= 1e-2 * tol
    # w_0 = sum_n exp(0) is the point count
    w0 = w2.flat[w2.size // 2]
    assert abs(w0.real - n) <= 3 * tol * scale_w and abs(w0.imag) <= 3 * tol * scale_w


def test_batch_matches_single_and_oracle(E):
    probs = synthdata.batch_problems(count=6, n_lo=2e3, n_hi=5e4)
    items, singles, refs = [], [], []
    for rec, model in probs:
        rec.n_targets = 500
        x, y, z = synthdata.make_np(rec)
        ek, ok, sigma, eps = _kernel(E, model)
        items.append(dict(x=_dev(x), y=_dev(y), kernel=ek, sigma=sigma, eps=eps))
        singles.append((x, y, z, ek, ok, sigma, eps))
    B = E.batch_setup(items)
    infos = B.solve()
    assert all(i["converged"] for i in infos)
    for i, (x, y, z, ek, ok, sigma, eps) in enumerate(singles):
        mu = B.predict(i, _dev(z)).double().cpu().numpy()
        par = B.params(i)
        if par["M"] <= 12000:
            ref = O.efgp(x, y, z, ok, sigma, eps)
            assert np.abs(mu - ref.mu).max() <= 10 * eps * np.abs(y).max(), i
        h = E.setup(_dev(x), _dev(y), ek, sigma, eps)
        h.solve()
        mu1 = h.predict(_dev(z)).double().cpu().numpy()
        assert np.abs(mu - mu1).max() <= 0.2 * 10 * eps * np.abs(y).max(), i


@pytest.mark.parametrize("name,n", [("matern2d", 20000), ("se3d", 0)])
def test_prior_sample_matches_oracle_type2(E, name, n):
    """A GP prior draw (Sec. 6): caller-supplied weights through efgp_set_beta,
    then the type-2 sum, against the oracle's direct sum with the same weights.
    N = 0 needs no data: the prior is drawn before any observation."""
    rec = synthdata.config(name, n=n)
    x, y, z = synthdata.make_np(rec)
    z = z[:5000]
    ek, ok, sigma, eps = _kernel(E, synthdata.MODELS[name])
    d = x.shape[1]
    h = E.setup(_dev(x), _dev(y), ek, sigma, eps)
    par = h.params()
    beta = E.prior_weights(par["M"], np.random.default_rng(5))
    h.set_beta(beta)
    f = h.predict(_dev(z)).double().cpu().numpy()
    f2 = h.sample_prior(_dev(z), np.random.default_rng(5)).double().cpu().numpy()
    h.close()
    hh, m = O.choose_h_m(ok, d, eps)
    assert m == par["m"]
    D = O.spectral_weights(ok, d, hh, m)
    ref = O.mean_at(z, beta, D, hh, m)
    assert np.abs(ref.imag).max() <= 1e-9 * np.abs(ref.real).max()
    # type-2 NUFFT error bound: tol sum_j |D_j beta_j|
    bound = 3 * (eps / 10) * np.abs(D * beta).sum()
    assert np.abs(f - ref.real).max() <= bound, (np.abs(f - ref.real).max(), bound)
    assert np.array_equal(f, f2)


def test_scheduled_batch_with_empty_and_large_problems(E):
    """The one-launch batched CG over problems of very different size: an
    empty problem (finishes at initialisation), a long-lengthscale small one
    and a short-lengthscale Matern-1/2 one whose FFT grid (L > 1000) is far
    beyond one thread-block cluster.  Each must agree with its own
    single-problem graph-captured solve."""
    specs = [(0, ("matern", 1.5, 0.2, 0.5, 1e-4)), (30_000, ("matern", 1.5, 0.25, 0.4, 1e-4)),
             (200_000, ("matern", 0.5, 0.03, 0.3, 1e-4))]
    items, cases = [], []
    for k, (n, model) in enumerate(specs):
        rec = synthdata.config("matern2d", n=n)
        rec.seed = 40 + k
        rec.targets, rec.n_targets = "iid", 2000
        x, y, z = synthdata.make_np(rec)
        ek, ok, sigma, eps = _kernel(E, model)
        items.append(dict(x=_dev(x), y=_dev(y), kernel=ek, sigma=sigma, eps=eps))
        cases.append((x, y, z, ek, sigma, eps))
    B = E.batch_setup(items)
    assert B.params(2)["L"] > 1000
    infos = B.solve()
    assert all(i["converged"] for i in infos), infos
    assert infos[0]["iters"] == 0
    for i, (x, y, z, ek, sigma, eps) in enumerate(cases):
        mu = B.predict(i, _dev(z)).double().cpu().numpy()
        if i == 0:
            assert np.all(mu == 0)
            continue
        h = E.setup(_dev(x), _dev(y), ek, sigma, eps, cg_mode=1)
        i1 = h.solve()
        mu1 = h.predict(_dev(z)).double().cpu().numpy()
        h.close()
        assert abs(i1["iters"] - infos[i]["iters"]) <= max(5, 0.1 * i1["iters"]), (i, i1, infos[i])
        assert np.abs(mu - mu1).max() <= 0.2 * 10 * eps * np.abs(y).max(), i
    B.close()


@pytest.mark.parametrize("model,d,n", [(("matern", 3.5, 0.3, 0.3, 1e-3), 2, 50_000),
                                       (("matern", 4.5, 0.1, 0.3, 1e-6), 1, 50_000)])
def test_matern_above_5_2_uniform_bound_parameters(E, model, d, n):
    """Matern nu > 5/2 takes (h, m) from the uniform bound eq. maternhm; the
    GPU path with those parameters against the oracle."""
    rec = synthdata.config("matern2d" if d == 2 else "se1d", n=n)
    rec.targets, rec.n_targets = "iid", 3000
    x, y, z = synthdata.make_np(rec)
    ek, ok, sigma, eps = _kernel(E, model)
    prec = "mixed" if eps >= 1e-4 else "fp64"
    h = E.setup(_dev(x), _dev(y), ek, sigma, eps, precision=prec)
    info = h.solve()
    mu = h.predict(_dev(z)).double().cpu().numpy()
    par = h.params()
    h.close()
    hh, m = O.choose_h_m(ok, d, eps)
    assert par["m"] == m and abs(par["h"] - hh) < 1e-12
    ref = O.efgp(x, y, z, ok, sigma, eps)
    assert info["converged"]
    assert np.abs(mu - ref.mu).max() <= 10 * eps * np.abs(y).max()


def test_scheduled_cg_bounded_wait_reports_timeout(E, monkeypatch):
    """EFGP_FAULT=queue_stall starts every problem in a phase whose items are
    all taken and never complete (a flag nothing sets): each block's bounded
    wait for work runs out, the kernel returns, the host reports
    EFGP_ETIMEOUT, and the same handle then solves normally."""
    from paper_2210_10210_gb300 import _capi
    rec = synthdata.config("matern2d", n=20_000)
    x, y, z = synthdata.make_np(rec)
    ek, ok, sigma, eps = _kernel(E, synthdata.MODELS["matern2d"])
    h = E.setup(_dev(x), _dev(y), ek, sigma, eps, cg_mode=3)
    monkeypatch.setenv("EFGP_FAULT", "queue_stall")
    with pytest.raises(E.EfgpError) as ei:
        h.solve()
    assert ei.value.status == _capi.EFGP_ETIMEOUT
    monkeypatch.delenv("EFGP_FAULT")
    info = h.solve()
    assert info["converged"]
    mu = h.predict(_dev(z[:2000])).double().cpu().numpy()
    h.close()
    ref = _oracle(("matern2d", 20_000, None, 2000), x, y, z[:2000], ok, sigma, eps)
    assert np.abs(mu - ref.mu).max() <= 10 * eps * np.abs(y).max()


def test_grid_cg_bounded_barrier_wait_reports_timeout(E, monkeypatch):
    """EFGP_FAULT=grid_stall starts the grid CG's barrier with more arrivals
    than blocks, so no barrier completes: every block's bounded wait runs out,
    the launch returns, the host reports EFGP_ETIMEOUT, and the same handle
    then solves normally."""
    from paper_2210_10210_gb300 import _capi
    rec = synthdata.config("matern2d", n=20_000)
    x, y, z = synthdata.make_np(rec)
    ek, ok, sigma, eps = _kernel(E, synthdata.MODELS["matern2d"])
    h = E.setup(_dev(x), _dev(y), ek, sigma, eps, cg_mode=4)
    monkeypatch.setenv("EFGP_FAULT", "grid_stall")
    with pytest.raises(E.EfgpError) as ei:
        h.solve()
    assert ei.value.status == _capi.EFGP_ETIMEOUT
    monkeypatch.delenv("EFGP_FAULT")
    info = h.solve()
    assert info["converged"]
    mu = h.predict(_dev(z[:2000])).double().cpu().numpy()
    h.close()
    ref = _oracle(("matern2d", 20_000, None, 2000), x, y, z[:2000], ok, sigma, eps)
    assert np.abs(mu - ref.mu).max() <= 10 * eps * np.abs(y).max()


def test_injected_allocation_failure_reports_enomem(E, monkeypatch):
    from paper_2210_10210_gb300 import _capi
    ek, _, sigma, eps = _kernel(E, synthdata.MODELS["matern2d"])
    x = torch.rand(1000, 2, device="cuda")
    y = torch.rand(1000, device="cuda")
    monkeypatch.setenv("EFGP_FAULT", "alloc")
    with pytest.raises(E.EfgpError) as ei:
        E.setup(x, y, ek, sigma, eps)
    assert ei.value.status == _capi.EFGP_ENOMEM
    monkeypatch.delenv("EFGP_FAULT")
    h = E.setup(x, y, ek, sigma, eps)
    assert h.solve()["converged"]
    h.close()


def test_many_targets_shared_memory_interpolation(E):
    """q >= 2^22 targets (the mean at all training points of a large
    problem) take the interpolation with the type-2 grid staged in shared
    memory: it must agree with the per-target gather path on a prefix and
    with the oracle on sampled targets."""
    name = "matern2d_1e9"
    rec = synthdata.config(name, n=50_000)
    x, y, _ = synthdata.make_np(rec)
    q = (1 << 22) + 1001
    z = synthdata.uniform_np(rec.seed, 77, 0, 2 * q).astype(np.float32).reshape(q, 2)
    ek, ok, sigma, eps = _kernel(E, synthdata.MODELS[name])
    h = E.setup(_dev(x), _dev(y), ek, sigma, eps)
    h.solve()
    zd = _dev(z)
    mu_all = h.predict(zd).double().cpu().numpy()
    mu_pre = h.predict(zd[:3000]).double().cpu().numpy()
    h.close()
    scale = np.abs(mu_all).max()
    assert np.abs(mu_all[:3000] - mu_pre).max() <= 1e-6 * scale
    idx = np.random.default_rng(9).choice(q, 1500, replace=False)
    ref = _oracle((name, 50_000, "smem", 1500), x, y, z[idx].astype(np.float64), ok, sigma, eps)
    assert np.abs(mu_all[idx] - ref.mu).max() <= 10 * eps * np.abs(y).max()


@pytest.mark.parametrize("name,n", [("matern2d", 100_000), ("se3d", 50_000)])
def test_autotuned_passes_match_default(E, name, n):
    """efgp_options.autotune re-chooses the line batch and thread count of each
    Toeplitz pass by timing; the solve must agree with the default choice."""
    rec = synthdata.config(name, n=n)
    x, y, z = synthdata.make_np(rec)
    z = z[:5000]
    ek, ok, sigma, eps = _kernel(E, synthdata.MODELS[name])
    out = []
    for tune in (0, 1):
        h = E.setup(_dev(x), _dev(y), ek, sigma, eps, autotune=tune)
        info = h.solve()
        assert info["converged"] and info["true_rel_residual"] <= 10 * eps, (tune, info)
        out.append((info, h.predict(_dev(z)).double().cpu().numpy()))
        h.close()
    (i0, m0), (i1, m1) = out
    assert abs(i0["iters"] - i1["iters"]) <= max(5, 0.1 * i0["iters"])
    # tuned line batches and radix orders round in another order: two
    # iterates stopping at the same residual agree to half the criterion
    assert np.abs(m0 - m1).max() <= 0.5 * 10 * eps * np.abs(y).max()


def test_device_apply_matches_host_apply(E):
    """efgp_apply_system_device (device arrays, stream-ordered) gives the same
    product as the host-pointer accessor."""
    rec = synthdata.config("matern2d", n=20_000)
    x, y, _ = synthdata.make_np(rec)
    ek, ok, sigma, eps = _kernel(E, synthdata.MODELS["matern2d"])
    h = E.setup(_dev(x), _dev(y), ek, sigma, eps)
    M = h.params()["M"]
    rng = np.random.default_rng(4)
    v = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    want = h.apply_system(v)
    vd = torch.from_numpy(v).cuda()
    out = torch.empty_like(vd)
    h.apply_system_device(vd, out)
    torch.cuda.synchronize()
    h.close()
    assert np.array_equal(out.cpu().numpy(), want)


def test_fused_setup_bounded_barrier_wait_reports_timeout(E, monkeypatch):
    """EFGP_FAULT=setup_stall presets the fused set-up's grid barrier with
    more arrivals than blocks: every block's bounded wait runs out after
    the chunk's scatter, the launch returns, the host reports EFGP_ETIMEOUT,
    and a new set-up then works."""
    from paper_2210_10210_gb300 import _capi
    rec = synthdata.config("matern2d_1e9", n=50_000)
    x, y, z = synthdata.make_np(rec)
    ek, ok, sigma, eps = _kernel(E, synthdata.MODELS["matern2d_1e9"])
    monkeypatch.setenv("EFGP_FAULT", "setup_stall")
    with pytest.raises(E.EfgpError) as ei:
        E.setup(_dev(x), _dev(y), ek, sigma, eps, setup_path=2, **_FUSED_PLAN)
    assert ei.value.status == _capi.EFGP_ETIMEOUT
    monkeypatch.delenv("EFGP_FAULT")
    h = E.setup(_dev(x), _dev(y), ek, sigma, eps, setup_path=2, **_FUSED_PLAN)
    assert h.phase_times()["setups_fused"] == 1
    assert h.solve()["converged"]
    h.close()
