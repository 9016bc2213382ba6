"""The allocation-free prediction entry point, called through the C ABI.

efgp_predict_noalloc serves callers that cannot allocate device memory when
they predict (real-time loops that must not block in an allocator, hosts that
reserve all device memory up front); it keeps its scratch grids in a fixed
array inside the library.
This file is collected last so that a failure here does not hide the result
of any other test.
"""
import ctypes as C

import numpy as np
import pytest

import synthdata

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


def _setup(E, name, n, precision="mixed"):
    rec = synthdata.config(name, n=n)
    x, y, z = synthdata.make_np(rec)
    fam, nu, ell, sigma, eps = synthdata.MODELS[name]
    h = E.setup(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), E.Kernel(fam, nu, ell), sigma, eps,
                precision=precision)
    h.solve()
    return h, z, y, eps


def _noalloc(E, h, zt, out):
    L = E._capi.lib()
    return L.efgp_predict_noalloc(h.ptr, zt.data_ptr(), zt.shape[0], out.data_ptr())


@pytest.mark.parametrize("name,n,precision", [("matern2d", 50_000, "mixed"), ("se3d", 20_000, "mixed"),
                                              ("se1d", 10_000, "fp64")])
def test_noalloc_matches_predict_twice(E, name, n, precision):
    h, z, y, eps = _setup(E, name, n, precision)
    zt = torch.from_numpy(z[:20_000]).cuda()
    ref = h.predict(zt).double().cpu().numpy()
    tol = 1e-3 * 10 * eps * np.abs(y).max()     # same kernels on the same data: rounding only
    for _ in range(2):                           # the second call reuses the array's old contents
        out = torch.full((zt.shape[0],), float("nan"), device="cuda",
                         dtype=torch.float64 if precision == "fp64" else torch.float32)
        assert _noalloc(E, h, zt, out) == 0, E._capi.lib().efgp_last_error()
        got = out.double().cpu().numpy()
        assert np.isfinite(got).all()
        assert np.abs(got - ref).max() <= tol
    h.close()


def test_noalloc_rejects_grids_beyond_its_array(E):
    # Matern-1/2 with a short length scale needs type-2 grids far above 16 MiB
    x = torch.rand(2000, 2, device="cuda")
    y = torch.rand(2000, device="cuda")
    h = E.setup(x, y, E.Kernel("matern", 0.5, 0.03), 0.5, 1e-4)
    h.solve()
    zt = torch.rand(10, 2, device="cuda")
    out = torch.empty(10, device="cuda")
    st = _noalloc(E, h, zt, out)
    assert st == 8                                   # EFGP_EUNSUPPORTED
    assert b"16777216" in E._capi.lib().efgp_last_error()
    h.close()


def test_noalloc_rejects_host_pointer_handles(E):
    rec = synthdata.config("matern2d", n=5000)
    x, y, z = synthdata.make_np(rec)
    h = E.setup(x, y, E.Kernel("matern", 1.5, 0.1), 0.3, 1e-4)    # host arrays -> host_io handle
    h.solve()
    zt = torch.from_numpy(z[:10]).cuda()
    out = torch.empty(10, device="cuda")
    assert _noalloc(E, h, zt, out) == 1               # EFGP_EINVAL
    h.close()
