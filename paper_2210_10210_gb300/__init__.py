"""Equispaced-Fourier Gaussian-process regression (EFGP) on one GB300 GPU.

A thin Python binding of the C ABI in include/efgp.h: it only marshals
arguments (pointers, sizes, dtypes) to libefgp.so, whose CUDA kernels run
every step of the method.  There is no CPU fallback: if the library has not
been built the calls raise.

    import paper_2210_10210_gb300 as efgp
    h = efgp.setup(x, y, kernel=efgp.Kernel("matern", nu=1.5, lengthscale=0.1), sigma=0.3, eps=1e-4)
    info = h.solve()
    mu = h.predict(targets)

x, y and targets may be CUDA torch tensors (used in place, on the current
stream) or host arrays (numpy or CPU tensors; copied by the library).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import _capi
from ._capi import efgp_kernel, efgp_options, efgp_params, efgp_problem, efgp_solve_info

__all__ = ["Kernel", "EfgpError", "plan", "setup", "Handle", "batch_setup", "Batch", "prior_weights", "version"]


class EfgpError(RuntimeError):
    def __init__(self, status, where=""):
        L = _capi.lib()
        msg = L.efgp_status_string(status).decode()
        detail = L.efgp_last_error().decode()
        super().__init__(f"{where}: {msg} ({status}){': ' + detail if detail else ''}")
        self.status = status


@dataclass(frozen=True)
class Kernel:
    """Covariance kernel: "se" (squared exponential) or "matern" (smoothness nu)."""
    family: str = "se"
    nu: float = 1.5
    lengthscale: float = 0.1
    variance: float = 1.0

    def c(self):
        fam = {"se": _capi.KERNEL_SE, "matern": _capi.KERNEL_MATERN}[self.family]
        return efgp_kernel(fam, float(self.nu), float(self.lengthscale), float(self.variance))


def version() -> str:
    return _capi.lib().efgp_version().decode()


def _check(status, where):
    if status != _capi.EFGP_OK:
        raise EfgpError(status, where)


def _is_cuda(a) -> bool:
    return hasattr(a, "is_cuda") and a.is_cuda


def _dtype_code(a) -> int:
    s = str(a.dtype)
    if "float64" in s:
        return _capi.F64
    if "float32" in s:
        return _capi.F32
    raise TypeError(f"unsupported dtype {a.dtype}; use float32 or float64")


def _host_array(a):
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(a)


def _options(precision="mixed", coord=_capi.F32, value=_capi.F32, host_io=0, stream=None, **kw) -> efgp_options:
    o = efgp_options()
    _capi.lib().efgp_default_options(C.byref(o))
    o.precision = {"mixed": _capi.MIXED, "fp64": _capi.FP64, "mixed_cg64": _capi.MIXED_CG64}[precision]
    o.coord_dtype = coord
    o.value_dtype = value
    o.host_io = host_io
    for k, v in kw.items():
        if v is None:
            continue
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    if stream is not None:
        o.stream = C.c_void_p(stream)
    return o


def _current_stream(device_tensor):
    """The caller's current stream, or None for the legacy default stream
    (the library then uses its own stream, ordered after the legacy one)."""
    import torch
    s = torch.cuda.current_stream(device_tensor.device).cuda_stream
    return s if s else None


def plan(d: int, n: int, kernel: Kernel, sigma: float, eps: float, precision="mixed", **opts) -> dict:
    """(h, m), FFT and NUFFT sizes chosen for a problem; needs no GPU."""
    p = efgp_params()
    k = kernel.c()
    o = _options(precision, **opts)
    _check(_capi.lib().efgp_plan(int(d), int(n), C.byref(k), float(sigma), float(eps), C.byref(o), C.byref(p)),
           "efgp_plan")
    return p.as_dict()


def prior_weights(M: int, rng) -> np.ndarray:
    """Weights beta on J_m (row-major, M = (2m+1)^d) with E[beta_j conj(beta_k)]
    = delta_jk and beta_{-j} = conj(beta_j), so that
    f(z) = sum_j D_j beta_j exp(2 pi i h j.z) is real with covariance
    sum_j D_j^2 exp(2 pi i h j.(z - z')) = ktilde(z - z') (eq. 110): a GP prior
    draw in the Fourier basis (Sec. 6).  Drawn on the host from the numpy
    Generator rng; the index of -j is M-1-j."""
    z = (rng.standard_normal(M) + 1j * rng.standard_normal(M)) / np.sqrt(2.0)
    beta = (z + np.conj(z[::-1])) / np.sqrt(2.0)
    beta[M // 2] = rng.standard_normal()        # j = 0: real, unit variance
    return beta


class Handle:
    """A set-up problem (owns device workspace until closed)."""

    def __init__(self, ptr, d, coord, value, host_io, keep=(), soa=False):
        self._p = ptr
        self.d = d
        self._soa = soa
        self._coord = coord
        self._value = value
        self._host_io = host_io
        self._keep = keep

    @property
    def ptr(self):
        return self._p

    def close(self):
        if self._p:
            _capi.lib().efgp_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> dict:
        p = efgp_params()
        _check(_capi.lib().efgp_get_params(self._p, C.byref(p)), "efgp_get_params")
        return p.as_dict()

    def solve(self, raise_on_notconv: bool = False) -> dict:
        info = efgp_solve_info()
        st = _capi.lib().efgp_solve(self._p, C.byref(info))
        if st not in (_capi.EFGP_OK, _capi.EFGP_ENOTCONV) or (raise_on_notconv and st != _capi.EFGP_OK):
            raise EfgpError(st, "efgp_solve")
        return {"iters": info.iters, "rel_residual": info.rel_residual,
                "true_rel_residual": info.true_rel_residual, "converged": bool(info.converged),
                "solve_ms": info.solve_ms, "status": st}

    def predict(self, targets, out=None):
        """Posterior mean at targets (q x d).  Device tensor in -> device tensor out."""
        L = _capi.lib()
        if self._host_io:
            z = _host_array(targets)
            q = z.shape[1] if self._soa else z.shape[0]
            mu = np.empty(q, dtype=np.float64 if self._value == _capi.F64 else np.float32) if out is None else out
            _check(L.efgp_predict(self._p, z.ctypes.data, q, mu.ctypes.data), "efgp_predict")
            return mu
        import torch
        if not _is_cuda(targets):
            raise ValueError("handle was set up with device inputs; pass CUDA targets")
        z = targets.contiguous()
        q = z.shape[1] if self._soa else z.shape[0]
        vdt = torch.float64 if self._value == _capi.F64 else torch.float32
        mu = torch.empty(q, dtype=vdt, device=z.device) if out is None else out
        _check(L.efgp_predict(self._p, z.data_ptr(), q, mu.data_ptr()), "efgp_predict")
        return mu

    def phase_times(self) -> dict:
        t = _capi.efgp_phase_times()
        _check(_capi.lib().efgp_get_phase_times(self._p, C.byref(t)), "efgp_get_phase_times")
        return t.as_dict()

    def beta(self) -> np.ndarray:
        p = self.params()
        buf = np.empty(2 * p["M"], dtype=np.float64)
        _check(_capi.lib().efgp_get_beta(self._p, buf.ctypes.data), "efgp_get_beta")
        return buf.view(np.complex128)

    def set_beta(self, beta):
        """Use caller-supplied weights (M complex) for predict (e.g. prior samples)."""
        b = np.ascontiguousarray(beta, dtype=np.complex128)
        _check(_capi.lib().efgp_set_beta(self._p, b.ctypes.data), "efgp_set_beta")

    def sample_prior(self, targets, rng):
        """One draw of the GP prior (covariance ktilde, eq. 110) at targets:
        weights from prior_weights(M, rng), then the type-2 sum."""
        self.set_beta(prior_weights(self.params()["M"], rng))
        return self.predict(targets)

    def system(self):
        """(w on J_{2m} as a (4m+1)^d complex array, b on J_m as an M vector)."""
        p = self.params()
        k4 = (4 * p["m"] + 1) ** self.d
        w = np.empty(2 * k4, dtype=np.float64)
        b = np.empty(2 * p["M"], dtype=np.float64)
        _check(_capi.lib().efgp_get_system(self._p, w.ctypes.data, b.ctypes.data), "efgp_get_system")
        return w.view(np.complex128).reshape((4 * p["m"] + 1,) * self.d), b.view(np.complex128)

    def apply_system_device(self, v, out):
        """out = A v on the device (complex128 CUDA tensors of M entries), stream-ordered."""
        assert v.dtype == out.dtype and v.is_contiguous() and out.is_contiguous()
        _check(_capi.lib().efgp_apply_system_device(self._p, v.data_ptr(), out.data_ptr()),
               "efgp_apply_system_device")

    def apply_system(self, v) -> np.ndarray:
        v = np.ascontiguousarray(v, dtype=np.complex128)
        out = np.empty_like(v)
        _check(_capi.lib().efgp_apply_system(self._p, v.ctypes.data, out.ctypes.data), "efgp_apply_system")
        return out


def setup(x, y, kernel: Kernel, sigma: float, eps: float, precision: str = "mixed", soa: bool = False,
          stream=None, **opts) -> Handle:
    """Steps 1-3 of the method for points x (N x d, or d x N with soa) and data y."""
    L = _capi.lib()
    dev = _is_cuda(x)
    if dev != _is_cuda(y):
        raise ValueError("x and y must both be CUDA tensors or both host arrays")
    if dev:
        xs, ys = x.contiguous(), y.contiguous()
        keep = (xs, ys)
        xp, yp = xs.data_ptr(), ys.data_ptr()
        if stream is None:
            stream = _current_stream(xs)
    else:
        xs, ys = _host_array(x), _host_array(y)
        keep = (xs, ys)
        xp, yp = xs.ctypes.data, ys.ctypes.data
    if soa:
        d, n = xs.shape
    else:
        n, d = (xs.shape[0], 1) if xs.ndim == 1 else xs.shape
    coord, value = _dtype_code(xs), _dtype_code(ys)
    o = _options(precision, coord, value, host_io=0 if dev else 1, stream=stream, x_layout=1 if soa else 0, **opts)
    k = kernel.c()
    ptr = C.c_void_p()
    _check(L.efgp_setup(xp if n else None, yp if n else None, n, d, C.byref(k), float(sigma), float(eps),
                        C.byref(o), C.byref(ptr)), "efgp_setup")
    return Handle(ptr.value, d, coord, value, 0 if dev else 1, keep if dev else (), soa=soa)


class Batch:
    """Many independent problems solved by one sequence of graph launches."""

    def __init__(self, ptr, n, value, host_io, keep):
        self._p = ptr
        self.n = n
        self._value = value
        self._host_io = host_io
        self._keep = keep

    def close(self):
        if self._p:
            _capi.lib().efgp_batch_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self):
        infos = (efgp_solve_info * self.n)()
        st = _capi.lib().efgp_batch_solve(self._p, infos)
        if st not in (_capi.EFGP_OK, _capi.EFGP_ENOTCONV):
            raise EfgpError(st, "efgp_batch_solve")
        return [{"iters": i.iters, "rel_residual": i.rel_residual, "converged": bool(i.converged),
                 "solve_ms": i.solve_ms} for i in infos]

    def params(self, i) -> dict:
        p = efgp_params()
        _check(_capi.lib().efgp_batch_get_params(self._p, i, C.byref(p)), "efgp_batch_get_params")
        return p.as_dict()

    def handle(self, i) -> Handle:
        """Non-owning view of problem i."""
        h = Handle(_capi.lib().efgp_batch_handle(self._p, i), 2, 0, self._value, self._host_io)
        h.close = lambda: None   # owned by the batch
        return h

    def predict(self, i, targets):
        L = _capi.lib()
        if self._host_io:
            z = _host_array(targets)
            mu = np.empty(z.shape[0], dtype=np.float64 if self._value == _capi.F64 else np.float32)
            _check(L.efgp_batch_predict(self._p, i, z.ctypes.data, z.shape[0], mu.ctypes.data), "efgp_batch_predict")
            return mu
        import torch
        z = targets.contiguous()
        vdt = torch.float64 if self._value == _capi.F64 else torch.float32
        mu = torch.empty(z.shape[0], dtype=vdt, device=z.device)
        _check(L.efgp_batch_predict(self._p, i, z.data_ptr(), z.shape[0], mu.data_ptr()), "efgp_batch_predict")
        return mu


def batch_setup(problems, precision: str = "mixed", **opts) -> Batch:
    """problems: list of dicts with x, y, kernel (Kernel), sigma, eps."""
    L = _capi.lib()
    n = len(problems)
    arr = (efgp_problem * n)()
    keep = []
    dev = _is_cuda(problems[0]["x"])
    coord = value = None
    for i, p in enumerate(problems):
        x, y = p["x"], p["y"]
        if dev:
            xs, ys = x.contiguous(), y.contiguous()
            xp, yp = xs.data_ptr(), ys.data_ptr()
        else:
            xs, ys = _host_array(x), _host_array(y)
            xp, yp = xs.ctypes.data, ys.ctypes.data
        keep += [xs, ys]
        coord, value = _dtype_code(xs), _dtype_code(ys)
        arr[i].x = xp
        arr[i].y = yp
        arr[i].N = xs.shape[0]
        arr[i].d = 1 if xs.ndim == 1 else xs.shape[1]
        arr[i].kern = p["kernel"].c()
        arr[i].sigma = float(p["sigma"])
        arr[i].eps = float(p["eps"])
    o = _options(precision, coord, value, host_io=0 if dev else 1, **opts)
    ptr = C.c_void_p()
    failed = C.c_int(-1)
    st = L.efgp_batch_setup(arr, n, C.byref(o), C.byref(ptr), C.byref(failed))
    if st != _capi.EFGP_OK:
        raise EfgpError(st, f"efgp_batch_setup (problem {failed.value})")
    return Batch(ptr.value, n, value, 0 if dev else 1, keep)
