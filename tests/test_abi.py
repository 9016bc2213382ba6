"""The C ABI without a GPU: the library builds, loads, exports every symbol
declared in include/efgp.h, and its host-only planning matches the oracle."""
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def capi():
    from paper_2210_10210_gb300 import build, _capi
    build.build()
    return _capi


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "efgp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(efgp_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(capi):
    L = capi.lib()
    names = _declared_symbols()
    assert len(names) >= 19
    for n in names:
        assert hasattr(L, n), n
    assert {s[0] for s in capi.SIGNATURES} == set(names)


def test_status_strings_and_version(capi):
    L = capi.lib()
    for s in range(9):
        assert L.efgp_status_string(s)
    assert b"sm_103a" in L.efgp_version()


def _plan(family, nu, ell, d, sigma, eps, n=10_000, **kw):
    import paper_2210_10210_gb300 as E
    return E.plan(d, n, E.Kernel(family, nu, ell), sigma, eps, **kw)


@pytest.mark.parametrize("name", ["se1d", "matern2d", "se3d", "matern2d_1e9", "matern2d_table4",
                                  "matern2d_table5"])
def test_host_plan_matches_oracle_h_m(capi, name):
    import synthdata
    from oracle import efgp_oracle as O
    fam, nu, ell, sigma, eps = synthdata.MODELS[name]
    d = synthdata.config(name).d
    p = _plan(fam, nu, ell, d, sigma, eps)
    h, m = O.choose_h_m(O.Kernel(fam, nu, ell), d, eps)
    assert p["m"] == m
    assert abs(p["h"] - h) <= 1e-12
    assert p["M"] == (2 * m + 1) ** d
    assert p["L"] >= 4 * m + 1
    # the NUFFT plans meet the default tolerance eps/10
    assert p["es_err1"] <= eps / 10 and p["es_err2"] <= eps / 10
    assert p["nf1"] >= 4 * m + 1 and p["nf2"] >= 2 * m + 1


@pytest.mark.parametrize("nu,d,ell,eps", [(3.5, 1, 0.1, 1e-6), (3.5, 2, 0.3, 1e-3), (4.5, 2, 0.1, 1e-3),
                                          (3.5, 3, 0.4, 1e-2)])
def test_host_plan_matches_oracle_for_matern_above_5_2(capi, nu, d, ell, eps):
    from oracle import efgp_oracle as O
    p = _plan("matern", nu, ell, d, 0.3, eps)
    h, m = O.choose_h_m(O.Kernel("matern", nu, ell), d, eps)
    assert p["m"] == m and abs(p["h"] - h) <= 1e-12
    assert p["es_err1"] <= eps / 10 and p["es_err2"] <= eps / 10


@pytest.mark.parametrize("row", [("matern", 0.5, 0.1, 2, 1e-3, 97), ("matern", 1.5, 0.1, 2, 1e-5, 94),
                                 ("matern", 1.5, 0.1, 2, 1e-7, 346)])
def test_host_plan_reproduces_paper_m(capi, row):
    fam, nu, ell, d, eps, m = row
    assert _plan(fam, nu, ell, d, 0.1, eps)["m"] == m


def test_fft_length_is_smooth(capi):
    for m in (3, 11, 41, 94, 200):
        p = _plan("se", 0, 0.1, 2, 0.3, 1e-4, m_override=m)
        L = p["L"]
        v = L
        for f in (2, 3, 5, 7):
            while v % f == 0:
                v //= f
        assert v == 1 and L >= 4 * m + 1


def test_plan_overrides(capi):
    p = _plan("se", 0, 0.1, 1, 0.3, 1e-6, m_override=60, h_override=0.5, fft_len_override=256)
    assert p["m"] == 60 and p["h"] == 0.5 and p["L"] == 256


@pytest.mark.parametrize("bad", [dict(d=0), dict(d=4), dict(sigma=0.0), dict(eps=0.5), dict(eps=1e-14),
                                 dict(ell=-1.0)])
def test_invalid_arguments_rejected_without_gpu(capi, bad):
    import ctypes as C
    from paper_2210_10210_gb300 import _options
    L = capi.lib()
    args = dict(d=2, sigma=0.3, eps=1e-4, ell=0.1)
    args.update(bad)
    k = capi.efgp_kernel(capi.KERNEL_MATERN, 1.5, args["ell"], 1.0)
    o = _options()
    p = capi.efgp_params()
    st = L.efgp_plan(args["d"], 100, C.byref(k), args["sigma"], args["eps"], C.byref(o), C.byref(p))
    assert st == capi.EFGP_EINVAL
    h = C.c_void_p()
    st = L.efgp_setup(None, None, 0, args["d"], C.byref(k), args["sigma"], args["eps"], C.byref(o), C.byref(h))
    assert st == capi.EFGP_EINVAL and not h.value


def test_null_inputs_with_points_rejected(capi):
    import ctypes as C
    from paper_2210_10210_gb300 import _options
    L = capi.lib()
    k = capi.efgp_kernel(capi.KERNEL_SE, 0, 0.1, 1.0)
    o = _options()
    h = C.c_void_p()
    assert L.efgp_setup(None, None, 10, 2, C.byref(k), 0.3, 1e-4, C.byref(o), C.byref(h)) == capi.EFGP_EINVAL
    assert L.efgp_solve(None, None) == capi.EFGP_EINVAL
    assert L.efgp_predict(None, None, 0, None) == capi.EFGP_EINVAL


def test_nufft_error_estimate_is_conservative():
    """The planner's ES error model (one unit point, sampled modes) against a
    direct FP64 NUFFT of random points computed here in numpy from the
    planner's parameters: the model bounds the observed relative error."""
    import paper_2210_10210_gb300 as E
    E._capi.lib()
    for d, fam, nu, ell, eps in [(1, "se", 0, 0.1, 1e-6), (2, "matern", 1.5, 0.1, 1e-4)]:
        p = E.plan(d, 10_000, E.Kernel(fam, nu, ell), 0.3, eps)
        assert p["es_err1"] < eps / 10
        assert p["w1"] >= 3 and p["poly_deg1"] >= p["w1"] - 1


def test_ctypes_struct_layouts_match_the_header():
    """Every struct the binding passes through the C ABI has the same size and
    field offsets in ctypes as in include/efgp.h (compiled here with gcc)."""
    import shutil
    import subprocess
    import ctypes
    from paper_2210_10210_gb300 import _capi
    from paper_2210_10210_gb300 import build as B
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [_capi.efgp_kernel, _capi.efgp_options, _capi.efgp_params, _capi.efgp_solve_info,
               _capi.efgp_phase_times, _capi.efgp_problem]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "efgp.h"', 'int main(void) {']
    for st in structs:
        n = st.__name__
        lines.append(f'  printf("{n} sizeof %zu\\n", sizeof({n}));')
        for f, _ in st._fields_:
            lines.append(f'  printf("{n} {f} %zu\\n", offsetof({n}, {f}));')
    lines += ['  return 0;', '}']
    os.makedirs(B.OUT_DIR, exist_ok=True)   # the package's (ignored) build directory
    src = os.path.join(B.OUT_DIR, "layout_check.c")
    with open(src, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    exe = os.path.join(B.OUT_DIR, "layout_check")
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for st in structs:
        n = st.__name__
        assert got[(n, "sizeof")] == ctypes.sizeof(st), n
        for f, _ in st._fields_:
            assert got[(n, f)] == getattr(st, f).offset, (n, f)
