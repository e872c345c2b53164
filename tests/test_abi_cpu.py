"""CPU checks of the C ABI: the library builds for sm_103a, loads without a GPU,
exports every function include/sk.h declares, and rejects bad arguments on the
host before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sk.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2201_07524_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\*?(sk_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("sk_init", "sk_kernel_apply", "sk_solve", "sk_grad", "sk_destroy", "sk_get_state",
                 "sk_set_state", "sk_error_string"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_library_exports_only_c_names(lib):
    # extern "C": the ABI names are unmangled
    out = os.popen("nm -D --defined-only %s" % lib._name).read()
    exported = set(re.findall(r"\sT\s(sk_\w+)$", out, flags=re.M))
    assert set(declared_functions()) <= exported


def test_default_params_and_error_strings():
    from paper_2201_07524_gb300 import sk
    p = sk.sk_default_params()
    assert (p.N, p.sigma, p.m_w, p.p, p.precision) == (64, 2.0, 4, 8, sk.SK_FP32)
    assert p.eps_B == 0.1 and p.eps_I == 0.0
    for code in range(10):
        assert sk.sk_error_string(code)
    assert sk.sk_error_string(999) == "unknown status"


def _init_status(d=2, n=4, m=4, eps=0.05, r=2.0, **prm):
    from paper_2201_07524_gb300 import sk
    x = np.zeros((n, max(d, 1)))
    y = np.zeros((m, max(d, 1)))
    a = np.full(n, 1.0 / max(n, 1))
    b = np.full(m, 1.0 / max(m, 1))
    p = sk.sk_default_params(**prm)
    h = ctypes.c_void_p()
    return sk._lib.sk_init(ctypes.byref(h), d, n, x.ctypes.data, a.ctypes.data, m, y.ctypes.data, b.ctypes.data,
                           eps, r, ctypes.byref(p), None), h


@pytest.mark.parametrize("kwargs", [
    dict(d=0), dict(d=4), dict(n=0), dict(m=0), dict(eps=0.0), dict(eps=-1.0), dict(r=0.5),
    dict(eps=float("nan")), dict(N=7), dict(N=6), dict(sigma=1.0), dict(sigma=1.5, N=64),
    dict(m_w=1), dict(m_w=9), dict(p=1), dict(p=13), dict(eps_B=0.0), dict(eps_B=0.5),
    dict(precision=2), dict(N=1024), dict(N=16, m_w=8),
])
def test_init_rejects_bad_arguments_on_host(kwargs):
    from paper_2201_07524_gb300 import sk
    st, h = _init_status(**kwargs)
    assert st == sk.SK_ERR_ARG
    assert not h.value


def test_null_plan_calls_are_rejected():
    from paper_2201_07524_gb300 import sk
    L = sk._lib
    assert L.sk_kernel_apply(None, 0, None, None, None) == sk.SK_ERR_ARG
    assert L.sk_solve(None, 1, 0.0, 1, None, None, None, None) == sk.SK_ERR_ARG
    assert L.sk_grad(None, None, None, None, None, None) == sk.SK_ERR_ARG
    assert L.sk_plan_info(None, None) == sk.SK_ERR_ARG
    assert L.sk_set_kernels(None, 0) == sk.SK_ERR_ARG
    assert L.sk_inject_fault(None, 0) == sk.SK_ERR_ARG
    assert L.sk_autotune(None, None, None) == sk.SK_ERR_ARG
    assert L.sk_launch_count(None) == -1
    L.sk_destroy(None)


def test_c_example_builds_and_checks_its_arguments(lib):
    # the plain-C example links against the library and rejects bad
    # arguments before touching the GPU
    import subprocess
    from paper_2201_07524_gb300 import build
    exe = build.build_example()
    assert os.path.exists(exe)
    assert subprocess.run([exe], capture_output=True).returncode == 2
    assert subprocess.run([exe, "4", "10", "10", "0.05", "3"], capture_output=True).returncode == 2
