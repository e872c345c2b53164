"""The no-allocation entry point, sk_direct_residual_noalloc.

It is for callers that may not allocate device memory (a framework's memory
pool owns the GPU's memory, or the service must not allocate after start-up):
they pass every input and output buffer, and the function keeps its
reduction scratch in a fixed device array inside the library.  These tests
call it through the C ABI and compare it with the plan-based direct method
(sk_kernel_apply with SK_METHOD_DIRECT) within the FP32 direct-summation
tolerance of the other tests (1e-5 relative per element), on two calls in a
row so the shared scratch is reused.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2201_07524_gb300 import workloads as wl   # noqa: E402

sk = pytest.importorskip("paper_2201_07524_gb300.sk")

TOL = 1e-5


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def _call(x, u, a, y, v, eps, r, t_out, stats):
    n, d = x.shape
    m = y.shape[0]
    return sk._lib.sk_direct_residual_noalloc(d, n, x.data_ptr(), u.data_ptr(), a.data_ptr(), m, y.data_ptr(),
                                              v.data_ptr(), eps, r, t_out.data_ptr(), stats.data_ptr(), None)


@pytest.mark.parametrize("d,r,n,m", [(3, 2.0, 3001, 2499), (2, 1.0, 3001, 2499), (1, 2.0, 3001, 2499),
                                     (3, 1.5, 3001, 2499),
                                     # n at the scratch limit: 4096 blocks share the ticket and the partials
                                     (3, 2.0, 2097152, 300)])
def test_noalloc_matches_plan_direct_method_twice(d, r, n, m):
    eps = 0.02
    xh = wl.uniform_ball(n, d, 0.2, 91)
    yh = wl.uniform_ball(m, d, 0.2, 92)
    ah, bh = wl.uniform_weights(n), wl.uniform_weights(m)
    plan = sk.sk_init(_dev(xh), _dev(ah), _dev(yh), _dev(bh), eps, r, sk.sk_default_params(precision=sk.SK_FP32))
    sk.sk_set_method(plan, sk.SK_METHOD_DIRECT)
    x, y, a = _dev(xh), _dev(yh), _dev(ah)
    t_out = torch.zeros(n, dtype=torch.float64, device="cuda")
    stats = torch.zeros(2, dtype=torch.float64, device="cuda")
    for call, seed in enumerate((93, 94)):       # two calls in a row share the scratch
        vh = wl.positive_vector(m, seed)
        uh = wl.positive_vector(n, seed + 10, low=1e-3, high=2e-3)
        want = np.zeros(n)
        sk.sk_kernel_apply(plan, 0, vh, want)     # existing entry point, host output
        st = _call(x, _dev(uh), a, y, _dev(vh), eps, r, t_out, stats)
        assert st == sk.SK_OK, sk.sk_error_string(st)
        torch.cuda.synchronize()
        got = t_out.cpu().numpy()
        assert np.max(np.abs(got - want) / want) <= TOL, call
        res2 = np.sum((uh * want - ah) ** 2)
        dot = np.sum(uh * want)
        s = stats.cpu().numpy()
        assert abs(s[0] - res2) <= TOL * res2, call
        assert abs(s[1] - dot) <= TOL * dot, call
    plan.close()


def test_noalloc_rejects_oversize_and_host_buffers():
    x = _dev(np.zeros((4, 2)))
    one = _dev(np.ones(4))
    t_out = torch.zeros(4, dtype=torch.float64, device="cuda")
    stats = torch.zeros(2, dtype=torch.float64, device="cuda")
    lib = sk._lib
    # n beyond the fixed scratch: rejected before any GPU work touches the buffers
    too_many = 2097152 + 1
    st = lib.sk_direct_residual_noalloc(2, too_many, x.data_ptr(), one.data_ptr(), one.data_ptr(), 4, x.data_ptr(),
                                        one.data_ptr(), 0.05, 2.0, t_out.data_ptr(), stats.data_ptr(), None)
    assert st == sk.SK_ERR_TOO_LARGE
    assert "scratch" in sk.sk_error_string(st)
    # host buffers are not accepted (copying them would need device memory)
    host = np.zeros(8)
    st = lib.sk_direct_residual_noalloc(2, 4, host.ctypes.data, one.data_ptr(), one.data_ptr(), 4, x.data_ptr(),
                                        one.data_ptr(), 0.05, 2.0, t_out.data_ptr(), stats.data_ptr(), None)
    assert st == sk.SK_ERR_ARG


def test_noalloc_rejects_overlapping_outputs():
    n, m = 64, 32
    x = _dev(wl.uniform_ball(n, 2, 0.2, 5))
    y = _dev(wl.uniform_ball(m, 2, 0.2, 6))
    u, a = _dev(np.ones(n)), _dev(np.full(n, 1.0 / n))
    v = _dev(np.ones(m))
    t_out = torch.zeros(n, dtype=torch.float64, device="cuda")
    stats = torch.zeros(2, dtype=torch.float64, device="cuda")
    lib = sk._lib
    # t_out on top of u, then stats_out inside t_out: refused on the host, nothing launched
    st = lib.sk_direct_residual_noalloc(2, n, x.data_ptr(), u.data_ptr(), a.data_ptr(), m, y.data_ptr(),
                                        v.data_ptr(), 0.05, 2.0, u.data_ptr(), stats.data_ptr(), None)
    assert st == sk.SK_ERR_ARG
    st = lib.sk_direct_residual_noalloc(2, n, x.data_ptr(), u.data_ptr(), a.data_ptr(), m, y.data_ptr(),
                                        v.data_ptr(), 0.05, 2.0, t_out.data_ptr(), t_out.data_ptr() + 8, None)
    assert st == sk.SK_ERR_ARG
    # pinned host memory is not device memory either
    pinned = torch.zeros(n, dtype=torch.float64).pin_memory()
    st = lib.sk_direct_residual_noalloc(2, n, x.data_ptr(), u.data_ptr(), a.data_ptr(), m, y.data_ptr(),
                                        v.data_ptr(), 0.05, 2.0, pinned.data_ptr(), stats.data_ptr(), None)
    assert st == sk.SK_ERR_ARG
