"""Parity of sk_grad (through the C ABI) with the oracle's dual_gradient.

Tolerances: the weight gradients eps (1/2 + log u) are elementwise FP64,
1e-13 relative.  The position gradients 2 u_i (x_i (K v)_i - (K (v y))_i) take
d + 1 fast summations with signed weights v (y_t - c_t); their error is the
fast summation's relative error times the weights' l1 norm, so each
element is compared against 4 max_i(u_i) R sum_j v_j (R the radius of the
clouds around the plan's centre) times 1e-5 (FP32) / 1e-6 (FP64) -- the
E_fs targets -- and the direct method to 1e-10 of the same scale.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import sinkhorn as osk         # noqa: E402
from paper_2201_07524_gb300 import workloads as wl   # noqa: E402

sk = pytest.importorskip("paper_2201_07524_gb300.sk")

TOL = {sk.SK_FP64: 1e-6, sk.SK_FP32: 1e-5}


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def make_plan(x, y, a, b, eps, r=2.0, precision=sk.SK_FP64, **kw):
    prm = sk.sk_default_params(precision=precision, **kw)
    return sk.sk_init(cuda(x), cuda(a), cuda(y), cuda(b), eps, r, prm)


def grads(plan, n, m, d, host=False):
    if host:
        out = [np.zeros(n), np.zeros(m), np.zeros(n * d), np.zeros(m * d)]
    else:
        out = [torch.zeros(k, dtype=torch.float64, device="cuda") for k in (n, m, n * d, m * d)]
    sk.sk_grad(plan, *out)
    torch.cuda.synchronize()
    res = [o if host else o.cpu().numpy() for o in out]
    return res[0], res[1], res[2].reshape(n, d), res[3].reshape(m, d)


def pos_scale(x, y, u, v):
    allp = np.vstack([x, y])
    c = 0.5 * (allp.min(axis=0) + allp.max(axis=0))
    R = np.max(np.linalg.norm(allp - c, axis=1))
    return 4.0 * R * max(u.max() * v.sum(), v.max() * u.sum())


@pytest.mark.parametrize("d,precision", [(2, sk.SK_FP64), (3, sk.SK_FP64), (2, sk.SK_FP32), (3, sk.SK_FP32),
                                         (1, sk.SK_FP64)])
def test_grad_matches_oracle_at_a_state(d, precision):
    n, m, eps = 700, 513, 0.05
    x = wl.uniform_ball(n, d, 0.2, 71)
    y = wl.uniform_ball(m, d, 0.2, 72)
    a, b = wl.dirichlet_weights(n, 73), wl.dirichlet_weights(m, 74)
    u, v = wl.positive_vector(n, 75), wl.positive_vector(m, 76)
    plan = make_plan(x, y, a, b, eps, precision=precision, N=64)
    sk.sk_set_state(plan, cuda(u), cuda(v))
    ga, gb, gx, gy = grads(plan, n, m, d)
    ea, eb, ex, ey = osk.dual_gradient(x, y, a, b, u, v, eps, 2.0)
    assert np.max(np.abs(ga - ea)) <= 1e-13 * np.max(np.abs(ea))
    assert np.max(np.abs(gb - eb)) <= 1e-13 * np.max(np.abs(eb))
    scale = pos_scale(x, y, u, v)
    assert np.max(np.abs(ex)) > 100 * TOL[precision] * scale      # the gradient is well above the tolerance
    assert np.max(np.abs(gx - ex)) <= TOL[precision] * scale
    assert np.max(np.abs(gy - ey)) <= TOL[precision] * scale


def test_grad_after_solve_matches_oracle_and_host_buffers():
    # converged state: the gradient of the value (envelope theorem), host outputs
    w = wl.SMALL_2D
    x, y = w.points()
    a, b = w.marginals()
    plan = make_plan(x, y, a, b, w.eps, precision=sk.SK_FP64)
    sk.sk_solve(plan, 200, result=False)
    ga, gb, gx, gy = grads(plan, w.n, w.m, w.d, host=True)
    ref = osk.sinkhorn_dense(x, a, y, b, w.eps, w.r, 200)
    ea, eb, ex, ey = osk.dual_gradient(x, y, a, b, ref["u"], ref["v"], w.eps, w.r)
    # u, v agree with the oracle to the fast summation's accuracy (relative 1e-6)
    assert np.max(np.abs(ga - ea)) <= 1e-6 * w.eps
    assert np.max(np.abs(gb - eb)) <= 1e-6 * w.eps
    scale = pos_scale(x, y, ref["u"], ref["v"])
    assert np.max(np.abs(gx - ex)) <= 1e-5 * scale
    assert np.max(np.abs(gy - ey)) <= 1e-5 * scale
    # translation invariance survives the fast summation
    assert np.max(np.abs(gx.sum(axis=0) + gy.sum(axis=0))) <= 1e-5 * scale * w.n


def test_grad_direct_method():
    n, m, d, eps = 300, 200, 2, 0.05
    x = wl.uniform_ball(n, d, 0.2, 81)
    y = wl.uniform_ball(m, d, 0.2, 82)
    a, b = wl.uniform_weights(n), wl.uniform_weights(m)
    u, v = wl.positive_vector(n, 83), wl.positive_vector(m, 84)
    plan = make_plan(x, y, a, b, eps)
    sk.sk_set_method(plan, sk.SK_METHOD_DIRECT)
    sk.sk_set_state(plan, cuda(u), cuda(v))
    _, _, gx, gy = grads(plan, n, m, d)
    _, _, ex, ey = osk.dual_gradient(x, y, a, b, u, v, eps, 2.0)
    scale = pos_scale(x, y, u, v)
    assert np.max(np.abs(gx - ex)) <= 1e-10 * scale
    assert np.max(np.abs(gy - ey)) <= 1e-10 * scale


def test_grad_positions_need_r2_weights_do_not():
    n, d = 200, 3
    x = wl.uniform_ball(n, d, 0.2, 91)
    y = wl.uniform_ball(n, d, 0.2, 92)
    a = wl.uniform_weights(n)
    plan = make_plan(x, y, a, a, 0.05, r=1.0, precision=sk.SK_FP32, N=32)
    gx = torch.zeros(n * d, dtype=torch.float64, device="cuda")
    with pytest.raises(sk.SkError) as e:
        sk.sk_grad(plan, grad_x=gx)
    assert e.value.status == sk.SK_ERR_UNSUPPORTED
    ga = torch.zeros(n, dtype=torch.float64, device="cuda")
    sk.sk_grad(plan, grad_a=ga)
    u = np.ones(n)
    assert np.allclose(ga.cpu().numpy(), 0.05 * (0.5 + np.log(u)), rtol=0, atol=1e-15)
    sk.sk_grad(plan)    # nothing requested: a no-op


# ------------------------------------------------------------ divergence
def test_divergence_matches_oracle():
    # FP64 fast summation: each value to 1e-5 relative (the Sinkhorn-value
    # target), the divergence to 1e-5 of the largest of them
    n, m, d, eps, iters = 600, 450, 2, 0.05, 100
    x = wl.uniform_ball(n, d, 0.2, 101)
    y = wl.gaussian_mixture(m, d, 4, 0.05, 0.1, 102)
    a, b = wl.dirichlet_weights(n, 103), wl.dirichlet_weights(m, 104)
    prm = sk.sk_default_params(precision=sk.SK_FP64)
    sd, sxy, sxx, syy = sk.sk_divergence(cuda(x), cuda(a), cuda(y), cuda(b), eps, 2.0, iters, params=prm)
    ref = [osk.sinkhorn_dense(p, wp, q, wq, eps, 2.0, iters)["s"]
           for p, wp, q, wq in ((x, a, y, b), (x, a, x, a), (y, b, y, b))]
    for got, want in zip((sxy, sxx, syy), ref):
        assert abs(got - want) <= 1e-5 * abs(want)
    scale = max(abs(v) for v in ref)
    assert abs(sd - osk.sinkhorn_divergence(x, a, y, b, eps, 2.0, iters)) <= 1e-5 * scale
    assert sd > 0.0


def test_divergence_of_a_measure_with_itself_is_zero():
    n, d = 800, 3
    x = wl.uniform_ball(n, d, 0.2, 111)
    a = wl.dirichlet_weights(n, 112)
    sd, sxy, sxx, syy = sk.sk_divergence(cuda(x), cuda(a), cuda(x), cuda(a), 0.05, 2.0, 50,
                                         params=sk.sk_default_params(precision=sk.SK_FP32, N=32))
    # the three plans see the same inputs; spreading adds with atomics, so
    # the values agree to FP32 rounding, not bit for bit
    assert abs(sxy - sxx) <= 1e-6 * abs(sxx) and abs(sxx - syy) <= 1e-6 * abs(sxx)
    assert abs(sd) <= 1e-6 * abs(sxx)
