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


def test_divergence_gradient_matches_oracle():
    n, m, d, eps, iters = 500, 400, 2, 0.05, 300
    x = wl.gaussian_mixture(n, d, 4, 0.05, 0.1, 121)
    y = wl.uniform_ball(m, d, 0.2, 122)
    a, b = wl.dirichlet_weights(n, 123), wl.dirichlet_weights(m, 124)
    g = [torch.zeros(k, dtype=torch.float64, device="cuda") for k in (n, m, n * d, m * d)]
    sk.sk_divergence(cuda(x), cuda(a), cuda(y), cuda(b), eps, 2.0, iters,
                     params=sk.sk_default_params(precision=sk.SK_FP64), grad_a=g[0], grad_b=g[1], grad_x=g[2],
                     grad_y=g[3])
    ga, gb, gx, gy = (t.cpu().numpy() for t in g)
    ea, eb, ex, ey = osk.sinkhorn_divergence_gradient(x, a, y, b, eps, 2.0, iters)
    # the weight gradients are defined up to a constant on each side's simplex
    for got, want in ((ga, ea), (gb, eb)):
        assert np.max(np.abs((got - got.mean()) - (want - want.mean()))) <= 1e-6 * eps
    o = osk.sinkhorn_dense(x, a, y, b, eps, 2.0, iters)
    _, _, tx, ty = osk.dual_gradient(x, y, a, b, o["u"], o["v"], eps, 2.0)
    scale = max(np.max(np.abs(tx)), np.max(np.abs(ty)))     # one term's size
    assert np.max(np.abs(gx.reshape(n, d) - ex)) <= 1e-5 * scale
    assert np.max(np.abs(gy.reshape(m, d) - ey)) <= 1e-5 * scale


def test_divergence_autograd_matches_direct_gradients():
    # torch.autograd over the divergence returns the gradients sk_divergence
    # computes, scaled by the incoming gradient
    n, m, d, eps, iters = 300, 250, 3, 0.05, 100
    x = cuda(wl.gaussian_mixture(n, d, 4, 0.05, 0.1, 141)).requires_grad_()
    y = cuda(wl.uniform_ball(m, d, 0.2, 142)).requires_grad_()
    a = cuda(wl.dirichlet_weights(n, 143)).requires_grad_()
    b = cuda(wl.dirichlet_weights(m, 144)).requires_grad_()
    prm = sk.sk_default_params(precision=sk.SK_FP64)
    sd = sk.sinkhorn_divergence(x, a, y, b, eps, 2.0, iters, params=prm)
    (3.0 * sd).backward()
    g = [torch.zeros(k, dtype=torch.float64, device="cuda") for k in (n, m, n * d, m * d)]
    ref = sk.sk_divergence(x.detach(), a.detach(), y.detach(), b.detach(), eps, 2.0, iters, params=prm,
                           grad_a=g[0], grad_b=g[1], grad_x=g[2], grad_y=g[3])
    # two separate solves: spreading adds with atomics, so agreement to rounding
    assert abs(float(sd.detach()) - ref[0]) <= 1e-12 * abs(ref[0])
    for got, want in ((a.grad, g[0]), (b.grad, g[1]), (x.grad.reshape(-1), g[2]), (y.grad.reshape(-1), g[3])):
        assert torch.allclose(got, 3.0 * want, rtol=0, atol=1e-10 * float(want.abs().max()))


def test_divergence_gradient_finite_differences():
    # the differentiation check on Gaussian-mixture clouds in 3-D (r = 2,
    # eps = 0.02): central differences with step 1e-4 of the divergence,
    # every solve converged (row residual <= 1e-13), on 64 random position
    # coordinates and two simplex directions of the weights.  FP64 plans.
    n = m = 1024
    d, eps, h = 3, 0.02, 1e-4
    x = wl.gaussian_mixture(n, d, 8, 0.03, 0.15, 131)
    y = wl.uniform_ball(m, d, 0.2, 132)
    a, b = wl.uniform_weights(n), wl.uniform_weights(m)
    prm = sk.sk_default_params(precision=sk.SK_FP64)

    def sd(xx, aa, yy, bb, grads=None):
        kw = {} if grads is None else dict(grad_a=grads[0], grad_b=grads[1], grad_x=grads[2], grad_y=grads[3])
        return sk.sk_divergence(cuda(xx), cuda(aa), cuda(yy), cuda(bb), eps, 2.0, 20000, tol=1e-13, params=prm,
                                **kw)[0]

    g = [np.zeros(k) for k in (n, m, n * d, m * d)]
    sd(x, a, y, b, g)
    gx, gy = g[2].reshape(n, d), g[3].reshape(m, d)
    rng = np.random.default_rng(133)
    worst = 0.0
    for k in range(64):
        arr, grad = (x, gx) if k % 2 == 0 else (y, gy)
        i, t = int(rng.integers(len(arr))), int(rng.integers(d))
        old = arr[i, t]
        arr[i, t] = old + h
        sp = sd(x, a, y, b)
        arr[i, t] = old - h
        sm = sd(x, a, y, b)
        arr[i, t] = old
        worst = max(worst, abs((sp - sm) / (2 * h) - grad[i, t]))
    scale = max(np.max(np.abs(gx)), np.max(np.abs(gy)))
    assert worst <= 1e-3 * scale
    for w, grad, first in ((a, g[0], True), (b, g[1], False)):
        dlt = rng.standard_normal(len(w))
        dlt -= dlt.mean()
        dlt *= 1e-3 * w.min() / np.max(np.abs(dlt))   # keeps the weights positive
        if first:
            sp, sm = sd(x, a + dlt, y, b), sd(x, a - dlt, y, b)
        else:
            sp, sm = sd(x, a, y, b + dlt), sd(x, a, y, b - dlt)
        assert abs((sp - sm) / 2 - float(grad @ dlt)) <= 1e-3 * abs(float(grad @ dlt)) + 1e-12
