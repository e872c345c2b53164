"""The log-domain iteration (Alg. 4, sk_set_domain) through the C ABI.

Tolerances: the log domain returns the value of the scaling domain at the
same plan and iteration count to 1e-6 relative (FP32; the two forms round
differently) and 1e-10 (FP64), and matches the FP64 log-sum-exp oracle to the
fast summation's accuracy (1e-6 relative in s, 1e-6 eps in the potentials).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import sinkhorn as osk         # noqa: E402
from paper_2201_07524_gb300 import workloads as wl   # noqa: E402

sk = pytest.importorskip("paper_2201_07524_gb300.sk")


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def make(x, y, a, b, eps, precision, N=64):
    prm = sk.sk_default_params(precision=precision, N=N)
    return sk.sk_init(cuda(x), cuda(a), cuda(y), cuda(b), eps, 2.0, prm)


def state(plan, n, m):
    u = torch.zeros(n, dtype=torch.float64, device="cuda")
    v = torch.zeros(m, dtype=torch.float64, device="cuda")
    sk.sk_get_state(plan, u=u, v=v)
    return u.cpu().numpy(), v.cpu().numpy()


@pytest.mark.parametrize("d,precision,tol", [(2, sk.SK_FP64, 1e-10), (3, sk.SK_FP32, 1e-6)])
def test_log_domain_matches_scaling_domain(d, precision, tol):
    n, m, eps = 3000, 2500, 0.03
    x = wl.uniform_ball(n, d, 0.2, 181)
    y = wl.gaussian_mixture(m, d, 4, 0.05, 0.1, 182)
    a, b = wl.dirichlet_weights(n, 183), wl.dirichlet_weights(m, 184)
    ps = make(x, y, a, b, eps, precision)
    pl = make(x, y, a, b, eps, precision)
    sk.sk_set_domain(pl, sk.SK_DOMAIN_LOG)
    _, rs = sk.sk_solve(ps, 40)
    _, rl = sk.sk_solve(pl, 40)
    assert abs(rl["s"] - rs["s"]) <= tol * abs(rs["s"])
    # the residuals agree down to each precision's noise floor, where the two
    # forms round differently (FP32 kernel sums: a few 1e-9 on these marginals)
    floor = 1e-12 if precision == sk.SK_FP64 else 5e-9
    assert abs(rl["err_row"] - rs["err_row"]) <= 1e-3 * rs["err_row"] + floor
    us, vs = state(ps, n, m)
    bl, gl = state(pl, n, m)
    assert np.max(np.abs(bl - eps * (np.log(us) + 0.5))) <= 10 * tol * eps * max(1.0, np.max(np.abs(np.log(us))))
    assert np.max(np.abs(gl - eps * (np.log(vs) + 0.5))) <= 10 * tol * eps * max(1.0, np.max(np.abs(np.log(vs))))


def test_log_domain_matches_log_oracle_from_zero_potentials():
    n, m, d, eps, it = 500, 400, 2, 0.02, 50
    x = wl.uniform_ball(n, d, 0.2, 191)
    y = wl.uniform_ball(m, d, 0.2, 192)
    a, b = wl.uniform_weights(n), wl.uniform_weights(m)
    plan = make(x, y, a, b, eps, sk.SK_FP64)
    sk.sk_set_domain(plan, sk.SK_DOMAIN_LOG)
    sk.sk_set_state(plan, cuda(np.zeros(n)), cuda(np.zeros(m)))       # the Set line of Alg. 4
    _, res = sk.sk_solve(plan, it)
    ref = osk.sinkhorn_log_dense(x, a, y, b, eps, 2.0, it)
    beta, gamma = state(plan, n, m)
    assert abs(res["s"] - ref["s"]) <= 1e-6 * abs(ref["s"])
    assert np.max(np.abs(beta - ref["beta"])) <= 1e-6 * eps
    assert np.max(np.abs(gamma - ref["gamma"])) <= 1e-6 * eps


def test_log_domain_survives_an_extreme_gauge():
    # (u, c v) and (u / c, c v) give the same iterates up to the gauge c, and
    # so the same value; with v = 1e-50 the scaling form's FP32 weights
    # underflow to zero, the log form's weights are shifted to at most e^(-1/2)
    n, m, d, eps = 2000, 1800, 3, 0.05
    x = wl.uniform_ball(n, d, 0.2, 201)
    y = wl.uniform_ball(m, d, 0.2, 202)
    a, b = wl.uniform_weights(n), wl.uniform_weights(m)
    ref = make(x, y, a, b, eps, sk.SK_FP32)
    _, rref = sk.sk_solve(ref, 30)
    tiny = 1e-50 * wl.positive_vector(m, 203)
    bad = make(x, y, a, b, eps, sk.SK_FP32)
    sk.sk_set_state(bad, cuda(np.ones(n)), cuda(tiny))
    st, _ = sk.sk_solve(bad, 30, raise_on_error=False)
    assert st == sk.SK_ERR_UNDERFLOW
    good = make(x, y, a, b, eps, sk.SK_FP32)
    sk.sk_set_state(good, cuda(np.ones(n)), cuda(tiny))
    sk.sk_set_domain(good, sk.SK_DOMAIN_LOG)
    st, res = sk.sk_solve(good, 30)
    assert st == sk.SK_OK
    assert abs(res["s"] - rref["s"]) <= 1e-5 * abs(rref["s"])


def test_log_domain_gradient_and_round_trip():
    n, m, d, eps = 700, 600, 2, 0.05
    x = wl.uniform_ball(n, d, 0.2, 211)
    y = wl.uniform_ball(m, d, 0.2, 212)
    a, b = wl.dirichlet_weights(n, 213), wl.dirichlet_weights(m, 214)
    plan = make(x, y, a, b, eps, sk.SK_FP64)
    sk.sk_solve(plan, 20, result=False)
    g1 = [np.zeros(k) for k in (n, m, n * d, m * d)]
    sk.sk_grad(plan, *g1)
    u0, v0 = state(plan, n, m)
    sk.sk_set_domain(plan, sk.SK_DOMAIN_LOG)
    g2 = [np.zeros(k) for k in (n, m, n * d, m * d)]
    sk.sk_grad(plan, *g2)
    for p, q in zip(g1, g2):
        assert np.max(np.abs(p - q)) <= 1e-9 * np.max(np.abs(p))
    sk.sk_set_domain(plan, sk.SK_DOMAIN_SCALING)
    u1, v1 = state(plan, n, m)
    assert np.max(np.abs(u1 / u0 - 1)) <= 1e-13 and np.max(np.abs(v1 / v0 - 1)) <= 1e-13


def test_log_domain_in_a_batch():
    n, d, eps = 1500, 2, 0.04
    x = wl.uniform_ball(n, d, 0.2, 221)
    y = wl.uniform_ball(n, d, 0.2, 222)
    a = wl.uniform_weights(n)
    p1, p2 = make(x, y, a, a, eps, sk.SK_FP32), make(x, y, a, a, eps, sk.SK_FP32)
    sk.sk_set_domain(p2, sk.SK_DOMAIN_LOG)
    st, res = sk.sk_solve_batch([p1, p2], 25)
    assert st == sk.SK_OK
    assert abs(res[0]["s"] - res[1]["s"]) <= 1e-6 * abs(res[0]["s"])
