"""Automatic parameter choice and batched solves, through the C ABI.

Tolerances: kernel sums with automatically chosen N and m_w meet the same
E_fs targets as the fixed-parameter tests (1e-5 FP32, 1e-6 FP64); a batched
solve reproduces the solves of the same plans one by one to 1e-6 relative in
s and 1e-5 in u, v (spreading adds with atomics, so FP32 results are not
bit-identical run to run), and batches of FP64 and FP32 plans match the dense
oracle's s to 1e-5 relative (u to 1e-4 per entry).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import sinkhorn as osk         # noqa: E402
from paper_2201_07524_gb300 import workloads as wl   # noqa: E402

sk = pytest.importorskip("paper_2201_07524_gb300.sk")

TOL_FS = {sk.SK_FP64: 1e-6, sk.SK_FP32: 1e-5}


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def auto_plan(x, y, a, b, eps, precision):
    prm = sk.sk_default_params(precision=precision)
    prm.N = 0
    prm.m_w = 0
    return sk.sk_init(cuda(x), cuda(a), cuda(y), cuda(b), eps, 2.0, prm)


@pytest.mark.parametrize("d,eps,precision", [(1, 0.005, sk.SK_FP64), (2, 0.01, sk.SK_FP32), (2, 0.1, sk.SK_FP64),
                                             (3, 0.02, sk.SK_FP32), (3, 0.1, sk.SK_FP32), (3, 0.05, sk.SK_FP64)])
def test_auto_parameters_meet_targets(d, eps, precision):
    n, m = 900, 700
    x = wl.uniform_ball(n, d, 0.2, 141)
    y = wl.uniform_ball(m, d, 0.2, 142)
    plan = auto_plan(x, y, wl.uniform_weights(n), wl.uniform_weights(m), eps, precision)
    info = sk.sk_plan_info(plan)
    assert info["N"] >= 16 and info["N"] & (info["N"] - 1) == 0 and info["m_w"] >= 2
    v = wl.positive_vector(m, 143)
    out = torch.zeros(n, dtype=torch.float64, device="cuda")
    sk.sk_kernel_apply(plan, 0, cuda(v), out)
    exact = osk.kernel_apply(x, y, v, eps, 2.0)
    err = float(np.max(np.abs(out.cpu().numpy() - exact)) / np.max(np.abs(exact)))
    assert err <= TOL_FS[precision], (info["N"], info["m_w"], err)


def _problems(count, seed, lo=500, hi=5000):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        d = int(rng.integers(2, 4))
        n, m = (int(np.exp(rng.uniform(np.log(lo), np.log(hi)))) for _ in range(2))
        eps = float(rng.uniform(0.01, 0.1))
        x = wl.uniform_ball(n, d, 0.2, seed * 1000 + 2 * k)
        y = wl.uniform_ball(m, d, 0.2, seed * 1000 + 2 * k + 1)
        out.append((x, y, wl.uniform_weights(n), wl.uniform_weights(m), eps))
    return out


def test_solve_batch_matches_solves_one_by_one():
    probs = _problems(12, 151)
    batch = [auto_plan(*p, sk.SK_FP32) for p in probs]
    alone = [auto_plan(*p, sk.SK_FP32) for p in probs]
    st, res = sk.sk_solve_batch(batch, 20)
    assert st == sk.SK_OK
    for plan_b, plan_a, rb, p in zip(batch, alone, res, probs):
        _, ra = sk.sk_solve(plan_a, 20)
        assert rb["iters"] == 20 and sk.sk_get_state(plan_b) == 20
        assert abs(rb["s"] - ra["s"]) <= 1e-6 * abs(ra["s"])
        ub = torch.zeros(len(p[0]), dtype=torch.float64, device="cuda")
        ua = torch.zeros(len(p[0]), dtype=torch.float64, device="cuda")
        sk.sk_get_state(plan_b, u=ub)
        sk.sk_get_state(plan_a, u=ua)
        assert float(torch.max(torch.abs(ub - ua) / ua)) <= 1e-5


def test_solve_batch_matches_oracle_fp64():
    probs = _problems(3, 161, lo=300, hi=900)
    plans = [auto_plan(*p, sk.SK_FP64) for p in probs]
    st, res = sk.sk_solve_batch(plans, 30)
    assert st == sk.SK_OK
    for (x, y, a, b, eps), r in zip(probs, res):
        ref = osk.sinkhorn_dense(x, a, y, b, eps, 2.0, 30)
        assert abs(r["s"] - ref["s"]) <= 1e-5 * abs(ref["s"])
    # a second call continues from the state the first left
    st, res2 = sk.sk_solve_batch(plans, 10)
    for (x, y, a, b, eps), r in zip(probs, res2):
        ref = osk.sinkhorn_dense(x, a, y, b, eps, 2.0, 40)
        assert abs(r["s"] - ref["s"]) <= 1e-5 * abs(ref["s"])


def test_solve_batch_fp32_and_mixed_d_match_oracle_per_problem():
    # one batch of FP32 and FP64 plans in d = 1, 2, 3, uneven n and m, eps in
    # [0.01, 0.1]: every problem's value and scaling vector against the dense
    # FP64 oracle after the same iteration count (value to 1e-5 relative, the
    # tolerance of the single solves; u to 1e-4 relative per entry)
    rng = np.random.default_rng(181)
    probs = []
    for k, (d, precision) in enumerate([(1, sk.SK_FP32), (2, sk.SK_FP32), (3, sk.SK_FP32), (2, sk.SK_FP64),
                                        (3, sk.SK_FP32), (1, sk.SK_FP64), (3, sk.SK_FP64), (2, sk.SK_FP32)]):
        n, m = (int(np.exp(rng.uniform(np.log(300), np.log(2500)))) for _ in range(2))
        eps = float(rng.uniform(0.01, 0.1))
        x = wl.uniform_ball(n, d, 0.2, 1810 + 2 * k)
        y = wl.uniform_ball(m, d, 0.2, 1811 + 2 * k)
        a, b = wl.dirichlet_weights(n, 1850 + k), wl.uniform_weights(m)
        probs.append((x, y, a, b, eps, precision))
    plans = [auto_plan(x, y, a, b, eps, precision) for x, y, a, b, eps, precision in probs]
    st, res = sk.sk_solve_batch(plans, 30)
    assert st == sk.SK_OK
    for (x, y, a, b, eps, precision), plan, r in zip(probs, plans, res):
        ref = osk.sinkhorn_dense(x, a, y, b, eps, 2.0, 30)
        assert abs(r["s"] - ref["s"]) <= 1e-5 * abs(ref["s"]), (x.shape, precision, r["s"], ref["s"])
        u = np.zeros(len(x))
        sk.sk_get_state(plan, u=u)
        assert np.max(np.abs(u - ref["u"]) / ref["u"]) <= 1e-4, (x.shape, precision)


def test_solve_batch_rejects_bad_arguments():
    x = wl.uniform_ball(300, 2, 0.2, 171)
    a = wl.uniform_weights(300)
    plan = auto_plan(x, x, a, a, 0.05, sk.SK_FP32)
    st, _ = sk.sk_solve_batch([plan, plan], 3, raise_on_error=False)
    assert st == sk.SK_ERR_ARG
    sk.sk_stage_times(plan, 1)
    st, _ = sk.sk_solve_batch([plan], 3, raise_on_error=False)
    assert st == sk.SK_ERR_ARG
    sk.sk_stage_times(plan, 0)
    st, _ = sk.sk_solve_batch([plan], 3)
    assert st == sk.SK_OK
