"""Pins for oracle.sinkhorn: closed forms, invariants and brute force that fix
what Alg. 1 and the kernel products compute, independently of the oracle code."""
import math

import numpy as np
import pytest

from oracle import lp
from oracle import sinkhorn as osk
from paper_2201_07524_gb300 import workloads as wl


# ---------------------------------------------------------------- Gibbs kernel

def test_gibbs_kernel_hand_values():
    # rows are sources x_i, columns targets y_j; distance 0.5 = |(0.3, 0.4)|
    x = np.array([[0.0, 0.0], [1.0, 0.0]])
    y = np.array([[0.3, 0.4], [0.0, 0.0], [1.0, 2.0]])
    K1 = osk.gibbs_kernel(x, y, eps=0.5, r=1.0)
    assert K1.shape == (2, 3)
    assert K1[0, 0] == pytest.approx(math.exp(-1.0), rel=1e-15)
    assert K1[0, 1] == 1.0
    assert K1[1, 2] == pytest.approx(math.exp(-2.0 / 0.5), rel=1e-15)
    d10 = math.hypot(1.0 - 0.3, 0.0 - 0.4)
    K2 = osk.gibbs_kernel(x, y, eps=0.25, r=2.0)
    assert K2[0, 0] == pytest.approx(math.exp(-1.0), rel=1e-15)
    assert K2[1, 0] == pytest.approx(math.exp(-d10 ** 2 / 0.25), rel=1e-14)
    K3 = osk.gibbs_kernel(x, y, eps=0.1, r=1.5)
    assert K3[1, 0] == pytest.approx(math.exp(-d10 ** 1.5 / 0.1), rel=1e-14)


def test_gibbs_kernel_gaussian_factorization():
    # r = 2: exp(-|x-y|^2/eps) = exp(-|x|^2/eps) exp(-|y|^2/eps) exp(2 x.y/eps)
    x = wl.uniform_ball(7, 3, 0.2, 11)
    y = wl.uniform_ball(5, 3, 0.2, 12)
    eps = 0.07
    fact = (np.exp(-np.sum(x * x, 1) / eps)[:, None] * np.exp(-np.sum(y * y, 1) / eps)[None, :]
            * np.exp(2.0 * (x @ y.T) / eps))
    np.testing.assert_allclose(osk.gibbs_kernel(x, y, eps, 2.0), fact, rtol=1e-13)


# ---------------------------------------------------------------- kernel products

def test_kernel_apply_unit_vectors_give_columns():
    x = wl.uniform_ball(9, 2, 0.2, 3)
    y = wl.uniform_ball(4, 2, 0.2, 4)
    eps, r = 0.03, 1.0
    for j in range(4):
        e = np.zeros(4)
        e[j] = 1.0
        t = osk.kernel_apply(x, y, e, eps, r, chunk=4)
        for i in range(9):
            dist = math.sqrt((x[i, 0] - y[j, 0]) ** 2 + (x[i, 1] - y[j, 1]) ** 2)
            assert t[i] == pytest.approx(math.exp(-dist / eps), rel=1e-14)
        tt = osk.kernel_apply_T(x, y, np.eye(9)[2], eps, r)
        assert tt[j] == pytest.approx(math.exp(-math.dist(x[2], y[j]) / eps), rel=1e-14)


@pytest.mark.parametrize("r,eps,exact", [
    # r = 2: the lattice sum of a well-resolved Gaussian equals its integral sqrt(pi eps)
    (2.0, 0.01, math.sqrt(math.pi * 0.01)),
    # r = 1: geometric series, sum_j h exp(-|j| h / eps) = h coth(h / (2 eps))
    (1.0, 0.05, 1e-4 / math.tanh(1e-4 / (2 * 0.05)))])
def test_kernel_apply_lattice_sum_1d(r, eps, exact):
    h = 1e-4
    y = (np.arange(-20000, 20001) * h)[:, None]
    x = np.array([[0.0]])
    t = osk.kernel_apply(x, y, np.full(len(y), h), eps, r)
    assert t[0] == pytest.approx(exact, rel=2e-7)


def test_kernel_apply_riemann_sum_2d_gaussian():
    # integral over R^2 of exp(-|y|^2/eps) = pi eps
    h = 2e-3
    g = np.arange(-300, 301) * h
    Y = np.stack(np.meshgrid(g, g, indexing="ij"), -1).reshape(-1, 2)
    t = osk.kernel_apply(np.array([[0.0, 0.0]]), Y, np.full(len(Y), h * h), 0.01, 2.0)
    assert t[0] == pytest.approx(math.pi * 0.01, rel=1e-10)


# ---------------------------------------------------------------- Alg. 1

def test_single_point_value_is_cost():
    x = np.array([[0.1, -0.05]])
    y = np.array([[-0.02, 0.13]])
    for r in (1.0, 2.0):
        res = osk.sinkhorn_dense(x, [1.0], y, [1.0], eps=0.05, r=r, iters=3)
        c = math.dist(x[0], y[0]) ** r
        assert res["s"] == pytest.approx(c, rel=1e-13)
        assert res["s_tilde"] == pytest.approx(c, rel=1e-13)
        assert res["H_pi"] == pytest.approx(0.0, abs=1e-14)


def test_two_by_two_closed_form():
    # Uniform marginals force pi = [[q, 1/2-q], [1/2-q, q]]; optimality of
    # pi = diag(u) K diag(v) gives q^2 / (1/2-q)^2 = K11 K22 / (K12 K21).
    x = np.array([[0.0], [0.3]])
    y = np.array([[0.05], [0.2]])
    eps, r = 0.04, 2.0
    C = (x - y.T) ** 2
    kappa = math.exp(-(C[0, 0] + C[1, 1] - C[0, 1] - C[1, 0]) / eps)
    q = math.sqrt(kappa) / (2 * (1 + math.sqrt(kappa)))
    pi = np.array([[q, 0.5 - q], [0.5 - q, q]])
    primal = float(np.sum(pi * C)) + eps * float(np.sum(pi * np.log(pi)))
    res = osk.sinkhorn_dense(x, [0.5, 0.5], y, [0.5, 0.5], eps, r, iters=200)
    np.testing.assert_allclose(res["pi"], pi, rtol=1e-12)
    assert res["s"] == pytest.approx(primal, rel=1e-12)


def _problem(n, m, d, seed, weights="dirichlet"):
    x = wl.uniform_ball(n, d, 0.2, seed)
    y = wl.uniform_ball(m, d, 0.2, seed + 1)
    if weights == "dirichlet":
        a, b = wl.dirichlet_weights(n, seed + 2), wl.dirichlet_weights(m, seed + 3)
    else:
        a, b = wl.uniform_weights(n), wl.uniform_weights(m)
    return x, a, y, b


def test_half_steps_make_one_marginal_exact():
    # After a u-update the row marginal is exact, after a v-update the column one.
    x, a, y, b = _problem(30, 40, 2, 5)
    res = osk.sinkhorn_dense(x, a, y, b, 0.05, 2.0, iters=6, record=True)
    K = res["K"]
    for step, (u, v) in enumerate(res["history"][1:], start=1):
        row, col = osk.marginal_residuals(u, v, a, b, K)
        if step % 2 == 1:
            assert row < 1e-15
        else:
            assert col < 1e-15


def test_objective_decrease_equals_kl_sum():
    # Lemma "Sinkhorniteration1": f(Delta) - f(Delta+1) = KL(p|pi 1) + KL(p~|pi^T 1), Delta >= 1.
    x, a, y, b = _problem(25, 20, 2, 8)
    res = osk.sinkhorn_dense(x, a, y, b, 0.03, 2.0, iters=8, record=True)
    K = res["K"]
    hist = res["history"]
    for delta in range(1, len(hist) - 1):
        u0, v0 = hist[delta]
        u1, v1 = hist[delta + 1]
        drop = osk.objective_f(u0, v0, a, b, K) - osk.objective_f(u1, v1, a, b, K)
        pi = osk.transport_plan(u0, v0, K)
        kl = osk.kl_divergence(a, pi.sum(1)) + osk.kl_divergence(b, pi.sum(0))
        assert drop >= -1e-15
        assert drop == pytest.approx(kl, rel=1e-9, abs=1e-15)


def test_dual_value_equals_primal_at_convergence():
    # s = eps(<a, log u> + <b, log v> + 1 - u^T K v) equals <pi, C> - eps H(pi)
    # once the marginals hold (Prop. "dual representation", vanishing duality gap).
    x, a, y, b = _problem(40, 30, 3, 13)
    eps = 0.05
    res = osk.sinkhorn_dense(x, a, y, b, eps, 2.0, iters=500)
    assert res["err_row"] < 1e-13
    primal = res["s_tilde"] - eps * res["H_pi"]
    assert res["s"] == pytest.approx(primal, rel=1e-11)
    K = res["K"]
    assert osk.dual_objective(res["u"], res["v"], a, b, K, eps) == pytest.approx(res["s"], rel=1e-12)


def test_sandwich_with_bruteforce_lp():
    # Lemma "Quality of the Sinkhorn approximation": s <= w_r <= s~ <= s + eps (H(P) + H(P~)).
    rng_seeds = [21, 22, 23]
    for seed in rng_seeds:
        x, a, y, b = _problem(6, 6, 2, seed, weights="uniform")
        for eps in (0.002, 0.02, 0.2):
            res = osk.sinkhorn_dense(x, a, y, b, eps, 2.0, iters=4000)
            w = lp.wasserstein_r_uniform(x, y, 2.0)
            assert res["s"] <= w + 1e-12
            assert w <= res["s_tilde"] + 1e-12
            assert res["s_tilde"] <= res["s"] + eps * (osk.entropy(a) + osk.entropy(b)) + 1e-12


def test_small_eps_approaches_lp():
    x, a, y, b = _problem(5, 5, 2, 31, weights="uniform")
    w = lp.wasserstein_r_uniform(x, y, 1.0)
    gaps = []
    for eps in (0.02, 0.005, 0.001):
        res = osk.sinkhorn_dense(x, a, y, b, eps, 1.0, iters=20000)
        gaps.append(abs(res["s_tilde"] - w))
    assert gaps[-1] < 1e-6
    assert gaps[0] > gaps[-1]


def test_large_eps_limit_is_independent_coupling():
    # eps -> inf: pi -> a b^T, so s + eps (H(a) + H(b)) -> sum_ij a_i b_j C_ij.
    x, a, y, b = _problem(12, 9, 2, 41)
    C = osk.cost_matrix(x, y, 2.0)
    indep = float(a @ C @ b)
    errs = []
    for eps in (1e2, 1e3, 1e4):
        res = osk.sinkhorn_dense(x, a, y, b, eps, 2.0, iters=50)
        errs.append(abs(res["s"] + eps * (osk.entropy(a) + osk.entropy(b)) - indep))
    assert errs[2] < 1e-5 * indep
    assert errs[0] > errs[1] > errs[2]


def test_swap_symmetry_and_permutation_invariance():
    x, a, y, b = _problem(20, 15, 2, 51)
    eps = 0.04
    s1 = osk.sinkhorn_dense(x, a, y, b, eps, 2.0, iters=800)
    s2 = osk.sinkhorn_dense(y, b, x, a, eps, 2.0, iters=800)
    assert s1["s"] == pytest.approx(s2["s"], rel=1e-11)
    perm = np.random.default_rng(0).permutation(20)
    s3 = osk.sinkhorn_dense(x[perm], a[perm], y, b, eps, 2.0, iters=800)
    assert s3["s"] == pytest.approx(s1["s"], rel=1e-11)
    np.testing.assert_allclose(s3["u"], s1["u"][perm], rtol=1e-9)


def test_translation_rule_for_squared_cost():
    # C'_ij = |x_i - y_j - t|^2 = C_ij - 2 <x_i - y_j, t> + |t|^2; the shift is constant
    # on couplings with fixed marginals, so s' = s - 2 <E_a x - E_b y, t> + |t|^2.
    x, a, y, b = _problem(18, 22, 2, 61)
    t = np.array([0.03, -0.02])
    eps = 0.05
    s0 = osk.sinkhorn_dense(x, a, y, b, eps, 2.0, iters=800)["s"]
    s1 = osk.sinkhorn_dense(x, a, y + t, b, eps, 2.0, iters=800)["s"]
    pred = s0 - 2 * float((a @ x - b @ y) @ t) + float(t @ t)
    assert s1 == pytest.approx(pred, rel=1e-10)


def test_matrix_free_matches_dense():
    x, a, y, b = _problem(33, 27, 3, 71)
    d = osk.sinkhorn_dense(x, a, y, b, 0.03, 1.0, iters=20)
    f = osk.sinkhorn_matrix_free(x, a, y, b, 0.03, 1.0, iters=20)
    np.testing.assert_allclose(f["u"], d["u"], rtol=1e-12)
    np.testing.assert_allclose(f["v"], d["v"], rtol=1e-12)
    assert f["s"] == pytest.approx(d["s"], rel=1e-12)


def test_entropy_and_kl_values():
    assert osk.entropy(np.full(8, 1 / 8)) == pytest.approx(math.log(8), rel=1e-15)
    assert osk.entropy([1.0, 0.0]) == 0.0
    p = np.array([0.2, 0.8])
    q = np.array([0.5, 0.5])
    assert osk.kl_divergence(p, q) == pytest.approx(0.2 * math.log(0.4) + 0.8 * math.log(1.6), rel=1e-15)
