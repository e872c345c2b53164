"""Pins of the oracle's gradient (dual_gradient) and Sinkhorn divergence.

The gradient is checked against things other than its own formula: central
differences of the dual function Eq. (27) (itself pinned in
test_oracle_sinkhorn.py), the envelope theorem at a converged dense solve
(differences of the re-solved value s), the one-point closed form and
translation invariance.  The divergence is checked against the one-point
closed form, the swap symmetry, sd(P, P) = 0 and non-negativity (Remark
"Entropy bias and Sinkhorn divergence")."""
import numpy as np
import pytest

from oracle import sinkhorn as osk


def _problem(n, m, d, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-0.3, 0.3, size=(n, d))
    y = rng.uniform(-0.3, 0.3, size=(m, d))
    a = rng.uniform(0.5, 1.5, size=n)
    b = rng.uniform(0.5, 1.5, size=m)
    return x, y, a / a.sum(), b / b.sum()


def _dual(x, y, a, b, u, v, eps, r):
    return osk.dual_objective(u, v, a, b, osk.gibbs_kernel(x, y, eps, r), eps)


@pytest.mark.parametrize("r", [1.0, 1.5, 2.0, 3.0])
def test_dual_gradient_matches_finite_differences(r):
    x, y, a, b = _problem(4, 5, 2, 11)
    rng = np.random.default_rng(12)
    u = rng.uniform(0.5, 2.0, size=4)
    v = rng.uniform(0.5, 2.0, size=5)
    eps, h = 0.2, 1e-6
    ga, gb, gx, gy = osk.dual_gradient(x, y, a, b, u, v, eps, r)
    for arr, g in ((x, gx), (y, gy)):
        for idx in np.ndindex(arr.shape):
            old = arr[idx]
            arr[idx] = old + h
            fp = _dual(x, y, a, b, u, v, eps, r)
            arr[idx] = old - h
            fm = _dual(x, y, a, b, u, v, eps, r)
            arr[idx] = old
            assert abs((fp - fm) / (2 * h) - g[idx]) < 1e-7 * max(1.0, abs(g[idx]))
    for arr, g in ((a, ga), (b, gb)):
        for i in range(len(arr)):
            old = arr[i]
            arr[i] = old + h
            fp = _dual(x, y, a, b, u, v, eps, r)
            arr[i] = old - h
            fm = _dual(x, y, a, b, u, v, eps, r)
            arr[i] = old
            assert abs((fp - fm) / (2 * h) - g[i]) < 1e-8


def _converged_value(x, a, y, b, eps, r):
    out = osk.sinkhorn_dense(x, a, y, b, eps, r, 4000)
    assert out["err_row"] < 1e-13
    return out


def test_envelope_theorem_positions():
    # at the maximizer the gradient of the value equals the dual gradient
    x, y, a, b = _problem(3, 4, 2, 21)
    eps, r, h = 0.3, 2.0, 1e-5
    out = _converged_value(x, a, y, b, eps, r)
    _, _, gx, gy = osk.dual_gradient(x, y, a, b, out["u"], out["v"], eps, r)
    for arr, g in ((x, gx), (y, gy)):
        for idx in np.ndindex(arr.shape):
            old = arr[idx]
            arr[idx] = old + h
            sp = _converged_value(x, a, y, b, eps, r)["s"]
            arr[idx] = old - h
            sm = _converged_value(x, a, y, b, eps, r)["s"]
            arr[idx] = old
            assert abs((sp - sm) / (2 * h) - g[idx]) < 1e-7


def test_envelope_theorem_weights():
    # along directions that keep a on the simplex, ds = <beta, da>
    x, y, a, b = _problem(4, 3, 2, 31)
    eps, r, h = 0.3, 2.0, 1e-6
    out = _converged_value(x, a, y, b, eps, r)
    ga, gb, _, _ = osk.dual_gradient(x, y, a, b, out["u"], out["v"], eps, r)
    rng = np.random.default_rng(32)
    for w, g, first in ((a, ga, True), (b, gb, False)):
        dlt = rng.standard_normal(len(w))
        dlt -= dlt.mean()
        wp, wm = w + h * dlt, w - h * dlt
        if first:
            sp = _converged_value(x, wp, y, b, eps, r)["s"]
            sm = _converged_value(x, wm, y, b, eps, r)["s"]
        else:
            sp = _converged_value(x, a, y, wp, eps, r)["s"]
            sm = _converged_value(x, a, y, wm, eps, r)["s"]
        assert abs((sp - sm) / (2 * h) - float(g @ dlt)) < 1e-7


@pytest.mark.parametrize("r", [1.0, 2.0, 3.0])
def test_single_pair_closed_form(r):
    # n = m = 1: pi = 1, s = ||x - y||^r, d/dx = r ||x - y||^(r-2) (x - y)
    x = np.array([[0.1, -0.2, 0.05]])
    y = np.array([[-0.15, 0.1, 0.2]])
    out = osk.sinkhorn_dense(x, [1.0], y, [1.0], 0.5, r, 5)
    _, _, gx, gy = osk.dual_gradient(x, y, [1.0], [1.0], out["u"], out["v"], 0.5, r)
    dist = np.linalg.norm(x - y)
    want = r * dist ** (r - 2) * (x - y)
    assert np.allclose(gx, want, rtol=1e-12, atol=0)
    assert np.allclose(gy, -want, rtol=1e-12, atol=0)
    assert abs(out["s"] - dist ** r) < 1e-12


def test_translation_invariance():
    # moving both clouds together leaves every cost unchanged
    x, y, a, b = _problem(5, 6, 3, 41)
    rng = np.random.default_rng(42)
    u = rng.uniform(0.5, 2.0, size=5)
    v = rng.uniform(0.5, 2.0, size=6)
    _, _, gx, gy = osk.dual_gradient(x, y, a, b, u, v, 0.1, 2.0)
    assert np.allclose(gx.sum(axis=0) + gy.sum(axis=0), 0.0, atol=1e-14)


def test_divergence_single_points_and_symmetry():
    x = np.array([[0.1, 0.0]])
    y = np.array([[-0.2, 0.3]])
    sd = osk.sinkhorn_divergence(x, [1.0], y, [1.0], 0.1, 2.0, 3)
    assert abs(sd - np.sum((x - y) ** 2)) < 1e-12
    xs, ys, a, b = _problem(5, 7, 2, 51)
    s1 = osk.sinkhorn_divergence(xs, a, ys, b, 0.05, 2.0, 300)
    s2 = osk.sinkhorn_divergence(ys, b, xs, a, 0.05, 2.0, 300)
    assert abs(s1 - s2) < 1e-10
    assert abs(osk.sinkhorn_divergence(xs, a, xs, a, 0.05, 2.0, 300)) < 1e-12


@pytest.mark.parametrize("seed", [61, 62, 63])
def test_divergence_is_nonnegative(seed):
    x, y, a, b = _problem(6, 5, 2, seed)
    assert osk.sinkhorn_divergence(x, a, y, b, 0.05, 2.0, 500) > 0.0


def test_divergence_gradient_matches_differences_at_convergence():
    x, y, a, b = _problem(4, 3, 2, 71)
    eps, r, h, it = 0.3, 2.0, 1e-5, 3000
    ga, gb, gx, gy = osk.sinkhorn_divergence_gradient(x, a, y, b, eps, r, it)
    for arr, g in ((x, gx), (y, gy)):
        for idx in np.ndindex(arr.shape):
            old = arr[idx]
            arr[idx] = old + h
            sp = osk.sinkhorn_divergence(x, a, y, b, eps, r, it)
            arr[idx] = old - h
            sm = osk.sinkhorn_divergence(x, a, y, b, eps, r, it)
            arr[idx] = old
            assert abs((sp - sm) / (2 * h) - g[idx]) < 1e-7
    rng = np.random.default_rng(72)
    for w, g, first in ((a, ga, True), (b, gb, False)):
        dlt = rng.standard_normal(len(w))
        dlt -= dlt.mean()
        if first:
            sp = osk.sinkhorn_divergence(x, w + h * dlt, y, b, eps, r, it)
            sm = osk.sinkhorn_divergence(x, w - h * dlt, y, b, eps, r, it)
        else:
            sp = osk.sinkhorn_divergence(x, a, y, w + h * dlt, eps, r, it)
            sm = osk.sinkhorn_divergence(x, a, y, w - h * dlt, eps, r, it)
        assert abs((sp - sm) / (2 * h) - float(g @ dlt)) < 1e-7


def test_divergence_gradient_vanishes_at_equal_measures():
    # sd(P, P~) >= 0 with equality at P~ = P: a minimum, so the position
    # gradient with respect to y vanishes there
    x, _, a, _ = _problem(5, 5, 2, 81)
    _, gb, gx, gy = osk.sinkhorn_divergence_gradient(x, a, x.copy(), a.copy(), 0.2, 2.0, 2000)
    assert np.max(np.abs(gy)) < 1e-12 and np.max(np.abs(gx)) < 1e-12
    assert np.max(np.abs(gb - gb.mean())) < 1e-12


# ------------------------------------------------------------ log domain
@pytest.mark.parametrize("iters", [1, 2, 7])
def test_log_domain_is_alg1_up_to_a_gauge(iters):
    # from beta = gamma = 0 (u = v = e^(-1/2)) against Alg. 1 from u = v = 1:
    # exp(beta/eps - 1/2) = e^(1/2) u and exp(gamma/eps - 1/2) = e^(-1/2) v,
    # which leaves pi and the value unchanged
    x, y, a, b = _problem(6, 5, 2, 91)
    eps = 0.1
    lg = osk.sinkhorn_log_dense(x, a, y, b, eps, 2.0, iters)
    ref = osk.sinkhorn_dense(x, a, y, b, eps, 2.0, iters)
    assert np.allclose(lg["beta"], eps * (np.log(ref["u"]) + 1.0), rtol=0, atol=1e-13)
    assert np.allclose(lg["gamma"], eps * np.log(ref["v"]), rtol=0, atol=1e-13)
    assert abs(lg["s"] - ref["s"]) < 1e-13
    assert abs(lg["err_row"] - ref["err_row"]) < 1e-13


def test_log_domain_survives_where_the_kernel_underflows():
    # eps small enough that the scaling form's u, v leave the FP64 range: the
    # log form keeps converging, and its dual value (a lower bound of the
    # entropic optimum) stays within the sandwich of Lemma "Quality of the
    # Sinkhorn approximation" around the brute-force optimum,
    # s <= w_r <= s + eps (H(a) + H(b)).
    from oracle import lp
    rng = np.random.default_rng(92)
    x = rng.uniform(-0.4, 0.4, size=(5, 2))
    y = rng.uniform(-0.4, 0.4, size=(5, 2))
    a = np.full(5, 0.2)
    eps = 1e-4
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        assert not np.all(np.isfinite(osk.sinkhorn_dense(x, a, y, a, eps, 2.0, 50)["u"]))
    lg = osk.sinkhorn_log_dense(x, a, y, a, eps, 2.0, 3000)
    assert np.all(np.isfinite(lg["beta"])) and lg["err_row"] < 1e-3
    w = lp.assignment_cost_bruteforce(osk.cost_matrix(x, y, 2.0))[0]
    assert lg["s"] <= w <= lg["s"] + eps * (osk.entropy(a) + osk.entropy(a))
