"""Pins for oracle.lp: the brute-force assignment against an independent
library solver and against the 1-D monotone-matching closed form."""
import numpy as np
import pytest

from oracle import lp
from oracle import sinkhorn as osk


def test_bruteforce_matches_scipy_assignment():
    scipy_opt = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(3)
    for n in (1, 2, 5, 7):
        C = rng.random((n, n))
        rows, cols = scipy_opt.linear_sum_assignment(C)
        val, perm = lp.assignment_cost_bruteforce(C)
        assert val == pytest.approx(C[rows, cols].sum() / n, rel=1e-14)
        assert C[np.arange(n), perm].sum() / n == pytest.approx(val, rel=1e-15)


def test_one_dimensional_monotone_matching():
    # For a convex cost |x - y|^r, r >= 1, in 1-D the sorted matching is optimal.
    rng = np.random.default_rng(5)
    x = rng.random((7, 1))
    y = rng.random((7, 1))
    for r in (1.0, 2.0, 3.0):
        w = lp.wasserstein_r_uniform(x, y, r)
        sorted_cost = np.mean(np.abs(np.sort(x[:, 0]) - np.sort(y[:, 0])) ** r)
        assert w == pytest.approx(sorted_cost, rel=1e-13)


def test_identical_clouds_cost_zero():
    x = np.random.default_rng(9).random((6, 2))
    assert lp.wasserstein_r_uniform(x, x[::-1], 2.0) == 0.0
    assert osk.cost_matrix(x, x, 2.0).diagonal().max() == 0.0
