"""Kantorovich linear program by brute force, for tiny inputs (test infrastructure).

Def. "Wasserstein distance" and Eqs. (Da)-(Dd): w_r = min sum_ij pi_ij d_ij^r
over couplings with marginals p and p~.  For n = m points with uniform weights
1/n the feasible set is (1/n) x the Birkhoff polytope, whose vertices are the
permutation matrices, so the minimum of the linear objective is attained at a
permutation: w_r = (1/n) min_sigma sum_i C_{i, sigma(i)}.  This module
enumerates all n! permutations; it is meant for n <= 8.
"""
import itertools

import numpy as np

from .sinkhorn import cost_matrix


def assignment_cost_bruteforce(C):
    """min over permutations sigma of (1/n) sum_i C[i, sigma(i)], plus the minimizer."""
    C = np.asarray(C, dtype=np.float64)
    n = C.shape[0]
    if C.shape != (n, n):
        raise ValueError("square cost matrix required")
    if n > 9:
        raise ValueError("brute force is for n <= 9")
    best, best_perm = np.inf, None
    rows = np.arange(n)
    for perm in itertools.permutations(range(n)):
        c = C[rows, perm].sum()
        if c < best:
            best, best_perm = c, perm
    return best / n, best_perm


def wasserstein_r_uniform(x, y, r):
    """w_r(P, P~) of Eq. (W0) for uniform empirical measures with n = m points."""
    return assignment_cost_bruteforce(cost_matrix(x, y, r))[0]
