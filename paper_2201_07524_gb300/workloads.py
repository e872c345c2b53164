"""Seeded synthetic point clouds and weights.

This module only draws inputs; it holds none of the method's arithmetic, so
the CUDA path's tests and the CPU oracle can both take their inputs from it.
All arrays are numpy float64 on the host.

Recipes (the paper's own synthetic workloads are i.i.d. uniform clouds,
Sec. 5.1; the named workloads below replace them with balls, disks and
Gaussian mixtures of the stated radii):

* ``uniform_ball``: direction = normalized standard normal vector, radius =
  R * U^(1/d) with U ~ Uniform(0, 1), so the density is uniform in the ball.
* ``gaussian_mixture``: K component means drawn by ``uniform_ball`` with
  radius R_mean; each point picks a component uniformly and adds an isotropic
  normal offset of standard deviation ``sigma``.
* ``dirichlet_weights``: Dirichlet(1, ..., 1), drawn as normalized Exp(1)
  variables.
* ``uniform_weights``: 1/n each.
"""
from dataclasses import dataclass, field

import numpy as np


def uniform_ball(n, d, radius, seed):
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((n, d))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    rad = radius * rng.random(n) ** (1.0 / d)
    return g * rad[:, None]


def gaussian_mixture(n, d, components, sigma, mean_radius, seed):
    rng = np.random.default_rng(seed)
    means = uniform_ball(components, d, mean_radius, seed + 7919)
    which = rng.integers(0, components, size=n)
    return means[which] + sigma * rng.standard_normal((n, d))


def dirichlet_weights(n, seed):
    rng = np.random.default_rng(seed)
    e = rng.exponential(1.0, size=n)
    return e / e.sum()


def uniform_weights(n):
    return np.full(n, 1.0 / n)


def positive_vector(n, seed, low=0.5, high=1.5):
    """A seeded positive vector to stand in for a scaling vector u or v."""
    rng = np.random.default_rng(seed)
    return low + (high - low) * rng.random(n)


@dataclass
class Workload:
    """One optimal-transport problem: clouds, weights and solver settings."""
    name: str
    d: int
    n: int
    m: int
    eps: float
    r: float
    iters: int
    N: int
    m_w: int
    sigma: float = 2.0
    precision: str = "fp32"
    source: str = "ball"          # "ball" or "gmm"
    seed_x: int = 1
    seed_y: int = 2
    weights: str = "uniform"      # "uniform" or "dirichlet"
    extra: dict = field(default_factory=dict)

    def points(self):
        if self.source == "gmm":
            x = gaussian_mixture(self.n, self.d, 8, 0.03, 0.15, self.seed_x)
        else:
            x = uniform_ball(self.n, self.d, 0.2, self.seed_x)
        y = uniform_ball(self.m, self.d, 0.2, self.seed_y)
        return x, y

    def marginals(self):
        if self.weights == "dirichlet":
            return dirichlet_weights(self.n, self.seed_x + 100), dirichlet_weights(self.m, self.seed_y + 100)
        return uniform_weights(self.n), uniform_weights(self.m)


# The problems the library is measured and checked on.
SMALL_2D = Workload("ball2d_n2000_eps0.05_fp64", d=2, n=2000, m=2000, eps=0.05, r=2.0,
                    iters=100, N=64, m_w=4, precision="fp64")
HEADLINE_3D = Workload("ball3d_n1e6_eps0.02_fp32", d=3, n=1_000_000, m=1_000_000, eps=0.02,
                       r=2.0, iters=100, N=64, m_w=4, precision="fp32")
GMM_2D = Workload("gmm2d_n1e6_eps0.01_fp32", d=2, n=1_000_000, m=1_000_000, eps=0.01, r=2.0,
                  iters=100, N=512, m_w=6, precision="fp32", source="gmm", weights="dirichlet")
BALL3D_R1 = Workload("ball3d_n4e6_r1_eps0.02_fp32", d=3, n=4_000_000, m=4_000_000, eps=0.02,
                     r=1.0, iters=100, N=128, m_w=4, precision="fp32", extra={"eps_I": 1.0 / 32})
