"""Pins for oracle.fastsum: derivatives against symbolic differentiation, the
regularized kernel's matching conditions, b_k against the Gaussian's Fourier
transform, the NDFTs against the FFT at grid nodes and against adjointness,
and Eq. (fastsum) against the exact product of Eq. (matexp)."""
import math

import numpy as np
import pytest

from oracle import fastsum as ofs
from oracle import sinkhorn as osk
from paper_2201_07524_gb300 import workloads as wl

sympy = pytest.importorskip("sympy")


def _sympy_derivs(expr, var, at, p):
    return [float(sympy.diff(expr, var, j).subs(var, at)) if j else float(expr.subs(var, at))
            for j in range(p)]


@pytest.mark.parametrize("r,eps,rho0", [(2.0, 0.02, 0.4), (1.0, 0.02, 0.03), (1.5, 0.05, 0.3),
                                        (3.0, 0.1, 0.25)])
def test_radial_derivatives_match_symbolic(r, eps, rho0):
    rho = sympy.Symbol("rho", positive=True)
    expr = sympy.exp(-rho ** sympy.nsimplify(r) / sympy.nsimplify(eps))
    ref = _sympy_derivs(expr, rho, sympy.nsimplify(rho0), 8)
    got = ofs.radial_derivatives(rho0, eps, r, 8)
    scale = max(abs(v) for v in ref)
    np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-13 * scale)


def _kb_value_and_derivs(L, eps, r, p, at):
    c = ofs.boundary_polynomial(L, eps, r, p)
    delta = 0.5 - L
    tau = (at - L) / delta
    out = []
    poly = np.polynomial.Polynomial(c)
    for j in range(p):
        out.append(poly.deriv(j)(tau) / delta ** j if j else poly(tau))
    return out


@pytest.mark.parametrize("r,eps,L,p", [(2.0, 0.02, 0.4, 8), (2.0, 0.05, 0.4, 6), (1.0, 0.02, 0.35, 5)])
def test_boundary_polynomial_two_point_conditions(r, eps, L, p):
    rho = sympy.Symbol("rho", positive=True)
    expr = sympy.exp(-rho ** sympy.nsimplify(r) / sympy.nsimplify(eps))
    at_L = _sympy_derivs(expr, rho, sympy.nsimplify(L), p)
    got_L = _kb_value_and_derivs(L, eps, r, p, L)
    scale = max(abs(v) for v in at_L)
    np.testing.assert_allclose(got_L, at_L, rtol=1e-9, atol=1e-10 * scale)
    got_half = _kb_value_and_derivs(L, eps, r, p, 0.5)
    assert np.all(np.abs(got_half[1:]) <= 1e-8 * scale)
    assert len(ofs.boundary_polynomial(L, eps, r, p)) == 2 * p - 1


def test_nearfield_polynomial_matching_conditions():
    eps, r, eps_I, p = 0.02, 1.0, 1.0 / 32, 6
    c = ofs.nearfield_polynomial(eps_I, eps, r, p)
    rho = sympy.Symbol("rho", positive=True)
    poly = sum(float(c[q]) * (rho / sympy.nsimplify(eps_I)) ** (2 * q) for q in range(p))
    expr = sympy.exp(-rho / sympy.nsimplify(eps))
    want = _sympy_derivs(expr, rho, sympy.nsimplify(eps_I), p)
    got = _sympy_derivs(poly, rho, sympy.nsimplify(eps_I), p)
    scale = max(abs(v) for v in want)
    np.testing.assert_allclose(got, want, rtol=1e-8, atol=1e-9 * scale)
    # even polynomial: no odd derivative at 0
    assert float(sympy.diff(poly, rho).subs(rho, 0)) == 0.0


def test_regularized_kernel_pieces():
    eps, r, L, p = 0.02, 2.0, 0.4, 8
    rng = np.random.default_rng(1)
    y = rng.uniform(-0.5, 0.5, size=(2000, 3))
    rho = np.linalg.norm(y, axis=1)
    kr = ofs.regularized_kernel(y, eps, r, L, p)
    inside = rho <= L
    np.testing.assert_allclose(kr[inside], np.exp(-rho[inside] ** 2 / eps), rtol=1e-15)
    # constant K_B(1/2) in the corners of the cube
    corner = rho > 0.5
    kb_half = ofs.regularized_kernel(np.array([[0.5, 0.0, 0.0]]), eps, r, L, p)[0]
    np.testing.assert_allclose(kr[corner], kb_half, rtol=1e-15)
    # continuity across rho = L and across the torus boundary
    # K_B matches p derivatives at L, so just past L it agrees with K's own
    # continuation to O(eta^p)
    for eta in (1e-4, 1e-3):
        b = ofs.regularized_kernel(np.array([[L + eta, 0, 0]]), eps, r, L, p)[0]
        assert b == pytest.approx(math.exp(-(L + eta) ** 2 / eps), rel=1e-10)
        a = ofs.regularized_kernel(np.array([[0.5 - eta, 0.0, 0.0]]), eps, r, L, p)[0]
        b = ofs.regularized_kernel(np.array([[-0.5 + eta, 0.0, 0.0]]), eps, r, L, p)[0]
        assert a == pytest.approx(b, rel=1e-12)
    # periodic: shifting by a lattice vector changes nothing
    # (adding integers rounds the coordinates, hence the loose tolerance)
    np.testing.assert_allclose(ofs.regularized_kernel(y + np.array([1.0, -1.0, 2.0]), eps, r, L, p), kr,
                               rtol=1e-10)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_fourier_coefficients_gaussian_closed_form(d):
    # A narrow Gaussian is already ~0 at rho = L and fully resolved by N, so the
    # normalized DFT of its samples is its continuous Fourier transform:
    # b_k = (pi eps)^{d/2} exp(-pi^2 eps |k|^2).
    # eps and N are such that exp(-L^2/eps) and the alias exp(-pi^2 eps N^2/4)
    # are both below 1e-13.
    N = {1: 64, 2: 64, 3: 48}[d]
    eps = 0.005
    b = ofs.fourier_coefficients(N, d, eps, 2.0, 0.4, 8)
    k = ofs.frequency_grid(N, d)
    want = (math.pi * eps) ** (d / 2) * np.exp(-math.pi ** 2 * eps * np.sum(k * k, axis=-1))
    np.testing.assert_allclose(b, want, atol=1e-12 * want.max())
    assert b[(N // 2,) * d] == pytest.approx((math.pi * eps) ** (d / 2), rel=1e-12)


def test_fourier_coefficients_interpolate_at_grid_nodes():
    N, d = 16, 2
    b = ofs.fourier_coefficients(N, d, 0.05, 2.0, 0.4, 6)
    nodes = ofs.frequency_grid(N, d).reshape(-1, d) / N
    vals = ofs.ndft(nodes, b, N)
    np.testing.assert_allclose(vals.real, ofs.regularized_kernel(nodes, 0.05, 2.0, 0.4, 6), atol=1e-14)
    assert np.abs(vals.imag).max() < 1e-14


@pytest.mark.parametrize("p", [4, 6, 8])
def test_fourier_coefficient_decay_reflects_smoothness(p):
    # K_R is C^{p-1} (K_B matches p-1 derivatives at L and is flat to order p-1
    # at 1/2), so the tail of |b_k| falls at least like |k|^{-p}; a missed
    # matching condition would leave a |k|^{-2} tail.
    N = 256
    b = ofs.fourier_coefficients(N, 1, 0.02, 2.0, 0.4, p)
    k = np.abs(np.arange(-N // 2, N // 2))
    t64 = np.abs(b[k > 64]).max()
    t96 = np.abs(b[k > 96]).max()
    assert math.log(t64 / t96) / math.log(1.5) >= p - 1


def test_adjoint_ndft_at_grid_nodes_is_fft():
    N, n, d = 8, 4, 2
    rng = np.random.default_rng(2)
    lidx = rng.integers(0, N, size=(n, d))
    w = rng.standard_normal(n)
    grid = np.zeros((N, N))
    np.add.at(grid, tuple(lidx.T), w)
    want = np.fft.fftshift(np.fft.fftn(grid))     # sum_l g_l e^{-2 pi i k l / N}, k in I_N
    got = ofs.adjoint_ndft(lidx / N, w, N)
    np.testing.assert_allclose(got, want, atol=1e-13)


def test_ndft_and_adjoint_are_adjoint():
    N = 10
    rng = np.random.default_rng(4)
    for d in (1, 2, 3):
        z = rng.random((13, d))
        w = rng.standard_normal(13)
        fh = rng.standard_normal((N,) * d) + 1j * rng.standard_normal((N,) * d)
        lhs = np.vdot(ofs.ndft(z, fh, N), w)                   # <A f, w>
        rhs = np.vdot(fh, ofs.adjoint_ndft(z, w, N))           # <f, A^H w>
        assert lhs == pytest.approx(rhs, rel=1e-12)


def test_ndft_small_brute_force():
    import cmath
    N = 4
    z = np.array([[0.1, 0.7], [0.33, 0.2]])
    fh = np.arange(16).reshape(4, 4) * (1 + 0.5j)
    got = ofs.ndft(z, fh, N)
    for j in range(2):
        acc = 0j
        for a in range(N):
            for c in range(N):
                acc += fh[a, c] * cmath.exp(2j * math.pi * ((a - 2) * z[j, 0] + (c - 2) * z[j, 1]))
        assert got[j] == pytest.approx(acc, rel=1e-13)


@pytest.mark.parametrize("d,N,eps", [(1, 64, 0.05), (2, 64, 0.05), (3, 32, 0.02)])
def test_fastsum_matches_exact_product(d, N, eps):
    # Eq. (fastsum) with the regularized kernel reproduces Eq. (matexp) up to the
    # kernel approximation error.
    n = 300 if d < 3 else 150
    x = wl.uniform_ball(n, d, 0.2, 3)
    y = wl.uniform_ball(n + 17, d, 0.2, 4)
    v = wl.positive_vector(n + 17, 5)
    exact = osk.kernel_apply(x, y, v, eps, 2.0)
    got = ofs.fastsum(x, y, v, eps, 2.0, N, np.zeros(3), 1.0, 0.1, 8)
    assert np.abs(got - exact).max() / np.abs(exact).max() < 1e-6


def test_fastsum_scaling_is_exact():
    # Moving and scaling the clouds into the torus leaves the sum unchanged.
    d, N, eps = 2, 64, 0.05
    x = wl.uniform_ball(200, d, 0.2, 6) + 0.3
    y = wl.uniform_ball(210, d, 0.2, 7) + 0.3
    v = wl.positive_vector(210, 8)
    exact = osk.kernel_apply(x, y, v, eps, 2.0)
    got = ofs.fastsum(x, y, v, eps, 2.0, N, np.array([0.3, 0.3, 0.0]), 0.5, 0.1, 8)
    assert np.abs(got - exact).max() / np.abs(exact).max() < 1e-6


def test_nearfield_correction_restores_r1_kernel():
    d, N, eps, eps_I, p = 2, 64, 0.05, 1.0 / 16, 6
    x = wl.uniform_ball(250, d, 0.2, 9)
    y = wl.uniform_ball(260, d, 0.2, 10)
    v = wl.positive_vector(260, 11)
    exact = osk.kernel_apply(x, y, v, eps, 1.0)
    with_nf = ofs.fastsum(x, y, v, eps, 1.0, N, np.zeros(3), 1.0, 0.1, p, eps_I)
    err_nf = np.abs(with_nf - exact).max() / np.abs(exact).max()
    # the same K_R without its correction misses the cusp at 0
    zx = ofs.torus_coordinates(x, np.zeros(3), 1.0)
    zy = ofs.torus_coordinates(y, np.zeros(3), 1.0)
    b = ofs.fourier_coefficients(N, d, eps, 1.0, 0.4, p, eps_I)
    no_nf = ofs.fastsum_trig(zx, zy, v, b)
    err_no = np.abs(no_nf - exact).max() / np.abs(exact).max()
    assert err_nf < 1e-4
    assert err_no > 100 * err_nf


def test_torus_coordinates_hand_values():
    # z = scale (x - center) + 1/2: the center lands on 1/2, offsets scale.
    c = np.array([0.3, -0.1, 0.0])
    z = ofs.torus_coordinates(np.array([[0.3, -0.1], [0.4, -0.3]]), c, 0.5)
    np.testing.assert_allclose(z, [[0.5, 0.5], [0.55, 0.4]], rtol=1e-15)
