"""NFFT-based fast summation, evaluated with exact trigonometric sums (test infrastructure).

Sec. 4.1 of the paper approximates the radial kernel K(y) = exp(-||y||^r / eps)
(Eq. (kernel_fun), with eps = 1/lambda) by an h-periodic trigonometric
polynomial K_RK(y) = sum_{k in I_N} b_k exp(2 pi i k.y / h) (Eq. (ansatz_NFFT)),
built from a regularized periodic kernel K~ ("Regularization of K"), and then
evaluates t_i = sum_j v_j K(x_i - y_j) through Eq. (fastsum).

This module takes h = 1 and works in torus coordinates (points already scaled
into the unit torus so that all differences have norm <= L = 1/2 - eps_B).  It
computes, in FP64 and by their plain definitions:

* the regularized kernel K_R (the paper's K~), with the boundary polynomial K_B
  on L < rho <= 1/2 and, for kernels that are not smooth at 0 (r not an even
  integer), a near-field polynomial K_I on rho < eps_I (Remark "Arithmetic
  complexity");
* its Fourier coefficients b_k on I_N = {-N/2, ..., N/2-1}^d as the
  normalized DFT of samples on the N^d grid;
* the adjoint NDFT h_k = sum_j w_j exp(-2 pi i k.z_j) and the NDFT
  f_j = sum_k f_k exp(2 pi i k.z_j) as direct sums (no window, no FFT);
* Eq. (fastsum) with those exact sums, and the direct near-field correction.

The paper leaves the boundary polynomial, the near-field polynomial and the way
b_k are obtained to the book it cites; the readings taken here are:

* K_B(rho) is the polynomial of degree 2p-2 in rho on [L, 1/2] whose
  derivatives of orders 0..p-1 equal those of K at rho = L and whose derivatives
  of orders 1..p-1 vanish at rho = 1/2 (two-point Taylor interpolation).
* K_I(rho) = sum_{q<p} c_q rho^(2q) matches the derivatives of orders 0..p-1 of
  K at rho = eps_I.
* b_k = N^-d sum_{l in I_N} K_R(l/N) exp(-2 pi i k.l/N).
* Since K is real, the summation result is the real part of the paper's sum
  over I_N.

Only tests/, smoke() and bench.py's CPU-baseline leg may use this module.
"""
import math

import numpy as np


def radial_kernel(rho, eps, r):
    """K(rho) = exp(-rho^r / eps) (Eq. (kernel_fun) with lambda = 1/eps)."""
    return np.exp(-np.asarray(rho, dtype=np.float64) ** r / eps)


def needs_nearfield(r):
    """True when K is not smooth at y = 0, i.e. r is not an even integer
    (Remark "Arithmetic complexity": r = 1 needs near-field regularization)."""
    return not (float(r).is_integer() and int(r) % 2 == 0)


def radial_derivatives(rho0, eps, r, p):
    """[K(rho0), K'(rho0), ..., K^(p-1)(rho0)] for K = exp(g), g = -rho^r / eps.

    Uses f' = g' f, hence f^(k+1) = sum_{j=0..k} binom(k, j) g^(j+1) f^(k-j),
    with g^(j)(rho) = -r (r-1) ... (r-j+1) rho^(r-j) / eps.
    """
    g = [-(rho0 ** r) / eps]
    for j in range(1, p):
        falling = 1.0
        for q in range(j):
            falling *= (r - q)
        g.append(-falling * rho0 ** (r - j) / eps)
    f = [math.exp(g[0])]
    for k in range(p - 1):
        f.append(sum(math.comb(k, j) * g[j + 1] * f[k - j] for j in range(k + 1)))
    return f


def boundary_polynomial(L, eps, r, p):
    """Coefficients c_0..c_{2p-2} of K_B(rho) = sum_i c_i tau^i, tau = (rho - L) / (1/2 - L).

    Conditions: K_B^(j)(L) = K^(j)(L) for j = 0..p-1 and K_B^(j)(1/2) = 0 for
    j = 1..p-1 (derivatives with respect to rho).  In tau the first set fixes
    c_j = K^(j)(L) delta^j / j! (delta = 1/2 - L) for j < p; the remaining
    p-1 coefficients solve the linear system of the conditions at tau = 1.
    """
    delta = 0.5 - L
    f = radial_derivatives(L, eps, r, p)
    low = [f[j] * delta ** j / math.factorial(j) for j in range(p)]
    nq = p - 1
    A = np.zeros((nq, nq))
    rhs = np.zeros(nq)
    for row, order in enumerate(range(1, p)):
        # d^order/dtau^order tau^e at tau = 1 equals e! / (e - order)!
        rhs[row] = -sum(low[e] * math.perm(e, order) for e in range(order, p))
        for q in range(nq):
            A[row, q] = math.perm(p + q, order)
    high = np.linalg.solve(A, rhs) if nq > 0 else np.zeros(0)
    return np.concatenate([np.array(low), high])


def nearfield_polynomial(eps_I, eps, r, p):
    """Coefficients c_0..c_{p-1} of K_I(rho) = sum_q c_q (rho/eps_I)^(2q).

    Conditions: K_I^(j)(eps_I) = K^(j)(eps_I) for j = 0..p-1.  Solved in the
    scaled variable s = rho/eps_I, where the j-th derivative of s^(2q) at s = 1
    is (2q)! / (2q-j)!.
    """
    f = radial_derivatives(eps_I, eps, r, p)
    A = np.zeros((p, p))
    rhs = np.array([f[j] * eps_I ** j for j in range(p)])
    for j in range(p):
        for q in range(p):
            A[j, q] = math.perm(2 * q, j) if 2 * q >= j else 0.0
    return np.linalg.solve(A, rhs)


def regularized_kernel(y, eps, r, L, p, eps_I=None):
    """K_R(y) on the unit torus (the paper's K~ with h = 1), y of shape (..., d).

    K_R = K_I(rho) for rho < eps_I (only when K is not smooth at 0),
          K(rho)   for rho <= L,
          K_B(rho) for L < rho <= 1/2,
          K_B(1/2) for rho > 1/2 inside [-1/2, 1/2]^d.
    ``y`` is first wrapped into [-1/2, 1/2)^d (h-periodicity).
    """
    y = np.asarray(y, dtype=np.float64)
    y = y - np.floor(y + 0.5)
    rho = np.sqrt(np.sum(y * y, axis=-1))
    cb = boundary_polynomial(L, eps, r, p)
    tau = (np.minimum(rho, 0.5) - L) / (0.5 - L)
    kb = np.polynomial.polynomial.polyval(tau, cb)
    out = np.where(rho <= L, radial_kernel(rho, eps, r), kb)
    if eps_I is not None and needs_nearfield(r):
        ci = nearfield_polynomial(eps_I, eps, r, p)
        ki = np.polynomial.polynomial.polyval((rho / eps_I) ** 2, ci)
        out = np.where(rho < eps_I, ki, out)
    return out


def frequency_grid(N, d):
    """The index set I_N = {-N/2, ..., N/2-1}^d as an array of shape (N,)*d + (d,)."""
    k = np.arange(-N // 2, N // 2)
    return np.stack(np.meshgrid(*([k] * d), indexing="ij"), axis=-1)


def fourier_coefficients(N, d, eps, r, L, p, eps_I=None):
    """b_k = N^-d sum_{l in I_N} K_R(l/N) exp(-2 pi i k.l / N), k in I_N.

    Returned real (K_R is real and even in each coordinate, so b is real) as an
    array of shape (N,)*d whose entry [k_1 + N/2, ..., k_d + N/2] is b_k.  The
    DFT is taken with numpy's FFT after moving l = 0 to the first position.
    """
    samples = regularized_kernel(frequency_grid(N, d) / N, eps, r, L, p, eps_I)
    bh = np.fft.fftn(np.fft.ifftshift(samples)) / float(N) ** d
    return np.fft.fftshift(bh).real


def _phase_factors(z, N, sign):
    """exp(sign 2 pi i k z_t) for k in I_N, one (n, N) array per dimension."""
    k = np.arange(-N // 2, N // 2)
    z = np.asarray(z, dtype=np.float64)
    return [np.exp(sign * 2j * np.pi * np.outer(z[:, t], k)) for t in range(z.shape[1])]


def adjoint_ndft(z, w, N):
    """h_k = sum_j w_j exp(-2 pi i k.z_j), k in I_N (the inner sum of Eq. (fastsum)).

    Direct sum over points; exp(-2 pi i k.z) is the product over dimensions of
    exp(-2 pi i k_t z_t).  Output shape (N,)*d indexed by k + N/2.
    """
    E = _phase_factors(z, N, -1.0)
    w = np.asarray(w, dtype=np.float64)
    letters = "abc"[: len(E)]
    spec = "j," + ",".join("j" + c for c in letters) + "->" + letters
    return np.einsum(spec, w, *E)


def ndft(z, fhat, N):
    """f_j = sum_{k in I_N} fhat_k exp(2 pi i k.z_j) (the outer sum of Eq. (fastsum))."""
    E = _phase_factors(z, N, +1.0)
    letters = "abc"[: len(E)]
    spec = letters + "," + ",".join("j" + c for c in letters) + "->j"
    return np.einsum(spec, fhat, *E)


def fastsum_trig(zx, zy, v, b):
    """Eq. (fastsum): t_i = Re sum_{k in I_N} b_k (sum_j v_j e^{-2 pi i k.y_j}) e^{2 pi i k.x_i},

    evaluated with the exact sums above (torus coordinates zx, zy).
    """
    N = b.shape[0]
    return ndft(zx, b * adjoint_ndft(zy, v, N), N).real


def nearfield_correction(zx, zy, v, eps, r, eps_I, p, chunk=256):
    """sum over pairs with ||x_i - y_j|| < eps_I of v_j (K - K_I)(||x_i - y_j||).

    Adding it to the fast sum of K_R restores the exact kernel near y = 0
    (Remark "Arithmetic complexity").  Direct O(n m) loop over row chunks.
    """
    zx = np.asarray(zx, dtype=np.float64)
    zy = np.asarray(zy, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    ci = nearfield_polynomial(eps_I, eps, r, p)
    out = np.zeros(zx.shape[0])
    for i0 in range(0, zx.shape[0], chunk):
        diff = zx[i0:i0 + chunk, None, :] - zy[None, :, :]
        rho = np.sqrt(np.sum(diff * diff, axis=-1))
        ki = np.polynomial.polynomial.polyval((rho / eps_I) ** 2, ci)
        corr = np.where(rho < eps_I, radial_kernel(rho, eps, r) - ki, 0.0)
        out[i0:i0 + chunk] = corr @ v
    return out


def torus_coordinates(x, center, scale):
    """z = scale (x - center) + 1/2: points moved into the unit torus so that the
    kernel in the new coordinates is exp(-rho^r / (eps scale^r))."""
    x = np.asarray(x, dtype=np.float64)
    return scale * (x - np.asarray(center, dtype=np.float64)[: x.shape[1]]) + 0.5


def fastsum(x, y, v, eps, r, N, center, scale, eps_B, p, eps_I=None):
    """What the NFFT path approximates before windowing: sum_j v_j K_R(x_i - y_j)
    (plus the near-field correction when K is not smooth at 0), computed through
    Eq. (fastsum) with exact trigonometric sums.  Differs from the exact product
    of Eq. (matexp) only by the kernel approximation error."""
    d = np.asarray(x).shape[1]
    zx = torus_coordinates(x, center, scale)
    zy = torus_coordinates(y, center, scale)
    eps_s = eps * scale ** r
    L = 0.5 - eps_B
    use_nf = needs_nearfield(r) and eps_I is not None
    b = fourier_coefficients(N, d, eps_s, r, L, p, eps_I if use_nf else None)
    t = fastsum_trig(zx, zy, v, b)
    if use_nf:
        t = t + nearfield_correction(zx, zy, v, eps_s, r, eps_I, p)
    return t
