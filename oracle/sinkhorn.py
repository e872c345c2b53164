"""Dense FP64 Sinkhorn and exact kernel-vector products (test infrastructure).

Notation: source points x_i (n of them, weights a = p), target points y_j
(m of them, weights b = p~), cost d_ij^r with d the Euclidean distance
(Eq. (dist)).  The paper writes the Gibbs kernel as exp(-lambda d^r); this
oracle takes eps = 1/lambda, so k_ij = exp(-d_ij^r / eps) and every 1/lambda
in the paper becomes a factor eps.  The scaling vectors u, v are the paper's
alpha, alpha~.

Only tests/, smoke() and bench.py's CPU-baseline leg may use this module.
"""
import numpy as np


def cost_matrix(x, y, r):
    """d_ij^r with d_ij = ||x_i - y_j||_2 (Eq. (dist), Def. "Wasserstein distance")."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    diff = x[:, None, :] - y[None, :, :]
    dist = np.sqrt(np.sum(diff * diff, axis=-1))
    return dist ** r


def gibbs_kernel(x, y, eps, r):
    """k_ij = exp(-d_ij^r / eps): the Gibbs kernel of Alg. 1 (with lambda = 1/eps)."""
    return np.exp(-cost_matrix(x, y, r) / eps)


def kernel_apply(x, y, v, eps, r, chunk=256):
    """t_i = sum_j v_j exp(-||x_i - y_j||^r / eps), i = 1..n (Eq. (matexp)).

    Matrix-free: rows are formed ``chunk`` at a time, so memory stays
    O(chunk * m) and the oracle reaches sizes where the dense K does not fit.
    """
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    out = np.empty(x.shape[0], dtype=np.float64)
    for i0 in range(0, x.shape[0], chunk):
        out[i0:i0 + chunk] = gibbs_kernel(x[i0:i0 + chunk], y, eps, r) @ v
    return out


def kernel_apply_T(x, y, u, eps, r, chunk=256):
    """t~_j = sum_i u_i exp(-||x_i - y_j||^r / eps), j = 1..m (Eq. (matexpt))."""
    return kernel_apply(y, x, u, eps, r, chunk)


def entropy(p):
    """H(P) = -sum_i p_i log p_i (Lemma "Quality of the Sinkhorn approximation"), 0 log 0 = 0."""
    p = np.asarray(p, dtype=np.float64)
    nz = p > 0
    return float(-np.sum(p[nz] * np.log(p[nz])))


def plan_entropy(pi):
    """H(pi) = -sum_ij pi_ij log pi_ij (Eq. (negentropy))."""
    return entropy(np.ravel(pi))


def transport_plan(u, v, K):
    """pi = diag(u) K diag(v) (Eq. (pi*))."""
    return u[:, None] * K * v[None, :]


def dual_objective(u, v, a, b, K, eps):
    """Dual function Eq. (27) with 1/lambda = eps:

    d(u, v) = eps sum_i a_i (1/2 + log u_i) + eps sum_j b_j (1/2 + log v_j)
              - eps sum_ij u_i k_ij v_j.
    With sum a = sum b = 1 this is the value Alg. 1 returns.
    """
    return float(eps * np.sum(a * (0.5 + np.log(u)))
                 + eps * np.sum(b * (0.5 + np.log(v)))
                 - eps * (u @ K @ v))


def sinkhorn_value(u, v, a, b, uKv, eps):
    """Result line of Alg. 1 / Alg. 3 with 1/lambda = eps:

    s = eps + eps sum_i a_i log u_i + eps sum_j b_j log v_j - eps u^T K v.
    ``uKv`` is u^T K v (Alg. 3 writes it as sum_j t~_j v_j).
    """
    return float(eps * (1.0 + np.sum(a * np.log(u)) + np.sum(b * np.log(v)) - uKv))


def marginal_residuals(u, v, a, b, K):
    """The two terms of Eq. (Error): ||pi 1 - p|| and ||pi^T 1 - p~|| (Euclidean)."""
    row = u * (K @ v) - a
    col = v * (K.T @ u) - b
    return float(np.linalg.norm(row)), float(np.linalg.norm(col))


def sinkhorn_dense(x, a, y, b, eps, r, iters, record=False):
    """Alg. 1 (standard Sinkhorn) with an explicit K, in FP64.

    Starts from u = 1_n, v = 1_m (the Set line of Alg. 1).  One iteration is the
    odd half-step u_i <- a_i / (K v)_i followed by the even half-step
    v_j <- b_j / (K^T u)_j (Eq. (S1), reading its second p_j as p~_j = b_j).
    ``iters`` counts such pairs, so Delta = 2 * iters half-steps are taken.

    Returns a dict with u, v, the result value ``s`` (Alg. 1 result line), the
    primal quantities <pi, C> = s~ (Eq. (15)) and H(pi), the final residuals of
    Eq. (Error) and, if ``record``, the states after every half-step.
    """
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    C = cost_matrix(x, y, r)
    K = np.exp(-C / eps)
    u = np.ones(len(a))
    v = np.ones(len(b))
    history = [(u.copy(), v.copy())] if record else None
    for _ in range(iters):
        u = a / (K @ v)            # Delta odd
        if record:
            history.append((u.copy(), v.copy()))
        v = b / (K.T @ u)          # Delta even
        if record:
            history.append((u.copy(), v.copy()))
    pi = transport_plan(u, v, K)
    err_row, err_col = marginal_residuals(u, v, a, b, K)
    uKv = float(u @ K @ v)
    return dict(
        u=u, v=v, K=K, C=C, pi=pi,
        s=sinkhorn_value(u, v, a, b, uKv, eps),
        s_tilde=float(np.sum(pi * C)),
        H_pi=plan_entropy(pi),
        err_row=err_row, err_col=err_col,
        history=history,
    )


def sinkhorn_matrix_free(x, a, y, b, eps, r, iters):
    """Alg. 1 with every K-product formed row-chunk by row-chunk (Eqs. (matexp),
    (matexpt)); the same iteration as ``sinkhorn_dense`` for sizes whose K does
    not fit in memory.  Returns u, v, s (Alg. 1 result line) and the final
    Eq. (Error) residuals."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    u = np.ones(len(a))
    v = np.ones(len(b))
    for _ in range(iters):
        u = a / kernel_apply(x, y, v, eps, r)
        v = b / kernel_apply_T(x, y, u, eps, r)
    Kv = kernel_apply(x, y, v, eps, r)
    KTu = kernel_apply_T(x, y, u, eps, r)
    uKv = float(u @ Kv)
    return dict(
        u=u, v=v,
        s=sinkhorn_value(u, v, a, b, uKv, eps),
        err_row=float(np.linalg.norm(u * Kv - a)),
        err_col=float(np.linalg.norm(v * KTu - b)),
    )


def kl_divergence(p, q):
    """D_KL(p | q) = sum_i p_i log(p_i / q_i) (Notations, Sec. 2)."""
    p = np.asarray(p, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    nz = p > 0
    return float(np.sum(p[nz] * np.log(p[nz] / q[nz])))


def objective_f(u, v, a, b, K):
    """f(u, v) = u^T K v - sum a log u - sum b log v (Eq. (objfunc)), here with
    the unnormalized K that Alg. 1 iterates with."""
    return float(u @ K @ v - np.sum(a * np.log(u)) - np.sum(b * np.log(v)))


def cost_gradient(x, y, r):
    """dC_ij / dx_i for C_ij = ||x_i - y_j||^r: r ||x_i - y_j||^(r-2) (x_i - y_j),
    shape (n, m, d).  Where x_i = y_j the cost is not differentiable for r < 2;
    there the value 0 (a subgradient) is taken."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    diff = x[:, None, :] - y[None, :, :]
    dist = np.sqrt(np.sum(diff * diff, axis=-1))
    scale = np.zeros_like(dist)
    nz = dist > 0
    scale[nz] = r * dist[nz] ** (r - 2.0)
    return scale[:, :, None] * diff


def dual_gradient(x, y, a, b, u, v, eps, r):
    """Gradient of the dual function Eq. (27) at fixed scaling vectors (u, v)
    with respect to the weights and the positions.

    Eq. (27) is d = eps sum_i a_i (1/2 + log u_i) + eps sum_j b_j (1/2 + log v_j)
    - eps sum_ij u_i k_ij v_j with k_ij = exp(-C_ij / eps), so
      d/da_i = eps (1/2 + log u_i)   (the dual variable beta_i of Eq. (13))
      d/db_j = eps (1/2 + log v_j)   (gamma_j)
      d/dx_i = sum_j pi_ij dC_ij/dx_i,  pi = diag(u) K diag(v)  (Eq. (pi*))
      d/dy_j = sum_i pi_ij dC_ij/dy_j = -sum_i pi_ij dC_ij/dx_i.
    At the maximizer of Eq. (14) this is the gradient of the value s
    (envelope theorem: the first-order conditions Eq. (S1) hold there).
    Returns (grad_a, grad_b, grad_x, grad_y)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    K = gibbs_kernel(x, y, eps, r)
    pi = transport_plan(np.asarray(u, dtype=np.float64), np.asarray(v, dtype=np.float64), K)
    G = cost_gradient(x, y, r)
    grad_x = np.einsum("ij,ijk->ik", pi, G)
    grad_y = -np.einsum("ij,ijk->jk", pi, G)
    grad_a = eps * (0.5 + np.log(u))
    grad_b = eps * (0.5 + np.log(v))
    return grad_a, grad_b, grad_x, grad_y


def sinkhorn_divergence(x, a, y, b, eps, r, iters):
    """Sinkhorn divergence sd(P, P~) = s(P, P~) - (s(P, P) + s(P~, P~)) / 2
    (Remark "Entropy bias and Sinkhorn divergence"), each term the Alg. 1
    result after ``iters`` iterations from u = v = 1."""
    sxy = sinkhorn_dense(x, a, y, b, eps, r, iters)["s"]
    sxx = sinkhorn_dense(x, a, x, a, eps, r, iters)["s"]
    syy = sinkhorn_dense(y, b, y, b, eps, r, iters)["s"]
    return sxy - 0.5 * (sxx + syy)


def sinkhorn_divergence_gradient(x, a, y, b, eps, r, iters):
    """Gradient of sd(P, P~) (Remark "Entropy bias and Sinkhorn divergence")
    with respect to a, b, x, y, from the dual gradients of its three terms at
    their Alg. 1 states after ``iters`` iterations.  In s(P, P) every point is
    both a source and a target, so its gradient is the sum of the two sides'.
    Returns (grad_a, grad_b, grad_x, grad_y)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    o = sinkhorn_dense(x, a, y, b, eps, r, iters)
    ga, gb, gx, gy = dual_gradient(x, y, a, b, o["u"], o["v"], eps, r)
    ox = sinkhorn_dense(x, a, x, a, eps, r, iters)
    xa1, xa2, xx1, xx2 = dual_gradient(x, x, a, a, ox["u"], ox["v"], eps, r)
    oy = sinkhorn_dense(y, b, y, b, eps, r, iters)
    yb1, yb2, yy1, yy2 = dual_gradient(y, y, b, b, oy["u"], oy["v"], eps, r)
    return (ga - 0.5 * (xa1 + xa2), gb - 0.5 * (yb1 + yb2),
            gx - 0.5 * (xx1 + xx2), gy - 0.5 * (yy1 + yy2))


def _logsumexp(z, axis):
    zmax = np.max(z, axis=axis, keepdims=True)
    zmax = np.where(np.isfinite(zmax), zmax, 0.0)
    return np.squeeze(zmax, axis=axis) + np.log(np.sum(np.exp(z - zmax), axis=axis))


def sinkhorn_log_dense(x, a, y, b, eps, r, iters, beta0=None, gamma0=None):
    """Alg. 4 (log-domain) in FP64 with the dual variables beta, gamma of
    Eq. (11), every kernel sum formed by the log-sum-exp trick:

      log t_i  = LSE_j (gamma_j / eps - 1/2 - C_ij / eps),
      beta_i  <- eps (log a_i - log t_i + 1/2)           (Delta odd)
      log t~_j = LSE_i (beta_i / eps - 1/2 - C_ij / eps),
      gamma_j <- eps (log b_j - log t~_j + 1/2)          (Delta even).

    The +1/2 is the first-order condition d/d beta_i of Eq. (11) set to zero
    (the update as printed in Alg. 4 leaves it out).  Starts from the Set line
    beta = gamma = 0 unless given.  Returns beta, gamma, the value of Eq. (11)
    at the final state (Alg. 4 result line: sum a beta + sum b gamma - eps sum_j
    t~_j exp(gamma_j / eps - 1/2), t~ formed from the final beta) and the
    Eq. (Error) residuals."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    C = cost_matrix(x, y, r)
    beta = np.zeros(len(a)) if beta0 is None else np.array(beta0, dtype=np.float64)
    gamma = np.zeros(len(b)) if gamma0 is None else np.array(gamma0, dtype=np.float64)
    for _ in range(iters):
        log_t = _logsumexp(gamma[None, :] / eps - 0.5 - C / eps, axis=1)
        beta = eps * (np.log(a) - log_t + 0.5)
        log_tt = _logsumexp(beta[:, None] / eps - 0.5 - C / eps, axis=0)
        gamma = eps * (np.log(b) - log_tt + 0.5)
    log_pi = beta[:, None] / eps - 0.5 + gamma[None, :] / eps - 0.5 - C / eps
    row = np.exp(_logsumexp(log_pi, axis=1)) - a
    col = np.exp(_logsumexp(log_pi, axis=0)) - b
    mass = float(np.exp(_logsumexp(log_pi.ravel(), axis=0)))
    s = float(a @ beta + b @ gamma - eps * mass)
    return dict(beta=beta, gamma=gamma, s=s, err_row=float(np.linalg.norm(row)),
                err_col=float(np.linalg.norm(col)))
