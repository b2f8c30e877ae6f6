"""Walk-generating matrix functions and the walk-based Laplacians, dense FP64.

Test infrastructure only (see the package header). Each function restates a
definition of Sec. 3 of the paper; the closed forms are checked against the
series definitions by the oracle's own tests, never assumed.
"""
import math

import numpy as np


# ------------------------------------------------------------------ walk counts
def nbt_counts(A, kmax):
    """p_0..p_kmax: nonbacktracking walk counts, Eq. Br (Sec. 3.2):
    p_0 = I, p_1 = A, p_2 = A^2 - D, p_k = A p_{k-1} + (I - D) p_{k-2}, k >= 3."""
    n = A.shape[0]
    I = np.eye(n)
    D = np.diag(A.sum(axis=1))
    p = [I, A.copy(), A @ A - D]
    for k in range(3, kmax + 1):
        p.append(A @ p[k - 1] + (I - D) @ p[k - 2])
    return p[: kmax + 1]


def btdw_counts(A, mu, kmax):
    """q_0..q_kmax: backtrack-downweighted walk counts, Eq. qrec (Sec. 3.2):
    q_0 = I, q_1 = A, q_2 = A^2 - mu D, and q_{k+1} = A q_k + mu (mu I - D) q_{k-1}.
    The recurrence is applied from k = 2 on (q_3 onwards); at k = 1 it would
    not reproduce the stated q_2."""
    n = A.shape[0]
    I = np.eye(n)
    D = np.diag(A.sum(axis=1))
    q = [I, A.copy(), A @ A - mu * D]
    for k in range(2, kmax):
        q.append(A @ q[k] + mu * (mu * I - D) @ q[k - 1])
    return q[: kmax + 1]


# ------------------------------------------------------------------ phi(A, c)
def resolvent_coeffs(alpha):
    """c = (1, alpha, alpha^2, ...): the resolvent f(x) = (1 - alpha x)^{-1} (Sec. 3.2.1)."""
    return lambda k: alpha ** k


def exp_coeffs(beta):
    """c_k = beta^k / k!: f(x) = exp(beta x) (Sec. 3.2.1 and Sec. 4.1.2)."""
    return lambda k: beta ** k / math.factorial(k)


def phi_series(A, mu, coeff, kmax=4000, rel_tol=1e-18):
    """phi(A, c) = sum_k c_k q_k(A) (Prop. whe-we-converge, Def. BDTW-Laplacian),
    summed term by term with the q_k of Eq. qrec until |c_k q_k|_max falls
    below rel_tol * |phi|_max for three consecutive terms."""
    n = A.shape[0]
    I = np.eye(n)
    D = np.diag(A.sum(axis=1))
    q_prev, q_cur = I, A.copy()
    phi = coeff(0) * I + coeff(1) * A
    small = 0
    q_next = A @ A - mu * D          # q_2
    for k in range(2, kmax + 1):
        term = coeff(k) * q_next
        phi = phi + term
        if np.abs(term).max() <= rel_tol * np.abs(phi).max():
            small += 1
            if small >= 3:
                return phi
        else:
            small = 0
        q_prev, q_cur = q_cur, q_next
        q_next = A @ q_cur + mu * (mu * I - D) @ q_prev
    raise RuntimeError("phi_series did not converge; is alpha * rho(Z) < 1?")


def resolvent_matrix(A, mu, alpha):
    """M_mu(alpha) = (1 - mu^2 alpha^2) I - alpha A + alpha^2 mu D.

    For mu = 1 this is the deformed Laplacian of Eq. deformed,
    I - alpha A - alpha^2 (I - D); for mu = 0 it is I - alpha A. The general-mu
    form is the extension the paper states after Prop. CGworks; it follows
    from Eq. qrec by multiplying sum_k alpha^k q_k by M_mu(alpha)."""
    n = A.shape[0]
    D = np.diag(A.sum(axis=1))
    return (1.0 - mu * mu * alpha * alpha) * np.eye(n) - alpha * A + alpha * alpha * mu * D


def phi_resolvent_closed(A, mu, alpha):
    """phi = (1 - mu^2 alpha^2) M_mu(alpha)^{-1} (Eq. deformed, general mu)."""
    n = A.shape[0]
    a = 1.0 - mu * mu * alpha * alpha
    return a * np.linalg.solve(resolvent_matrix(A, mu, alpha), np.eye(n))


def f_of_symmetric(A, f):
    """f(A) = Q f(Lambda) Q^T for symmetric A (spectral definition of a matrix
    function, used for the all-walk case mu = 0, Def. transformedlaplacian)."""
    lam, Q = np.linalg.eigh(A)
    return (Q * f(lam)) @ Q.T


def phi_allwalk_resolvent_eig(A, alpha):
    return f_of_symmetric(A, lambda x: 1.0 / (1.0 - alpha * x))


def phi_allwalk_exp_eig(A, beta):
    return f_of_symmetric(A, lambda x: np.exp(beta * x))


# ------------------------------------------------------------------ Laplacians
def walk_degrees(phi):
    """t(f) = phi 1: total communicability / walk degrees D_f (Sec. 3.1)."""
    return phi.sum(axis=1)


def walk_laplacian(phi):
    """L = diag(phi 1) - phi (Eq. f-laplacian, Eq. weighted_laplacian)."""
    return np.diag(walk_degrees(phi)) - phi


def apply_laplacian(phi, V):
    """L V = D_f (.) V - phi V, column by column."""
    return walk_degrees(phi)[:, None] * V - phi @ V


def diffusion(Lap, U0, taus):
    """u(tau) = exp(-tau L) u0 for each tau (Eq. diffusion_on_G_with_downweighted_walk,
    column form; L is symmetric so p0 exp(-t L) is its transpose). Uses the
    symmetric eigendecomposition of L."""
    lam, Q = np.linalg.eigh(Lap)
    C = Q.T @ U0
    return [Q @ (np.exp(-t * lam)[:, None] * C) for t in taus]


def markov_stationary(phi):
    """Stationary distribution of P = I - D^{-1} L with D = diag(phi 1).

    The paper defines the chain through Eq. let_there_be_markov; the values
    printed in Fig. 1 correspond to D = diag(phi 1) (the walk degrees), for
    which P = D^{-1} phi is row-stochastic and pi = phi 1 / (1^T phi 1)."""
    d = walk_degrees(phi)
    P = phi / d[:, None]
    w, V = np.linalg.eig(P.T)
    i = int(np.argmin(np.abs(w - 1.0)))
    pi = np.real(V[:, i])
    return pi / pi.sum()


def markov_evolve(phi, P0, steps):
    """Distributions of the discrete-time chain p_{s+1} = p_s P of Sec. 3.3
    (Eq. let_there_be_markov) with D = diag(phi 1), i.e. P = D^{-1} phi, after
    each step count in `steps` (non-decreasing). P0 holds start distributions
    as columns; in column form a step is p <- P^T p."""
    d = walk_degrees(phi)
    P = phi / d[:, None]
    out, cur, s = [], np.array(P0, dtype=np.float64), 0
    for t in steps:
        while s < t:
            cur = P.T @ cur
            s += 1
        out.append(cur.copy())
    return out
