"""Spectral quantities that fix the admissible parameters (Prop. whe-we-converge,
Prop. CGworks, Sec. 4.1.2). Dense FP64; test infrastructure only."""
import numpy as np

from .walks import resolvent_matrix


def companion(A, mu):
    """Z = [[O, I], [mu (mu I - D), A]] (Eq. Zdef)."""
    n = A.shape[0]
    D = np.diag(A.sum(axis=1))
    Z = np.zeros((2 * n, 2 * n))
    Z[:n, n:] = np.eye(n)
    Z[n:, :n] = mu * (mu * np.eye(n) - D)
    Z[n:, n:] = A
    return Z


def rho_companion(A, mu):
    """rho(Z), the spectral radius bounding the resolvent's alpha (Prop. whe-we-converge)."""
    return float(np.abs(np.linalg.eigvals(companion(A, mu))).max())


def lambda_max(A):
    """Largest eigenvalue of the symmetric adjacency (= rho(A))."""
    return float(np.linalg.eigvalsh(A)[-1])


def lambda_min_resolvent(A, mu, t):
    return float(np.linalg.eigvalsh(resolvent_matrix(A, mu, t))[0])


def first_singular_t(A, mu, lo=0.0, hi=None, iters=200):
    """First t > 0 at which M_mu(t) becomes singular, by bisection on the sign
    of lambda_min(M_mu(t)). det M_mu(t) = 0 exactly when 1/t is an eigenvalue
    of Z, and M_mu(0) = I, so the root is 1 / rho(Z) when rho(Z) is a real
    eigenvalue of Z (the Perron root for a connected graph)."""
    if hi is None:
        hi = 1.0
        while lambda_min_resolvent(A, mu, hi) > 0.0 and hi < 1e6:
            hi *= 2.0
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if lambda_min_resolvent(A, mu, mid) > 0.0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)
