"""Trace of phi and the exchangeable Nystrom trace estimator (Alg. 1, step
"XNysTrace(Y, Omega)"; the estimator is the one of Epperly, Tropp and
Webber's XTrace paper, which the paper cites for it). Dense FP64; test
infrastructure only.

Reading used for the details the paper leaves open:
  * test vectors: the columns omega_i of Omega, exactly as given;
  * no stabilising shift (the operators estimated here are positive
    definite with bounded condition number, so Omega_{-i}^T A Omega_{-i} is
    well conditioned); the pseudo-inverse is a plain Moore-Penrose inverse;
  * estimate = mean_i t_i, error estimate = std(t_i) / sqrt(M) with the
    sample standard deviation (divisor M - 1).
"""
import numpy as np


def exact_trace(phi):
    return float(np.trace(phi))


def nystrom(Y, Om):
    """Nystrom approximation A_hat = Y (Om^T Y)^+ Y^T from Y = A Om."""
    return Y @ np.linalg.pinv(Om.T @ Y) @ Y.T


def xnystrace(A, Omega):
    """Literal leave-one-out definition: for i = 1..M the Nystrom
    approximation A_hat_(i) is built from the other M - 1 test vectors and
    t_i = tr(A_hat_(i)) + omega_i^T (A - A_hat_(i)) omega_i.
    Returns (mean t_i, std(t_i) / sqrt(M), t)."""
    n, M = Omega.shape
    Y = A @ Omega
    t = np.empty(M)
    for i in range(M):
        keep = [j for j in range(M) if j != i]
        Ah = nystrom(Y[:, keep], Omega[:, keep])
        w = Omega[:, i]
        t[i] = np.trace(Ah) + w @ (A @ w) - w @ (Ah @ w)
    return float(t.mean()), float(t.std(ddof=1) / np.sqrt(M)), t


def return_probability(Lap, ts):
    """p(t) = tr(exp(-t L)) / n (Sec. 4.4, Eq. average_return_probabilities),
    from the eigenvalues of the symmetric L."""
    lam = np.linalg.eigvalsh(Lap)
    return np.array([np.exp(-t * lam).sum() / len(lam) for t in ts])


def xnys_return_probability(Lap, Omega, ts):
    """Alg. 1 with exact Y(t): the literal leave-one-out XNysTrace of
    exp(-t L) with the test vectors Omega, divided by n, for each t.
    Returns a list of (estimate, error estimate)."""
    lam, Q = np.linalg.eigh(Lap)
    n = len(lam)
    out = []
    for t in ts:
        E = (Q * np.exp(-t * lam)) @ Q.T
        est, err, _ = xnystrace(E, Omega)
        out.append((est / n, err / n))
    return out
