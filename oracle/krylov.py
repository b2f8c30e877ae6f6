"""Plain CPU FP64 Krylov evaluation of the walk Laplacians (Sec. 4), the
steps in the paper's order: each phi V is one conjugate-gradient solve with
the deformed Laplacian M (Sec. 4.2), and exp(-tau L) u0 is the Lanczos
approximation |u0| Q_m exp(-tau T_m) e_1 (Sec. 4.1), with exp(-tau T_m)
from the symmetric eigendecomposition of the small tridiagonal T_m.

scipy.sparse supplies the sparse matrix-vector product; numpy the small
eigendecomposition. Nothing is blocked or fused. Iteration counts are
returned so that timings can be expressed in operator applications.
Test infrastructure only (see the package header).
"""
import numpy as np
import scipy.sparse as sp


def adjacency(row_ptr, col_idx, n):
    return sp.csr_matrix((np.ones(len(col_idx)), np.asarray(col_idx), np.asarray(row_ptr)), shape=(n, n))


def resolvent_operator(A, mu, alpha):
    """M_mu(alpha) = (1 - mu^2 alpha^2) I - alpha A + alpha^2 mu D (sparse)."""
    n = A.shape[0]
    d = np.asarray(A.sum(axis=1)).ravel()
    return sp.csr_matrix((1.0 - mu * mu * alpha * alpha) * sp.eye(n) - alpha * A + alpha * alpha * mu * sp.diags(d))


def cg(M, B, tol, maxit=10000):
    """Conjugate gradients (Hestenes and Stiefel), one recurrence per column of
    B run side by side; stops a column when |r| <= tol |b|. Returns (X, iterations
    of the slowest column)."""
    B = np.asarray(B, dtype=np.float64)
    one = B.ndim == 1
    if one:
        B = B[:, None]
    X = np.zeros_like(B)
    R = B.copy()
    P = R.copy()
    g = (R * R).sum(0)
    bn = np.sqrt(g)
    active = bn > 0
    it = 0
    while active.any() and it < maxit:
        Q = M @ P
        a = np.where(active, g / np.where(active, (P * Q).sum(0), 1.0), 0.0)
        X += a * P
        R -= a * Q
        gn = (R * R).sum(0)
        it += 1
        active = active & (np.sqrt(gn) > tol * bn)
        beta = np.where(active, gn / np.where(g > 0, g, 1.0), 0.0)
        P = R + beta * P
        g = gn
    return (X[:, 0] if one else X), it


class ResolventLaplacian:
    """Apply L = D_f - phi with phi = a M^{-1} (resolvent walk Laplacian)."""

    def __init__(self, A, mu, alpha, tol=1e-12):
        self.M = resolvent_operator(A, mu, alpha)
        self.a = 1.0 - mu * mu * alpha * alpha
        self.tol = tol
        self.applications = 0
        n = A.shape[0]
        x, it = cg(self.M, self.a * np.ones(n), tol)
        self.applications += it
        self.Df = x

    def apply(self, V):
        X, it = cg(self.M, self.a * V, self.tol)
        self.applications += it
        return (self.Df[:, None] * V if V.ndim == 2 else self.Df * V) - X


def lanczos_expmv(apply_L, u0, taus, tol=1e-10, m_max=400, check=4):
    """exp(-tau L) u0 for each tau by the Lanczos process on the symmetric L
    (no reorthogonalisation), stopping when the approximations of two checks
    apart agree to tol |y|. Returns (list of vectors, Lanczos steps)."""
    n = u0.shape[0]
    beta0 = np.linalg.norm(u0)
    if beta0 == 0:
        return [np.zeros(n) for _ in taus], 0
    V = [u0 / beta0]
    al, be = [], []
    prev = None
    m = 0
    for j in range(m_max):
        w = apply_L(V[j])
        a = V[j] @ w
        w = w - a * V[j] - (be[-1] * V[j - 1] if j > 0 else 0.0)
        b = np.linalg.norm(w)
        al.append(a)
        be.append(b)
        m = j + 1
        done = b <= 1e-13 * (abs(a) + (be[-2] if j > 0 else 0.0))
        if m % check == 0 or done or m == m_max:
            T = np.diag(al) + np.diag(be[:-1], 1) + np.diag(be[:-1], -1)
            lam, Q = np.linalg.eigh(T)
            ys = [Q @ (np.exp(-t * lam) * Q[0]) for t in taus]
            if done:
                prev = ys
                break
            if prev is not None:
                # an approximation that underflowed to zero is not converged:
                # exp(-tau L) conserves the mass of u0 (L 1 = 0), the Krylov
                # space just has not reached the slow modes yet
                ok = all(np.linalg.norm(y) > 0 and
                         np.linalg.norm(y - np.concatenate([p, np.zeros(len(y) - len(p))])) <= tol * np.linalg.norm(y)
                         for y, p in zip(ys, prev))
                if ok:
                    prev = ys
                    break
            prev = ys
        if done:
            break
        V.append(w / b)
    Vm = np.stack(V[:m], axis=1)
    return [beta0 * (Vm @ y) for y in prev], m


def rho_companion_sparse(A, mu):
    """rho(Z) for Z = [[O, I], [mu (mu I - D), A]] (Eq. Zdef) by ARPACK on Z as
    an operator (largest-modulus eigenvalue)."""
    from scipy.sparse.linalg import LinearOperator, eigs

    n = A.shape[0]
    d = np.asarray(A.sum(axis=1)).ravel()

    def zmv(v):
        x, y = v[:n], v[n:]
        return np.concatenate([y, mu * (mu - d) * x + A @ y])

    Z = LinearOperator((2 * n, 2 * n), matvec=zmv, dtype=np.float64)
    return float(np.abs(eigs(Z, k=1, which="LM", return_eigenvectors=False, tol=1e-10)[0]))
