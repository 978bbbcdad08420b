"""Unrestarted GMRES with modified Gram-Schmidt Arnoldi and Givens rotations,
x0 = 0, stopping at ||b - A x|| / ||b|| <= tol (the solver of Algorithm 2;
restart, start vector and orthogonalization are not specified by the paper)."""
import numpy as np


def gmres(matvec, b, tol, maxit):
    """Solve A x = b for the operator `matvec` (Algorithm 2's GMRES on the
    two-body system, Algorithm 3 as the matvec).  Returns x and a record
    with the iteration count, the final relative residual and its history."""
    n = b.size
    beta = np.linalg.norm(b)
    hist = [1.0]
    if beta == 0.0:
        return np.zeros_like(b), {"iters": 0, "relres": 0.0, "hist": hist}
    V = np.zeros((maxit + 1, n))
    H = np.zeros((maxit + 1, maxit))
    cs = np.zeros(maxit)
    sn = np.zeros(maxit)
    g = np.zeros(maxit + 1)
    g[0] = beta
    V[0] = b.ravel() / beta
    j = 0
    for j in range(maxit):
        w = matvec(V[j].reshape(b.shape)).ravel()
        for i in range(j + 1):
            H[i, j] = V[i] @ w
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] > 0:
            V[j + 1] = w / H[j + 1, j]
        for i in range(j):
            t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
            H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
            H[i, j] = t
        den = np.hypot(H[j, j], H[j + 1, j])
        cs[j] = H[j, j] / den
        sn[j] = H[j + 1, j] / den
        H[j, j] = den
        H[j + 1, j] = 0.0
        g[j + 1] = -sn[j] * g[j]
        g[j] = cs[j] * g[j]
        hist.append(abs(g[j + 1]) / beta)
        if hist[-1] <= tol:
            break
    k = j + 1
    y = np.zeros(k)
    for i in range(k - 1, -1, -1):
        y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
    x = (V[:k].T @ y).reshape(b.shape)
    return x, {"iters": k, "relres": hist[-1], "hist": hist}
