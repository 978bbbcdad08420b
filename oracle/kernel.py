"""Stokeslet blocks, rigid-body matrices and truncated pseudo-inverses (FP64).

Vector layout everywhere: a field over n points is a length-2n vector with
the x and y components of point j at entries 2j and 2j+1.
"""
import numpy as np


def stokeslet(X, Y, mu=1.0):
    """2D Stokeslet matrix S(X, Y), eq. (stokeslet2d), Sec. 3:
    S(x, y) = 1/(4 pi mu) [ -log|x-y| I + (x-y)(x-y)^T / |x-y|^2 ].
    X: (m, 2) targets, Y: (n, 2) sources -> (2m, 2n)."""
    X = np.asarray(X, dtype=np.float64).reshape(-1, 2)
    Y = np.asarray(Y, dtype=np.float64).reshape(-1, 2)
    dx = X[:, None, 0] - Y[None, :, 0]
    dy = X[:, None, 1] - Y[None, :, 1]
    r2 = dx * dx + dy * dy
    lg = 0.5 * np.log(r2)
    c = 1.0 / (4.0 * np.pi * mu)
    S = np.empty((X.shape[0], 2, Y.shape[0], 2))
    S[:, 0, :, 0] = c * (-lg + dx * dx / r2)
    S[:, 0, :, 1] = c * (dx * dy / r2)
    S[:, 1, :, 0] = S[:, 0, :, 1]
    S[:, 1, :, 1] = c * (-lg + dy * dy / r2)
    return S.reshape(2 * X.shape[0], 2 * Y.shape[0])


def stokeslet_in(X, Y, mu=1.0, dtype=np.float64):
    """The Stokeslet matrix of eq. (stokeslet2d) with every operation carried
    out in `dtype` (np.float64, or np.longdouble for an extended-precision
    reference: 80-bit on x86-64, IEEE binary128 on aarch64).  The inputs are
    taken as exact values of that type."""
    X = np.asarray(X).reshape(-1, 2).astype(dtype)
    Y = np.asarray(Y).reshape(-1, 2).astype(dtype)
    dx = X[:, None, 0] - Y[None, :, 0]
    dy = X[:, None, 1] - Y[None, :, 1]
    r2 = dx * dx + dy * dy
    lg = np.log(r2) / dtype(2)
    pi = dtype(4) * np.arctan(dtype(1))
    c = dtype(1) / (dtype(4) * pi * dtype(mu))
    S = np.empty((X.shape[0], 2, Y.shape[0], 2), dtype=dtype)
    S[:, 0, :, 0] = c * (-lg + dx * dx / r2)
    S[:, 0, :, 1] = c * (dx * dy / r2)
    S[:, 1, :, 0] = S[:, 0, :, 1]
    S[:, 1, :, 1] = c * (-lg + dy * dy / r2)
    return S.reshape(2 * X.shape[0], 2 * Y.shape[0])


def rigid_matrix(pts, c):
    """Rigid-body matrix of eq. (Kmat), Sec. 3.4: rows [I_2, (y - c)^perp] per
    point, with (a, b)^perp = (-b, a) (Sec. 1, after eq. (rigidbc)).  (2n, 3).  K^T lam gives (sum lam_x,
    sum lam_y, sum lam . (y - c)^perp); B [v; w] gives v + w (x - c)^perp."""
    pts = np.asarray(pts, dtype=np.float64).reshape(-1, 2)
    d = pts - np.asarray(c, dtype=np.float64)[None, :]
    K = np.zeros((pts.shape[0], 2, 3))
    K[:, 0, 0] = 1.0
    K[:, 1, 1] = 1.0
    K[:, 0, 2] = -d[:, 1]
    K[:, 1, 2] = d[:, 0]
    return K.reshape(-1, 3)


def rigid_projector(K):
    """L = K (K^T K)^{-1} K^T, the projector onto rigid-body source strengths
    (Sec. 4.1, before eq. (phi_eq))."""
    return K @ np.linalg.solve(K.T @ K, K.T)


class TSVD:
    """Truncated pseudo-inverse applied backward-stably as in eq. (howG+), Sec. 3.1:
    x = V Sigma^+ (U^T b), keeping singular values > eps * sigma_1."""

    def __init__(self, A, eps):
        U, s, Vt = np.linalg.svd(A, full_matrices=False)
        r = int(np.sum(s > eps * s[0]))
        self.rank = r
        self.s = s
        self.Ut = U[:, :r].T.copy()
        self.VSi = (Vt[:r].T / s[:r]).copy()

    def apply(self, b):
        """x = V Sigma^+ (U^T b): U^T b first, as eq. (howG+) prescribes."""
        return self.VSi @ (self.Ut @ b)


def blockdiag(*mats):
    """Block-diagonal matrix of the given blocks (the blkdiag of the pair
    systems, e.g. blockdiag(K^(1,2)T, K^(2,1)T) in eq. (force_ext))."""
    rows = sum(m.shape[0] for m in mats)
    cols = sum(m.shape[1] for m in mats)
    out = np.zeros((rows, cols))
    i = j = 0
    for m in mats:
        out[i:i + m.shape[0], j:j + m.shape[1]] = m
        i += m.shape[0]
        j += m.shape[1]
    return out
