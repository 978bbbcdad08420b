"""Global fine MFS on a small cluster, solved densely (the one-body baseline
of Sec. 6.1 with the union of the fine discretizations of all close pairs,
Remark "Unknowns with one-body preconditioning").  Used to pin the two-body
scheme: no compression, no preconditioner, one truncated-SVD least squares.
"""
import numpy as np

from .geometry import contacts, fine_sets, ring
from .kernel import TSVD, blockdiag, rigid_matrix, rigid_projector, stokeslet


def _unique_rows(pts, tol=1e-13):
    out = []
    for q in pts:
        if not any(np.hypot(*(q - o)) < tol for o in out):
            out.append(q)
    return np.array(out)


def fine_cluster(centres, radii, p):
    """Per-disk fine sources and nodes: every disk carries the proxies, the
    shielding-ellipse sources and the Moebius nodes of all of its close pairs
    (coincident proxy rings are merged, Remark "Combining fine sources").
    Disks without contacts keep N_fp proxies and ceil(a_f N_fp) nodes."""
    P = len(radii)
    Ys = [[] for _ in range(P)]
    Xs = [[] for _ in range(P)]
    pairs = contacts(centres, radii, p.delta_c)
    for i, k in pairs:
        fs = fine_sets(centres[i], radii[i], centres[k], radii[k], p)
        Ys[i].append(fs["Y1"]); Ys[k].append(fs["Y2"])
        Xs[i].append(fs["X1"]); Xs[k].append(fs["X2"])
    for i in range(P):
        if not Ys[i]:
            Ys[i].append(ring(centres[i], radii[i] * p.Rf_eff, p.Nfp))
            Xs[i].append(ring(centres[i], radii[i], int(np.ceil(p.af * p.Nfp))))
        Ys[i] = _unique_rows(np.concatenate(Ys[i]))
        Xs[i] = _unique_rows(np.concatenate(Xs[i]))
    return Ys, Xs


def solve(centres, radii, p, problem, data, eps=1e-11, points=None):
    """Resistance: S lam = g at all fine nodes, forces f = sum lam, torques
    sum lam . (y - c)^perp (eq. (force_eq)).  Mobility: [S (I - L) + B K^T]
    lam_bar = -S lam_0 with fine K, B, L per disk and [v; w] = -K^T lam_bar
    (eqs. (tosolve), (u0_def), (rbm_ansatz)).  With points (n, 2), also the
    flow field there: sum S(x, Y) lam (resistance) or sum S(x, Y) [(I - L)
    lam_bar + lam_0] (mobility, eq. (mob)); returns (result, field)."""
    centres = np.asarray(centres, dtype=np.float64)
    radii = np.asarray(radii, dtype=np.float64)
    Ys, Xs = fine_cluster(centres, radii, p)
    P = len(radii)
    Y = np.concatenate(Ys)
    X = np.concatenate(Xs)
    S = stokeslet(X, Y, p.mu)
    Ks = [rigid_matrix(Ys[i], centres[i]) for i in range(P)]
    Bs = [rigid_matrix(Xs[i], centres[i]) for i in range(P)]
    K = blockdiag(*Ks)
    data = np.asarray(data, dtype=np.float64).reshape(P, 3)
    if problem == "resistance":
        g = np.concatenate([Bs[i] @ data[i] for i in range(P)])
        lam = TSVD(S, eps).apply(g)
        out = (K.T @ lam).reshape(P, 3)
        if points is None:
            return out
        return out, (stokeslet(points, Y, p.mu) @ lam).reshape(-1, 2)
    L = blockdiag(*[rigid_projector(Ki) for Ki in Ks])
    B = blockdiag(*Bs)
    M = S @ (np.eye(L.shape[0]) - L) + B @ K.T
    lam0 = np.concatenate([Ks[i] @ np.linalg.solve(Ks[i].T @ Ks[i], data[i]) for i in range(P)])
    lb = TSVD(M, eps).apply(-S @ lam0)
    out = (-(K.T @ lb)).reshape(P, 3)
    if points is None:
        return out
    strength = (np.eye(L.shape[0]) - L) @ lb + lam0
    return out, (stokeslet(points, Y, p.mu) @ strength).reshape(-1, 2)
