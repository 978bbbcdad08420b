"""Pair precompute: fine local solve and peanut compression (Sec. 3.2-3.4,
Sec. 4.3-4.4, Algorithm 2 precomputation loop)."""
import numpy as np

from .geometry import coarse_sources, fine_sets, peanut
from .kernel import TSVD, blockdiag, rigid_matrix, rigid_projector, stokeslet


def pair_blocks(c1, r1, c2, r2, ob1, ob2, p, problem, rho, keep=False):
    """Coarse-to-coarse correction A (4N_c x 4N_c) and extraction matrix E
    (6 x 4N_c) of one close pair.

    Resistance (Sec. 3.2-3.4):
      F = S(X_f, Y_f), blkQ = [[0, Q21], [Q12, 0]] with Q21 = S(X_f on 1, Y^2),
      Q12 = S(X_f on 2, Y^1) (eq. (sys2b) and the symmetrizing remark),
      Z = F^+ blkQ (truncated at eps_trunc_fine, eq. (bfm)),
      C = S(z, Y^(1-2)), D = S(z, Y_f) (eq. (peanut)),
      A = -C^+ D Z (eq. (Amat)),
      beta = -Z lam_bar_pair, so the fine-source force/torque correction is
      E = -blockdiag(Kf1^T, Kf2^T) Z (eqs. (force_syst), (force_ext); the
      printed eq. (force_ext) drops the minus sign and the transposes).
    Mobility (Sec. 4.3-4.4, projected maps after eq. (peanut_mob)):
      Q's carry (I - L), F = S(X_f, Y_f)(I - Lf) + blockdiag(Bf1 Kf1^T,
      Bf2 Kf2^T), C = S(z, Y^(1-2))(I - L^pair), D = S(z, Y_f)(I - Lf);
      velocities get -Kf^T beta = +Kf^T Z lam_bar (eq. (rbm2)), so
      E = +blockdiag(Kf1^T, Kf2^T) Z.
    """
    mu = p.mu
    fs = fine_sets(c1, r1, c2, r2, p)
    Yf1, Yf2, Xf1, Xf2 = fs["Y1"], fs["Y2"], fs["X1"], fs["X2"]
    Yf = np.concatenate([Yf1, Yf2])
    Xf = np.concatenate([Xf1, Xf2])
    Y1 = coarse_sources(c1, r1, p)
    Y2 = coarse_sources(c2, r2, p)
    F = stokeslet(Xf, Yf, mu)
    Q21 = stokeslet(Xf1, Y2, mu)
    Q12 = stokeslet(Xf2, Y1, mu)
    Kf1 = rigid_matrix(Yf1, c1)
    Kf2 = rigid_matrix(Yf2, c2)
    z = peanut(c1, r1, c2, r2, rho, p.Mp)
    C = stokeslet(z, np.concatenate([Y1, Y2]), mu)
    D = stokeslet(z, Yf, mu)
    if problem == "mobility":
        Lf = blockdiag(rigid_projector(Kf1), rigid_projector(Kf2))
        Pf = np.eye(Lf.shape[0]) - Lf
        Bf1 = rigid_matrix(Xf1, c1)
        Bf2 = rigid_matrix(Xf2, c2)
        F = F @ Pf + blockdiag(Bf1 @ Kf1.T, Bf2 @ Kf2.T)
        Q21 = Q21 @ ob2.proj
        Q12 = Q12 @ ob1.proj
        C = C @ blockdiag(ob1.proj, ob2.proj)
        D = D @ Pf
    n1 = Q21.shape[0]
    nc = Q21.shape[1]
    blkQ = np.zeros((F.shape[0], 2 * nc))
    blkQ[:n1, nc:] = Q21
    blkQ[n1:, :nc] = Q12
    Fp = TSVD(F, p.eps_trunc_fine)
    Z = Fp.apply(blkQ)
    Cp = TSVD(C, p.eps_trunc)
    A = -Cp.apply(D @ Z)
    Kf = blockdiag(Kf1, Kf2)
    E = (-1.0 if problem == "resistance" else 1.0) * (Kf.T @ Z)
    out = {"A": A, "E": E, "rank_F": Fp.rank, "rank_C": Cp.rank,
           "shape_F": F.shape, "n_enh": (fs["n_enh1"], fs["n_enh2"]),
           "fine_residual": float(np.linalg.norm(F @ Z - blkQ) / np.linalg.norm(blkQ)),
           "peanut_residual": float(np.linalg.norm(C @ A + D @ Z) / np.linalg.norm(D @ Z))}
    if keep:
        out.update(F=F, blkQ=blkQ, Z=Z, C=C, D=D, Yf=Yf, Xf=Xf, z=z, Kf=Kf)
    return out
