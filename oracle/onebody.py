"""One-body MFS factors (Sec. 3.1 resistance, Sec. 4.1 mobility)."""
import numpy as np

from .geometry import coarse_nodes, coarse_sources
from .kernel import TSVD, rigid_matrix, rigid_projector, stokeslet


class OneBody:
    """Self-interaction block and its truncated pseudo-inverse for a disk of
    radius r (translation invariant, so shared by all disks of that radius).

    resistance: P = S(X, Y), lam_bar = P^+ mu (eq. (howG+)).
    mobility:   S_L = P (I - L) + B K^T, lam_bar = S_L^+ mu (eq. (SL)),
                strengths fed to Stokeslet sums are (I - L) lam_bar
                (eq. (phi_eq)).
    """

    def __init__(self, r, p, problem):
        c = np.zeros(2)
        self.r = r
        self.Y = coarse_sources(c, r, p)
        self.X = coarse_nodes(c, r, p)
        self.P = stokeslet(self.X, self.Y, p.mu)
        self.K = rigid_matrix(self.Y, c)
        self.B = rigid_matrix(self.X, c)
        n = 2 * p.Nc
        if problem == "resistance":
            self.proj = np.eye(n)
            M = self.P
        else:
            self.L = rigid_projector(self.K)
            self.proj = np.eye(n) - self.L
            M = self.P @ self.proj + self.B @ self.K.T
        self.M = M
        self.pinv = TSVD(M, p.eps_trunc)

    def apply_pinv(self, mu):
        """lam_bar = P^+ mu (resistance) or S_L^+ mu (mobility)."""
        return self.pinv.apply(mu)
