"""Method parameters (Sec. 5 and Sec. 6; defaults as in Sec. 6.2)."""
from dataclasses import dataclass, replace

from .geometry import radius_rule


@dataclass(frozen=True)
class Params:
    Nc: int = 60            # coarse sources per disk
    Mc: int = 72            # coarse collocation nodes per disk
    Rc: float = 0.0         # source radius; 0 -> 1 - log(1e12)/N_c (Sec. 6)
    Nfp: int = 150          # fine proxy sources per disk (Sec. 6.2)
    Nell: int = 80          # ellipse parameter N_ell (Sec. 6.2)
    Mp: int = 200           # peanut nodes (Sec. 6.2)
    gamma: float = 0.3      # ellipse shape (Sec. 5)
    af: float = 1.2         # fine equispaced nodes = ceil(af * Nfp) (Sec. 5)
    r_mob: float = 0.6      # Moebius parameter r (Sec. 5)
    aell: float = 5.0       # Moebius nodes = aell * Nell (Sec. 5)
    delta_c: float = 0.2    # contact threshold (Sec. 6)
    eps_trunc: float = 1e-14        # SVD truncation (Sec. 6.2)
    eps_trunc_fine: float = 1e-11   # truncation for the fine solve (Sec. 6.2)
    mu: float = 1.0         # viscosity (never given a value in the paper)
    tol: float = 1e-7       # GMRES tolerance (Sec. 6.2)
    maxit: int = 300
    rho: float = 0.0        # peanut rolling radius; 0 -> smallest disk radius

    def __post_init__(self):
        if not (0.0 < self.Rc_eff < 1.0) or not (0.0 < self.Rf_eff < 1.0):
            raise ValueError("source radii must lie in (0, 1): N_c and N_fp must exceed "
                             "log(1e12) ~ 27.6 when the radius rule is used")

    @property
    def Rc_eff(self):
        return self.Rc if self.Rc > 0 else radius_rule(self.Nc)

    @property
    def Rf_eff(self):
        return radius_rule(self.Nfp)

    def with_(self, **kw):
        return replace(self, **kw)


# Two unit disks at gap 1e-3: 36 coarse sources on radius 0.7, 72 nodes,
# 400 fine proxies per disk, FP64, GMRES tol 1e-10.
PAIR_SMALL = Params(Nc=36, Mc=72, Rc=0.7, Nfp=400, tol=1e-10)
# Packings: N_c = 60 (72 vector unknowns per body), paper fine parameters.
PACKING = Params(Nc=60, Mc=72)
POLY = Params(Nc=60, Mc=72, delta_c=0.1)
