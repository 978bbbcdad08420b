"""Flow evaluation at new boundary nodes and the relative boundary residual:
the flowEval branch of Algorithm 2 (coarse strengths lam, lam_bar and the
fine strengths beta of every close pair returned for evaluation), eq. (bfm)
for beta, and Sec. 6.1 eqs. (residual_x) and (residual).

Test infrastructure only (see oracle/__init__.py).  Written from the
definitions: the two-body representation of the flow is the sum of every
disk's one-body field (with the completion flow for mobility, eq. (mob)) and,
for every close pair, its correction field.  Outside a pair's peanut that
correction is represented by the compressed coarse strengths lam~ (eq.
(peanut), eq. (peanut_mob)); on the pair's own boundary it must be the fine
sources beta themselves (Algorithm 3's discussion of Step 2b: the coarse
correction cannot replace the fine sources on the pair).  So at a node x on
disk i,

  u(x) = sum_k S(x, Y^k) [sigma^(k) + lam_0^(k)]
         - sum_{pairs c containing i} S(x, Y^(c)) proj(lam~^(c))
         + sum_{pairs c containing i} S(x, Y_f^(c)) proj_f(beta^(c)),

sigma = proj(lam_bar + sum lam~) as in Algorithm 3, Y^(c) the coarse sources
of both disks of pair c, beta^(c) = -F^+ blkQ lam_bar^(pair) = -Z lam_bar
(eq. (bfm) with the reading of eq. (force_ext)), proj = I - L and proj_f =
I - L_f for mobility (eq. (chi_mob)), identities for resistance.  lam_0 is
the completion-flow strength (mobility only).  The boundary data are g(x) =
v + omega (x - c)^perp with the prescribed (resistance) or computed
(mobility) rigid velocities.
"""
import numpy as np

from .geometry import ring
from .kernel import rigid_projector, stokeslet_in


def eval_nodes(c, r, m):
    """m new boundary nodes, half a spacing off the angle-0 ring: angles
    2 pi (j + 1/2) / m."""
    return ring(c, r, m, offset=0.5)


def boundary_flow(sysm, mu, data, m_eval, dtype=np.float64):
    """u and g at m_eval new nodes on every boundary, [P, m_eval, 2] each, for
    the solution mu of the system (its pair blocks must keep the fine
    solution Z, the fine sources Yf and the fine rigid matrix Kf: System(...,
    keep_fine=True)).  data: the resistance problem's velocities, or the
    mobility problem's forces and torques.  dtype: the precision of the sums
    (np.longdouble for an extended-precision reference)."""
    P, p = sysm.P, sysm.p
    n = 2 * p.Nc
    mob = sysm.problem == "mobility"
    mu = np.asarray(mu, dtype=np.float64).reshape(P, 2 * p.Mc)
    data = np.asarray(data, dtype=np.float64).reshape(P, 3)
    lb = sysm.lam_bar(mu)
    lam = lb.copy()
    tild = []
    for (i, k), blk in zip(sysm.pairs, sysm.blocks):
        t = blk["A"] @ np.concatenate([lb[i], lb[k]])
        lam[i] += t[:n]
        lam[k] += t[n:]
        tild.append(t)
    sig = np.stack([sysm.proj(i, lam[i]) for i in range(P)])
    lam0 = sysm.completion_strengths(data) if mob else np.zeros_like(sig)
    src = sig + lam0
    vel = sysm.post(mu) if mob else data
    X = np.stack([eval_nodes(sysm.centres[i], sysm.radii[i], m_eval) for i in range(P)])
    u = np.zeros((P, m_eval * 2), dtype=dtype)
    for i in range(P):
        acc = np.zeros(2 * m_eval, dtype=dtype)
        for k in range(P):
            acc = acc + stokeslet_in(X[i], sysm.Y[k], p.mu, dtype) @ src[k].astype(dtype)
        for (a, b), blk, t in zip(sysm.pairs, sysm.blocks, tild):
            if i not in (a, b):
                continue
            Yc = np.concatenate([sysm.Y[a], sysm.Y[b]])
            tc = np.concatenate([sysm.proj(a, t[:n]), sysm.proj(b, t[n:])])
            acc = acc - stokeslet_in(X[i], Yc, p.mu, dtype) @ tc.astype(dtype)
            beta = -(blk["Z"] @ np.concatenate([lb[a], lb[b]]))
            if mob:
                beta = beta - rigid_projector(blk["Kf"]) @ beta
            acc = acc + stokeslet_in(X[i], blk["Yf"], p.mu, dtype) @ beta.astype(dtype)
        u[i] = acc
    rel = X - sysm.centres[:, None, :]
    g = np.empty((P, m_eval, 2))
    g[:, :, 0] = vel[:, 0:1] - vel[:, 2:3] * rel[:, :, 1]
    g[:, :, 1] = vel[:, 1:2] + vel[:, 2:3] * rel[:, :, 0]
    return u.astype(np.float64).reshape(P, m_eval, 2), g


def boundary_residual(sysm, mu, data, m_eval, dtype=np.float64):
    """Pointwise residual eps(x) = |u(x) - g(x)| (eq. (residual_x)) at the new
    nodes: per disk its maximum [P], and the relative boundary residual of
    eq. (residual), max_x eps(x) / max_i max_x |g^(i)(x)|."""
    u, g = boundary_flow(sysm, mu, data, m_eval, dtype)
    eps = np.hypot(u[:, :, 0] - g[:, :, 0], u[:, :, 1] - g[:, :, 1])
    gmax = np.hypot(g[:, :, 0], g[:, :, 1]).max()
    return eps.max(axis=1), float(eps.max() / gmax)
