"""The global two-body system: matvec (Algorithm 3), right-hand sides,
post-processing and solve drivers (Algorithm 2; Sec. 4 for mobility)."""
import numpy as np

from .geometry import coarse_nodes, coarse_sources, contacts
from .gmres import gmres
from .kernel import stokeslet, stokeslet_in
from .onebody import OneBody
from .pairs import pair_blocks


def stokes_sum(Xt, Ys, sig, mu, chunk=32):
    """u(x_m) = sum_n S(x_m, y_n) sig_n by direct summation (eq. (stokes_sum));
    Xt (m, 2), Ys (n, 2), sig (n, 2) -> (m, 2)."""
    Xt = Xt.reshape(-1, 2)
    Ys = Ys.reshape(-1, 2)
    sig = sig.reshape(-1, 2)
    out = np.zeros((Xt.shape[0], 2))
    c = 1.0 / (4.0 * np.pi * mu)
    for a in range(0, Xt.shape[0], chunk):
        xs = Xt[a:a + chunk]
        dx = xs[:, None, 0] - Ys[None, :, 0]
        dy = xs[:, None, 1] - Ys[None, :, 1]
        r2 = dx * dx + dy * dy
        lg = 0.5 * np.log(r2)
        dot = (dx * sig[None, :, 0] + dy * sig[None, :, 1]) / r2
        out[a:a + chunk, 0] = c * np.sum(-lg * sig[None, :, 0] + dot * dx, axis=1)
        out[a:a + chunk, 1] = c * np.sum(-lg * sig[None, :, 1] + dot * dy, axis=1)
    return out


class System:
    """Geometry, one-body factors and pair blocks of one problem.

    problem: "resistance" or "mobility".  blocks: optional list of
    {"A", "E"} per contact to use instead of computing them.  keep_fine:
    also keep each pair's fine solution Z, fine sources Yf and fine rigid
    matrix Kf (the flowEval data of Algorithm 2, for oracle.flow).
    """

    def __init__(self, centres, radii, p, problem, blocks=None, dense_limit=2.5e9, keep_fine=False):
        self.p = p
        self.problem = problem
        self.centres = np.asarray(centres, dtype=np.float64)
        self.radii = np.asarray(radii, dtype=np.float64)
        P = self.P = len(self.radii)
        self.onebody = {}
        for r in np.unique(self.radii):
            self.onebody[float(r)] = OneBody(float(r), p, problem)
        self.ob = [self.onebody[float(r)] for r in self.radii]
        self.X = np.stack([coarse_nodes(self.centres[i], self.radii[i], p) for i in range(P)])
        self.Y = np.stack([coarse_sources(self.centres[i], self.radii[i], p) for i in range(P)])
        self.pairs = contacts(self.centres, self.radii, p.delta_c)
        self.rho = p.rho if p.rho > 0 else float(self.radii.min())
        if blocks is None:
            blocks = [pair_blocks(self.centres[i], self.radii[i], self.centres[k], self.radii[k],
                                  self.ob[i], self.ob[k], p, problem, self.rho, keep=keep_fine)
                      for i, k in self.pairs]
            if keep_fine:
                keys = ("A", "E", "Z", "Yf", "Kf", "rank_F", "rank_C")
                blocks = [{q: b[q] for q in keys} for b in blocks]
        self.blocks = blocks
        nbytes = (2 * P * p.Mc) * (2 * P * p.Nc) * 8
        self.S_all = None
        if nbytes <= dense_limit:
            self.S_all = stokeslet(self.X.reshape(-1, 2), self.Y.reshape(-1, 2), p.mu)

    # -- pieces of Algorithm 3 -------------------------------------------
    def lam_bar(self, mu):
        """Step 1a: lam_bar^(i) = Pi^+ mu^(i) (eq. (howG+) / eq. (SL))."""
        return np.stack([self.ob[i].apply_pinv(mu[i].ravel()) for i in range(self.P)])

    def proj(self, i, lam):
        """Strengths fed to Stokeslet sums: lam itself for resistance,
        (I - L) lam for mobility (Sec. 4.4)."""
        return self.ob[i].proj @ lam

    def far_field(self, sig, targets):
        """Step 2a over the given target disks, every source included."""
        if self.S_all is not None:
            u = (self.S_all @ sig.ravel()).reshape(self.P, -1)
            return u[targets]
        Xt = self.X[targets].reshape(-1, 2)
        return stokes_sum(Xt, self.Y.reshape(-1, 2), sig.reshape(-1, 2), self.p.mu).reshape(len(targets), -1)

    def matvec(self, mu, targets=None):
        """Algorithm 3 for the resistance problem, and for mobility with every
        Stokeslet strength replaced by its projection (I - L) lam (Sec. 4.4).
        mu: (P, 2 M_c).  Returns u at the target disks (all by default)."""
        P, p = self.P, self.p
        mu = mu.reshape(P, 2 * p.Mc)
        targets = np.arange(P) if targets is None else np.asarray(targets)
        lb = self.lam_bar(mu)                                   # Step 1a
        lam = lb.copy()
        tildes = []
        n = 2 * p.Nc
        for (i, k), blk in zip(self.pairs, self.blocks):         # Step 1b
            t = blk["A"] @ np.concatenate([lb[i], lb[k]])
            lam[i] += t[:n]
            lam[k] += t[n:]
            tildes.append(t)
        sig = np.stack([self.proj(i, lam[i]) for i in range(P)])
        u = self.far_field(sig, targets)                         # Step 2a
        pos = {int(t): a for a, t in enumerate(targets)}
        mu_S = lambda a, b: stokeslet(self.X[a], self.Y[b], p.mu)  # S^(ab)
        for (i, k), t in zip(self.pairs, tildes):                # Step 2b
            ti = self.proj(i, t[:n])
            tk = self.proj(k, t[n:])
            if i in pos:
                # - [P S^(ik)] lam~  - H^(k,i) mu^(k), H^(k,i) = S^(ik) Pi^+ (proj.)
                u[pos[i]] -= self.ob[i].P @ ti + mu_S(i, k) @ (tk + self.proj(k, lb[k]))
            if k in pos:
                u[pos[k]] -= mu_S(k, i) @ (ti + self.proj(i, lb[i])) + self.ob[k].P @ tk
        for i in targets:                                        # identity fix
            u[pos[int(i)]] -= self.ob[i].P @ self.proj(i, lb[i]) - mu[i]
        return u

    def matvec_exclusion(self, mu, targets=None, dtype=np.float64):
        """Algorithm 3 with Step 2b and the identity step carried out before
        the Stokeslet sums instead of after them.  Expanding Step 2b, every
        self term and every close partner's own one-body and pair-correction
        strengths cancel exactly, which leaves

          u^(i) = mu^(i) + sum_{k not in C(i), k != i} S^(ik) sigma^(k)
                + sum_{k in C(i)} S^(ik) proj_k( sum_{n in C(k), n != i} lam~_k^(k-n) )

        (C(i): the close partners of i; lam~_k^(k-n): the correction that pair
        (k, n) adds to disk k in Step 1b; sigma = proj(lam)).  Nothing is
        added and subtracted again.  Every operation after the one-body and
        pair blocks (Step 1a, Step 1b, projections, the sums) runs in `dtype`;
        with np.longdouble this is an extended-precision evaluation of the
        same FP64 inputs (blocks, factors, points, mu).  Returns u at the
        target disks (all by default) as float64."""
        P, p = self.P, self.p
        n = 2 * p.Nc
        targets = np.arange(P) if targets is None else np.asarray(targets)
        mu = np.asarray(mu, dtype=np.float64).reshape(P, 2 * p.Mc).astype(dtype)
        lb = np.stack([self.ob[i].pinv.VSi.astype(dtype) @ (self.ob[i].pinv.Ut.astype(dtype) @ mu[i])
                       for i in range(P)])                                  # Step 1a
        lam = lb.copy()
        corr = {}                                                            # corr[(a, b)]: pair (a, b)'s share on a
        for (i, k), blk in zip(self.pairs, self.blocks):                     # Step 1b
            t = blk["A"].astype(dtype) @ np.concatenate([lb[i], lb[k]])
            lam[i] += t[:n]
            lam[k] += t[n:]
            corr[(i, k)], corr[(k, i)] = t[:n], t[n:]
        prj = {float(r): ob.proj.astype(dtype) for r, ob in self.onebody.items()}
        proj = lambda k, v: prj[float(self.radii[k])] @ v
        partners = {i: set() for i in range(P)}
        for i, k in self.pairs:
            partners[i].add(k)
            partners[k].add(i)
        u = np.empty((len(targets), 2 * p.Mc), dtype=dtype)
        for a, i in enumerate(targets):
            i = int(i)
            acc = mu[i].copy()
            for k in range(P):
                if k == i:
                    continue
                if k in partners[i]:
                    own = np.zeros(n, dtype=dtype)
                    for m in sorted(partners[k] - {i}):
                        own = own + corr[(k, m)]
                    s_k = proj(k, own)
                else:
                    s_k = proj(k, lam[k])
                acc = acc + stokeslet_in(self.X[i], self.Y[k], p.mu, dtype) @ s_k
            u[a] = acc
        return u.astype(np.float64)

    def exclusion_condition(self, mu, targets=None):
        """Rounding scale of the exclusion form's sums at the target disks:
        the 2-norm of the sum of |S^(ik)| |s_k| over the terms that those sums
        add, divided by the 2-norm of the result.  An FP64 evaluation of the
        sums, in any order, errs by about eps_64 times this (relative), and so
        does an FP64 evaluation of the strengths s_k that feed them (a
        relative error of eps in s_k moves the result by that much)."""
        P, p = self.P, self.p
        n = 2 * p.Nc
        targets = np.arange(P) if targets is None else np.asarray(targets)
        mu = np.asarray(mu, dtype=np.float64).reshape(P, 2 * p.Mc)
        lb = self.lam_bar(mu)
        lam = lb.copy()
        corr = {}
        for (i, k), blk in zip(self.pairs, self.blocks):
            t = blk["A"] @ np.concatenate([lb[i], lb[k]])
            lam[i] += t[:n]
            lam[k] += t[n:]
            corr[(i, k)], corr[(k, i)] = t[:n], t[n:]
        partners = {i: set() for i in range(P)}
        for i, k in self.pairs:
            partners[i].add(k)
            partners[k].add(i)
        absum = np.zeros((len(targets), 2 * p.Mc))
        for a, i in enumerate(targets):
            i = int(i)
            absum[a] = np.abs(mu[i])
            for k in range(P):
                if k == i:
                    continue
                if k in partners[i]:
                    s_k = self.proj(k, sum((corr[(k, m)] for m in partners[k] - {i}), np.zeros(n)))
                else:
                    s_k = self.proj(k, lam[k])
                absum[a] += np.abs(stokeslet(self.X[i], self.Y[k], p.mu)) @ np.abs(s_k)
        u = self.matvec_exclusion(mu, targets)
        return float(np.linalg.norm(absum) / np.linalg.norm(u))

    # -- right-hand sides and post-processing ----------------------------
    def rhs_resistance(self, vel):
        """g^(i) at the coarse nodes, eq. (rigidbc): v + omega (x - c)^perp."""
        vel = np.asarray(vel, dtype=np.float64).reshape(self.P, 3)
        g = np.zeros((self.P, self.p.Mc, 2))
        rel = self.X - self.centres[:, None, :]
        g[:, :, 0] = vel[:, 0:1] - vel[:, 2:3] * rel[:, :, 1]
        g[:, :, 1] = vel[:, 1:2] + vel[:, 2:3] * rel[:, :, 0]
        return g.reshape(self.P, -1)

    def completion_strengths(self, ft):
        """lam_0^(i) = K (K^T K)^{-1} [f; t]^(i), so that K^T lam_0 = [f; t]
        (Sec. 4.1, completion flow)."""
        ft = np.asarray(ft, dtype=np.float64).reshape(self.P, 3)
        return np.stack([self.ob[i].K @ np.linalg.solve(self.ob[i].K.T @ self.ob[i].K, ft[i])
                         for i in range(self.P)])

    def rhs_mobility(self, ft, targets=None):
        """b = -u_0, u_0^(i) = sum_k S(X^(i), Y^(k)) lam_0^(k) (eq. (u0_def))."""
        lam0 = self.completion_strengths(ft)
        targets = np.arange(self.P) if targets is None else np.asarray(targets)
        return -self.far_field(lam0, targets)

    def post(self, mu):
        """Resistance: [f; t]^(i) = K^T lam_bar^(i) + sum_pairs E lam_bar_pair
        (eq. (two_force)).  Mobility: [v; omega]^(i) = -K^T lam_bar^(i) +
        sum_pairs E lam_bar_pair (eqs. (rbm_ansatz), (rbm2))."""
        lb = self.lam_bar(mu.reshape(self.P, -1))
        sgn = 1.0 if self.problem == "resistance" else -1.0
        out = np.stack([sgn * (self.ob[i].K.T @ lb[i]) for i in range(self.P)])
        for (i, k), blk in zip(self.pairs, self.blocks):
            e = blk["E"] @ np.concatenate([lb[i], lb[k]])
            out[i] += e[:3]
            out[k] += e[3:]
        return out

    def solve(self, data, tol=None, maxit=None):
        """Algorithm 2 (resistance: data = (v_x, v_y, omega) per disk, returns
        (f_x, f_y, t)); Sec. 4 (mobility: data = (f_x, f_y, t), returns
        (v_x, v_y, omega))."""
        p = self.p
        tol = p.tol if tol is None else tol
        maxit = p.maxit if maxit is None else maxit
        b = self.rhs_resistance(data) if self.problem == "resistance" else self.rhs_mobility(data)
        mu, info = gmres(lambda x: self.matvec(x), b, tol, maxit)
        info["mu"] = mu
        return self.post(mu), info
