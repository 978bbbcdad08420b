"""Point sets of the coarse and fine MFS discretizations and contact detection.

All sets are in global coordinates, counterclockwise, angle 0 along +x.
"""
import math

import numpy as np


def radius_rule(N, eps=1e-12):
    """Source-circle radius R = 1 - log(1/eps)/N (Sec. 6, before Remark r:cpu)."""
    return 1.0 - math.log(1.0 / eps) / N


def ring(c, rad, n, offset=0.0):
    """n equispaced points on the circle of radius rad about c, starting at
    angle 2 pi offset / n in the global frame (the coarse and proxy rings of
    Sec. 3 and Sec. 5)."""
    t = 2.0 * np.pi * (np.arange(n) + offset) / n
    return np.stack([c[0] + rad * np.cos(t), c[1] + rad * np.sin(t)], axis=1)


def coarse_sources(c, r, p):
    """N_c sources equispaced on the concentric circle of radius R_c (Sec. 3,
    after eq. (stokes_sum); Sec. 5); scaled by the disk radius r."""
    return ring(c, r * p.Rc_eff, p.Nc)


def coarse_nodes(c, r, p):
    """M_c collocation nodes equispaced on the boundary (Sec. 5)."""
    return ring(c, r, p.Mc)


def contacts(centres, radii, delta_c):
    """Close pairs (i < k) with gap |c_i - c_k| - r_i - r_k <= delta_c
    (Sec. 6, first paragraph; Algorithm 2, precomputation).  Brute force."""
    P = len(radii)
    out = []
    for i in range(P):
        d = np.hypot(centres[i + 1:, 0] - centres[i, 0], centres[i + 1:, 1] - centres[i, 1])
        gap = d - radii[i] - radii[i + 1:]
        for k in np.nonzero(gap <= delta_c)[0]:
            out.append((i, i + 1 + int(k)))
    return out


def limiting_points(d, r1, r2):
    """Distances p1 (from c1) and p2 (from c2) of the two limiting points of
    the circles, i.e. where successive image reflections accumulate.  For
    r1 = r2 = 1, d = 2 + delta this is R_acc(delta) = 1 + delta/2 -
    sqrt(delta + delta^2/4) (Sec. 5).  Unequal radii go beyond the paper,
    which treats equal disks only: parity unpinned against it, pinned by the
    two points being mutual inverses in both circles."""
    a = d * d + r1 * r1 - r2 * r2
    p1 = (a - math.sqrt(max(a * a - 4.0 * d * d * r1 * r1, 0.0))) / (2.0 * d)
    b = d * d + r2 * r2 - r1 * r1
    p2 = (b - math.sqrt(max(b * b - 4.0 * d * d * r2 * r2, 0.0))) / (2.0 * d)
    return p1, p2


def shield_ellipse(a, rad, Rf, Nell, gamma):
    """Shielding ellipse nodes in body-local complex coordinates (Sec. 5):
    z(theta) = a/2 [1 + cos(theta + i alpha)], alpha = arccosh(1 + 2 gamma
    (rad - a)/a), theta_j = (j + 1/2) pi / N_ell, j = 0..2N_ell-1, keeping
    |z| > rad*R_f.  Foci at 0 and a, rightmost point a + gamma (rad - a)."""
    alpha = math.acosh(1.0 + 2.0 * gamma * (rad - a) / a)
    th = (np.arange(2 * Nell) + 0.5) * np.pi / Nell
    z = 0.5 * a * (1.0 + np.cos(th + 1j * alpha))
    return z[np.abs(z) > rad * Rf]


def mobius_angles(M, r):
    """Pair-adapted node angles (Sec. 5): theta_j = 2 pi j / M and
    theta~_j = pi + arg((e^{i theta} + r)/(1 + r e^{i theta})); nodes
    cluster at theta~ = pi."""
    th = 2.0 * np.pi * np.arange(M) / M
    e = np.exp(1j * th)
    return np.pi + np.angle((e + r) / (1.0 + r * e))


def fine_sets(c1, r1, c2, r2, p):
    """Fine sources and collocation nodes of a close pair (Sec. 5).

    Sources per disk: N_fp proxies on radius r*R_f (not rotated with the
    pair) plus, when the limiting point lies outside the proxy circle, the
    shielding-ellipse nodes, placed as c1 + e^{i phi} z for disk 1 and
    c2 - e^{i phi} z for disk 2 (phi = direction c1 -> c2).
    Nodes per disk: ceil(a_f N_fp) equispaced plus a_ell N_ell Moebius nodes
    whose dense end faces the partner.
    """
    c1 = np.asarray(c1, dtype=np.float64)
    c2 = np.asarray(c2, dtype=np.float64)
    dvec = c2 - c1
    d = float(np.hypot(*dvec))
    phi = math.atan2(dvec[1], dvec[0])
    rot = complex(math.cos(phi), math.sin(phi))
    Rf = p.Rf_eff
    p1, p2 = limiting_points(d, r1, r2)
    out = {}
    for tag, c, rad, a, sgn in (("1", c1, r1, p1, 1.0), ("2", c2, r2, p2, -1.0)):
        prox = ring(c, rad * Rf, p.Nfp)
        if a > rad * Rf:
            z = sgn * rot * shield_ellipse(a, rad, Rf, p.Nell, p.gamma)
            enh = np.stack([c[0] + z.real, c[1] + z.imag], axis=1)
        else:
            enh = np.zeros((0, 2))
        out["Y" + tag] = np.concatenate([prox, enh], axis=0)
        neq = int(math.ceil(p.af * p.Nfp))
        eq = ring(c, rad, neq)
        tt = mobius_angles(int(round(p.aell * p.Nell)), p.r_mob)
        ang = phi + tt - np.pi if tag == "1" else phi + tt
        mob = np.stack([c[0] + rad * np.cos(ang), c[1] + rad * np.sin(ang)], axis=1)
        out["X" + tag] = np.concatenate([eq, mob], axis=0)
        out["n_enh" + tag] = enh.shape[0]
    out["d"] = d
    out["phi"] = phi
    return out


def peanut(c1, r1, c2, r2, rho, Mp):
    """Peanut proxy surface of a pair (Sec. 3.3, Fig. peanut_fig): the curve
    traced by rolling a disk of radius rho around the pair -- the outer arcs
    of both disks joined by two concave waist arcs of radius rho.  M_p nodes
    uniform in arc length, at arc-length positions (p + 1/2) L / M_p
    measured counterclockwise from the upper tangent point on disk 1."""
    c1 = np.asarray(c1, dtype=np.float64)
    c2 = np.asarray(c2, dtype=np.float64)
    dvec = c2 - c1
    d = float(np.hypot(*dvec))
    phi = math.atan2(dvec[1], dvec[0])
    # pair frame: c1 = (0, 0), c2 = (d, 0); rolling-disk centres (wx, +-wy)
    R1, R2 = r1 + rho, r2 + rho
    wx = (d * d + R1 * R1 - R2 * R2) / (2.0 * d)
    wy = math.sqrt(R1 * R1 - wx * wx)
    th1 = math.atan2(wy, wx)              # upper tangent direction seen from c1
    th2 = math.atan2(wy, wx - d)          # upper tangent direction seen from c2
    a1 = math.atan2(wy, -wx)              # c1 seen from the lower rolling centre
    a2 = math.atan2(wy, d - wx)           # c2 seen from the lower rolling centre
    # arcs in counterclockwise order of the whole curve
    arcs = [
        ("c", (0.0, 0.0), r1, th1, 2 * np.pi - th1),       # disk 1 outer, ccw
        ("c", (wx, -wy), rho, a1, a2),                      # lower waist, cw
        ("c", (d, 0.0), r2, -th2, th2),                     # disk 2 outer, ccw
        ("c", (wx, wy), rho, -a2, -a1),                     # upper waist, cw
    ]
    lens = [rad * abs(t1 - t0) for _, _, rad, t0, t1 in arcs]
    L = sum(lens)
    s = (np.arange(Mp) + 0.5) * L / Mp
    pts = np.zeros((Mp, 2))
    start = 0.0
    for (_, cen, rad, t0, t1), ln in zip(arcs, lens):
        m = (s >= start) & (s < start + ln)
        t = t0 + (t1 - t0) * (s[m] - start) / ln
        pts[m, 0] = cen[0] + rad * np.cos(t)
        pts[m, 1] = cen[1] + rad * np.sin(t)
        start += ln
    cph, sph = math.cos(phi), math.sin(phi)
    out = np.empty_like(pts)
    out[:, 0] = c1[0] + cph * pts[:, 0] - sph * pts[:, 1]
    out[:, 1] = c1[1] + sph * pts[:, 0] + cph * pts[:, 1]
    return out
