"""Pins of the CPU oracle against facts fixed by the paper and by the
mathematics, independent of the oracle's own formulas (CPU only)."""
import math

import numpy as np
import pytest

import workloads as w
from oracle import bruteforce
from oracle.geometry import (contacts, fine_sets, limiting_points, mobius_angles, peanut,
                             radius_rule, shield_ellipse)
from oracle.kernel import stokeslet
from oracle.params import PACKING, PAIR_SMALL
from oracle.system import System


# ---------------------------------------------------------------- kernel
def test_stokeslet_symmetry_and_stokes_equations():
    """S(x,y) = S(y,x) = S(x,y)^T, and a single Stokeslet field is
    divergence-free and satisfies mu Lap u = grad p with the Stokeslet
    pressure p = (x-y).F / (2 pi |x-y|^2) (checked by finite differences)."""
    rng = np.random.default_rng(0)
    X = rng.uniform(-3, 3, (5, 2))
    Y = rng.uniform(-3, 3, (4, 2))
    S = stokeslet(X, Y)
    St = stokeslet(Y, X)
    assert np.allclose(S, St.T, atol=1e-15)
    for m in range(5):
        blk = S[2 * m:2 * m + 2, 0:2]
        assert np.allclose(blk, blk.T, atol=1e-15)
    F = np.array([0.7, -1.3])
    y0 = np.array([[0.1, -0.2]])
    u = lambda x: (stokeslet(np.atleast_2d(x), y0) @ F)
    x0 = np.array([1.3, 0.4])
    h = 1e-4
    ex, ey = np.array([h, 0]), np.array([0, h])
    div = (u(x0 + ex)[0] - u(x0 - ex)[0] + u(x0 + ey)[1] - u(x0 - ey)[1]) / (2 * h)
    assert abs(div) < 1e-8
    lap = (u(x0 + ex) + u(x0 - ex) + u(x0 + ey) + u(x0 - ey) - 4 * u(x0)) / h ** 2
    p = lambda x: (x - y0[0]) @ F / (2 * math.pi * np.sum((x - y0[0]) ** 2))
    gp = np.array([(p(x0 + ex) - p(x0 - ex)) / (2 * h), (p(x0 + ey) - p(x0 - ey)) / (2 * h)])
    assert np.allclose(lap, gp, atol=1e-5)


# ------------------------------------------------------- closed forms
@pytest.mark.parametrize("a", [1.0, 0.8, 1.2])
def test_single_disk_resistance_closed_form(a):
    """Translation: a Stokeslet F plus a potential dipole at the centre moves
    the circle rigidly with V = F (1/2 - log a) / (4 pi mu), so the force on
    the fluid is F = 4 pi mu V / (1/2 - log a) (= 8 pi mu V for the unit
    disk; singular at a = sqrt(e), Remark r:uinfty).  Rotation: a rotlet gives
    t = 4 pi mu a^2 omega and zero force."""
    s = System(np.zeros((1, 2)), np.array([a]), PACKING, "resistance")
    ft, info = s.solve(np.array([[1.0, -0.5, 0.0]]), tol=1e-13)
    F = 4 * math.pi / (0.5 - math.log(a))
    assert np.allclose(ft[0], [F, -0.5 * F, 0.0], rtol=1e-10, atol=1e-10 * F)
    ft, _ = s.solve(np.array([[0.0, 0.0, 1.0]]), tol=1e-13)
    assert np.allclose(ft[0], [0, 0, 4 * math.pi * a * a], rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("a", [1.0, 0.8, 1.2])
def test_single_disk_exterior_field_closed_form(a):
    """Off the surface, the one-body MFS field of a rigid disk is the exact
    one.  Translation with velocity V: a Stokeslet F at the centre plus the
    potential dipole D = a^2 F / (8 pi mu), which cancels the Stokeslet's
    (x.F) x / r^2 part on r = a, so u = V there with F = 4 pi mu V /
    (1/2 - log a).  Rotation with omega: the rotlet u = a^2 omega (-y, x) / r^2.
    The ring of coarse sources reproduces both at r = 1.5a .. 4a to rounding
    (its aliasing terms decay like (R_c a / r)^N_c)."""
    from oracle.onebody import OneBody
    from oracle.system import stokes_sum
    mu = PACKING.mu
    ob = OneBody(a, PACKING, "resistance")
    th = np.linspace(0.0, 2 * np.pi, 37, endpoint=False)
    V = np.array([1.0, -0.5])
    lam = ob.apply_pinv(np.tile(V, PACKING.Mc)).reshape(-1, 2)
    F = lam.sum(0)
    assert np.allclose(F, 4 * np.pi * mu * V / (0.5 - math.log(a)), rtol=1e-12)
    for rr in (1.5, 2.0, 4.0):
        X = np.stack([rr * a * np.cos(th), rr * a * np.sin(th)], 1)
        r2 = (X ** 2).sum(1)[:, None]
        xF = (X @ F)[:, None]
        exact = (-0.5 * np.log(r2) * F + xF * X / r2) / (4 * np.pi * mu) \
            + a * a / (8 * np.pi * mu) * (F / r2 - 2 * xF * X / r2 ** 2)
        u = stokes_sum(X, ob.Y, lam, mu)
        assert np.abs(u - exact).max() < 1e-12 * np.abs(exact).max(), rr
    w_ = 1.0
    lam = ob.apply_pinv(np.stack([-w_ * ob.X[:, 1], w_ * ob.X[:, 0]], 1).ravel()).reshape(-1, 2)
    for rr in (1.5, 3.0):
        X = np.stack([rr * a * np.cos(th), rr * a * np.sin(th)], 1)
        exact = (a * a * w_ / (X ** 2).sum(1))[:, None] * np.stack([-X[:, 1], X[:, 0]], 1)
        u = stokes_sum(X, ob.Y, lam, mu)
        assert np.abs(u - exact).max() < 1e-12 * np.abs(exact).max(), rr


@pytest.mark.parametrize("a", [1.0, 0.9])
def test_single_disk_mobility_closed_form(a):
    """Inverse of the above: v = f (1/2 - log a)/(4 pi mu), omega = t/(4 pi mu a^2)."""
    s = System(np.zeros((1, 2)), np.array([a]), PACKING, "mobility")
    v, _ = s.solve(np.array([[0.3, 1.1, -2.0]]), tol=1e-13)
    m = (0.5 - math.log(a)) / (4 * math.pi)
    assert np.allclose(v[0], [0.3 * m, 1.1 * m, -2.0 / (4 * math.pi * a * a)], rtol=1e-10, atol=1e-12)


# ------------------------------------------------------- algebra of Alg. 3
@pytest.mark.parametrize("problem", ["resistance", "mobility"])
def test_isolated_pair_matvec_is_identity(problem):
    """For P = 2 the Step 2b subtraction cancels every pair-internal term:
    the two-body system matrix of an isolated pair is exactly I (Sec. 3.5,
    'approximately the identity', exact in Algorithm 3's algebra)."""
    pk = w.two_disks(1e-2)
    s = System(pk.centres, pk.radii, PACKING, problem)
    assert len(s.pairs) == 1
    mu = w.smooth_surface_vector(2, PACKING.Mc, 7).reshape(2, -1)
    u = s.matvec(mu)
    # rounding of the large cancelling terms in the literal form
    assert np.max(np.abs(u - mu)) < 1e-9 * np.max(np.abs(mu))


def test_no_contacts_reduces_to_one_body_system():
    """Without close pairs Algorithm 3 is the one-body preconditioned system,
    eq. (resistance): identity diagonal blocks and S^(ik) P^+ off-diagonal."""
    c = np.array([[0.0, 0.0], [2.6, 0.4], [-0.3, 2.7]])
    s = System(c, np.ones(3), PACKING, "resistance")
    assert s.pairs == []
    mu = w.smooth_surface_vector(3, PACKING.Mc, 3).reshape(3, -1)
    u = s.matvec(mu)
    ob = s.ob[0]
    pinv = ob.pinv.VSi @ ob.pinv.Ut
    for i in range(3):
        ref = mu[i].copy()
        for k in range(3):
            if k != i:
                ref = ref + stokeslet(s.X[i], s.Y[k]) @ (pinv @ mu[k])
        assert np.allclose(u[i], ref, atol=1e-11)


def test_gmres_matches_dense_solve():
    """GMRES on Algorithm 3 agrees with a dense direct solve of the same
    square 2 M_c P system (matrix assembled column by column)."""
    c = np.array([[0.0, 0.0], [2.02, 0.0], [4.3, 0.5], [1.0, 2.3]])
    p = PACKING.with_(Nc=32, Mc=40, Rc=0.6, Nfp=60, Nell=20, Mp=80)
    s = System(c, np.ones(4), p, "mobility")
    n = 4 * 2 * p.Mc
    A = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = s.matvec(e.reshape(4, -1)).ravel()
    b = s.rhs_mobility(w.forces_torques(4, 9)).ravel()
    x_dense = np.linalg.solve(A, b)
    _, info = s.solve(w.forces_torques(4, 9), tol=1e-13)
    # unit-vector columns are non-smooth inputs: the literal form's cancelling
    # terms leave ~1e-7 rounding in the assembled matrix
    assert np.linalg.norm(info["mu"].ravel() - x_dense) < 1e-5 * np.linalg.norm(x_dense)


# ------------------------------------------------------- physics
def test_two_disk_resistance_matrix_symmetric_positive_definite():
    """Lorentz reciprocity: the 6x6 resistance matrix of two close disks is
    symmetric; it is positive definite once the pair is small enough that the
    w = 0 problem of Remark r:uinfty is not near its singular scale (radius
    0.3, gap 3e-4).  Mirror symmetry about the line of centres zeros the
    coupling between motion along the line and the other modes."""
    a = 0.3
    c = a * np.array([[0.0, 0.0], [2.001, 0.0]])
    s = System(c, a * np.ones(2), PACKING, "resistance")
    R = np.zeros((6, 6))
    for j in range(6):
        e = np.zeros(6)
        e[j] = 1.0
        R[:, j] = s.solve(e.reshape(2, 3), tol=1e-12)[0].ravel()
    assert np.linalg.norm(R - R.T) < 1e-8 * np.linalg.norm(R)
    assert np.linalg.eigvalsh(0.5 * (R + R.T)).min() > 0
    along, other = [0, 3], [1, 2, 4, 5]
    assert np.max(np.abs(R[np.ix_(along, other)])) < 1e-8 * np.abs(R).max()
    # lubrication: squeeze resistance far above the isolated-disk value
    assert R[0, 0] > 100 * 4 * math.pi / (0.5 - math.log(a))


def test_squeeze_resistance_grows_as_gap_shrinks():
    fx = []
    for gap in (1e-1, 1e-2, 1e-3):
        pk = w.two_disks(gap)
        s = System(pk.centres, pk.radii, PACKING, "resistance")
        fx.append(s.solve(np.array([[1.0, 0, 0], [-1.0, 0, 0]]), tol=1e-12)[0][0, 0])
    assert fx[0] < fx[1] < fx[2]
    # 2D squeeze flow between cylinders: force ~ delta^(-3/2)
    slope = math.log(fx[2] / fx[1]) / math.log(10)
    assert 1.3 < slope < 1.7


def test_zero_net_force_under_pure_rotation():
    s = System(np.zeros((1, 2)), np.ones(1), PACKING, "resistance")
    ft, _ = s.solve(np.array([[0.0, 0.0, 2.5]]), tol=1e-13)
    assert np.all(np.abs(ft[0, :2]) < 1e-11)


@pytest.mark.parametrize("gap,tol", [(1e-1, 1e-8), (1e-2, 1e-4)])
def test_two_way_consistency(gap, tol):
    """Mobility output fed to the resistance solve returns the input forces
    (Sec. 6.1, 'two-way error'), to a level set by the boundary residual."""
    pk = w.two_disks(gap)
    ft = np.array([[1.0, 0.3, 0.2], [-1.0, -0.3, -0.5]])
    v, _ = System(pk.centres, pk.radii, PACKING, "mobility").solve(ft, tol=1e-12)
    ft2, _ = System(pk.centres, pk.radii, PACKING, "resistance").solve(v, tol=1e-12)
    assert np.max(np.abs(ft2 - ft)) < tol


def test_isolated_pair_equals_fine_brute_force():
    """For an isolated pair the two-body scheme is the pair's fine MFS: its
    forces match a dense global fine solve (no compression, no
    preconditioning), which pins Z, E and the force extraction."""
    pk = w.two_disks(1e-2)
    vel = np.array([[1.0, 0.3, 0.2], [-0.5, -0.3, 0.4]])
    p = PACKING.with_(Nfp=100)
    fb = bruteforce.solve(pk.centres, pk.radii, p, "resistance", vel)
    ft, _ = System(pk.centres, pk.radii, p, "resistance").solve(vel, tol=1e-13)
    assert np.linalg.norm(ft - fb) < 1e-8 * np.linalg.norm(fb)



@pytest.mark.parametrize("problem", ["resistance", "mobility"])
@pytest.mark.parametrize("gap", [1e-1, 1e-2, 1e-3])
def test_unequal_pair_against_fine_brute_force(problem, gap):
    """Disks of radii 0.8 and 1.2 (the unequal-radius extension: limiting
    points of unequal circles, rolling radius 0.8): the two-body solution
    matches the dense fine MFS of the pair within the 1e-5 solve target
    (measured 4e-10 to 1e-5; equal radii give 3e-11 to 4e-6)."""
    c = np.array([[0.0, 0.0], [0.8 + 1.2 + gap, 0.0]])
    r = np.array([0.8, 1.2])
    data = (np.array([[1.0, 0.3, 0.2], [-0.5, -0.3, 0.4]]) if problem == "resistance"
            else np.array([[1.0, 0.3, 0.2], [-1.0, -0.3, -0.5]]))
    p = PACKING.with_(Nfp=100)
    fb = bruteforce.solve(c, r, p, problem, data)
    out, _ = System(c, r, p, problem).solve(data, tol=1e-13)
    assert np.linalg.norm(out - fb) < 3e-5 * np.linalg.norm(fb)


@pytest.mark.slow
@pytest.mark.parametrize("problem,geom,tol", [
    ("resistance", "chain", 5e-6), ("mobility", "chain", 5e-6), ("mobility", "triangle", 5e-4)])
def test_three_disks_against_fine_brute_force(problem, geom, tol):
    """Three disks with two or three close contacts: the pairwise-corrected,
    peanut-compressed solution approaches the dense fine MFS.  (A closed
    triangle under resistance traps a fluid pocket -- a three-body effect
    that pair corrections do not carry, cf. Remark 'Clustering' -- so it is
    not used.)"""
    geoms = {"chain": np.array([[0, 0], [2.01, 0], [4.02, 0.3]]),
             "triangle": np.array([[0, 0], [2.01, 0], [1.005, 2.01 * np.sqrt(3) / 2]])}
    c = geoms[geom]
    data = np.array([[1.0, 0.3, 0.2], [-0.5, -0.3, 0.4], [-0.5, 0.0, -0.1]])
    fb = bruteforce.solve(c, np.ones(3), PACKING, problem, data)
    out, _ = System(c, np.ones(3), PACKING, problem).solve(data, tol=1e-12)
    assert np.linalg.norm(out - fb) < tol * np.linalg.norm(fb)


# ------------------------------------------------------- geometry
def test_accumulation_radius_and_limiting_points():
    """R_acc(delta) = 1 + delta/2 - sqrt(delta + delta^2/4) (Sec. 5) is the
    limiting point of two unit circles: the point inverse to itself under
    reflection in both circles (image accumulation)."""
    for delta in (1e-3, 1e-2, 0.1):
        p1, p2 = limiting_points(2 + delta, 1.0, 1.0)
        racc = 1 + delta / 2 - math.sqrt(delta + delta ** 2 / 4)
        assert abs(p1 - racc) < 1e-14 and abs(p2 - racc) < 1e-14
    d, r1, r2 = 2.05, 0.8, 1.2
    p1, p2 = limiting_points(d, r1, r2)
    # mutual inverses in circle 1 (centre 0) and circle 2 (centre d)
    assert abs((d - p2) * p1 - r1 ** 2) < 1e-12
    assert abs((d - p1) * p2 - r2 ** 2) < 1e-12


def test_shield_ellipse_foci_and_tip():
    """Ellipse with foci 0 and a, rightmost point a + gamma (1 - a); nodes kept
    only outside the proxy circle."""
    a, Rf, gamma = 0.969, 0.9309, 0.3
    alpha = math.acosh(1 + 2 * gamma * (1 - a) / a)
    z_all = 0.5 * a * (1 + np.cos(np.linspace(0, 2 * np.pi, 50) + 1j * alpha))
    s = np.abs(z_all) + np.abs(z_all - a)
    assert np.allclose(s, s[0], atol=1e-12)
    assert abs(0.5 * a * (1 + math.cosh(alpha)) - (a + gamma * (1 - a))) < 1e-14
    z = shield_ellipse(a, 1.0, Rf, 80, gamma)
    assert len(z) > 0 and np.all(np.abs(z) > Rf)



@pytest.mark.parametrize("r1,r2", [(0.8, 1.2), (1.2, 0.8)])
def test_shield_ellipse_for_unequal_radii(r1, r2):
    """For a disk of radius r1 facing a disk of radius r2 at gap 1e-3, the
    shielding nodes lie on one ellipse whose foci are the disk centre and the
    limiting point a (constant sum of focal distances), stay outside r1 R_f,
    and reach no further than a + gamma (r1 - a) toward the partner (Sec. 5,
    with r1 for the unit radius)."""
    d = r1 + r2 + 1e-3
    a, _ = limiting_points(d, r1, r2)
    Rf, gamma = 0.9309, 0.3
    z = shield_ellipse(a, r1, Rf, 80, gamma)
    assert len(z) > 0 and np.all(np.abs(z) > r1 * Rf)
    s = np.abs(z) + np.abs(z - a)
    assert np.allclose(s, s[0], rtol=1e-12)
    tip = a + gamma * (r1 - a)
    assert np.all(z.real <= tip + 1e-12) and z.real.max() > tip - 1e-3
    assert 0 < a < r1


def test_fine_sets_counts_and_orientation():
    p = PAIR_SMALL
    pk = w.two_disks(1e-3)
    fs = fine_sets(pk.centres[0], 1.0, pk.centres[1], 1.0, p)
    assert fs["n_enh1"] == fs["n_enh2"] > 0
    assert fs["Y1"].shape[0] == p.Nfp + fs["n_enh1"]
    assert fs["X1"].shape[0] == math.ceil(p.af * p.Nfp) + int(p.aell * p.Nell)
    # enhancing sources lie between the centre and the partner
    enh = fs["Y1"][p.Nfp:]
    assert np.all(enh[:, 0] > 0)
    # proxies on radius R_f, not rotated
    assert np.allclose(np.hypot(*fs["Y1"][:p.Nfp].T), radius_rule(p.Nfp))
    assert np.allclose(fs["Y1"][0], [radius_rule(p.Nfp), 0.0])
    # Moebius nodes cluster toward the partner
    mob = fs["X1"][math.ceil(p.af * p.Nfp):]
    assert np.sum(mob[:, 0] > 0.9) > 4 * np.sum(mob[:, 0] < -0.9)
    # a wide gap keeps no ellipse sources (R_acc <= R_f)
    fs2 = fine_sets([0, 0], 1.0, [2.15, 0], 1.0, PACKING)
    assert fs2["n_enh1"] == 0


def test_mobius_map_fixed_points():
    t = mobius_angles(8, 0.6)
    assert abs(t[0] - math.pi) < 1e-15           # theta = 0 -> pi
    assert abs((t[4] % (2 * math.pi))) < 1e-12   # theta = pi -> 2 pi = 0


def test_peanut_is_the_rolling_disk_envelope():
    """Every peanut node lies on one of the four arcs, outside both disks, and
    a disk of radius rho placed against the curve at that node touches but
    does not overlap the pair; nodes are uniform in arc length and the
    length is 6 pi - 8 atan2(h, d/2) for unit disks and rho = 1."""
    for gap in (1e-3, 0.15):
        d = 2 + gap
        c1, c2 = np.array([0.3, -0.2]), np.array([0.3, -0.2]) + d * np.array([math.cos(0.7), math.sin(0.7)])
        z = peanut(c1, 1.0, c2, 1.0, 1.0, 400)
        d1 = np.hypot(*(z - c1).T)
        d2 = np.hypot(*(z - c2).T)
        assert np.all(d1 >= 1 - 1e-12) and np.all(d2 >= 1 - 1e-12)
        on_disk = (np.abs(d1 - 1) < 1e-12) | (np.abs(d2 - 1) < 1e-12)
        # waist nodes: distance exactly 1 from a rolling centre at distance 2 from both
        h = math.sqrt(4 - (d / 2) ** 2)
        mid = 0.5 * (c1 + c2)
        n = np.array([-(c2 - c1)[1], (c2 - c1)[0]]) / d
        wu, wd = mid + h * n, mid - h * n
        on_waist = (np.abs(np.hypot(*(z - wu).T) - 1) < 1e-12) | (np.abs(np.hypot(*(z - wd).T) - 1) < 1e-12)
        assert np.all(on_disk | on_waist)
        seg = np.hypot(*(np.roll(z, -1, axis=0) - z).T)
        L = 6 * math.pi - 8 * math.atan2(h, d / 2)
        assert abs(seg.sum() - L) < 1e-3
        assert np.std(seg) < 1e-3 * seg.mean()



@pytest.mark.parametrize("r1,r2", [(0.8, 1.2), (1.2, 0.9), (1.0, 1.0)])
def test_peanut_envelope_for_unequal_radii(r1, r2):
    """The peanut of two disks of different radii with rolling radius rho =
    min(r1, r2) (reading of Sec. 3.3 for unequal disks): the rolling disk
    touches both disks at the two points W with |W - c_i| = r_i + rho (found
    here as circle intersections).  Every node lies outside both disks and
    outside both rolling disks, on a disk circle or on a rolling circle; the
    nodes are uniform along one closed curve."""
    for gap in (1e-3, 0.1):
        rho = min(r1, r2)
        c1 = np.array([0.4, -0.1])
        d = r1 + r2 + gap
        u = np.array([math.cos(-1.1), math.sin(-1.1)])
        c2 = c1 + d * u
        z = peanut(c1, r1, c2, r2, rho, 600)
        # rolling centres: intersections of |W - c1| = r1 + rho and |W - c2| = r2 + rho
        R1, R2 = r1 + rho, r2 + rho
        a = (R1 ** 2 - R2 ** 2 + d ** 2) / (2 * d)
        hh = math.sqrt(R1 ** 2 - a ** 2)
        nrm = np.array([-u[1], u[0]])
        W = [c1 + a * u + hh * nrm, c1 + a * u - hh * nrm]
        for Wk in W:
            assert abs(np.hypot(*(Wk - c1)) - R1) < 1e-12 and abs(np.hypot(*(Wk - c2)) - R2) < 1e-12
        d1 = np.hypot(*(z - c1).T)
        d2 = np.hypot(*(z - c2).T)
        dw = [np.hypot(*(z - Wk).T) for Wk in W]
        tol = 1e-12
        assert np.all(d1 >= r1 - tol) and np.all(d2 >= r2 - tol)
        assert np.all(dw[0] >= rho - tol) and np.all(dw[1] >= rho - tol)
        on = (np.abs(d1 - r1) < tol) | (np.abs(d2 - r2) < tol) | (np.abs(dw[0] - rho) < tol) | \
             (np.abs(dw[1] - rho) < tol)
        assert np.all(on)
        # both disks and both waists are represented
        assert np.any(np.abs(d1 - r1) < tol) and np.any(np.abs(d2 - r2) < tol)
        assert np.any(np.abs(dw[0] - rho) < tol) and np.any(np.abs(dw[1] - rho) < tol)
        seg = np.hypot(*(np.roll(z, -1, axis=0) - z).T)
        assert np.std(seg) < 1e-3 * seg.mean()


def test_params_reject_nonpositive_source_radius():
    with pytest.raises(ValueError):
        PACKING.with_(Nc=24)


def test_contacts_brute_force():
    pk = w.packing_p100()
    cs = contacts(pk.centres, pk.radii, 0.2)
    ref = set()
    for i in range(pk.P):
        for k in range(i + 1, pk.P):
            if np.hypot(*(pk.centres[i] - pk.centres[k])) - 2 <= 0.2:
                ref.add((i, k))
    assert set(cs) == ref and len(cs) > 10


def test_squeeze_force_matches_reynolds_lubrication():
    """Two unit disks approaching each other at relative speed V across a gap
    delta: the lubrication (Reynolds) asymptote of the force is
    F = (3 pi / 2) mu V (a / delta)^(3/2), derived from the thin-film flux
    balance for two cylinders, independent of the paper.  The oracle's force
    at delta = 1e-3 lies within 0.5 % of it (the correction is O(delta))."""
    c = np.array([[0.0, 0.0], [2.0 + 1e-3, 0.0]])
    s = System(c, np.ones(2), PAIR_SMALL, "resistance")
    f, _ = s.solve(np.array([[1.0, 0, 0], [-1.0, 0, 0]]))
    lead = 1.5 * math.pi * 1.0 * 2.0 * (1.0 / 1e-3) ** 1.5
    assert f[0][0] == pytest.approx(lead, rel=5e-3)
    assert f[1][0] == pytest.approx(-f[0][0], rel=1e-10)


def test_matvec_on_sampled_targets_equals_full_rows():
    """The oracle's matvec evaluated on a subset of target disks (as the
    full-size P = 10^4 check uses it) equals those rows of the full matvec:
    Step 2a over every source, the Step 2b terms of pairs that touch a sampled
    disk, and the identity step, with the dense far field (to rounding) and
    with the chunked direct sum."""
    p = PAIR_SMALL
    c = np.array([[0.0, 0.0], [2.05, 0.0], [4.2, 0.3], [0.5, 2.3], [2.7, 2.2]])
    r = np.ones(5)
    mu = w.smooth_surface_vector(5, p.Mc, 3).reshape(5, -1)
    dense = System(c, r, p, "mobility")
    assert len(dense.pairs) >= 2
    chunked = System(c, r, p, "mobility", blocks=dense.blocks, dense_limit=0)
    full = dense.matvec(mu)
    for targets in ([1], [0, 3], [2, 4, 1]):
        t = np.sort(np.asarray(targets))
        np.testing.assert_allclose(dense.matvec(mu, t), full[t], rtol=0, atol=1e-12 * np.abs(full).max())
        # the chunked sum adds the same terms in another order; with the real
        # pair blocks the literal form cancels strengths ~1e6 |mu|, so the
        # two orders differ at ~1e-16 x 1e6 of the field
        np.testing.assert_allclose(chunked.matvec(mu, t), full[t], rtol=0, atol=1e-9 * np.abs(full).max())


@pytest.mark.parametrize("problem", ["resistance", "mobility"])
@pytest.mark.parametrize("gap", [1e-1, 1e-2, 1e-3])
def test_pair_solves_have_small_residuals(problem, gap):
    """The two least-squares problems of a close pair are solved, at the
    paper's parameters: the fine local solve F Z = blkQ (eq. (bfm)) and the
    peanut compression C A = -D Z (eq. (Amat)) leave relative residuals at the
    discretisation level (measured 1e-12..2e-5 and 1e-8..2e-7 here), while a
    sign, index or transposition error in Z, D or A leaves O(1)."""
    from oracle.onebody import OneBody
    from oracle.pairs import pair_blocks
    ob = OneBody(1.0, PACKING, problem)
    out = pair_blocks(np.array([0.0, 0.0]), 1.0, np.array([2.0 + gap, 0.0]), 1.0, ob, ob, PACKING, problem, 1.0)
    assert out["fine_residual"] < 1e-4
    assert out["peanut_residual"] < 1e-4


@pytest.mark.parametrize("problem", ["resistance", "mobility"])
def test_exclusion_form_equals_literal_algorithm3(problem):
    """Algorithm 3 adds every source in Step 2a and then, in Step 2b and the
    identity step, takes out the self terms and the pair-internal terms.  The
    same vector is reached without any cancellation: u^(i) = mu^(i) plus the
    fields of the disks that are not close to i with their full strengths,
    plus, for each close partner k, the field of k's corrections from its
    other pairs only (its own lam_bar and the (i, k) correction are already
    inside the two-body solve).  This exclusion form is the one the device
    matvec evaluates; written out here directly from the definitions, it
    agrees with the literal form to rounding, so a sign, index or swapped
    operand in the oracle's Step 2b (or in the exclusion bookkeeping) fails."""
    p = PAIR_SMALL
    c = np.array([[0.0, 0.0], [2.05, 0.0], [4.2, 0.3], [0.5, 2.3], [2.7, 2.2]])
    s = System(c, np.ones(5), p, problem)
    P, n = s.P, 2 * p.Nc
    assert len(s.pairs) >= 2
    mu = w.smooth_surface_vector(P, p.Mc, 3).reshape(P, -1)
    lb = s.lam_bar(mu)
    lam = lb.copy()
    corr = {}                      # corr[(a, b)]: correction that pair (a, b) adds to disk a
    for (i, k), blk in zip(s.pairs, s.blocks):
        t = blk["A"] @ np.concatenate([lb[i], lb[k]])
        lam[i] += t[:n]
        lam[k] += t[n:]
        corr[(i, k)], corr[(k, i)] = t[:n], t[n:]
    sig = [s.proj(i, lam[i]) for i in range(P)]
    u = np.empty_like(mu)
    for i in range(P):
        acc = mu[i].copy()
        for k in range(P):
            if k == i:
                continue
            if (k, i) in corr:
                own = sum((v for (a, b), v in corr.items() if a == k and b != i), np.zeros(n))
                acc += stokeslet(s.X[i], s.Y[k], p.mu) @ s.proj(k, own)
            else:
                acc += stokeslet(s.X[i], s.Y[k], p.mu) @ sig[k]
        u[i] = acc
    lit = s.matvec(mu)
    # the literal form cancels strengths up to ~1e4 |mu|: rounding ~1e-16 x 1e4
    assert np.linalg.norm(u - lit) < 1e-11 * np.linalg.norm(lit)
    # the oracle's own exclusion-form evaluation (the reference for the device
    # matvec) is the same vector, in FP64 and in extended precision, on all
    # disks and on a subset of target disks
    for dt in (np.float64, np.longdouble):
        ex = s.matvec_exclusion(mu, dtype=dt)
        assert np.linalg.norm(ex - lit) < 1e-11 * np.linalg.norm(lit)
        assert np.linalg.norm(ex - u) < 1e-13 * np.linalg.norm(u)
    sub = s.matvec_exclusion(mu, targets=[1, 3], dtype=np.longdouble)
    assert np.linalg.norm(sub - u[[1, 3]]) < 1e-13 * np.linalg.norm(u[[1, 3]])
    assert 1.0 <= s.exclusion_condition(mu) < 1e6


def test_extended_precision_stokeslet_sum_against_mpmath():
    """The extended-precision reference evaluates cancelling sums that FP64
    cannot: a ring of 60 Stokeslets whose strengths are one high Fourier mode
    (m = 25) of amplitude 1e8 has a field that decays like (rho/|z|)^25 away
    from the ring, so the direct sum cancels ~15 digits.  Against a 50-digit
    mpmath evaluation of the same sum, np.longdouble reaches its own
    eps x condition number while FP64 misses by orders of magnitude more."""
    mpmath = pytest.importorskip("mpmath")
    from oracle.kernel import stokeslet_in
    mpmath.mp.dps = 50
    N, m, rho, amp = 60, 25, 0.54, 1e8
    th = 2 * np.pi * np.arange(N) / N
    Y = np.stack([rho * np.cos(th), rho * np.sin(th)], -1)
    s = np.stack([amp * np.cos(m * th), amp * np.sin(m * th)], -1).ravel()
    X = np.array([[1.05, 0.3], [-0.7, 0.9]])
    ref = []
    for x in X:
        ux = uy = mpmath.mpf(0)
        for j in range(N):
            dx = mpmath.mpf(x[0]) - mpmath.mpf(Y[j, 0])
            dy = mpmath.mpf(x[1]) - mpmath.mpf(Y[j, 1])
            r2 = dx * dx + dy * dy
            lg = mpmath.log(r2) / 2
            sx, sy = mpmath.mpf(s[2 * j]), mpmath.mpf(s[2 * j + 1])
            dot = (dx * sx + dy * sy) / r2
            ux += -lg * sx + dot * dx
            uy += -lg * sy + dot * dy
        c = 1 / (4 * mpmath.pi)
        ref += [float(c * ux), float(c * uy)]
    ref = np.array(ref)
    scale = np.abs(stokeslet(X, Y)) @ np.abs(s)
    cond = np.linalg.norm(scale) / np.linalg.norm(ref)
    assert cond > 1e6                            # a badly conditioned sum
    e64 = np.linalg.norm(stokeslet(X, Y) @ s - ref) / np.linalg.norm(ref)
    ext = (stokeslet_in(X, Y, 1.0, np.longdouble) @ s.astype(np.longdouble)).astype(np.float64)
    eext = np.linalg.norm(ext - ref) / np.linalg.norm(ref)
    epsx = float(np.finfo(np.longdouble).eps)
    assert eext < max(100 * epsx * cond, 1e-15)
    assert e64 > 10 * eext


@pytest.mark.parametrize("case", ["pair_1e-2", "pair_1e-3", "chain_resistance", "chain_mobility"])
def test_fine_brute_force_converges_under_refinement(case):
    """The dense fine MFS that the compressed scheme is pinned to converges as
    its near-contact resolution is refined: N_ell (shielding-ellipse sources
    and 5 N_ell Moebius nodes per contact, Sec. 5) from coarse to twice the
    paper's 80.  The distance to the finest level falls steadily to the
    truncation floor, and the paper's N_ell = 80 is already within 1e-6 of it
    at gap 1e-3.  Nodes whose dense end faced away from the partner would
    stall near 4e-2."""
    vel2 = np.array([[1.0, 0.3, 0.2], [-0.5, -0.3, 0.4]])
    vel3 = np.array([[1.0, 0.3, 0.2], [-0.5, -0.3, 0.4], [-0.5, 0.0, -0.1]])
    chain = np.array([[0.0, 0.0], [2.01, 0.0], [4.02, 0.3]])
    setups = {
        "pair_1e-2": (w.two_disks(1e-2).centres, "resistance", vel2, (10, 20, 30, 40, 60, 80)),
        "pair_1e-3": (w.two_disks(1e-3).centres, "resistance", vel2, (40, 60, 80, 100, 160)),
        "chain_resistance": (chain, "resistance", vel3, (10, 20, 30, 40, 60, 80)),
        "chain_mobility": (chain, "mobility", vel3, (10, 20, 30, 40, 60, 80)),
    }
    c, problem, data, levels = setups[case]
    r = np.ones(len(c))
    out = {n: bruteforce.solve(c, r, PACKING.with_(Nell=n, Nfp=100), problem, data) for n in levels}
    ref = out[levels[-1]]
    err = [np.linalg.norm(out[n] - ref) / np.linalg.norm(ref) for n in levels[:-1]]
    floor = 1e-9
    for a, b in zip(err, err[1:]):
        assert b < a or b < floor, err               # steady until the truncation floor
    assert err[-1] < floor, err                      # the last two levels agree
    assert err[0] > 1e3 * err[-1], err               # and the coarsest level is far from them
    if case == "pair_1e-3":
        assert err[levels.index(80)] < 1e-6, err


# ------------------------------------------------- flow evaluation (flowEval)
@pytest.mark.parametrize("problem", ["resistance", "mobility"])
def test_boundary_flow_single_disk_is_rigid(problem):
    """A single disk: the one-body MFS reproduces the exact rigid-body flow,
    so the pointwise residual (eq. (residual_x)) at new boundary nodes is at
    rounding level."""
    from oracle import flow
    s = System(np.zeros((1, 2)), np.array([1.0]), PACKING, problem, keep_fine=True)
    data = np.array([[1.0, -0.5, 0.3]])
    _, info = s.solve(data, tol=1e-13)
    _, rel = flow.boundary_residual(s, info["mu"], data, 100)
    assert rel < 1e-12


@pytest.mark.slow
@pytest.mark.parametrize("problem,gap", [("resistance", 1e-1), ("resistance", 1e-3), ("mobility", 1e-2),
                                         ("mobility", 1e-3)])
def test_boundary_flow_of_a_pair_matches_fine_brute_force(problem, gap):
    """Two unit disks at the paper's parameters: the two-body flow at 100 new
    nodes per boundary (one-body fields, the other pairs' compressed
    corrections, the pair's own fine sources beta = -Z lam_bar) equals the
    flow of the dense fine MFS of the same pair (no compression, no
    preconditioner) to 5e-6, and its relative boundary residual (eq.
    (residual)) is within 5 times the brute force's own (plus 1e-8): the
    peanut compression and the one-body stand-in of Step 2b add their own error.  Leaving
    out the fine sources, or taking them with the wrong sign, breaks both."""
    from oracle import bruteforce, flow
    pk = w.two_disks(gap)
    s = System(pk.centres, pk.radii, PACKING, problem, keep_fine=True)
    data = np.array([[1.0, 0.3, 0.2], [-0.5, -0.3, 0.4]])
    _, info = s.solve(data, tol=1e-13)
    u, g = flow.boundary_flow(s, info["mu"], data, 100)
    X = np.concatenate([flow.eval_nodes(pk.centres[i], 1.0, 100) for i in range(2)])
    _, ubf = bruteforce.solve(pk.centres, pk.radii, PACKING, problem, data, points=X)
    err = np.linalg.norm(u.reshape(-1, 2) - ubf) / np.linalg.norm(ubf)
    assert err < 5e-6
    _, rel = flow.boundary_residual(s, info["mu"], data, 100)
    gv = g.reshape(-1, 2)
    rel_bf = np.hypot(*(ubf - gv).T).max() / np.hypot(*gv.T).max()
    assert rel <= 5 * rel_bf + 1e-8
    # planted: the pair's fine sources with the wrong sign
    for b in s.blocks:
        b["Z"] = -b["Z"]
    u2, _ = flow.boundary_flow(s, info["mu"], data, 100)
    assert np.linalg.norm(u2.reshape(-1, 2) - ubf) / np.linalg.norm(ubf) > 1e-2
