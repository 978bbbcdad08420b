"""Seeded synthetic workloads: disk packings and rigid-body inputs.

This module is the one piece shared by the CPU oracle and the GPU path. It
holds geometry generation and random draws only -- none of the MFS method's
arithmetic (no Stokeslets, no contact lists, no least squares).

Packings follow the generator of Sec. 6.2 (square lattice, then Metropolis
accept/reject sweeps that keep every disk inside the box and every gap at or
above a prescribed minimum), with two other starts: a hexagonal lattice for
polydisperse packings whose largest disks do not fit a square lattice at the
target area fraction, and random sequential placement for the P=100
workload.  Every draw uses numpy's PCG64 with a fixed seed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Packing:
    centres: np.ndarray          # (P, 2) float64
    radii: np.ndarray            # (P,) float64
    box: tuple                   # (Lx, Ly) of the rectangular domain
    meta: dict = field(default_factory=dict)

    @property
    def P(self) -> int:
        return int(self.centres.shape[0])


class _Grid:
    """Uniform cell list over the box [0, Lx) x [0, Ly) for gap queries."""

    def __init__(self, centres, Lx, Ly, cell):
        self.nx = max(1, int(math.floor(Lx / cell)))
        self.ny = max(1, int(math.floor(Ly / cell)))
        self.cx = Lx / self.nx
        self.cy = Ly / self.ny
        self.cells: dict[tuple[int, int], list[int]] = {}
        self.key: dict[int, tuple[int, int]] = {}
        for i, c in enumerate(centres):
            self.add(i, c)

    def _k(self, c):
        return (min(self.nx - 1, max(0, int(c[0] / self.cx))),
                min(self.ny - 1, max(0, int(c[1] / self.cy))))

    def add(self, i, c):
        k = self._k(c)
        self.cells.setdefault(k, []).append(i)
        self.key[i] = k

    def move(self, i, c):
        k = self._k(c)
        if k != self.key[i]:
            self.cells[self.key[i]].remove(i)
            self.cells.setdefault(k, []).append(i)
            self.key[i] = k

    def near(self, c):
        kx, ky = self._k(c)
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                lst = self.cells.get((kx + dx, ky + dy))
                if lst:
                    yield from lst


def _admissible(i, c, centres, radii, Lx, Ly, gmin, grid, skip=()):
    r = radii[i]
    if c[0] - r < 0 or c[1] - r < 0 or c[0] + r > Lx or c[1] + r > Ly:
        return False
    for k in grid.near(c):
        if k == i or k in skip:
            continue
        d = math.hypot(c[0] - centres[k, 0], c[1] - centres[k, 1])
        if d - r - radii[k] < gmin:
            return False
    return True


def _sweeps(centres, radii, Lx, Ly, gmin, rng, nsweep, step):
    """Metropolis sweeps: visit disks in order, propose a uniform random
    displacement, accept only if the disk stays in the box and keeps every
    gap >= gmin (Sec. 6.2)."""
    P = len(radii)
    grid = _Grid(centres, Lx, Ly, 2.0 * radii.max() + max(gmin, 0.25) + 1e-9)
    accepted = 0
    for _ in range(nsweep):
        disp = rng.uniform(-step, step, size=(P, 2))
        for i in range(P):
            c = centres[i] + disp[i]
            if _admissible(i, c, centres, radii, Lx, Ly, gmin, grid):
                centres[i] = c
                grid.move(i, c)
                accepted += 1
    return accepted / max(1, nsweep * P)


def _min_gap_pairs(centres, radii, cutoff):
    """All pairs with gap < cutoff, via sorting on x (geometry helper only)."""
    order = np.argsort(centres[:, 0])
    xs = centres[order, 0]
    rmax = radii.max()
    out = []
    for a in range(len(order)):
        i = order[a]
        b = a + 1
        while b < len(order) and xs[b] - xs[a] <= 2 * rmax + cutoff:
            k = order[b]
            g = math.hypot(*(centres[i] - centres[k])) - radii[i] - radii[k]
            if g < cutoff:
                out.append((min(i, k), max(i, k), g))
            b += 1
    return out


def _lattice(P, area, phi, hexagonal, rng):
    """P sites of a square or hexagonal lattice whose box gives area fraction
    phi; returns (sites, Lx, Ly)."""
    if hexagonal:
        ncol = max(1, int(round(math.sqrt(P * math.sqrt(3) / 2))))
        nrow = int(math.ceil(P / ncol))
        # spacing s with area / (ncol*s * nrow*s*sqrt(3)/2) = phi
        s = math.sqrt(area / (phi * ncol * nrow * math.sqrt(3) / 2))
        sites = np.array([((a + 0.5 + 0.5 * (b % 2) - 0.25) * s, (b + 0.5) * s * math.sqrt(3) / 2)
                          for b in range(nrow) for a in range(ncol)])
        Lx, Ly = ncol * s, nrow * s * math.sqrt(3) / 2
    else:
        n = int(math.ceil(math.sqrt(P)))
        s = math.sqrt(area / phi) / n
        sites = np.array([((a + 0.5) * s, (b + 0.5) * s) for b in range(n) for a in range(n)])
        Lx = Ly = n * s
    pick = np.sort(rng.permutation(len(sites))[:P])
    return sites[pick].copy(), Lx, Ly, s


def _rsa(P, radii, Lx, Ly, gmin, rng, max_tries=10 ** 7):
    """Random sequential placement: uniform trial positions, rejected if they
    leave the box or come closer than gmin to a placed disk."""
    centres = np.zeros((P, 2))
    placed = 0
    tries = 0
    grid = _Grid(np.zeros((0, 2)), Lx, Ly, 2.0 * radii.max() + gmin + 1e-9)
    while placed < P:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("random sequential placement did not finish")
        r = radii[placed]
        c = np.array([rng.uniform(r, Lx - r), rng.uniform(r, Ly - r)])
        ok = True
        for k in grid.near(c):
            if math.hypot(c[0] - centres[k, 0], c[1] - centres[k, 1]) - r - radii[k] < gmin:
                ok = False
                break
        if ok:
            centres[placed] = c
            grid.add(placed, c)
            placed += 1
    return centres


def _snap_closest(centres, radii, Lx, Ly, gmin, target_gap):
    """Move one disk of the closest pair along the line of centres so that the
    pair's gap equals target_gap, if that keeps the packing admissible."""
    pairs = _min_gap_pairs(centres, radii, 0.5)
    if not pairs:
        return None
    for i, k, g in sorted(pairs, key=lambda t: t[2])[:20]:
        d = centres[k] - centres[i]
        dist = np.linalg.norm(d)
        new = centres[i] + d / dist * (radii[i] + radii[k] + target_gap)
        grid = _Grid(centres, Lx, Ly, 2.0 * radii.max() + 0.25)
        if _admissible(k, new, centres, radii, Lx, Ly, min(gmin, target_gap) * 0.999, grid,
                       skip=(i,)):
            centres[k] = new
            return (int(i), int(k), float(target_gap))
    return None


def packing(P, phi, seed, gmin=1e-3, radii=None, nsweep=10, start="square",
            snap_gap=None, step=None):
    """Random disk packing at area fraction phi in a rectangular box.

    start="square" (Sec. 6.2): square lattice at the target area fraction;
    start="hex": hexagonal lattice (needed when the largest disks do not fit a
    square lattice at phi); start="rsa": random sequential placement.  Then
    nsweep Metropolis sweeps with minimum gap gmin.  snap_gap: finally set the
    closest pair's gap to this value (one disk moved along the line of
    centres) when that keeps every other gap >= gmin.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    if radii is None:
        radii = np.ones(P)
    radii = np.asarray(radii, dtype=np.float64)
    area = float(np.pi * np.sum(radii ** 2))
    if start == "rsa":
        Lx = Ly = math.sqrt(area / phi)
        centres = _rsa(P, radii, Lx, Ly, gmin, rng)
        s = 2.0
    else:
        centres, Lx, Ly, s = _lattice(P, area, phi, start == "hex", rng)
        radii = radii[rng.permutation(P)]
        lattice_gap = s - 2 * radii.max()
        if lattice_gap < gmin:
            raise ValueError(f"lattice spacing {s:.4f} too small for radii up to {radii.max()}")
    if step is None:
        step = max(0.05, 0.5 * (s - 2 * radii.max()))
    acc = _sweeps(centres, radii, Lx, Ly, gmin, rng, nsweep, step)
    snapped = None
    if snap_gap is not None:
        snapped = _snap_closest(centres, radii, Lx, Ly, gmin, snap_gap)
    return Packing(centres=np.ascontiguousarray(centres), radii=np.ascontiguousarray(radii),
                   box=(Lx, Ly), meta={"P": P, "phi": phi, "seed": seed, "gmin": gmin,
                                       "start": start, "accept": acc, "snapped": snapped})


def gap_stats(pk: Packing, cutoff=0.2):
    pairs = _min_gap_pairs(pk.centres, pk.radii, cutoff)
    g = np.array([t[2] for t in pairs]) if pairs else np.zeros(0)
    return {"n_candidate": int(len(g)), "min_gap": float(g.min()) if len(g) else None,
            "frac_below_0.05": float(np.mean(g < 0.05)) if len(g) else 0.0}


# --- the named workloads --------------------------------------------------

def two_disks(gap=1e-3):
    """Two unit disks at the given gap along x."""
    c = np.array([[0.0, 0.0], [2.0 + gap, 0.0]])
    return Packing(centres=c, radii=np.ones(2), box=(8.0, 8.0), meta={"P": 2, "gap": gap})


def packing_p100(seed=2):
    """P=100 unit disks at area fraction 0.40: random sequential placement
    with minimum gap 1e-2, Metropolis sweeps, closest pair snapped to 1e-2."""
    return packing(100, 0.40, seed, gmin=1e-2, start="rsa", nsweep=20, snap_gap=1e-2, step=0.3)


def packing_p1000_poly(seed=3):
    """P=1000 disks with radii ~ U[0.8, 1.2] at area fraction 0.60, minimum
    gap 1e-3, from a hexagonal lattice."""
    rng = np.random.Generator(np.random.PCG64(seed + 1000))
    r = rng.uniform(0.8, 1.2, size=1000)
    return packing(1000, 0.60, seed, gmin=1e-3, radii=r, start="hex", nsweep=10,
                   snap_gap=1e-3)


def packing_p10000(seed=4, nsweep=6):
    """P=10^4 unit disks at area fraction 0.65 from a square lattice
    (spacing 2.198) with Metropolis sweeps at minimum gap 1e-3; closest pair
    snapped to 1e-3 (Sec. 6.2, Fig. 2)."""
    return packing(10000, 0.65, seed, gmin=1e-3, nsweep=nsweep, snap_gap=1e-3)


def cluster(P, delta, seed, max_tries=200000):
    """Random cluster of P unit disks in which every disk has separation
    exactly delta from at least one other (Sec. 6.1): disk 0 at the origin;
    each next disk at distance 2 + delta from a uniformly drawn earlier disk,
    in a uniform random direction, kept only if every other separation is at
    least delta.  Returns a Packing whose box bounds the cluster."""
    rng = np.random.Generator(np.random.PCG64(seed))
    c = np.zeros((P, 2))
    n, tries = 1, 0
    while n < P:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("cluster: no admissible placement found")
        j = int(rng.integers(n))
        a = rng.uniform(0.0, 2.0 * np.pi)
        x = c[j] + (2.0 + delta) * np.array([np.cos(a), np.sin(a)])
        d = np.hypot(c[:n, 0] - x[0], c[:n, 1] - x[1]) - 2.0
        d[j] = delta
        if d.min() >= delta * (1.0 - 1e-12):
            c[n] = x
            n += 1
    lo, hi = c.min(axis=0) - 1.0, c.max(axis=0) + 1.0
    return Packing(centres=c, radii=np.ones(P), box=(float(hi[0] - lo[0]), float(hi[1] - lo[1])),
                   meta={"P": P, "delta": delta, "seed": seed, "tries": tries})


def move_disks(pk: Packing, n_move, seed, frac=0.3, shift=(0.0, 0.0)):
    """One step of a moving geometry: n_move distinct disks (drawn without
    replacement) each displaced, one after the other, in a uniform random
    direction by frac times its current smallest gap to any other disk (so
    its gaps stay >= (1 - frac) times their values just before its move),
    then every centre shifted by `shift`.  Returns (new centres [P, 2], moved disk indices)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    c = pk.centres.copy()
    r = pk.radii
    idx = rng.choice(pk.P, size=n_move, replace=False)
    for j in idx:
        d = np.hypot(c[:, 0] - c[j, 0], c[:, 1] - c[j, 1]) - r - r[j]
        d[j] = np.inf
        a = rng.uniform(0.0, 2.0 * np.pi)
        c[j] += frac * d.min() * np.array([np.cos(a), np.sin(a)])
    c += np.asarray(shift, dtype=np.float64)
    return c, np.sort(idx)


def rigid_velocities(P, seed):
    """(v_x, v_y, omega) per disk, each N(0,1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((P, 3))


def forces_torques(P, seed):
    """(f_x, f_y, t) per disk, each N(0,1), forces shifted to zero net force
    (Sec. 6.1); torques are not shifted."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ft = rng.standard_normal((P, 3))
    ft[:, :2] -= ft[:, :2].mean(axis=0, keepdims=True)
    return ft


def smooth_surface_vector(P, Mc, seed, modes=4):
    """A smooth surface field per disk: low Fourier modes in the node angle
    (a realistic matvec input, unlike iid noise)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    th = 2 * np.pi * np.arange(Mc) / Mc
    out = np.zeros((P, Mc, 2))
    for m in range(modes + 1):
        a = rng.standard_normal((P, 2, 2)) / (1 + m) ** 2
        out[:, :, 0] += a[:, 0, 0:1] * np.cos(m * th) + a[:, 0, 1:2] * np.sin(m * th)
        out[:, :, 1] += a[:, 1, 0:1] * np.cos(m * th) + a[:, 1, 1:2] * np.sin(m * th)
    return out


def serving_stream(n, seed=0, pmin=50, pmax=5000, mean_gap_s=0.02):
    """Seeded request stream: Poisson arrivals (mean mean_gap_s apart); each a
    square-lattice packing with P log-uniform in [pmin, pmax], area fraction
    uniform in [0.3, 0.65], minimum gap log-uniform in [1e-3, 1e-1] (the
    closest pair snapped to it), resistance or mobility with probability 1/2,
    inputs N(0, 1) as rigid_velocities / forces_torques.  A square lattice of
    ceil(sqrt(P))^2 sites reaches only area fraction P pi / ((2 + gmin)
    ceil(sqrt(P)))^2 with every gap >= gmin, which is below 0.65 for small P
    that are not squares; the drawn area fraction is capped there (a draw
    under the cap is unchanged).
    Returns a list of (arrival_s, Packing, problem (0 resistance, 1 mobility),
    inputs [P, 3])."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out, t = [], 0.0
    for q in range(n):
        t += float(rng.exponential(mean_gap_s))
        P = int(round(math.exp(rng.uniform(math.log(pmin), math.log(pmax)))))
        phi = float(rng.uniform(0.3, 0.65))
        gmin = float(10 ** rng.uniform(-3, -1))
        n_side = int(math.ceil(math.sqrt(P)))
        phi = min(phi, (1 - 1e-9) * P * math.pi / ((2 + gmin) * n_side) ** 2)
        problem = int(rng.integers(0, 2))
        pk = packing(P, phi, 1000 + q, gmin=gmin, start="square", nsweep=3, snap_gap=gmin)
        data = rigid_velocities(P, 5000 + q) if problem == 0 else forces_torques(P, 5000 + q)
        out.append((t, pk, problem, data))
    return out
