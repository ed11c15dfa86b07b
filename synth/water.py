"""Seeded synthetic water boxes (rigid TIP3P geometry) with monovalent ions.

Recipe (stated once, used by every test and benchmark):
  * sites: water oxygens and ions.  Up to ``RSA_MAX_SITES`` sites are placed by
    random sequential addition (uniform proposals, rejected when closer than
    ``dmin`` = 2.5 A to an accepted site, tested in batches against a hash grid);
    larger systems (and the batched replicas) use a jittered rectangular
    lattice (node counts chosen so the lattice has at least as many nodes as
    sites, a random subset of nodes, uniform jitter of up to +-0.25 A per
    coordinate).  Both keep sites >= 2.5 A apart.
  * water: O at the site, the two H at 0.9572 A with H-O-H = 104.52 deg, in a
    uniformly random orientation (random unit quaternion).
  * charges: O -0.834 e, H +0.417 e, Na+ +1 e, Cl- -1 e.  Ions replace random
    sites.
  * periodic boxes fold every atom into [0, L); open boxes keep oxygens at
    least one O-H length from the faces so that every atom lies in [0, L].
Nothing here computes any part of the multilevel summation.
"""
import math
from dataclasses import dataclass, field

import numpy as np

TIP3P = {"qO": -0.834, "qH": 0.417, "rOH": 0.9572, "angle_deg": 104.52}
RSA_MAX_SITES = 60000


def _random_rotations(rng, n):
    """Uniform random rotation matrices from unit quaternions (Shoemake)."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    w, x = a * np.sin(2 * np.pi * u2), a * np.cos(2 * np.pi * u2)
    y, z = b * np.sin(2 * np.pi * u3), b * np.cos(2 * np.pi * u3)
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def _rsa_sites(rng, n, L, lo, hi, periodic, dmin):
    """Random sequential addition in the box [lo, hi]^3 (per dim)."""
    L = np.asarray(L, float)
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    span = hi - lo
    c = dmin / math.sqrt(3.0)                 # at most one site per hash cell
    nc = np.maximum(1, np.ceil((L if periodic else span) / c).astype(int))
    w = (L if periodic else span) / nc
    reach = int(math.ceil(dmin / w.min()))
    grid = -np.ones(int(nc.prod()), dtype=np.int64)
    sites = np.empty((n, 3))
    count = 0
    offs = np.array([(i, j, k) for i in range(-reach, reach + 1) for j in range(-reach, reach + 1)
                     for k in range(-reach, reach + 1)])
    stall = 0
    while count < n:
        need = n - count
        B = int(min(max(4 * need, 4096), 400000))
        cand = lo + rng.random((B, 3)) * span
        ci = np.floor((cand - (0.0 if periodic else lo)) / w).astype(int)
        ci = np.minimum(ci, nc - 1)
        ok = grid[(ci[:, 2] * nc[1] + ci[:, 1]) * nc[0] + ci[:, 0]] < 0
        cand, ci = cand[ok], ci[ok]
        # conflicts with accepted sites
        bad = np.zeros(len(cand), bool)
        for o in offs:
            cj = ci + o
            if periodic:
                cj %= nc
                valid = np.ones(len(cj), bool)
            else:
                valid = np.all((cj >= 0) & (cj < nc), axis=1)
                cj = np.clip(cj, 0, nc - 1)
            occ = grid[(cj[:, 2] * nc[1] + cj[:, 1]) * nc[0] + cj[:, 0]]
            m = valid & (occ >= 0)
            if m.any():
                d = cand[m] - sites[occ[m]]
                if periodic:
                    d -= L * np.round(d / L)
                bad[np.where(m)[0][np.einsum("ij,ij->i", d, d) < dmin * dmin]] = True
        cand, ci = cand[~bad], ci[~bad]
        # conflicts inside the batch: keep the earlier proposal
        flat = (ci[:, 2] * nc[1] + ci[:, 1]) * nc[0] + ci[:, 0]
        _, first = np.unique(flat, return_index=True)
        keep = np.zeros(len(cand), bool)
        keep[first] = True
        cand, ci, flat = cand[keep], ci[keep], flat[keep]
        tmp = -np.ones(int(nc.prod()), dtype=np.int64)
        tmp[flat] = np.arange(len(cand))
        bad = np.zeros(len(cand), bool)
        for o in offs:
            if not o.any():
                continue
            cj = ci + o
            if periodic:
                cj %= nc
                valid = np.ones(len(cj), bool)
            else:
                valid = np.all((cj >= 0) & (cj < nc), axis=1)
                cj = np.clip(cj, 0, nc - 1)
            oth = tmp[(cj[:, 2] * nc[1] + cj[:, 1]) * nc[0] + cj[:, 0]]
            m = valid & (oth >= 0) & (oth < np.arange(len(cand)))
            if m.any():
                d = cand[m] - cand[oth[m]]
                if periodic:
                    d -= L * np.round(d / L)
                bad[np.where(m)[0][np.einsum("ij,ij->i", d, d) < dmin * dmin]] = True
        cand, flat = cand[~bad], flat[~bad]
        take = min(len(cand), n - count)
        if take == 0:
            stall += 1
            if stall > 50:
                raise RuntimeError("random sequential addition stalled; density too high")
            continue
        stall = 0
        sites[count:count + take] = cand[:take]
        grid[flat[:take]] = np.arange(count, count + take)
        count += take
    return sites


def _lattice_sites(rng, n, L, lo, hi, periodic, dmin, jitter=0.25):
    """Jittered rectangular lattice, random subset of nodes.  Node counts per
    dimension start at the ~3.06 A water-density spacing and grow (the
    coarsest dimension first) until the lattice holds n nodes; the jitter
    shrinks if needed so that sites stay at least dmin apart."""
    span = (np.asarray(L, float) if periodic else np.asarray(hi, float) - np.asarray(lo, float))
    a = (float(np.prod(span)) / n) ** (1.0 / 3.0)
    m = np.maximum(1, np.floor(span / a).astype(int))
    nodes = (lambda mm: span / mm) if periodic else (lambda mm: span / np.maximum(mm - 1, 1))
    while int(m.prod()) < n:
        m[int(np.argmax(nodes(m)))] += 1
    step = nodes(m)
    jit = min(jitter, 0.499 * (float(step.min()) - dmin))
    if jit < 0:
        raise ValueError("lattice too dense for the minimum spacing")
    idx = rng.choice(int(m.prod()), size=n, replace=False)
    ijk = np.stack([idx % m[0], (idx // m[0]) % m[1], idx // (m[0] * m[1])], axis=1)
    base = (np.asarray(lo, float) if not periodic else 0.0) + ijk * step
    if periodic:
        base = base + 0.5 * step
    pos = base + rng.uniform(-jit, jit, size=(n, 3))
    if not periodic:
        pos = np.clip(pos, lo, hi)
    return pos


def make_water_box(L, n_water, n_na=0, n_cl=0, seed=0, periodic=True, dmin=2.5, method="auto"):
    """Returns (pos float64[N,3], q float64[N]) for n_water rigid TIP3P waters
    (atoms O, H, H per molecule) followed by n_na Na+ and n_cl Cl- ions."""
    rng = np.random.default_rng(seed)
    L = np.broadcast_to(np.asarray(L, float), (3,)).copy()
    n_sites = n_water + n_na + n_cl
    margin = 0.0 if periodic else TIP3P["rOH"] + 1e-6
    lo, hi = np.full(3, margin), L - margin
    if method == "auto":
        method = "rsa" if n_sites <= RSA_MAX_SITES else "lattice"
    place = _rsa_sites if method == "rsa" else _lattice_sites
    sites = place(rng, n_sites, L, lo, hi, periodic, dmin)
    perm = rng.permutation(n_sites)
    wsites, ions = sites[perm[:n_water]], sites[perm[n_water:]]
    th = math.radians(TIP3P["angle_deg"]) / 2.0
    r = TIP3P["rOH"]
    h_local = np.array([[r * math.sin(th), 0.0, r * math.cos(th)],
                        [-r * math.sin(th), 0.0, r * math.cos(th)]])
    R = _random_rotations(rng, n_water)
    H = wsites[:, None, :] + np.einsum("nij,kj->nki", R, h_local)
    pos = np.empty((3 * n_water + n_na + n_cl, 3))
    pos[0:3 * n_water:3] = wsites
    pos[1:3 * n_water:3] = H[:, 0]
    pos[2:3 * n_water:3] = H[:, 1]
    pos[3 * n_water:] = ions
    q = np.empty(len(pos))
    q[0:3 * n_water:3] = TIP3P["qO"]
    q[1:3 * n_water:3] = TIP3P["qH"]
    q[2:3 * n_water:3] = TIP3P["qH"]
    q[3 * n_water:3 * n_water + n_na] = 1.0
    q[3 * n_water + n_na:] = -1.0
    if periodic:
        pos = np.mod(pos, L)
        pos[pos >= L] -= L[np.nonzero(pos >= L)[1]]
    return pos, q


@dataclass
class Workload:
    """One named synthetic system together with its MSM parameters."""
    name: str
    box: float
    periodic: bool
    n_water: int
    n_na: int
    n_cl: int
    cutoff: float
    spacing: float
    order: int
    split: int
    levels: int = 0
    precision: str = "mixed"
    seed: int = 0
    notes: dict = field(default_factory=dict)

    @property
    def n_atoms(self):
        return 3 * self.n_water + self.n_na + self.n_cl

    def make(self, seed=None):
        return make_water_box(self.box, self.n_water, self.n_na, self.n_cl,
                              seed=self.seed if seed is None else seed, periodic=self.periodic)


WORKLOADS = {
    # open 30 A cube, 1,000 waters; a=12, h=2.5, cubic, Taylor C1, top grid <= 8^3
    "water3k_open": Workload("water3k_open", 30.0, False, 1000, 0, 0, 12.0, 2.5, 3, 1,
                             precision="fp64", seed=11),
    # periodic 62.2 A, 7,852 waters + 2 Na+ (net +2 e); a=10, h=2.0, cubic
    "water23k": Workload("water23k", 62.2, True, 7852, 2, 0, 10.0, 2.0, 3, 2, seed=12),
    # periodic 216.8 A, 354,930 waters + 919 Na+ + 919 Cl- (0.15 M); a=12, h=2.5, quintic
    "water1m": Workload("water1m", 216.8, True, 354930, 919, 919, 12.0, 2.5, 5, 2, seed=13),
    # periodic 340 A, 1,364,300 waters + 3,550 Na+ + 3,550 Cl- = 4.1M atoms; a=10, h=1.5, quintic, l=5
    "water4m": Workload("water4m", 340.0, True, 1364300, 3550, 3550, 10.0, 1.5, 5, 2, levels=5,
                        seed=15),
}


def workload(name):
    return WORKLOADS[name]


def replica_sizes(n_rep=64, lo=5000, hi=50000, seed=14):
    """Atom counts log-uniform in [lo, hi], rounded to a multiple of 3 (waters)."""
    rng = np.random.default_rng(seed)
    n = np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_rep))
    return (np.round(n / 3.0).astype(int) * 3).tolist()


def replica_boxes(n_rep=64, lo=5000, hi=50000, density=0.1, seed=14, method="lattice"):
    """The batched-replica workload: n_rep periodic water boxes whose atom
    counts are log-uniform in [lo, hi] (multiples of 3), each at the given
    atom density, L = (N / density)^(1/3).  Returns [(L, pos, q), ...]."""
    out = []
    for r, n in enumerate(replica_sizes(n_rep, lo, hi, seed)):
        L = (n / density) ** (1.0 / 3.0)
        pos, q = make_water_box(L, n // 3, 0, 0, seed=seed * 1000 + r, periodic=True, method=method)
        out.append((L, pos, q))
    return out


def spatial_subsample(pos, box, n_pick, seed=0):
    """Indices of the n_pick atoms nearest to a random point (minimum image):
    a compact spatial patch of the system."""
    rng = np.random.default_rng(seed)
    c = rng.random(3) * np.asarray(box, float)
    d = pos - c
    d -= np.asarray(box, float) * np.round(d / np.asarray(box, float))
    r2 = np.einsum("ij,ij->i", d, d)
    return np.sort(np.argpartition(r2, n_pick - 1)[:n_pick])
