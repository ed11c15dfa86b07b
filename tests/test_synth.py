"""The synthetic inputs follow their stated recipe: TIP3P geometry and
charges, ion counts and net charge, sites at least dmin apart (minimum image
in periodic boxes), atoms inside the box, the workloads' atom counts, the
log-uniform replica sizes, and the point-charge plasmas of the MD tests."""
import math

import numpy as np
import pytest
from scipy.spatial import cKDTree

from synth import TIP3P, WORKLOADS, make_ion_system, make_water_box, replica_sizes


@pytest.mark.parametrize("periodic,method", [(True, "rsa"), (True, "lattice"), (False, "rsa"), (False, "lattice")])
def test_water_box_recipe(periodic, method):
    L, nw, nna, ncl = 24.0, 420, 3, 2
    pos, q = make_water_box(L, nw, nna, ncl, seed=5, periodic=periodic, method=method)
    assert pos.shape == (3 * nw + nna + ncl, 3) and q.shape == (len(pos),)
    # charges per atom kind, net charge
    np.testing.assert_array_equal(q[0:3 * nw:3], TIP3P["qO"])
    np.testing.assert_array_equal(q[1:3 * nw:3], TIP3P["qH"])
    np.testing.assert_array_equal(q[2:3 * nw:3], TIP3P["qH"])
    assert np.all(q[3 * nw:3 * nw + nna] == 1.0) and np.all(q[3 * nw + nna:] == -1.0)
    assert q.sum() == pytest.approx(nna - ncl, abs=1e-9)

    def mi(d):
        return d - L * np.round(d / L) if periodic else d
    O, H1, H2 = pos[0:3 * nw:3], pos[1:3 * nw:3], pos[2:3 * nw:3]
    d1, d2 = mi(H1 - O), mi(H2 - O)
    np.testing.assert_allclose(np.linalg.norm(d1, axis=1), TIP3P["rOH"], rtol=1e-12)
    np.testing.assert_allclose(np.linalg.norm(d2, axis=1), TIP3P["rOH"], rtol=1e-12)
    cosang = (d1 * d2).sum(1) / (np.linalg.norm(d1, axis=1) * np.linalg.norm(d2, axis=1))
    np.testing.assert_allclose(np.degrees(np.arccos(cosang)), TIP3P["angle_deg"], rtol=1e-10)
    # sites (oxygens and ions) at least 2.5 A apart
    sites = np.vstack([O, pos[3 * nw:]])
    tree = cKDTree(np.mod(sites, L) if periodic else sites, boxsize=L if periodic else None)
    assert len(tree.query_pairs(2.5 - 1e-9)) == 0
    # inside the box
    if periodic:
        assert pos.min() >= 0.0 and pos.max() < L
    else:
        assert pos.min() >= 0.0 and pos.max() <= L


def test_orientations_are_not_aligned():
    pos, _ = make_water_box(30.0, 600, 0, 0, seed=9, periodic=True)
    O, H1, H2 = pos[0::3], pos[1::3], pos[2::3]
    bis = (H1 + H2) / 2.0 - O
    bis -= 30.0 * np.round(bis / 30.0)
    bis /= np.linalg.norm(bis, axis=1)[:, None]
    # uniform random orientations: the mean bisector is near zero, each axis's mean square near 1/3
    assert np.abs(bis.mean(axis=0)).max() < 0.1
    np.testing.assert_allclose((bis ** 2).mean(axis=0), 1.0 / 3.0, atol=0.05)


def test_workload_sizes():
    assert WORKLOADS["water3k_open"].n_atoms == 3000
    assert WORKLOADS["water23k"].n_atoms == 23558
    assert WORKLOADS["water1m"].n_atoms == 1066628
    assert WORKLOADS["water4m"].n_atoms == 4100000
    w = WORKLOADS["water23k"]
    pos, q = w.make()
    assert len(q) == 23558 and q.sum() == pytest.approx(2.0, abs=1e-9)
    # water density ~0.1 atoms per cubic A in the periodic boxes
    for name in ("water23k", "water1m", "water4m"):
        w = WORKLOADS[name]
        assert 0.095 < w.n_atoms / w.box ** 3 < 0.107, name


def test_replica_sizes_log_uniform():
    n = np.array(replica_sizes(64))
    assert len(n) == 64 and np.all(n % 3 == 0)
    assert n.min() >= 5000 - 3 and n.max() <= 50000 + 3
    u = (np.log(n) - math.log(5000)) / (math.log(50000) - math.log(5000))
    assert 0.35 < u.mean() < 0.65                    # log-uniform, not uniform in n
    assert replica_sizes(64) == replica_sizes(64)    # seeded


@pytest.mark.parametrize("kind", ["plasma", "salt"])
def test_ion_system_recipe(kind):
    pos, q, im, vel = make_ion_system(20.0, 150, seed=3, kind=kind, kT=0.05, mass=2.0)
    assert pos.shape == (150, 3) and vel.shape == (150, 3)
    if kind == "plasma":
        assert np.all(q == 1.0)
    else:
        assert q.sum() == 0.0 and set(np.unique(q)) == {-1.0, 1.0}
    np.testing.assert_array_equal(im, 0.5)
    np.testing.assert_allclose(vel.sum(axis=0), 0.0, atol=1e-12)   # no net momentum
    assert 0.5 < (vel ** 2).mean() / (0.05 / 2.0) < 1.5             # variance kT / m
    tree = cKDTree(np.mod(pos, 20.0), boxsize=20.0)
    assert len(tree.query_pairs(2.8 - 1e-9)) == 0
