"""Seeded point-charge systems for the molecular-dynamics tests: ions on a
jittered lattice (at least dmin apart), charges, masses and thermal
velocities.  No multilevel-summation arithmetic."""
import numpy as np

from .water import _lattice_sites


def make_ion_system(L, n, seed=0, kind="plasma", dmin=2.8, mass=1.0, kT=0.05, periodic=True):
    """Returns (pos [n,3], q [n], inv_mass [n], vel [n,3]), float64.

    kind "plasma": every ion +1 (a one-component plasma: like charges only,
    so nothing collapses under the bare Coulomb force); "salt": alternating
    +1 / -1.  Velocities are Gaussian with variance kT / mass per component,
    shifted so that the total momentum is zero."""
    rng = np.random.default_rng(seed)
    Lv = np.broadcast_to(np.asarray(L, float), (3,)).copy()
    lo = np.zeros(3) if periodic else np.full(3, 1.0)
    hi = Lv if periodic else Lv - 1.0
    pos = _lattice_sites(rng, n, Lv, lo, hi, periodic, dmin)
    if kind == "plasma":
        q = np.ones(n)
    elif kind == "salt":
        q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    else:
        raise ValueError("kind must be 'plasma' or 'salt'")
    inv_mass = np.full(n, 1.0 / mass)
    vel = rng.normal(0.0, np.sqrt(kT / mass), size=(n, 3))
    vel -= vel.mean(axis=0)
    return pos, q, inv_mass, vel
