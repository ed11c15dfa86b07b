"""Velocity Verlet molecular dynamics around the oracle's MSM force.

TEST INFRASTRUCTURE ONLY (as the rest of this package): the tests, and
nothing on the product path, call it.

The scheme is the velocity Verlet of the thesis proposal (Sec. "Molecular
Dynamics"): from r(t), v(t) and the acceleration a(t) = F(t)/m,

    v(t + dt/2) = v(t) + a(t) dt/2
    r(t + dt)   = r(t) + v(t + dt/2) dt
    r(t + dt)  -> U(r(t + dt)) -> a(t + dt)
    v(t + dt)   = v(t + dt/2) + a(t + dt) dt/2

written out step by step in FP64 with numpy.  ``velocity_verlet`` takes any
force routine, so that the integrator can be pinned on its own (a harmonic
force, whose discrete trajectory has a closed form); ``md_run`` plugs in the
oracle's MSM evaluation.
"""
import numpy as np

from . import msm


def velocity_verlet(force, r, v, inv_mass, dt, nsteps, f0=None, wrap=None):
    """nsteps velocity Verlet steps.  force(r) returns (F [n,3], potential
    energy); inv_mass [n] (0 fixes an atom); f0 = F(r) if already known; wrap
    maps positions back into the box after each drift (periodic boxes).
    Returns (r, v, F, records) with records [nsteps, 6] = (potential,
    kinetic, total, momentum x, y, z) after each step."""
    r = np.array(r, dtype=np.float64, copy=True)
    v = np.array(v, dtype=np.float64, copy=True)
    im = np.asarray(inv_mass, dtype=np.float64)
    F = force(r)[0] if f0 is None else np.array(f0, dtype=np.float64, copy=True)
    moving = im > 0
    m = np.zeros_like(im)
    m[moving] = 1.0 / im[moving]
    records = np.zeros((nsteps, 6))
    for s in range(nsteps):
        v = v + 0.5 * dt * F * im[:, None]          # v(t + dt/2)
        r = r + dt * v                               # r(t + dt)
        if wrap is not None:
            r = wrap(r)
        F, U = force(r)                              # F(t + dt) from U(r(t + dt))
        v = v + 0.5 * dt * F * im[:, None]          # v(t + dt)
        K = 0.5 * float(np.sum(m * np.sum(v * v, axis=1)))
        records[s] = (U, K, U + K, *np.sum(m[:, None] * v, axis=0))
    return r, v, F, records


def md_run(P, pos, vel, inv_mass, q, dt, nsteps, f0=None):
    """velocity_verlet with the oracle's MSM force and energy (parameters P);
    periodic boxes wrap positions into [0, L)."""
    q = np.asarray(q, dtype=np.float64)
    box = np.asarray(P.box, dtype=np.float64)

    def force(r):
        out = msm(P, r, q)
        return out["F"], out["E"]

    wrap = (lambda r: r - box * np.floor(r / box)) if P.periodic else None
    return velocity_verlet(force, pos, vel, inv_mass, dt, nsteps, f0=f0, wrap=wrap)
