"""Parareal integration of one window (Sec. "Parareal Method", Eq. parareal).

TEST INFRASTRUCTURE ONLY (as the rest of this package).

Time points T_k = T_0 + k dT, k = 0..W.  Iteration 0 is the coarse sweep
lambda_{k+1} = G(lambda_k); each further iteration evaluates the fine
propagator F at every point of the previous iterate, then sweeps

    lambda_{k+1}^{new} = G(lambda_k^{new}) + F(lambda_k^{old}) - G(lambda_k^{old})

from lambda_0 (fixed).  ``parareal`` is the generic driver (any state type
with the given combine and change rules); ``md_parareal`` instantiates it for
molecular dynamics with F = velocity Verlet on the oracle's MSM force and G =
velocity Verlet on the cutoff method's force (the parareal section's
simplest coarse propagator) or on MSM with coarser parameters.
"""
import numpy as np

from . import cutoff_sum
from .md import md_run, velocity_verlet


def parareal(fine, coarse, combine, change, converged, lam0, window, max_iter):
    """Returns (lam [window+1 states], history [iterate 0..K], changes [K])
    where change(new, old) measures an iteration over the whole window (new
    and old iterates, lists of states) and the driver stops once
    converged(change) holds (or after max_iter)."""
    lam = [lam0]
    g = []
    for k in range(window):                     # iteration 0: the coarse sweep
        g.append(coarse(lam[k]))
        lam.append(g[k])
    history = [list(lam)]
    changes = []
    for _ in range(max_iter):
        f = [fine(lam[k]) for k in range(window)]   # independent: parallel in time
        new = [lam0]
        for k in range(window):
            g_new = coarse(new[k])
            new.append(combine(g_new, f[k], g[k]))
            g[k] = g_new
        ch = change(new, lam)
        lam = new
        history.append(list(lam))
        changes.append(ch)
        if converged(ch):
            break
    return lam, history, changes


def md_parareal(P_fine, P_coarse, pos0, vel0, inv_mass, q, window, dt_fine, steps_fine, dt_coarse, steps_coarse,
                max_iter, tol, coarse_method="cutoff"):
    """Parareal MD: states (r, v); positions combined through the minimum
    image of F - G and wrapped when periodic; an iteration has converged
    when no position moved more than tol and no velocity more than
    tol / dT (dT = steps_fine dt_fine).  Returns (lam, history, changes)
    with changes [(largest position change, largest velocity change)]."""
    q = np.asarray(q, dtype=np.float64)
    im = np.asarray(inv_mass, dtype=np.float64)
    box = np.asarray(P_fine.box, dtype=np.float64)
    periodic = bool(P_fine.periodic)
    span = abs(dt_fine * steps_fine)

    def fine(state):
        r, v, _, _ = md_run(P_fine, state[0], state[1], im, q, dt_fine, steps_fine)
        return (r, v)

    def cutoff_force(r):
        out = cutoff_sum(P_coarse, r, q)
        return out["F"], out["E"]

    wrap = (lambda r: r - box * np.floor(r / box)) if periodic else None

    def coarse(state):
        if coarse_method == "msm":   # MSM with the coarse parameters (shorter cutoff, coarser grid)
            r, v, _, _ = md_run(P_coarse, state[0], state[1], im, q, dt_coarse, steps_coarse)
        else:
            r, v, _, _ = velocity_verlet(cutoff_force, state[0], state[1], im, dt_coarse, steps_coarse, wrap=wrap)
        return (r, v)

    def min_image(d):
        return d - box * np.round(d / box) if periodic else d

    def combine(g_new, f, g):
        r = g_new[0] + min_image(f[0] - g[0])
        if periodic:
            r = wrap(r)
        return (r, g_new[1] + (f[1] - g[1]))

    def change(new, old):
        dr = max(float(np.abs(min_image(a[0] - b[0])).max(initial=0.0)) for a, b in zip(new[1:], old[1:]))
        dv = max(float(np.abs(a[1] - b[1]).max(initial=0.0)) for a, b in zip(new[1:], old[1:]))
        return (dr, dv)

    def converged(ch):
        return ch[0] <= tol and ch[1] * span <= tol

    return parareal(fine, coarse, combine, change, converged, (np.array(pos0, float), np.array(vel0, float)),
                    window, max_iter)
