"""Pins of the oracle's velocity Verlet MD (Sec. "Molecular Dynamics", the
velocity Verlet scheme) against things other than itself.

- The integrator alone, on a harmonic force, where the discrete map has an
  exact quadratic invariant, v^2 + w^2 (1 - w^2 dt^2 / 4) x^2, and the
  trajectory converges to x0 cos(wt) + v0/w sin(wt) at second order.  A full
  instead of a half kick, a kick with the old force, or a drift with the old
  velocity breaks both.
- The integrator with the MSM force: exact time reversibility (negate the
  velocities and the trajectory retraces itself), and total energy conserved
  up to fluctuations that shrink as dt^2, which holds only if the force is
  the exact negative gradient of the energy the oracle reports.
"""
import numpy as np
import pytest

from synth import make_ion_system


def harmonic(k):
    def force(r):
        return -k * r, 0.5 * k * float(np.sum(r * r))
    return force


def test_velocity_verlet_harmonic_invariant(oracle):
    from oracle.md import velocity_verlet
    k, m, dt = 2.5, 0.7, 0.05
    w2 = k / m
    r0 = np.array([[0.9, -0.4, 0.2]])
    v0 = np.array([[0.1, 0.3, -0.8]])
    r, v, F, rec = velocity_verlet(harmonic(k), r0, v0, np.array([1.0 / m]), dt, 4000)
    Q0 = np.sum(v0 ** 2 + w2 * (1.0 - w2 * dt * dt / 4.0) * r0 ** 2, axis=0)
    Q = np.sum(v ** 2 + w2 * (1.0 - w2 * dt * dt / 4.0) * r ** 2, axis=0)
    np.testing.assert_allclose(Q, Q0, rtol=1e-12)
    # the plain energy is not invariant: it oscillates at O(dt^2)
    E = rec[:, 2]
    assert 1e-6 < (E.max() - E.min()) / E[0] < 1e-2
    np.testing.assert_allclose(F, -k * r, rtol=1e-15)


def test_velocity_verlet_second_order_convergence(oracle):
    from oracle.md import velocity_verlet
    k, m, T = 3.0, 1.3, 2.0
    w = np.sqrt(k / m)
    r0 = np.array([[0.5, 0.0, -0.25]])
    v0 = np.array([[0.0, 0.7, 0.1]])
    exact = r0 * np.cos(w * T) + v0 / w * np.sin(w * T)
    errs = []
    for nsteps in (100, 200, 400):
        r, _, _, _ = velocity_verlet(harmonic(k), r0, v0, np.array([1.0 / m]), T / nsteps, nsteps)
        errs.append(np.abs(r - exact).max())
    for e1, e2 in zip(errs, errs[1:]):
        assert 3.6 < e1 / e2 < 4.4          # global error ~ dt^2


def test_velocity_verlet_fixed_atoms_and_momentum(oracle):
    """inv_mass 0 fixes an atom; with a force that sums to zero (pairwise
    springs) the momentum of the moving atoms is conserved exactly."""
    from oracle.md import velocity_verlet

    def springs(r):
        d = r[:, None, :] - r[None, :, :]
        return -0.4 * d.sum(axis=1), 0.2 * float(np.sum(d * d)) / 2.0
    rng = np.random.default_rng(5)
    r0, v0 = rng.normal(size=(6, 3)), rng.normal(size=(6, 3))
    im = np.array([1.0, 0.5, 2.0, 1.0, 0.25, 1.0])
    r, v, _, rec = velocity_verlet(springs, r0, v0, im, 0.01, 300)
    p0 = np.sum(v0 / im[:, None], axis=0)
    np.testing.assert_allclose(rec[:, 3:], np.broadcast_to(p0, (300, 3)), rtol=1e-11, atol=1e-12)
    im[2] = 0.0
    r, v, _, rec = velocity_verlet(springs, r0, v0, im, 0.01, 50)
    np.testing.assert_allclose(r[2], r0[2] + 50 * 0.01 * v0[2], rtol=1e-13, atol=1e-14)  # drifts at constant v
    np.testing.assert_array_equal(v[2], v0[2])


def small_plasma():
    pos, q, im, vel = make_ion_system(16.0, 24, seed=11, kind="plasma", kT=0.05)
    return pos, q, im, vel


def test_md_msm_time_reversible(oracle):
    from oracle.md import md_run
    P = oracle.Params(box=(16.0,) * 3, periodic=True, cutoff=6.0, spacing=2.0, order=3, split=2)
    pos, q, im, vel = small_plasma()
    r1, v1, F1, _ = md_run(P, pos, vel, im, q, 0.05, 20)
    assert np.abs(r1 - pos).max() > 0.05                 # the atoms did move
    r2, v2, _, _ = md_run(P, r1, -v1, im, q, 0.05, 20, f0=F1)
    d = r2 - pos
    d -= 16.0 * np.round(d / 16.0)                       # across the periodic wrap
    assert np.abs(d).max() < 1e-10
    np.testing.assert_allclose(-v2, vel, atol=1e-10)


def test_md_msm_energy_fluctuation_scales_as_dt2(oracle):
    from oracle.md import md_run
    P = oracle.Params(box=(16.0,) * 3, periodic=True, cutoff=6.0, spacing=2.0, order=3, split=2)
    pos, q, im, vel = small_plasma()
    spread = []
    for dt, n in ((0.1, 20), (0.05, 40)):
        _, _, _, rec = md_run(P, pos, vel, im, q, dt, n)
        E = rec[:, 2]
        spread.append(np.abs(E - E[0]).max() / rec[:, 1].mean())
    assert spread[0] < 1e-4
    assert 3.0 < spread[0] / spread[1] < 5.5


# ------------------------------------------------------------- parareal ----
def test_parareal_linear_closed_form(oracle):
    """Linear propagators F(y) = f y, G(y) = g y: iterate k of the parareal
    recursion is lambda_n^k = sum_{j <= min(k, n)} C(n, j) (f - g)^j g^(n-j)
    y0 (the binomial expansion of (g + (f - g))^n truncated at order k), so
    iterate k is exact for n <= k."""
    from math import comb
    from oracle.parareal import parareal
    f, g, y0, W = 0.93, 0.71, 1.7, 7
    lam, hist, ch = parareal(lambda y: f * y, lambda y: g * y, lambda gn, fo, go: gn + fo - go,
                             lambda new, old: max(abs(a - b) for a, b in zip(new, old)), lambda c: False,
                             y0, W, W + 1)
    assert len(hist) == W + 2
    for k, it in enumerate(hist):
        for n in range(W + 1):
            want = y0 * sum(comb(n, j) * (f - g) ** j * g ** (n - j) for j in range(min(k, n) + 1))
            assert it[n] == pytest.approx(want, rel=1e-13)
        for n in range(min(k, W) + 1):
            assert it[n] == pytest.approx(y0 * f ** n, rel=1e-13)      # exact up to point k
    assert ch[-1] == pytest.approx(0.0, abs=1e-15)        # iterate W + 1 repeats iterate W


def test_md_parareal_reaches_the_sequential_fine_trajectory(oracle):
    """After `window` iterations every time point equals the sequential fine
    propagation (velocity Verlet on the MSM force) from the start; the
    iterations before are exact up to their own index."""
    from oracle.md import md_run
    from oracle.parareal import md_parareal
    P = oracle.Params(box=(16.0,) * 3, periodic=True, cutoff=6.0, spacing=2.0, order=3, split=2)
    pos, q, im, vel = small_plasma()
    W, dtf, sf = 3, 0.05, 4
    lam, hist, ch = md_parareal(P, P, pos, vel, im, q, W, dtf, sf, 0.1, 2, W, 0.0)
    r, v = pos, vel
    for n in range(1, W + 1):
        r, v, _, _ = md_run(P, r, v, im, q, dtf, sf)
        d = lam[n][0] - r
        d -= 16.0 * np.round(d / 16.0)
        assert np.abs(d).max() < 1e-11
        np.testing.assert_allclose(lam[n][1], v, atol=1e-11)
        # iterate 0 (coarse only) is already off at n = 1; iterate n is exact at n
        d0 = hist[0][n][0] - r
        assert np.abs(d0 - 16.0 * np.round(d0 / 16.0)).max() > 1e-6
        dn = hist[n][n][0] - r
        assert np.abs(dn - 16.0 * np.round(dn / 16.0)).max() < 1e-11
    assert ch[0][0] > ch[-1][0]
