"""Pins of the FP64 oracle against things other than itself.

Each test fixes one part of the oracle by a value the thesis proposal prints
(tests/golden/paper_values.json), a textbook closed form or constant
(tests/golden/textbook_values.json), an exact mathematical identity, an
invariance, or brute force on tiny inputs.  A plausible slip anywhere in the
oracle (a dropped term, a wrong sign, a transposed operator, a missing self
term, a wrong grid index) fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

from conftest import rel_rms
from synth import make_water_box, WORKLOADS

GOLD = os.path.join(os.path.dirname(__file__), "golden")
PAPER = json.load(open(os.path.join(GOLD, "paper_values.json")))
TEXT = json.load(open(os.path.join(GOLD, "textbook_values.json")))


# ---------------------------------------------------------------- gamma ----
def test_gamma_C2_equals_printed_polynomial(oracle):
    c0, c1, c2 = PAPER["gamma_C2_coefficients"]["value"]
    for rho in np.linspace(0.0, 0.999, 57):
        assert oracle.gamma(2, rho) == pytest.approx(c0 + c1 * rho ** 2 + c2 * rho ** 4, abs=1e-15)
    for rho in [1.0, 1.3, 2.0, 7.5]:
        assert oracle.gamma(2, rho) == pytest.approx(1.0 / rho, rel=1e-15)


@pytest.mark.parametrize("m", [1, 2, 3])
def test_gamma_matches_inverse_to_order_m(m, oracle):
    # value and first derivative meet 1/rho at rho = 1 for every m (C1 at least)
    assert oracle.gamma(m, 1.0 - 1e-12) == pytest.approx(1.0, abs=1e-10)
    assert oracle.dgamma(m, 1.0 - 1e-12) == pytest.approx(-1.0, abs=1e-10)
    # for m >= 2 also the second derivative (2/rho^3 = 2 at rho = 1)
    e = 1e-5
    d2 = (oracle.dgamma(m, 1.0 - e) - oracle.dgamma(m, 1.0 - 3 * e)) / (2 * e)
    if m >= 2:
        assert d2 == pytest.approx(2.0, abs=1e-3)
    else:
        assert abs(d2 - 2.0) > 0.5       # C1 smoothing has a kink in curvature
    # gamma(0) is the constant term of the truncated series: 3/2, 15/8, 35/16
    assert oracle.gamma(m, 0.0) == pytest.approx({1: 1.5, 2: 1.875, 3: 2.1875}[m], abs=1e-15)


@pytest.mark.parametrize("m", [1, 2, 3])
def test_dgamma_is_derivative(m, oracle):
    for rho in [0.1, 0.4, 0.77, 0.98, 1.2, 3.0]:
        e = 1e-6
        fd = (oracle.gamma(m, rho + e) - oracle.gamma(m, rho - e)) / (2 * e)
        assert oracle.dgamma(m, rho) == pytest.approx(fd, abs=1e-8)


# ------------------------------------------------------- kernel splitting --
@pytest.mark.parametrize("l", [1, 2, 3, 5])
@pytest.mark.parametrize("m", [1, 2])
def test_splitting_telescopes_to_coulomb(l, m, oracle):
    """Eq. msmgrid: 1/r = g* + g^0 + ... + g^{l-2} + g^{l-1} for every r."""
    a = 9.0
    for r in [0.3, 1.0, 4.5, 8.99, 9.01, 17.0, 30.0, 70.0, 200.0]:
        s = oracle.gstar(m, a, r) + sum(oracle.glevel(m, a, k, r) for k in range(l - 1)) \
            + oracle.gtop(m, a, l - 1, r)
        assert s == pytest.approx(1.0 / r, rel=1e-13)


def test_level_kernels_have_compact_support(oracle):
    a = 10.0
    assert oracle.gstar(2, a, a) == 0.0 and oracle.gstar(2, a, 1.5 * a) == 0.0
    assert abs(oracle.gstar(2, a, a * (1 - 1e-9))) < 1e-12          # continuous at r = a
    for k in range(4):
        rk = a * 2 ** (k + 1)
        assert oracle.glevel(2, a, k, rk) == 0.0
        assert abs(oracle.glevel(2, a, k, rk * (1 - 1e-9))) < 1e-12
        # level scaling g^k(r) = 2^-k g^0(r / 2^k)
        for r in [0.0, 3.0, 11.0, 17.0]:
            assert oracle.glevel(2, a, k, r * 2 ** k) == pytest.approx(
                oracle.glevel(2, a, 0, r) / 2 ** k, rel=1e-13, abs=1e-16)


def test_dgstar_is_derivative(oracle):
    a = 12.0
    for r in [0.5, 2.0, 7.0, 11.9]:
        e = 1e-6
        fd = (oracle.gstar(2, a, r + e) - oracle.gstar(2, a, r - e)) / (2 * e)
        assert oracle.dgstar(2, a, r) == pytest.approx(fd, rel=1e-6, abs=1e-10)


# ------------------------------------------------------------ basis Phi ----
@pytest.mark.parametrize("p,S,deg", [(3, 2, 2), (5, 3, 4)])
def test_Phi_interpolates_and_reproduces_polynomials(p, S, deg, oracle):
    assert oracle.Phi(p, 0.0) == 1.0
    for n in range(1, S + 2):
        assert oracle.Phi(p, n) == 0.0 and oracle.Phi(p, -n) == 0.0
    for x in np.linspace(0.0, 1.0, 23):
        for j in range(deg + 1):
            s = sum(oracle.Phi(p, x - n) * n ** j for n in range(-S - 1, S + 3))
            assert s == pytest.approx(x ** j, abs=1e-12), (p, x, j)
        # one degree higher is not reproduced everywhere (order is exactly deg+1)
    bad = max(abs(sum(oracle.Phi(p, x - n) * n ** (deg + 1) for n in range(-S - 1, S + 3))
                  - x ** (deg + 1)) for x in np.linspace(0.05, 0.95, 19))
    assert bad > 1e-3


def test_cubic_Phi_is_keys_kernel(oracle):
    for x in np.linspace(-2.5, 2.5, 101):
        t = abs(x)
        if t <= 1:
            w = 1.5 * t ** 3 - 2.5 * t ** 2 + 1
        elif t < 2:
            w = -0.5 * t ** 3 + 2.5 * t ** 2 - 4 * t + 2
        else:
            w = 0.0
        assert oracle.Phi(3, x) == pytest.approx(w, abs=1e-14)


@pytest.mark.parametrize("p", [3, 5])
def test_Phi_is_C1_and_dPhi_is_derivative(p, oracle):
    S = (p + 1) // 2
    e = 1e-6
    for x in np.linspace(-S - 0.5, S + 0.5, 77):
        fd = (oracle.Phi(p, x + e) - oracle.Phi(p, x - e)) / (2 * e)
        assert oracle.dPhi(p, x) == pytest.approx(fd, abs=1e-7)
    for knot in range(0, S + 1):
        assert oracle.dPhi(p, knot - 1e-10) == pytest.approx(oracle.dPhi(p, knot + 1e-10), abs=1e-8)


def test_restriction_weights_are_exact_rationals(oracle):
    for name, p in [("cubic", 3), ("quintic", 5)]:
        total = 0.0
        for d, w in TEXT["restriction_weights"][name]:
            assert oracle.Phi(p, d / 2.0) == w
            total += w * (1 if d == 0 else 2)
        assert total == 2.0      # the 1-D restriction stencil sums to 2


# ------------------------------------------------------------- geometry ----
def test_geometry_readings(oracle):
    P = oracle.Params(box=(62.2,) * 3, periodic=True, cutoff=10.0, spacing=2.0, order=3)
    G = oracle.geometry(P)
    assert [n[0] for n in G.n] == [32, 16, 8] and G.h[0] == pytest.approx(62.2 / 32)
    P = oracle.Params(box=(216.8,) * 3, periodic=True, cutoff=12.0, spacing=2.5, order=5)
    assert [n[0] for n in oracle.geometry(P).n] == [96, 48, 24, 12, 6]      # 86.72 -> 3*32
    P = oracle.Params(box=(340.0,) * 3, periodic=True, cutoff=10.0, spacing=1.5, order=5, levels=5)
    assert [n[0] for n in oracle.geometry(P).n] == [240, 120, 60, 30, 15]   # 226.7 -> 15*16
    # open 30 A, h = 2.5, cubic (S = 2): level 0 spans -1..14 (16 points);
    # level 1 spans ceil((-1-3)/2) = -2 .. floor((14+3)/2) = 8 (11 points);
    # level 2 spans -2 .. floor((8+3)/2) = 5 (8 points) -> stop (<= 8)
    P = oracle.Params(box=(30.0,) * 3, periodic=False, cutoff=12.0, spacing=2.5, order=3, split=1)
    G = oracle.geometry(P)
    assert [n[0] for n in G.n] == [16, 11, 8] and [lo[0] for lo in G.lo] == [-1, -2, -2]


# --------------------------------------------- grid transfer operators ----
def _small_system(periodic, seed=1, L=24.0, nw=300):
    return make_water_box(L, nw, 2, 2, seed=seed, periodic=periodic)


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("order", [3, 5])
def test_charge_conservation_and_transposes(periodic, order, oracle):
    pos, q = _small_system(periodic)
    P = oracle.Params(box=(24.0,) * 3, periodic=periodic, cutoff=6.0, spacing=1.5, order=order,
                      levels=3)
    G = oracle.geometry(P)
    q0 = oracle.anterpolate(P, G, pos, q)
    assert q0.sum() == pytest.approx(q.sum(), abs=1e-11)          # partition of unity
    q1 = oracle.restrict(P, G, 0, q0)
    assert q1.sum() == pytest.approx(q0.sum(), abs=1e-11)
    rng = np.random.default_rng(5)
    # prolongation is the transpose of restriction: <R x, y> = <x, P y>
    x, y = rng.standard_normal(G.shape(0)), rng.standard_normal(G.shape(1))
    Py = oracle.prolongate(P, G, 0, y, np.zeros(G.shape(0)))
    assert np.vdot(oracle.restrict(P, G, 0, x), y) == pytest.approx(np.vdot(x, Py), rel=1e-12)
    # interpolation is the transpose of anterpolation: sum_mu q0_mu u_mu = sum_j q_j u(r_j)
    u = rng.standard_normal(G.shape(0))
    ul, _ = oracle.interpolate(P, G, pos, u)
    assert np.vdot(q0, u) == pytest.approx(np.dot(q, ul), rel=1e-12)


def _brute_lattice(oracle, P, G, k, qk, kernel):
    """sum over every pair of grid points (and, periodic, over images)."""
    n = G.n[k]
    hk = [G.h[d] * 2 ** k for d in range(3)]
    idx = np.array([(x, y, z) for z in range(n[2]) for y in range(n[1]) for x in range(n[0])])
    flat = qk.reshape(-1)
    out = np.zeros(len(idx))
    imgs = [(0, 0, 0)]
    if P.periodic:
        R = 1
        imgs = [(i, j, l) for i in range(-R, R + 1) for j in range(-R, R + 1) for l in range(-R, R + 1)]
    for a, mu in enumerate(idx):
        s = 0.0
        for b, nu in enumerate(idx):
            for im in imgs:
                d = [(mu[c] - nu[c] + im[c] * n[c]) * hk[c] for c in range(3)]
                s += kernel(math.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2)) * flat[b]
        out[a] = s
    return out.reshape(qk.shape)


@pytest.mark.parametrize("periodic", [True, False])
def test_lattice_cutoff_equals_brute_force(periodic, oracle):
    P = oracle.Params(box=(9.0,) * 3, periodic=periodic, cutoff=2.0, spacing=1.5, order=3, levels=2)
    G = oracle.geometry(P)
    rng = np.random.default_rng(2)
    for k in range(G.levels - 1):
        qk = rng.standard_normal(G.shape(k))
        got = oracle.lattice_cutoff(P, G, k, qk)
        ref = _brute_lattice(oracle, P, G, k, qk, lambda r: oracle.glevel(P.split, P.cutoff, k, r))
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)
        q2 = rng.standard_normal(G.shape(k))    # symmetric operator
        assert np.vdot(got, q2) == pytest.approx(np.vdot(qk, oracle.lattice_cutoff(P, G, k, q2)), rel=1e-12)


def test_open_top_level_equals_brute_force(oracle):
    P = oracle.Params(box=(8.0,) * 3, periodic=False, cutoff=2.0, spacing=2.0, order=3, levels=2)
    G = oracle.geometry(P)
    qt = np.random.default_rng(3).standard_normal(G.shape(1))
    got = oracle.top_level(P, G, qt)
    ref = _brute_lattice(oracle, P, G, 1, qt, lambda r: oracle.gtop(P.split, P.cutoff, 1, r))
    np.testing.assert_allclose(got, ref, rtol=1e-12)


# ---------------------------------------------------------------- Ewald ----
def _rocksalt(ncell, r0):
    base = [(0, 0, 0, 1), (1, 1, 0, 1), (1, 0, 1, 1), (0, 1, 1, 1),
            (1, 0, 0, -1), (0, 1, 0, -1), (0, 0, 1, -1), (1, 1, 1, -1)]
    pos, q = [], []
    for i in range(ncell):
        for j in range(ncell):
            for k in range(ncell):
                for (x, y, z, s) in base:
                    pos.append(((2 * i + x) * r0, (2 * j + y) * r0, (2 * k + z) * r0))
                    q.append(float(s))
    return np.array(pos), np.array(q), 2 * ncell * r0


def test_ewald_reproduces_madelung_constant(oracle):
    pos, q, L = _rocksalt(2, 2.82)
    E = oracle.ewald_sum((L,) * 3, pos, q)["E"]
    M = TEXT["madelung_nacl"]["value"]
    assert E / (len(q) / 2) == pytest.approx(-M / 2.82, rel=1e-10)


def test_ewald_independent_of_splitting_parameter(oracle):
    pos, q = make_water_box(20.0, 200, 1, 0, seed=4, periodic=True)   # net charge +1
    a = oracle.ewald_sum((20.0,) * 3, pos, q, eps_exp=5.0)
    b = oracle.ewald_sum((20.0,) * 3, pos, q, eps_exp=6.5)
    assert a["E"] == pytest.approx(b["E"], rel=1e-10)
    assert rel_rms(a["F"], b["F"]) < 1e-9


def test_direct_sum_closed_form(oracle):
    pos = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0]])
    q = np.array([2.0, -0.5])
    D = oracle.direct_sum(pos, q)
    assert D["E"] == pytest.approx(2.0 * -0.5 / 5.0, rel=1e-15)
    # force on atom 0 is attractive, |F| = |q1 q2| / r^2 along the line
    np.testing.assert_allclose(D["F"][0], [0.024, 0.032, 0.0], rtol=1e-14)
    np.testing.assert_allclose(D["F"][1], -D["F"][0], rtol=1e-15)


@pytest.mark.parametrize("periodic", [True, False])
def test_short_range_link_cells_equal_brute_force(periodic, oracle):
    pos, q = make_water_box(40.0, 1500, 3, 3, seed=6, periodic=periodic)
    P = oracle.Params(box=(40.0,) * 3, periodic=periodic, cutoff=9.0, spacing=2.0, order=3)
    a = oracle.short_range(P, pos, q, method="brute")
    b = oracle.short_range(P, pos, q, method="cells")
    np.testing.assert_allclose(a[0], b[0], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(a[1], b[1], rtol=1e-12, atol=1e-12)


# ---------------------------------------------- whole method vs textbook ----
def test_open_msm_vs_direct_sum_water3k(oracle):
    w = WORKLOADS["water3k_open"]
    pos, q = w.make()
    D = oracle.direct_sum(pos, q)
    # the workload's own setting: Taylor C1, cubic, a = 12, h = 2.5
    P = oracle.Params(box=(w.box,) * 3, periodic=False, cutoff=w.cutoff, spacing=w.spacing,
                      order=w.order, split=w.split)
    R = oracle.msm(P, pos, q)
    band = PAPER["force_rel_error_band_from_8A"]["value"][1]
    e_c1 = rel_rms(R["F"], D["F"])
    assert e_c1 < band
    assert abs(R["E"] - D["E"]) / abs(D["E"]) < 1e-4
    # the paper's quoted setting (C2, cubic, a = 12, h = 2): below 1%
    g = PAPER["force_rel_error_bound_C2_cubic"]
    P2 = oracle.Params(box=(w.box,) * 3, periodic=False, cutoff=g["setting"]["cutoff"],
                       spacing=g["setting"]["spacing"], order=3, split=2)
    R2 = oracle.msm(P2, pos, q)
    assert rel_rms(R2["F"], D["F"]) < g["value"]
    assert rel_rms(R2["F"], D["F"]) < e_c1          # smoother splitting is more accurate
    # error shrinks with order and with h
    P3 = oracle.Params(box=(w.box,) * 3, periodic=False, cutoff=12.0, spacing=2.0, order=5, split=2)
    assert rel_rms(oracle.msm(P3, pos, q)["F"], D["F"]) < rel_rms(R2["F"], D["F"])
    P4 = oracle.Params(box=(w.box,) * 3, periodic=False, cutoff=12.0, spacing=1.25, order=3, split=1)
    assert rel_rms(oracle.msm(P4, pos, q)["F"], D["F"]) < e_c1
    # net force: small against the force scale but not zero (no momentum conservation)
    net = np.linalg.norm(R["F"].sum(0))
    scale = np.sqrt((D["F"] ** 2).sum())
    assert 0.0 < net < 0.05 * scale


@pytest.mark.parametrize("charged", [False, True])
def test_periodic_msm_vs_ewald(charged, oracle):
    pos, q = make_water_box(30.0, 900, 0, 0, seed=3, periodic=True)
    if charged:
        pos = np.vstack([pos, [[5.0, 5.0, 5.0], [20.0, 20.0, 20.0]]])
        q = np.concatenate([q, [1.0, 1.0]])
    Ew = oracle.ewald_sum((30.0,) * 3, pos, q)
    P = oracle.Params(box=(30.0,) * 3, periodic=True, cutoff=12.0, spacing=2.0, order=3, split=2)
    R = oracle.msm(P, pos, q)
    assert rel_rms(R["F"], Ew["F"]) < PAPER["force_rel_error_bound_C2_cubic"]["value"]
    assert abs(R["E"] - Ew["E"]) / abs(Ew["E"]) < 1e-4
    P5 = oracle.Params(box=(30.0,) * 3, periodic=True, cutoff=12.0, spacing=2.0, order=5, split=2)
    assert rel_rms(oracle.msm(P5, pos, q)["F"], Ew["F"]) < rel_rms(R["F"], Ew["F"])


def test_periodic_top_kernel_is_finite_and_symmetric(oracle):
    P = oracle.Params(box=(30.0,) * 3, periodic=True, cutoff=6.0, spacing=2.0, order=3, split=2)
    G = oracle.geometry(P)
    M = G.n[-1][0]
    for n in [(0, 0, 0), (1, 0, 0), (1, 2, 3)]:
        k = oracle.top_kernel_periodic(P, G, n)
        assert np.isfinite(k)
        assert k == pytest.approx(oracle.top_kernel_periodic(P, G, [(-v) % M for v in n]), rel=1e-12)
        assert k == pytest.approx(oracle.top_kernel_periodic(P, G, (n[2], n[0], n[1])), rel=1e-12)


# ----------------------------------------------------------- invariants ----
def _params_small(periodic, order=3):
    return dict(box=(24.0,) * 3, periodic=periodic, cutoff=8.0, spacing=2.0, order=order, split=2)


@pytest.mark.parametrize("periodic", [True, False])
def test_linearity_in_charges(periodic, oracle):
    pos, q = _small_system(periodic)
    P = oracle.Params(**_params_small(periodic))
    a = oracle.msm(P, pos, q)
    b = oracle.msm(P, pos, -2.5 * q)
    assert b["E"] == pytest.approx(6.25 * a["E"], rel=1e-12)
    np.testing.assert_allclose(b["phi"], -2.5 * a["phi"], rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("periodic", [True, False])
def test_permutation_invariance(periodic, oracle):
    pos, q = _small_system(periodic)
    P = oracle.Params(**_params_small(periodic))
    a = oracle.msm(P, pos, q)
    perm = np.random.default_rng(8).permutation(len(q))
    b = oracle.msm(P, pos[perm], q[perm])
    assert b["E"] == pytest.approx(a["E"], rel=1e-12)
    np.testing.assert_allclose(b["F"], a["F"][perm], rtol=1e-10, atol=1e-12)


def test_periodic_translation_by_grid_vectors(oracle):
    pos, q = _small_system(True)
    P = oracle.Params(**_params_small(True))
    G = oracle.geometry(P)
    assert G.levels >= 2
    # every level is invariant under shifts by the top-level spacing 2^(l-1) h
    ht = np.array(G.h) * 2 ** (G.levels - 1)
    a = oracle.msm(P, pos, q)
    shift = ht * np.array([1, -2, 3])
    b = oracle.msm(P, np.mod(pos + shift, 24.0), q)
    assert b["E"] == pytest.approx(a["E"], rel=1e-11)
    np.testing.assert_allclose(b["F"], a["F"], rtol=1e-8, atol=1e-10)
    # a shift by one finest-grid cell (half a coarse cell) or off the grid
    # changes the result, but only within the method's error
    for frac in [np.array(G.h), 0.37 * np.array(G.h)]:
        c = oracle.msm(P, np.mod(pos + frac, 24.0), q)
        assert c["E"] != pytest.approx(a["E"], rel=1e-11)
        assert abs(c["E"] - a["E"]) / abs(a["E"]) < 1e-4


@pytest.mark.parametrize("periodic,order", [(True, 3), (False, 3), (True, 5)])
def test_forces_are_minus_energy_gradient(periodic, order, oracle):
    pos, q = make_water_box(18.0, 120, 1, 1, seed=9, periodic=periodic)
    P = oracle.Params(box=(18.0,) * 3, periodic=periodic, cutoff=6.0, spacing=1.5, order=order, split=2)
    R = oracle.msm(P, pos, q)
    rng = np.random.default_rng(10)
    e = 1e-5
    for i in rng.choice(len(q), 5, replace=False):
        for d in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, d] += e
            pm[i, d] -= e
            fd = -(oracle.msm(P, pp, q)["E"] - oracle.msm(P, pm, q)["E"]) / (2 * e)
            assert R["F"][i, d] == pytest.approx(fd, rel=1e-6, abs=1e-7)
        qp, qm = q.copy(), q.copy()
        qp[i] += e
        qm[i] -= e
        fdq = (oracle.msm(P, pos, qp)["E"] - oracle.msm(P, pos, qm)["E"]) / (2 * e)
        assert R["phi"][i] == pytest.approx(fdq, rel=1e-7, abs=1e-8)


def test_two_charges_and_single_charge(oracle):
    """Two opposite unit charges at distance r: E -> -1/r and |F| -> 1/r^2
    within the method's error, which shrinks as h is refined.  The forces on
    the two atoms are opposite only within that error (the grid part carries a
    small self force: MSM does not conserve momentum)."""
    def run(h, r):
        P = oracle.Params(box=(40.0,) * 3, periodic=False, cutoff=8.0, spacing=h, order=3, split=2)
        pos = np.array([[10.0, 11.0, 12.0], [10.0 + r, 11.0, 12.0]])
        return oracle.msm(P, pos, np.array([1.0, -1.0]))
    for r in [3.0, 9.0, 17.0]:
        c, f = run(2.0, r), run(1.0, r)
        err_c = abs(c["E"] + 1.0 / r) * r
        err_f = abs(f["E"] + 1.0 / r) * r
        assert err_c < 2e-2 and err_f < err_c
        assert abs(c["F"][0][0] * r ** 2 - 1.0) < 6e-2
        assert abs(f["F"][0][0] * r ** 2 - 1.0) < abs(c["F"][0][0] * r ** 2 - 1.0)
        assert np.linalg.norm(c["F"][0] + c["F"][1]) < 6e-2 / r ** 2
    # one charge: the self term removes gamma(0)/a; what remains is the grid's
    # interpolation residual of the smooth kernel at r = 0
    P = oracle.Params(box=(40.0,) * 3, periodic=False, cutoff=8.0, spacing=2.0, order=3, split=2)
    R1 = oracle.msm(P, np.array([[13.3, 14.1, 15.7]]), np.array([1.0]))
    assert abs(R1["E"]) < 1e-2 * oracle.self_coefficient(P)


def test_single_level_top_only(oracle):
    pos, q = make_water_box(20.0, 250, 0, 0, seed=12, periodic=False)
    D = oracle.direct_sum(pos, q)
    P = oracle.Params(box=(20.0,) * 3, periodic=False, cutoff=8.0, spacing=2.0, order=3, split=2, levels=1)
    R = oracle.msm(P, pos, q)
    assert R["geometry"].levels == 1
    assert rel_rms(R["F"], D["F"]) < 0.01


# ---- the cutoff method (the parareal section's coarse propagator G) ----

def test_cutoff_sum_two_charges_closed_form(oracle):
    """Two charges: inside the cutoff E = q1 q2 / r and F = +-q1 q2 d / r^3
    (like charges repel); beyond it nothing, with open and periodic boxes
    (minimum image across the boundary)."""
    for periodic, pos in [(False, [[2.0, 3.0, 4.0], [5.0, 7.0, 4.0]]),    # r = 5
                          (True, [[0.5, 10.0, 10.0], [19.5 - 4.0, 10.0, 10.0]])]:  # image r = 5
        P = oracle.Params(box=(20.0,) * 3, periodic=periodic, cutoff=6.0, spacing=2.0)
        q = np.array([0.8, -1.3])
        out = oracle.cutoff_sum(P, np.array(pos), q)
        assert out["E"] == pytest.approx(0.8 * -1.3 / 5.0, rel=1e-14)
        d = np.array(pos[0]) - np.array(pos[1])
        if periodic:
            d -= 20.0 * np.round(d / 20.0)
        f0 = 0.8 * -1.3 * d / 125.0
        np.testing.assert_allclose(out["F"][0], f0, rtol=1e-13, atol=1e-16)
        np.testing.assert_allclose(out["F"][1], -f0, rtol=1e-13, atol=1e-16)
        P4 = oracle.Params(box=(20.0,) * 3, periodic=periodic, cutoff=4.9, spacing=2.0)
        far = oracle.cutoff_sum(P4, np.array(pos), q)
        assert far["E"] == 0.0 and np.all(far["F"] == 0.0)


def test_cutoff_sum_equals_direct_sum_when_nothing_is_cut(oracle):
    """An open box with a cutoff beyond its diagonal: the cutoff method is the
    plain Coulomb sum (an independent routine, no minimum image, no cutoff)."""
    pos, q = make_water_box(14.0, 60, 1, 1, seed=71, periodic=False)
    P = oracle.Params(box=(14.0,) * 3, periodic=False, cutoff=30.0, spacing=2.0)
    a, b = oracle.cutoff_sum(P, pos, q), oracle.direct_sum(pos, q)
    assert a["E"] == pytest.approx(b["E"], rel=1e-13)
    np.testing.assert_allclose(a["F"], b["F"], rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(a["phi"], b["phi"], rtol=1e-12, atol=1e-13)


def test_cutoff_sum_forces_are_the_energy_gradient_and_scale(oracle):
    """Central finite differences of E give -F (no pair within the step of
    the cutoff edge); E(alpha q) = alpha^2 E."""
    pos, q = make_water_box(16.0, 80, 1, 1, seed=72, periodic=True)
    P = oracle.Params(box=(16.0,) * 3, periodic=True, cutoff=6.5, spacing=2.0)
    ref = oracle.cutoff_sum(P, pos, q)
    h = 1e-5
    rng = np.random.default_rng(72)
    checked = 0
    for i in rng.choice(len(q), 12, replace=False):
        d = pos - pos[i]
        d -= 16.0 * np.round(d / 16.0)
        r = np.sqrt((d ** 2).sum(1))
        r[i] = 0.0
        if np.any(np.abs(r[r > 0] - 6.5) < 1e-3):
            continue
        for c in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, c] += h
            pm[i, c] -= h
            fd = -(oracle.cutoff_sum(P, pp, q)["E"] - oracle.cutoff_sum(P, pm, q)["E"]) / (2 * h)
            assert fd == pytest.approx(ref["F"][i, c], rel=1e-6, abs=1e-8)
        checked += 1
    assert checked >= 6
    assert oracle.cutoff_sum(P, pos, 1.7 * q)["E"] == pytest.approx(1.7 ** 2 * ref["E"], rel=1e-13)


# ---- Wolf summation (damped, shifted-force form), a coarse function of the
# parareal section: pinned by the rock-salt Madelung constant, by its alpha = 0
# limit against the independently pinned cutoff method, by the continuity of
# the pair potential and force at R, and by finite differences.

def test_wolf_sum_reproduces_madelung_constant(oracle):
    """Wolf's damped, charge-neutralised sum converges to the lattice sum: on
    a periodic rock-salt crystal (nearest-neighbour distance 2.82 A, 4,096
    ions) its energy per ion pair is -M/r0 to 1e-7 at alpha = 0.2/A,
    R = 20 A and to 1e-6 at alpha = 0.25/A, R = 15 A (M: the textbook
    Madelung constant)."""
    pos, q, L = _rocksalt(8, 2.82)
    M = TEXT["madelung_nacl"]["value"]
    for alpha, R, tol in [(0.2, 20.0, 1e-7), (0.25, 15.0, 1e-6)]:
        P = oracle.Params(box=(L,) * 3, periodic=True, cutoff=R, spacing=2.0)
        out = oracle.wolf_sum(P, pos, q, alpha)
        assert out["E"] / (len(q) / 2) == pytest.approx(-M / 2.82, rel=tol), (alpha, R)
        # a perfect crystal: every ion feels no net force
        assert np.abs(out["F"]).max() < 1e-9


def test_wolf_sum_alpha_zero_is_the_shifted_force_cutoff(oracle):
    """alpha = 0: v(r) = 1/r - 1/R + (r - R)/R^2 within R and the self term
    q_i^2/(2R).  Built here from the cutoff method's potentials (an
    independently pinned routine) plus per-pair sums of q_j and q_j r."""
    pos, q = make_water_box(18.0, 120, 2, 2, seed=81, periodic=True)
    R = 7.0
    P = oracle.Params(box=(18.0,) * 3, periodic=True, cutoff=R, spacing=2.0)
    w = oracle.wolf_sum(P, pos, q, 0.0)
    c = oracle.cutoff_sum(P, pos, q)
    d = pos[:, None, :] - pos[None, :, :]
    d -= 18.0 * np.round(d / 18.0)
    r = np.sqrt((d ** 2).sum(-1))
    inside = (r < R) & ~np.eye(len(q), dtype=bool)
    s0 = (inside * q[None, :]).sum(1)
    s1 = (inside * q[None, :] * r).sum(1)
    phi = c["phi"] - s0 / R + (s1 - R * s0) / R ** 2 - q / R
    np.testing.assert_allclose(w["phi"], phi, rtol=1e-11, atol=1e-12)
    assert w["E"] == pytest.approx(0.5 * float(np.dot(q, phi)), rel=1e-12)


def test_wolf_pair_vanishes_with_its_derivative_at_the_cutoff(oracle):
    """Shifted force: v(R) = 0 and v'(R) = 0, for several alpha; two charges
    just inside and just outside R have the same energy (the self terms) and
    no force; inside, E(r) = -integral_r^R F dr of the oracle's own force."""
    R = 9.0
    for alpha in [0.0, 0.15, 0.3]:
        v, dv = oracle.wolf_pair(alpha, R, R * (1 - 1e-12))
        assert abs(v) < 1e-12 and abs(dv) < 1e-11
        P = oracle.Params(box=(40.0,) * 3, periodic=False, cutoff=R, spacing=2.0)
        q = np.array([0.7, -1.1])
        Es = []
        for r in [R * (1 - 1e-9), R * (1 + 1e-9)]:
            out = oracle.wolf_sum(P, np.array([[10.0, 10.0, 10.0], [10.0 + r, 10.0, 10.0]]), q, alpha)
            Es.append(out["E"])
            assert np.abs(out["F"]).max() < 1e-9
        self_e = -oracle.wolf_self_coefficient(alpha, R) * float((q ** 2).sum())
        assert Es[0] == pytest.approx(self_e, rel=1e-9) and Es[1] == pytest.approx(self_e, rel=1e-12)
        # energy at r = 3 from the force integrated (Simpson) from r to R
        s = np.linspace(3.0, R, 2001)
        fx = [oracle.wolf_sum(P, np.array([[10.0, 10.0, 10.0], [10.0 + x, 10.0, 10.0]]), q, alpha)["F"][1, 0]
              for x in s]
        h = s[1] - s[0]
        integral = h / 3 * (fx[0] + fx[-1] + 4 * sum(fx[1:-1:2]) + 2 * sum(fx[2:-1:2]))
        E3 = oracle.wolf_sum(P, np.array([[10.0, 10.0, 10.0], [13.0, 10.0, 10.0]]), q, alpha)["E"]
        assert E3 - self_e == pytest.approx(integral, rel=1e-9)


def test_wolf_sum_gradients_and_accuracy_against_ewald(oracle):
    """Central finite differences give F = -dE/dr and phi = dE/dq (step 1e-5 A;
    a pair within the step of R limits the difference to O(step) there); on a neutral
    periodic water box (alpha = 0.2/A, R = 11 A) the energy is within 1 % and
    the forces within 5 % rel-RMS of the Ewald sum (the method's own accuracy
    on a disordered system)."""
    pos, q = make_water_box(24.0, 450, 3, 3, seed=5, periodic=True)
    P = oracle.Params(box=(24.0,) * 3, periodic=True, cutoff=11.0, spacing=2.0)
    ref = oracle.wolf_sum(P, pos, q, 0.2)
    rng = np.random.default_rng(82)
    h = 1e-5
    for i in rng.choice(len(q), 6, replace=False):
        for c in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, c] += h
            pm[i, c] -= h
            fd = -(oracle.wolf_sum(P, pp, q, 0.2)["E"] - oracle.wolf_sum(P, pm, q, 0.2)["E"]) / (2 * h)
            # v is C1 at R (v'' jumps there): a pair within h of R costs O(h) in the difference
            assert fd == pytest.approx(ref["F"][i, c], rel=1e-6, abs=1e-7)
        qp, qm = q.copy(), q.copy()
        qp[i] += h
        qm[i] -= h
        fd = (oracle.wolf_sum(P, pos, qp, 0.2)["E"] - oracle.wolf_sum(P, pos, qm, 0.2)["E"]) / (2 * h)
        assert fd == pytest.approx(ref["phi"][i], rel=1e-7, abs=1e-9)
    ew = oracle.ewald_sum((24.0,) * 3, pos, q)
    assert ref["E"] == pytest.approx(ew["E"], rel=1e-2)
    assert rel_rms(ref["F"], ew["F"]) < 0.05
