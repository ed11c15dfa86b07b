"""FP64 CPU oracle of one multilevel-summation (MSM) energy+force evaluation.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the CUDA library
never does, and the two share no code.

The arithmetic lives in ``msm_oracle.c`` (plain loops, double precision); this
module marshals numpy arrays into it and composes the steps of the long-range
algorithm in the order the thesis proposal lists them (Sec. "Multilevel
Summation Method"): anterpolation, then restriction and lattice cutoff for
k = 0..l-2, the top level, prolongation for k = l-2..0, interpolation; the
short-range part u_short = sum_j g*(r_i, r_j) q_j is added, and
U_i = k_c (u_short + u_long) with forces F_i = -dU/dr_i.
"""
import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

MAXLEV = 16


class _Params(C.Structure):
    _fields_ = [("box", C.c_double * 3), ("periodic", C.c_int), ("cutoff", C.c_double),
                ("spacing", C.c_double), ("levels", C.c_int), ("order", C.c_int),
                ("split", C.c_int)]


class _Geom(C.Structure):
    _fields_ = [("levels", C.c_int), ("h", C.c_double * 3),
                ("lo", (C.c_int * 3) * MAXLEV), ("n", (C.c_int * 3) * MAXLEV)]


@dataclass
class Params:
    """MSM parameters: box edges L (A), periodicity, cutoff a, spacing h,
    levels l (0 = automatic), order p (3 cubic / 5 quintic), Taylor smoothing
    order m (paper prints m = 2), Coulomb prefactor k_c."""
    box: tuple
    periodic: bool
    cutoff: float
    spacing: float
    levels: int = 0
    order: int = 3
    split: int = 2
    coulomb_k: float = 1.0

    def _c(self):
        p = _Params()
        for d in range(3):
            p.box[d] = float(self.box[d])
        p.periodic = int(bool(self.periodic))
        p.cutoff = float(self.cutoff)
        p.spacing = float(self.spacing)
        p.levels = int(self.levels)
        p.order = int(self.order)
        p.split = int(self.split)
        return p


_lib = None
_D = C.POINTER(C.c_double)
_I64 = C.POINTER(C.c_int64)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P, G = C.POINTER(_Params), C.POINTER(_Geom)
        sig = {
            "orc_gamma": (C.c_double, [C.c_int, C.c_double]),
            "orc_dgamma": (C.c_double, [C.c_int, C.c_double]),
            "orc_gstar": (C.c_double, [C.c_int, C.c_double, C.c_double]),
            "orc_dgstar": (C.c_double, [C.c_int, C.c_double, C.c_double]),
            "orc_glevel": (C.c_double, [C.c_int, C.c_double, C.c_int, C.c_double]),
            "orc_gtop": (C.c_double, [C.c_int, C.c_double, C.c_int, C.c_double]),
            "orc_Phi": (C.c_double, [C.c_int, C.c_double]),
            "orc_dPhi": (C.c_double, [C.c_int, C.c_double]),
            "orc_geometry": (C.c_int, [P, G]),
            "orc_anterpolate": (C.c_int, [P, G, C.c_int64, _D, _D, _D]),
            "orc_restrict": (C.c_int, [P, G, C.c_int, _D, _D]),
            "orc_prolongate": (C.c_int, [P, G, C.c_int, _D, _D]),
            "orc_lattice_cutoff": (C.c_int, [P, G, C.c_int, _D, _D]),
            "orc_top_level": (C.c_int, [P, G, _D, _D]),
            "orc_top_kernel_periodic": (C.c_double, [P, G, C.POINTER(C.c_int)]),
            "orc_interpolate": (C.c_int, [P, G, C.c_int64, _D, _D, C.c_int64, _I64, _D, _D]),
            "orc_short_range_brute": (C.c_int, [P, C.c_int64, _D, _D, C.c_int64, _I64, _D, _D]),
            "orc_short_range_cells": (C.c_int, [P, C.c_int64, _D, _D, _D, _D]),
            "orc_direct_sum": (C.c_double, [C.c_int64, _D, _D, C.c_int64, _I64, _D, _D]),
            "orc_cutoff_sum": (C.c_double, [P, C.c_int64, _D, _D, C.c_int64, _I64, _D, _D]),
            "orc_wolf_sum": (C.c_double, [P, C.c_double, C.c_int64, _D, _D, C.c_int64, _I64, _D, _D]),
            "orc_wolf_pair": (C.c_double, [C.c_double, C.c_double, C.c_double, _D]),
            "orc_wolf_self_coefficient": (C.c_double, [C.c_double, C.c_double]),
            "orc_ewald_sum": (C.c_double, [_D, C.c_double, C.c_int64, _D, _D, _D, _D]),
            "orc_ewald_psi_reg": (C.c_double, [_D, C.c_double, _D]),
            "orc_self_coefficient": (C.c_double, [P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_D)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


# -- scalar functions (Eq. msmgrid kernels, gamma, Phi) ----------------------
def gamma(m, rho):
    return lib().orc_gamma(int(m), float(rho))


def dgamma(m, rho):
    return lib().orc_dgamma(int(m), float(rho))


def gstar(m, a, r):
    return lib().orc_gstar(int(m), float(a), float(r))


def dgstar(m, a, r):
    return lib().orc_dgstar(int(m), float(a), float(r))


def glevel(m, a, k, r):
    return lib().orc_glevel(int(m), float(a), int(k), float(r))


def gtop(m, a, k, r):
    return lib().orc_gtop(int(m), float(a), int(k), float(r))


def Phi(p, x):
    return lib().orc_Phi(int(p), float(x))


def dPhi(p, x):
    return lib().orc_dPhi(int(p), float(x))


# -- geometry ----------------------------------------------------------------
@dataclass
class Geometry:
    levels: int
    h: tuple
    lo: list   # per level, 3 ints
    n: list    # per level, 3 ints (x fastest in memory: arrays are [nz, ny, nx])

    def shape(self, k):
        return (self.n[k][2], self.n[k][1], self.n[k][0])


def geometry(P: Params) -> Geometry:
    g = _Geom()
    rc = lib().orc_geometry(C.byref(P._c()), C.byref(g))
    if rc != 0:
        raise ValueError("oracle: unsupported grid geometry")
    return Geometry(g.levels, tuple(g.h), [tuple(g.lo[k]) for k in range(g.levels)],
                    [tuple(g.n[k]) for k in range(g.levels)])


def _cgeom(G: Geometry):
    g = _Geom()
    g.levels = G.levels
    for d in range(3):
        g.h[d] = G.h[d]
    for k in range(G.levels):
        for d in range(3):
            g.lo[k][d] = G.lo[k][d]
            g.n[k][d] = G.n[k][d]
    return g


# -- the steps of the long-range part, in the paper's order -----------------
def anterpolate(P, G, pos, q):
    pos, q = _f64(pos, (-1, 3)), _f64(q)
    q0 = np.zeros(G.shape(0))
    rc = lib().orc_anterpolate(C.byref(P._c()), C.byref(_cgeom(G)), len(q), _dp(pos), _dp(q), _dp(q0))
    if rc:
        raise ValueError("oracle: atom outside the open box")
    return q0


def restrict(P, G, k, qk):
    qk = _f64(qk)
    out = np.zeros(G.shape(k + 1))
    lib().orc_restrict(C.byref(P._c()), C.byref(_cgeom(G)), k, _dp(qk), _dp(out))
    return out


def lattice_cutoff(P, G, k, qk):
    qk = _f64(qk)
    out = np.zeros(G.shape(k))
    lib().orc_lattice_cutoff(C.byref(P._c()), C.byref(_cgeom(G)), k, _dp(qk), _dp(out))
    return out


def top_level(P, G, qt):
    qt = _f64(qt)
    out = np.zeros(G.shape(G.levels - 1))
    lib().orc_top_level(C.byref(P._c()), C.byref(_cgeom(G)), _dp(qt), _dp(out))
    return out


def top_kernel_periodic(P, G, n):
    arr = (C.c_int * 3)(*[int(v) for v in n])
    return lib().orc_top_kernel_periodic(C.byref(P._c()), C.byref(_cgeom(G)), arr)


def prolongate(P, G, k, u_coarse, u_cut):
    """Returns u^k = u^{k,cutoff} + sum_mu phi^{k+1}_mu(r^k_nu) u^{k+1}_mu."""
    uc = _f64(u_coarse)
    uf = np.array(u_cut, dtype=np.float64, copy=True)
    lib().orc_prolongate(C.byref(P._c()), C.byref(_cgeom(G)), k, _dp(uc), _dp(uf))
    return uf


def _targets(targets):
    if targets is None:
        return None, 0, None
    t = np.ascontiguousarray(targets, dtype=np.int64)
    return t, len(t), t.ctypes.data_as(_I64)


def interpolate(P, G, pos, u0, targets=None):
    pos, u0 = _f64(pos, (-1, 3)), _f64(u0)
    t, nt, tp = _targets(targets)
    cnt = nt if t is not None else len(pos)
    phi, grad = np.zeros(cnt), np.zeros((cnt, 3))
    rc = lib().orc_interpolate(C.byref(P._c()), C.byref(_cgeom(G)), len(pos), _dp(pos), _dp(u0),
                               nt, tp, _dp(phi), _dp(grad))
    if rc:
        raise ValueError("oracle: atom outside the open box")
    return phi, grad


def short_range(P, pos, q, targets=None, method="auto"):
    """u_short and the short-range force F_short = -q_i grad u_short."""
    pos, q = _f64(pos, (-1, 3)), _f64(q)
    n = len(q)
    if method == "auto":
        method = "cells" if (targets is None and n > 20000) else "brute"
    if method == "cells" and targets is None:
        phi, F = np.zeros(n), np.zeros((n, 3))
        rc = lib().orc_short_range_cells(C.byref(P._c()), n, _dp(pos), _dp(q), _dp(phi), _dp(F))
        if rc == 0:
            return phi, F
    t, nt, tp = _targets(targets)
    cnt = nt if t is not None else n
    phi, F = np.zeros(cnt), np.zeros((cnt, 3))
    lib().orc_short_range_brute(C.byref(P._c()), n, _dp(pos), _dp(q), nt, tp, _dp(phi), _dp(F))
    return phi, F


def self_coefficient(P):
    return lib().orc_self_coefficient(C.byref(P._c()))


def msm(P: Params, pos, q, targets=None, keep_grids=False, short_method="auto"):
    """One MSM evaluation (Sec. "Multilevel Summation Method").

    Returns a dict with phi (dE/dq_i) and F (-dE/dr_i) for all atoms or for
    the listed targets, E = 1/2 sum q_i phi_i (whole systems only), and the
    short/long parts.  Reading of the self term: the constant q_i gamma(0)/a
    (the smooth kernel at r = 0) is removed from phi_i.
    """
    pos, q = _f64(pos, (-1, 3)), _f64(q)
    G = geometry(P)
    l = G.levels
    # anterpolation
    qg = [anterpolate(P, G, pos, q)]
    ucut = []
    # restriction and lattice cutoff, k = 0..l-2
    for k in range(l - 1):
        qg.append(restrict(P, G, k, qg[k]))
        ucut.append(lattice_cutoff(P, G, k, qg[k]))
    # top level
    ug = [None] * l
    ug[l - 1] = top_level(P, G, qg[l - 1])
    # prolongation, k = l-2..0
    for k in range(l - 2, -1, -1):
        ug[k] = prolongate(P, G, k, ug[k + 1], ucut[k])
    # interpolation
    phi_long, grad_long = interpolate(P, G, pos, ug[0], targets)
    # short range
    phi_s, F_s = short_range(P, pos, q, targets, short_method)
    qt = q if targets is None else q[np.asarray(targets)]
    phi = phi_s + phi_long - qt * self_coefficient(P)
    F = F_s - qt[:, None] * grad_long
    kc = P.coulomb_k
    out = {"phi": kc * phi, "F": kc * F, "phi_short": kc * phi_s, "F_short": kc * F_s,
           "phi_long": kc * phi_long, "F_long": -kc * qt[:, None] * grad_long, "geometry": G}
    if targets is None:
        out["E"] = 0.5 * float(np.dot(q, out["phi"]))
    if keep_grids:
        out["q_grids"] = qg
        out["u_cut"] = ucut
        out["u_grids"] = ug
    return out


def direct_sum(pos, q, targets=None, coulomb_k=1.0):
    """Open-boundary Coulomb sum (Eq. coulomb with 1/2 and i != j)."""
    pos, q = _f64(pos, (-1, 3)), _f64(q)
    t, nt, tp = _targets(targets)
    cnt = nt if t is not None else len(q)
    phi, F = np.zeros(cnt), np.zeros((cnt, 3))
    E = lib().orc_direct_sum(len(q), _dp(pos), _dp(q), nt, tp, _dp(phi), _dp(F))
    out = {"phi": coulomb_k * phi, "F": coulomb_k * F}
    if t is None:
        out["E"] = coulomb_k * E
    return out


def cutoff_sum(P: Params, pos, q, targets=None):
    """The cutoff method (the parareal section's simplest coarse propagator
    G): the Coulomb law over pairs within the cutoff P.cutoff only (minimum
    image when periodic), E = 1/2 sum q_i phi_i."""
    pos, q = _f64(pos, (-1, 3)), _f64(q)
    t, nt, tp = _targets(targets)
    cnt = nt if t is not None else len(q)
    phi, F = np.zeros(cnt), np.zeros((cnt, 3))
    E = lib().orc_cutoff_sum(C.byref(P._c()), len(q), _dp(pos), _dp(q), nt, tp, _dp(phi), _dp(F))
    kc = P.coulomb_k
    out = {"phi": kc * phi, "F": kc * F}
    if t is None:
        out["E"] = kc * E
    return out


def wolf_sum(P: Params, pos, q, alpha, targets=None):
    """Wolf summation in its damped, shifted-force form (Wolf et al. 1999;
    force-shifted as in Fennell and Gezelter 2006), one of the coarse
    functions of the parareal section: pair potential
    v(r) = erfc(alpha r)/r - erfc(alpha R)/R + c1 (r - R) within R = P.cutoff,
    self term -c_s q_i^2; returns phi = dE/dq, F = -dE/dr and E (no targets)."""
    pos, q = _f64(pos, (-1, 3)), _f64(q)
    t, nt, tp = _targets(targets)
    cnt = nt if t is not None else len(q)
    phi, F = np.zeros(cnt), np.zeros((cnt, 3))
    E = lib().orc_wolf_sum(C.byref(P._c()), float(alpha), len(q), _dp(pos), _dp(q), nt, tp, _dp(phi), _dp(F))
    kc = P.coulomb_k
    out = {"phi": kc * phi, "F": kc * F}
    if t is None:
        out["E"] = kc * E
    return out


def wolf_pair(alpha, R, r):
    """(v(r), v'(r)) of the Wolf pair potential above."""
    d = C.c_double(0.0)
    v = lib().orc_wolf_pair(float(alpha), float(R), float(r), C.byref(d))
    return v, d.value


def wolf_self_coefficient(alpha, R):
    return lib().orc_wolf_self_coefficient(float(alpha), float(R))


def ewald_sum(box, pos, q, eps_exp=6.0, coulomb_k=1.0):
    """Textbook Ewald sum (tin-foil boundary, neutralising background)."""
    pos, q = _f64(pos, (-1, 3)), _f64(q)
    L = _f64(box)
    phi, F = np.zeros(len(q)), np.zeros((len(q), 3))
    E = lib().orc_ewald_sum(_dp(L), float(eps_exp), len(q), _dp(pos), _dp(q), _dp(phi), _dp(F))
    return {"E": coulomb_k * E, "phi": coulomb_k * phi, "F": coulomb_k * F}


def ewald_psi_reg(box, r, eps_exp=6.0):
    L = _f64(box)
    rr = _f64(r)
    return lib().orc_ewald_psi_reg(_dp(L), float(eps_exp), _dp(rr))
