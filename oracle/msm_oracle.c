/*
 * msm_oracle.c -- plain, slow FP64 CPU oracle for one multilevel-summation
 * (MSM) energy-and-force evaluation of Coulomb electrostatics.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant generator
 * with the CUDA library.
 *
 * Every function follows one passage of the thesis proposal "Large-Scale
 * Molecular Dynamics Simulations for Highly Parallel Infrastructures"
 * (Pazurikova, 2014), Sec. "Multilevel Summation Method":
 *   - kernel splitting, Eqs. split / msmgrid (the g*, g^k, g^{l-1} kernels);
 *   - the Taylor smoothing gamma (the printed C2 member, and its C1/C3
 *     siblings from the same Taylor series);
 *   - the nodal basis phi^k_mu = Phi(x)Phi(y)Phi(z) with grid spacing 2^k h;
 *   - the six-step long-range algorithm (anterpolation, restriction, lattice
 *     cutoff, top level, prolongation, interpolation) and the short-range part
 *     u_short = sum_j g*(r_i, r_j) q_j;
 *   - forces F_i = -dU/dr_i (Sec. "Simulation loop").
 * The readings taken where the text is silent (grid geometry, periodic top
 * level, self term, the quintic basis) are stated at each function.
 *
 * Everything is double precision and written as the plain definition: loops
 * over the support of each basis function or kernel, no blocking, no fusion.
 * OpenMP only splits loops over independent outputs.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXLEV 16

/* Parameters of one MSM evaluation (same meaning as the method's symbols). */
typedef struct {
  double box[3];    /* L_x, L_y, L_z (Angstrom); atoms live in [0, L) */
  int periodic;     /* 1: periodic in x, y, z; 0: open boundaries */
  double cutoff;    /* a: short-range cutoff of g* */
  double spacing;   /* h: requested finest spacing (periodic: upper bound) */
  int levels;       /* l: number of grids; 0 chooses automatically */
  int order;        /* p: 3 (cubic) or 5 (quintic) interpolation */
  int split;        /* m: Taylor smoothing order (1, 2 or 3); paper prints m=2 */
} orc_params;

/* Grid geometry of all levels. Level k has spacing 2^k h[d]; its points have
 * absolute indices lo[k][d] .. lo[k][d]+n[k][d]-1 and sit at x = index*2^k h. */
typedef struct {
  int levels;
  double h[3];
  int lo[ORC_MAXLEV][3];
  int n[ORC_MAXLEV][3];
} orc_geom;

/* ------------------------------------------------------------------------ */
/* Smoothing function gamma (Sec. MSM, the printed Taylor smoothing).        */
/* For rho >= 1, gamma = 1/rho.  For rho < 1 it is the Taylor polynomial of  */
/* s^(-1/2) about s = 1 in s = rho^2, truncated after the (s-1)^m term.  The */
/* paper prints m = 2: 15/8 - 5/4 rho^2 + 3/8 rho^4.                         */
/* ------------------------------------------------------------------------ */
static double taylor_coef(int j) {
  /* binomial(-1/2, j) = prod_{i<j} (-1/2 - i) / j! */
  double c = 1.0;
  for (int i = 0; i < j; ++i) c *= (-0.5 - i) / (double)(i + 1);
  return c;
}

double orc_gamma(int m, double rho) {
  if (rho >= 1.0) return 1.0 / rho;
  double x = rho * rho - 1.0, sum = 0.0, xp = 1.0;
  for (int j = 0; j <= m; ++j) {
    sum += taylor_coef(j) * xp;
    xp *= x;
  }
  return sum;
}

double orc_dgamma(int m, double rho) {
  if (rho >= 1.0) return -1.0 / (rho * rho);
  double x = rho * rho - 1.0, sum = 0.0, xp = 1.0;
  for (int j = 1; j <= m; ++j) {
    sum += taylor_coef(j) * j * xp; /* d/ds of (s-1)^j */
    xp *= x;
  }
  return sum * 2.0 * rho;           /* ds/drho = 2 rho */
}

/* The kernels of Eq. msmgrid, as functions of the distance r. */
double orc_gstar(int m, double a, double r) { /* 1/r - gamma(r/a)/a */
  if (r >= a) return 0.0;                      /* both parts equal 1/r */
  return 1.0 / r - orc_gamma(m, r / a) / a;
}
double orc_dgstar(int m, double a, double r) { /* derivative of g* in r */
  if (r >= a) return 0.0;
  return -1.0 / (r * r) - orc_dgamma(m, r / a) / (a * a);
}
double orc_glevel(int m, double a, int k, double r) { /* g^k, k <= l-2 */
  double ak = ldexp(a, k), ak1 = ldexp(a, k + 1);
  if (r >= ak1) return 0.0;                     /* both parts equal 1/r */
  return orc_gamma(m, r / ak) / ak - orc_gamma(m, r / ak1) / ak1;
}
double orc_gtop(int m, double a, int k, double r) { /* g^{l-1} with k = l-1 */
  double ak = ldexp(a, k);
  return orc_gamma(m, r / ak) / ak;
}

/* ------------------------------------------------------------------------ */
/* Nodal basis Phi (Sec. MSM: phi^k_mu = Phi((x-x_mu)/2^k h) Phi(..) Phi(..)).*/
/* p = 3: the cubic numerical Hermite (C1) interpolant the paper names.      */
/* p = 5: the C1 quintic of the same family (reading; not printed).          */
/* ------------------------------------------------------------------------ */
double orc_Phi(int p, double x) {
  double t = fabs(x);
  if (p == 3) {
    if (t <= 1.0) return (1.0 - t) * (1.0 + t - 1.5 * t * t);
    if (t <= 2.0) return -0.5 * (t - 1.0) * (2.0 - t) * (2.0 - t);
    return 0.0;
  }
  if (t <= 1.0) return (1.0 - t * t) * (2.0 - t) * (6.0 + 3.0 * t - 5.0 * t * t) / 12.0;
  if (t <= 2.0) return (t - 1.0) * (t - 2.0) * (t - 3.0) * (5.0 * t * t - 9.0 * t - 4.0) / 24.0;
  if (t <= 3.0) return -(t - 1.0) * (t - 2.0) * (t - 3.0) * (t - 3.0) * (t - 4.0) / 24.0;
  return 0.0;
}

double orc_dPhi(int p, double x) { /* dPhi/dx */
  double t = fabs(x), s = (x < 0.0) ? -1.0 : 1.0, d;
  if (p == 3) {
    if (t <= 1.0) d = -5.0 * t + 4.5 * t * t;                     /* of 1 - 5/2 t^2 + 3/2 t^3 */
    else if (t <= 2.0) d = -1.5 * t * t + 5.0 * t - 4.0;           /* of -t^3/2 + 5/2 t^2 - 4t + 2 */
    else d = 0.0;
    return s * d;
  }
  /* quintic: differentiate the products with the product rule */
  if (t <= 1.0) {
    double A = 1.0 - t * t, B = 2.0 - t, C = 6.0 + 3.0 * t - 5.0 * t * t;
    d = (-2.0 * t * B * C - A * C + A * B * (3.0 - 10.0 * t)) / 12.0;
  } else if (t <= 2.0) {
    double f[4] = {t - 1.0, t - 2.0, t - 3.0, 5.0 * t * t - 9.0 * t - 4.0};
    double df[4] = {1.0, 1.0, 1.0, 10.0 * t - 9.0};
    d = 0.0;
    for (int i = 0; i < 4; ++i) {
      double prod = df[i];
      for (int j = 0; j < 4; ++j) if (j != i) prod *= f[j];
      d += prod;
    }
    d /= 24.0;
  } else if (t <= 3.0) {
    double f[5] = {t - 1.0, t - 2.0, t - 3.0, t - 3.0, t - 4.0};
    d = 0.0;
    for (int i = 0; i < 5; ++i) {
      double prod = 1.0;
      for (int j = 0; j < 5; ++j) if (j != i) prod *= f[j];
      d += prod;
    }
    d = -d / 24.0;
  } else {
    d = 0.0;
  }
  return s * d;
}

/* ------------------------------------------------------------------------ */
/* Grid geometry (the paper fixes only "spacing 2^k h"; reading):           */
/*  periodic: M0 = smallest m*2^j >= L/h with m <= 8 (auto levels) or the     */
/*    smallest multiple of 2^(l-1) >= L/h (given l); h_eff = L/M0; level k    */
/*    has M0/2^k points; auto levels halve while every dim is even and the   */
/*    largest dim exceeds 8.                                                 */
/*  open: h_eff = h; level 0 spans indices -(S-1) .. floor(L/h)+S with       */
/*    S = (p+1)/2; level k+1 spans every coarse point whose basis function   */
/*    touches a level-k point; auto levels stop once the largest dim is <= 8 */
/*    or stops shrinking.                                                    */
/* ------------------------------------------------------------------------ */
static int floordiv(int a, int b) { return (a >= 0) ? a / b : -((-a + b - 1) / b); }
static int ceildiv(int a, int b) { return -floordiv(-a, b); }

int orc_geometry(const orc_params* P, orc_geom* G) {
  int S = (P->order + 1) / 2;
  memset(G, 0, sizeof(*G));
  if (P->periodic) {
    int M0[3];
    for (int d = 0; d < 3; ++d) {
      double x = P->box[d] / P->spacing;
      long best = -1;
      if (P->levels > 0) {
        long m = 1L << (P->levels - 1);
        best = (long)ceil(x / (double)m - 1e-12) * m;
        if (best < m) best = m;
      } else {
        for (int j = 0; j < 30; ++j)
          for (long m = 1; m <= 8; ++m) {
            long c = m << j;
            if ((double)c >= x - 1e-9 && (best < 0 || c < best)) best = c;
          }
      }
      M0[d] = (int)best;
      G->h[d] = P->box[d] / (double)M0[d];
    }
    int l = P->levels;
    if (l <= 0) {
      int cur[3] = {M0[0], M0[1], M0[2]};
      l = 1;
      for (;;) {
        int mx = cur[0] > cur[1] ? cur[0] : cur[1];
        mx = mx > cur[2] ? mx : cur[2];
        if (mx <= 8 || (cur[0] & 1) || (cur[1] & 1) || (cur[2] & 1)) break;
        for (int d = 0; d < 3; ++d) cur[d] /= 2;
        ++l;
      }
    }
    if (l > ORC_MAXLEV) return -1;
    G->levels = l;
    for (int k = 0; k < l; ++k)
      for (int d = 0; d < 3; ++d) {
        G->lo[k][d] = 0;
        G->n[k][d] = M0[d] >> k;
        if ((G->n[k][d] << k) != M0[d]) return -1;
      }
    return 0;
  }
  for (int d = 0; d < 3; ++d) {
    G->h[d] = P->spacing;
    G->lo[0][d] = -(S - 1);
    G->n[0][d] = (int)floor(P->box[d] / P->spacing) + S - G->lo[0][d] + 1;
  }
  int l = 1;
  for (;;) {
    if (P->levels > 0 && l >= P->levels) break;
    if (l >= ORC_MAXLEV) return -1;
    int nlo[3], nn[3], mx_cur = 0, mx_next = 0;
    for (int d = 0; d < 3; ++d) {
      int lo = G->lo[l - 1][d], hi = lo + G->n[l - 1][d] - 1;
      nlo[d] = ceildiv(lo - (2 * S - 1), 2);
      nn[d] = floordiv(hi + (2 * S - 1), 2) - nlo[d] + 1;
      if (G->n[l - 1][d] > mx_cur) mx_cur = G->n[l - 1][d];
      if (nn[d] > mx_next) mx_next = nn[d];
    }
    if (P->levels <= 0 && (mx_cur <= 8 || mx_next >= mx_cur)) break;
    for (int d = 0; d < 3; ++d) {
      G->lo[l][d] = nlo[d];
      G->n[l][d] = nn[d];
    }
    ++l;
  }
  G->levels = l;
  return 0;
}

static int64_t npts(const orc_geom* G, int k) {
  return (int64_t)G->n[k][0] * G->n[k][1] * G->n[k][2];
}

/* Map an absolute level-k index along dim d to its array slot; -1 if the
 * point is not on the (open) grid.  Periodic grids wrap. */
static int slot(const orc_params* P, const orc_geom* G, int k, int d, int idx) {
  int n = G->n[k][d];
  if (P->periodic) {
    int r = idx % n;
    return r < 0 ? r + n : r;
  }
  int s = idx - G->lo[k][d];
  return (s >= 0 && s < n) ? s : -1;
}

/* Periodic positions are folded into [0, L); open positions must lie in [0, L]. */
static int atom_coord(const orc_params* P, const double* r, double* out) {
  for (int d = 0; d < 3; ++d) {
    double x = r[d], L = P->box[d];
    if (P->periodic) {
      x = fmod(x, L);
      if (x < 0.0) x += L;
      if (x >= L) x -= L;
    } else if (!(x >= 0.0 && x <= L)) {
      return -1;
    }
    out[d] = x;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Anterpolation: q^0_mu = sum_j phi^0_mu(r_j) q_j.                          */
/* Each atom is visited once; the loop covers the 2S points per dimension    */
/* where its basis weights can be nonzero (Phi vanishes elsewhere).          */
/* ------------------------------------------------------------------------ */
int orc_anterpolate(const orc_params* P, const orc_geom* G, int64_t n, const double* pos,
                    const double* q, double* q0) {
  int S = (P->order + 1) / 2, W = 2 * S;
  memset(q0, 0, sizeof(double) * npts(G, 0));
  for (int64_t j = 0; j < n; ++j) {
    double x[3];
    if (atom_coord(P, pos + 3 * j, x)) return -2;
    double w[3][6];
    int s[3][6];
    for (int d = 0; d < 3; ++d) {
      double t = x[d] / G->h[d];
      int base = (int)floor(t) - (S - 1);
      for (int i = 0; i < W; ++i) {
        w[d][i] = orc_Phi(P->order, t - (double)(base + i));
        s[d][i] = slot(P, G, 0, d, base + i);
        if (s[d][i] < 0 && w[d][i] != 0.0) return -3;
      }
    }
    for (int c = 0; c < W; ++c)
      for (int b = 0; b < W; ++b)
        for (int a = 0; a < W; ++a) {
          double wt = w[0][a] * w[1][b] * w[2][c];
          if (wt == 0.0) continue;
          q0[((int64_t)s[2][c] * G->n[0][1] + s[1][b]) * G->n[0][0] + s[0][a]] += wt * q[j];
        }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Restriction: q^{k+1}_mu = sum_nu phi^{k+1}_mu(r^k_nu) q^k_nu.  Level-k     */
/* point nu sits at nu*h_k and coarse point mu at 2*mu*h_k, so the weight is  */
/* prod_d Phi((nu_d - 2 mu_d)/2), nonzero for |nu_d - 2 mu_d| < 2S.          */
/* ------------------------------------------------------------------------ */
int orc_restrict(const orc_params* P, const orc_geom* G, int k, const double* qf, double* qc) {
  int S = (P->order + 1) / 2, R = 2 * S - 1;
  int nc[3] = {G->n[k + 1][0], G->n[k + 1][1], G->n[k + 1][2]};
#pragma omp parallel for collapse(2) schedule(static)
  for (int cz = 0; cz < nc[2]; ++cz)
    for (int cy = 0; cy < nc[1]; ++cy)
      for (int cx = 0; cx < nc[0]; ++cx) {
        int mu[3] = {G->lo[k + 1][0] + cx, G->lo[k + 1][1] + cy, G->lo[k + 1][2] + cz};
        double sum = 0.0;
        for (int dz = -R; dz <= R; ++dz)
          for (int dy = -R; dy <= R; ++dy)
            for (int dx = -R; dx <= R; ++dx) {
              int nu[3] = {2 * mu[0] + dx, 2 * mu[1] + dy, 2 * mu[2] + dz};
              double wt = orc_Phi(P->order, dx / 2.0) * orc_Phi(P->order, dy / 2.0) *
                          orc_Phi(P->order, dz / 2.0);
              if (wt == 0.0) continue;
              int sx = slot(P, G, k, 0, nu[0]), sy = slot(P, G, k, 1, nu[1]),
                  sz = slot(P, G, k, 2, nu[2]);
              if (sx < 0 || sy < 0 || sz < 0) continue; /* open grid: no point there */
              sum += wt * qf[((int64_t)sz * G->n[k][1] + sy) * G->n[k][0] + sx];
            }
        qc[((int64_t)cz * nc[1] + cy) * nc[0] + cx] = sum;
      }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Prolongation: u^k_nu = u^{k,cutoff}_nu + sum_mu phi^{k+1}_mu(r^k_nu)       */
/* u^{k+1}_mu.  Adds into uf, which holds u^{k,cutoff} on entry.             */
/* ------------------------------------------------------------------------ */
int orc_prolongate(const orc_params* P, const orc_geom* G, int k, const double* uc, double* uf) {
  int S = (P->order + 1) / 2, R = 2 * S - 1;
  int nf[3] = {G->n[k][0], G->n[k][1], G->n[k][2]};
  int nc[3] = {G->n[k + 1][0], G->n[k + 1][1], G->n[k + 1][2]};
#pragma omp parallel for collapse(2) schedule(static)
  for (int fz = 0; fz < nf[2]; ++fz)
    for (int fy = 0; fy < nf[1]; ++fy)
      for (int fx = 0; fx < nf[0]; ++fx) {
        int nu[3] = {G->lo[k][0] + fx, G->lo[k][1] + fy, G->lo[k][2] + fz};
        double sum = 0.0;
        /* every coarse mu with |nu - 2 mu| <= R, per dimension */
        for (int mz = floordiv(nu[2] - R + 1, 2); 2 * mz <= nu[2] + R; ++mz)
          for (int my = floordiv(nu[1] - R + 1, 2); 2 * my <= nu[1] + R; ++my)
            for (int mx = floordiv(nu[0] - R + 1, 2); 2 * mx <= nu[0] + R; ++mx) {
              double wt = orc_Phi(P->order, (nu[0] - 2 * mx) / 2.0) *
                          orc_Phi(P->order, (nu[1] - 2 * my) / 2.0) *
                          orc_Phi(P->order, (nu[2] - 2 * mz) / 2.0);
              if (wt == 0.0) continue;
              int sx = slot(P, G, k + 1, 0, mx), sy = slot(P, G, k + 1, 1, my),
                  sz = slot(P, G, k + 1, 2, mz);
              if (sx < 0 || sy < 0 || sz < 0) continue;
              sum += wt * uc[((int64_t)sz * nc[1] + sy) * nc[0] + sx];
            }
        uf[((int64_t)fz * nf[1] + fy) * nf[0] + fx] += sum;
      }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Lattice cutoff on level k <= l-2: u^{k,cutoff}_mu = sum_nu g^k(r_mu, r_nu) */
/* q^k_nu.  g^k vanishes for r >= 2^(k+1) a, so nu runs over the offsets     */
/* inside that radius; periodic grids sum over all images by wrapping.       */
/* ------------------------------------------------------------------------ */
int orc_lattice_cutoff(const orc_params* P, const orc_geom* G, int k, const double* qk,
                       double* uk) {
  double hk[3] = {ldexp(G->h[0], k), ldexp(G->h[1], k), ldexp(G->h[2], k)};
  double rc = ldexp(P->cutoff, k + 1);
  int ext[3];
  for (int d = 0; d < 3; ++d) ext[d] = (int)ceil(rc / hk[d]);
  /* list of offsets with nonzero g^k, evaluated straight from the definition */
  int64_t cap = (int64_t)(2 * ext[0] + 1) * (2 * ext[1] + 1) * (2 * ext[2] + 1);
  int* off = (int*)malloc(sizeof(int) * 3 * cap);
  double* val = (double*)malloc(sizeof(double) * cap);
  int64_t nt = 0;
  for (int dz = -ext[2]; dz <= ext[2]; ++dz)
    for (int dy = -ext[1]; dy <= ext[1]; ++dy)
      for (int dx = -ext[0]; dx <= ext[0]; ++dx) {
        double r = sqrt(pow(dx * hk[0], 2) + pow(dy * hk[1], 2) + pow(dz * hk[2], 2));
        double g = orc_glevel(P->split, P->cutoff, k, r);
        if (g == 0.0) continue;
        off[3 * nt] = dx; off[3 * nt + 1] = dy; off[3 * nt + 2] = dz;
        val[nt++] = g;
      }
  int n0 = G->n[k][0], n1 = G->n[k][1], n2 = G->n[k][2];
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < n2; ++z)
    for (int y = 0; y < n1; ++y)
      for (int x = 0; x < n0; ++x) {
        int mu[3] = {G->lo[k][0] + x, G->lo[k][1] + y, G->lo[k][2] + z};
        double sum = 0.0;
        for (int64_t t = 0; t < nt; ++t) {
          int sx = slot(P, G, k, 0, mu[0] + off[3 * t]);
          int sy = slot(P, G, k, 1, mu[1] + off[3 * t + 1]);
          int sz = slot(P, G, k, 2, mu[2] + off[3 * t + 2]);
          if (sx < 0 || sy < 0 || sz < 0) continue;
          sum += val[t] * qk[((int64_t)sz * n1 + sy) * n0 + sx];
        }
        uk[((int64_t)z * n1 + y) * n0 + x] = sum;
      }
  free(off);
  free(val);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Ewald summation of the periodic Coulomb kernel (textbook, tin-foil        */
/* boundary, uniform neutralising background).  Used as the periodic        */
/* reference and to build the periodic top-level kernel.                    */
/*   psi(r) = sum_m erfc(alpha|r+mL|)/|r+mL|                                 */
/*          + (4 pi/V) sum_{k!=0} exp(-k^2/4alpha^2)/k^2 cos(k.r)            */
/*          - pi/(alpha^2 V)                                                 */
/* orc_ewald_psi_reg returns psi(r) - 1/r, which is finite at r = 0.         */
/* ------------------------------------------------------------------------ */
typedef struct {
  double L[3], alpha, rcut, kcut;
} orc_ewald;

static void ewald_defaults(const double* L, double eps_exp, orc_ewald* E) {
  double Lmin = L[0] < L[1] ? L[0] : L[1];
  Lmin = Lmin < L[2] ? Lmin : L[2];
  for (int d = 0; d < 3; ++d) E->L[d] = L[d];
  E->rcut = 0.5 * Lmin;
  E->alpha = eps_exp / E->rcut;       /* erfc(alpha rcut) ~ exp(-eps_exp^2) */
  E->kcut = 2.0 * E->alpha * eps_exp; /* exp(-k^2/4alpha^2) ~ exp(-eps_exp^2) */
}

double orc_ewald_psi_reg(const double* L, double eps_exp, const double* r) {
  orc_ewald E;
  ewald_defaults(L, eps_exp, &E);
  double V = L[0] * L[1] * L[2], a = E.alpha, sum = 0.0;
  int mr[3];
  for (int d = 0; d < 3; ++d) mr[d] = (int)ceil(E.rcut / L[d]) + 1;
  for (int mz = -mr[2]; mz <= mr[2]; ++mz)
    for (int my = -mr[1]; my <= mr[1]; ++my)
      for (int mx = -mr[0]; mx <= mr[0]; ++mx) {
        double d[3] = {r[0] + mx * L[0], r[1] + my * L[1], r[2] + mz * L[2]};
        double s = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        if (mx == 0 && my == 0 && mz == 0) {
          /* erfc(as)/s - 1/s = -erf(as)/s, limit -2a/sqrt(pi) at s = 0 */
          sum += (s > 0.0) ? -erf(a * s) / s : -2.0 * a / sqrt(M_PI);
        } else if (s < E.rcut) {
          sum += erfc(a * s) / s;
        }
      }
  int kr[3];
  for (int d = 0; d < 3; ++d) kr[d] = (int)ceil(E.kcut * L[d] / (2.0 * M_PI));
  double rec = 0.0;
  for (int nz = -kr[2]; nz <= kr[2]; ++nz)
    for (int ny = -kr[1]; ny <= kr[1]; ++ny)
      for (int nx = -kr[0]; nx <= kr[0]; ++nx) {
        if (nx == 0 && ny == 0 && nz == 0) continue;
        double k[3] = {2.0 * M_PI * nx / L[0], 2.0 * M_PI * ny / L[1], 2.0 * M_PI * nz / L[2]};
        double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        if (k2 > E.kcut * E.kcut) continue;
        rec += exp(-k2 / (4.0 * a * a)) / k2 * cos(k[0] * r[0] + k[1] * r[1] + k[2] * r[2]);
      }
  return sum + 4.0 * M_PI / V * rec - M_PI / (a * a * V);
}

/* Ewald energy, per-atom potential and forces of point charges.  Returns E;
 * phi[i] = dE/dq_i, F[i] = -dE/dr_i.  eps_exp sets the accuracy. */
double orc_ewald_sum(const double* L, double eps_exp, int64_t n, const double* pos,
                     const double* q, double* phi, double* F) {
  orc_ewald E;
  ewald_defaults(L, eps_exp, &E);
  double V = L[0] * L[1] * L[2], a = E.alpha, Q = 0.0;
  for (int64_t i = 0; i < n; ++i) Q += q[i];
  int mr[3], kr[3];
  for (int d = 0; d < 3; ++d) {
    /* with rcut <= L/2 only the minimum image can lie inside rcut */
    mr[d] = (E.rcut <= 0.5 * L[d]) ? 0 : (int)ceil(E.rcut / L[d]) + 1;
    kr[d] = (int)ceil(E.kcut * L[d] / (2.0 * M_PI));
  }
  /* real space */
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < n; ++i) {
    double p = 0.0, f[3] = {0.0, 0.0, 0.0};
    for (int64_t j = 0; j < n; ++j) {
      double base[3];
      for (int d = 0; d < 3; ++d) {
        double dd = pos[3 * i + d] - pos[3 * j + d];
        base[d] = dd - L[d] * floor(dd / L[d] + 0.5); /* minimum image */
      }
      for (int mz = -mr[2]; mz <= mr[2]; ++mz)
        for (int my = -mr[1]; my <= mr[1]; ++my)
          for (int mx = -mr[0]; mx <= mr[0]; ++mx) {
            if (i == j && mx == 0 && my == 0 && mz == 0) continue;
            double d[3] = {base[0] + mx * L[0], base[1] + my * L[1], base[2] + mz * L[2]};
            double s = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            if (s >= E.rcut) continue;
            double e = erfc(a * s) / s;
            p += q[j] * e;
            double fr = q[j] * (e + 2.0 * a / sqrt(M_PI) * exp(-a * a * s * s)) / (s * s);
            for (int c = 0; c < 3; ++c) f[c] += fr * d[c];
          }
    }
    phi[i] = p - 2.0 * a / sqrt(M_PI) * q[i] - M_PI * Q / (a * a * V);
    for (int c = 0; c < 3; ++c) F[3 * i + c] = q[i] * f[c];
  }
  /* reciprocal space, k and -k together (half space nz>0 | (nz=0, ny>0) | ...) */
  int nkx = 2 * kr[0] + 1, nky = 2 * kr[1] + 1, nkz = 2 * kr[2] + 1;
  int64_t nk = (int64_t)nkx * nky * nkz;
  double* rec_phi = (double*)calloc((size_t)n, sizeof(double));
  double* rec_f = (double*)calloc((size_t)3 * n, sizeof(double));
  for (int64_t t = 0; t < nk; ++t) {
    int nx = (int)(t % nkx) - kr[0], ny = (int)((t / nkx) % nky) - kr[1],
        nz = (int)(t / ((int64_t)nkx * nky)) - kr[2];
    if (!(nz > 0 || (nz == 0 && ny > 0) || (nz == 0 && ny == 0 && nx > 0))) continue;
    double k[3] = {2.0 * M_PI * nx / L[0], 2.0 * M_PI * ny / L[1], 2.0 * M_PI * nz / L[2]};
    double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    if (k2 > E.kcut * E.kcut) continue;
    double pref = 2.0 * 4.0 * M_PI / V * exp(-k2 / (4.0 * a * a)) / k2; /* x2 for -k */
    double C = 0.0, Sn = 0.0;
#pragma omp parallel for reduction(+ : C, Sn) schedule(static)
    for (int64_t j = 0; j < n; ++j) {
      double kr_ = k[0] * pos[3 * j] + k[1] * pos[3 * j + 1] + k[2] * pos[3 * j + 2];
      C += q[j] * cos(kr_);
      Sn += q[j] * sin(kr_);
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      double kr_ = k[0] * pos[3 * i] + k[1] * pos[3 * i + 1] + k[2] * pos[3 * i + 2];
      double c = cos(kr_), s = sin(kr_);
      rec_phi[i] += pref * (c * C + s * Sn);
      double fm = pref * q[i] * (s * C - c * Sn);
      for (int d = 0; d < 3; ++d) rec_f[3 * i + d] += fm * k[d];
    }
  }
  double En = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    phi[i] += rec_phi[i];
    for (int d = 0; d < 3; ++d) F[3 * i + d] += rec_f[3 * i + d];
    En += 0.5 * q[i] * phi[i];
  }
  free(rec_phi);
  free(rec_f);
  return En;
}

/* ------------------------------------------------------------------------ */
/* Top level: u^{l-1}_mu = sum_nu g^{l-1}(r_mu, r_nu) q^{l-1}_nu, all pairs. */
/* Open boundaries: g^{l-1} itself.  Periodic (reading): the sum over nu     */
/* runs over all periodic images, and the conditionally convergent image sum */
/* of g^{l-1} is taken as the Ewald kernel minus the image sum of the        */
/* compactly supported remainder s = 1/r - g^{l-1} (support r < 2^(l-1) a):  */
/*   K(r) = [psi(r) - 1/r] + g^{l-1}(r) - sum_{m != 0} s(|r + mL|).          */
/* With this kernel the periodic MSM approximates the Ewald energy (tin-foil,*/
/* neutralising background) for any net charge.                             */
/* ------------------------------------------------------------------------ */
static double top_remainder(const orc_params* P, int top, double r) {
  double A = ldexp(P->cutoff, top);
  if (r >= A) return 0.0;
  return 1.0 / r - orc_gtop(P->split, P->cutoff, top, r);
}

double orc_top_kernel_periodic(const orc_params* P, const orc_geom* G, const int* n) {
  int top = G->levels - 1;
  double r[3];
  for (int d = 0; d < 3; ++d) {
    int M = G->n[top][d], m = ((n[d] % M) + M) % M;
    if (2 * m > M) m -= M;                      /* minimum-image representative */
    r[d] = m * ldexp(G->h[d], top);
  }
  double rr = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  double K = orc_ewald_psi_reg(P->box, 6.0, r) + orc_gtop(P->split, P->cutoff, top, rr);
  double A = ldexp(P->cutoff, top);
  int mr[3];
  for (int d = 0; d < 3; ++d) mr[d] = (int)ceil(A / P->box[d]) + 1;
  for (int mz = -mr[2]; mz <= mr[2]; ++mz)
    for (int my = -mr[1]; my <= mr[1]; ++my)
      for (int mx = -mr[0]; mx <= mr[0]; ++mx) {
        if (mx == 0 && my == 0 && mz == 0) continue;
        double d[3] = {r[0] + mx * P->box[0], r[1] + my * P->box[1], r[2] + mz * P->box[2]};
        K -= top_remainder(P, top, sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]));
      }
  return K;
}

int orc_top_level(const orc_params* P, const orc_geom* G, const double* qt, double* ut) {
  int top = G->levels - 1;
  int n0 = G->n[top][0], n1 = G->n[top][1], n2 = G->n[top][2];
  int64_t np = (int64_t)n0 * n1 * n2;
  double* Ktab = NULL;
  if (P->periodic) { /* the periodic kernel depends on (mu - nu) mod M only */
    Ktab = (double*)malloc(sizeof(double) * np);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < np; ++t) {
      int n[3] = {(int)(t % n0), (int)((t / n0) % n1), (int)(t / ((int64_t)n0 * n1))};
      Ktab[t] = orc_top_kernel_periodic(P, G, n);
    }
  }
  double ht[3] = {ldexp(G->h[0], top), ldexp(G->h[1], top), ldexp(G->h[2], top)};
#pragma omp parallel for schedule(static)
  for (int64_t m = 0; m < np; ++m) {
    int mu[3] = {(int)(m % n0), (int)((m / n0) % n1), (int)(m / ((int64_t)n0 * n1))};
    double sum = 0.0;
    for (int64_t v = 0; v < np; ++v) {
      int nu[3] = {(int)(v % n0), (int)((v / n0) % n1), (int)(v / ((int64_t)n0 * n1))};
      double K;
      if (P->periodic) {
        int dn[3];
        for (int d = 0; d < 3; ++d) {
          int M = G->n[top][d];
          dn[d] = ((mu[d] - nu[d]) % M + M) % M;
        }
        K = Ktab[((int64_t)dn[2] * n1 + dn[1]) * n0 + dn[0]];
      } else {
        double r = sqrt(pow((mu[0] - nu[0]) * ht[0], 2) + pow((mu[1] - nu[1]) * ht[1], 2) +
                        pow((mu[2] - nu[2]) * ht[2], 2));
        K = orc_gtop(P->split, P->cutoff, top, r);
      }
      sum += K * qt[v];
    }
    ut[m] = sum;
  }
  free(Ktab);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Interpolation: u_i^long = sum_mu phi^0_mu(r_i) u^0_mu, and its gradient   */
/* sum_mu grad phi^0_mu(r_i) u^0_mu (for the forces).                        */
/* targets == NULL evaluates all n atoms; else the listed atom indices.      */
/* ------------------------------------------------------------------------ */
int orc_interpolate(const orc_params* P, const orc_geom* G, int64_t n, const double* pos,
                    const double* u0, int64_t nt, const int64_t* targets, double* phi,
                    double* grad) {
  int S = (P->order + 1) / 2, W = 2 * S, bad = 0;
  int64_t cnt = targets ? nt : n;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (int64_t t = 0; t < cnt; ++t) {
    int64_t i = targets ? targets[t] : t;
    double x[3];
    if (atom_coord(P, pos + 3 * i, x)) { bad |= 1; continue; }
    double w[3][6], dw[3][6];
    int s[3][6];
    for (int d = 0; d < 3; ++d) {
      double tt = x[d] / G->h[d];
      int base = (int)floor(tt) - (S - 1);
      for (int a = 0; a < W; ++a) {
        w[d][a] = orc_Phi(P->order, tt - (base + a));
        dw[d][a] = orc_dPhi(P->order, tt - (base + a)) / G->h[d];
        s[d][a] = slot(P, G, 0, d, base + a);
        if (s[d][a] < 0) { w[d][a] = 0.0; dw[d][a] = 0.0; s[d][a] = 0; }
      }
    }
    double p = 0.0, g[3] = {0.0, 0.0, 0.0};
    for (int c = 0; c < W; ++c)
      for (int b = 0; b < W; ++b)
        for (int a = 0; a < W; ++a) {
          double u = u0[((int64_t)s[2][c] * G->n[0][1] + s[1][b]) * G->n[0][0] + s[0][a]];
          p += w[0][a] * w[1][b] * w[2][c] * u;
          g[0] += dw[0][a] * w[1][b] * w[2][c] * u;
          g[1] += w[0][a] * dw[1][b] * w[2][c] * u;
          g[2] += w[0][a] * w[1][b] * dw[2][c] * u;
        }
    phi[t] = p;
    for (int d = 0; d < 3; ++d) grad[3 * t + d] = g[d];
  }
  return bad ? -2 : 0;
}

/* ------------------------------------------------------------------------ */
/* Short-range part: u_i^short = sum_{j != i} g*(|r_i - r_j|) q_j, nonzero   */
/* only for r < a, and its force F_i = -q_i grad_i u_i^short.  Periodic      */
/* boxes use the minimum image (requires a <= L/2).                          */
/* orc_short_range_brute checks every j for each target.                     */
/* ------------------------------------------------------------------------ */
static void min_image(const orc_params* P, double* d) {
  if (!P->periodic) return;
  for (int c = 0; c < 3; ++c) d[c] -= P->box[c] * floor(d[c] / P->box[c] + 0.5);
}

int orc_short_range_brute(const orc_params* P, int64_t n, const double* pos, const double* q,
                          int64_t nt, const int64_t* targets, double* phi, double* F) {
  int64_t cnt = targets ? nt : n;
  double a = P->cutoff;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t t = 0; t < cnt; ++t) {
    int64_t i = targets ? targets[t] : t;
    double p = 0.0, f[3] = {0.0, 0.0, 0.0};
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      double d[3] = {pos[3 * i] - pos[3 * j], pos[3 * i + 1] - pos[3 * j + 1],
                     pos[3 * i + 2] - pos[3 * j + 2]};
      min_image(P, d);
      double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      if (r >= a) continue;
      p += q[j] * orc_gstar(P->split, a, r);
      double dg = orc_dgstar(P->split, a, r);
      for (int c = 0; c < 3; ++c) f[c] -= q[i] * q[j] * dg * d[c] / r;
    }
    phi[t] = p;
    for (int c = 0; c < 3; ++c) F[3 * t + c] = f[c];
  }
  return 0;
}

/* Link-cell variant (Sec. "Short-range interactions": atoms are binned into
 * cells no narrower than a and each atom examines its own and the 26
 * neighbouring cells).  Same result as the brute-force form; used for whole
 * systems that are too large for the O(N^2) loop.  Needs >= 3 cells per
 * periodic dimension; callers fall back to the brute-force form otherwise. */
int orc_short_range_cells(const orc_params* P, int64_t n, const double* pos, const double* q,
                          double* phi, double* F) {
  int nc[3];
  double w[3];
  for (int d = 0; d < 3; ++d) {
    nc[d] = (int)floor(P->box[d] / P->cutoff);
    if (nc[d] < 1) nc[d] = 1;
    if (P->periodic && nc[d] < 3) return -1;
    w[d] = P->box[d] / nc[d];
  }
  int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
  int64_t* head = (int64_t*)malloc(sizeof(int64_t) * ncell);
  int64_t* next = (int64_t*)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
  int* cell = (int*)malloc(sizeof(int) * 3 * (n > 0 ? n : 1));
  for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
  for (int64_t j = n - 1; j >= 0; --j) {
    double x[3];
    if (atom_coord(P, pos + 3 * j, x)) { free(head); free(next); free(cell); return -2; }
    for (int d = 0; d < 3; ++d) {
      int c = (int)floor(x[d] / w[d]);
      cell[3 * j + d] = c < 0 ? 0 : (c >= nc[d] ? nc[d] - 1 : c);
    }
    int64_t id = ((int64_t)cell[3 * j + 2] * nc[1] + cell[3 * j + 1]) * nc[0] + cell[3 * j];
    next[j] = head[id];
    head[id] = j;
  }
  double a = P->cutoff;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < n; ++i) {
    double p = 0.0, f[3] = {0.0, 0.0, 0.0};
    for (int oz = -1; oz <= 1; ++oz)
      for (int oy = -1; oy <= 1; ++oy)
        for (int ox = -1; ox <= 1; ++ox) {
          int c[3] = {cell[3 * i] + ox, cell[3 * i + 1] + oy, cell[3 * i + 2] + oz};
          int skip = 0;
          for (int d = 0; d < 3; ++d) {
            if (P->periodic) c[d] = (c[d] + nc[d]) % nc[d];
            else if (c[d] < 0 || c[d] >= nc[d]) skip = 1;
          }
          if (skip) continue;
          for (int64_t j = head[((int64_t)c[2] * nc[1] + c[1]) * nc[0] + c[0]]; j >= 0; j = next[j]) {
            if (j == i) continue;
            double d[3] = {pos[3 * i] - pos[3 * j], pos[3 * i + 1] - pos[3 * j + 1],
                           pos[3 * i + 2] - pos[3 * j + 2]};
            min_image(P, d);
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            if (r >= a) continue;
            p += q[j] * orc_gstar(P->split, a, r);
            double dg = orc_dgstar(P->split, a, r);
            for (int k = 0; k < 3; ++k) f[k] -= q[i] * q[j] * dg * d[k] / r;
          }
        }
    phi[i] = p;
    for (int k = 0; k < 3; ++k) F[3 * i + k] = f[k];
  }
  free(head);
  free(next);
  free(cell);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Direct Coulomb sum with open boundaries (Eq. coulomb, read with the 1/2    */
/* and i != j): phi_i = sum_{j!=i} q_j/r_ij, F_i = q_i sum_j q_j r_ij/r^3,    */
/* E = 1/2 sum_i q_i phi_i.                                                  */
/* ------------------------------------------------------------------------ */
double orc_direct_sum(int64_t n, const double* pos, const double* q, int64_t nt,
                      const int64_t* targets, double* phi, double* F) {
  int64_t cnt = targets ? nt : n;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t t = 0; t < cnt; ++t) {
    int64_t i = targets ? targets[t] : t;
    double p = 0.0, f[3] = {0.0, 0.0, 0.0};
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      double d[3] = {pos[3 * i] - pos[3 * j], pos[3 * i + 1] - pos[3 * j + 1],
                     pos[3 * i + 2] - pos[3 * j + 2]};
      double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      p += q[j] / r;
      for (int c = 0; c < 3; ++c) f[c] += q[i] * q[j] * d[c] / (r * r * r);
    }
    phi[t] = p;
    for (int c = 0; c < 3; ++c) F[3 * t + c] = f[c];
  }
  double E = 0.0;
  if (!targets)
    for (int64_t i = 0; i < n; ++i) E += 0.5 * q[i] * phi[i];
  return E;
}

/* Cutoff method (the simplest coarse propagator G of the parareal section:  */
/* the Coulomb law summed only over atoms within a constant cutoff a, all    */
/* farther pairs neglected): phi_i = sum_{j!=i, r_ij<a} q_j/r_ij, F_i =       */
/* q_i sum_{j!=i, r_ij<a} q_j (r_i - r_j)/r_ij^3 (the gradient inside the     */
/* cutoff), E = 1/2 sum_i q_i phi_i.  Minimum image when periodic (a <= L/2). */
/* Brute force over every pair.                                              */
double orc_cutoff_sum(const orc_params* P, int64_t n, const double* pos, const double* q, int64_t nt,
                      const int64_t* targets, double* phi, double* F) {
  int64_t cnt = targets ? nt : n;
  double a = P->cutoff;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t t = 0; t < cnt; ++t) {
    int64_t i = targets ? targets[t] : t;
    double p = 0.0, f[3] = {0.0, 0.0, 0.0};
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      double d[3] = {pos[3 * i] - pos[3 * j], pos[3 * i + 1] - pos[3 * j + 1],
                     pos[3 * i + 2] - pos[3 * j + 2]};
      min_image(P, d);
      double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      if (r >= a) continue;
      p += q[j] / r;
      for (int c = 0; c < 3; ++c) f[c] += q[i] * q[j] * d[c] / (r * r * r);
    }
    phi[t] = p;
    for (int c = 0; c < 3; ++c) F[3 * t + c] = f[c];
  }
  double E = 0.0;
  if (!targets)
    for (int64_t i = 0; i < n; ++i) E += 0.5 * q[i] * phi[i];
  return E;
}

/* Wolf summation (Wolf, Keblinski, Phillpot and Eggebrecht, J. Chem. Phys. */
/* 110, 8254 (1999)), one of the coarse functions G the proposal lists for   */
/* the parareal method (Sec. "Proposed Solutions"; the thesis gives no       */
/* formula).  Reading taken: the damped, shifted-force form, whose pair      */
/* potential and its derivative both vanish at the cutoff R = P->cutoff (the */
/* force-shifted variant of Fennell and Gezelter, J. Chem. Phys. 124, 234104 */
/* (2006)), so that the forces are the exact gradient of the energy:         */
/*   v(r) = erfc(alpha r)/r - erfc(alpha R)/R + c1 (r - R),  r < R,          */
/*   c1   = erfc(alpha R)/R^2 + (2 alpha/sqrt(pi)) exp(-alpha^2 R^2)/R,      */
/*   E    = 1/2 sum_i sum_{j != i, r_ij < R} q_i q_j v(r_ij) - c_s sum q_i^2, */
/*   c_s  = erfc(alpha R)/(2R) + alpha/sqrt(pi)   (charge-neutralising shell  */
/*          and damping self terms of Wolf's sum),                            */
/*   phi_i = dE/dq_i = sum_j q_j v(r_ij) - 2 c_s q_i,  E = 1/2 sum q_i phi_i, */
/*   F_i  = -dE/dr_i = -q_i sum_j q_j v'(r_ij) (r_i - r_j)/r_ij.             */
/* alpha = 0 is the shifted-force Coulomb cutoff.  Minimum image when        */
/* periodic (R <= L/2).  Brute force over every pair; erfc from the C         */
/* library.                                                                  */
double orc_wolf_self_coefficient(double alpha, double R) { return erfc(alpha * R) / (2.0 * R) + alpha / sqrt(M_PI); }

double orc_wolf_pair(double alpha, double R, double r, double* dvdr) {
  const double two_a_sqrtpi = 2.0 * alpha / sqrt(M_PI);
  const double c1 = erfc(alpha * R) / (R * R) + two_a_sqrtpi * exp(-alpha * alpha * R * R) / R;
  if (dvdr) *dvdr = (r < R) ? -erfc(alpha * r) / (r * r) - two_a_sqrtpi * exp(-alpha * alpha * r * r) / r + c1 : 0.0;
  if (r >= R) return 0.0;
  return erfc(alpha * r) / r - erfc(alpha * R) / R + c1 * (r - R);
}

double orc_wolf_sum(const orc_params* P, double alpha, int64_t n, const double* pos, const double* q, int64_t nt,
                    const int64_t* targets, double* phi, double* F) {
  int64_t cnt = targets ? nt : n;
  const double R = P->cutoff, cs = orc_wolf_self_coefficient(alpha, R);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t t = 0; t < cnt; ++t) {
    int64_t i = targets ? targets[t] : t;
    double p = 0.0, f[3] = {0.0, 0.0, 0.0};
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      double d[3] = {pos[3 * i] - pos[3 * j], pos[3 * i + 1] - pos[3 * j + 1],
                     pos[3 * i + 2] - pos[3 * j + 2]};
      min_image(P, d);
      double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      if (r >= R) continue;
      double dv = 0.0;
      p += q[j] * orc_wolf_pair(alpha, R, r, &dv);
      for (int c = 0; c < 3; ++c) f[c] -= q[i] * q[j] * dv * d[c] / r;
    }
    phi[t] = p - 2.0 * cs * q[i];
    for (int c = 0; c < 3; ++c) F[3 * t + c] = f[c];
  }
  double E = 0.0;
  if (!targets)
    for (int64_t i = 0; i < n; ++i) E += 0.5 * q[i] * phi[i];
  return E;
}

/* Self term (reading): the grid part of u_i contains atom i's own charge     */
/* through the smooth kernel, whose value at r = 0 is gamma(0)/a; that       */
/* constant is removed from phi_i.  Exposed for the assembly step.           */
double orc_self_coefficient(const orc_params* P) { return orc_gamma(P->split, 0.0) / P->cutoff; }
