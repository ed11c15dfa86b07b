// plan.cpp -- host side of an MSM plan: parameter checks, grid geometry,
// short-range cells, the level stencil and the top-level kernel (FP64), and
// the device workspace.
//
// Geometry (the thesis fixes only that level k has spacing 2^k h, Sec.
// "Multilevel Summation Method"):
//   periodic: M0 per dimension is the smallest m * 2^j >= L/h with m <= 8
//     (levels chosen automatically) or the smallest multiple of 2^(l-1) >= L/h
//     (levels given); h_eff = L/M0; level k has M0/2^k points; automatic
//     levels halve while every dimension is even and the largest exceeds 8.
//   open: h_eff = h; level 0 spans indices -(S-1) .. floor(L/h)+S, with
//     S = (p+1)/2 the support half-width of Phi; level k+1 spans every coarse
//     point whose basis function reaches a level-k point; automatic levels
//     stop when the largest dimension is <= 8 or stops shrinking.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "msm_internal.h"

namespace msm {

namespace {

int fdiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }
int cdiv(int a, int b) { return -fdiv(-a, b); }

// Taylor smoothing gamma(rho) (printed C2 member and its C1/C3 siblings), in
// s = rho^2 for rho < 1 and 1/rho beyond.
double smooth(int m, double rho) {
  if (rho >= 1.0) return 1.0 / rho;
  double s = rho * rho;
  switch (m) {
    case 1: return 1.5 - 0.5 * s;
    case 2: return 1.875 + s * (-1.25 + 0.375 * s);
    default: return 2.1875 + s * (-2.1875 + s * (1.3125 - 0.3125 * s));
  }
}

// g^k of Eq. msmgrid for k <= l-2 (compact support r < 2^(k+1) a).
double level_kernel(int m, double a, int k, double r) {
  double ak = std::ldexp(a, k);
  if (r >= 2.0 * ak) return 0.0;
  return smooth(m, r / ak) / ak - smooth(m, r / (2.0 * ak)) / (2.0 * ak);
}

// g^{l-1}: the top-level kernel gamma(r/A)/A with A = 2^(l-1) a.
double top_kernel(int m, double A, double r) { return smooth(m, r / A) / A; }

// Periodic Coulomb kernel minus 1/r (Ewald: tin-foil boundary, uniform
// neutralising background), finite at r = 0.  alpha is chosen so that the
// real-space images within rc = min(L) and the reciprocal vectors with
// |k| < 2 * 5.9 * alpha both converge below 1e-15.
double ewald_minus_coulomb(const double L[3], const double r[3]) {
  double Lmin = std::fmin(L[0], std::fmin(L[1], L[2]));
  const double eta = 5.9;
  double rc = Lmin, alpha = eta / rc, kc = 2.0 * alpha * eta;
  double V = L[0] * L[1] * L[2];
  double real = 0.0;
  int im[3];
  for (int d = 0; d < 3; ++d) im[d] = (int)std::ceil(rc / L[d]) + 1;
  for (int a = -im[0]; a <= im[0]; ++a)
    for (int b = -im[1]; b <= im[1]; ++b)
      for (int c = -im[2]; c <= im[2]; ++c) {
        double x = r[0] + a * L[0], y = r[1] + b * L[1], z = r[2] + c * L[2];
        double s = std::sqrt(x * x + y * y + z * z);
        if (a == 0 && b == 0 && c == 0)
          real += (s == 0.0) ? -2.0 * alpha / std::sqrt(M_PI) : -std::erf(alpha * s) / s;
        else if (s < rc)
          real += std::erfc(alpha * s) / s;
      }
  double recip = 0.0;
  int km[3];
  for (int d = 0; d < 3; ++d) km[d] = (int)std::ceil(kc * L[d] / (2.0 * M_PI));
  for (int a = 0; a <= km[0]; ++a)       // half space a > 0, plus a = 0 planes
    for (int b = -km[1]; b <= km[1]; ++b)
      for (int c = -km[2]; c <= km[2]; ++c) {
        if (a == 0 && (b < 0 || (b == 0 && c <= 0))) continue;
        double kx = 2.0 * M_PI * a / L[0], ky = 2.0 * M_PI * b / L[1], kz = 2.0 * M_PI * c / L[2];
        double k2 = kx * kx + ky * ky + kz * kz;
        if (k2 > kc * kc) continue;
        recip += 2.0 * std::exp(-k2 / (4.0 * alpha * alpha)) / k2 *
                 std::cos(kx * r[0] + ky * r[1] + kz * r[2]);
      }
  return real + 4.0 * M_PI / V * recip - M_PI / (alpha * alpha * V);
}

int geometry(const msm_params& p, Plan* P) {
  int S = P->S;
  if (p.periodic) {
    int M0[3];
    for (int d = 0; d < 3; ++d) {
      double x = p.box[d] / p.spacing;
      long best = -1;
      if (p.levels > 0) {
        long m = 1L << (p.levels - 1);
        long c = (long)std::ceil(x / (double)m - 1e-12);
        best = (c < 1 ? 1 : c) * m;
      } else {
        for (int j = 0; j < 30; ++j)
          for (long m = 1; m <= 8; ++m) {
            long c = m << j;
            if ((double)c >= x - 1e-9 && (best < 0 || c < best)) best = c;
          }
      }
      if (best <= 0 || best > (1L << 20)) return MSM_ERR_UNSUPPORTED;
      M0[d] = (int)best;
      P->h[d] = p.box[d] / (double)M0[d];
    }
    int l = p.levels;
    if (l <= 0) {
      int c[3] = {M0[0], M0[1], M0[2]};
      l = 1;
      while (std::max(c[0], std::max(c[1], c[2])) > 8 && !(c[0] & 1) && !(c[1] & 1) && !(c[2] & 1)) {
        for (int d = 0; d < 3; ++d) c[d] /= 2;
        ++l;
      }
    }
    if (l > kMaxLevels) return MSM_ERR_UNSUPPORTED;
    P->levels = l;
    for (int k = 0; k < l; ++k)
      for (int d = 0; d < 3; ++d) {
        P->lo[k][d] = 0;
        P->n[k][d] = M0[d] >> k;
        if ((P->n[k][d] << k) != M0[d]) return MSM_ERR_UNSUPPORTED;
      }
    return MSM_OK;
  }
  for (int d = 0; d < 3; ++d) {
    P->h[d] = p.spacing;
    P->lo[0][d] = -(S - 1);
    P->n[0][d] = (int)std::floor(p.box[d] / p.spacing) + 2 * S;
  }
  int l = 1;
  for (;;) {
    if (p.levels > 0 && l >= p.levels) break;
    if (l >= kMaxLevels) return MSM_ERR_UNSUPPORTED;
    int nlo[3], nn[3], cur = 0, nxt = 0;
    for (int d = 0; d < 3; ++d) {
      int lo = P->lo[l - 1][d], hi = lo + P->n[l - 1][d] - 1;
      nlo[d] = cdiv(lo - (2 * S - 1), 2);
      nn[d] = fdiv(hi + (2 * S - 1), 2) - nlo[d] + 1;
      cur = std::max(cur, P->n[l - 1][d]);
      nxt = std::max(nxt, nn[d]);
    }
    if (p.levels <= 0 && (cur <= 8 || nxt >= cur)) break;
    for (int d = 0; d < 3; ++d) {
      P->lo[l][d] = nlo[d];
      P->n[l][d] = nn[d];
    }
    ++l;
  }
  P->levels = l;
  return MSM_OK;
}

template <typename T>
cudaError_t upload(void** dst, const std::vector<T>& v) {
  cudaError_t e = cudaMalloc(dst, sizeof(T) * (v.empty() ? 1 : v.size()));
  if (e != cudaSuccess) return e;
  if (v.empty()) return cudaSuccess;
  return cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
}

template <typename T>
void build_segments(const Plan& P, const std::vector<double>& G, const int E[3],
                    std::vector<Segment<T>>& segs, std::vector<int>& start) {
  int nx = 2 * E[0] + 1, ny = 2 * E[1] + 1;
  auto at = [&](int dx, int dy, int dz) {
    return G[((size_t)(dz + E[2]) * ny + (dy + E[1])) * nx + (dx + E[0])];
  };
  start.assign(2 * E[2] + 2, 0);
  for (int dz = -E[2]; dz <= E[2]; ++dz) {
    start[dz + E[2]] = (int)segs.size();
    for (int dy = -E[1]; dy <= E[1]; ++dy) {
      int X = -1;
      for (int dx = 0; dx <= E[0]; ++dx)
        if (at(dx, dy, dz) != 0.0) X = dx;
      if (X < 0) continue;
      for (int dx0 = -X; dx0 <= X; dx0 += kSeg) {
        Segment<T> s;
        s.dy = dy;
        s.dx0 = dx0;
        for (int j = 0; j < kSeg; ++j) {
          int dx = dx0 + j;
          s.g[j] = (dx <= X) ? (T)at(dx, dy, dz) : (T)0;
        }
        segs.push_back(s);
      }
    }
  }
  start[2 * E[2] + 1] = (int)segs.size();
  (void)P;
}

// Row pairs of the stencil for the packed FP32 kernel, whose lanes own two
// adjacent output rows (y, y + 1): input row y + e feeds row y through the
// taps of row e and row y + 1 through those of row e - 1, so one window load
// serves both.  Entry (dz, e, dx0), e = -Ey..Ey+1, holds the pairs
// (G(dx0 + j, e, dz), G(dx0 + j, e - 1, dz)) over the union of the two rows'
// x extents (zero where a row has no tap).
void build_row_pairs(const std::vector<double>& G, const int E[3], std::vector<Segment2>& segs,
                     std::vector<int>& start) {
  const int nx = 2 * E[0] + 1, ny = 2 * E[1] + 1;
  auto at = [&](int dx, int dy, int dz) -> double {
    if (dy < -E[1] || dy > E[1] || dx < -E[0] || dx > E[0]) return 0.0;
    return G[((size_t)(dz + E[2]) * ny + (dy + E[1])) * nx + (dx + E[0])];
  };
  auto extent = [&](int dy, int dz) {  // largest |dx| with a nonzero tap, -1 for an empty row
    int X = -1;
    for (int dx = 0; dx <= E[0]; ++dx)
      if (at(dx, dy, dz) != 0.0) X = dx;
    return X;
  };
  start.assign(2 * E[2] + 2, 0);
  for (int dz = -E[2]; dz <= E[2]; ++dz) {
    start[dz + E[2]] = (int)segs.size();
    for (int e = -E[1]; e <= E[1] + 1; ++e) {
      const int X = std::max(extent(e, dz), extent(e - 1, dz));
      if (X < 0) continue;
      for (int dx0 = -X; dx0 <= X; dx0 += kSeg) {
        Segment2 s;
        s.dy = e;
        s.dx0 = dx0;
        for (int j = 0; j < kSeg; ++j) {
          const int dx = dx0 + j;
          s.g[j] = dx <= X ? make_float2((float)at(dx, e, dz), (float)at(dx, e - 1, dz)) : make_float2(0.f, 0.f);
        }
        segs.push_back(s);
      }
    }
  }
  start[2 * E[2] + 1] = (int)segs.size();
}

}  // namespace

int64_t grid_points(const Plan& P, int k) { return (int64_t)P.n[k][0] * P.n[k][1] * P.n[k][2]; }

int validate_params(const msm_params* pp) {
  const msm_params& p = *pp;
  for (int d = 0; d < 3; ++d)
    if (!(p.box[d] > 0.0) || !std::isfinite(p.box[d])) return MSM_ERR_INVALID_ARG;
  if (!(p.cutoff > 0.0) || !(p.spacing > 0.0) || !std::isfinite(p.cutoff) || !std::isfinite(p.spacing))
    return MSM_ERR_INVALID_ARG;
  if (p.order != 3 && p.order != 5) return MSM_ERR_INVALID_ARG;
  if (p.splitting < 1 || p.splitting > 3) return MSM_ERR_INVALID_ARG;
  if (p.precision != MSM_FP64 && p.precision != MSM_MIXED) return MSM_ERR_INVALID_ARG;
  if (p.levels < 0 || p.levels > kMaxLevels) return MSM_ERR_INVALID_ARG;
  if (p.max_atoms < 1 || p.max_atoms > (int64_t)1 << 30) return MSM_ERR_INVALID_ARG;
  if (!std::isfinite(p.coulomb_k)) return MSM_ERR_INVALID_ARG;
  if (p.periodic) {
    for (int d = 0; d < 3; ++d)
      if (p.cutoff > 0.5 * p.box[d]) return MSM_ERR_CUTOFF_GT_HALF_BOX;
    for (int d = 0; d < 3; ++d)
      if ((int)std::floor(p.box[d] / (0.5 * p.cutoff)) < 5) return MSM_ERR_UNSUPPORTED;
  }
  return MSM_OK;
}

int validate_tuning(const msm_tuning* t) {
  if (!t) return MSM_OK;
  if (t->cell_fill < 0 || t->cell_fill > 256 || t->patch_cells < 0 || t->patch_cells > 4 || t->lattice_waves < 0 ||
      t->lattice_waves > 64)
    return MSM_ERR_INVALID_ARG;
  if (t->pair_targets != 0 && t->pair_targets != 8 && t->pair_targets != 32) return MSM_ERR_INVALID_ARG;
  if (t->batch_persistent != 0 && t->batch_persistent != 1) return MSM_ERR_INVALID_ARG;
  if (t->lattice_method < 0 || t->lattice_method > 2) return MSM_ERR_INVALID_ARG;
  if (t->pair_runs < 0 || t->pair_runs > 2) return MSM_ERR_INVALID_ARG;
  if (t->lattice_txn < 0 || t->lattice_tyn < 0 || t->lattice_txn > 32 || t->lattice_tyn > 32 ||
      (t->lattice_txn == 0) != (t->lattice_tyn == 0) || t->lattice_txn * t->lattice_tyn > 32)
    return MSM_ERR_INVALID_ARG;
  return MSM_OK;
}

int plan_geometry(const msm_params* pp, Plan* P) {
  const int vrc = validate_params(pp);
  if (vrc != MSM_OK) return vrc;
  P->P = *pp;
  P->fp64 = (pp->precision == MSM_FP64);
  P->S = (pp->order + 1) / 2;
  P->W = 2 * P->S;
  return geometry(*pp, P);
}

int build_plan(const msm_params* pp, const msm_tuning* tune, Plan* P) {
  const msm_params& p = *pp;
  int vrc = validate_params(pp);
  if (vrc != MSM_OK) return vrc;
  int trc = validate_tuning(tune);
  if (trc != MSM_OK) return trc;
  msm_tuning TU = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (tune) TU = *tune;
  const double fill = TU.cell_fill > 0 ? TU.cell_fill : 24.0;
  P->lattice_waves = TU.lattice_waves > 0 ? TU.lattice_waves : 8;
  P->pair_targets = TU.pair_targets > 0 ? TU.pair_targets : 32;
  P->lattice_txn = TU.lattice_txn;
  P->batch_persistent = TU.batch_persistent;
  const int lattice_method = TU.lattice_method > 0 ? TU.lattice_method : 2;
  P->lattice_tyn = TU.lattice_tyn;
  P->wolf_alpha = 2.4 / p.cutoff;  // alpha R = 2.4 (0.2 per length unit at R = 12) until msm_set_wolf_alpha
  for (int d = 0; d < 3; ++d)
    if (!(p.box[d] > 0.0) || !std::isfinite(p.box[d])) return MSM_ERR_INVALID_ARG;
  if (!(p.cutoff > 0.0) || !(p.spacing > 0.0) || !std::isfinite(p.cutoff) || !std::isfinite(p.spacing))
    return MSM_ERR_INVALID_ARG;
  if (p.order != 3 && p.order != 5) return MSM_ERR_INVALID_ARG;
  if (p.splitting < 1 || p.splitting > 3) return MSM_ERR_INVALID_ARG;
  if (p.precision != MSM_FP64 && p.precision != MSM_MIXED) return MSM_ERR_INVALID_ARG;
  if (p.levels < 0 || p.levels > kMaxLevels) return MSM_ERR_INVALID_ARG;
  if (p.max_atoms < 1 || p.max_atoms > (int64_t)1 << 30) return MSM_ERR_INVALID_ARG;
  if (!std::isfinite(p.coulomb_k)) return MSM_ERR_INVALID_ARG;
  if (p.periodic) {
    for (int d = 0; d < 3; ++d)
      if (p.cutoff > 0.5 * p.box[d]) return MSM_ERR_CUTOFF_GT_HALF_BOX;
  }
  P->P = p;
  P->fp64 = (p.precision == MSM_FP64);
  P->S = (p.order + 1) / 2;
  P->W = 2 * P->S;
  int rc = geometry(p, P);
  if (rc != MSM_OK) return rc;
  P->gamma0 = smooth(p.splitting, 0.0);

  // short-range cells: width >= a/2 (neighbours within two cells), widened
  // toward ~24 atoms per cell (tunable) at the plan's capacity density so that the 32
  // lanes of a warp stay busy (the bounding-box culling absorbs the larger
  // candidate volume)
  double vol = p.box[0] * p.box[1] * p.box[2];
  double wfill = std::cbrt(fill * vol / (double)p.max_atoms);
  // (cells may be wider than a: the neighbour rows then shrink to +-1 cell)
  double wmin = std::max(0.5 * p.cutoff, wfill);
  for (int d = 0; d < 3; ++d) {
    // the cell count nearest to the target width, but cells at least a/2 wide
    int c = std::min((int)std::lround(p.box[d] / wmin), (int)std::floor(p.box[d] / (0.5 * p.cutoff)));
    if (p.periodic && c < 5) c = (int)std::floor(p.box[d] / (0.5 * p.cutoff));
    if (c < 1) c = 1;
    if (p.periodic && c < 5) return MSM_ERR_UNSUPPORTED;  // the 5-cell walk would alias images
    if (c > 1024) c = 1024;
    P->nc[d] = c;
    P->cw[d] = p.box[d] / c;
  }
  P->ncell = P->nc[0] * P->nc[1] * P->nc[2];
  // target runs by default on large boxes, where they were measured faster
  // (1.63 against 1.72 ms at 42,875 cells); small boxes run too few warps
  // for the longer row walks of a run (1.15-1.9x slower at 343-1,000 cells)
  P->pair_runs = TU.pair_runs == 1 || (TU.pair_runs == 0 && P->ncell >= 16384);
  std::vector<int4> offs;
  for (int oz = -2; oz <= 2; ++oz)
    for (int oy = -2; oy <= 2; ++oy)
      for (int ox = -2; ox <= 2; ++ox) {
        int o[3] = {ox, oy, oz};
        double g2 = 0.0;
        for (int d = 0; d < 3; ++d) {
          double gap = std::max(std::abs(o[d]) - 1, 0) * P->cw[d];
          g2 += gap * gap;
        }
        if (g2 >= p.cutoff * p.cutoff) continue;  // no pair of points closer than a
        offs.push_back(make_int4(ox, oy, oz, 0));
      }
  P->noff = (int)offs.size();
  // the same offsets grouped by (dy, dz) into contiguous x runs (cells are numbered x fastest)
  std::vector<int4> rowv;
  for (int oz = -2; oz <= 2; ++oz)
    for (int oy = -2; oy <= 2; ++oy) {
      int xlo = 99, xhi = -99;
      for (auto& o : offs)
        if (o.y == oy && o.z == oz) {
          xlo = std::min(xlo, o.x);
          xhi = std::max(xhi, o.x);
        }
      if (xlo > xhi) continue;
      if (oy == 0 && oz == 0) {  // the home cell (offset 0) is evaluated separately, with the self test
        if (xlo <= -1) rowv.push_back(make_int4(oy, oz, xlo, -1));
        if (xhi >= 1) rowv.push_back(make_int4(oy, oz, 1, xhi));
      } else {
        rowv.push_back(make_int4(oy, oz, xlo, xhi));
      }
    }
  P->nrows = (int)rowv.size();
  // the packed pair kernel builds its row table one row per lane; with cells
  // at least a/2 wide there are at most 5 x 5 (dy, dz) rows plus the split
  // home row
  if (P->nrows > 32) return MSM_ERR_UNSUPPORTED;
  // anterpolation patch: B^3 cells reach at most floor(B cw/h) + 2S + 5
  // points per dimension (with margin for rounding); keep it in shared memory
  // (FP64 sums, or two 32-bit integer sums per point on the mixed path)
  {
    const int cap = P->fp64 ? 24 : 29;
    auto patch_dim = [&](int b) {
      int pd = 0;
      for (int d = 0; d < 3; ++d) pd = std::max(pd, (int)std::floor(b * P->cw[d] / P->h[d]) + 2 * P->S + 5);
      return pd;
    };
    // the largest patch (at most the requested one) that fits: batched launches
    int B = TU.patch_cells > 0 ? TU.patch_cells : 4;
    while (B >= 1 && patch_dim(B) > cap) --B;
    if (B < 1) return MSM_ERR_UNSUPPORTED;  // cells wider than a patch can hold
    P->ablk_batch = B;
    P->apd_batch = patch_dim(B);
    if (TU.patch_cells == 0 && !P->fp64) {
      // one system alone, mixed precision: by default smaller patches for
      // small systems, down to 2 cells a side until the patch blocks fill the
      // 152 SMs once (water23k: 0.40 -> 0.34 ms serialised; the FP64 path
      // measured 2 % slower with them); a batch fills the GPU with its replicas
      auto blocks = [&](int b) {
        int64_t nb = 1;
        for (int d = 0; d < 3; ++d) nb *= (P->nc[d] + b - 1) / b;
        return nb;
      };
      while (B > 2 && blocks(B) < 152) --B;
    }
    P->ablk = B;
    P->apd = patch_dim(B);
  }

  // level stencil G0(n) = g^0(|h o n|) on the level-0 lattice; level k uses
  // 2^-k G0 because g^k(2^k r) = 2^-k g^0(r).
  double R = 2.0 * p.cutoff;
  for (int d = 0; d < 3; ++d) {
    P->E[d] = (int)std::ceil(R / P->h[d]);
    while (P->E[d] > 0 && P->E[d] * P->h[d] >= R) --P->E[d];
  }
  // FFT form of the lattice cutoff (periodic levels whose sizes factor into
  // radices 2, 3, 5, 7; built after the workspace below).  It has no window
  // to fit, so a stencil too many grid spacings wide for the stencil kernel's
  // shared memory is refused only where the stencil would run.
  bool want_fft = p.periodic && lattice_method == 2 && P->levels > 1;
  for (int k = 0; k + 1 < P->levels && want_fft; ++k)
    for (int d = 0; d < 3; ++d)
      if (!fft_size_ok(P->n[k][d])) want_fft = false;
  P->stencil_fits = lattice_fits(*P);
  if (!P->stencil_fits && !want_fft) return MSM_ERR_UNSUPPORTED;  // cutoff too many grid spacings wide
  if (P->lattice_txn > 0 && P->stencil_fits && !lattice_tile_fits(*P, P->lattice_txn, P->lattice_tyn))
    return MSM_ERR_INVALID_ARG;
  std::vector<double> G((size_t)(2 * P->E[0] + 1) * (2 * P->E[1] + 1) * (2 * P->E[2] + 1), 0.0);
  double taps = 0;
  for (int dz = -P->E[2]; dz <= P->E[2]; ++dz)
    for (int dy = -P->E[1]; dy <= P->E[1]; ++dy)
      for (int dx = -P->E[0]; dx <= P->E[0]; ++dx) {
        double x = dx * P->h[0], y = dy * P->h[1], z = dz * P->h[2];
        double g = level_kernel(p.splitting, p.cutoff, 0, std::sqrt(x * x + y * y + z * z));
        G[((size_t)(dz + P->E[2]) * (2 * P->E[1] + 1) + (dy + P->E[1])) * (2 * P->E[0] + 1) +
          (dx + P->E[0])] = g;
        if (g != 0.0) taps += 1;
      }
  P->stencil_taps = taps;

  // top-level kernel table (FP64)
  int top = P->levels - 1;
  double ht[3];
  for (int d = 0; d < 3; ++d) ht[d] = std::ldexp(P->h[d], top);
  double A = std::ldexp(p.cutoff, top);
  std::vector<double> K;
  if (p.periodic) {
    // K(r) = [psi(r) - 1/r] + g^{l-1}(r) - sum_{m != 0} s(|r + mL|), with
    // s = 1/r - g^{l-1} supported on r < A: the image sum of g^{l-1} made
    // convergent by the Ewald kernel psi (tin-foil, neutralising background).
    for (int d = 0; d < 3; ++d) P->top_table_dims[d] = P->n[top][d];
    K.resize((size_t)P->n[top][0] * P->n[top][1] * P->n[top][2]);
    int img[3];
    for (int d = 0; d < 3; ++d) img[d] = (int)std::ceil(A / p.box[d]) + 1;
    for (int c = 0; c < P->n[top][2]; ++c)
      for (int b = 0; b < P->n[top][1]; ++b)
        for (int a = 0; a < P->n[top][0]; ++a) {
          int m[3] = {a, b, c};
          double r[3];
          for (int d = 0; d < 3; ++d) {
            int M = P->n[top][d], v = m[d];
            if (2 * v > M) v -= M;
            r[d] = v * ht[d];
          }
          double rr = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
          double val = ewald_minus_coulomb(p.box, r) + top_kernel(p.splitting, A, rr);
          for (int i = -img[0]; i <= img[0]; ++i)
            for (int j = -img[1]; j <= img[1]; ++j)
              for (int l2 = -img[2]; l2 <= img[2]; ++l2) {
                if (i == 0 && j == 0 && l2 == 0) continue;
                double x = r[0] + i * p.box[0], y = r[1] + j * p.box[1], z = r[2] + l2 * p.box[2];
                double s = std::sqrt(x * x + y * y + z * z);
                if (s < A) val -= 1.0 / s - top_kernel(p.splitting, A, s);
              }
          K[((size_t)c * P->n[top][1] + b) * P->n[top][0] + a] = val;
        }
  } else {
    for (int d = 0; d < 3; ++d) P->top_table_dims[d] = 2 * P->n[top][d] - 1;
    K.resize((size_t)P->top_table_dims[0] * P->top_table_dims[1] * P->top_table_dims[2]);
    for (int c = 0; c < P->top_table_dims[2]; ++c)
      for (int b = 0; b < P->top_table_dims[1]; ++b)
        for (int a = 0; a < P->top_table_dims[0]; ++a) {
          double x = (a - (P->n[top][0] - 1)) * ht[0], y = (b - (P->n[top][1] - 1)) * ht[1],
                 z = (c - (P->n[top][2] - 1)) * ht[2];
          K[((size_t)c * P->top_table_dims[1] + b) * P->top_table_dims[0] + a] =
              top_kernel(p.splitting, A, std::sqrt(x * x + y * y + z * z));
        }
  }

  // ---- device workspace ----
  DeviceBuffers& D = P->d;
  size_t T = P->fp64 ? sizeof(double) : sizeof(float);
  int64_t cap = p.max_atoms;
  P->cap = cap;
  {  // one energy partial per interpolation block (blocks of ablk^3 cells)
    int64_t nb = 1;
    for (int d = 0; d < 3; ++d) nb *= (P->nc[d] + P->ablk - 1) / P->ablk;
    P->nblk_partial = (int)std::max<int64_t>(nb, 1);
  }
  cudaError_t e = cudaSuccess;
  auto M = [&](void** ptr, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(ptr, bytes ? bytes : 16);
  };
  M((void**)&D.key, sizeof(int) * cap);
  M((void**)&D.rank, sizeof(int) * cap);
  M((void**)&D.perm, sizeof(int) * cap);
  M((void**)&D.count, sizeof(int) * (size_t)P->ncell);
  M((void**)&D.csum, sizeof(int) * (size_t)(P->ncell / 4096 + 1));
  if (e == cudaSuccess) e = cudaMemset(D.count, 0, sizeof(int) * (size_t)P->ncell);  // kept zero between evaluations
  M((void**)&D.cell_start, sizeof(int) * (P->ncell + 1));
  M(&D.atoms, 4 * T * cap);
  M(&D.gfrac, 4 * T * cap);
  M((void**)&D.gbase, sizeof(int4) * cap);
  M(&D.phis, T * cap);
  M(&D.fs, 4 * T * cap);
  M(&D.glong, 4 * T * cap);
  for (int k = 0; k < P->levels; ++k) {
    size_t np = (size_t)grid_points(*P, k);
    M(&D.gq[k], sizeof(double) * np);  // charge grids are FP64 in every mode
    M(&D.gu[k], T * np);
    M(&D.aq[k], sizeof(double) * np);
    M(&D.au[k], T * np);
  }
  // temporaries of the separable passes: the largest level pair, per dimension
  size_t tsize = (size_t)grid_points(*P, 0);
  for (int k = 0; k + 1 < P->levels; ++k) {
    size_t t = 1;
    for (int d = 0; d < 3; ++d) t *= (size_t)std::max(P->n[k][d], P->n[k + 1][d]);
    tsize = std::max(tsize, t);
  }
  for (int i = 0; i < 2; ++i) M(&D.tmp[i], sizeof(double) * tsize);
  P->tmp_elems = (int64_t)tsize;
  M(&D.lparts, T * (size_t)(P->stencil_fits ? lattice_parts_elems(*P) : 0));
  size_t ntop = (size_t)grid_points(*P, top);
  M((void**)&D.topq, sizeof(double) * ntop);
  M((void**)&D.topu, sizeof(double) * ntop);
  M((void**)&D.partial, sizeof(double) * P->nblk_partial);
  M((void**)&D.scalars, sizeof(double) * 8);
  M((void**)&D.md_partial, sizeof(double) * 4 * kMdBlocks);
  M((void**)&D.md_step, sizeof(int));
  M((void**)&D.status, sizeof(int));
  if (want_fft) {  // complex FP64 per point of every lattice level (the kernel's transforms use level 0's share)
    size_t pts = 0;
    for (int k = 0; k + 1 < P->levels; ++k) pts += (size_t)grid_points(*P, k);
    M(&D.fft_work, 16 * pts);
  }
  if (e != cudaSuccess) return MSM_ERR_OOM;
  if (cudaMemset(D.status, 0, sizeof(int)) != cudaSuccess) return MSM_ERR_CUDA;
  if (want_fft) {
    // the folded kernel of level k on its own grid: taps n wrapped modulo the
    // level's dimensions (the images of the sphere where it is wider than the
    // grid), values G0(n) (the level factor is applied with the transform)
    for (int k = 0; k + 1 < P->levels; ++k) {
      const int M0 = P->n[k][0], M1 = P->n[k][1], M2 = P->n[k][2];
      std::vector<double> Kg((size_t)M0 * M1 * M2, 0.0);
      for (int dz = -P->E[2]; dz <= P->E[2]; ++dz)
        for (int dy = -P->E[1]; dy <= P->E[1]; ++dy)
          for (int dx = -P->E[0]; dx <= P->E[0]; ++dx) {
            const double g = G[((size_t)(dz + P->E[2]) * (2 * P->E[1] + 1) + (dy + P->E[1])) * (2 * P->E[0] + 1) +
                               (dx + P->E[0])];
            if (g == 0.0) continue;
            const int x = ((dx % M0) + M0) % M0, y = ((dy % M1) + M1) % M1, z = ((dz % M2) + M2) % M2;
            Kg[((size_t)z * M1 + y) * M0 + x] += g;
          }
      if (fft_build_level(*P, k, Kg, D.fft_work) != cudaSuccess) return MSM_ERR_CUDA;
    }
    // the pass tables of both sweeps: level k at offset sum_{j<k} N_j of the
    // workspace, in complex elements of the plan's precision
    const size_t cs = P->fp64 ? 2 * sizeof(double) : 2 * sizeof(float);
    for (int dir = 0; dir < 2; ++dir) {
      std::vector<FftBatchItem> items;
      size_t off = 0;
      for (int k = 0; k + 1 < P->levels; ++k) {
        items.push_back(FftBatchItem{&P->fftl[k], (const double*)(dir ? D.aq[k] : D.gq[k]), dir ? D.au[k] : D.gu[k],
                                     (char*)D.fft_work + cs * off});
        off += (size_t)grid_points(*P, k);
      }
      if (fft_batch_build(items, P->fp64, &P->fftb[dir]) != cudaSuccess) return MSM_ERR_CUDA;
    }
    P->lattice_fft = true;
  }
  if (upload((void**)&D.topK, K) != cudaSuccess) return MSM_ERR_OOM;
  if (upload((void**)&D.cell_off, offs) != cudaSuccess) return MSM_ERR_OOM;
  if (upload((void**)&D.cell_rows, rowv) != cudaSuccess) return MSM_ERR_OOM;
  if (P->fp64) {
    std::vector<R4<double>> sh;
    for (auto& o : offs) sh.push_back({o.x * P->cw[0], o.y * P->cw[1], o.z * P->cw[2], 0.0});
    if (upload(&D.cell_shift, sh) != cudaSuccess) return MSM_ERR_OOM;
  } else {
    std::vector<R4<float>> sh;
    for (auto& o : offs)
      sh.push_back({(float)(o.x * P->cw[0]), (float)(o.y * P->cw[1]), (float)(o.z * P->cw[2]), 0.f});
    if (upload(&D.cell_shift, sh) != cudaSuccess) return MSM_ERR_OOM;
  }
  if (P->stencil_fits) {  // the stencil kernel's segment tables (unused, and not built, past its window)
    std::vector<int> start;
    if (P->fp64) {
      std::vector<Segment<double>> segs;
      build_segments<double>(*P, G, P->E, segs, start);
      P->nseg = (int)segs.size();
      if (upload(&D.seg, segs) != cudaSuccess) return MSM_ERR_OOM;
    } else {
      std::vector<Segment2> segs2;
      build_row_pairs(G, P->E, segs2, start);
      P->nseg = (int)segs2.size();
      if (upload(&D.seg2, segs2) != cudaSuccess) return MSM_ERR_OOM;
    }
    if (upload((void**)&D.seg_start, start) != cudaSuccess) return MSM_ERR_OOM;
  }
  int least = 0, greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
      cudaStreamCreateWithPriority(&P->side, cudaStreamNonBlocking, greatest) != cudaSuccess ||
      cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming) != cudaSuccess)
    return MSM_ERR_CUDA;
  return MSM_OK;
}

void free_plan(Plan* P) {
  DeviceBuffers& D = P->d;
  void* ptrs[] = {D.key, D.rank, D.perm, D.count, D.csum, D.cell_start, D.atoms,
                  D.gfrac, D.gbase, D.phis, D.fs, D.glong, D.topK, D.topq, D.topu, D.seg, D.seg2, D.cell_shift, D.cell_rows,
                  D.seg_start, D.cell_off, D.partial, D.scalars, D.md_partial, D.md_step, D.status, D.hpos, D.hq,
                  D.hphi, D.hforce, D.henergy, D.lparts, D.fft_work};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (D.hstatus) cudaFreeHost(D.hstatus);
  for (int i = 0; i < 2; ++i)
    if (D.tmp[i]) cudaFree(D.tmp[i]);
  for (int k = 0; k < kMaxLevels; ++k) fft_free_level(P->fftl[k]);
  for (int dir = 0; dir < 2; ++dir) {
    fft_batch_free(P->fftb[dir]);
    P->fftb[dir] = nullptr;
  }
  for (int k = 0; k < kMaxLevels; ++k) {
    if (D.gq[k]) cudaFree(D.gq[k]);
    if (D.gu[k]) cudaFree(D.gu[k]);
    if (D.aq[k]) cudaFree(D.aq[k]);
    if (D.au[k]) cudaFree(D.au[k]);
  }
  D = DeviceBuffers();
  if (P->side) cudaStreamDestroy(P->side);
  if (P->ev_fork) cudaEventDestroy(P->ev_fork);
  if (P->ev_join) cudaEventDestroy(P->ev_join);
  P->side = nullptr;
  P->ev_fork = P->ev_join = nullptr;
}

}  // namespace msm
