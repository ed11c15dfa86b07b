// kernels_pair.cu -- short-range part of MSM (Sec. "Multilevel Summation
// Method"): u_i^short = sum_{j != i, r_ij < a} q_j g*(r_ij) with
// g*(r) = 1/r - gamma(r/a)/a (Eq. msmgrid), and the force
// F_i = -q_i grad_i u_i^short.
//
// One warp owns one cell of the sort-binned atoms (cells at least a/2 wide):
// its lanes hold up to 32 target atoms and walk the neighbour cells within
// reach (offsets whose closest points are nearer than a).  Source atoms are
// shifted into the target cell's frame (every difference is between small
// cell-local coordinates), culled against the bounding box of the targets,
// and queued in the warp's shared memory; full queues are broadcast to the
// lanes in unrolled batches.  Each pair costs one rsqrt and ~20 FP32
// operations; rejected pairs are masked, not branched.  Mixed precision sums
// each batch in FP32 and folds the batch sums into the running totals with an
// error-free TwoSum (compensated accumulation).
#include <climits>
#include <cmath>
#include <new>

#include "msm_internal.h"

namespace msm {

namespace {

template <typename T, int M>
struct Smooth;  // gamma(rho) and d gamma / d s as polynomials in s = rho^2 < 1

template <typename T>
struct Smooth<T, 1> {
  __device__ static T g(T s) { return T(1.5) - T(0.5) * s; }
  __device__ static T gs(T) { return T(-0.5); }
};
template <typename T>
struct Smooth<T, 2> {
  __device__ static T g(T s) { return T(1.875) + s * (T(-1.25) + T(0.375) * s); }
  __device__ static T gs(T s) { return T(-1.25) + T(0.75) * s; }
};
template <typename T>
struct Smooth<T, 3> {
  __device__ static T g(T s) {
    return T(2.1875) + s * (T(-2.1875) + s * (T(1.3125) - T(0.3125) * s));
  }
  __device__ static T gs(T s) { return T(-2.1875) + s * (T(2.625) - T(0.9375) * s); }
};

// error-free transformation s + x = t + err; the error goes to the compensation term
template <typename T>
__device__ __forceinline__ void two_sum_add(T& s, T& c, T x) {
  T t = s + x;
  T bp = t - s;
  c += (s - (t - bp)) + (x - bp);
  s = t;
}

// Cutoff constants are precomputed on the host in both precisions: a divide
// in FP64 on every thread would cost dozens of FP64-pipe operations.
struct PairArgs {
  int nc[3];
  int periodic;
  int noff;
  double a2, inv_a, inv_a2, two_inv_a3;
  float a2f, inv_af, inv_a2f, two_inv_a3f;
};

// Constants of the Wolf pair function (damped, shifted force) with damping
// alpha and cutoff R = a: v(r) = erfc(alpha r)/r - vR + c1 (r - R),
// vR = erfc(alpha R)/R, c1 = erfc(alpha R)/R^2 + c2 exp(-alpha^2 R^2)/R,
// c2 = 2 alpha/sqrt(pi).
template <typename T>
struct WolfC {
  T alpha, alpha2, c2, vR, c1, R;
};

template <typename T>
WolfC<T> wolf_consts(double alpha, double R) {
  const double c2 = 2.0 * alpha / std::sqrt(M_PI);
  const double vR = std::erfc(alpha * R) / R;
  const double c1 = std::erfc(alpha * R) / (R * R) + c2 * std::exp(-alpha * alpha * R * R) / R;
  return WolfC<T>{(T)alpha, (T)(alpha * alpha), (T)c2, (T)vR, (T)c1, (T)R};
}

__device__ __forceinline__ float d_erfc(float x) { return erfcf(x); }
__device__ __forceinline__ double d_erfc(double x) { return erfc(x); }
__device__ __forceinline__ float d_exp(float x) { return expf(x); }
__device__ __forceinline__ double d_exp(double x) { return exp(x); }

template <typename T>
struct CutoffConsts;
template <>
struct CutoffConsts<double> {
  __device__ static void get(const PairArgs& A, double& a2, double& ia, double& ia2, double& t3) {
    a2 = A.a2; ia = A.inv_a; ia2 = A.inv_a2; t3 = A.two_inv_a3;
  }
};

PairArgs pair_args(const Plan& P) {
  PairArgs A;
  for (int d = 0; d < 3; ++d) A.nc[d] = P.nc[d];
  A.periodic = P.P.periodic;
  A.noff = P.noff;
  const double a = P.P.cutoff;
  A.a2 = a * a;
  A.inv_a = 1.0 / a;
  A.inv_a2 = 1.0 / (a * a);
  A.two_inv_a3 = 2.0 / (a * a * a);
  A.a2f = (float)A.a2;
  A.inv_af = (float)A.inv_a;
  A.inv_a2f = (float)A.inv_a2;
  A.two_inv_a3f = (float)A.two_inv_a3;
  return A;
}

constexpr int kWarps = 4;
#ifndef MSM_PAIR_BATCH
#define MSM_PAIR_BATCH 64
#endif
#ifndef MSM_PAIR_MINB
#define MSM_PAIR_MINB 6
#endif
constexpr int kBatch = MSM_PAIR_BATCH;  // sources per queue drain (pairs per lane per drain)
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float fast_rsqrt(float x) {  // one MUFU.RSQ; inputs are >= a^2/... never denormal
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ double fast_rsqrt(double x) { return rsqrt(x); }

template <typename T>
__device__ __forceinline__ T far_away() { return T(1e18); }

// Pair functions: K = 0 is MSM's short-range kernel g*(r) = 1/r - gamma(r/a)/a
// (zero with its derivative at r = a); K = 1 is the plain Coulomb law 1/r of
// the cutoff method (the parareal section's coarse propagator G), which is
// not zero at a, so sources beyond the cutoff are masked; K = 2 is Wolf
// summation's damped, shifted-force pair potential (another coarse function
// of that section), masked beyond a as well.
constexpr int kPairMSM = 0, kPairCutoff = 1, kPairWolf = 2;

// One pair, scalar: target ai against source b (skipped at r = 0, the atom
// itself, and beyond the cutoff); adds q_j times the pair potential to pphi
// and f (r_i - r_j) to (px, py, pz) with f = q_j v'(r)/r.
template <typename T, int M, int K>
__device__ __forceinline__ void pair1(const R4<T>& ai, const R4<T>& b, T a2, T inv_a, T inv_a2, T two_inv_a3,
                                      const WolfC<T>& W, T& pphi, T& px, T& py, T& pz) {
  const T dx = ai.x - b.x, dy = ai.y - b.y, dz = ai.z - b.z;
  const T r2 = dx * dx + dy * dy + dz * dz;
  const bool ok = (r2 < a2) && (r2 > T(0));  // inside the cutoff, not the atom itself
  const T r2s = ok ? r2 : a2;
  const T qj = ok ? b.w : T(0);
  const T rinv = fast_rsqrt(r2s);
  T f;
  if (K == kPairMSM) {
    const T s = r2s * inv_a2;
    pphi += qj * (rinv - Smooth<T, M>::g(s) * inv_a);
    f = qj * (-(rinv * rinv * rinv) - two_inv_a3 * Smooth<T, M>::gs(s));
  } else if (K == kPairWolf) {  // f = q_j v'(r) / r
    const T r = r2s * rinv;
    const T e = d_erfc(W.alpha * r), g = W.c2 * d_exp(-W.alpha2 * r2s);
    pphi += qj * (e * rinv - W.vR + W.c1 * (r - W.R));
    f = qj * (W.c1 * rinv - (e * rinv + g) * rinv * rinv);
  } else {
    pphi += qj * rinv;
    f = -qj * (rinv * rinv * rinv);
  }
  px += f * dx;
  py += f * dy;
  pz += f * dz;
}

// One batch: the lane's target atom against the kBatch queued sources.
template <typename T, int M, bool COMP, int K = kPairMSM, int NB = kBatch>
__device__ __forceinline__ void pair_batch(const R4<T>* __restrict__ Q, const R4<T>& ai, T a2, T inv_a,
                                           T inv_a2, T two_inv_a3, const WolfC<T>& W, T& phi, T& fx, T& fy,
                                           T& fz, T& cphi, T& cfx, T& cfy, T& cfz) {
  T pphi = 0, px = 0, py = 0, pz = 0;
#pragma unroll 8
  for (int jj = 0; jj < NB; ++jj) pair1<T, M, K>(ai, Q[jj], a2, inv_a, inv_a2, two_inv_a3, W, pphi, px, py, pz);
  if (COMP) {
    two_sum_add(phi, cphi, pphi);
    two_sum_add(fx, cfx, px);
    two_sum_add(fy, cfy, py);
    two_sum_add(fz, cfz, pz);
  } else {
    phi += pphi;
    fx += px;
    fy += py;
    fz += pz;
  }
}

// One warp per cell.  For every neighbour cell in reach, the warp stages 32
// source atoms at a time (shifted into the target cell's frame), drops those
// farther than a from the bounding box of its target atoms, and appends the
// rest to a per-warp queue in shared memory; each full queue of kBatch
// sources is one fully unrolled batch of pair evaluations.
template <typename T, int M, bool COMP, int K>
__global__ void __launch_bounds__(32 * kWarps) k_short_range(
    const R4<T>* __restrict__ atoms, const int* __restrict__ cell_start,
    const int4* __restrict__ offs, const R4<T>* __restrict__ shifts, PairArgs A, WolfC<T> W, int ncell,
    T* __restrict__ phis, R4<T>* __restrict__ fs) {
  __shared__ R4<T> queue[kWarps][2 * kBatch];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  R4<T>* Q = queue[warp];
  const int cell = blockIdx.x * kWarps + warp;
  if (cell >= ncell) return;  // warp-uniform
  const int cx = cell % A.nc[0], cy = (cell / A.nc[0]) % A.nc[1], cz = cell / (A.nc[0] * A.nc[1]);
  T a2, inv_a, inv_a2, two_inv_a3;
  CutoffConsts<T>::get(A, a2, inv_a, inv_a2, two_inv_a3);
  const R4<T> dummy = {far_away<T>(), far_away<T>(), far_away<T>(), T(0)};
  const int i0 = cell_start[cell], i1 = cell_start[cell + 1];
  for (int ib = i0; ib < i1; ib += 32) {
    const int i = ib + lane;
    const bool iv = i < i1;
    R4<T> ai = iv ? atoms[i] : R4<T>{T(0), T(0), T(0), T(0)};
    // bounding box of this chunk's target atoms
    T lx = iv ? ai.x : far_away<T>(), ly = iv ? ai.y : far_away<T>(), lz = iv ? ai.z : far_away<T>();
    T hx = iv ? ai.x : -far_away<T>(), hy = iv ? ai.y : -far_away<T>(), hz = iv ? ai.z : -far_away<T>();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lx = min(lx, __shfl_xor_sync(kFull, lx, o));
      ly = min(ly, __shfl_xor_sync(kFull, ly, o));
      lz = min(lz, __shfl_xor_sync(kFull, lz, o));
      hx = max(hx, __shfl_xor_sync(kFull, hx, o));
      hy = max(hy, __shfl_xor_sync(kFull, hy, o));
      hz = max(hz, __shfl_xor_sync(kFull, hz, o));
    }
    T phi = 0, fx = 0, fy = 0, fz = 0, cphi = 0, cfx = 0, cfy = 0, cfz = 0;
    int qn = 0;  // queued sources (warp-uniform)
    for (int o = 0; o < A.noff; ++o) {
      const int4 off = offs[o];
      int nx = cx + off.x, ny = cy + off.y, nz = cz + off.z;
      if (A.periodic) {
        nx = (nx + A.nc[0]) % A.nc[0];
        ny = (ny + A.nc[1]) % A.nc[1];
        nz = (nz + A.nc[2]) % A.nc[2];
      } else if (nx < 0 || ny < 0 || nz < 0 || nx >= A.nc[0] || ny >= A.nc[1] || nz >= A.nc[2]) {
        continue;
      }
      const int nb = (nz * A.nc[1] + ny) * A.nc[0] + nx;
      const R4<T> sh = shifts[o];
      const int j0 = cell_start[nb], j1 = cell_start[nb + 1];
      for (int jb = j0; jb < j1; jb += 32) {
        const int j = jb + lane;
        R4<T> aj = dummy;
        if (j < j1) {
          aj = atoms[j];
          aj.x += sh.x;
          aj.y += sh.y;
          aj.z += sh.z;
        }
        const T ex = max(max(lx - aj.x, aj.x - hx), T(0));
        const T ey = max(max(ly - aj.y, aj.y - hy), T(0));
        const T ez = max(max(lz - aj.z, aj.z - hz), T(0));
        const bool keep = (j < j1) && (ex * ex + ey * ey + ez * ez < a2);
        const unsigned bal = __ballot_sync(kFull, keep);
        if (keep) Q[qn + __popc(bal & ((1u << lane) - 1u))] = aj;
        qn += __popc(bal);
        __syncwarp();
        if (qn >= kBatch) {
          pair_batch<T, M, COMP, K>(Q, ai, a2, inv_a, inv_a2, two_inv_a3, W, phi, fx, fy, fz, cphi, cfx, cfy, cfz);
          __syncwarp();
          if (lane < qn - kBatch) Q[lane] = Q[kBatch + lane];
          qn -= kBatch;
          __syncwarp();
        }
      }
    }
    if (qn > 0) {  // last partial batch, padded with far-away zero charges
      for (int t = lane; t < kBatch; t += 32)
        if (t >= qn) Q[t] = dummy;
      __syncwarp();
      pair_batch<T, M, COMP, K>(Q, ai, a2, inv_a, inv_a2, two_inv_a3, W, phi, fx, fy, fz, cphi, cfx, cfy, cfz);
      __syncwarp();
    }
    if (iv) {
      phis[i] = phi + cphi;
      const T qi = ai.w;
      fs[i] = R4<T>{-qi * (fx + cfx), -qi * (fy + cfy), -qi * (fz + cfz), T(0)};
    }
  }
}

// ---- mixed precision: packed FP32x2 arithmetic (two sources per instruction) ----
// The queue is stored as four FP32 arrays (x, y, z, q), so sources j..j+3
// load as one float4 per array and feed FFMA2/FMUL2/FADD2 as two pairs.  With
// d = r_j - r_i, f' = q_j (1/r^3 + 2 gamma_s(s)/a^3) and
// F_i = -q_i sum_j f' d, which needs no negations in the loop.  The home cell
// (the only one that holds the target itself) goes through the scalar batch
// with the self test; every other cell skips that test.  Far-away padding
// sits at 1e6 so that the unmasked polynomial stays finite.
struct alignas(16) QueueF {
  float x[2 * kBatch], y[2 * kBatch], z[2 * kBatch], q[2 * kBatch];
};

// gamma(r/a)/a and (2/a^3) dgamma/ds written straight as polynomials in r^2
// (host-scaled coefficients, duplicated into float2 pairs):
//   pot = 1/r - sum_k G[k] r2^k,   f' = 1/r^3 + sum_k D[k] r2^k.
// Beyond the cutoff r2 is clamped to a^2: pot and f' are zero there up to
// FP32 rounding (a few 1e-8 / a per source, measured to leave the energy and
// forces of the 1.07M-atom water box unchanged at the 1e-8 / 1e-7 level).
struct PairCoef {
  float2 G[4];
  float2 D[3];
};

template <int M>
__device__ __forceinline__ float2 poly_g(const PairCoef& C, float2 r2) {
  float2 t = C.G[M];
#pragma unroll
  for (int k = M - 1; k >= 0; --k) t = __ffma2_rn(t, r2, C.G[k]);
  return t;
}
template <int M>
__device__ __forceinline__ float2 poly_d(const PairCoef& C, float2 r2) {
  float2 t = C.D[M - 1];
#pragma unroll
  for (int k = M - 2; k >= 0; --k) t = __ffma2_rn(t, r2, C.D[k]);
  return t;
}

// One packed step: the lane's target (negated coordinates nax, nay, naz)
// against two sources (bx, by, bz, bq); adds q_j times the pair potential to
// sphi and f' d to (sx, sy, sz) with d = r_j - r_i.  Outside the home cell a
// source is never at r = 0; SELF (the home cell, which holds the target
// itself) drops a source at r = 0: its charge becomes 0 and r^2 becomes a^2.
template <int M, int K, bool SELF = false>
__device__ __forceinline__ void pair2(float2 bx, float2 by, float2 bz, float2 bq, float2 nax, float2 nay, float2 naz,
                                      float a2, const PairCoef& C, const WolfC<float>& W, float2& sphi, float2& sx,
                                      float2& sy, float2& sz) {
  const float2 dx = __fadd2_rn(bx, nax), dy = __fadd2_rn(by, nay), dz = __fadd2_rn(bz, naz);
  float2 r2 = __fmul2_rn(dx, dx);
  r2 = __ffma2_rn(dy, dy, r2);
  r2 = __ffma2_rn(dz, dz, r2);
  if (SELF) {
    bq = make_float2(r2.x > 0.f ? bq.x : 0.f, r2.y > 0.f ? bq.y : 0.f);
    r2 = make_float2(r2.x > 0.f ? r2.x : a2, r2.y > 0.f ? r2.y : a2);
  }
  float2 fp;
  if (K == kPairMSM) {
    // a source beyond the cutoff is evaluated at r = a, where g* and its
    // derivative vanish (C1 smoothing): no select on q_j is needed
    r2 = make_float2(fminf(r2.x, a2), fminf(r2.y, a2));
    const float2 qj = bq;
    const float2 rinv = make_float2(fast_rsqrt(r2.x), fast_rsqrt(r2.y));
    const float2 pot = __fadd2_rn(rinv, poly_g<M>(C, r2));  // G holds -gamma coefficients
    sphi = __ffma2_rn(qj, pot, sphi);
    fp = __fmul2_rn(__ffma2_rn(__fmul2_rn(rinv, rinv), rinv, poly_d<M>(C, r2)), qj);
  } else if (K == kPairWolf) {
    // damped shifted force within the cutoff; erfc(x) by Abramowitz and
    // Stegun 7.1.26, t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) exp(-x^2),
    // t = 1 / (1 + p x), |error| < 1.5e-7 for x >= 0, whose exp(-x^2) is the
    // force term's exp(-alpha^2 r^2) as well
    const bool okx = r2.x < a2, oky = r2.y < a2;
    const float2 r2s = make_float2(okx ? r2.x : a2, oky ? r2.y : a2);
    const float2 q = make_float2(okx ? bq.x : 0.f, oky ? bq.y : 0.f);
    const float2 ri = make_float2(fast_rsqrt(r2s.x), fast_rsqrt(r2s.y));
    const float2 r = __fmul2_rn(r2s, ri);
    const float2 al = make_float2(W.alpha, W.alpha);
    const float2 x = __fmul2_rn(al, r);
    const float2 den = __ffma2_rn(make_float2(0.3275911f, 0.3275911f), x, make_float2(1.f, 1.f));
    const float2 t = make_float2(__fdividef(1.f, den.x), __fdividef(1.f, den.y));
    float2 poly = make_float2(1.061405429f, 1.061405429f);
    poly = __ffma2_rn(poly, t, make_float2(-1.453152027f, -1.453152027f));
    poly = __ffma2_rn(poly, t, make_float2(1.421413741f, 1.421413741f));
    poly = __ffma2_rn(poly, t, make_float2(-0.284496736f, -0.284496736f));
    poly = __ffma2_rn(poly, t, make_float2(0.254829592f, 0.254829592f));
    const float2 ex = make_float2(__expf(-W.alpha2 * r2s.x), __expf(-W.alpha2 * r2s.y));
    const float2 e = __fmul2_rn(__fmul2_rn(poly, t), ex);  // erfc(alpha r)
    const float2 er = __fmul2_rn(e, ri);
    // q (erfc(alpha r) / r - v_R + c1 (r - R)) and -v'(r) / r = q ((e/r + c2 ex) / r^2 - c1 / r)
    const float2 c1v = make_float2(W.c1, W.c1);
    const float2 pot = __ffma2_rn(c1v, __fadd2_rn(r, make_float2(-W.R, -W.R)), __fadd2_rn(er, make_float2(-W.vR, -W.vR)));
    sphi = __ffma2_rn(q, pot, sphi);
    const float2 inner = __ffma2_rn(make_float2(W.c2, W.c2), ex, er);
    fp = __fmul2_rn(q, __ffma2_rn(__fmul2_rn(inner, ri), ri, __fmul2_rn(make_float2(-W.c1, -W.c1), ri)));
  } else {  // plain Coulomb within the cutoff
    const float2 qj = make_float2(r2.x < a2 ? bq.x : 0.f, r2.y < a2 ? bq.y : 0.f);
    const float2 rinv = make_float2(fast_rsqrt(r2.x), fast_rsqrt(r2.y));
    sphi = __ffma2_rn(qj, rinv, sphi);
    fp = __fmul2_rn(__fmul2_rn(__fmul2_rn(rinv, rinv), rinv), qj);
  }
  sx = __ffma2_rn(fp, dx, sx);
  sy = __ffma2_rn(fp, dy, sy);
  sz = __ffma2_rn(fp, dz, sz);
}

template <int M, int K, int NB = kBatch, bool SELF = false>
__device__ __forceinline__ void pair_batch_f2(const QueueF& Q, float2 nax, float2 nay, float2 naz, float a2,
                                              const PairCoef& C, const WolfC<float>& W, float& phi, float& px,
                                              float& py, float& pz, float& cphi, float& cpx, float& cpy,
                                              float& cpz) {
  float2 sphi = make_float2(0.f, 0.f), sx = sphi, sy = sphi, sz = sphi;
  // sources jj..jj+3 load as one float4 per coordinate (two packed halves)
  auto four = [&](int jj) {
    const float4 x4 = *reinterpret_cast<const float4*>(&Q.x[jj]);
    const float4 y4 = *reinterpret_cast<const float4*>(&Q.y[jj]);
    const float4 z4 = *reinterpret_cast<const float4*>(&Q.z[jj]);
    const float4 q4 = *reinterpret_cast<const float4*>(&Q.q[jj]);
    pair2<M, K, SELF>(make_float2(x4.x, x4.y), make_float2(y4.x, y4.y), make_float2(z4.x, z4.y),
                      make_float2(q4.x, q4.y), nax, nay, naz, a2, C, W, sphi, sx, sy, sz);
    pair2<M, K, SELF>(make_float2(x4.z, x4.w), make_float2(y4.z, y4.w), make_float2(z4.z, z4.w),
                      make_float2(q4.z, q4.w), nax, nay, naz, a2, C, W, sphi, sx, sy, sz);
  };
#pragma unroll
  for (int jj = 0; jj < NB; jj += 4) four(jj);
  two_sum_add(phi, cphi, sphi.x + sphi.y);
  two_sum_add(px, cpx, sx.x + sx.y);
  two_sum_add(py, cpy, sy.x + sy.y);
  two_sum_add(pz, cpz, sz.x + sz.y);
}

// Rows of neighbour cells: for each (dy, dz) the cells cx+xlo..cx+xhi of one x
// row are contiguous in the sorted atom array (cells are numbered x fastest),
// so a whole row is one or two contiguous atom ranges ("segments"; two when
// the row wraps around a periodic box).  At the start of a cell the lanes
// build the cell's segment table together, one row per lane (all cell-start
// loads in flight at once), and a warp scan lays the segments end to end
// into one flat source index space.  The warp then walks that space in full
// chunks of 32 sources, loading the next chunk's atoms before it works on the
// current one.  The x offset of a source's cell follows from comparing its
// index with the cell starts inside its segment.
constexpr int kMaxRows = 32;  // rows per cell: cells at least a/2 wide give at most 26

struct SegTable {
  int4 rec[2 * kMaxRows + 1];   // (first atom, flat start, x offset of the first cell, -); sentinel at the end
  int4 bnd[2 * kMaxRows];       // first atom of the segment's 2nd..5th cell (INT_MAX where absent)
  float2 shift[2 * kMaxRows];   // (y, z) shift of the row
};

// Arguments of the packed pair kernel (one system).
struct PairKArgs {
  const R4<float>* atoms;
  const int* cell_start;
  const int4* rows;
  int nrows;
  PairArgs A;
  PairCoef C;
  WolfC<float> W;
  float cwx, cwy, cwz;
  int ncell;
  float* phis;
  R4<float>* fs;
  // target runs (short_range_run_body): cell of every input atom, the sorted
  // order's input indices and the atom count
  const int* key;
  const int* perm;
  int natoms;
};

// The segment table of cell (cx, cy, cz), built by the warp (lane r: row r);
// returns the number of sources in the flat index space.
__device__ __forceinline__ int build_seg_table(SegTable& T, const PairKArgs& K, int cx, int cy, int cz, int lane) {
  const int* __restrict__ cell_start = K.cell_start;
  const int4* __restrict__ rows = K.rows;
  const int nrows = K.nrows;
  const PairArgs& A = K.A;
  const int ncx = A.nc[0], ncy = A.nc[1], ncz = A.nc[2];
  const float cwy = K.cwy, cwz = K.cwz;
  int len[2] = {0, 0}, j0s[2] = {0, 0}, ox0s[2] = {0, 0};
  int4 bnds[2] = {make_int4(INT_MAX, INT_MAX, INT_MAX, INT_MAX), make_int4(INT_MAX, INT_MAX, INT_MAX, INT_MAX)};
  float2 sh = make_float2(0.f, 0.f);
  if (lane < nrows) {
    const int4 row = rows[lane];  // (dy, dz, xlo, xhi): x offsets xlo..xhi of this row
    int ny = cy + row.x, nz = cz + row.y;
    bool inside = true;
    if (A.periodic) {
      ny += (ny < 0) ? ncy : ((ny >= ncy) ? -ncy : 0);
      nz += (nz < 0) ? ncz : ((nz >= ncz) ? -ncz : 0);
    } else if (ny < 0 || nz < 0 || ny >= ncy || nz >= ncz) {
      inside = false;
    }
    const int rbase = (nz * ncy + ny) * ncx;
    sh = make_float2(row.x * cwy, row.y * cwz);
#pragma unroll
    for (int seg = 0; seg < 2; ++seg) {
      int ox0 = 0, ox1 = -1;  // empty unless set below
      if (!inside) {
      } else if (A.periodic) {
        const int xa = cx + row.z, xb = cx + row.w;  // may leave [0, ncx) by at most 2
        if (xa < 0) {
          if (seg == 0) { ox0 = row.z; ox1 = -cx - 1; } else { ox0 = -cx; ox1 = row.w; }
        } else if (xb >= ncx) {
          if (seg == 0) { ox0 = row.z; ox1 = ncx - 1 - cx; } else { ox0 = ncx - cx; ox1 = row.w; }
        } else if (seg == 0) {
          ox0 = row.z; ox1 = row.w;
        }
      } else if (seg == 0) {
        ox0 = max(row.z, -cx);
        ox1 = min(row.w, ncx - 1 - cx);
      }
      if (ox0 <= ox1) {
        int x0 = cx + ox0, x1 = cx + ox1;
        if (A.periodic) {
          x0 += (x0 < 0) ? ncx : ((x0 >= ncx) ? -ncx : 0);
          x1 += (x1 < 0) ? ncx : ((x1 >= ncx) ? -ncx : 0);
        }
        const int j0 = cell_start[rbase + x0], j1 = cell_start[rbase + x1 + 1];
        int bb[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) bb[t] = (x0 + 1 + t <= x1) ? cell_start[rbase + x0 + 1 + t] : INT_MAX;
        len[seg] = j1 - j0;
        j0s[seg] = j0;
        ox0s[seg] = ox0;
        bnds[seg] = make_int4(bb[0], bb[1], bb[2], bb[3]);
      }
    }
  }
  int total;
  {
    const int mine = len[0] + len[1];
    int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    total = __shfl_sync(kFull, incl, 31);
    const int start = incl - mine;
    if (lane < nrows) {
#pragma unroll
      for (int seg = 0; seg < 2; ++seg) {
        T.rec[2 * lane + seg] = make_int4(j0s[seg], seg ? start + len[0] : start, ox0s[seg], 0);
        T.bnd[2 * lane + seg] = bnds[seg];
        T.shift[2 * lane + seg] = sh;
      }
    }
    if (lane == 0) T.rec[2 * nrows] = make_int4(0, INT_MAX, 0, 0);
    __syncwarp();
  }

  return total;
}

template <int M, int KIND>
__device__ __forceinline__ void short_range_f2_body(const PairKArgs& K, int blk) {
  const R4<float>* __restrict__ atoms = K.atoms;
  const int* __restrict__ cell_start = K.cell_start;
  const int ncell = K.ncell;
  const PairArgs& A = K.A;
  const PairCoef C = K.C;
  const WolfC<float> W = K.W;
  const float cwx = K.cwx;
  float* __restrict__ phis = K.phis;
  R4<float>* __restrict__ fs = K.fs;
  __shared__ QueueF queue[kWarps];
  __shared__ SegTable tables[kWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  QueueF& Q = queue[warp];
  SegTable& T = tables[warp];
  const int cell = blk * kWarps + warp;
  if (cell >= ncell) return;  // warp-uniform
  const int ncx = A.nc[0], ncy = A.nc[1];
  const int cx = cell % ncx, cy = (cell / ncx) % ncy, cz = cell / (ncx * ncy);
  const float a2 = A.a2f;
  const float FAR = 1e6f;
  const int i0 = cell_start[cell], i1 = cell_start[cell + 1];
  const int total = build_seg_table(T, K, cx, cy, cz, lane);

  for (int ib = i0; ib < i1; ib += 32) {
    const int i = ib + lane;
    const bool iv = i < i1;
    const R4<float> ai = iv ? atoms[i] : R4<float>{0.f, 0.f, 0.f, 0.f};
    float lx = iv ? ai.x : FAR, ly = iv ? ai.y : FAR, lz = iv ? ai.z : FAR;
    float hx = iv ? ai.x : -FAR, hy = iv ? ai.y : -FAR, hz = iv ? ai.z : -FAR;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lx = fminf(lx, __shfl_xor_sync(kFull, lx, o));
      ly = fminf(ly, __shfl_xor_sync(kFull, ly, o));
      lz = fminf(lz, __shfl_xor_sync(kFull, lz, o));
      hx = fmaxf(hx, __shfl_xor_sync(kFull, hx, o));
      hy = fmaxf(hy, __shfl_xor_sync(kFull, hy, o));
      hz = fmaxf(hz, __shfl_xor_sync(kFull, hz, o));
    }
    const float2 nax = make_float2(-ai.x, -ai.x), nay = make_float2(-ai.y, -ai.y), naz = make_float2(-ai.z, -ai.z);
    float phi = 0.f, px = 0.f, py = 0.f, pz = 0.f, cphi = 0.f, cpx = 0.f, cpy = 0.f, cpz = 0.f;
    // home cell: packed batches of 32 with the self test (the queue is empty here)
    for (int jb = i0; jb < i1; jb += 32) {
      const int j = jb + lane;
      const R4<float> h = (j < i1) ? atoms[j] : R4<float>{FAR, FAR, FAR, 0.f};
      Q.x[lane] = h.x;
      Q.y[lane] = h.y;
      Q.z[lane] = h.z;
      Q.q[lane] = h.w;
      __syncwarp();
      pair_batch_f2<M, KIND, 32, true>(Q, nax, nay, naz, a2, C, W, phi, px, py, pz, cphi, cpx, cpy, cpz);
      __syncwarp();
    }
    // ---- the neighbour rows: flat source index t in [0, total), 32 per step ----
    int seg = 0;  // this lane's segment cursor (t only grows)
    // source t: its atom index and cell x offset (t < total)
    auto locate = [&](int t, int& j, int& ox, float2& shv) {
      while (T.rec[seg + 1].y <= t) ++seg;
      const int4 r = T.rec[seg];
      const int4 b = T.bnd[seg];
      j = r.x + (t - r.y);
      ox = r.z + (j >= b.x) + (j >= b.y) + (j >= b.z) + (j >= b.w);
      shv = T.shift[seg];
    };
    R4<float> an = {FAR, FAR, FAR, 0.f};
    int oxn = 0;
    float2 shn = make_float2(0.f, 0.f);
    if (lane < total) {
      int j;
      locate(lane, j, oxn, shn);
      an = atoms[j];
    }
    int qn = 0;  // queued sources (warp-uniform)
    for (int t0 = 0; t0 < total; t0 += 32) {
      const bool valid = t0 + lane < total;
      R4<float> aj = an;
      const int ox = oxn;
      const float2 shv = shn;
      if (t0 + 32 + lane < total) {  // next chunk's load goes out before this chunk's work
        int j;
        locate(t0 + 32 + lane, j, oxn, shn);
        an = atoms[j];
      }
      aj.x += ox * cwx;
      aj.y += shv.x;
      aj.z += shv.y;
      const float ex = fmaxf(fmaxf(lx - aj.x, aj.x - hx), 0.f);
      const float ey = fmaxf(fmaxf(ly - aj.y, aj.y - hy), 0.f);
      const float ez = fmaxf(fmaxf(lz - aj.z, aj.z - hz), 0.f);
      const bool keep = valid && (ex * ex + ey * ey + ez * ez < a2);
      const unsigned bal = __ballot_sync(kFull, keep);
      if (keep) {
        const int p = qn + __popc(bal & ((1u << lane) - 1u));
        Q.x[p] = aj.x;
        Q.y[p] = aj.y;
        Q.z[p] = aj.z;
        Q.q[p] = aj.w;
      }
      qn += __popc(bal);
      __syncwarp();
      if (qn >= kBatch) {
        pair_batch_f2<M, KIND>(Q, nax, nay, naz, a2, C, W, phi, px, py, pz, cphi, cpx, cpy, cpz);
        __syncwarp();
        if (lane < qn - kBatch) {
          Q.x[lane] = Q.x[kBatch + lane];
          Q.y[lane] = Q.y[kBatch + lane];
          Q.z[lane] = Q.z[kBatch + lane];
          Q.q[lane] = Q.q[kBatch + lane];
        }
        qn -= kBatch;
        __syncwarp();
      }
    }
    if (qn > 0) {  // last partial batch, padded with far-away zero charges
      for (int t = lane; t < kBatch; t += 32)
        if (t >= qn) {
          Q.x[t] = FAR;
          Q.y[t] = FAR;
          Q.z[t] = FAR;
          Q.q[t] = 0.f;
        }
      __syncwarp();
      pair_batch_f2<M, KIND>(Q, nax, nay, naz, a2, C, W, phi, px, py, pz, cphi, cpx, cpy, cpz);
      __syncwarp();
    }
    if (iv) {
      phis[i] = phi + cphi;
      const float qi = ai.w;
      fs[i] = R4<float>{-qi * (px + cpx), -qi * (py + cpy), -qi * (pz + cpz), 0.f};
    }
  }
}

// ---- target clusters (mixed precision) ----
// The warp takes its cell's atoms 32 at a time (a pass) as up to kClPass
// clusters of kCl consecutive atoms (slabs of the cell across x, since
// binning sorts each cell by x), and culls every source against each
// cluster's own bounding box.  Each cluster has its own queue; a full queue of kCD
// sources is drained by the whole warp on that one cluster: lane 4 i + jl
// evaluates target i of the cluster against sources 16 jl .. 16 jl + 15
// (packed FP32x2), the four partial sums of a target are added across its
// four lanes by two shuffles, and lane 4 i + c, which owns target (c, i),
// folds them into its compensated totals.  The home cell goes through the
// scalar pair with the self test.  Queue arrays leave 4 floats of padding
// after every 16 sources, so that the four source lanes' float4 loads fall
// on distinct banks.
constexpr int kCl = 8, kClPass = 4, kCD = 64, kCQ = kCD + 32;
constexpr int kCQP = kCQ + (kCQ / 16) * 4;
__device__ __forceinline__ int cq_slot(int p) { return p + ((p >> 4) << 2); }
struct alignas(16) ClQueue {
  float x[kCQP], y[kCQP], z[kCQP], q[kCQP];
};

template <int M, int KIND>
__device__ __forceinline__ void cl_drain(const ClQueue& Q, float tx, float ty, float tz, int jl, float a2,
                                         const PairCoef& C, const WolfC<float>& W, float& s0, float& s1, float& s2,
                                         float& s3) {
  const float2 nax = make_float2(-tx, -tx), nay = make_float2(-ty, -ty), naz = make_float2(-tz, -tz);
  float2 sphi = make_float2(0.f, 0.f), sx = sphi, sy = sphi, sz = sphi;
  const int b = cq_slot(16 * jl);
#pragma unroll
  for (int k = 0; k < 16; k += 4) {
    const float4 x4 = *reinterpret_cast<const float4*>(&Q.x[b + k]);
    const float4 y4 = *reinterpret_cast<const float4*>(&Q.y[b + k]);
    const float4 z4 = *reinterpret_cast<const float4*>(&Q.z[b + k]);
    const float4 q4 = *reinterpret_cast<const float4*>(&Q.q[b + k]);
    pair2<M, KIND>(make_float2(x4.x, x4.y), make_float2(y4.x, y4.y), make_float2(z4.x, z4.y),
                   make_float2(q4.x, q4.y), nax, nay, naz, a2, C, W, sphi, sx, sy, sz);
    pair2<M, KIND>(make_float2(x4.z, x4.w), make_float2(y4.z, y4.w), make_float2(z4.z, z4.w),
                   make_float2(q4.z, q4.w), nax, nay, naz, a2, C, W, sphi, sx, sy, sz);
  }
  s0 = sphi.x + sphi.y;
  s1 = sx.x + sx.y;
  s2 = sy.x + sy.y;
  s3 = sz.x + sz.y;
}

// The four partial sums of target i, spread over lanes 4 i .. 4 i + 3, added
// (every lane of the group gets the total).
__device__ __forceinline__ void cl_reduce(float& s0, float& s1, float& s2, float& s3) {
#pragma unroll
  for (int o = 1; o <= 2; o <<= 1) {
    s0 += __shfl_xor_sync(kFull, s0, o);
    s1 += __shfl_xor_sync(kFull, s1, o);
    s2 += __shfl_xor_sync(kFull, s2, o);
    s3 += __shfl_xor_sync(kFull, s3, o);
  }
}

template <int M, int KIND>
__device__ __forceinline__ void short_range_c8_body(const PairKArgs& K, int blk) {
  const R4<float>* __restrict__ atoms = K.atoms;
  const int* __restrict__ cell_start = K.cell_start;
  const int ncell = K.ncell;
  const PairArgs& A = K.A;
  const PairCoef C = K.C;
  const WolfC<float> W = K.W;
  const float cwx = K.cwx;
  float* __restrict__ phis = K.phis;
  R4<float>* __restrict__ fs = K.fs;
  __shared__ ClQueue queues[kWarps][kClPass];
  __shared__ R4<float> home[kWarps][32];
  __shared__ SegTable tables[kWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cell = blk * kWarps + warp;
  if (cell >= ncell) return;  // warp-uniform
  const int ncx = A.nc[0], ncy = A.nc[1];
  const int cx = cell % ncx, cy = (cell / ncx) % ncy, cz = cell / (ncx * ncy);
  const float a2 = A.a2f, inv_a = A.inv_af, inv_a2s = A.inv_a2f, two_inv_a3 = A.two_inv_a3f;
  const float FAR = 1e6f;
  const int i0 = cell_start[cell], i1 = cell_start[cell + 1];
  if (i0 == i1) return;  // warp-uniform
  SegTable& T = tables[warp];
  ClQueue* Q = queues[warp];
  const int total = build_seg_table(T, K, cx, cy, cz, lane);
  const int jl = lane & 3, ti = lane >> 2;
  for (int base = i0; base < i1; base += kCl * kClPass) {
    const int ncl = min(kClPass, (i1 - base + kCl - 1) / kCl);
    // lane 4 i + c owns target (c, i), atom base + 8 c + i
    const int t_atom = base + kCl * jl + ti;
    const bool tv = t_atom < i1;
    const R4<float> ai = tv ? atoms[t_atom] : R4<float>{FAR, FAR, FAR, 0.f};
    // bounding box of each cluster (over the lanes with the same lane & 3),
    // then every cluster's box in every lane
    float lx = tv ? ai.x : FAR, ly = tv ? ai.y : FAR, lz = tv ? ai.z : FAR;
    float hx = tv ? ai.x : -FAR, hy = tv ? ai.y : -FAR, hz = tv ? ai.z : -FAR;
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) {
      lx = fminf(lx, __shfl_xor_sync(kFull, lx, o));
      ly = fminf(ly, __shfl_xor_sync(kFull, ly, o));
      lz = fminf(lz, __shfl_xor_sync(kFull, lz, o));
      hx = fmaxf(hx, __shfl_xor_sync(kFull, hx, o));
      hy = fmaxf(hy, __shfl_xor_sync(kFull, hy, o));
      hz = fmaxf(hz, __shfl_xor_sync(kFull, hz, o));
    }
    float blx[kClPass], bly[kClPass], blz[kClPass], bhx[kClPass], bhy[kClPass], bhz[kClPass];
#pragma unroll
    for (int c = 0; c < kClPass; ++c) {
      blx[c] = __shfl_sync(kFull, lx, c);
      bly[c] = __shfl_sync(kFull, ly, c);
      blz[c] = __shfl_sync(kFull, lz, c);
      bhx[c] = __shfl_sync(kFull, hx, c);
      bhy[c] = __shfl_sync(kFull, hy, c);
      bhz[c] = __shfl_sync(kFull, hz, c);
    }
    float phi = 0.f, px = 0.f, py = 0.f, pz = 0.f, cphi = 0.f, cpx = 0.f, cpy = 0.f, cpz = 0.f;
    // the home cell: cluster c's targets against all the cell's atoms, lane
    // 4 i + jl taking sources jl, jl + 4, ... (scalar, with the self test)
    for (int jb = i0; jb < i1; jb += 32) {
      const int j = jb + lane;
      home[warp][lane] = (j < i1) ? atoms[j] : R4<float>{FAR, FAR, FAR, 0.f};
      __syncwarp();
#pragma unroll 1
      for (int c = 0; c < ncl; ++c) {
        const int src = 4 * ti + c;
        const R4<float> t = {__shfl_sync(kFull, ai.x, src), __shfl_sync(kFull, ai.y, src),
                             __shfl_sync(kFull, ai.z, src), 0.f};
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k)
          pair1<float, M, KIND>(t, home[warp][jl + 4 * k], a2, inv_a, inv_a2s, two_inv_a3, W, s0, s1, s2, s3);
        cl_reduce(s0, s1, s2, s3);
        if (jl == c) {  // both paths sum grad_i u_i (scalar: f (r_i - r_j); packed: f' (r_j - r_i), f' = -f)
          two_sum_add(phi, cphi, s0);
          two_sum_add(px, cpx, s1);
          two_sum_add(py, cpy, s2);
          two_sum_add(pz, cpz, s3);
        }
      }
      __syncwarp();
    }
    // the neighbour rows: flat source index t in [0, total), 32 per step
    int seg = 0;
    auto locate = [&](int t, int& j, int& ox, float2& shv) {
      while (T.rec[seg + 1].y <= t) ++seg;
      const int4 r = T.rec[seg];
      const int4 b = T.bnd[seg];
      j = r.x + (t - r.y);
      ox = r.z + (j >= b.x) + (j >= b.y) + (j >= b.z) + (j >= b.w);
      shv = T.shift[seg];
    };
    R4<float> an = {FAR, FAR, FAR, 0.f};
    int oxn = 0;
    float2 shn = make_float2(0.f, 0.f);
    if (lane < total) {
      int j;
      locate(lane, j, oxn, shn);
      an = atoms[j];
    }
    int qn[kClPass];
#pragma unroll
    for (int c = 0; c < kClPass; ++c) qn[c] = 0;
    auto drain = [&](int c) {
      const int src = 4 * ti + c;
      const float tx = __shfl_sync(kFull, ai.x, src), ty = __shfl_sync(kFull, ai.y, src),
                  tz = __shfl_sync(kFull, ai.z, src);
      float s0, s1, s2, s3;
      cl_drain<M, KIND>(Q[c], tx, ty, tz, jl, a2, C, W, s0, s1, s2, s3);
      cl_reduce(s0, s1, s2, s3);
      if (jl == c) {
        two_sum_add(phi, cphi, s0);
        two_sum_add(px, cpx, s1);
        two_sum_add(py, cpy, s2);
        two_sum_add(pz, cpz, s3);
      }
    };
    for (int t0 = 0; t0 < total; t0 += 32) {
      const bool valid = t0 + lane < total;
      R4<float> aj = an;
      const int ox = oxn;
      const float2 shv = shn;
      if (t0 + 32 + lane < total) {  // next chunk's load goes out before this chunk's work
        int j;
        locate(t0 + 32 + lane, j, oxn, shn);
        an = atoms[j];
      }
      aj.x += ox * cwx;
      aj.y += shv.x;
      aj.z += shv.y;
      const unsigned lt = (1u << lane) - 1u;
#pragma unroll
      for (int c = 0; c < kClPass; ++c) {
        if (c < ncl) {
          const float ex = fmaxf(fmaxf(blx[c] - aj.x, aj.x - bhx[c]), 0.f);
          const float ey = fmaxf(fmaxf(bly[c] - aj.y, aj.y - bhy[c]), 0.f);
          const float ez = fmaxf(fmaxf(blz[c] - aj.z, aj.z - bhz[c]), 0.f);
          const bool keep = valid && (ex * ex + ey * ey + ez * ez < a2);
          const unsigned bal = __ballot_sync(kFull, keep);
          if (keep) {
            const int p = cq_slot(qn[c] + __popc(bal & lt));
            Q[c].x[p] = aj.x;
            Q[c].y[p] = aj.y;
            Q[c].z[p] = aj.z;
            Q[c].q[p] = aj.w;
          }
          qn[c] += __popc(bal);
        }
      }
      __syncwarp();
#pragma unroll
      for (int c = 0; c < kClPass; ++c) {
        if (c < ncl && qn[c] >= kCD) {
          drain(c);
          __syncwarp();
          if (lane < qn[c] - kCD) {
            const int from = cq_slot(kCD + lane), to = cq_slot(lane);
            Q[c].x[to] = Q[c].x[from];
            Q[c].y[to] = Q[c].y[from];
            Q[c].z[to] = Q[c].z[from];
            Q[c].q[to] = Q[c].q[from];
          }
          qn[c] -= kCD;
          __syncwarp();
        }
      }
    }
    // last partial queues, padded with far-away zero charges
#pragma unroll
    for (int c = 0; c < kClPass; ++c) {
      if (c < ncl && qn[c] > 0) {
        for (int t = qn[c] + lane; t < kCD; t += 32) {
          const int p = cq_slot(t);
          Q[c].x[p] = FAR;
          Q[c].y[p] = FAR;
          Q[c].z[p] = FAR;
          Q[c].q[p] = 0.f;
        }
        __syncwarp();
        drain(c);
        __syncwarp();
      }
    }
    if (tv) {
      phis[t_atom] = phi + cphi;
      const float qi = ai.w;
      fs[t_atom] = R4<float>{-qi * (px + cpx), -qi * (py + cpy), -qi * (pz + cpz), 0.f};
    }
  }
}

// ---- target runs (mixed precision) ----
// Warp w takes the 32 consecutive sorted atoms 32 w .. 32 w + 31 as its
// targets, whatever cells they belong to, so that no lane idles for want of
// a cell's atoms (~25 per cell at the default fill).  Binning sorts each cell
// by x and numbers cells x fastest, so a run of a cell row is a slab of it
// 32 atoms thick.  The run is cut into pieces of one row and at most three
// consecutive cells (nearly always one piece); a piece is a pass as in the
// one-cell kernel, about its first cell c0 and span s = its last cell - c0:
// the targets enter c0's frame shifted by whole cells, the home block is the
// atoms of cells c0 .. c0 + s with the self test, and the neighbour rows are
// the plan's rows widened by s cells in +x (the home row without the piece's
// own cells), walked as one flat index space, culled against the piece's
// bounding box and queued.  A periodic row then spans up to seven cells, so
// the runs need at least seven cells in x.
constexpr int kRunBnd = 6;  // boundaries inside a row segment of up to 7 cells
struct SegTableR {
  int4 rec[2 * kMaxRows + 1];         // (first atom, flat start, x offset of the first cell, -); sentinel at the end
  int4 bnd[2 * kMaxRows];             // first atom of the segment's 2nd..5th cell (INT_MAX where absent)
  int2 bnd2[2 * kMaxRows];            // ... of its 6th and 7th cell
  float2 shift[2 * kMaxRows];         // (y, z) shift of the row
};

// The segment table of the rows about cells (cx .. cx + span, cy, cz): as
// build_seg_table, each row widened by span cells in +x (the home row's
// right part moved past the piece's cells), then narrowed to the cells a
// source within a of the targets' bounding box (lx..hx, ly..hy, lz..hz, in
// the frame of cell cx) can lie in: a row at y gap gy and z gap gz from the
// box reaches sqrt(a^2 - gy^2 - gz^2) beyond it in x (with a margin for
// rounding; the culling tests each source exactly).
__device__ __forceinline__ int build_seg_table_run(SegTableR& T, const PairKArgs& K, int cx, int cy, int cz, int span,
                                                   float lx, float ly, float lz, float hx, float hy, float hz,
                                                   int lane) {
  const int* __restrict__ cell_start = K.cell_start;
  const PairArgs& A = K.A;
  const int ncx = A.nc[0], ncy = A.nc[1], ncz = A.nc[2];
  const int nrows = K.nrows;
  const float cwy = K.cwy, cwz = K.cwz;
  int len[2] = {0, 0}, j0s[2] = {0, 0}, ox0s[2] = {0, 0};
  int bb[2][kRunBnd];
#pragma unroll
  for (int g = 0; g < 2; ++g)
#pragma unroll
    for (int t = 0; t < kRunBnd; ++t) bb[g][t] = INT_MAX;
  float2 sh = make_float2(0.f, 0.f);
  if (lane < nrows) {
    int4 row = K.rows[lane];  // (dy, dz, xlo, xhi)
    if (row.x == 0 && row.y == 0) {
      if (row.z > 0) { row.z += span; row.w += span; }  // the home row's right part
    } else {
      row.w += span;
    }
    const float gy = fmaxf(fmaxf(row.x * cwy - hy, ly - (row.x + 1) * cwy), 0.f);
    const float gz = fmaxf(fmaxf(row.y * cwz - hz, lz - (row.y + 1) * cwz), 0.f);
    const float r2 = A.a2f - gy * gy - gz * gz;
    bool inside = r2 > 0.f;
    if (inside) {
      const float reach = sqrtf(r2) * 1.0001f + 1e-3f;
      row.z = max(row.z, (int)floorf((lx - reach) / K.cwx));
      row.w = min(row.w, (int)floorf((hx + reach) / K.cwx));
      inside = row.z <= row.w;
    }
    int ny = cy + row.x, nz = cz + row.y;
    if (A.periodic) {
      ny += (ny < 0) ? ncy : ((ny >= ncy) ? -ncy : 0);
      nz += (nz < 0) ? ncz : ((nz >= ncz) ? -ncz : 0);
    } else if (ny < 0 || nz < 0 || ny >= ncy || nz >= ncz) {
      inside = false;
    }
    const int rbase = (nz * ncy + ny) * ncx;
    sh = make_float2(row.x * cwy, row.y * cwz);
#pragma unroll
    for (int seg = 0; seg < 2; ++seg) {
      int ox0 = 0, ox1 = -1;
      if (!inside) {
      } else if (A.periodic) {  // at most 7 <= ncx cells: the row wraps at one end at most
        const int xa = cx + row.z, xb = cx + row.w;
        if (xa < 0) {
          if (seg == 0) { ox0 = row.z; ox1 = -cx - 1; } else { ox0 = -cx; ox1 = row.w; }
        } else if (xb >= ncx) {
          if (seg == 0) { ox0 = row.z; ox1 = ncx - 1 - cx; } else { ox0 = ncx - cx; ox1 = row.w; }
        } else if (seg == 0) {
          ox0 = row.z; ox1 = row.w;
        }
      } else if (seg == 0) {
        ox0 = max(row.z, -cx);
        ox1 = min(row.w, ncx - 1 - cx);
      }
      if (ox0 <= ox1) {
        int x0 = cx + ox0, x1 = cx + ox1;
        if (A.periodic) {
          x0 += (x0 < 0) ? ncx : ((x0 >= ncx) ? -ncx : 0);
          x1 += (x1 < 0) ? ncx : ((x1 >= ncx) ? -ncx : 0);
        }
        const int j0 = cell_start[rbase + x0], j1 = cell_start[rbase + x1 + 1];
#pragma unroll
        for (int t = 0; t < kRunBnd; ++t) bb[seg][t] = (x0 + 1 + t <= x1) ? cell_start[rbase + x0 + 1 + t] : INT_MAX;
        len[seg] = j1 - j0;
        j0s[seg] = j0;
        ox0s[seg] = ox0;
      }
    }
  }
  const int mine = len[0] + len[1];
  int incl = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  const int total = __shfl_sync(kFull, incl, 31);
  const int start = incl - mine;
  if (lane < nrows) {
#pragma unroll
    for (int seg = 0; seg < 2; ++seg) {
      T.rec[2 * lane + seg] = make_int4(j0s[seg], seg ? start + len[0] : start, ox0s[seg], 0);
      T.bnd[2 * lane + seg] = make_int4(bb[seg][0], bb[seg][1], bb[seg][2], bb[seg][3]);
      T.bnd2[2 * lane + seg] = make_int2(bb[seg][4], bb[seg][5]);
      T.shift[2 * lane + seg] = sh;
    }
  }
  if (lane == 0) T.rec[2 * nrows] = make_int4(0, INT_MAX, 0, 0);
  __syncwarp();
  return total;
}

template <int M, int KIND>
__device__ __forceinline__ void short_range_run_body(const PairKArgs& K, int blk) {
  const R4<float>* __restrict__ atoms = K.atoms;
  const int* __restrict__ cell_start = K.cell_start;
  const PairArgs& A = K.A;
  const PairCoef C = K.C;
  const WolfC<float> W = K.W;
  const float cwx = K.cwx;
  float* __restrict__ phis = K.phis;
  R4<float>* __restrict__ fs = K.fs;
  __shared__ QueueF queue[kWarps];
  __shared__ SegTableR tables[kWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  QueueF& Q = queue[warp];
  SegTableR& T = tables[warp];
  const int s0 = 32 * (blk * kWarps + warp);
  if (s0 >= K.natoms) return;  // warp-uniform
  const int nval = min(32, K.natoms - s0);
  const int ncx = A.nc[0], ncy = A.nc[1];
  const float a2 = A.a2f;
  const float FAR = 1e6f;
  // the lane's target: its sorted record and its cell (cells ascend with the lane)
  const bool sv = lane < nval;
  const int mycell = sv ? K.key[K.perm[s0 + lane]] : INT_MAX;
  const R4<float> me = sv ? atoms[s0 + lane] : R4<float>{0.f, 0.f, 0.f, 0.f};
  for (int l0 = 0; l0 < nval;) {  // one piece per step (warp-uniform)
    const int c0 = __shfl_sync(kFull, mycell, l0);
    const int cx = c0 % ncx, cy = (c0 / ncx) % ncy, cz = c0 / (ncx * ncy);
    const int climit = c0 + min(2, ncx - 1 - cx);  // the piece stays in the row, three cells at most
    const bool inp = lane >= l0 && mycell <= climit;  // lanes l0 .. l1 - 1
    const unsigned pb = __ballot_sync(kFull, inp);
    const int l1 = 32 - __clz(pb);
    const int span = __shfl_sync(kFull, mycell, l1 - 1) - c0;
    // cell boundaries inside the piece: atoms of cell c0 + 1 and c0 + 2 begin here
    const int h0 = cell_start[c0];
    const int b1 = span >= 1 ? cell_start[c0 + 1] : INT_MAX;
    const int b2 = span >= 2 ? cell_start[c0 + 2] : INT_MAX;
    const int h1 = cell_start[c0 + span + 1];
    // the target in c0's frame
    R4<float> ai = me;
    ai.x = __fmaf_rn((float)(inp ? mycell - c0 : 0), cwx, ai.x);  // the same rounding as the home block's
    float lx = inp ? ai.x : FAR, ly = inp ? ai.y : FAR, lz = inp ? ai.z : FAR;
    float hx = inp ? ai.x : -FAR, hy = inp ? ai.y : -FAR, hz = inp ? ai.z : -FAR;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lx = fminf(lx, __shfl_xor_sync(kFull, lx, o));
      ly = fminf(ly, __shfl_xor_sync(kFull, ly, o));
      lz = fminf(lz, __shfl_xor_sync(kFull, lz, o));
      hx = fmaxf(hx, __shfl_xor_sync(kFull, hx, o));
      hy = fmaxf(hy, __shfl_xor_sync(kFull, hy, o));
      hz = fmaxf(hz, __shfl_xor_sync(kFull, hz, o));
    }
    const float2 nax = make_float2(-ai.x, -ai.x), nay = make_float2(-ai.y, -ai.y), naz = make_float2(-ai.z, -ai.z);
    float phi = 0.f, px = 0.f, py = 0.f, pz = 0.f, cphi = 0.f, cpx = 0.f, cpy = 0.f, cpz = 0.f;
    // the home block: the atoms of the piece's cells, 32 at a time, with the self test
    for (int jb = h0; jb < h1; jb += 32) {
      const int j = jb + lane;
      R4<float> h = (j < h1) ? atoms[j] : R4<float>{FAR, FAR, FAR, 0.f};
      if (j < h1) h.x = __fmaf_rn((float)((j >= b1) + (j >= b2)), cwx, h.x);
      Q.x[lane] = h.x;
      Q.y[lane] = h.y;
      Q.z[lane] = h.z;
      Q.q[lane] = h.w;
      __syncwarp();
      pair_batch_f2<M, KIND, 32, true>(Q, nax, nay, naz, a2, C, W, phi, px, py, pz, cphi, cpx, cpy, cpz);
      __syncwarp();
    }
    // the neighbour rows: flat source index t in [0, total), 32 per step
    const int total = build_seg_table_run(T, K, cx, cy, cz, span, lx, ly, lz, hx, hy, hz, lane);
    int seg = 0;
    auto locate = [&](int t, int& j, int& ox, float2& shv) {
      while (T.rec[seg + 1].y <= t) ++seg;
      const int4 r = T.rec[seg];
      const int4 b = T.bnd[seg];
      const int2 b2 = T.bnd2[seg];
      j = r.x + (t - r.y);
      ox = r.z + (j >= b.x) + (j >= b.y) + (j >= b.z) + (j >= b.w) + (j >= b2.x) + (j >= b2.y);
      shv = T.shift[seg];
    };
    R4<float> an = {FAR, FAR, FAR, 0.f};
    int oxn = 0;
    float2 shn = make_float2(0.f, 0.f);
    if (lane < total) {
      int j;
      locate(lane, j, oxn, shn);
      an = atoms[j];
    }
    int qn = 0;
    for (int t0 = 0; t0 < total; t0 += 32) {
      const bool valid = t0 + lane < total;
      R4<float> aj = an;
      const int ox = oxn;
      const float2 shv = shn;
      if (t0 + 32 + lane < total) {
        int j;
        locate(t0 + 32 + lane, j, oxn, shn);
        an = atoms[j];
      }
      aj.x += ox * cwx;
      aj.y += shv.x;
      aj.z += shv.y;
      const float ex = fmaxf(fmaxf(lx - aj.x, aj.x - hx), 0.f);
      const float ey = fmaxf(fmaxf(ly - aj.y, aj.y - hy), 0.f);
      const float ez = fmaxf(fmaxf(lz - aj.z, aj.z - hz), 0.f);
      const bool keep = valid && (ex * ex + ey * ey + ez * ez < a2);
      const unsigned bal = __ballot_sync(kFull, keep);
      if (keep) {
        const int p = qn + __popc(bal & ((1u << lane) - 1u));
        Q.x[p] = aj.x;
        Q.y[p] = aj.y;
        Q.z[p] = aj.z;
        Q.q[p] = aj.w;
      }
      qn += __popc(bal);
      __syncwarp();
      if (qn >= kBatch) {
        pair_batch_f2<M, KIND>(Q, nax, nay, naz, a2, C, W, phi, px, py, pz, cphi, cpx, cpy, cpz);
        __syncwarp();
        if (lane < qn - kBatch) {
          Q.x[lane] = Q.x[kBatch + lane];
          Q.y[lane] = Q.y[kBatch + lane];
          Q.z[lane] = Q.z[kBatch + lane];
          Q.q[lane] = Q.q[kBatch + lane];
        }
        qn -= kBatch;
        __syncwarp();
      }
    }
    if (qn > 0) {  // last partial batch, padded with far-away zero charges
      for (int t = lane; t < kBatch; t += 32)
        if (t >= qn) {
          Q.x[t] = FAR;
          Q.y[t] = FAR;
          Q.z[t] = FAR;
          Q.q[t] = 0.f;
        }
      __syncwarp();
      pair_batch_f2<M, KIND>(Q, nax, nay, naz, a2, C, W, phi, px, py, pz, cphi, cpx, cpy, cpz);
      __syncwarp();
    }
    if (inp) {
      const int i = s0 + lane;
      phis[i] = phi + cphi;
      const float qi = me.w;
      fs[i] = R4<float>{-qi * (px + cpx), -qi * (py + cpy), -qi * (pz + cpz), 0.f};
    }
    l0 = l1;
  }
}

template <int M, int KIND>
__global__ void __launch_bounds__(32 * kWarps, MSM_PAIR_MINB) k_short_range_run(PairKArgs a) {
  short_range_run_body<M, KIND>(a, blockIdx.x);
}

template <int M>
__global__ void __launch_bounds__(32 * kWarps, MSM_PAIR_MINB) kb_short_range_run(const PairKArgs* __restrict__ tab,
                                                                   const int* __restrict__ first, int nrep) {
  const int r = batch_rep(first, nrep, blockIdx.x);
  short_range_run_body<M, kPairMSM>(tab[r], blockIdx.x - first[r]);
}

template <int M, int KIND>
__global__ void __launch_bounds__(32 * kWarps, MSM_PAIR_MINB) k_short_range_f2(PairKArgs a) {
  short_range_f2_body<M, KIND>(a, blockIdx.x);
}

template <int M, int KIND>
__global__ void __launch_bounds__(32 * kWarps, 4) k_short_range_c8(PairKArgs a) {
  short_range_c8_body<M, KIND>(a, blockIdx.x);
}

template <int M>
__global__ void __launch_bounds__(32 * kWarps, 4) kb_short_range_c8(const PairKArgs* __restrict__ tab,
                                                                   const int* __restrict__ first, int nrep) {
  const int r = batch_rep(first, nrep, blockIdx.x);
  short_range_c8_body<M, kPairMSM>(tab[r], blockIdx.x - first[r]);
}

template <int M>
__global__ void __launch_bounds__(32 * kWarps, MSM_PAIR_MINB) kb_short_range_f2(const PairKArgs* __restrict__ tab,
                                                                   const int* __restrict__ first, int nrep) {
  const int r = batch_rep(first, nrep, blockIdx.x);
  short_range_f2_body<M, kPairMSM>(tab[r], blockIdx.x - first[r]);
}

template <typename T, bool COMP, int K>
void launch_t(Plan& P, cudaStream_t st, double alpha = 0.0) {
  PairArgs A = pair_args(P);
  const WolfC<T> W = wolf_consts<T>(alpha, P.P.cutoff);
  int blocks = (P.ncell + kWarps - 1) / kWarps;
  auto* at = (const R4<T>*)P.d.atoms;
  auto* sh = (const R4<T>*)P.d.cell_shift;
  auto* ph = (T*)P.d.phis;
  auto* fs = (R4<T>*)P.d.fs;
  switch (P.P.splitting) {
    case 1:
      k_short_range<T, 1, COMP, K><<<blocks, 32 * kWarps, 0, st>>>(at, P.d.cell_start, P.d.cell_off, sh, A, W,
                                                               P.ncell, ph, fs);
      break;
    case 2:
      k_short_range<T, 2, COMP, K><<<blocks, 32 * kWarps, 0, st>>>(at, P.d.cell_start, P.d.cell_off, sh, A, W,
                                                               P.ncell, ph, fs);
      break;
    default:
      k_short_range<T, 3, COMP, K><<<blocks, 32 * kWarps, 0, st>>>(at, P.d.cell_start, P.d.cell_off, sh, A, W,
                                                               P.ncell, ph, fs);
      break;
  }
}

}  // namespace

PairKArgs pair_kargs(const Plan& P) {
  PairKArgs K;
  K.A = pair_args(P);
  K.W = wolf_consts<float>(0.0, P.P.cutoff);
  K.atoms = (const R4<float>*)P.d.atoms;
  K.cell_start = P.d.cell_start;
  K.rows = P.d.cell_rows;
  K.nrows = P.nrows;
  K.ncell = P.ncell;
  K.phis = (float*)P.d.phis;
  K.fs = (R4<float>*)P.d.fs;
  // gamma coefficients c_k (Taylor series of s^(-1/2) about s = 1, truncated at m)
  static const double c[4][4] = {{0, 0, 0, 0}, {1.5, -0.5, 0, 0}, {1.875, -1.25, 0.375, 0},
                                 {2.1875, -2.1875, 1.3125, -0.3125}};
  const int m = P.P.splitting;
  const double a = P.P.cutoff;
  for (int k = 0; k < 4; ++k) {
    float g = (k <= m) ? (float)(-c[m][k] / std::pow(a, 2 * k + 1)) : 0.f;
    K.C.G[k] = make_float2(g, g);
  }
  for (int k = 0; k < 3; ++k) {
    float d = (k + 1 <= m) ? (float)(2.0 * (k + 1) * c[m][k + 1] / std::pow(a, 2 * k + 3)) : 0.f;
    K.C.D[k] = make_float2(d, d);
  }
  K.cwx = (float)P.cw[0];
  K.cwy = (float)P.cw[1];
  K.cwz = (float)P.cw[2];
  K.key = P.d.key;
  K.perm = P.d.perm;
  K.natoms = 0;
  return K;
}

// Target runs apply to a plan whose pair kernel takes a cell's targets
// (pair_targets 32) and whose periodic rows hold at least seven cells.
static bool use_runs(const Plan& P) {
  return P.pair_runs && P.pair_targets != kCl && (!P.P.periodic || P.nc[0] >= 7);
}

template <int KIND>
void launch_f2(Plan& P, int64_t n, cudaStream_t st, double alpha = 0.0) {
  PairKArgs K = pair_kargs(P);
  K.W = wolf_consts<float>(alpha, P.P.cutoff);
  K.natoms = (int)n;
  const int blocks = (P.ncell + kWarps - 1) / kWarps;
  if (use_runs(P)) {  // runs of 32 consecutive atoms
    const int br = (int)(((n + 31) / 32 + kWarps - 1) / kWarps);
    if (KIND == kPairCutoff) k_short_range_run<2, kPairCutoff><<<br, 32 * kWarps, 0, st>>>(K);  // M unused
    else if (KIND == kPairWolf) k_short_range_run<2, kPairWolf><<<br, 32 * kWarps, 0, st>>>(K);
    else if (P.P.splitting == 1) k_short_range_run<1, kPairMSM><<<br, 32 * kWarps, 0, st>>>(K);
    else if (P.P.splitting == 2) k_short_range_run<2, kPairMSM><<<br, 32 * kWarps, 0, st>>>(K);
    else k_short_range_run<3, kPairMSM><<<br, 32 * kWarps, 0, st>>>(K);
    return;
  }
  if (P.pair_targets == kCl) {  // clusters of 8 targets
    if (KIND == kPairCutoff) k_short_range_c8<2, kPairCutoff><<<blocks, 32 * kWarps, 0, st>>>(K);  // M unused
    else if (KIND == kPairWolf) k_short_range_c8<2, kPairWolf><<<blocks, 32 * kWarps, 0, st>>>(K);
    else if (P.P.splitting == 1) k_short_range_c8<1, kPairMSM><<<blocks, 32 * kWarps, 0, st>>>(K);
    else if (P.P.splitting == 2) k_short_range_c8<2, kPairMSM><<<blocks, 32 * kWarps, 0, st>>>(K);
    else k_short_range_c8<3, kPairMSM><<<blocks, 32 * kWarps, 0, st>>>(K);
    return;
  }
  if (KIND == kPairCutoff) k_short_range_f2<2, kPairCutoff><<<blocks, 32 * kWarps, 0, st>>>(K);  // M unused
  else if (KIND == kPairWolf) k_short_range_f2<2, kPairWolf><<<blocks, 32 * kWarps, 0, st>>>(K);
  else if (P.P.splitting == 1) k_short_range_f2<1, kPairMSM><<<blocks, 32 * kWarps, 0, st>>>(K);
  else if (P.P.splitting == 2) k_short_range_f2<2, kPairMSM><<<blocks, 32 * kWarps, 0, st>>>(K);
  else k_short_range_f2<3, kPairMSM><<<blocks, 32 * kWarps, 0, st>>>(K);
}

cudaError_t launch_short_range(Plan& P, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (P.fp64) launch_t<double, false, kPairMSM>(P, st);
  else launch_f2<kPairMSM>(P, n, st);
  P.launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_cutoff_pairs(Plan& P, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (P.fp64) launch_t<double, false, kPairCutoff>(P, st);
  else launch_f2<kPairCutoff>(P, n, st);
  P.launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_wolf_pairs(Plan& P, int64_t n, double alpha, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (P.fp64) launch_t<double, false, kPairWolf>(P, st, alpha);
  else launch_f2<kPairWolf>(P, n, st, alpha);
  P.launches += 1;
  return cudaGetLastError();
}

struct PairBatch {
  BatchTable<PairKArgs> cells;  // kWarps cells (or target runs) per block
  int splitting = 2;
  int targets = 8;  // the first replica's pair_targets
  bool runs = false;  // every replica takes target runs
};

cudaError_t pair_batch_build(const std::vector<BatchRep>& reps, PairBatch** out) {
  *out = nullptr;
  PairBatch* b = new (std::nothrow) PairBatch();
  if (!b) return cudaErrorMemoryAllocation;
  std::vector<PairKArgs> ka;
  std::vector<int> kb;
  b->runs = !reps.empty();
  for (const BatchRep& r : reps) b->runs = b->runs && use_runs(*r.plan);
  for (const BatchRep& r : reps) {
    PairKArgs K = pair_kargs(*r.plan);
    K.natoms = (int)r.n;
    ka.push_back(K);
    if (b->runs) kb.push_back(r.n > 0 ? (int)(((r.n + 31) / 32 + kWarps - 1) / kWarps) : 0);
    else kb.push_back(r.n > 0 ? (r.plan->ncell + kWarps - 1) / kWarps : 0);
    b->splitting = r.plan->P.splitting;
  }
  if (!reps.empty()) b->targets = reps[0].plan->pair_targets;
  cudaError_t e = make_table(b->cells, ka, kb);
  if (e != cudaSuccess) {
    pair_batch_free(b);
    return e;
  }
  *out = b;
  return cudaSuccess;
}

cudaError_t pair_batch_launch(PairBatch* b, cudaStream_t st) {
  const int nb = b->cells.total;
  if (nb == 0) return cudaSuccess;
  if (b->runs) {
    if (b->splitting == 1) kb_short_range_run<1><<<nb, 32 * kWarps, 0, st>>>(b->cells.args, b->cells.first, b->cells.nrep);
    else if (b->splitting == 2)
      kb_short_range_run<2><<<nb, 32 * kWarps, 0, st>>>(b->cells.args, b->cells.first, b->cells.nrep);
    else kb_short_range_run<3><<<nb, 32 * kWarps, 0, st>>>(b->cells.args, b->cells.first, b->cells.nrep);
    return cudaGetLastError();
  }
  if (b->targets == kCl) {
    if (b->splitting == 1) kb_short_range_c8<1><<<nb, 32 * kWarps, 0, st>>>(b->cells.args, b->cells.first, b->cells.nrep);
    else if (b->splitting == 2)
      kb_short_range_c8<2><<<nb, 32 * kWarps, 0, st>>>(b->cells.args, b->cells.first, b->cells.nrep);
    else kb_short_range_c8<3><<<nb, 32 * kWarps, 0, st>>>(b->cells.args, b->cells.first, b->cells.nrep);
    return cudaGetLastError();
  }
  if (b->splitting == 1) kb_short_range_f2<1><<<nb, 32 * kWarps, 0, st>>>(b->cells.args, b->cells.first, b->cells.nrep);
  else if (b->splitting == 2) kb_short_range_f2<2><<<nb, 32 * kWarps, 0, st>>>(b->cells.args, b->cells.first, b->cells.nrep);
  else kb_short_range_f2<3><<<nb, 32 * kWarps, 0, st>>>(b->cells.args, b->cells.first, b->cells.nrep);
  return cudaGetLastError();
}

void pair_batch_free(PairBatch* b) {
  if (!b) return;
  b->cells.release();
  delete b;
}

}  // namespace msm
