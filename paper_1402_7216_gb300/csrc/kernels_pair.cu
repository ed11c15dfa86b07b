// kernels_pair.cu -- short-range part of MSM (Sec. "Multilevel Summation
// Method"): u_i^short = sum_{j != i, r_ij < a} q_j g*(r_ij) with
// g*(r) = 1/r - gamma(r/a)/a (Eq. msmgrid), and the force
// F_i = -q_i grad_i u_i^short.
//
// One warp owns one cell of the sort-binned atoms (cells at least a/2 wide):
// its lanes hold up to 32 target atoms and walk the neighbour cells within
// reach (offsets whose closest points are nearer than a).  Source atoms of a
// neighbour cell are staged in the warp's shared memory (shifted into the
// target cell's frame, so every difference is between small cell-local
// coordinates) and broadcast to the lanes.  Each pair costs one rsqrt and
// ~20 FP32 operations; rejected pairs are masked, not branched.  Mixed
// precision sums each staged chunk in FP32 and folds the chunk sums into the
// running totals with an error-free TwoSum (compensated accumulation).
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

__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }

// error-free transformation s + x = t + err; the error goes to the compensation term
template <typename T>
__device__ __forceinline__ void two_sum_add(T& s, T& c, T x) {
  T t = s + x;
  T bp = t - s;
  c += (s - (t - bp)) + (x - bp);
  s = t;
}

struct PairArgs {
  int nc[3];
  double cw[3];
  int periodic;
  int noff;
  double a;
};

constexpr int kWarps = 4;

template <typename T, int M, bool COMP>
__global__ void __launch_bounds__(32 * kWarps) k_short_range(
    const R4<T>* __restrict__ atoms, const int* __restrict__ cell_start,
    const int4* __restrict__ offs, PairArgs A, int ncell, T* __restrict__ phis,
    R4<T>* __restrict__ fs) {
  __shared__ R4<T> sj[kWarps][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cell = blockIdx.x * kWarps + warp;
  if (cell >= ncell) return;  // warp-uniform
  const int cx = cell % A.nc[0], cy = (cell / A.nc[0]) % A.nc[1], cz = cell / (A.nc[0] * A.nc[1]);
  const T a2 = T(A.a * A.a), inv_a = T(1.0 / A.a), inv_a2 = T(1.0 / (A.a * A.a));
  const T two_inv_a3 = T(2.0 / (A.a * A.a * A.a));
  const int i0 = cell_start[cell], i1 = cell_start[cell + 1];
  for (int ib = i0; ib < i1; ib += 32) {
    const int i = ib + lane;
    const bool iv = i < i1;
    R4<T> ai = iv ? atoms[i] : R4<T>{T(0), T(0), T(0), T(0)};
    T phi = 0, fx = 0, fy = 0, fz = 0;
    T cphi = 0, cfx = 0, cfy = 0, cfz = 0;
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
      const T sx = T(off.x * A.cw[0]), sy = T(off.y * A.cw[1]), sz = T(off.z * A.cw[2]);
      const int j0 = cell_start[nb], j1 = cell_start[nb + 1];
      for (int jb = j0; jb < j1; jb += 32) {
        const int j = jb + lane;
        if (j < j1) {
          R4<T> aj = atoms[j];
          aj.x += sx;
          aj.y += sy;
          aj.z += sz;
          sj[warp][lane] = aj;
        }
        __syncwarp();
        const int cnt = min(32, j1 - jb);
        T pphi = 0, px = 0, py = 0, pz = 0;
        for (int jj = 0; jj < cnt; ++jj) {
          const R4<T> b = sj[warp][jj];
          const T dx = ai.x - b.x, dy = ai.y - b.y, dz = ai.z - b.z;
          const T r2 = dx * dx + dy * dy + dz * dz;
          const bool ok = (r2 < a2) && (r2 > T(0));
          const T r2s = ok ? r2 : a2;
          const T rinv = rsq(r2s);
          const T s = r2s * inv_a2;
          const T qj = ok ? b.w : T(0);
          pphi += qj * (rinv - Smooth<T, M>::g(s) * inv_a);
          const T f = qj * (-(rinv * rinv * rinv) - two_inv_a3 * Smooth<T, M>::gs(s));
          px += f * dx;
          py += f * dy;
          pz += f * dz;
        }
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
        __syncwarp();
      }
    }
    if (iv) {
      phis[i] = phi + cphi;
      const T qi = ai.w;
      fs[i] = R4<T>{-qi * (fx + cfx), -qi * (fy + cfy), -qi * (fz + cfz), T(0)};
    }
  }
}

template <typename T, bool COMP>
void launch_t(Plan& P, cudaStream_t st) {
  PairArgs A;
  for (int d = 0; d < 3; ++d) {
    A.nc[d] = P.nc[d];
    A.cw[d] = P.cw[d];
  }
  A.periodic = P.P.periodic;
  A.noff = P.noff;
  A.a = P.P.cutoff;
  int blocks = (P.ncell + kWarps - 1) / kWarps;
  auto* at = (const R4<T>*)P.d.atoms;
  auto* ph = (T*)P.d.phis;
  auto* fs = (R4<T>*)P.d.fs;
  switch (P.P.splitting) {
    case 1:
      k_short_range<T, 1, COMP><<<blocks, 32 * kWarps, 0, st>>>(at, P.d.cell_start, P.d.cell_off, A,
                                                               P.ncell, ph, fs);
      break;
    case 2:
      k_short_range<T, 2, COMP><<<blocks, 32 * kWarps, 0, st>>>(at, P.d.cell_start, P.d.cell_off, A,
                                                               P.ncell, ph, fs);
      break;
    default:
      k_short_range<T, 3, COMP><<<blocks, 32 * kWarps, 0, st>>>(at, P.d.cell_start, P.d.cell_off, A,
                                                               P.ncell, ph, fs);
      break;
  }
}

}  // namespace

cudaError_t launch_short_range(Plan& P, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (P.fp64) launch_t<double, false>(P, st);
  else launch_t<float, true>(P, st);
  P.launches += 1;
  return cudaGetLastError();
}

}  // namespace msm
