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

struct PairArgs {
  int nc[3];
  int periodic;
  int noff;
  double a;
};

constexpr int kWarps = 4;
constexpr int kBatch = 32;       // pairs per lane per batch (one queue drain)
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float fast_rsqrt(float x) {  // one MUFU.RSQ; inputs are >= a^2/... never denormal
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ double fast_rsqrt(double x) { return rsqrt(x); }

template <typename T>
__device__ __forceinline__ T far_away() { return T(1e18); }

// One batch: the lane's target atom against the kBatch queued sources.
template <typename T, int M, bool COMP>
__device__ __forceinline__ void pair_batch(const R4<T>* __restrict__ Q, const R4<T>& ai, T a2, T inv_a,
                                           T inv_a2, T two_inv_a3, T& phi, T& fx, T& fy, T& fz, T& cphi,
                                           T& cfx, T& cfy, T& cfz) {
  T pphi = 0, px = 0, py = 0, pz = 0;
#pragma unroll 8
  for (int jj = 0; jj < kBatch; ++jj) {
    const R4<T> b = Q[jj];
    const T dx = ai.x - b.x, dy = ai.y - b.y, dz = ai.z - b.z;
    const T r2 = dx * dx + dy * dy + dz * dz;
    const bool ok = (r2 < a2) && (r2 > T(0));   // inside the cutoff, not the atom itself
    const T r2s = ok ? r2 : a2;
    const T qj = ok ? b.w : T(0);
    const T rinv = fast_rsqrt(r2s);
    const T s = r2s * inv_a2;
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
}

// One warp per cell.  For every neighbour cell in reach, the warp stages 32
// source atoms at a time (shifted into the target cell's frame), drops those
// farther than a from the bounding box of its target atoms, and appends the
// rest to a per-warp queue in shared memory; each full queue of kBatch
// sources is one fully unrolled batch of pair evaluations.
template <typename T, int M, bool COMP>
__global__ void __launch_bounds__(32 * kWarps) k_short_range(
    const R4<T>* __restrict__ atoms, const int* __restrict__ cell_start,
    const int4* __restrict__ offs, const R4<T>* __restrict__ shifts, PairArgs A, int ncell,
    T* __restrict__ phis, R4<T>* __restrict__ fs) {
  __shared__ R4<T> queue[kWarps][2 * kBatch];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  R4<T>* Q = queue[warp];
  const int cell = blockIdx.x * kWarps + warp;
  if (cell >= ncell) return;  // warp-uniform
  const int cx = cell % A.nc[0], cy = (cell / A.nc[0]) % A.nc[1], cz = cell / (A.nc[0] * A.nc[1]);
  const T a2 = T(A.a * A.a), inv_a = T(1.0 / A.a), inv_a2 = T(1.0 / (A.a * A.a));
  const T two_inv_a3 = T(2.0 / (A.a * A.a * A.a));
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
          pair_batch<T, M, COMP>(Q, ai, a2, inv_a, inv_a2, two_inv_a3, phi, fx, fy, fz, cphi, cfx, cfy, cfz);
          __syncwarp();
          if (lane < qn - kBatch) Q[lane] = Q[kBatch + lane];
          qn -= kBatch;
          __syncwarp();
        }
      }
    }
    if (qn > 0) {  // last partial batch, padded with far-away zero charges
      if (lane >= qn) Q[lane] = dummy;
      __syncwarp();
      pair_batch<T, M, COMP>(Q, ai, a2, inv_a, inv_a2, two_inv_a3, phi, fx, fy, fz, cphi, cfx, cfy, cfz);
      __syncwarp();
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
  for (int d = 0; d < 3; ++d) A.nc[d] = P.nc[d];
  A.periodic = P.P.periodic;
  A.noff = P.noff;
  A.a = P.P.cutoff;
  int blocks = (P.ncell + kWarps - 1) / kWarps;
  auto* at = (const R4<T>*)P.d.atoms;
  auto* sh = (const R4<T>*)P.d.cell_shift;
  auto* ph = (T*)P.d.phis;
  auto* fs = (R4<T>*)P.d.fs;
  switch (P.P.splitting) {
    case 1:
      k_short_range<T, 1, COMP><<<blocks, 32 * kWarps, 0, st>>>(at, P.d.cell_start, P.d.cell_off, sh, A,
                                                               P.ncell, ph, fs);
      break;
    case 2:
      k_short_range<T, 2, COMP><<<blocks, 32 * kWarps, 0, st>>>(at, P.d.cell_start, P.d.cell_off, sh, A,
                                                               P.ncell, ph, fs);
      break;
    default:
      k_short_range<T, 3, COMP><<<blocks, 32 * kWarps, 0, st>>>(at, P.d.cell_start, P.d.cell_off, sh, A,
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
