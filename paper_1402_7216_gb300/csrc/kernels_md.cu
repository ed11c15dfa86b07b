// kernels_md.cu -- molecular dynamics around the MSM force: the velocity
// Verlet scheme of the thesis proposal (Sec. "Molecular Dynamics"): from
// r(t), v(t) and a(t) = F(t)/m,
//   v(t + dt/2) = v(t) + a(t) dt/2,  r(t + dt) = r(t) + v(t + dt/2) dt,
//   F(t + dt) from U(r(t + dt)),     v(t + dt) = v(t + dt/2) + a(t + dt) dt/2.
// The force evaluation between the two half steps is the ordinary MSM
// evaluation; these kernels are the drift before it and the kick after it,
// with the step's energies and momentum reduced in a fixed order (the record
// does not depend on scheduling).  Everything is FP64: the per-atom work is a
// few operations against one MSM evaluation, and FP64 keeps the trajectory
// state exact to the caller's precision.
#include "msm_internal.h"

namespace msm {
namespace {

constexpr int kMdThreads = 256;

struct MdBox {
  double L[3], inv_L[3];
  int periodic;
};

// v += a dt/2, r += v dt, and a periodic box wraps r back into [0, L).
__global__ void __launch_bounds__(kMdThreads) k_md_drift(int64_t n, double* __restrict__ pos,
                                                          double* __restrict__ vel, const double* __restrict__ force,
                                                          const double* __restrict__ inv_mass, double dt, MdBox B) {
  const double half = 0.5 * dt;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double im = inv_mass[i];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double v = vel[3 * i + d] + half * im * force[3 * i + d];
      double x = pos[3 * i + d] + dt * v;
      if (B.periodic) {
        x -= B.L[d] * floor(x * B.inv_L[d]);
        if (x >= B.L[d]) x -= B.L[d];  // rounding of the product can land on L itself
        if (x < 0.0) x = 0.0;
      }
      vel[3 * i + d] = v;
      pos[3 * i + d] = x;
    }
  }
}

// Fixed-order block sum of four values (thread 0 returns them).
__device__ __forceinline__ void block_sum4(double v[4]) {
  __shared__ double red[kMdThreads / 32][4];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < 4; ++c)
    for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
  if (lane == 0)
#pragma unroll
    for (int c = 0; c < 4; ++c) red[w][c] = v[c];
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      v[c] = lane < kMdThreads / 32 ? red[lane][c] : 0.0;
      for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
    }
  }
}

// v += a dt/2 with the new force, then per-block kinetic energy 1/2 m v^2
// and momentum m v (atoms with inv_mass 0 are fixed: they take no kick and
// carry neither).
__global__ void __launch_bounds__(kMdThreads) k_md_kick(int64_t n, double* __restrict__ vel,
                                                         const double* __restrict__ force,
                                                         const double* __restrict__ inv_mass, double dt,
                                                         double* __restrict__ partial) {
  const double half = 0.5 * dt;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double im = inv_mass[i];
    double v[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      v[d] = vel[3 * i + d] + half * im * force[3 * i + d];
      vel[3 * i + d] = v[d];
    }
    if (im > 0.0) {
      const double m = 1.0 / im;
      acc[0] += 0.5 * m * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
      acc[1] += m * v[0];
      acc[2] += m * v[1];
      acc[3] += m * v[2];
    }
  }
  block_sum4(acc);
  if (threadIdx.x == 0)
#pragma unroll
    for (int c = 0; c < 4; ++c) partial[4 * blockIdx.x + c] = acc[c];
}

// The step's record {potential, kinetic, total, momentum x, y, z}: the
// block partials summed in block order.
// (potential may point at record[0]: the evaluation's energy output)
__global__ void __launch_bounds__(kMdThreads) k_md_record(const double* __restrict__ partial, int nb,
                                                           const double* potential, double* record) {
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[c] += partial[4 * b + c];
  block_sum4(acc);
  if (threadIdx.x == 0) {
    const double u = *potential;
    record[0] = u;
    record[1] = acc[0];
    record[2] = u + acc[0];
    record[3] = acc[1];
    record[4] = acc[2];
    record[5] = acc[3];
  }
}

int md_blocks(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(kMdBlocks, (n + kMdThreads - 1) / kMdThreads)); }

}  // namespace

cudaError_t launch_md_drift(Plan& P, int64_t n, double* pos, double* vel, const double* force,
                            const double* inv_mass, double dt, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  MdBox B;
  for (int d = 0; d < 3; ++d) {
    B.L[d] = P.P.box[d];
    B.inv_L[d] = 1.0 / P.P.box[d];
  }
  B.periodic = P.P.periodic;
  k_md_drift<<<md_blocks(n), kMdThreads, 0, st>>>(n, pos, vel, force, inv_mass, dt, B);
  P.launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_md_kick(Plan& P, int64_t n, double* vel, const double* force, const double* inv_mass, double dt,
                           const double* potential, double* record, cudaStream_t st) {
  const int nb = md_blocks(n);
  if (n > 0) k_md_kick<<<nb, kMdThreads, 0, st>>>(n, vel, force, inv_mass, dt, P.d.md_partial);
  else cudaMemsetAsync(P.d.md_partial, 0, sizeof(double) * 4, st);
  k_md_record<<<1, kMdThreads, 0, st>>>(P.d.md_partial, nb, potential, record);
  P.launches += 2;
  return cudaGetLastError();
}

}  // namespace msm
