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
// (potential may point at record[0]: the evaluation's energy output).  With
// a step counter the record goes to record + 6 * counter, and the counter
// advances: a step replayed from a CUDA graph writes the next record.
__global__ void __launch_bounds__(kMdThreads) k_md_record(const double* __restrict__ partial, int nb,
                                                           const double* potential, double* record, int* counter) {
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[c] += partial[4 * b + c];
  block_sum4(acc);
  if (threadIdx.x == 0) {
    const double u = *potential;
    if (counter) record += 6 * (size_t)(*counter)++;
    record[0] = u;
    record[1] = acc[0];
    record[2] = u + acc[0];
    record[3] = acc[1];
    record[4] = acc[2];
    record[5] = acc[3];
  }
}

// Fixed-order block maximum of two non-negative values (thread 0 returns them).
__device__ __forceinline__ void block_max2(double v[2]) {
  __shared__ double red[kMdThreads / 32][2];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < 2; ++c)
    for (int o = 16; o > 0; o >>= 1) v[c] = fmax(v[c], __shfl_down_sync(0xffffffffu, v[c], o));
  if (lane == 0) {
    red[w][0] = v[0];
    red[w][1] = v[1];
  }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      v[c] = lane < kMdThreads / 32 ? red[lane][c] : 0.0;
      for (int o = 16; o > 0; o >>= 1) v[c] = fmax(v[c], __shfl_down_sync(0xffffffffu, v[c], o));
    }
  }
}

// The parareal correction (Eq. parareal) of one time point:
//   lambda_{n+1}^{k+1} = G(lambda_n^{k+1}) + F(lambda_n^k) - G(lambda_n^k)
// for positions and velocities.  In a periodic box the position difference
// F - G is taken as its minimum image and the result is wrapped into [0, L)
// (the two propagations may have wrapped an atom differently).  The kernel
// also keeps G(lambda_n^{k+1}) for the next iteration and records the largest
// change of the point against its previous iterate (positions, velocities).
__global__ void __launch_bounds__(kMdThreads) k_parareal_correct(int64_t n, MdBox B, const double* __restrict__ gnew_pos,
                                                                  const double* __restrict__ gnew_vel,
                                                                  const double* __restrict__ f_pos,
                                                                  const double* __restrict__ f_vel,
                                                                  double* __restrict__ g_pos, double* __restrict__ g_vel,
                                                                  double* __restrict__ lam_pos,
                                                                  double* __restrict__ lam_vel,
                                                                  double* __restrict__ partial) {
  double ch[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int64_t k = 3 * i + d;
      double df = f_pos[k] - g_pos[k];
      if (B.periodic) df -= B.L[d] * rint(df * B.inv_L[d]);
      double x = gnew_pos[k] + df;
      if (B.periodic) {
        x -= B.L[d] * floor(x * B.inv_L[d]);
        if (x >= B.L[d]) x -= B.L[d];
        if (x < 0.0) x = 0.0;
      }
      double dx = x - lam_pos[k];
      if (B.periodic) dx -= B.L[d] * rint(dx * B.inv_L[d]);
      const double v = gnew_vel[k] + (f_vel[k] - g_vel[k]);
      ch[0] = fmax(ch[0], fabs(dx));
      ch[1] = fmax(ch[1], fabs(v - lam_vel[k]));
      lam_pos[k] = x;
      lam_vel[k] = v;
      g_pos[k] = gnew_pos[k];
      g_vel[k] = gnew_vel[k];
    }
  }
  block_max2(ch);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = ch[0];
    partial[2 * blockIdx.x + 1] = ch[1];
  }
}

__global__ void __launch_bounds__(kMdThreads) k_parareal_change(const double* __restrict__ partial, int nb,
                                                                 double* __restrict__ change) {
  double ch[2] = {0.0, 0.0};
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    ch[0] = fmax(ch[0], partial[2 * b]);
    ch[1] = fmax(ch[1], partial[2 * b + 1]);
  }
  block_max2(ch);
  if (threadIdx.x == 0) {
    change[0] = ch[0];
    change[1] = ch[1];
  }
}

MdBox md_box(const Plan& P) {
  MdBox B;
  for (int d = 0; d < 3; ++d) {
    B.L[d] = P.P.box[d];
    B.inv_L[d] = 1.0 / P.P.box[d];
  }
  B.periodic = P.P.periodic;
  return B;
}

int md_blocks(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(kMdBlocks, (n + kMdThreads - 1) / kMdThreads)); }

}  // namespace

cudaError_t launch_md_drift(Plan& P, int64_t n, double* pos, double* vel, const double* force,
                            const double* inv_mass, double dt, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_md_drift<<<md_blocks(n), kMdThreads, 0, st>>>(n, pos, vel, force, inv_mass, dt, md_box(P));
  P.launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_md_kick(Plan& P, int64_t n, double* vel, const double* force, const double* inv_mass, double dt,
                           const double* potential, double* record, int* counter, cudaStream_t st) {
  const int nb = md_blocks(n);
  if (n > 0) {
    k_md_kick<<<nb, kMdThreads, 0, st>>>(n, vel, force, inv_mass, dt, P.d.md_partial);
  } else {
    const cudaError_t e = cudaMemsetAsync(P.d.md_partial, 0, sizeof(double) * 4, st);
    if (e != cudaSuccess) return e;
  }
  k_md_record<<<1, kMdThreads, 0, st>>>(P.d.md_partial, nb, potential, record, counter);
  P.launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_parareal_correct(Plan& P, int64_t n, const double* gnew_pos, const double* gnew_vel,
                                    const double* f_pos, const double* f_vel, double* g_pos, double* g_vel,
                                    double* lam_pos, double* lam_vel, double* change, cudaStream_t st) {
  const int nb = md_blocks(n);
  if (n > 0)
    k_parareal_correct<<<nb, kMdThreads, 0, st>>>(n, md_box(P), gnew_pos, gnew_vel, f_pos, f_vel, g_pos, g_vel, lam_pos,
                                                  lam_vel, P.d.md_partial);
  else if (const cudaError_t e = cudaMemsetAsync(P.d.md_partial, 0, sizeof(double) * 2, st); e != cudaSuccess)
    return e;
  k_parareal_change<<<1, kMdThreads, 0, st>>>(P.d.md_partial, nb, change);
  P.launches += 2;
  return cudaGetLastError();
}

}  // namespace msm
