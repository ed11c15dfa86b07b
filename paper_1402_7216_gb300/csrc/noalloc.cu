// noalloc.cu -- msm_energy_noalloc: the energy reduction E = 1/2 sum_i q_i phi_i
// with its scratch (one FP64 partial sum per 256 atoms) in a file-scope device
// array instead of plan-owned memory, so the call allocates nothing.
//
// Why: some callers must not allocate device memory while they run -- for
// example an MD engine that owns all device memory through its own pool, or a
// time-step loop that cannot afford cudaMalloc, which may synchronise the
// device and stall other streams.  Such callers still pass their own inputs
// and output; the scratch is this array, which every GPU that loads the
// library keeps until the process exits.
#include <mutex>

#include "msm_internal.h"

namespace msm {
namespace {

constexpr int kBlock = 256;
constexpr int kMaxPartials = 65536;  // n <= 256 * 65536 = 16,777,216 atoms (512 KiB of scratch)
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partials[kMaxPartials];

// Host-side cache of the array's device address, one per device.  In host
// code the symbol itself is only a stand-in, not a device address.
double* g_partials_addr[kMaxDevices] = {nullptr};
std::mutex g_partials_mu;

__global__ void __launch_bounds__(kBlock) k_qphi_partials(int64_t n, const double* __restrict__ q,
                                                          const double* __restrict__ phi,
                                                          double* __restrict__ partials) {
  __shared__ double red[kBlock / 32];
  int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  double v = (i < n) ? q[i] * phi[i] : 0.0;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = (threadIdx.x < kBlock / 32) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;  // every partial in [0, nb) is written
  }
}

__global__ void __launch_bounds__(1024) k_partials_final(const double* __restrict__ partials, int nb,
                                                         double* __restrict__ energy) {
  __shared__ double red[32];
  double v = 0.0;
  for (int i = threadIdx.x; i < nb; i += 1024) v += partials[i];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = red[threadIdx.x];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *energy = 0.5 * s;
  }
}

// Looks up the scratch array's device address for the current device (once
// per device; the first call on a device does this set-up).
cudaError_t partials_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_partials_mu);
  if (!g_partials_addr[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_partials_addr[dev] = p;
  }
  *out = g_partials_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace msm

extern "C" int msm_energy_noalloc(int64_t n, const double* q, const double* phi, double* energy,
                                  void* cuda_stream) {
  using namespace msm;
  if (n < 0 || !energy || (n > 0 && (!q || !phi))) return MSM_ERR_INVALID_ARG;
  int64_t nb = (n + kBlock - 1) / kBlock;
  if (nb > kMaxPartials) return MSM_ERR_TOO_MANY_ATOMS;
  double* partials = nullptr;
  if (partials_for_current_device(&partials) != cudaSuccess) return MSM_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (nb > 0) k_qphi_partials<<<(unsigned)nb, kBlock, 0, st>>>(n, q, phi, partials);
  k_partials_final<<<1, 1024, 0, st>>>(partials, (int)nb, energy);
  return cudaGetLastError() == cudaSuccess ? MSM_OK : MSM_ERR_CUDA;
}
