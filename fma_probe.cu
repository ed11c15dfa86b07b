// fma_probe.cu -- FP32 FMA throughput of this GPU, measured: the denominator
// of the roofline fractions of the ALU-bound kernels (pair sums, lattice
// cutoff).  Each thread runs independent chains of packed (two-lane) or
// scalar fused multiply-adds long enough that issue, not latency, limits it.
// Measurement support of bench.py, built as its own library (fma_probe.so),
// not part of the MSM library or its C ABI.
//
//   int fma_probe(int packed, int64_t iters, int blocks, float* out, void* stream)
// blocks x 256 threads each run iters iterations of 16 independent FMAs (8
// packed two-lane FMAs when packed != 0, else 16 scalar ones) and write one
// float each to out [blocks * 256] (device): FLOP = blocks * 256 * iters * 32
// per launch.  Asynchronous on stream.  Returns 0, -1 for bad arguments, -7
// when the launch fails.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kProbeChains = 8;  // independent accumulators per thread

__global__ void __launch_bounds__(256) k_fma_probe_packed(int64_t iters, float a, float b, float* __restrict__ out) {
  float2 acc[kProbeChains];
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) acc[c] = make_float2(threadIdx.x * 1e-3f + c, c * 0.5f);
  const float2 m = make_float2(a, a), d = make_float2(b, b);
  for (int64_t i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) acc[c] = __ffma2_rn(acc[c], m, d);
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) s += acc[c].x + acc[c].y;
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_fma_probe_scalar(int64_t iters, float a, float b, float* __restrict__ out) {
  float acc[2 * kProbeChains];
#pragma unroll
  for (int c = 0; c < 2 * kProbeChains; ++c) acc[c] = threadIdx.x * 1e-3f + c;
  for (int64_t i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < 2 * kProbeChains; ++c) acc[c] = fmaf(acc[c], a, b);
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < 2 * kProbeChains; ++c) s += acc[c];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int fma_probe(int packed, int64_t iters, int blocks, float* out, void* stream) {
  if (iters < 0 || blocks < 1 || !out) return -1;
  cudaStream_t st = (cudaStream_t)stream;
  // a = 1 - 2^-20 and b = 2^-10 keep every chain finite and away from denormals
  const float a = 0.99999904632568359375f, b = 0.0009765625f;
  if (packed) k_fma_probe_packed<<<blocks, 256, 0, st>>>(iters, a, b, out);
  else k_fma_probe_scalar<<<blocks, 256, 0, st>>>(iters, a, b, out);
  return cudaGetLastError() == cudaSuccess ? 0 : -7;
}
