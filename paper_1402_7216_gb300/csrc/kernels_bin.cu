// kernels_bin.cu -- atom binning by sort (link cells, Sec. "Short-range
// interactions": atoms are binned into cells so that each atom only examines
// nearby cells).  The cell key of every atom is sorted by a stable LSD radix
// sort (8-bit digits, per-block histograms, one scan, stable scatter ranked
// with warp match), so the binning takes no scatter atomics on global memory
// and the order inside a cell is the input order (deterministic).
// The gather then writes the sorted atoms in the layouts the later passes
// read: cell-local coordinates for the pair sums, and fractional level-0 grid
// coordinates plus the first support index for the grid passes.
#include <cmath>

#include "msm_internal.h"

namespace msm {

namespace {

constexpr int kChunk = 4096;   // atoms per radix block
constexpr int kThreads = 256;  // = radix size

// Folds x into [0, L) (multiplying by the reciprocal: FP64 division is slow).
__device__ __forceinline__ double fold(double x, double L, double inv_L) {
  double y = x - L * floor(x * inv_L);
  if (y >= L) y -= L;
  if (y < 0.0) y += L;
  return y;
}

struct BinArgs {
  double box[3];
  double inv_box[3];
  double cw[3];
  double inv_cw[3];
  double inv_h[3];
  int nc[3];
  int fmax[3];  // open grids: largest floor(x/h) the level-0 grid covers
  int periodic;
  int S;
};

__global__ void k_keys(const double* __restrict__ pos, const double* __restrict__ q, int n,
                       BinArgs A, int* __restrict__ keys, int* __restrict__ idx,
                       int* __restrict__ status) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double x[3] = {pos[3 * (size_t)i], pos[3 * (size_t)i + 1], pos[3 * (size_t)i + 2]};
  int bad = 0;
  if (!isfinite(x[0]) || !isfinite(x[1]) || !isfinite(x[2]) || !isfinite(q[i])) bad |= kStatusNonfinite;
  int c[3];
  for (int d = 0; d < 3; ++d) {
    double v = x[d];
    if (A.periodic) {
      v = isfinite(v) ? fold(v, A.box[d], A.inv_box[d]) : 0.0;
    } else if (!(v >= 0.0 && v <= A.box[d])) {
      bad |= kStatusOutside;
      v = 0.0;
    }
    int ci = (int)floor(v * A.inv_cw[d]);
    c[d] = ci < 0 ? 0 : (ci >= A.nc[d] ? A.nc[d] - 1 : ci);
  }
  if (bad) atomicOr(status, bad);
  keys[i] = (c[2] * A.nc[1] + c[1]) * A.nc[0] + c[0];
  idx[i] = i;
}

__global__ void __launch_bounds__(kThreads) k_hist(const int* __restrict__ keys, int n, int shift,
                                                   int* __restrict__ hist, int nblk) {
  __shared__ int h[256];
  int t = threadIdx.x, b = blockIdx.x;
  h[t] = 0;
  __syncthreads();
  int end = min(n, (b + 1) * kChunk);
  for (int i = b * kChunk + t; i < end; i += kThreads) atomicAdd(&h[(keys[i] >> shift) & 255], 1);
  __syncthreads();
  hist[t * nblk + b] = h[t];
}

// Exclusive scan of `total` ints in place, one block of 1024 threads walking
// the array in coalesced tiles of 1024 (warp-shuffle scan inside a tile, a
// running carry between tiles).
__global__ void __launch_bounds__(1024) k_scan(int* __restrict__ data, int total) {
  __shared__ int wsum[32];
  __shared__ int carry_s;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (t == 0) carry_s = 0;
  __syncthreads();
  for (int base = 0; base < total; base += 1024) {
    const int i = base + t;
    const int v = (i < total) ? data[i] : 0;
    int x = v;  // inclusive warp scan
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int w = wsum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      wsum[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    const int carry = carry_s;
    const int excl = carry + (warp > 0 ? wsum[warp - 1] : 0) + x - v;
    if (i < total) data[i] = excl;
    __syncthreads();
    if (t == 1023) carry_s = excl + v;
    __syncthreads();
  }
}

// Stable scatter: inside a block, items are ranked in index order (warp
// match for ranks inside a warp, a per-digit prefix over the warps), on top of
// the block's scanned digit offset.
__global__ void __launch_bounds__(kThreads) k_scatter(const int* __restrict__ kin,
                                                      const int* __restrict__ iin,
                                                      int* __restrict__ kout, int* __restrict__ iout,
                                                      const int* __restrict__ hist, int n, int shift,
                                                      int nblk) {
  __shared__ int s_off[256];
  __shared__ int s_w[kThreads / 32][256];
  int t = threadIdx.x, lane = t & 31, warp = t >> 5, b = blockIdx.x;
  s_off[t] = hist[t * nblk + b];
  int base = b * kChunk;
  for (int sub = 0; sub < kChunk && base + sub < n; sub += kThreads) {
    for (int e = t; e < (kThreads / 32) * 256; e += kThreads) (&s_w[0][0])[e] = 0;
    __syncthreads();
    int i = base + sub + t;
    bool valid = i < n;
    int key = valid ? kin[i] : 0;
    int digit = valid ? ((key >> shift) & 255) : 256;
    unsigned peers = __match_any_sync(0xffffffffu, digit);
    int rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && lane == __ffs(peers) - 1) s_w[warp][digit] = __popc(peers);
    __syncthreads();
    {
      int run = s_off[t];
      for (int w = 0; w < kThreads / 32; ++w) {
        int c = s_w[w][t];
        s_w[w][t] = run;
        run += c;
      }
      s_off[t] = run;
    }
    __syncthreads();
    if (valid) {
      int p = s_w[warp][digit] + rank;
      kout[p] = key;
      iout[p] = iin[i];
    }
    __syncthreads();
  }
}

__global__ void k_cell_start(const int* __restrict__ keys, int n, int ncell, int* __restrict__ cs) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c > ncell) return;
  int lo = 0, hi = n;  // first position with key >= c
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (keys[mid] < c) lo = mid + 1;
    else hi = mid;
  }
  cs[c] = lo;
}

template <typename T>
__global__ void k_gather(const double* __restrict__ pos, const double* __restrict__ q, int n,
                         BinArgs A, const int* __restrict__ keys, const int* __restrict__ idx,
                         R4<T>* __restrict__ atoms, R4<T>* __restrict__ gfrac,
                         int4* __restrict__ gbase) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  int i = idx[s], key = keys[s];
  int c[3] = {key % A.nc[0], (key / A.nc[0]) % A.nc[1], key / (A.nc[0] * A.nc[1])};
  double qi = q[i];
  T loc[3], fr[3];
  int bs[3];
  for (int d = 0; d < 3; ++d) {
    double v = pos[3 * (size_t)i + d];
    if (A.periodic) v = isfinite(v) ? fold(v, A.box[d], A.inv_box[d]) : 0.0;
    else v = fmin(fmax(v, 0.0), A.box[d]);
    loc[d] = (T)(v - c[d] * A.cw[d]);
    double t = v * A.inv_h[d];
    double fl = floor(t);
    if (!A.periodic && fl > (double)A.fmax[d]) fl = (double)A.fmax[d];  // x = L rounding up
    fr[d] = (T)(t - fl);
    bs[d] = (int)fl - (A.S - 1);
  }
  atoms[s] = R4<T>{loc[0], loc[1], loc[2], (T)qi};
  gfrac[s] = R4<T>{fr[0], fr[1], fr[2], (T)qi};
  gbase[s] = make_int4(bs[0], bs[1], bs[2], 0);
}

}  // namespace

cudaError_t launch_binning(Plan& P, int64_t n64, const double* pos, const double* q, cudaStream_t st) {
  int n = (int)n64;
  DeviceBuffers& D = P.d;
  BinArgs A;
  for (int d = 0; d < 3; ++d) {
    A.box[d] = P.P.box[d];
    A.inv_box[d] = 1.0 / P.P.box[d];
    A.cw[d] = P.cw[d];
    A.inv_cw[d] = 1.0 / P.cw[d];
    A.inv_h[d] = 1.0 / P.h[d];
    A.nc[d] = P.nc[d];
    A.fmax[d] = P.n[0][d] - 2 * P.S;
  }
  A.periodic = P.P.periodic;
  A.S = P.S;
  if (n > 0) {
    k_keys<<<(n + 255) / 256, 256, 0, st>>>(pos, q, n, A, D.keys[0], D.idx[0], D.status);
    int nblk = (n + kChunk - 1) / kChunk;
    int cur = 0;
    for (int pass = 0; pass < P.key_passes; ++pass) {
      int shift = 8 * pass;
      k_hist<<<nblk, kThreads, 0, st>>>(D.keys[cur], n, shift, D.hist, nblk);
      k_scan<<<1, 1024, 0, st>>>(D.hist, 256 * nblk);
      k_scatter<<<nblk, kThreads, 0, st>>>(D.keys[cur], D.idx[cur], D.keys[cur ^ 1], D.idx[cur ^ 1],
                                           D.hist, n, shift, nblk);
      cur ^= 1;
    }
    P.launches += 1 + 3 * P.key_passes;
    if (cur != 0) {  // keep the sorted result in slot 0
      P.launches += 2;
      cudaMemcpyAsync(D.keys[0], D.keys[1], sizeof(int) * n, cudaMemcpyDeviceToDevice, st);
      cudaMemcpyAsync(D.idx[0], D.idx[1], sizeof(int) * n, cudaMemcpyDeviceToDevice, st);
    }
  }
  k_cell_start<<<(P.ncell + 1 + 255) / 256, 256, 0, st>>>(D.keys[0], n, P.ncell, D.cell_start);
  P.launches += 1 + (n > 0 ? 1 : 0);
  if (n > 0) {
    if (P.fp64)
      k_gather<double><<<(n + 255) / 256, 256, 0, st>>>(pos, q, n, A, D.keys[0], D.idx[0],
                                                        (R4<double>*)D.atoms, (R4<double>*)D.gfrac,
                                                        D.gbase);
    else
      k_gather<float><<<(n + 255) / 256, 256, 0, st>>>(pos, q, n, A, D.keys[0], D.idx[0],
                                                       (R4<float>*)D.atoms, (R4<float>*)D.gfrac,
                                                       D.gbase);
  }
  return cudaGetLastError();
}

}  // namespace msm
