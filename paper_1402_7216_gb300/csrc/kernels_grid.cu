// kernels_grid.cu -- the long-range steps of MSM (Sec. "Multilevel Summation
// Method"), in the order the thesis lists them:
//   anterpolation   q^0_mu = sum_j phi^0_mu(r_j) q_j
//   restriction     q^{k+1}_mu = sum_nu phi^{k+1}_mu(r^k_nu) q^k_nu
//   lattice cutoff  u^{k,cutoff}_mu = sum_nu g^k(r^k_mu, r^k_nu) q^k_nu
//   top level       u^{l-1}_mu = sum_nu g^{l-1}(r_mu, r_nu) q^{l-1}_nu (all pairs)
//   prolongation    u^k_mu = u^{k,cutoff}_mu + sum_nu phi^{k+1}_nu(r^k_mu) u^{k+1}_nu
//   interpolation   u_i^long = sum_mu phi^0_mu(r_i) u^0_mu (and its gradient)
// with phi^k_mu = Phi(x)Phi(y)Phi(z) on spacing 2^k h, Phi the C1 cubic
// (numerical Hermite) or C1 quintic interpolant.  Grids are dense arrays,
// x fastest.  The adjoint (backward) pass reuses the same kernels: the
// transpose of interpolation is anterpolation, the transpose of prolongation
// is restriction, and the lattice and top kernels are symmetric.
#include <algorithm>
#include <cmath>
#include <new>
#include <type_traits>

#include "msm_internal.h"

namespace msm {

namespace {

// ---- nodal basis Phi ----
// Piece j of Phi covers |d| in [j, j+1]; it is written as a polynomial in the
// local coordinate u = |d| - j in [0, 1], where every coefficient is small,
// so FP32 evaluation keeps full relative accuracy (expanding in |d| instead
// would cancel terms up to ~60 against weights of ~0.01).
//   cubic   P0 = 1 - 5/2 u^2 + 3/2 u^3          P1 = -u (1 - u)^2 / 2
//   quintic Q0 = (1 - u^2)(2 - u)(6 + 3u - 5u^2)/12
//           Q1 = u (u - 1)(u - 2)(5u^2 + u - 8)/24
//           Q2 = -(u + 1) u (u - 1)^2 (u - 2)/24
template <typename T, int ORDER>
struct Basis;

template <typename T>
struct Basis<T, 3> {
  static constexpr int S = 2;
  __device__ static T p(int j, T u) {
    return j == 0 ? T(1) + u * u * (T(-2.5) + T(1.5) * u) : u * (T(-0.5) + u * (T(1) - T(0.5) * u));
  }
  __device__ static T dp(int j, T u) {
    return j == 0 ? u * (T(-5) + T(4.5) * u) : T(-0.5) + u * (T(2) - T(1.5) * u);
  }
};

template <typename T>
struct Basis<T, 5> {
  static constexpr int S = 3;
  __device__ static T p(int j, T u) {
    if (j == 0)
      return T(1) + u * u * (T(-25.0 / 12) + u * (T(5.0 / 12) + u * (T(13.0 / 12) - T(5.0 / 12) * u)));
    if (j == 1)
      return u * (T(-16.0 / 24) + u * (T(26.0 / 24) + u * (T(-1.0 / 24) + u * (T(-14.0 / 24) + T(5.0 / 24) * u))));
    return u * (T(2.0 / 24) + u * (T(-3.0 / 24) + u * (T(-1.0 / 24) + u * (T(3.0 / 24) - T(1.0 / 24) * u))));
  }
  __device__ static T dp(int j, T u) {
    if (j == 0)
      return u * (T(-50.0 / 12) + u * (T(15.0 / 12) + u * (T(52.0 / 12) - T(25.0 / 12) * u)));
    if (j == 1)
      return T(-16.0 / 24) + u * (T(52.0 / 24) + u * (T(-3.0 / 24) + u * (T(-56.0 / 24) + T(25.0 / 24) * u)));
    return T(2.0 / 24) + u * (T(-6.0 / 24) + u * (T(-3.0 / 24) + u * (T(12.0 / 24) - T(5.0 / 24) * u)));
  }
};

// Weights of the 2S support points base + s (s = 0..2S-1) for an atom at
// fractional offset f in [0,1) past grid point base + S - 1.  The signed
// distance to point s is d = f + S - 1 - s: piece S-1-s at u = f for s < S,
// piece s-S at u = 1 - f beyond.
template <typename T, int ORDER>
__device__ __forceinline__ void weights(T f, T* w) {
  constexpr int S = Basis<T, ORDER>::S;
  const T g = T(1) - f;
#pragma unroll
  for (int s = 0; s < 2 * S; ++s)
    w[s] = (s < S) ? Basis<T, ORDER>::p(S - 1 - s, f) : Basis<T, ORDER>::p(s - S, g);
}

// dPhi/dd at the same points (d > 0 for s < S, d < 0 beyond).
template <typename T, int ORDER>
__device__ __forceinline__ void dweights(T f, T* w) {
  constexpr int S = Basis<T, ORDER>::S;
  const T g = T(1) - f;
#pragma unroll
  for (int s = 0; s < 2 * S; ++s)
    w[s] = (s < S) ? Basis<T, ORDER>::dp(S - 1 - s, f) : -Basis<T, ORDER>::dp(s - S, g);
}

struct GridDims {
  int n[3];
  int lo[3];
  int periodic;
};

__device__ __forceinline__ int slot(int idx, int n, int lo, int periodic) {
  if (periodic) {
    int r = idx % n;
    return r < 0 ? r + n : r;
  }
  return idx - lo;  // callers only pass indices inside the open grid
}

// ---- anterpolation: per-block shared-memory patches ----
// A block owns B x B x B short-range cells; the level-0 points their atoms
// can reach form a patch of at most PD^3 points held in shared memory.  Each
// atom adds its (2S)^3 weighted charges into the patch (shared-memory
// atomics); the block then adds the patch into the global FP64 grid, so
// global atomics only meet where neighbouring patches overlap.
struct AnterpArgs {
  int nc[3];        // short-range cells per dimension
  int B;            // cells per block side
  int pd;           // patch points per dimension
  double cw_h[3];   // cell width in units of h
};

// One thread per atom, and the lanes of a warp take atoms from different
// cells of the block: the block's atoms are listed rank-major (the first atom
// of every cell, then the second of every cell, ...), so consecutive threads
// work on different cells.  Atoms of one cell share most of their support,
// so this keeps the shared-memory atomics of one warp instruction on
// different points, and no lane idles while others finish a fuller cell.
constexpr int kAnterpMaxAtoms = 4096;  // atoms per block listed in shared memory

__device__ __forceinline__ int block_cells(const AnterpArgs& A, const int* __restrict__ cell_start, const int* c0,
                                           int* cstart, int* ccount) {
  int k = 0;
  for (int bz = 0; bz < A.B; ++bz)
    for (int by = 0; by < A.B; ++by)
      for (int bx = 0; bx < A.B; ++bx) {
        int x = c0[0] + bx, y = c0[1] + by, z = c0[2] + bz;
        if (x >= A.nc[0] || y >= A.nc[1] || z >= A.nc[2]) continue;
        int c = (z * A.nc[1] + y) * A.nc[0] + x;
        cstart[k] = cell_start[c];
        ccount[k] = cell_start[c + 1] - cell_start[c];
        ++k;
      }
  return k;
}

// Rank-major list of the block's atoms (warp 0 builds it); returns the count,
// or -1 when the block holds more atoms than the list can take.
__device__ __forceinline__ int build_rank_list(int nk, const int* cstart, const int* ccount, int* list,
                                               int* maxc_s) {
  const int lane = threadIdx.x & 31;
  int total = 0;
  if (threadIdx.x < 32) {
    int mx = 0;
    for (int c = lane; c < nk; c += 32) mx = max(mx, ccount[c]);
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    for (int r = 0; r < mx; ++r)
      for (int cb = 0; cb < nk; cb += 32) {
        const int c = cb + lane;
        const bool has = c < nk && ccount[c] > r;
        const unsigned bal = __ballot_sync(0xffffffffu, has);
        const int p = total + __popc(bal & ((1u << lane) - 1u));
        if (has && p < kAnterpMaxAtoms) list[p] = cstart[c] + r;
        total += __popc(bal);
      }
    if (lane == 0) *maxc_s = total;
  }
  __syncthreads();
  total = *maxc_s;
  return total > kAnterpMaxAtoms ? -1 : total;
}

template <typename T, typename ACC, int ORDER>
__global__ void __launch_bounds__(256) k_anterp_patch(const R4<T>* __restrict__ gfrac,
                                                      const int4* __restrict__ gbase,
                                                      const int* __restrict__ cell_start, AnterpArgs A,
                                                      GridDims G, double* __restrict__ grid,
                                                      const double* __restrict__ dscale, double factor) {
  constexpr int S = Basis<T, ORDER>::S, W = 2 * S;
  extern __shared__ unsigned char smem_raw[];
  ACC* patch = reinterpret_cast<ACC*>(smem_raw);
  __shared__ int cstart[64], ccount[64], list[kAnterpMaxAtoms], tot_s;
  const int PD = A.pd, np = PD * PD * PD, tid = threadIdx.x;
  const int c0[3] = {(int)blockIdx.x * A.B, (int)blockIdx.y * A.B, (int)blockIdx.z * A.B};
  const int lo0 = (int)floor(c0[0] * A.cw_h[0]) - S - 1;
  const int lo1 = (int)floor(c0[1] * A.cw_h[1]) - S - 1;
  const int lo2 = (int)floor(c0[2] * A.cw_h[2]) - S - 1;
  for (int e = tid; e < np; e += blockDim.x) patch[e] = ACC(0);
  __shared__ int nk_s;
  if (tid == 0) nk_s = block_cells(A, cell_start, c0, cstart, ccount);
  __syncthreads();
  const int nk = nk_s;
  int total = build_rank_list(nk, cstart, ccount, list, &tot_s);
  const T sc_all = T(factor * (dscale ? *dscale : 1.0));
  const int count = total >= 0 ? total : 0;
  for (int kk = tid; kk < count; kk += blockDim.x) {
    const int i = list[kk];
    const R4<T> f = gfrac[i];
    const int4 b = gbase[i];
    const T qi = sc_all * f.w;
    T wx[W], wy[W], wz[W];
    weights<T, ORDER>(f.x, wx);
    weights<T, ORDER>(f.y, wy);
    weights<T, ORDER>(f.z, wz);
    const int px = b.x - lo0, py = b.y - lo1, pz = b.z - lo2;
    if (px >= 0 && py >= 0 && pz >= 0 && px + W <= PD && py + W <= PD && pz + W <= PD) {
#pragma unroll
      for (int c = 0; c < W; ++c) {
        const T qz = qi * wz[c];
#pragma unroll
        for (int bb = 0; bb < W; ++bb) {
          const T qyz = qz * wy[bb];
          ACC* row = patch + ((pz + c) * PD + py + bb) * PD + px;
#pragma unroll
          for (int a = 0; a < W; ++a) atomicAdd(row + a, ACC(qyz * wx[a]));
        }
      }
    } else {  // outside the patch (cannot happen for atoms inside their cells): straight to the grid
      for (int c = 0; c < W; ++c)
        for (int bb = 0; bb < W; ++bb)
          for (int a = 0; a < W; ++a) {
            int sx = slot(b.x + a, G.n[0], G.lo[0], G.periodic), sy = slot(b.y + bb, G.n[1], G.lo[1], G.periodic),
                sz = slot(b.z + c, G.n[2], G.lo[2], G.periodic);
            atomicAdd(grid + ((size_t)sz * G.n[1] + sy) * G.n[0] + sx, (double)(qi * wz[c] * wy[bb] * wx[a]));
          }
    }
  }
  if (total < 0) {  // more atoms than the list holds: one thread per atom, straight to the grid
    for (int c = 0; c < nk; ++c)
      for (int m = tid; m < ccount[c]; m += blockDim.x) {
        const int i = cstart[c] + m;
        const R4<T> f = gfrac[i];
        const int4 b = gbase[i];
        const T qi = sc_all * f.w;
        T wx[W], wy[W], wz[W];
        weights<T, ORDER>(f.x, wx);
        weights<T, ORDER>(f.y, wy);
        weights<T, ORDER>(f.z, wz);
        for (int cc = 0; cc < W; ++cc)
          for (int bb = 0; bb < W; ++bb)
            for (int a = 0; a < W; ++a) {
              int sx = slot(b.x + a, G.n[0], G.lo[0], G.periodic), sy = slot(b.y + bb, G.n[1], G.lo[1], G.periodic),
                  sz = slot(b.z + cc, G.n[2], G.lo[2], G.periodic);
              atomicAdd(grid + ((size_t)sz * G.n[1] + sy) * G.n[0] + sx, (double)(qi * wz[cc] * wy[bb] * wx[a]));
            }
      }
  }
  __syncthreads();
  for (int e = tid; e < np; e += blockDim.x) {
    const ACC v = patch[e];
    if (v == ACC(0)) continue;
    int ix = lo0 + e % PD, iy = lo1 + (e / PD) % PD, iz = lo2 + e / (PD * PD);
    if (!G.periodic && (ix < G.lo[0] || iy < G.lo[1] || iz < G.lo[2] || ix >= G.lo[0] + G.n[0] ||
                        iy >= G.lo[1] + G.n[1] || iz >= G.lo[2] + G.n[2]))
      continue;
    int sx = slot(ix, G.n[0], G.lo[0], G.periodic), sy = slot(iy, G.n[1], G.lo[1], G.periodic),
        sz = slot(iz, G.n[2], G.lo[2], G.periodic);
    atomicAdd(grid + ((size_t)sz * G.n[1] + sy) * G.n[0] + sx, (double)v);
  }
}

// ---- mixed precision: exact fixed-point patch sums ----
// Shared-memory FP32 atomic adds return through a compare-and-swap round
// trip, while 32-bit integer reductions are fire-and-forget.  So the mixed
// plan accumulates each patch point as two integer sums: a contribution
// c = q_j w (|w| <= 1) becomes t = c 2^12, a coarse part round(t) and a
// residual round((t - round(t)) 2^19), each added with an integer reduction.
// The patch sums are then exact, independent of order, at a resolution of
// 2^-31.  Integer sums wrap modulo 2^32, so only the final sums must fit:
// the coarse sum stays below 2^31 while |q_j| * (atoms of the block) <= 2^18
// for every atom in the patch, and the residuals (|.| <= 2^18, one per atom)
// of at most kAnterpMaxAtoms = 2^12 atoms stay below 2^30.  An atom with a
// larger charge (or |q_j| >= 2^10) goes straight to the FP64 grid.  The device-side scale (the
// adjoint's upstream gradient) multiplies the patch sums when they are
// flushed, so the fixed-point resolution is relative to the charges alone.
constexpr float kFxMagic = 12582912.0f;  // 1.5 * 2^23: adding it rounds |x| < 2^22 to an integer
constexpr float kFxCoarse = 4096.0f;     // 2^12
constexpr float kFxFine = 524288.0f;     // 2^19

__device__ __forceinline__ void fx_split(float t, int& hi, int& lo) {
  const float m = __fadd_rn(t, kFxMagic);
  hi = __float_as_int(m) - __float_as_int(kFxMagic);
  const float r = __fsub_rn(t, __fsub_rn(m, kFxMagic));  // t - round(t), exact
  lo = __float_as_int(__fmaf_rn(r, kFxFine, kFxMagic)) - __float_as_int(kFxMagic);
}

// Bank-ordered atom list.  Every tap of an atom sits at a fixed offset from
// the patch index of its first support point, so two lanes whose atoms' first
// points share a shared-memory bank (index mod 32) collide on every one of
// their (2S)^3 reductions.  The block therefore buckets its atoms by that
// bank and lays the list out in rounds of 32 slots, slot L of round r holding
// the r-th atom of bucket L: the 32 lanes of a warp instruction then touch 32
// different banks.  Buckets fuller than the round count R = ceil(total/32)
// spill into the empty slots of the others (those lanes share a bank with one
// other lane).  Integer sums do not depend on the order, so neither the
// bucket ranks nor the spill order affect the result.  Returns the slot count
// 32 R (unfilled slots hold -1); scratch (at least total + 32 R ints) is the
// not yet zeroed patch, else the list stays as it is.
__device__ __forceinline__ int bank_order(int* list, int total, const int4* __restrict__ gbase, int lo0, int lo1,
                                          int lo2, int PD, int* scratch, int nscratch) {
  __shared__ int bcnt[32], bempty[33], ovf;
  const int R = (total + 31) >> 5, nslot = R << 5;
  if (total == 0 || nscratch < total + nslot) return total;  // block-uniform
  const int tid = threadIdx.x;
  if (tid < 32) bcnt[tid] = 0;
  if (tid == 0) ovf = 0;
  __syncthreads();
  for (int kk = tid; kk < total; kk += blockDim.x) {
    const int4 b = gbase[list[kk]];
    const int key = (((b.z - lo2) * PD + (b.y - lo1)) * PD + (b.x - lo0)) & 31;
    scratch[kk] = key | (atomicAdd(&bcnt[key], 1) << 5);
  }
  __syncthreads();
  if (tid < 32) {  // empty slots of bucket L: rounds bcnt[L] .. R-1; exclusive prefix over L
    const int e = max(0, R - bcnt[tid]);
    int incl = e;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (tid >= o) incl += y;
    }
    bempty[tid] = incl - e;
    if (tid == 31) bempty[32] = incl;
  }
  int* slots = scratch + total;
  for (int e = tid; e < nslot; e += blockDim.x) slots[e] = -1;
  __syncthreads();
  for (int kk = tid; kk < total; kk += blockDim.x) {
    const int key = scratch[kk] & 31, r = scratch[kk] >> 5;
    int slot;
    if (r < R) {
      slot = (r << 5) | key;
    } else {
      const int o = atomicAdd(&ovf, 1);  // o < total empty slots, since 32 R >= total
      int L = 0;
      while (bempty[L + 1] <= o) ++L;
      slot = ((bcnt[L] + (o - bempty[L])) << 5) | L;
    }
    slots[slot] = list[kk];
  }
  __syncthreads();
  for (int e = tid; e < nslot; e += blockDim.x) list[e] = slots[e];
  __syncthreads();
  return nslot;
}

// One atom's (2S)^3 weighted charges straight into the fixed-point grid
// (global 64-bit integer reductions, 2^-31 units, computed in FP64); kept out
// of line so that the patch loop holds its weights in registers.
template <int ORDER>
__device__ __noinline__ void anterp_atom_global(const R4<float> f, const int4 b, const GridDims G,
                                                unsigned long long* __restrict__ gfx) {
  constexpr int W = 2 * Basis<float, ORDER>::S;
  float wx[W], wy[W], wz[W];
  weights<float, ORDER>(f.x, wx);
  weights<float, ORDER>(f.y, wy);
  weights<float, ORDER>(f.z, wz);
  const double qd = 2147483648.0 * (double)f.w;  // 2^31 q
#pragma unroll
  for (int c = 0; c < W; ++c) {
    const int sz = slot(b.z + c, G.n[2], G.lo[2], G.periodic);
#pragma unroll
    for (int bb = 0; bb < W; ++bb) {
      const int sy = slot(b.y + bb, G.n[1], G.lo[1], G.periodic);
      unsigned long long* row = gfx + ((size_t)sz * G.n[1] + sy) * G.n[0];
#pragma unroll
      for (int a = 0; a < W; ++a)
        atomicAdd(row + slot(b.x + a, G.n[0], G.lo[0], G.periodic),
                  (unsigned long long)__double2ll_rn(qd * (double)(wz[c] * wy[bb] * wx[a])));
    }
  }
}

template <int ORDER>
__device__ __forceinline__ void anterp_fx_body(const R4<float>* __restrict__ gfrac, const int4* __restrict__ gbase,
                                               const int* __restrict__ cell_start, const AnterpArgs& A,
                                               const GridDims& G, unsigned long long* __restrict__ gfx, int bx, int by,
                                               int bz) {
  constexpr int S = Basis<float, ORDER>::S, W = 2 * S;
  extern __shared__ unsigned char smem_raw[];
  const int PD = A.pd, np = PD * PD * PD, tid = threadIdx.x;
  int* phi_ = reinterpret_cast<int*>(smem_raw);  // coarse sums
  int* plo = phi_ + np;                          // residual sums
  __shared__ int cstart[64], ccount[64], list[kAnterpMaxAtoms + 32], tot_s, nk_s;  // + one round of slots
  const int c0[3] = {bx * A.B, by * A.B, bz * A.B};
  const int lo0 = (int)floor(c0[0] * A.cw_h[0]) - S - 1;
  const int lo1 = (int)floor(c0[1] * A.cw_h[1]) - S - 1;
  const int lo2 = (int)floor(c0[2] * A.cw_h[2]) - S - 1;
  if (tid == 0) nk_s = block_cells(A, cell_start, c0, cstart, ccount);
  __syncthreads();
  const int nk = nk_s;
  const int total = build_rank_list(nk, cstart, ccount, list, &tot_s);
  // |q_j| <= 2^18 / (atoms in the patch) bounds the coarse sums; |q_j| < 2^10
  // keeps |t| < 2^22, where the magic-number rounding of fx_split is exact
  const float qmax = fminf(262144.0f / (float)max(total, 1), 1023.0f);
  const int count = total >= 0 ? bank_order(list, total, gbase, lo0, lo1, lo2, PD, phi_, 2 * np) : 0;
  for (int e = tid; e < 2 * np; e += blockDim.x) phi_[e] = 0;
  __syncthreads();
  for (int kk = tid; kk < count; kk += blockDim.x) {
    const int i = list[kk];
    if (i < 0) continue;  // unfilled slot of the bank-ordered list
    const R4<float> f = gfrac[i];
    const int4 b = gbase[i];
    float wx[W], wy[W], wz[W];
    weights<float, ORDER>(f.x, wx);
    weights<float, ORDER>(f.y, wy);
    weights<float, ORDER>(f.z, wz);
    const int px = b.x - lo0, py = b.y - lo1, pz = b.z - lo2;
    if (fabsf(f.w) < qmax && px >= 0 && py >= 0 && pz >= 0 && px + W <= PD && py + W <= PD && pz + W <= PD) {
      const float qs = f.w * kFxCoarse;
#pragma unroll
      for (int c = 0; c < W; ++c) {
        const float qz = qs * wz[c];
#pragma unroll
        for (int bb = 0; bb < W; ++bb) {
          const float qyz = qz * wy[bb];
          const int off = ((pz + c) * PD + py + bb) * PD + px;
#pragma unroll
          for (int a = 0; a < W; ++a) {
            int h, l;
            fx_split(qyz * wx[a], h, l);
            atomicAdd(phi_ + off + a, h);
            atomicAdd(plo + off + a, l);
          }
        }
      }
    } else {  // large charge, or outside the patch: straight to the global grid
      anterp_atom_global<ORDER>(f, b, G, gfx);
    }
  }
  if (total < 0) {  // more atoms than the list holds: one thread per atom, straight to the grid
    for (int c = 0; c < nk; ++c)
      for (int m = tid; m < ccount[c]; m += blockDim.x) {
        const int i = cstart[c] + m;
        anterp_atom_global<ORDER>(gfrac[i], gbase[i], G, gfx);
      }
  }
  __syncthreads();
  // flush: the point's value in 2^-31 units, h 2^19 + l, added to the global
  // fixed-point grid with an integer reduction (no FP64 arithmetic)
  for (int e = tid; e < np; e += blockDim.x) {
    const int h = phi_[e], l = plo[e];
    if ((h | l) == 0) continue;
    int ix = lo0 + e % PD, iy = lo1 + (e / PD) % PD, iz = lo2 + e / (PD * PD);
    if (!G.periodic && (ix < G.lo[0] || iy < G.lo[1] || iz < G.lo[2] || ix >= G.lo[0] + G.n[0] ||
                        iy >= G.lo[1] + G.n[1] || iz >= G.lo[2] + G.n[2]))
      continue;
    int sx = slot(ix, G.n[0], G.lo[0], G.periodic), sy = slot(iy, G.n[1], G.lo[1], G.periodic),
        sz = slot(iz, G.n[2], G.lo[2], G.periodic);
    atomicAdd(gfx + ((size_t)sz * G.n[1] + sy) * G.n[0] + sx,
              (unsigned long long)((long long)h * 524288LL + (long long)l));
  }
}

template <int ORDER>
__global__ void __launch_bounds__(256) k_anterp_fx(const R4<float>* __restrict__ gfrac, const int4* __restrict__ gbase,
                                                   const int* __restrict__ cell_start, AnterpArgs A, GridDims G,
                                                   unsigned long long* __restrict__ gfx) {
  anterp_fx_body<ORDER>(gfrac, gbase, cell_start, A, G, gfx, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Fixed-point level-0 charges (2^-31 units) to the FP64 grid, times the
// device-side scale: one conversion per grid point.
__device__ __forceinline__ void fx_to_f64_body(const unsigned long long* __restrict__ gfx, double* __restrict__ q0,
                                               int64_t count, const double* __restrict__ dscale, double factor,
                                               int64_t i) {
  if (i >= count) return;
  const double sc = factor * (dscale ? *dscale : 1.0) * (1.0 / 2147483648.0);
  q0[i] = (double)(long long)gfx[i] * sc;
}

__global__ void k_fx_to_f64(const unsigned long long* __restrict__ gfx, double* __restrict__ q0, int64_t count,
                            const double* __restrict__ dscale, double factor) {
  fx_to_f64_body(gfx, q0, count, dscale, factor, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

// ---- restriction and prolongation: separable 1-D passes ----
// phi^{k+1}_mu(r^k_nu) = prod_d Phi((nu_d - 2 mu_d)/2), so restriction is
// three 1-D filters (x, then y, then z) and prolongation, its transpose, the
// same filters in reverse order.  1-D weights Phi(d/2): cubic d = 0, +-1,
// +-3 -> 1, 9/16, -1/16; quintic d = 0, +-1, +-3, +-5 -> 1, 75/128, -25/256,
// 3/256 (Phi vanishes at the other integers).
template <int ORDER>
__device__ __forceinline__ double rweight(int ad) {
  if (ad == 0) return 1.0;
  if (ORDER == 3) return ad == 1 ? 9.0 / 16 : -1.0 / 16;
  return ad == 1 ? 75.0 / 128 : (ad == 3 ? -25.0 / 256 : 3.0 / 256);
}

struct AxisArgs {
  int nin[3], nout[3];  // array dims (x, y, z) of input and output
  int axis;             // 0, 1, 2
  int lo_in, lo_out;    // first absolute index along the axis
  int periodic;
};

// The output point t of an axis pass as (x, y, z): 32-bit divisions while
// the grid has fewer than 2^32 points (64-bit integer division is a long
// software sequence on the GPU), 64-bit beyond.
__device__ __forceinline__ void axis_point(int64_t t, const int nout[3], int64_t np, int c[3]) {
  if (np <= 0xffffffffLL) {
    const unsigned tu = (unsigned)t, n0 = (unsigned)nout[0], n1 = (unsigned)nout[1];
    const unsigned q = tu / n0;
    c[0] = (int)(tu - q * n0);
    c[1] = (int)(q % n1);
    c[2] = (int)(q / n1);
  } else {
    c[0] = (int)(t % nout[0]);
    c[1] = (int)((t / nout[0]) % nout[1]);
    c[2] = (int)(t / ((int64_t)nout[0] * nout[1]));
  }
}

// index s into [0, n) on a periodic axis: s is at most a few taps outside,
// so a wrap by additions replaces the integer modulo
__device__ __forceinline__ int wrap_periodic(int s, int n) {
  while (s < 0) s += n;
  while (s >= n) s -= n;
  return s;
}

// restriction along one axis: out[.., c, ..] = sum_d w(d) in[.., 2(lo_out + c) + d - lo_in, ..]
template <typename T, int ORDER>
__device__ __forceinline__ void restrict_axis_body(const T* __restrict__ in, T* __restrict__ out, const AxisArgs& A,
                                                   int64_t t) {
  constexpr int R = ORDER;  // taps reach |d| <= 2S - 1 = ORDER
  int64_t np = (int64_t)A.nout[0] * A.nout[1] * A.nout[2];
  if (t >= np) return;
  int c[3];
  axis_point(t, A.nout, np, c);
  int64_t stride = A.axis == 0 ? 1 : (A.axis == 1 ? (int64_t)A.nin[0] : (int64_t)A.nin[0] * A.nin[1]);
  int cc = c[A.axis];
  c[A.axis] = 0;
  const T* base = in + ((int64_t)c[2] * A.nin[1] + c[1]) * A.nin[0] + c[0];
  int n = A.nin[A.axis];
  int nu0 = 2 * (A.lo_out + cc);
  T sum = 0;
#pragma unroll
  for (int d = -R; d <= R; ++d) {
    if (d != 0 && (d & 1) == 0) continue;
    int s = nu0 + d - A.lo_in;
    if (A.periodic) {
      s = wrap_periodic(s, n);
    } else if (s < 0 || s >= n) {
      continue;
    }
    sum += T(rweight<ORDER>(d < 0 ? -d : d)) * base[s * stride];
  }
  out[t] = sum;
}

template <typename T, int ORDER>
__global__ void k_restrict_axis(const T* __restrict__ in, T* __restrict__ out, AxisArgs A) {
  restrict_axis_body<T, ORDER>(in, out, A, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

// prolongation along one axis: out[.., f, ..] (+)= sum_mu w(nu - 2 mu) in[.., mu - lo_in, ..]
template <typename T, int ORDER>
__device__ __forceinline__ void prolong_axis_body(const T* __restrict__ in, T* __restrict__ out, const AxisArgs& A,
                                                  int accumulate, int64_t t) {
  constexpr int R = ORDER;
  int64_t np = (int64_t)A.nout[0] * A.nout[1] * A.nout[2];
  if (t >= np) return;
  int c[3];
  axis_point(t, A.nout, np, c);
  int64_t stride = A.axis == 0 ? 1 : (A.axis == 1 ? (int64_t)A.nin[0] : (int64_t)A.nin[0] * A.nin[1]);
  int f = c[A.axis];
  c[A.axis] = 0;
  const T* base = in + ((int64_t)c[2] * A.nin[1] + c[1]) * A.nin[0] + c[0];
  int n = A.nin[A.axis];
  int nu = A.lo_out + f;
  T sum = 0;
#pragma unroll
  for (int d = -R; d <= R; ++d) {  // nu - 2 mu = d, d = 0 or odd
    if (d != 0 && (d & 1) == 0) continue;
    if (((nu - d) & 1) != 0) continue;
    int s = (nu - d) / 2 - A.lo_in;
    if (A.periodic) {
      s = wrap_periodic(s, n);
    } else if (s < 0 || s >= n) {
      continue;
    }
    sum += T(rweight<ORDER>(d < 0 ? -d : d)) * base[s * stride];
  }
  out[t] = accumulate ? out[t] + sum : sum;
}

template <typename T, int ORDER>
__global__ void k_prolong_axis(const T* __restrict__ in, T* __restrict__ out, AxisArgs A, int accumulate) {
  prolong_axis_body<T, ORDER>(in, out, A, accumulate, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

// ---- restriction and prolongation in one pass (small levels) ----
// The tensor product of the three axis passes above, each output point
// gathering its taps directly: the same taps in the same order and the same
// association (restriction: x innermost, then y, then z; prolongation: z
// innermost, then y, then x), so the result is bit-identical to the three
// passes; one launch instead of three and no temporaries.  Used where the
// gathered taps are few enough (see direct_budget).
struct Grid3Args {
  int nin[3], nout[3];  // array dims (x, y, z) of input and output
  int lo_in[3], lo_out[3];
  int periodic;
};

// The 1-D taps of a restriction output c in the axis pass's order (offsets
// -R, .., -1, 0, 1, .., R, odd or 0): input indices and weights in fixed
// slots; an open grid's taps outside the grid get weight 0 (adding 0 * v
// leaves a sum unchanged, so the result stays that of the pass, which skips
// them).
template <typename T, int ORDER>
__device__ __forceinline__ void restrict_taps(int c, int lo_out, int lo_in, int n, int periodic, int* s, T* w) {
  constexpr int R = ORDER;
  const int nu0 = 2 * (lo_out + c);
  int k = 0;
#pragma unroll
  for (int d = -R; d <= R; ++d) {
    if (d != 0 && (d & 1) == 0) continue;
    int t = nu0 + d - lo_in;
    T wt = T(rweight<ORDER>(d < 0 ? -d : d));
    if (periodic) {
      t = wrap_periodic(t, n);
    } else if (t < 0 || t >= n) {
      t = 0;
      wt = T(0);
    }
    s[k] = t;
    w[k] = wt;
    ++k;
  }
}

// The 1-D taps of a prolongation output f: an even index nu takes the one
// coarse point nu / 2 (offset 0), an odd one the ORDER + 1 points of the odd
// offsets -R .. R, in the axis pass's order; fixed slots as above.  Returns
// the slot count (1 or ORDER + 1).
template <typename T, int ORDER>
__device__ __forceinline__ int prolong_taps(int f, int lo_out, int lo_in, int n, int periodic, int* s, T* w) {
  constexpr int R = ORDER;
  const int nu = lo_out + f;
  if ((nu & 1) == 0) {
    int t = nu / 2 - lo_in;
    T wt = T(1);
    if (periodic) {
      t = wrap_periodic(t, n);
    } else if (t < 0 || t >= n) {
      t = 0;
      wt = T(0);
    }
    s[0] = t;
    w[0] = wt;
    return 1;
  }
  int k = 0;
#pragma unroll
  for (int d = -R; d <= R; d += 2) {  // the odd offsets
    int t = (nu - d) / 2 - lo_in;
    T wt = T(rweight<ORDER>(d < 0 ? -d : d));
    if (periodic) {
      t = wrap_periodic(t, n);
    } else if (t < 0 || t >= n) {
      t = 0;
      wt = T(0);
    }
    s[k] = t;
    w[k] = wt;
    ++k;
  }
  return R + 1;
}

template <typename T, int ORDER>
__global__ void k_restrict3(const T* __restrict__ in, T* __restrict__ out, Grid3Args A) {
  constexpr int NT = ORDER + 2;  // offsets 0 and the odd ones up to ORDER
  const int np = A.nout[0] * A.nout[1] * A.nout[2];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= np) return;
  const int c[3] = {t % A.nout[0], (t / A.nout[0]) % A.nout[1], t / (A.nout[0] * A.nout[1])};
  int sx[NT], sy[NT], sz[NT];
  T wx[NT], wy[NT], wz[NT];
  restrict_taps<T, ORDER>(c[0], A.lo_out[0], A.lo_in[0], A.nin[0], A.periodic, sx, wx);
  restrict_taps<T, ORDER>(c[1], A.lo_out[1], A.lo_in[1], A.nin[1], A.periodic, sy, wy);
  restrict_taps<T, ORDER>(c[2], A.lo_out[2], A.lo_in[2], A.nin[2], A.periodic, sz, wz);
  T acc = 0;
#pragma unroll
  for (int iz = 0; iz < NT; ++iz) {
    T ay = 0;
#pragma unroll
    for (int iy = 0; iy < NT; ++iy) {
      const T* row = in + ((size_t)sz[iz] * A.nin[1] + sy[iy]) * A.nin[0];
      T ax = 0;
#pragma unroll
      for (int ix = 0; ix < NT; ++ix) ax += wx[ix] * row[sx[ix]];
      ay += wy[iy] * ax;
    }
    acc += wz[iz] * ay;
  }
  out[t] = acc;
}

template <typename T, int ORDER>
__global__ void k_prolong3(const T* __restrict__ in, T* __restrict__ out, Grid3Args A) {
  constexpr int NO = ORDER + 1;  // the odd offsets
  const int np = A.nout[0] * A.nout[1] * A.nout[2];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= np) return;
  const int f[3] = {t % A.nout[0], (t / A.nout[0]) % A.nout[1], t / (A.nout[0] * A.nout[1])};
  int sx[NO], sy[NO], sz[NO];
  T wx[NO], wy[NO], wz[NO];
  const int kx = prolong_taps<T, ORDER>(f[0], A.lo_out[0], A.lo_in[0], A.nin[0], A.periodic, sx, wx);
  const int ky = prolong_taps<T, ORDER>(f[1], A.lo_out[1], A.lo_in[1], A.nin[1], A.periodic, sy, wy);
  const int kz = prolong_taps<T, ORDER>(f[2], A.lo_out[2], A.lo_in[2], A.nin[2], A.periodic, sz, wz);
  T acc = 0;
#pragma unroll
  for (int ix = 0; ix < NO; ++ix) {
    if (ix < kx) {
      T ay = 0;
#pragma unroll
      for (int iy = 0; iy < NO; ++iy) {
        if (iy < ky) {
          T az = 0;
#pragma unroll
          for (int iz = 0; iz < NO; ++iz)
            if (iz < kz) az += wz[iz] * in[((size_t)sz[iz] * A.nin[1] + sy[iy]) * A.nin[0] + sx[ix]];
          ay += wy[iy] * az;
        }
      }
      acc += wx[ix] * ay;
    }
  }
  out[t] = out[t] + acc;  // onto u^{k, cutoff}
}

// ---- lattice cutoff: z-streaming shared-memory planes, register tiles ----
// A block of 4 warps owns a brick of outputs 32 (x) x LBY (y) x 4 (z); warp w
// owns plane z0 + w.  The input planes are staged one at a time in shared
// memory (a 2-D window with halo Ex, Ey; odd row pitch so the lanes of a warp
// sit on distinct banks); for staged plane zi, warp w applies the stencil rows
// of dz = zi - (z0 + w) as segments of 8 taps along x on register tiles of
// 8 consecutive x outputs per lane.  Coarse levels with few bricks split the
// input planes over several blocks (nsplit) that add their partial sums into
// the zeroed output; per-plane partial sums are folded into the totals with
// TwoSum in mixed precision.
//   FP64: one row per lane (LBY = 8), scalar FMA.
//   FP32: two rows per lane (LBY = 16) packed into float2, one FFMA2 per two
//         outputs, coefficients stored pre-duplicated as float2 pairs.
constexpr int LBX = 32, LBZ = 4, LPX = 8;
constexpr int kLatticeLP = 8;   // x outputs per lane of the FP32 lattice kernel (8 or 16)
constexpr int kLatticeZ = 4;    // warps (output planes) per block of the FP32 lattice kernel
constexpr size_t kLatticeSmemMax = 200 * 1024;  // dynamic shared memory the FP32 lattice kernels may use

template <typename T>
__device__ __forceinline__ void two_sum_add(T& s, T& c, T x) {
  T t = s + x;
  T bp = t - s;
  c += (s - (t - bp)) + (x - bp);
  s = t;
}

// Stages plane zi of q into plane[] (rows SY, staged width SXw, pitch SX).
template <typename T>
__device__ __forceinline__ void stage_plane(T* plane, const T* __restrict__ q, const GridDims& G, int zi, int x0,
                                            int y0, int Ex, int Ey, int SXw, int SX, int SY) {
  int gz;
  bool zok;
  if (G.periodic) {
    gz = zi % G.n[2];
    if (gz < 0) gz += G.n[2];
    zok = true;
  } else {
    gz = zi;
    zok = (zi >= 0 && zi < G.n[2]);
  }
  for (int e = threadIdx.x; e < SY * SXw; e += blockDim.x) {
    int xx = e % SXw, yy = e / SXw;
    int gx = x0 - Ex + xx, gy = y0 - Ey + yy;
    T v = T(0);
    if (G.periodic) {
      gx %= G.n[0];
      if (gx < 0) gx += G.n[0];
      gy %= G.n[1];
      if (gy < 0) gy += G.n[1];
      v = q[((size_t)gz * G.n[1] + gy) * G.n[0] + gx];
    } else if (zok && gx >= 0 && gx < G.n[0] && gy >= 0 && gy < G.n[1]) {
      v = q[((size_t)gz * G.n[1] + gy) * G.n[0] + gx];
    }
    plane[yy * SX + xx] = v;
  }
}

struct LatticeArgs {
  int Ex, Ey, Ez;
  int nsplit;  // blocks sharing one brick's input planes
  int nbz;     // bricks along z
  int txn, tyn;  // FP32 kernel: lanes along x (LP outputs each) and along y (two rows each) of a warp's tile
};

// When several blocks share a brick's input planes (L.nsplit > 1), block
// part writes its partial sums to up[part][point] and k_lattice_reduce adds
// the parts in order: no atomics, so the sums are reproducible.
template <typename T, bool COMP>
__global__ void __launch_bounds__(128) k_lattice(const T* __restrict__ q, T* __restrict__ u, T* __restrict__ up,
                                                 GridDims G, const Segment<T>* __restrict__ seg,
                                                 const int* __restrict__ seg_start, LatticeArgs L, T scale) {
  constexpr int LBY = 8;
  extern __shared__ unsigned char smem_raw[];
  T* plane = reinterpret_cast<T*>(smem_raw);
  const int Ex = L.Ex, Ey = L.Ey, Ez = L.Ez;
  const int SXw = LBX + 2 * Ex + kSeg, SX = SXw | 1, SY = LBY + 2 * Ey;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, tx = lane & 3, ty = lane >> 2;
  const int bz = blockIdx.z % L.nbz, part = blockIdx.z / L.nbz;
  const int x0 = blockIdx.x * LBX, y0 = blockIdx.y * LBY, z0 = bz * LBZ, zo = z0 + warp;
  const int nplanes = LBZ + 2 * Ez, per = (nplanes + L.nsplit - 1) / L.nsplit;
  const int zbeg = z0 - Ez + part * per, zend = min(z0 - Ez + nplanes, zbeg + per);
  T acc[LPX], cmp[LPX];
#pragma unroll
  for (int j = 0; j < LPX; ++j) acc[j] = cmp[j] = T(0);
  for (int zi = zbeg; zi < zend; ++zi) {
    __syncthreads();
    stage_plane(plane, q, G, zi, x0, y0, Ex, Ey, SXw, SX, SY);
    __syncthreads();
    const int dz = zi - zo;
    if (dz < -Ez || dz > Ez || zo >= G.n[2]) continue;  // warp-uniform
    T part_[LPX];
#pragma unroll
    for (int j = 0; j < LPX; ++j) part_[j] = T(0);
    const int s1 = seg_start[dz + Ez + 1];
    for (int s = seg_start[dz + Ez]; s < s1; ++s) {
      const Segment<T> sg = seg[s];
      const T* row = plane + (ty + Ey + sg.dy) * SX + tx * LPX + Ex + sg.dx0;
      T win[LPX + kSeg - 1];
#pragma unroll
      for (int k = 0; k < LPX + kSeg - 1; ++k) win[k] = row[k];
#pragma unroll
      for (int k = 0; k < kSeg; ++k)
#pragma unroll
        for (int j = 0; j < LPX; ++j) part_[j] += sg.g[k] * win[j + k];
    }
#pragma unroll
    for (int j = 0; j < LPX; ++j) {
      if (COMP) two_sum_add(acc[j], cmp[j], part_[j]);
      else acc[j] += part_[j];
    }
  }
  if (zo >= G.n[2]) return;
  const int y = y0 + ty;
  if (y >= G.n[1]) return;
#pragma unroll
  for (int j = 0; j < LPX; ++j) {
    int x = x0 + tx * LPX + j;
    if (x >= G.n[0]) continue;
    T v = scale * (acc[j] + cmp[j]);
    const size_t o = ((size_t)zo * G.n[1] + y) * G.n[0] + x;
    if (L.nsplit > 1) up[(size_t)part * G.n[0] * G.n[1] * G.n[2] + o] = v;
    else u[o] = v;
  }
}

// Window offsets of a block, computed once (the periodic wrap costs integer
// divisions): col[xx] = grid x index of window column xx (-1 outside an open
// grid), row[yy] = (grid y index) * n_x (-1 outside).
__device__ __forceinline__ void window_offsets(const GridDims& G, int x0, int y0, int Ex, int Ey, int SXw, int SY,
                                               int* col, int* row) {
  for (int t = threadIdx.x; t < SXw + SY; t += blockDim.x) {
    const bool isx = t < SXw;
    const int n = isx ? G.n[0] : G.n[1];
    int g = isx ? x0 - Ex + t : y0 - Ey + (t - SXw);
    if (G.periodic) {
      g %= n;
      if (g < 0) g += n;
    } else if (g < 0 || g >= n) {
      g = -1;
    }
    if (isx) col[t] = g;
    else row[t - SXw] = g < 0 ? -1 : g * G.n[0];
  }
}

// Asynchronous staging of one plane (cp.async: global -> shared without
// registers); points outside an open grid are zero-filled (source size 0).
// Each thread walks the window with a fixed stride of blockDim.x elements,
// stepping its (row, column) incrementally.  Window rows are stored even rows
// first, then odd rows (row yy at yy / 2 + (yy odd) * SY / 2): lanes reading
// rows 2 ty + c then read rows ty apart, one odd row stride SX apart, which
// keeps the lanes of a warp on distinct banks.
__device__ __forceinline__ void stage_plane_async(float* plane, const float* __restrict__ q, const GridDims& G,
                                                  int zi, const int* col, const int* row, int SXw, int SX, int SY) {
  int gz;
  bool zok;
  if (G.periodic) {
    gz = zi % G.n[2];
    if (gz < 0) gz += G.n[2];
    zok = true;
  } else {
    gz = zi;
    zok = (zi >= 0 && zi < G.n[2]);
  }
  const float* qz = q + (size_t)(zok ? gz : 0) * G.n[1] * G.n[0];
  const int step = blockDim.x, dyy = step / SXw, dxx = step - dyy * SXw;
  int xx = threadIdx.x % SXw, yy = threadIdx.x / SXw;
  for (; yy < SY; ) {
    const int gx = col[xx], go = row[yy];
    const bool ok = zok && gx >= 0 && go >= 0;
    const float* src = ok ? qz + go + gx : q;
    unsigned dst = (unsigned)__cvta_generic_to_shared(plane + ((yy >> 1) + (yy & 1) * (SY >> 1)) * SX + xx);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(src), "r"(ok ? 4 : 0));
    xx += dxx;
    yy += dyy;
    if (xx >= SXw) {
      xx -= SXw;
      ++yy;
    }
  }
}

// FP32: each lane owns LP consecutive x outputs of two adjacent rows (y,
// y + 1), packed into float2 (one FFMA2 per two outputs); a warp covers TXN LP
// (x) x 2 TYN (y) of one plane.  An input row y + e feeds both outputs, row y
// through the taps of stencil row e and row y + 1 through those of row e - 1,
// so the table holds those coefficient pairs and one shared load serves both
// rows (against two rows TYN apart with one coefficient each: 5% faster on
// the 1.07M-atom system, 9% on the 64-replica batch).  The next input plane
// is staged by cp.async while the current one is applied (double buffer).  A
// segment of 8 taps is applied as a sliding window: input column k feeds the
// outputs j = k - t of every tap t, so one shared load serves up to 8 FFMA2
// (LP + 7 loads per 8 LP FFMA2); the row pairing costs 2 Ey + 2 input rows per
// output pair instead of 2 Ey + 1.  The block's warps share each input plane
// and apply to it different stencil planes dz, of unequal size, so a warp
// may wait at the plane's barrier; stepping the warps through dz together
// (each on its own input plane, a ring of kLatticeZ + 1 buffers) removes the
// wait but measured 15-20% slower, the larger ring costing resident blocks.  Taps accumulate straight into the outputs (summing each
// plane first measured no different on the 1.07M-atom system: mixed-vs-FP64
// energy 4.4e-8, force 4.9e-7).
// TXC, TYC: the warp tile fixed at compile time (the common 32 x 16 tile),
// or 0 to take it from L (other shapes, batches of uneven grids).
template <int LP, int TXC, int TYC>
__device__ __forceinline__ void lattice_f2_body(const float* __restrict__ q, float* __restrict__ u,
                                                float* __restrict__ up, const GridDims G,
                                                const Segment2* __restrict__ seg, const int* __restrict__ seg_start,
                                                const LatticeArgs L, float scale, int bx, int by, int bzs) {
  const int TXN = TXC ? TXC : L.txn, TYN = TYC ? TYC : L.tyn, TW = LP * TXN, LBY = 2 * TYN;  // tile: TW (x) by LBY (y)
  extern __shared__ unsigned char smem_raw[];
  const int Ex = L.Ex, Ey = L.Ey, Ez = L.Ez;
  const int SXw = TW + 2 * Ex + kSeg, SX = SXw | 1, SY = LBY + 2 * Ey;
  float* buf0 = reinterpret_cast<float*>(smem_raw);
  float* buf1 = buf0 + SX * SY;
  int* col = reinterpret_cast<int*>(buf1 + SX * SY);  // window offsets (SXw + SY ints)
  int* row = col + SXw;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, tx = lane % TXN, ty = lane / TXN;
  const bool active = (TXC * TYC == 32) || ty < TYN;  // lanes past TXN * TYN only help with staging
  const int bz = bzs % L.nbz, part = bzs / L.nbz;
  const int x0 = bx * TW, y0 = by * LBY, z0 = bz * kLatticeZ, zo = z0 + warp;
  const int nplanes = kLatticeZ + 2 * Ez, per = (nplanes + L.nsplit - 1) / L.nsplit;
  const int zbeg = z0 - Ez + part * per, zend = min(z0 - Ez + nplanes, zbeg + per);
  float2 acc[LP];  // (row 2 ty, row 2 ty + 1) of the LP x outputs
#pragma unroll
  for (int j = 0; j < LP; ++j) acc[j] = make_float2(0.f, 0.f);
  window_offsets(G, x0, y0, Ex, Ey, SXw, SY, col, row);
  __syncthreads();
  if (zbeg < zend) stage_plane_async(buf0, q, G, zbeg, col, row, SXw, SX, SY);
  asm volatile("cp.async.commit_group;\n" ::);
  for (int zi = zbeg; zi < zend; ++zi) {
    float* cur = ((zi - zbeg) & 1) ? buf1 : buf0;
    float* nxt = ((zi - zbeg) & 1) ? buf0 : buf1;
    if (zi + 1 < zend) stage_plane_async(nxt, q, G, zi + 1, col, row, SXw, SX, SY);
    asm volatile("cp.async.commit_group;\n" ::);
    asm volatile("cp.async.wait_group 1;\n" ::);  // plane zi has landed (this thread's copies)
    __syncthreads();                               // ... and everyone else's
    const int dz = zi - zo;
    if (active && dz >= -Ez && dz <= Ez && zo < G.n[2]) {
      const int s1 = seg_start[dz + Ez + 1];
#pragma unroll 2  // the next segment's coefficients load under this one's FMAs
      for (int s = seg_start[dz + Ez]; s < s1; ++s) {
        const Segment2 sg = seg[s];
        const int c = Ey + sg.dy;  // window row 2 ty + c, stored at ty + c / 2 (+ SY / 2 when c is odd)
        const float* r0 = cur + (ty + (c >> 1) + (c & 1) * (SY >> 1)) * SX + tx * LP + Ex + sg.dx0;
#pragma unroll
        for (int k = 0; k < LP + kSeg - 1; ++k) {
          const float v = r0[k];
          const float2 w = make_float2(v, v);
#pragma unroll
          for (int t = 0; t < kSeg; ++t)
            if (k - t >= 0 && k - t < LP) acc[k - t] = __ffma2_rn(sg.g[t], w, acc[k - t]);
        }
      }
    }
    __syncthreads();  // the buffer just read is restaged two planes from now
  }
  asm volatile("cp.async.wait_group 0;\n" ::);
  if (zo >= G.n[2] || !active) return;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int y = y0 + 2 * ty + r;
    if (y >= G.n[1]) continue;
#pragma unroll
    for (int j = 0; j < LP; ++j) {
      int x = x0 + tx * LP + j;
      if (x >= G.n[0]) continue;
      float v = scale * (r == 0 ? acc[j].x : acc[j].y);
      const size_t o = ((size_t)zo * G.n[1] + y) * G.n[0] + x;
      if (L.nsplit > 1) up[(size_t)part * G.n[0] * G.n[1] * G.n[2] + o] = v;  // summed in order by k_lattice_reduce
      else u[o] = v;
    }
  }
}

template <int LP, int TXC, int TYC>
__global__ void __launch_bounds__(32 * kLatticeZ, 6) k_lattice_f2(const float* __restrict__ q, float* __restrict__ u,
                                                               float* __restrict__ up, GridDims G,
                                                               const Segment2* __restrict__ seg,
                                                               const int* __restrict__ seg_start, LatticeArgs L,
                                                               float scale) {
  lattice_f2_body<LP, TXC, TYC>(q, u, up, G, seg, seg_start, L, scale, blockIdx.x, blockIdx.y, blockIdx.z);
}

// u[i] = sum over the parts p = 0..nsplit-1 of up[p][i], in that order.
template <typename T>
__device__ __forceinline__ void lattice_reduce_body(const T* __restrict__ up, T* __restrict__ u, int64_t np,
                                                    int nsplit, int64_t i) {
  if (i >= np) return;
  T v = up[i];
  for (int p = 1; p < nsplit; ++p) v += up[(size_t)p * np + i];
  u[i] = v;
}

template <typename T>
__global__ void __launch_bounds__(256) k_lattice_reduce(const T* __restrict__ up, T* __restrict__ u, int64_t np,
                                                        int nsplit) {
  lattice_reduce_body<T>(up, u, np, nsplit, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

// ---- top level: all pairs of the coarsest grid, FP64 ----
// One warp per output point: the lanes split the sum over the points of the
// coarsest grid and combine their FP64 partial sums with shuffles.
template <typename T>
__device__ __forceinline__ void top_body(const double* __restrict__ qt, T* __restrict__ ut, double* __restrict__ ut64,
                                         const GridDims& G, const double* __restrict__ K, int tx, int ty,
                                         int64_t m) {
  const int lane = threadIdx.x & 31;
  const int n0 = G.n[0], n1 = G.n[1], n2 = G.n[2];
  const int np = n0 * n1 * n2;
  if (m >= np) return;  // warp-uniform
  const int mx = (int)(m % n0), my = (int)((m / n0) % n1), mz = (int)(m / ((int64_t)n0 * n1));
  double sum = 0.0;
  for (int v = lane; v < np; v += 32) {
    const int vx = v % n0, vy = (v / n0) % n1, vz = v / (n0 * n1);
    int dx = mx - vx, dy = my - vy, dz = mz - vz;
    if (G.periodic) {
      dx += dx < 0 ? n0 : 0;
      dy += dy < 0 ? n1 : 0;
      dz += dz < 0 ? n2 : 0;
    } else {
      dx += n0 - 1;
      dy += n1 - 1;
      dz += n2 - 1;
    }
    sum += K[((size_t)dz * ty + dy) * tx + dx] * qt[v];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if (lane == 0) {
    ut[m] = (T)sum;
    ut64[m] = sum;
  }
}

constexpr int kTopWarps = 4;  // output points per block of the top-level kernel

template <typename T>
__global__ void __launch_bounds__(32 * kTopWarps) k_top(const double* __restrict__ qt, T* __restrict__ ut,
                                                        double* __restrict__ ut64, GridDims G,
                                                        const double* __restrict__ K, int tx, int ty, int tz) {
  top_body<T>(qt, ut, ut64, G, K, tx, ty, (int64_t)blockIdx.x * kTopWarps + (threadIdx.x >> 5));
  (void)tz;
}

// ---- interpolation at the atoms and assembly (forward) ----
template <typename T, int ORDER>
__device__ __forceinline__ void interp_atom(const R4<T>& f, const int4& b, const T* __restrict__ u0,
                                            const GridDims& G, const T inv_h[3], T& p, T g[3]) {
  constexpr int W = 2 * Basis<T, ORDER>::S;
  T wx[W], wy[W], wz[W], dx[W], dy[W], dz[W];
  weights<T, ORDER>(f.x, wx);
  weights<T, ORDER>(f.y, wy);
  weights<T, ORDER>(f.z, wz);
  dweights<T, ORDER>(f.x, dx);
  dweights<T, ORDER>(f.y, dy);
  dweights<T, ORDER>(f.z, dz);
  int ix[W], iy[W], iz[W];
#pragma unroll
  for (int s = 0; s < W; ++s) {
    ix[s] = slot(b.x + s, G.n[0], G.lo[0], G.periodic);
    iy[s] = slot(b.y + s, G.n[1], G.lo[1], G.periodic);
    iz[s] = slot(b.z + s, G.n[2], G.lo[2], G.periodic);
  }
  T P = 0, Gx = 0, Gy = 0, Gz = 0;
#pragma unroll
  for (int c = 0; c < W; ++c) {
    T pz = 0, gxz = 0, gyz = 0;
#pragma unroll
    for (int bb = 0; bb < W; ++bb) {
      const T* row = u0 + ((size_t)iz[c] * G.n[1] + iy[bb]) * G.n[0];
      T sa = 0, sd = 0;
#pragma unroll
      for (int a = 0; a < W; ++a) {
        T v = __ldg(row + ix[a]);
        sa += wx[a] * v;
        sd += dx[a] * v;
      }
      pz += wy[bb] * sa;
      gxz += wy[bb] * sd;
      gyz += dy[bb] * sa;
    }
    P += wz[c] * pz;
    Gx += wz[c] * gxz;
    Gy += wz[c] * gyz;
    Gz += dz[c] * pz;
  }
  p = P;
  g[0] = Gx * inv_h[0];
  g[1] = Gy * inv_h[1];
  g[2] = Gz * inv_h[2];
}

template <int BLOCK>
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[BLOCK / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (w == 0) {
    s = (lane < BLOCK / 32) ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  return s;  // valid in thread 0
}

struct AssembleArgs {
  double self_c;  // gamma(0)/a
  double kc;      // Coulomb prefactor
  double inv_h[3];
  float self_cf, kcf;  // the same in FP32 (mixed plans assemble in FP32)
};

// Per-atom assembly of phi_i, F_i (forward) and of dL/dq_i, dL/dr_i
// (adjoint).  The mixed plan works in FP32 and converts once per output (FP64
// operations, conversions included, issue at 1/64 of the FP32 rate here); the
// FP64 plan works in FP64.
template <typename T>
struct Assemble;
template <>
struct Assemble<float> {
  template <typename OUT>
  __device__ static double forward(const AssembleArgs& A, float q, float phis, float p, const R4<float>& s,
                                   const float g[3], int o, OUT* phi_out, OUT* force_out) {
    const float phi = A.kcf * ((phis + p) - q * A.self_cf);
    if (phi_out) phi_out[o] = (OUT)phi;
    if (force_out) {
      force_out[3 * (size_t)o + 0] = (OUT)(A.kcf * (s.x - q * g[0]));
      force_out[3 * (size_t)o + 1] = (OUT)(A.kcf * (s.y - q * g[1]));
      force_out[3 * (size_t)o + 2] = (OUT)(A.kcf * (s.z - q * g[2]));
    }
    return (double)(q * phi);
  }
  template <typename OUT>
  __device__ static void backward(const AssembleArgs& A, float gg, float q, float phis, const R4<float>& s,
                                  const R4<float>& gl, float v, const float gv[3], int o, OUT* grad_pos,
                                  OUT* grad_q) {
    const float hg = 0.5f * gg;
    if (grad_q) grad_q[o] = (OUT)(A.kcf * (gg * (phis - q * A.self_cf) + hg * gl.w + v));
    if (grad_pos) {
      grad_pos[3 * (size_t)o + 0] = (OUT)(A.kcf * (-gg * s.x + hg * q * gl.x + q * gv[0]));
      grad_pos[3 * (size_t)o + 1] = (OUT)(A.kcf * (-gg * s.y + hg * q * gl.y + q * gv[1]));
      grad_pos[3 * (size_t)o + 2] = (OUT)(A.kcf * (-gg * s.z + hg * q * gl.z + q * gv[2]));
    }
  }
};
template <>
struct Assemble<double> {
  template <typename OUT>
  __device__ static double forward(const AssembleArgs& A, double q, double phis, double p, const R4<double>& s,
                                   const double g[3], int o, OUT* phi_out, OUT* force_out) {
    const double phi = A.kc * (phis + p - q * A.self_c);
    if (phi_out) phi_out[o] = (OUT)phi;
    if (force_out) {
      force_out[3 * (size_t)o + 0] = (OUT)(A.kc * (s.x - q * g[0]));
      force_out[3 * (size_t)o + 1] = (OUT)(A.kc * (s.y - q * g[1]));
      force_out[3 * (size_t)o + 2] = (OUT)(A.kc * (s.z - q * g[2]));
    }
    return q * phi;
  }
  template <typename OUT>
  __device__ static void backward(const AssembleArgs& A, double gg, double q, double phis, const R4<double>& s,
                                  const R4<double>& gl, double v, const double gv[3], int o, OUT* grad_pos,
                                  OUT* grad_q) {
    if (grad_q) grad_q[o] = (OUT)(A.kc * (gg * (phis - q * A.self_c) + 0.5 * gg * gl.w + v));
    if (grad_pos) {
      grad_pos[3 * (size_t)o + 0] = (OUT)(A.kc * (-gg * s.x + 0.5 * gg * q * gl.x + q * gv[0]));
      grad_pos[3 * (size_t)o + 1] = (OUT)(A.kc * (-gg * s.y + 0.5 * gg * q * gl.y + q * gv[1]));
      grad_pos[3 * (size_t)o + 2] = (OUT)(A.kc * (-gg * s.z + 0.5 * gg * q * gl.z + q * gv[2]));
    }
  }
};

// Interpolation through the same per-block patches: a block stages the u^0
// points its atoms can reach (PD^3, wrapped) in shared memory, then each
// thread gathers its atoms' (2S)^3 taps from there.
template <typename T, int ORDER>
__device__ __forceinline__ void interp_patch_atom(const R4<T>& f, const int4& b, const T* __restrict__ patch, int PD,
                                                  int lo0, int lo1, int lo2, const T* __restrict__ u0,
                                                  const GridDims& G, const T ih[3], T& p, T g[3]) {
  constexpr int W = 2 * Basis<T, ORDER>::S;
  const int px = b.x - lo0, py = b.y - lo1, pz = b.z - lo2;
  if (px >= 0 && py >= 0 && pz >= 0 && px + W <= PD && py + W <= PD && pz + W <= PD) {
    T wx[W], wy[W], wz[W], dx[W], dy[W], dz[W];
    weights<T, ORDER>(f.x, wx);
    weights<T, ORDER>(f.y, wy);
    weights<T, ORDER>(f.z, wz);
    dweights<T, ORDER>(f.x, dx);
    dweights<T, ORDER>(f.y, dy);
    dweights<T, ORDER>(f.z, dz);
    T P = 0, Gx = 0, Gy = 0, Gz = 0;
#pragma unroll
    for (int c = 0; c < W; ++c) {
      T pzv = 0, gxz = 0, gyz = 0;
#pragma unroll
      for (int bb = 0; bb < W; ++bb) {
        const T* row = patch + ((pz + c) * PD + py + bb) * PD + px;
        T sa = 0, sd = 0;
#pragma unroll
        for (int a = 0; a < W; ++a) {
          T v = row[a];
          sa += wx[a] * v;
          sd += dx[a] * v;
        }
        pzv += wy[bb] * sa;
        gxz += wy[bb] * sd;
        gyz += dy[bb] * sa;
      }
      P += wz[c] * pzv;
      Gx += wz[c] * gxz;
      Gy += wz[c] * gyz;
      Gz += dz[c] * pzv;
    }
    p = P;
    g[0] = Gx * ih[0];
    g[1] = Gy * ih[1];
    g[2] = Gz * ih[2];
  } else {
    interp_atom<T, ORDER>(f, b, u0, G, ih, p, g);
  }
}

// Lists the block's atoms (rank-major, then bank-ordered with the patch as
// scratch: the gathers of one warp instruction then read 32 different banks)
// and stages the patch of u^0 for the block at cell block c0.  Returns the
// slot count of the list (unfilled slots hold -1), or -1 when the block holds
// more atoms than the list takes.
template <typename T>
__device__ __forceinline__ int stage_interp_block(const AnterpArgs& A, const int* __restrict__ cell_start,
                                                  const int4* __restrict__ gbase, const T* __restrict__ u0,
                                                  const GridDims& G, T* patch, int lo0, int lo1, int lo2, int* cstart,
                                                  int* ccount, int* list, int* nk_s, int* tot_s, int bx, int by,
                                                  int bz) {
  const int PD = A.pd, np = PD * PD * PD;
  const int c0[3] = {bx * A.B, by * A.B, bz * A.B};
  if (threadIdx.x == 0) *nk_s = block_cells(A, cell_start, c0, cstart, ccount);
  __syncthreads();
  int total = build_rank_list(*nk_s, cstart, ccount, list, tot_s);
  if (total >= 0)
    total = bank_order(list, total, gbase, lo0, lo1, lo2, PD, reinterpret_cast<int*>(patch),
                       np * (int)(sizeof(T) / sizeof(int)));
  for (int e = threadIdx.x; e < np; e += blockDim.x) {
    int ix = lo0 + e % PD, iy = lo1 + (e / PD) % PD, iz = lo2 + e / (PD * PD);
    T v = T(0);
    if (G.periodic) {
      v = u0[((size_t)slot(iz, G.n[2], 0, 1) * G.n[1] + slot(iy, G.n[1], 0, 1)) * G.n[0] + slot(ix, G.n[0], 0, 1)];
    } else if (ix >= G.lo[0] && iy >= G.lo[1] && iz >= G.lo[2] && ix < G.lo[0] + G.n[0] && iy < G.lo[1] + G.n[1] &&
               iz < G.lo[2] + G.n[2]) {
      v = u0[((size_t)(iz - G.lo[2]) * G.n[1] + (iy - G.lo[1])) * G.n[0] + (ix - G.lo[0])];
    }
    patch[e] = v;
  }
  __syncthreads();
  return total;
}

// Arguments of the interpolation kernels (one system): the forward kernel
// writes phi_out, force_out, fs.w, glong and the per-block energy partials;
// the adjoint kernel reads fs and glong and writes grad_pos, grad_q.
template <typename T, typename OUT>
struct InterpKArgs {
  const R4<T>* gfrac;
  const int4* gbase;
  const int* perm;
  const int* cell_start;
  AnterpArgs AA;
  const T* u0;  // u^0 (forward) or the adjoint grid (backward)
  GridDims G;
  AssembleArgs A;
  const T* phis;
  R4<T>* fs;
  R4<T>* glong;
  OUT* phi_out;
  OUT* force_out;
  double* partial;
  const double* gE;
  OUT* grad_pos;
  OUT* grad_q;
  int nbx, nby;  // blocks along x and y
};

// GATHER: interpolate only (u_long and its gradient into glong; no pair
// results needed, so this runs while the pair sums are still being computed),
// else also assemble phi, F and the energy partials.
template <typename T, int ORDER, typename OUT, bool GATHER = false>
__device__ __forceinline__ void interp_fwd_body(
    const R4<T>* __restrict__ gfrac, const int4* __restrict__ gbase, const int* __restrict__ perm,
    const int* __restrict__ cell_start, const AnterpArgs& AA, const T* __restrict__ u0, const GridDims& G,
    const AssembleArgs& A, const T* __restrict__ phis, R4<T>* __restrict__ fs, R4<T>* __restrict__ glong,
    OUT* __restrict__ phi_out, OUT* __restrict__ force_out, double* __restrict__ partial, int bx, int by, int bz,
    int lin) {
  constexpr int S = Basis<T, ORDER>::S;
  extern __shared__ unsigned char smem_raw[];
  T* patch = reinterpret_cast<T*>(smem_raw);
  __shared__ int cstart[64], ccount[64], list[kAnterpMaxAtoms + 32], nk_s, tot_s;  // + one round of slots
  const int c0[3] = {bx * AA.B, by * AA.B, bz * AA.B};
  const int lo0 = (int)floor(c0[0] * AA.cw_h[0]) - S - 1;
  const int lo1 = (int)floor(c0[1] * AA.cw_h[1]) - S - 1;
  const int lo2 = (int)floor(c0[2] * AA.cw_h[2]) - S - 1;
  const int total = stage_interp_block<T>(AA, cell_start, gbase, u0, G, patch, lo0, lo1, lo2, cstart, ccount, list,
                                          &nk_s, &tot_s, bx, by, bz);
  const T ih[3] = {T(A.inv_h[0]), T(A.inv_h[1]), T(A.inv_h[2])};
  double e = 0.0;
  const int nk = nk_s;
  // atoms from the list, or (over-full block) walked cell by cell
  const int nlist = total >= 0 ? total : 0;
  int walk_c = 0, walk_m = threadIdx.x;
  for (int kk = threadIdx.x;; kk += blockDim.x) {
    int i;
    if (total >= 0) {
      if (kk >= nlist) break;
      i = list[kk];
      if (i < 0) continue;  // unfilled slot of the bank-ordered list
    } else {
      while (walk_c < nk && walk_m >= ccount[walk_c]) walk_m -= ccount[walk_c++];
      if (walk_c >= nk) break;
      i = cstart[walk_c] + walk_m;
      walk_m += blockDim.x;
    }
    const R4<T> f = gfrac[i];
    T p, g[3];
    interp_patch_atom<T, ORDER>(f, gbase[i], patch, AA.pd, lo0, lo1, lo2, u0, G, ih, p, g);
    if (!GATHER) e += Assemble<T>::forward(A, f.w, phis[i], p, fs[i], g, perm[i], phi_out, force_out);
    glong[i] = R4<T>{g[0], g[1], g[2], p};
  }
  if (!GATHER) {
    double bsum = block_sum<256>(e);
    if (threadIdx.x == 0) partial[lin] = bsum;
  }
}

template <typename T, int ORDER, typename OUT>
__device__ __forceinline__ void interp_fwd_call(const InterpKArgs<T, OUT>& K, int bx, int by, int bz, int lin) {
  interp_fwd_body<T, ORDER, OUT>(K.gfrac, K.gbase, K.perm, K.cell_start, K.AA, K.u0, K.G, K.A, K.phis, K.fs, K.glong,
                                 K.phi_out, K.force_out, K.partial, bx, by, bz, lin);
}

template <typename T, int ORDER>
__global__ void __launch_bounds__(256, 3) k_interp_gather(const R4<T>* __restrict__ gfrac,
                                                          const int4* __restrict__ gbase,
                                                          const int* __restrict__ cell_start, AnterpArgs AA,
                                                          const T* __restrict__ u0, GridDims G, AssembleArgs A,
                                                          R4<T>* __restrict__ glong) {
  interp_fwd_body<T, ORDER, double, true>(gfrac, gbase, nullptr, cell_start, AA, u0, G, A, nullptr, nullptr, glong,
                                          nullptr, nullptr, nullptr, blockIdx.x, blockIdx.y, blockIdx.z, 0);
}

// Assembly after the pair sums and the gather: phi_i, F_i in the caller's
// order and the per-block energy partials (grid-stride over sorted atoms).
template <typename T, typename OUT>
__global__ void __launch_bounds__(256) k_interp_assemble(int64_t n, const int* __restrict__ perm,
                                                         const R4<T>* __restrict__ gfrac, const T* __restrict__ phis,
                                                         const R4<T>* __restrict__ fs,
                                                         const R4<T>* __restrict__ glong, AssembleArgs A,
                                                         OUT* __restrict__ phi_out, OUT* __restrict__ force_out,
                                                         double* __restrict__ partial) {
  double e = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
    const R4<T> gl = glong[i];
    const T g[3] = {gl.x, gl.y, gl.z};
    e += Assemble<T>::forward(A, gfrac[i].w, phis[i], gl.w, fs[i], g, perm[i], phi_out, force_out);
  }
  const double bsum = block_sum<256>(e);
  if (threadIdx.x == 0) partial[blockIdx.x] = bsum;
}

__device__ __forceinline__ void energy_final_body(const double* __restrict__ partial, int nb,
                                                  double* __restrict__ energy) {
  double v = 0.0;
  for (int i = threadIdx.x; i < nb; i += 1024) v += partial[i];
  double s = block_sum<1024>(v);
  if (threadIdx.x == 0) *energy = 0.5 * s;
}

__global__ void __launch_bounds__(1024) k_energy_final(const double* __restrict__ partial, int nb,
                                                       double* __restrict__ energy) {
  energy_final_body(partial, nb, energy);
}

// adjoint assembly: av0 = M (anterpolated 1/2 gE q) on the grid
template <typename T, int ORDER, typename OUT>
__device__ __forceinline__ void interp_bwd_body(
    const R4<T>* __restrict__ gfrac, const int4* __restrict__ gbase, const int* __restrict__ perm,
    const int* __restrict__ cell_start, const AnterpArgs& AA, const T* __restrict__ av0, const GridDims& G,
    const AssembleArgs& A, const T* __restrict__ phis, const R4<T>* __restrict__ fs,
    const R4<T>* __restrict__ glong, const double* __restrict__ gE, OUT* __restrict__ grad_pos,
    OUT* __restrict__ grad_q, int bx, int by, int bz) {
  constexpr int S = Basis<T, ORDER>::S;
  extern __shared__ unsigned char smem_raw[];
  T* patch = reinterpret_cast<T*>(smem_raw);
  __shared__ int cstart[64], ccount[64], list[kAnterpMaxAtoms + 32], nk_s, tot_s;  // + one round of slots
  const int c0[3] = {bx * AA.B, by * AA.B, bz * AA.B};
  const int lo0 = (int)floor(c0[0] * AA.cw_h[0]) - S - 1;
  const int lo1 = (int)floor(c0[1] * AA.cw_h[1]) - S - 1;
  const int lo2 = (int)floor(c0[2] * AA.cw_h[2]) - S - 1;
  const int total = stage_interp_block<T>(AA, cell_start, gbase, av0, G, patch, lo0, lo1, lo2, cstart, ccount,
                                          list, &nk_s, &tot_s, bx, by, bz);
  const T ih[3] = {T(A.inv_h[0]), T(A.inv_h[1]), T(A.inv_h[2])};
  const T gg = (T)*gE;
  const int nk = nk_s, nlist = total >= 0 ? total : 0;
  int walk_c = 0, walk_m = threadIdx.x;
  for (int kk = threadIdx.x;; kk += blockDim.x) {
    int i;
    if (total >= 0) {
      if (kk >= nlist) break;
      i = list[kk];
      if (i < 0) continue;  // unfilled slot of the bank-ordered list
    } else {
      while (walk_c < nk && walk_m >= ccount[walk_c]) walk_m -= ccount[walk_c++];
      if (walk_c >= nk) break;
      i = cstart[walk_c] + walk_m;
      walk_m += blockDim.x;
    }
    const R4<T> f = gfrac[i];
    T v, gv[3];
    interp_patch_atom<T, ORDER>(f, gbase[i], patch, AA.pd, lo0, lo1, lo2, av0, G, ih, v, gv);
    Assemble<T>::backward(A, gg, f.w, phis[i], fs[i], glong[i], v, gv, perm[i], grad_pos, grad_q);
  }
}

template <typename T, int ORDER, typename OUT>
__device__ __forceinline__ void interp_bwd_call(const InterpKArgs<T, OUT>& K, int bx, int by, int bz) {
  interp_bwd_body<T, ORDER, OUT>(K.gfrac, K.gbase, K.perm, K.cell_start, K.AA, K.u0, K.G, K.A, K.phis, K.fs, K.glong,
                                 K.gE, K.grad_pos, K.grad_q, bx, by, bz);
}

template <typename T, int ORDER, typename OUT>
__global__ void __launch_bounds__(256) k_interp_bwd(
    const R4<T>* __restrict__ gfrac, const int4* __restrict__ gbase, const int* __restrict__ perm,
    const int* __restrict__ cell_start, AnterpArgs AA, const T* __restrict__ av0, GridDims G, AssembleArgs A,
    const T* __restrict__ phis, const R4<T>* __restrict__ fs, const R4<T>* __restrict__ glong,
    const double* __restrict__ gE, OUT* __restrict__ grad_pos, OUT* __restrict__ grad_q) {
  interp_bwd_body<T, ORDER, OUT>(gfrac, gbase, perm, cell_start, AA, av0, G, A, phis, fs, glong, gE, grad_pos, grad_q,
                                 blockIdx.x, blockIdx.y, blockIdx.z);
}

template <typename T>
__global__ void k_to_double(const T* __restrict__ src, double* __restrict__ dst, int64_t count) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) dst[i] = (double)src[i];
}

GridDims dims_of(const Plan& P, int k) {
  GridDims G;
  for (int d = 0; d < 3; ++d) {
    G.n[d] = P.n[k][d];
    G.lo[d] = P.lo[k][d];
  }
  G.periodic = P.P.periodic;
  return G;
}

AssembleArgs assemble_args(const Plan& P) {
  AssembleArgs A;
  A.self_c = P.gamma0 / P.P.cutoff;
  A.kc = P.P.coulomb_k;
  for (int d = 0; d < 3; ++d) A.inv_h[d] = 1.0 / P.h[d];
  A.self_cf = (float)A.self_c;
  A.kcf = (float)A.kc;
  return A;
}

unsigned blocks_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

// batch: the patch of the batched launches (replicas fill the GPU together,
// so they keep the larger patch that a small system alone gives up)
AnterpArgs patch_args(const Plan& P, bool batch = false) {
  AnterpArgs A;
  for (int d = 0; d < 3; ++d) {
    A.nc[d] = P.nc[d];
    A.cw_h[d] = P.cw[d] / P.h[d];
  }
  A.B = batch ? P.ablk_batch : P.ablk;
  A.pd = batch ? P.apd_batch : P.apd;
  return A;
}

template <typename T, typename ACC, int ORDER>
void anterp_t(Plan& P, void* grid0, const double* dscale, double factor, cudaStream_t st) {
  AnterpArgs A;
  for (int d = 0; d < 3; ++d) {
    A.nc[d] = P.nc[d];
    A.cw_h[d] = P.cw[d] / P.h[d];
  }
  A.B = P.ablk;
  A.pd = P.apd;
  dim3 grid(blocks_for(P.nc[0], A.B), blocks_for(P.nc[1], A.B), blocks_for(P.nc[2], A.B));
  size_t sm = sizeof(ACC) * (size_t)A.pd * A.pd * A.pd;
  k_anterp_patch<T, ACC, ORDER><<<grid, 256, sm, st>>>((const R4<T>*)P.d.gfrac, P.d.gbase, P.d.cell_start, A,
                                                     dims_of(P, 0), (double*)grid0, dscale, factor);
}

// Mixed precision: patch sums into the fixed-point grid (in the restriction
// temporary tmp[0], free until the first restriction pass), then one
// conversion to the FP64 level-0 grid that applies the scale.
template <int ORDER>
void anterp_fx(Plan& P, int64_t n, void* grid0, const double* dscale, double factor, cudaStream_t st) {
  const int64_t np = grid_points(P, 0);
  auto* gfx = (unsigned long long*)P.d.tmp[0];
  cudaMemsetAsync(gfx, 0, sizeof(unsigned long long) * (size_t)np, st);
  P.launches += 2;
  if (n > 0) {
    AnterpArgs A = patch_args(P);
    dim3 grid(blocks_for(P.nc[0], A.B), blocks_for(P.nc[1], A.B), blocks_for(P.nc[2], A.B));
    size_t sm = 2 * sizeof(int) * (size_t)A.pd * A.pd * A.pd;  // coarse and residual sums
    k_anterp_fx<ORDER><<<grid, 256, sm, st>>>((const R4<float>*)P.d.gfrac, P.d.gbase, P.d.cell_start, A,
                                              dims_of(P, 0), gfx);
    P.launches += 1;
  }
  k_fx_to_f64<<<blocks_for(np, 256), 256, 0, st>>>(gfx, (double*)grid0, np, dscale, factor);
}

cudaError_t launch_anterpolate(Plan& P, int64_t n, void* grid0, const double* dscale, double factor,
                               cudaStream_t st) {
  if (!P.fp64) {
    if (P.P.order == 3) anterp_fx<3>(P, n, grid0, dscale, factor, st);
    else anterp_fx<5>(P, n, grid0, dscale, factor, st);
    return cudaGetLastError();
  }
  size_t bytes = sizeof(double) * (size_t)grid_points(P, 0);
  cudaMemsetAsync(grid0, 0, bytes, st);
  P.launches += 1 + (n > 0 ? 1 : 0);
  if (n <= 0) return cudaGetLastError();
  if (P.P.order == 3) anterp_t<double, double, 3>(P, grid0, dscale, factor, st);
  else anterp_t<double, double, 5>(P, grid0, dscale, factor, st);
  return cudaGetLastError();
}

// dst = factor * dscale[0] * src over the level-0 grid (FP64)
__global__ void k_scale_grid(const double* __restrict__ src, double* __restrict__ dst, int64_t count,
                             const double* __restrict__ dscale, double factor) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  dst[i] = src[i] * (factor * *dscale);
}

cudaError_t launch_scale_grid(Plan& P, const void* src, void* dst, const double* dscale, double factor,
                              cudaStream_t st) {
  P.launches += 1;
  const int64_t np = grid_points(P, 0);
  k_scale_grid<<<blocks_for(np, 256), 256, 0, st>>>((const double*)src, (double*)dst, np, dscale, factor);
  return cudaGetLastError();
}

// Whether a level's restriction or prolongation runs as one gathering pass:
// on plans whose finest grid has at most 64^3 points, whose evaluations are
// bound by their chains of small launches (measured 4-7 % faster on 23,558 and
// 3,000 atoms; on the 1.07 M-atom box, where the grid passes run beside the
// pair sums, the three-pass form was 1 % faster), and where the gathered taps
// (points times at most (ORDER + 2)^3) stay few (this GPU's FP64 rate is 1/64
// of its FP32 rate).
static bool direct_pass(const Plan& P, int64_t points, bool fp64_values) {
  if (grid_points(P, 0) > ((int64_t)1 << 18)) return false;
  const int64_t nt = P.P.order + 2;
  const int64_t taps = points * nt * nt * nt;
  return taps <= (fp64_values ? ((int64_t)1 << 17) : ((int64_t)1 << 26));
}

static Grid3Args grid3_args(const Plan& P, int kin, int kout) {
  Grid3Args A;
  for (int d = 0; d < 3; ++d) {
    A.nin[d] = P.n[kin][d];
    A.nout[d] = P.n[kout][d];
    A.lo_in[d] = P.lo[kin][d];
    A.lo_out[d] = P.lo[kout][d];
  }
  A.periodic = P.P.periodic;
  return A;
}

cudaError_t launch_restrict(Plan& P, int k, const void* fine, void* coarse, cudaStream_t st) {
  const int* nf = P.n[k];
  const int* nc = P.n[k + 1];
  const int64_t ncp = (int64_t)nc[0] * nc[1] * nc[2];
  if (direct_pass(P, ncp, true)) {
    P.launches += 1;
    const Grid3Args A = grid3_args(P, k, k + 1);
    if (P.P.order == 3) k_restrict3<double, 3><<<blocks_for(ncp, 128), 128, 0, st>>>((const double*)fine, (double*)coarse, A);
    else k_restrict3<double, 5><<<blocks_for(ncp, 128), 128, 0, st>>>((const double*)fine, (double*)coarse, A);
    return cudaGetLastError();
  }
  P.launches += 3;
  double* t1 = (double*)P.d.tmp[0];
  double* t2 = (double*)P.d.tmp[1];
  const double* src[3] = {(const double*)fine, t1, t2};
  double* dst[3] = {t1, t2, (double*)coarse};
  int cur[3] = {nf[0], nf[1], nf[2]};
  for (int ax = 0; ax < 3; ++ax) {
    AxisArgs A;
    for (int d = 0; d < 3; ++d) A.nin[d] = cur[d];
    cur[ax] = nc[ax];
    for (int d = 0; d < 3; ++d) A.nout[d] = cur[d];
    A.axis = ax;
    A.lo_in = P.lo[k][ax];
    A.lo_out = P.lo[k + 1][ax];
    A.periodic = P.P.periodic;
    unsigned nb = blocks_for((int64_t)cur[0] * cur[1] * cur[2], 256);
    if (P.P.order == 3) k_restrict_axis<double, 3><<<nb, 256, 0, st>>>(src[ax], dst[ax], A);
    else k_restrict_axis<double, 5><<<nb, 256, 0, st>>>(src[ax], dst[ax], A);
  }
  return cudaGetLastError();
}

template <typename T>
void prolong_t(Plan& P, int k, const T* coarse, T* fine, cudaStream_t st) {
  const int* nf = P.n[k];
  const int* nc = P.n[k + 1];
  T* s1 = (T*)P.d.tmp[0];
  T* s2 = (T*)P.d.tmp[1];
  const T* src[3] = {coarse, s1, s2};
  T* dst[3] = {s1, s2, fine};
  int cur[3] = {nc[0], nc[1], nc[2]};
  for (int i = 0; i < 3; ++i) {
    int ax = 2 - i;  // z, then y, then x
    AxisArgs A;
    for (int d = 0; d < 3; ++d) A.nin[d] = cur[d];
    cur[ax] = nf[ax];
    for (int d = 0; d < 3; ++d) A.nout[d] = cur[d];
    A.axis = ax;
    A.lo_in = P.lo[k + 1][ax];
    A.lo_out = P.lo[k][ax];
    A.periodic = P.P.periodic;
    unsigned nb = blocks_for((int64_t)cur[0] * cur[1] * cur[2], 256);
    int acc = (i == 2) ? 1 : 0;  // the last pass adds onto u^{k,cutoff}
    if (P.P.order == 3) k_prolong_axis<T, 3><<<nb, 256, 0, st>>>(src[i], dst[i], A, acc);
    else k_prolong_axis<T, 5><<<nb, 256, 0, st>>>(src[i], dst[i], A, acc);
  }
}

cudaError_t launch_prolong(Plan& P, int k, const void* coarse, void* fine, cudaStream_t st) {
  const int64_t nfp = grid_points(P, k);
  if (direct_pass(P, nfp, P.fp64)) {
    P.launches += 1;
    const Grid3Args A = grid3_args(P, k + 1, k);
    const unsigned nb = blocks_for(nfp, 256);
    if (P.fp64) {
      if (P.P.order == 3) k_prolong3<double, 3><<<nb, 256, 0, st>>>((const double*)coarse, (double*)fine, A);
      else k_prolong3<double, 5><<<nb, 256, 0, st>>>((const double*)coarse, (double*)fine, A);
    } else {
      if (P.P.order == 3) k_prolong3<float, 3><<<nb, 256, 0, st>>>((const float*)coarse, (float*)fine, A);
      else k_prolong3<float, 5><<<nb, 256, 0, st>>>((const float*)coarse, (float*)fine, A);
    }
    return cudaGetLastError();
  }
  P.launches += 3;
  if (P.fp64) prolong_t<double>(P, k, (const double*)coarse, (double*)fine, st);
  else prolong_t<float>(P, k, (const float*)coarse, (float*)fine, st);
  return cudaGetLastError();
}

__device__ __forceinline__ void f64_to_f32_body(const double* __restrict__ src, float* __restrict__ dst,
                                                int64_t count, int64_t i) {
  if (i < count) dst[i] = (float)src[i];
}

__global__ void k_f64_to_f32(const double* __restrict__ src, float* __restrict__ dst, int64_t count) {
  f64_to_f32_body(src, dst, count, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

// Warp tile of the FP32 lattice kernel for an n0 x n1 plane: txn lanes of
// kLatticeLP x outputs by tyn lanes of two rows (txn * tyn <= 32).  Every
// tile costs one warp's pass over the stencil whatever its idle lanes, plus
// the staging of its input window; the cost counts both (a warp's stencil
// pass at a plane is ~14,000 instructions, staging ~1/3 instruction per
// window element), so ragged small grids get tiles that fit them.
static size_t lattice_smem(int txn, int tyn, const int E[3]);

static void lattice_tile(int n0, int n1, const int E[3], int& txn, int& tyn) {
  double best = -1.0;
  txn = 4;
  tyn = 8;
  for (int a = 1; a <= 32; ++a)
    for (int b = 1; a * b <= 32; ++b) {
      if (lattice_smem(a, b, E) > kLatticeSmemMax) continue;
      const double tiles = (double)((n0 + kLatticeLP * a - 1) / (kLatticeLP * a)) * ((n1 + 2 * b - 1) / (2 * b));
      const double window = (double)(kLatticeLP * a + 2 * E[0] + kSeg) * (2 * b + 2 * E[1]);
      const double cost = tiles * (14000.0 + window / 3.0);
      if (best < 0 || cost < best) {
        best = cost;
        txn = a;
        tyn = b;
      }
    }
}

static size_t lattice_smem(int txn, int tyn, const int E[3]) {
  const int SXw = kLatticeLP * txn + 2 * E[0] + kSeg, SX = SXw | 1, SY = 2 * tyn + 2 * E[1];
  return sizeof(float) * 2 * SX * SY + sizeof(int) * (SXw + SY);
}

// Lattice cutoff of level k from the FP64 charges qk.  Mixed precision first
// converts the level's charges to FP32 once (on GB300 the conversion runs on
// the slow FP64 pipe, so it must not sit in the per-tap loop).
template <typename T>
void lattice_t(Plan& P, int k, const double* qk64, T* uk, cudaStream_t st) {
  GridDims G = dims_of(P, k);
  const bool f32 = !std::is_same<T, double>::value;
  const T* qk = (const T*)qk64;
  if (f32) {
    float* qf = (float*)P.d.tmp[0];  // free between the restriction and the prolongation passes
    k_f64_to_f32<<<blocks_for(grid_points(P, k), 256), 256, 0, st>>>(qk64, qf, grid_points(P, k));
    P.launches += 1;
    qk = (const T*)qf;
  }
  LatticeArgs L;
  L.Ex = P.E[0];
  L.Ey = P.E[1];
  L.Ez = P.E[2];
  // one system: the 32 x 16 tile, fixed at compile time, on every level (the
  // runtime-tile kernel is slower per tap than the saving on ragged coarse
  // levels), unless the plan's tuning names another tile for level 0
  lattice_tile_of(P, k, L.txn, L.tyn);
  const int TW = f32 ? kLatticeLP * L.txn : LBX, LBY = f32 ? 2 * L.tyn : 8;
  const int LBZb = f32 ? kLatticeZ : LBZ;  // output planes (warps) per block
  L.nbz = (int)blocks_for(G.n[2], LBZb);
  L.nsplit = lattice_nsplit(P, k);
  T* up = (T*)P.d.lparts;
  dim3 grid(blocks_for(G.n[0], TW), blocks_for(G.n[1], LBY), L.nbz * L.nsplit);
  int SX = (LBX + 2 * P.E[0] + kSeg) | 1, SY = LBY + 2 * P.E[1];
  // FP32 double-buffers its planes and keeps the window offsets (SXw + SY ints)
  size_t sm = f32 ? lattice_smem(L.txn, L.tyn, P.E) : sizeof(T) * SX * SY;
  T scale = (T)std::ldexp(1.0, -k);
  if (f32) {
    if (L.txn == 4 && L.tyn == 8)
      k_lattice_f2<kLatticeLP, 4, 8><<<grid, 32 * kLatticeZ, sm, st>>>((const float*)qk, (float*)uk, (float*)up, G,
                                                                      (const Segment2*)P.d.seg2, P.d.seg_start, L,
                                                                      (float)scale);
    else
      k_lattice_f2<kLatticeLP, 0, 0><<<grid, 32 * kLatticeZ, sm, st>>>((const float*)qk, (float*)uk, (float*)up, G,
                                                                      (const Segment2*)P.d.seg2, P.d.seg_start, L,
                                                                      (float)scale);
  } else {
    k_lattice<T, false><<<grid, 128, sm, st>>>(qk, uk, up, G, (const Segment<T>*)P.d.seg, P.d.seg_start, L, scale);
  }
  if (L.nsplit > 1) {
    const int64_t np = grid_points(P, k);
    k_lattice_reduce<T><<<blocks_for(np, 256), 256, 0, st>>>(up, uk, np, L.nsplit);
    P.launches += 1;
  }
}

// Warp tile of the FP32 lattice kernel at level k of a single system: the
// plan's tuned tile on level 0, else 4 x 8 (32 x 16 outputs).
void lattice_tile_of(const Plan& P, int k, int& txn, int& tyn) {
  if (k == 0 && P.lattice_txn > 0) {
    txn = P.lattice_txn;
    tyn = P.lattice_tyn;
  } else {
    txn = 4;
    tyn = 8;
  }
}

// Blocks that share one brick's input planes at level k (several on small
// levels, so that the launch still fills the GPU: lattice_waves blocks per SM).
int lattice_nsplit(const Plan& P, int k) {
  GridDims G = dims_of(P, k);
  int txn, tyn;
  lattice_tile_of(P, k, txn, tyn);
  const int TW = P.fp64 ? LBX : kLatticeLP * txn, LBY = P.fp64 ? 8 : 2 * tyn;
  const int LBZb = P.fp64 ? LBZ : kLatticeZ;
  const int64_t bricks = (int64_t)blocks_for(G.n[0], TW) * blocks_for(G.n[1], LBY) * blocks_for(G.n[2], LBZb);
  const int64_t target = (int64_t)P.lattice_waves * 152 * 4 / LBZb;
  return (int)std::min<int64_t>(LBZb + 2 * P.E[2], std::max<int64_t>(1, (target + bricks - 1) / bricks));
}

// Elements of the plan's split-partial buffer: the largest nsplit x points of
// any level whose lattice cutoff is split.
int64_t lattice_parts_elems(const Plan& P) {
  int64_t m = 0;
  for (int k = 0; k + 1 < P.levels; ++k) {
    const int ns = lattice_nsplit(P, k);
    if (ns > 1) m = std::max<int64_t>(m, (int64_t)ns * grid_points(P, k));
  }
  return m;
}

bool lattice_fits(const Plan& P) {
  if (P.fp64) {
    const int SX = (LBX + 2 * P.E[0] + kSeg) | 1, SY = 8 + 2 * P.E[1];
    return sizeof(double) * SX * SY <= 48 * 1024;
  }
  return lattice_smem(4, 8, P.E) <= kLatticeSmemMax;
}

bool lattice_tile_fits(const Plan& P, int txn, int tyn) {
  return P.fp64 || lattice_smem(txn, tyn, P.E) <= kLatticeSmemMax;
}

cudaError_t launch_lattice(Plan& P, int k, const void* qk, void* uk, cudaStream_t st) {
  P.launches += 1;
  if (P.fp64) lattice_t<double>(P, k, (const double*)qk, (double*)uk, st);
  else lattice_t<float>(P, k, (const double*)qk, (float*)uk, st);
  return cudaGetLastError();
}

cudaError_t launch_top(Plan& P, const void* qt, void* ut, cudaStream_t st) {
  P.launches += 1;
  int top = P.levels - 1;
  GridDims G = dims_of(P, top);
  unsigned nb = blocks_for(grid_points(P, top), kTopWarps);
  if (P.fp64)
    k_top<double><<<nb, 32 * kTopWarps, 0, st>>>((const double*)qt, (double*)ut, P.d.topu, G, P.d.topK,
                                     P.top_table_dims[0], P.top_table_dims[1], P.top_table_dims[2]);
  else
    k_top<float><<<nb, 32 * kTopWarps, 0, st>>>((const double*)qt, (float*)ut, P.d.topu, G, P.d.topK,
                                    P.top_table_dims[0], P.top_table_dims[1], P.top_table_dims[2]);
  return cudaGetLastError();
}


#define INTERP_FWD_ARGS(K)                                                                                   \
  K.gfrac, K.gbase, K.perm, K.cell_start, K.AA, K.u0, K.G, K.A, K.phis, K.fs, K.glong, K.phi_out, K.force_out, \
      K.partial
#define INTERP_BWD_ARGS(K) \
  K.gfrac, K.gbase, K.perm, K.cell_start, K.AA, K.u0, K.G, K.A, K.phis, K.fs, K.glong, K.gE, K.grad_pos, K.grad_q

// Interpolation arguments of plan P (forward: grid u^0; backward: the adjoint grid).
template <typename T, typename OUT>
InterpKArgs<T, OUT> interp_kargs(Plan& P, bool backward, OUT* phi, OUT* force, const double* gE, OUT* grad_pos,
                                 OUT* grad_q, double* partial, bool batch = false) {
  InterpKArgs<T, OUT> K;
  K.gfrac = (const R4<T>*)P.d.gfrac;
  K.gbase = P.d.gbase;
  K.perm = P.d.perm;
  K.cell_start = P.d.cell_start;
  K.AA = patch_args(P, batch);
  K.u0 = (const T*)(backward ? P.d.au[0] : P.d.gu[0]);
  K.G = dims_of(P, 0);
  K.A = assemble_args(P);
  K.phis = (const T*)P.d.phis;
  K.fs = (R4<T>*)P.d.fs;
  K.glong = (R4<T>*)P.d.glong;
  K.phi_out = phi;
  K.force_out = force;
  K.partial = partial;
  K.gE = gE;
  K.grad_pos = grad_pos;
  K.grad_q = grad_q;
  K.nbx = (int)blocks_for(P.nc[0], K.AA.B);
  K.nby = (int)blocks_for(P.nc[1], K.AA.B);
  return K;
}

cudaError_t launch_interp_gather(Plan& P, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  AnterpArgs AA = patch_args(P);
  dim3 grid(blocks_for(P.nc[0], AA.B), blocks_for(P.nc[1], AA.B), blocks_for(P.nc[2], AA.B));
  size_t sm = (P.fp64 ? 8 : 4) * (size_t)AA.pd * AA.pd * AA.pd;
  const GridDims G = dims_of(P, 0);
  const AssembleArgs A = assemble_args(P);
#define MSM_GATHER(T, O)                                                                                          \
  k_interp_gather<T, O><<<grid, 256, sm, st>>>((const R4<T>*)P.d.gfrac, P.d.gbase, P.d.cell_start, AA,            \
                                               (const T*)P.d.gu[0], G, A, (R4<T>*)P.d.glong)
  if (P.fp64) {
    if (P.P.order == 3) MSM_GATHER(double, 3);
    else MSM_GATHER(double, 5);
  } else {
    if (P.P.order == 3) MSM_GATHER(float, 3);
    else MSM_GATHER(float, 5);
  }
#undef MSM_GATHER
  P.launches += 1;
  return cudaGetLastError();
}

template <typename OUT>
cudaError_t launch_interp_assemble(Plan& P, int64_t n, double* energy, OUT* phi, OUT* force, cudaStream_t st) {
  const int nb = (int)std::max<int64_t>(0, std::min<int64_t>(P.nblk_partial, (n + 255) / 256));
  const AssembleArgs A = assemble_args(P);
  if (nb > 0) {
    if (P.fp64)
      k_interp_assemble<double, OUT><<<nb, 256, 0, st>>>(n, P.d.perm, (const R4<double>*)P.d.gfrac,
                                                        (const double*)P.d.phis, (const R4<double>*)P.d.fs,
                                                        (const R4<double>*)P.d.glong, A, phi, force, P.d.partial);
    else
      k_interp_assemble<float, OUT><<<nb, 256, 0, st>>>(n, P.d.perm, (const R4<float>*)P.d.gfrac,
                                                       (const float*)P.d.phis, (const R4<float>*)P.d.fs,
                                                       (const R4<float>*)P.d.glong, A, phi, force, P.d.partial);
  }
  k_energy_final<<<1, 1024, 0, st>>>(P.d.partial, nb, energy);
  P.launches += 1 + (nb > 0 ? 1 : 0);
  return cudaGetLastError();
}

template cudaError_t launch_interp_assemble<double>(Plan&, int64_t, double*, double*, double*, cudaStream_t);
template cudaError_t launch_interp_assemble<float>(Plan&, int64_t, double*, float*, float*, cudaStream_t);

template <typename OUT>
cudaError_t launch_interp_backward(Plan& P, int64_t n, const double* gE, OUT* grad_pos, OUT* grad_q,
                                   cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  AnterpArgs AA = patch_args(P);
  dim3 grid(blocks_for(P.nc[0], AA.B), blocks_for(P.nc[1], AA.B), blocks_for(P.nc[2], AA.B));
  size_t sm = (P.fp64 ? 8 : 4) * (size_t)AA.pd * AA.pd * AA.pd;
  P.launches += 1;
  if (P.fp64) {
    auto K = interp_kargs<double, OUT>(P, true, nullptr, nullptr, gE, grad_pos, grad_q, nullptr);
    if (P.P.order == 3) k_interp_bwd<double, 3, OUT><<<grid, 256, sm, st>>>(INTERP_BWD_ARGS(K));
    else k_interp_bwd<double, 5, OUT><<<grid, 256, sm, st>>>(INTERP_BWD_ARGS(K));
  } else {
    auto K = interp_kargs<float, OUT>(P, true, nullptr, nullptr, gE, grad_pos, grad_q, nullptr);
    if (P.P.order == 3) k_interp_bwd<float, 3, OUT><<<grid, 256, sm, st>>>(INTERP_BWD_ARGS(K));
    else k_interp_bwd<float, 5, OUT><<<grid, 256, sm, st>>>(INTERP_BWD_ARGS(K));
  }
  return cudaGetLastError();
}


template cudaError_t launch_interp_backward<double>(Plan&, int64_t, const double*, double*, double*, cudaStream_t);
template cudaError_t launch_interp_backward<float>(Plan&, int64_t, const double*, float*, float*, cudaStream_t);

cudaError_t launch_grid_to_double(Plan& P, const void* src, double* dst, int64_t count, bool is_double,
                                  cudaStream_t st) {
  unsigned nb = blocks_for(count, 256);
  if (count <= 0) return cudaSuccess;
  if (P.fp64 || is_double) k_to_double<double><<<nb, 256, 0, st>>>((const double*)src, dst, count);
  else k_to_double<float><<<nb, 256, 0, st>>>((const float*)src, dst, count);
  return cudaGetLastError();
}


// ---- the cutoff method: assembly of phi, F and E from the pair sums ----
// phi_i = k_c u_i, F_i = k_c (pair forces), E = 1/2 k_c sum_i q_i u_i; per-block
// FP64 partials (grid-stride over the sorted atoms) and k_energy_final.
template <typename T, typename OUT>
__global__ void __launch_bounds__(256) k_cutoff_assemble(int64_t n, const int* __restrict__ perm,
                                                         const R4<T>* __restrict__ atoms, const T* __restrict__ phis,
                                                         const R4<T>* __restrict__ fs, T kc, T selfc, OUT* __restrict__ phi_out,
                                                         OUT* __restrict__ force_out, double* __restrict__ partial) {
  double e = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
    const T p = phis[i] - selfc * atoms[i].w;  // selfc: the method's self term (0 for the cutoff method)
    const R4<T> f = fs[i];
    const int o = perm[i];
    if (phi_out) phi_out[o] = (OUT)(kc * p);
    if (force_out) {
      force_out[3 * (size_t)o + 0] = (OUT)(kc * f.x);
      force_out[3 * (size_t)o + 1] = (OUT)(kc * f.y);
      force_out[3 * (size_t)o + 2] = (OUT)(kc * f.z);
    }
    e += (double)(atoms[i].w * (kc * p));
  }
  const double bsum = block_sum<256>(e);
  if (threadIdx.x == 0) partial[blockIdx.x] = bsum;
}

template <typename OUT>
cudaError_t launch_cutoff_assemble(Plan& P, int64_t n, double* energy, OUT* phi, OUT* force, cudaStream_t st,
                                   double self_c) {
  const int nb = (int)std::max<int64_t>(0, std::min<int64_t>(P.nblk_partial, (n + 255) / 256));
  if (nb > 0) {
    if (P.fp64)
      k_cutoff_assemble<double, OUT><<<nb, 256, 0, st>>>(n, P.d.perm, (const R4<double>*)P.d.atoms,
                                                        (const double*)P.d.phis, (const R4<double>*)P.d.fs,
                                                        P.P.coulomb_k, self_c, phi, force, P.d.partial);
    else
      k_cutoff_assemble<float, OUT><<<nb, 256, 0, st>>>(n, P.d.perm, (const R4<float>*)P.d.atoms,
                                                       (const float*)P.d.phis, (const R4<float>*)P.d.fs,
                                                       (float)P.P.coulomb_k, (float)self_c, phi, force,
                                                       P.d.partial);
  }
  k_energy_final<<<1, 1024, 0, st>>>(P.d.partial, nb, energy);
  P.launches += 1 + (nb > 0 ? 1 : 0);
  return cudaGetLastError();
}

template cudaError_t launch_cutoff_assemble<double>(Plan&, int64_t, double*, double*, double*, cudaStream_t, double);
template cudaError_t launch_cutoff_assemble<float>(Plan&, int64_t, double*, float*, float*, cudaStream_t, double);

// ---- batches: every grid pass as one launch over all replicas ----
namespace {

constexpr int kEw = 256;  // threads per block of the batched elementwise kernels

struct ZeroKArgs {
  unsigned* p;
  int64_t words;
};
struct FxKArgs {
  const unsigned long long* gfx;
  double* q0;
  int64_t count;
  const double* dscale;
  double factor;
};
template <typename T>
struct AxisKArgs {
  const T* in;
  T* out;
  AxisArgs A;
  int acc;
};
struct ConvKArgs {
  const double* src;
  float* dst;
  int64_t count;
};
struct AntKArgs {
  const R4<float>* gfrac;
  const int4* gbase;
  const int* cell_start;
  AnterpArgs A;
  GridDims G;
  unsigned long long* gfx;
  int nbx, nby;
};
struct LatKArgs {
  const float* q;
  float* u;
  float* up;  // split partials (nsplit > 1)
  GridDims G;
  const Segment2* seg;
  const int* seg_start;
  LatticeArgs L;
  float scale;
  int nbx, nby;
};
struct TopKArgs {
  const double* qt;
  float* ut;
  double* ut64;
  GridDims G;
  const double* K;
  int tx, ty;
};
struct EnergyKArgs {
  const double* partial;
  int nb;
  double* energy;
};
struct ReduceKArgs {
  const float* up;
  float* u;
  int64_t np;
  int nsplit;
};

__device__ __forceinline__ int64_t ew_index(const int* __restrict__ first, int r) {
  return (int64_t)(blockIdx.x - first[r]) * kEw + threadIdx.x;
}

__global__ void __launch_bounds__(kEw) kb_zero(const ZeroKArgs* __restrict__ tab, const int* __restrict__ first,
                                               int nrep) {
  const int r = batch_rep(first, nrep, blockIdx.x);
  const int64_t i = ew_index(first, r);
  if (i < tab[r].words) tab[r].p[i] = 0u;
}

__global__ void __launch_bounds__(kEw) kb_fx_to_f64(const FxKArgs* __restrict__ tab, const int* __restrict__ first,
                                                    int nrep) {
  const int r = batch_rep(first, nrep, blockIdx.x);
  const FxKArgs& a = tab[r];
  fx_to_f64_body(a.gfx, a.q0, a.count, a.dscale, a.factor, ew_index(first, r));
}

template <int ORDER>
__global__ void __launch_bounds__(kEw) kb_restrict_axis(const AxisKArgs<double>* __restrict__ tab,
                                                        const int* __restrict__ first, int nrep) {
  const int r = batch_rep(first, nrep, blockIdx.x);
  const AxisKArgs<double>& a = tab[r];
  restrict_axis_body<double, ORDER>(a.in, a.out, a.A, ew_index(first, r));
}

template <int ORDER>
__global__ void __launch_bounds__(kEw) kb_prolong_axis(const AxisKArgs<float>* __restrict__ tab,
                                                       const int* __restrict__ first, int nrep) {
  const int r = batch_rep(first, nrep, blockIdx.x);
  const AxisKArgs<float>& a = tab[r];
  prolong_axis_body<float, ORDER>(a.in, a.out, a.A, a.acc, ew_index(first, r));
}

__global__ void __launch_bounds__(kEw) kb_lattice_reduce(const ReduceKArgs* __restrict__ tab,
                                                         const int* __restrict__ first, int nrep) {
  const int r = batch_rep(first, nrep, blockIdx.x);
  const ReduceKArgs& a = tab[r];
  lattice_reduce_body<float>(a.up, a.u, a.np, a.nsplit, ew_index(first, r));
}

__global__ void __launch_bounds__(kEw) kb_f64_to_f32(const ConvKArgs* __restrict__ tab, const int* __restrict__ first,
                                                     int nrep) {
  const int r = batch_rep(first, nrep, blockIdx.x);
  f64_to_f32_body(tab[r].src, tab[r].dst, tab[r].count, ew_index(first, r));
}

template <int ORDER>
__global__ void __launch_bounds__(256, 2) kb_anterp_fx(const AntKArgs* __restrict__ tab, const int* __restrict__ first,
                                                    int nrep) {
  const int r = batch_rep(first, nrep, blockIdx.x);
  const AntKArgs& a = tab[r];
  const int b = blockIdx.x - first[r];
  anterp_fx_body<ORDER>(a.gfrac, a.gbase, a.cell_start, a.A, a.G, a.gfx, b % a.nbx, (b / a.nbx) % a.nby,
                        b / (a.nbx * a.nby));
}

__global__ void __launch_bounds__(32 * kLatticeZ, 6) kb_lattice_f2(const LatKArgs* __restrict__ tab,
                                                                   const int* __restrict__ first, int nrep) {
  const int r = batch_rep(first, nrep, blockIdx.x);
  const LatKArgs& a = tab[r];
  const int b = blockIdx.x - first[r];
  lattice_f2_body<kLatticeLP, 0, 0>(a.q, a.u, a.up, a.G, a.seg, a.seg_start, a.L, a.scale, b % a.nbx,
                                    (b / a.nbx) % a.nby, b / (a.nbx * a.nby));
}

__global__ void __launch_bounds__(32 * kTopWarps) kb_top(const TopKArgs* __restrict__ tab,
                                                         const int* __restrict__ first, int nrep) {
  const int r = batch_rep(first, nrep, blockIdx.x);
  const TopKArgs& a = tab[r];
  top_body<float>(a.qt, a.ut, a.ut64, a.G, a.K, a.tx, a.ty,
                  (int64_t)(blockIdx.x - first[r]) * kTopWarps + (threadIdx.x >> 5));
}

template <int ORDER>
__global__ void __launch_bounds__(256, 2) kb_interp_fwd(const InterpKArgs<float, double>* __restrict__ tab,
                                                     const int* __restrict__ first, int nrep) {
  const int r = batch_rep(first, nrep, blockIdx.x);
  const InterpKArgs<float, double>& K = tab[r];
  const int b = blockIdx.x - first[r];
  interp_fwd_call<float, ORDER, double>(K, b % K.nbx, (b / K.nbx) % K.nby, b / (K.nbx * K.nby), b);
}

template <int ORDER>
__global__ void __launch_bounds__(256, 2) kb_interp_bwd(const InterpKArgs<float, double>* __restrict__ tab,
                                                     const int* __restrict__ first, int nrep) {
  const int r = batch_rep(first, nrep, blockIdx.x);
  const InterpKArgs<float, double>& K = tab[r];
  const int b = blockIdx.x - first[r];
  interp_bwd_call<float, ORDER, double>(K, b % K.nbx, (b / K.nbx) % K.nby, b / (K.nbx * K.nby));
}

__global__ void __launch_bounds__(1024) kb_energy_final(const EnergyKArgs* __restrict__ tab,
                                                        const int* __restrict__ first, int nrep) {
  const int r = batch_rep(first, nrep, blockIdx.x);
  energy_final_body(tab[r].partial, tab[r].nb, tab[r].energy);
}

int ew_blocks(int64_t count) { return (int)((count + kEw - 1) / kEw); }

}  // namespace

// ---- persistent chains (a measured alternative to one launch per pass) ----
// The restriction and the prolongation of a sweep are chains of small
// dependent passes (three axes per level pair).  A persistent form runs a
// whole chain in one cooperative launch: the co-resident blocks take the
// virtual blocks of each pass in turn (the same tables and element bodies as
// the per-pass launches) and meet at a grid barrier between passes.  The
// barrier is a counter and a generation word in device memory; every wait is
// bounded, and a wait that gives up posts kStatusTimeout and ends its block.
struct PassDesc {
  const void* args;   // the pass's table of per-replica arguments
  const int* first;   // its block offsets
  int nrep;
  int total;          // virtual blocks of kEw elements over all replicas
};
constexpr int kGridSpin = 1 << 22;  // polls of the generation word before a barrier gives up

// All blocks of the grid arrive, the last one releases the others.  bar[0]:
// arrivals of the current barrier, bar[1]: generation.
__device__ bool grid_barrier(unsigned* bar, unsigned nblocks, int* status) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) + 1u == nblocks) {
      bar[0] = 0u;  // nobody arrives at the next barrier before the generation moves
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      for (int it = 0; *gen == g; ++it) {
        if (it >= kGridSpin) {
          ok = 0;
          atomicOr(status, kStatusTimeout);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

template <int ORDER>
__global__ void __launch_bounds__(kEw) kb_restrict_chain(const PassDesc* __restrict__ passes, int npass,
                                                         unsigned* bar, int* status) {
  for (int p = 0; p < npass; ++p) {
    const PassDesc d = passes[p];
    const AxisKArgs<double>* tab = reinterpret_cast<const AxisKArgs<double>*>(d.args);
    for (int b = blockIdx.x; b < d.total; b += gridDim.x) {
      const int r = batch_rep(d.first, d.nrep, b);
      restrict_axis_body<double, ORDER>(tab[r].in, tab[r].out, tab[r].A, (int64_t)(b - d.first[r]) * kEw + threadIdx.x);
    }
    if (p + 1 < npass && !grid_barrier(bar, gridDim.x, status)) return;
  }
}

template <int ORDER>
__global__ void __launch_bounds__(kEw) kb_prolong_chain(const PassDesc* __restrict__ passes, int npass,
                                                        unsigned* bar, int* status) {
  for (int p = 0; p < npass; ++p) {
    const PassDesc d = passes[p];
    const AxisKArgs<float>* tab = reinterpret_cast<const AxisKArgs<float>*>(d.args);
    for (int b = blockIdx.x; b < d.total; b += gridDim.x) {
      const int r = batch_rep(d.first, d.nrep, b);
      prolong_axis_body<float, ORDER>(tab[r].in, tab[r].out, tab[r].A, tab[r].acc,
                                      (int64_t)(b - d.first[r]) * kEw + threadIdx.x);
    }
    if (p + 1 < npass && !grid_barrier(bar, gridDim.x, status)) return;
  }
}

struct GridBatch {
  int order = 3;
  int maxlev = 1;
  bool has_backward = false;
  BatchTable<ZeroKArgs> zero_fx;
  BatchTable<AntKArgs> anterp;
  BatchTable<FxKArgs> fx[2];
  std::vector<BatchTable<AxisKArgs<double>>> restr[2];  // [dir][3 k + axis]
  BatchTable<ConvKArgs> conv[2];
  BatchTable<ReduceKArgs> reduce_u[2];  // split lattice partials -> u, in part order
  float* lparts[2] = {nullptr, nullptr};
  BatchTable<LatKArgs> lattice[2];
  FftBatch* fft[2] = {nullptr, nullptr};  // the FFT form, when every replica's plan took it
  BatchTable<TopKArgs> top[2];
  std::vector<BatchTable<AxisKArgs<float>>> prol[2];  // [dir][3 k + pass]
  BatchTable<InterpKArgs<float, double>> interp[2];
  BatchTable<EnergyKArgs> energy;
  // persistent chains: pass descriptors of the restriction and prolongation
  // of each direction, barrier words, the status word they post to
  bool persistent = false;
  PassDesc* chain_restr[2] = {nullptr, nullptr};
  PassDesc* chain_prol[2] = {nullptr, nullptr};
  int n_restr = 0, n_prol = 0;
  unsigned* bar = nullptr;
  int* status = nullptr;
  int chain_blocks = 0;
  // the adjoint direction's temporaries, one block per replica
  std::vector<void*> scratch1;
};

void grid_batch_free(GridBatch* b) {
  if (!b) return;
  b->zero_fx.release();
  b->anterp.release();
  for (int d = 0; d < 2; ++d) {
    b->fx[d].release();
    for (auto& t : b->restr[d]) t.release();
    b->conv[d].release();
    b->reduce_u[d].release();
    if (b->lparts[d]) cudaFree(b->lparts[d]);
    b->lattice[d].release();
    fft_batch_free(b->fft[d]);
    b->top[d].release();
    for (auto& t : b->prol[d]) t.release();
    b->interp[d].release();
  }
  b->energy.release();
  for (int d = 0; d < 2; ++d) {
    if (b->chain_restr[d]) cudaFree(b->chain_restr[d]);
    if (b->chain_prol[d]) cudaFree(b->chain_prol[d]);
  }
  if (b->bar) cudaFree(b->bar);
  for (void* p : b->scratch1) cudaFree(p);
  delete b;
}

cudaError_t grid_batch_build(const std::vector<BatchRep>& reps, bool backward, GridBatch** out) {
  *out = nullptr;
  GridBatch* B = new (std::nothrow) GridBatch();
  if (!B) return cudaErrorMemoryAllocation;
  const int R = (int)reps.size();
  B->order = reps.empty() ? 3 : reps[0].plan->P.order;
  B->has_backward = backward;
  for (const BatchRep& r : reps) B->maxlev = std::max(B->maxlev, r.plan->levels);
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  {  // anterpolation into the fixed-point grids (tmp[0]); the same kernels for both directions
    std::vector<ZeroKArgs> za;
    std::vector<AntKArgs> aa;
    std::vector<int> zb, ab;
    size_t sm = 0;
    for (const BatchRep& r : reps) {
      Plan& P = *r.plan;
      const int64_t np = grid_points(P, 0);
      za.push_back(ZeroKArgs{(unsigned*)P.d.tmp[0], 2 * np});
      zb.push_back(ew_blocks(2 * np));
      AntKArgs a;
      a.gfrac = (const R4<float>*)P.d.gfrac;
      a.gbase = P.d.gbase;
      a.cell_start = P.d.cell_start;
      a.A = patch_args(P, true);
      a.G = dims_of(P, 0);
      a.gfx = (unsigned long long*)P.d.tmp[0];
      a.nbx = (int)blocks_for(P.nc[0], a.A.B);
      a.nby = (int)blocks_for(P.nc[1], a.A.B);
      aa.push_back(a);
      ab.push_back(r.n > 0 ? a.nbx * a.nby * (int)blocks_for(P.nc[2], a.A.B) : 0);
      sm = std::max(sm, 2 * sizeof(int) * (size_t)a.A.pd * a.A.pd * a.A.pd);
    }
    chk(make_table(B->zero_fx, za, zb));
    chk(make_table(B->anterp, aa, ab, sm));
  }
  // the adjoint direction's own temporaries (restriction and prolongation,
  // the FFT workspace or the stencil's FP32 charges, the top level's FP64
  // values), so that its level chain can run beside the forward's
  struct Scratch {
    void* tmp[2] = {nullptr, nullptr};
    void* fftw = nullptr;
    double* topu = nullptr;
  };
  std::vector<Scratch> S1(reps.size());
  if (backward)
    for (size_t i = 0; i < reps.size() && e == cudaSuccess; ++i) {
      Plan& P = *reps[i].plan;
      size_t lat = 0;
      for (int k = 0; k + 1 < P.levels; ++k) lat += (size_t)grid_points(P, k);
      const size_t tmpb = sizeof(double) * (size_t)P.tmp_elems, fftb = P.lattice_fft ? 16 * lat : 0;
      const size_t topb = sizeof(double) * (size_t)grid_points(P, P.levels - 1);
      char* base = nullptr;
      chk(cudaMalloc((void**)&base, 2 * tmpb + fftb + topb));
      if (e != cudaSuccess) break;
      B->scratch1.push_back(base);
      S1[i].tmp[0] = base;
      S1[i].tmp[1] = base + tmpb;
      S1[i].fftw = base + 2 * tmpb;
      S1[i].topu = reinterpret_cast<double*>(base + 2 * tmpb + fftb);
    }
  for (int dir = 0; dir < (backward ? 2 : 1); ++dir) {
    // this direction's temporaries of replica r
    auto tmp_of = [&](const BatchRep& r, int i) -> void* {
      return dir ? S1[&r - &reps[0]].tmp[i] : r.plan->d.tmp[i];
    };
    std::vector<FxKArgs> fa;
    std::vector<int> fb;
    for (const BatchRep& r : reps) {
      Plan& P = *r.plan;
      const int64_t np = grid_points(P, 0);
      fa.push_back(FxKArgs{(const unsigned long long*)P.d.tmp[0], (double*)(dir ? P.d.aq[0] : P.d.gq[0]), np,
                           dir ? r.grad_energy : nullptr, dir ? 0.5 : 1.0});
      fb.push_back(ew_blocks(np));
    }
    chk(make_table(B->fx[dir], fa, fb));
    // restriction k -> k+1: three axis passes (fine -> tmp[0] -> tmp[1] -> coarse), FP64
    B->restr[dir].resize(3 * std::max(B->maxlev - 1, 0));
    for (int k = 0; k + 1 < B->maxlev; ++k)
      for (int ax = 0; ax < 3; ++ax) {
        std::vector<AxisKArgs<double>> ra;
        std::vector<int> rb;
        for (const BatchRep& r : reps) {
          Plan& P = *r.plan;
          AxisKArgs<double> a{};
          int nb = 0;
          if (k + 1 < P.levels) {
            void* const* q = dir ? P.d.aq : P.d.gq;
            const double* src[3] = {(const double*)q[k], (const double*)tmp_of(r, 0), (const double*)tmp_of(r, 1)};
            double* dst[3] = {(double*)tmp_of(r, 0), (double*)tmp_of(r, 1), (double*)q[k + 1]};
            int cur[3] = {P.n[k][0], P.n[k][1], P.n[k][2]};
            for (int a2 = 0; a2 < ax; ++a2) cur[a2] = P.n[k + 1][a2];
            for (int d = 0; d < 3; ++d) a.A.nin[d] = cur[d];
            cur[ax] = P.n[k + 1][ax];
            for (int d = 0; d < 3; ++d) a.A.nout[d] = cur[d];
            a.A.axis = ax;
            a.A.lo_in = P.lo[k][ax];
            a.A.lo_out = P.lo[k + 1][ax];
            a.A.periodic = P.P.periodic;
            a.in = src[ax];
            a.out = dst[ax];
            a.acc = 0;
            nb = ew_blocks((int64_t)cur[0] * cur[1] * cur[2]);
          }
          ra.push_back(a);
          rb.push_back(nb);
        }
        chk(make_table(B->restr[dir][3 * k + ax], ra, rb));
      }
    // lattice cutoff of every level below the top.  FFT form (every plan
    // periodic and built with it): five launches over all levels of all
    // replicas, level k of a replica working at offset sum_{j<k} N_j of its
    // plan's complex workspace
    bool all_fft = true;
    for (const BatchRep& r : reps) all_fft = all_fft && r.plan->lattice_fft;
    if (all_fft) {
      std::vector<FftBatchItem> items;
      for (const BatchRep& r : reps) {
        Plan& P = *r.plan;
        void* const* q = dir ? P.d.aq : P.d.gq;
        void* const* u = dir ? P.d.au : P.d.gu;
        int64_t off = 0;
        for (int k = 0; k + 1 < P.levels; ++k) {
          void* work = dir ? S1[&r - &reps[0]].fftw : P.d.fft_work;
          items.push_back(FftBatchItem{&P.fftl[k], (const double*)q[k], u[k],
                                       (char*)work + 2 * sizeof(float) * (size_t)off});
          off += grid_points(P, k);
        }
      }
      chk(fft_batch_build(items, false, &B->fft[dir]));
    }
    // otherwise the stencil, all in one launch: FP32 copies of the charges at
    // offsets of tmp[0], the outputs zeroed where several blocks add into them
    if (!all_fft) {
      std::vector<ConvKArgs> ca;
      std::vector<LatKArgs> la;
      std::vector<int> cb, lb;
      size_t sm = 0;
      for (const BatchRep& r : reps) {
        Plan& P = *r.plan;
        void* const* q = dir ? P.d.aq : P.d.gq;
        void* const* u = dir ? P.d.au : P.d.gu;
        int64_t off = 0;
        for (int k = 0; k + 1 < P.levels; ++k) {
          const int64_t np = grid_points(P, k);
          float* qf = (float*)tmp_of(r, 0) + off;
          off += np;
          ca.push_back(ConvKArgs{(const double*)q[k], qf, np});
          cb.push_back(ew_blocks(np));
          GridDims G = dims_of(P, k);
          LatKArgs a;
          if (k == 0 && P.lattice_txn > 0) {  // the plan's tuned tile on its finest level
            a.L.txn = P.lattice_txn;
            a.L.tyn = P.lattice_tyn;
          } else {
            lattice_tile(G.n[0], G.n[1], P.E, a.L.txn, a.L.tyn);
          }
          const int TW = kLatticeLP * a.L.txn, LBY = 2 * a.L.tyn;
          a.q = qf;
          a.u = (float*)u[k];
          a.G = G;
          a.seg = (const Segment2*)P.d.seg2;
          a.seg_start = P.d.seg_start;
          a.L.Ex = P.E[0];
          a.L.Ey = P.E[1];
          a.L.Ez = P.E[2];
          a.L.nbz = (int)blocks_for(G.n[2], kLatticeZ);
          a.nbx = (int)blocks_for(G.n[0], TW);
          a.nby = (int)blocks_for(G.n[1], LBY);
          a.L.nsplit = 1;  // set below, once the bricks of every replica and level are known
          a.scale = (float)std::ldexp(1.0, -k);
          a.up = nullptr;
          la.push_back(a);
          lb.push_back(a.nbx * a.nby * a.L.nbz);
          sm = std::max(sm, lattice_smem(a.L.txn, a.L.tyn, P.E));
        }
      }
      // one launch holds the bricks of every replica and level, so the input
      // planes are split over several blocks only while the whole launch
      // falls short of lattice_waves blocks per SM
      int64_t bricks = 0;
      for (int b : lb) bricks += b;
      const int64_t target = (int64_t)reps[0].plan->lattice_waves * 152 * 4 / kLatticeZ;
      const int nsplit = (int)std::max<int64_t>(1, (target + bricks - 1) / std::max<int64_t>(bricks, 1));
      // split grids write their parts to one buffer of the graph, reduced in
      // part order afterwards (reproducible sums)
      int64_t elems = 0;
      for (size_t i = 0; i < la.size(); ++i) {
        la[i].L.nsplit = std::min(nsplit, kLatticeZ + 2 * la[i].L.Ez);
        lb[i] *= la[i].L.nsplit;
        if (la[i].L.nsplit > 1) elems += (int64_t)la[i].L.nsplit * la[i].G.n[0] * la[i].G.n[1] * la[i].G.n[2];
      }
      if (elems > 0) chk(cudaMalloc((void**)&B->lparts[dir], sizeof(float) * (size_t)elems));
      std::vector<ReduceKArgs> ra;
      std::vector<int> rb;
      int64_t off = 0;
      for (size_t i = 0; i < la.size(); ++i) {
        const int64_t np = (int64_t)la[i].G.n[0] * la[i].G.n[1] * la[i].G.n[2];
        if (la[i].L.nsplit > 1 && B->lparts[dir]) {
          la[i].up = B->lparts[dir] + off;
          ra.push_back(ReduceKArgs{la[i].up, la[i].u, np, la[i].L.nsplit});
          rb.push_back(ew_blocks(np));
          off += (int64_t)la[i].L.nsplit * np;
        }
      }
      chk(make_table(B->conv[dir], ca, cb));
      chk(make_table(B->lattice[dir], la, lb, sm));
      chk(make_table(B->reduce_u[dir], ra, rb));
    }
    {  // top level of every replica
      std::vector<TopKArgs> ta;
      std::vector<int> tb;
      for (const BatchRep& r : reps) {
        Plan& P = *r.plan;
        const int top = P.levels - 1;
        void* const* q = dir ? P.d.aq : P.d.gq;
        void* const* u = dir ? P.d.au : P.d.gu;
        ta.push_back(TopKArgs{(const double*)q[top], (float*)u[top], dir ? S1[&r - &reps[0]].topu : P.d.topu,
                              dims_of(P, top), P.d.topK,
                              P.top_table_dims[0], P.top_table_dims[1]});
        tb.push_back((int)blocks_for(grid_points(P, top), kTopWarps));
      }
      chk(make_table(B->top[dir], ta, tb));
    }
    // prolongation k+1 -> k: three passes (coarse -> tmp[0] -> tmp[1] -> fine, the last one adding), FP32
    B->prol[dir].resize(3 * std::max(B->maxlev - 1, 0));
    for (int k = B->maxlev - 2; k >= 0; --k)
      for (int i = 0; i < 3; ++i) {
        std::vector<AxisKArgs<float>> pa;
        std::vector<int> pb;
        for (const BatchRep& r : reps) {
          Plan& P = *r.plan;
          AxisKArgs<float> a{};
          int nb = 0;
          if (k + 1 < P.levels) {
            void* const* u = dir ? P.d.au : P.d.gu;
            const float* src[3] = {(const float*)u[k + 1], (const float*)tmp_of(r, 0), (const float*)tmp_of(r, 1)};
            float* dst[3] = {(float*)tmp_of(r, 0), (float*)tmp_of(r, 1), (float*)u[k]};
            int cur[3] = {P.n[k + 1][0], P.n[k + 1][1], P.n[k + 1][2]};
            for (int j = 0; j < i; ++j) cur[2 - j] = P.n[k][2 - j];
            const int ax = 2 - i;  // z, then y, then x
            for (int d = 0; d < 3; ++d) a.A.nin[d] = cur[d];
            cur[ax] = P.n[k][ax];
            for (int d = 0; d < 3; ++d) a.A.nout[d] = cur[d];
            a.A.axis = ax;
            a.A.lo_in = P.lo[k + 1][ax];
            a.A.lo_out = P.lo[k][ax];
            a.A.periodic = P.P.periodic;
            a.in = src[i];
            a.out = dst[i];
            a.acc = (i == 2) ? 1 : 0;
            nb = ew_blocks((int64_t)cur[0] * cur[1] * cur[2]);
          }
          pa.push_back(a);
          pb.push_back(nb);
        }
        chk(make_table(B->prol[dir][3 * k + i], pa, pb));
      }
    {  // interpolation and assembly
      std::vector<InterpKArgs<float, double>> ia;
      std::vector<int> ib;
      std::vector<EnergyKArgs> ea;
      std::vector<int> eb;
      size_t sm = 0;
      for (const BatchRep& r : reps) {
        Plan& P = *r.plan;
        auto K = dir ? interp_kargs<float, double>(P, true, nullptr, nullptr, r.grad_energy, r.grad_pos, r.grad_q,
                                                   nullptr, true)
                     : interp_kargs<float, double>(P, false, r.phi, r.force, nullptr, nullptr, nullptr, P.d.partial,
                                                   true);
        const int nb = K.nbx * K.nby * (int)blocks_for(P.nc[2], K.AA.B);
        ia.push_back(K);
        ib.push_back(r.n > 0 ? nb : 0);
        sm = std::max(sm, sizeof(float) * (size_t)K.AA.pd * K.AA.pd * K.AA.pd);
        ea.push_back(EnergyKArgs{P.d.partial, r.n > 0 ? nb : 0, r.energy});
        eb.push_back(1);
      }
      chk(make_table(B->interp[dir], ia, ib, sm));
      if (dir == 0) chk(make_table(B->energy, ea, eb));
    }
  }
  (void)R;
  // persistent chains (replica 0's plan asks for them): one cooperative launch
  // per chain, as many blocks as are co-resident
  if (e == cudaSuccess && !reps.empty() && reps[0].plan->batch_persistent) {
    const bool o3 = B->order == 3;
    int dev = 0, nsm = 0, per_r = 0, per_p = 0;
    chk(cudaGetDevice(&dev));
    chk(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    chk(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_r, (const void*)(o3 ? kb_restrict_chain<3> : kb_restrict_chain<5>), kEw, 0));
    chk(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_p, (const void*)(o3 ? kb_prolong_chain<3> : kb_prolong_chain<5>), kEw, 0));
    B->chain_blocks = nsm * std::max(1, std::min(per_r, per_p));
    for (int dir = 0; dir < (backward ? 2 : 1) && e == cudaSuccess; ++dir) {
      std::vector<PassDesc> rd, pd;
      for (int k = 0; k + 1 < B->maxlev; ++k)
        for (int ax = 0; ax < 3; ++ax) {
          const auto& t = B->restr[dir][3 * k + ax];
          if (t.total > 0) rd.push_back(PassDesc{t.args, t.first, t.nrep, t.total});
        }
      for (int k = B->maxlev - 2; k >= 0; --k)
        for (int i = 0; i < 3; ++i) {
          const auto& t = B->prol[dir][3 * k + i];
          if (t.total > 0) pd.push_back(PassDesc{t.args, t.first, t.nrep, t.total});
        }
      B->n_restr = (int)rd.size();
      B->n_prol = (int)pd.size();
      chk(cudaMalloc((void**)&B->chain_restr[dir], sizeof(PassDesc) * std::max<size_t>(1, rd.size())));
      chk(cudaMalloc((void**)&B->chain_prol[dir], sizeof(PassDesc) * std::max<size_t>(1, pd.size())));
      if (e == cudaSuccess && !rd.empty())
        chk(cudaMemcpy(B->chain_restr[dir], rd.data(), sizeof(PassDesc) * rd.size(), cudaMemcpyHostToDevice));
      if (e == cudaSuccess && !pd.empty())
        chk(cudaMemcpy(B->chain_prol[dir], pd.data(), sizeof(PassDesc) * pd.size(), cudaMemcpyHostToDevice));
    }
    chk(cudaMalloc((void**)&B->bar, 2 * sizeof(unsigned)));
    if (e == cudaSuccess) chk(cudaMemset(B->bar, 0, 2 * sizeof(unsigned)));
    B->status = reps[0].plan->d.status;
    B->persistent = true;
  }
  if (e != cudaSuccess) {
    grid_batch_free(B);
    return e;
  }
  *out = B;
  return cudaSuccess;
}

// One chain as a cooperative launch.
template <typename K>
cudaError_t launch_chain(GridBatch* B, K kernel, PassDesc* passes, int npass, cudaStream_t st) {
  if (npass == 0) return cudaSuccess;
  void* args[] = {(void*)&passes, (void*)&npass, (void*)&B->bar, (void*)&B->status};
  return cudaLaunchCooperativeKernel((const void*)kernel, dim3(B->chain_blocks), dim3(kEw), args, 0, st);
}

template <typename A, typename K>
void launch_table(const BatchTable<A>& t, K kernel, int threads, cudaStream_t st) {
  if (t.total > 0) kernel<<<t.total, threads, t.smem, st>>>(t.args, t.first, t.nrep);
}

cudaError_t grid_batch_front(GridBatch* B, bool backward, cudaStream_t st) {
  if (backward && !B->has_backward) return cudaErrorInvalidValue;
  const bool o3 = B->order == 3;
  launch_table(B->zero_fx, kb_zero, kEw, st);
  launch_table(B->anterp, o3 ? kb_anterp_fx<3> : kb_anterp_fx<5>, 256, st);
  launch_table(B->fx[0], kb_fx_to_f64, kEw, st);
  if (backward) launch_table(B->fx[1], kb_fx_to_f64, kEw, st);
  return cudaGetLastError();
}

bool grid_batch_persistent(const GridBatch* B) { return B->persistent; }

cudaError_t grid_batch_levels(GridBatch* B, int d, cudaStream_t st) {
  if (d == 1 && !B->has_backward) return cudaErrorInvalidValue;
  const bool o3 = B->order == 3;
  if (B->persistent) {
    cudaError_t e = launch_chain(B, o3 ? kb_restrict_chain<3> : kb_restrict_chain<5>, B->chain_restr[d], B->n_restr, st);
    if (e != cudaSuccess) return e;
  } else {
    for (int k = 0; k + 1 < B->maxlev; ++k)
      for (int ax = 0; ax < 3; ++ax)
        launch_table(B->restr[d][3 * k + ax], o3 ? kb_restrict_axis<3> : kb_restrict_axis<5>, kEw, st);
  }
  if (B->fft[d]) {
    cudaError_t e = fft_batch_launch(B->fft[d], st);
    if (e != cudaSuccess) return e;
  } else {
    launch_table(B->conv[d], kb_f64_to_f32, kEw, st);
    launch_table(B->lattice[d], kb_lattice_f2, 32 * kLatticeZ, st);
    launch_table(B->reduce_u[d], kb_lattice_reduce, kEw, st);
  }
  launch_table(B->top[d], kb_top, 32 * kTopWarps, st);
  if (B->persistent) {
    cudaError_t e = launch_chain(B, o3 ? kb_prolong_chain<3> : kb_prolong_chain<5>, B->chain_prol[d], B->n_prol, st);
    if (e != cudaSuccess) return e;
  } else {
    for (int k = B->maxlev - 2; k >= 0; --k)
      for (int i = 0; i < 3; ++i)
        launch_table(B->prol[d][3 * k + i], o3 ? kb_prolong_axis<3> : kb_prolong_axis<5>, kEw, st);
  }
  return cudaGetLastError();
}

cudaError_t grid_batch_interp(GridBatch* B, bool backward, cudaStream_t st) {
  const bool o3 = B->order == 3;
  if (backward) {
    if (!B->has_backward) return cudaErrorInvalidValue;
    launch_table(B->interp[1], o3 ? kb_interp_bwd<3> : kb_interp_bwd<5>, 256, st);
  } else {
    launch_table(B->interp[0], o3 ? kb_interp_fwd<3> : kb_interp_fwd<5>, 256, st);
    launch_table(B->energy, kb_energy_final, 1024, st);
  }
  return cudaGetLastError();
}

// Opts the patch kernels into more than 48 KB of dynamic shared memory.  Done
// once per process when the first plan is built, so that no configuration call
// happens while a stream is being captured into a graph.
cudaError_t configure_kernels() {
  cudaError_t e = cudaSuccess;
  auto set = [&](const void* f) {
    cudaError_t r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLatticeSmemMax);
    if (r != cudaSuccess) e = r;
  };
  set((const void*)k_interp_gather<float, 3>);
  set((const void*)k_interp_gather<float, 5>);
  set((const void*)k_interp_gather<double, 3>);
  set((const void*)k_interp_gather<double, 5>);
  set((const void*)k_lattice_f2<kLatticeLP, 4, 8>);
  set((const void*)k_lattice_f2<kLatticeLP, 0, 0>);
  set((const void*)kb_lattice_f2);
  set((const void*)kb_anterp_fx<3>);
  set((const void*)kb_anterp_fx<5>);
  set((const void*)kb_interp_fwd<3>);
  set((const void*)kb_interp_fwd<5>);
  set((const void*)kb_interp_bwd<3>);
  set((const void*)kb_interp_bwd<5>);
  set((const void*)k_anterp_fx<3>);
  set((const void*)k_anterp_fx<5>);
  set((const void*)k_anterp_patch<double, double, 3>);
  set((const void*)k_anterp_patch<double, double, 5>);
  set((const void*)k_interp_bwd<float, 3, double>);
  set((const void*)k_interp_bwd<float, 3, float>);
  set((const void*)k_interp_bwd<float, 5, double>);
  set((const void*)k_interp_bwd<float, 5, float>);
  set((const void*)k_interp_bwd<double, 3, double>);
  set((const void*)k_interp_bwd<double, 3, float>);
  set((const void*)k_interp_bwd<double, 5, double>);
  set((const void*)k_interp_bwd<double, 5, float>);
  if (e == cudaSuccess) e = configure_fft_kernels();
  return e;
}

}  // namespace msm
