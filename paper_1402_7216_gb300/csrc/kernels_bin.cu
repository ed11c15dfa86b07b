// kernels_bin.cu -- atom binning (link cells, Sec. "Short-range interactions":
// atoms are binned into cells so that each atom only examines nearby cells).
//
// A counting sort over cells in five launches:
//   k_bin_count    cell key of every atom; a provisional rank inside the cell
//                  from one warp-aggregated atomic per (warp, cell)
//   k_cell_sums    per-chunk sums of the cell counts
//   k_cell_scan    exclusive scan -> cell_start; resets the counts to zero
//                  for the next evaluation
//   k_bin_perm     perm[cell_start + rank] = atom index
//   k_cell_fill    one warp per cell: orders the cell's atoms by the key
//                  (slab, input index) -- the slab is the atom's place on
//                  256 slabs across the cell in x, so that a row of cells
//                  (cells are numbered x fastest) is sorted by x and any
//                  run of consecutive atoms of a row is a compact slab of it
//                  (the pair kernel's 32-atom target runs);
//                  each atom's final rank is the number of the cell's atoms
//                  with a smaller key -- and writes their sorted records:
//                  cell-local coordinates for the pair sums, fractional
//                  level-0 grid coordinates and the first support index for
//                  the grid passes, and the permutation back to input order.
// The provisional ranks follow the order in which the atomics were served;
// the reordering makes the sorted order a function of the input alone, so
// every later pass sums in the same order on every run and the results are
// bit-reproducible.  A cell of more than kOrderMax atoms (over 20 times the
// default cell fill) keeps the atomic order: still correct, only its
// rounding may vary between runs.
//
// Precision.  The FP64 plan folds and bins in FP64.  The mixed plan takes no
// FP64 arithmetic at all (this GPU issues FP64 at 1/64 of the FP32 rate): an
// FP64 coordinate is split with integer operations into hi + lo (two floats,
// 24 + 29 significant bits), cell and grid origins are FP32 pairs whose
// leading part times any index is exact, and the differences that matter,
// hi - k*c_hi, are exact by Sterbenz' lemma.  The cell-local coordinate and
// the fractional grid coordinate therefore carry a single FP32 rounding, as
// if they had been computed in FP64 and rounded.  FP32 inputs (hi = x, lo = 0)
// take the same path.  Positions outside [0, L) of a periodic box are folded
// in FP64 first (rare).
#include <cmath>
#include <cstring>
#include <new>
#include <type_traits>

#include "msm_internal.h"

namespace msm {

namespace {

constexpr int kScanChunk = 4096;  // cells per block of the cell scan (1024 threads x 4)
constexpr int kFillWarps = 8;     // cells per block of k_cell_fill
constexpr int kOrderMax = 512;    // largest cell that k_cell_fill puts in key order

// Folds x into [0, L) (multiplying by the reciprocal: FP64 division is slow).
__device__ __forceinline__ double fold(double x, double L, double inv_L) {
  double y = x - L * floor(x * inv_L);
  if (y >= L) y -= L;
  if (y < 0.0) y += L;
  return y;
}

struct BinArgs {
  // FP64 plan
  double box[3], inv_box[3], cw[3], inv_cw[3], h[3], inv_h[3];
  // mixed plan: c = c_hi + c_lo with k * c_hi exact for every index k in use
  float cw_hi[3], cw_lo[3], cwf[3], inv_cwf[3];
  float h_hi[3], h_lo[3], hf[3], inv_hf[3];
  long long box_bits[3];  // bit pattern of L as a double (inside test for FP64 inputs)
  int box_bits32[3];      // ... of float(L) (FP32 inputs)
  int nc[3];
  int fmax[3];  // open grids: largest floor(x/h) the level-0 grid covers
  int periodic;
  int S;
};

// Splits a finite y >= 0 into hi + lo with integer operations only: hi keeps
// the leading 24 significant bits (truncated), lo the next 29 (so hi + lo
// equals y to 2^-48 relative).  y < 2^-126 maps to 0.
__device__ __forceinline__ void split_nonneg(double y, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(y);
  const int e = (int)(b >> 52);  // biased exponent (the sign bit is 0)
  if (e < 897) {
    hi = 0.f;
    lo = 0.f;
    return;
  }
  hi = __int_as_float(((e - 896) << 23) | (int)((unsigned)(b >> 29) & 0x7fffffu));
  const unsigned ml = (unsigned)b & 0x1fffffffu;
  lo = (e >= 949) ? __fmul_rn(__uint2float_rn(ml), __int_as_float((e - 948) << 23)) : 0.f;
}
__device__ __forceinline__ void split_nonneg(float y, float& hi, float& lo) {
  hi = (y > 0.f) ? y : 0.f;  // -0 -> 0
  lo = 0.f;
}

__device__ __forceinline__ bool finite_bits(double x) {
  return ((unsigned long long)__double_as_longlong(x) >> 52 & 0x7ff) != 0x7ff;
}
__device__ __forceinline__ bool finite_bits(float x) { return ((unsigned)__float_as_int(x) >> 23 & 0xff) != 0xff; }

// 0 <= x < L (periodic, strict) or 0 <= x <= L (open), decided on the bit
// pattern: non-negative IEEE values order like their bit patterns.  A false
// "outside" for x == float(L) < L only sends the atom through the fold.
__device__ __forceinline__ bool inside_bits(double x, const BinArgs& A, int d, bool closed) {
  long long b = __double_as_longlong(x);
  if (b == (long long)0x8000000000000000ull) b = 0;  // -0
  return b >= 0 && (closed ? b <= A.box_bits[d] : b < A.box_bits[d]);
}
__device__ __forceinline__ bool inside_bits(float x, const BinArgs& A, int d, bool closed) {
  int b = __float_as_int(x);
  if (b == (int)0x80000000u) b = 0;
  return b >= 0 && (closed ? b <= A.box_bits32[d] : b < A.box_bits32[d]);
}

// x - k * c for x = hi + lo, c = c_hi + c_lo: k * c_hi is exact and so is
// hi - k * c_hi (Sterbenz), so the result is rounded once.
__device__ __forceinline__ float offset_from(float hi, float lo, int k, float c_hi, float c_lo) {
  const float kf = (float)k;
  return __fadd_rn(__fsub_rn(hi, __fmul_rn(kf, c_hi)), __fsub_rn(lo, __fmul_rn(kf, c_lo)));
}

// One coordinate on the mixed plan: the folded coordinate as hi + lo
// (status bits to `bad`), its cell index, and its level-0 floor index and
// fraction.  Every step uses explicitly rounded intrinsics, so the count and
// scatter kernels reach the same decisions.
template <typename IO>
__device__ __forceinline__ void prep_mixed(IO x, const BinArgs& A, int d, int& bad, float& hi, float& lo) {
  if (!finite_bits(x)) {
    bad |= kStatusNonfinite;
    hi = lo = 0.f;
  } else if (inside_bits(x, A, d, !A.periodic)) {
    split_nonneg(x, hi, lo);
  } else if (A.periodic) {
    split_nonneg(fold((double)x, A.box[d], A.inv_box[d]), hi, lo);
  } else {
    bad |= kStatusOutside;
    hi = lo = 0.f;
  }
}

__device__ __forceinline__ int cell_mixed(float hi, float lo, const BinArgs& A, int d) {
  const int nc = A.nc[d];
  int k = min((int)__fmul_rz(hi, A.inv_cwf[d]), nc - 1);
  const float loc = offset_from(hi, lo, k, A.cw_hi[d], A.cw_lo[d]);
  if (loc < 0.f && k > 0) --k;
  else if (loc >= A.cwf[d] && k < nc - 1) ++k;
  return k;
}

__device__ __forceinline__ void grid_mixed(float hi, float lo, const BinArgs& A, int d, int& b, float& fr) {
  b = (int)__fmul_rz(hi, A.inv_hf[d]);
  if (!A.periodic) b = min(b, A.fmax[d]);
  float dist = offset_from(hi, lo, b, A.h_hi[d], A.h_lo[d]);
  if (dist < 0.f && b > 0) {
    --b;
    dist = offset_from(hi, lo, b, A.h_hi[d], A.h_lo[d]);
  } else if (dist >= A.hf[d] && (A.periodic || b < A.fmax[d])) {
    ++b;
    dist = offset_from(hi, lo, b, A.h_hi[d], A.h_lo[d]);
  }
  fr = __fmul_rn(dist, A.inv_hf[d]);
}

// The same on the FP64 plan (FP64 arithmetic throughout).
template <typename IO>
__device__ __forceinline__ double prep_fp64(IO xin, const BinArgs& A, int d, int& bad) {
  const double v = (double)xin;
  if (!finite_bits(xin)) {
    bad |= kStatusNonfinite;
    return 0.0;
  }
  if (A.periodic) return fold(v, A.box[d], A.inv_box[d]);
  if (!(v >= 0.0 && v <= A.box[d])) {
    bad |= kStatusOutside;
    return 0.0;
  }
  return v;
}

__device__ __forceinline__ int cell_fp64(double v, const BinArgs& A, int d) {
  const int ci = (int)floor(__dmul_rn(v, A.inv_cw[d]));
  return ci < 0 ? 0 : (ci >= A.nc[d] ? A.nc[d] - 1 : ci);
}

__device__ __forceinline__ void grid_fp64(double v, const BinArgs& A, int d, int& b, double& fr) {
  const double t = v * A.inv_h[d];
  double fl = floor(t);
  if (!A.periodic && fl > (double)A.fmax[d]) fl = (double)A.fmax[d];  // x = L rounding up
  b = (int)fl;
  fr = t - fl;
}

// Arguments of the count and scatter kernels (one replica).
template <typename IO>
struct BinKArgs {
  const IO* pos;
  const IO* q;
  int n;
  BinArgs A;
  int* count;
  int* key;
  int* rank;
  int* status;
  const int* cell_start;
  void* atoms;
  void* gfrac;
  int4* gbase;
  int* perm;
  int ncell;
};

template <typename IO, bool FP64>
__device__ __forceinline__ void bin_count_body(const IO* __restrict__ pos, const IO* __restrict__ q, int n,
                                               const BinArgs& A, int* __restrict__ count, int* __restrict__ key_out,
                                               int* __restrict__ rank_out, int* __restrict__ status, int blk) {
  const int i = blk * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const bool valid = i < n;
  int key = -1, bad = 0;
  if (valid) {
    int c[3];
    for (int d = 0; d < 3; ++d) {
      const IO x = pos[3 * (size_t)i + d];
      if (FP64) {
        c[d] = cell_fp64(prep_fp64(x, A, d, bad), A, d);
      } else {
        float hi, lo;
        prep_mixed(x, A, d, bad, hi, lo);
        c[d] = cell_mixed(hi, lo, A, d);
      }
    }
    if (!finite_bits(q[i])) bad |= kStatusNonfinite;
    key = (c[2] * A.nc[1] + c[1]) * A.nc[0] + c[0];
  }
  if (bad) atomicOr(status, bad);
  // one atomic per distinct cell in the warp
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  const int leader = __ffs(peers) - 1;
  int base = 0;
  if (valid && lane == leader) base = atomicAdd(&count[key], __popc(peers));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (valid) {
    key_out[i] = key;
    rank_out[i] = base + __popc(peers & ((1u << lane) - 1u));
  }
}

template <typename IO, bool FP64>
__global__ void __launch_bounds__(256) k_bin_count(const IO* __restrict__ pos, const IO* __restrict__ q, int n,
                                                   BinArgs A, int* __restrict__ count, int* __restrict__ key_out,
                                                   int* __restrict__ rank_out, int* __restrict__ status) {
  bin_count_body<IO, FP64>(pos, q, n, A, count, key_out, rank_out, status, blockIdx.x);
}

template <typename IO, bool FP64>
__global__ void __launch_bounds__(256) kb_bin_count(const BinKArgs<IO>* __restrict__ tab, const int* __restrict__ first,
                                                    int nrep) {
  const int r = batch_rep(first, nrep, blockIdx.x);
  const BinKArgs<IO>& a = tab[r];
  bin_count_body<IO, FP64>(a.pos, a.q, a.n, a.A, a.count, a.key, a.rank, a.status, blockIdx.x - first[r]);
}

template <int NT>
__device__ __forceinline__ int block_reduce_sum(int v, int* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  v = (lane < NT / 32) ? red[lane] : 0;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  return v;
}

struct ScanKArgs {
  int* count;
  int ncell;
  int* sums;
  int* cell_start;
};

__device__ __forceinline__ void cell_sums_body(const int* __restrict__ count, int ncell, int* __restrict__ sums,
                                               int blk) {
  __shared__ int red[32];
  const int c0 = blk * kScanChunk + 4 * threadIdx.x;
  int v = 0;
  for (int t = 0; t < 4; ++t) v += (c0 + t < ncell) ? count[c0 + t] : 0;
  v = block_reduce_sum<1024>(v, red);
  if (threadIdx.x == 0) sums[blk] = v;
}

__global__ void __launch_bounds__(1024) k_cell_sums(const int* __restrict__ count, int ncell, int* __restrict__ sums) {
  cell_sums_body(count, ncell, sums, blockIdx.x);
}

__global__ void __launch_bounds__(1024) kb_cell_sums(const ScanKArgs* __restrict__ tab, const int* __restrict__ first,
                                                     int nrep) {
  const int r = batch_rep(first, nrep, blockIdx.x);
  cell_sums_body(tab[r].count, tab[r].ncell, tab[r].sums, blockIdx.x - first[r]);
}

// cell_start[c] = sum of count[0..c); count[c] = 0 afterwards.
__device__ __forceinline__ void cell_scan_body(int* __restrict__ count, int ncell, const int* __restrict__ sums,
                                               int* __restrict__ cell_start, int blk) {
  __shared__ int red[32], wsum[32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  // this block's offset: the sums of the chunks before it
  int pre = 0;
  for (int b = t; b < blk; b += 1024) pre += sums[b];
  pre = block_reduce_sum<1024>(pre, red);
  const int c0 = blk * kScanChunk + 4 * t;
  int v[4], tot = 0;
  for (int k = 0; k < 4; ++k) {
    v[k] = (c0 + k < ncell) ? count[c0 + k] : 0;
    tot += v[k];
  }
  int x = tot;  // inclusive warp scan of the thread totals
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = wsum[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    wsum[lane] = w;
  }
  __syncthreads();
  int run = pre + (warp > 0 ? wsum[warp - 1] : 0) + x - tot;
  for (int k = 0; k < 4; ++k) {
    const int c = c0 + k;
    if (c < ncell) {
      cell_start[c] = run;
      count[c] = 0;
    }
    run += v[k];
  }
  if (c0 <= ncell - 1 && ncell - 1 < c0 + 4) cell_start[ncell] = run;  // end marker, by the last cell's thread
}

__global__ void __launch_bounds__(1024) k_cell_scan(int* __restrict__ count, int ncell,
                                                    const int* __restrict__ sums, int* __restrict__ cell_start) {
  cell_scan_body(count, ncell, sums, cell_start, blockIdx.x);
}

__global__ void __launch_bounds__(1024) kb_cell_scan(const ScanKArgs* __restrict__ tab, const int* __restrict__ first,
                                                     int nrep) {
  const int r = batch_rep(first, nrep, blockIdx.x);
  cell_scan_body(tab[r].count, tab[r].ncell, tab[r].sums, tab[r].cell_start, blockIdx.x - first[r]);
}

// perm[cell_start[key] + provisional rank] = i
__device__ __forceinline__ void bin_perm_body(int n, const int* __restrict__ key_in, const int* __restrict__ rank_in,
                                              const int* __restrict__ cell_start, int* __restrict__ perm, int blk) {
  const int i = blk * blockDim.x + threadIdx.x;
  if (i >= n) return;
  perm[cell_start[key_in[i]] + rank_in[i]] = i;
}

__global__ void __launch_bounds__(256) k_bin_perm(int n, const int* __restrict__ key_in,
                                                  const int* __restrict__ rank_in, const int* __restrict__ cell_start,
                                                  int* __restrict__ perm) {
  bin_perm_body(n, key_in, rank_in, cell_start, perm, blockIdx.x);
}

// Slab of atom i across its cell `key` in x (0..kSlabs-1), from its
// cell-local x coordinate (the same arithmetic as the records below).
constexpr int kSlabs = 256;
template <typename IO, bool FP64>
__device__ __forceinline__ int slab_code(const IO* __restrict__ pos, const BinArgs& A, int key, int i) {
  const int kx = key % A.nc[0];
  int bad = 0, sx;
  if (FP64) {
    const double v = prep_fp64(pos[3 * (size_t)i], A, 0, bad);
    sx = (int)((v - kx * A.cw[0]) * (kSlabs * A.inv_cw[0]));
  } else {
    float hi, lo;
    prep_mixed(pos[3 * (size_t)i], A, 0, bad, hi, lo);
    sx = (int)(offset_from(hi, lo, kx, A.cw_hi[0], A.cw_lo[0]) * (kSlabs * A.inv_cwf[0]));
  }
  return min(max(sx, 0), kSlabs - 1);
}

// The sorted records of atom i at slot s of cell `key` (the atom's cell as
// k_bin_count found it: the same functions on the same input).
template <typename IO, bool FP64>
__device__ __forceinline__ void write_records(const IO* __restrict__ pos, const IO* __restrict__ q, const BinArgs& A,
                                              int key, int i, int s, void* __restrict__ atoms_v,
                                              void* __restrict__ gfrac_v, int4* __restrict__ gbase,
                                              int* __restrict__ perm) {
  const int kc[3] = {key % A.nc[0], (key / A.nc[0]) % A.nc[1], key / (A.nc[0] * A.nc[1])};
  int bad = 0, bs[3];
  if (FP64) {
    double loc[3], fr[3];
    for (int d = 0; d < 3; ++d) {
      const double v = prep_fp64(pos[3 * (size_t)i + d], A, d, bad);
      loc[d] = v - kc[d] * A.cw[d];
      grid_fp64(v, A, d, bs[d], fr[d]);
    }
    const double qi = finite_bits(q[i]) ? (double)q[i] : 0.0;
    reinterpret_cast<R4<double>*>(atoms_v)[s] = R4<double>{loc[0], loc[1], loc[2], qi};
    reinterpret_cast<R4<double>*>(gfrac_v)[s] = R4<double>{fr[0], fr[1], fr[2], qi};
  } else {
    float loc[3], fr[3];
    for (int d = 0; d < 3; ++d) {
      float hi, lo;
      prep_mixed(pos[3 * (size_t)i + d], A, d, bad, hi, lo);
      loc[d] = offset_from(hi, lo, kc[d], A.cw_hi[d], A.cw_lo[d]);
      grid_mixed(hi, lo, A, d, bs[d], fr[d]);
    }
    const float qi = finite_bits(q[i]) ? (float)q[i] : 0.f;
    reinterpret_cast<R4<float>*>(atoms_v)[s] = R4<float>{loc[0], loc[1], loc[2], qi};
    reinterpret_cast<R4<float>*>(gfrac_v)[s] = R4<float>{fr[0], fr[1], fr[2], qi};
  }
  gbase[s] = make_int4(bs[0] - (A.S - 1), bs[1] - (A.S - 1), bs[2] - (A.S - 1), 0);
  perm[s] = i;
}

// One atom's records in registers (computed once from one read of its
// position) and its slab, from the same cell-local coordinates as
// slab_code and write_records above.
template <bool FP64>
struct CellRec {
  using T = typename std::conditional<FP64, double, float>::type;
  T loc[3], fr[3], q;
  int bs[3];
};

template <typename IO, bool FP64>
__device__ __forceinline__ int make_record(const IO* __restrict__ pos, const IO* __restrict__ q, const BinArgs& A,
                                           int key, int i, CellRec<FP64>& R) {
  const int kc[3] = {key % A.nc[0], (key / A.nc[0]) % A.nc[1], key / (A.nc[0] * A.nc[1])};
  int bad = 0, code = 0;
  for (int d = 0; d < 3; ++d) {
    if (FP64) {
      const double v = prep_fp64(pos[3 * (size_t)i + d], A, d, bad);
      R.loc[d] = v - kc[d] * A.cw[d];
      if (d == 0) code = (int)((v - kc[d] * A.cw[d]) * (kSlabs * A.inv_cw[d]));
      double fr;
      grid_fp64(v, A, d, R.bs[d], fr);
      R.fr[d] = fr;
    } else {
      float hi, lo;
      prep_mixed(pos[3 * (size_t)i + d], A, d, bad, hi, lo);
      const float loc = offset_from(hi, lo, kc[d], A.cw_hi[d], A.cw_lo[d]);
      R.loc[d] = loc;
      if (d == 0) code = (int)(loc * (kSlabs * A.inv_cwf[d]));
      float fr;
      grid_mixed(hi, lo, A, d, R.bs[d], fr);
      R.fr[d] = fr;
    }
  }
  code = min(max(code, 0), kSlabs - 1);
  R.q = finite_bits(q[i]) ? (typename CellRec<FP64>::T)q[i] : (typename CellRec<FP64>::T)0;
  return code;
}

template <bool FP64>
__device__ __forceinline__ void store_record(const CellRec<FP64>& R, const BinArgs& A, int i, int s,
                                             void* __restrict__ atoms_v, void* __restrict__ gfrac_v,
                                             int4* __restrict__ gbase, int* __restrict__ perm) {
  using T = typename CellRec<FP64>::T;
  reinterpret_cast<R4<T>*>(atoms_v)[s] = R4<T>{R.loc[0], R.loc[1], R.loc[2], R.q};
  reinterpret_cast<R4<T>*>(gfrac_v)[s] = R4<T>{R.fr[0], R.fr[1], R.fr[2], R.q};
  gbase[s] = make_int4(R.bs[0] - (A.S - 1), R.bs[1] - (A.S - 1), R.bs[2] - (A.S - 1), 0);
  perm[s] = i;
}

// One warp per cell: the cell's atoms (perm, in provisional order) are put in
// (slab, index) order and their records written.  A cell of at most 32
// atoms (nearly every cell) takes one atom per lane: the lane reads its
// atom's position once, keeps the records in registers, ranks its key among
// the cell's keys and stores at that rank.  Larger cells go through the keys
// in shared memory (idx: the warp's kOrderMax keys) and recompute the
// records.
template <typename IO, bool FP64>
__device__ __forceinline__ void cell_fill_body(const IO* __restrict__ pos, const IO* __restrict__ q,
                                               const BinArgs& A, const int* __restrict__ cell_start,
                                               void* __restrict__ atoms_v, void* __restrict__ gfrac_v,
                                               int4* __restrict__ gbase, int* __restrict__ perm, int ncell, int cell,
                                               long long* __restrict__ idx) {
  if (cell >= ncell) return;  // warp-uniform
  const int lane = threadIdx.x & 31;
  const int s0 = cell_start[cell], m = cell_start[cell + 1] - s0;
  if (m <= 32) {
    CellRec<FP64> R;
    long long k = 0x7fffffffffffffffll;  // lanes past the cell rank after every atom
    int i = 0;
    if (lane < m) {
      i = perm[s0 + lane];
      k = ((long long)make_record<IO, FP64>(pos, q, A, cell, i, R) << 32) | (long long)i;
      idx[lane] = k;
    }
    __syncwarp();
    if (lane < m) {
      int r = 0;
      for (int j = 0; j < m; ++j) r += idx[j] < k;  // keys are distinct: r is a permutation of 0..m-1
      store_record<FP64>(R, A, i, s0 + r, atoms_v, gfrac_v, gbase, perm);
    }
    __syncwarp();
  } else if (m <= kOrderMax) {
    for (int t = lane; t < m; t += 32) {
      const int i = perm[s0 + t];
      idx[t] = ((long long)slab_code<IO, FP64>(pos, A, cell, i) << 32) | (long long)i;
    }
    __syncwarp();
    for (int t = lane; t < m; t += 32) {
      const long long k = idx[t];
      int r = 0;
      for (int j = 0; j < m; ++j) r += idx[j] < k;  // keys are distinct: r is a permutation of 0..m-1
      write_records<IO, FP64>(pos, q, A, cell, (int)(k & 0xffffffffll), s0 + r, atoms_v, gfrac_v, gbase, perm);
    }
    __syncwarp();
  } else {
    for (int t = lane; t < m; t += 32)
      write_records<IO, FP64>(pos, q, A, cell, perm[s0 + t], s0 + t, atoms_v, gfrac_v, gbase, perm);
  }
}

template <typename IO, bool FP64>
__global__ void __launch_bounds__(32 * kFillWarps) k_cell_fill(const IO* __restrict__ pos, const IO* __restrict__ q,
                                                               BinArgs A, const int* __restrict__ cell_start,
                                                               void* __restrict__ atoms_v, void* __restrict__ gfrac_v,
                                                               int4* __restrict__ gbase, int* __restrict__ perm,
                                                               int ncell) {
  __shared__ long long idx[kFillWarps][kOrderMax];
  const int w = threadIdx.x >> 5;
  cell_fill_body<IO, FP64>(pos, q, A, cell_start, atoms_v, gfrac_v, gbase, perm, ncell, blockIdx.x * kFillWarps + w,
                           idx[w]);
}

// Batched forms: the atom-indexed kernels take 256 atoms per block, the cell
// fill kFillWarps cells per block (tables `atoms` and `cells`).
__global__ void __launch_bounds__(256) kb_bin_perm(const BinKArgs<double>* __restrict__ tab,
                                                   const int* __restrict__ first, int nrep) {
  const int r = batch_rep(first, nrep, blockIdx.x);
  const BinKArgs<double>& a = tab[r];
  bin_perm_body(a.n, a.key, a.rank, a.cell_start, a.perm, blockIdx.x - first[r]);
}

template <typename IO, bool FP64>
__global__ void __launch_bounds__(32 * kFillWarps) kb_cell_fill(const BinKArgs<IO>* __restrict__ tab,
                                                                const int* __restrict__ first, int nrep) {
  __shared__ long long idx[kFillWarps][kOrderMax];
  const int r = batch_rep(first, nrep, blockIdx.x);
  const BinKArgs<IO>& a = tab[r];
  const int w = threadIdx.x >> 5;
  cell_fill_body<IO, FP64>(a.pos, a.q, a.A, a.cell_start, a.atoms, a.gfrac, a.gbase, a.perm, a.ncell,
                           (blockIdx.x - first[r]) * kFillWarps + w, idx[w]);
}

// Veltkamp-style split c = hi + lo with hi holding `hb` significant bits.
void split_const(double c, int hb, float& hi, float& lo) {
  int ex = 0;
  const double f = std::frexp(c, &ex);  // c = f * 2^ex, f in [0.5, 1)
  const double h = std::ldexp(std::floor(std::ldexp(f, hb)), ex - hb);
  hi = (float)h;
  lo = (float)(c - h);
}

int bits_for(int kmax) {
  int b = 1;
  while ((1 << b) <= kmax) ++b;
  return b;
}

BinArgs bin_args(const Plan& P) {
  BinArgs A;
  for (int d = 0; d < 3; ++d) {
    const double L = P.P.box[d];
    A.box[d] = L;
    A.inv_box[d] = 1.0 / L;
    A.cw[d] = P.cw[d];
    A.inv_cw[d] = 1.0 / P.cw[d];
    A.h[d] = P.h[d];
    A.inv_h[d] = 1.0 / P.h[d];
    A.nc[d] = P.nc[d];
    A.fmax[d] = P.n[0][d] - 2 * P.S;
    // leading parts short enough that index * leading part is exact in FP32
    split_const(P.cw[d], 24 - bits_for(P.nc[d] + 1), A.cw_hi[d], A.cw_lo[d]);
    split_const(P.h[d], 24 - bits_for(P.n[0][d] + 2), A.h_hi[d], A.h_lo[d]);
    A.cwf[d] = (float)P.cw[d];
    A.inv_cwf[d] = (float)(1.0 / P.cw[d]);
    A.hf[d] = (float)P.h[d];
    A.inv_hf[d] = (float)(1.0 / P.h[d]);
    double Ld = L;
    float Lf = (float)L;
    std::memcpy(&A.box_bits[d], &Ld, 8);
    std::memcpy(&A.box_bits32[d], &Lf, 4);
  }
  A.periodic = P.P.periodic;
  A.S = P.S;
  return A;
}

}  // namespace

template <typename IO>
cudaError_t launch_binning(Plan& P, int64_t n64, const IO* pos, const IO* q, cudaStream_t st) {
  const int n = (int)n64;
  DeviceBuffers& D = P.d;
  const BinArgs A = bin_args(P);
  const unsigned nb = (unsigned)((n + 255) / 256);
  const unsigned nsc = (unsigned)((P.ncell + kScanChunk - 1) / kScanChunk);
  if (n > 0) {
    if (P.fp64)
      k_bin_count<IO, true><<<nb, 256, 0, st>>>(pos, q, n, A, D.count, D.key, D.rank, D.status);
    else
      k_bin_count<IO, false><<<nb, 256, 0, st>>>(pos, q, n, A, D.count, D.key, D.rank, D.status);
  }
  k_cell_sums<<<nsc, 1024, 0, st>>>(D.count, P.ncell, D.csum);
  k_cell_scan<<<nsc, 1024, 0, st>>>(D.count, P.ncell, D.csum, D.cell_start);
  if (n > 0) {
    const unsigned nf = (unsigned)((P.ncell + kFillWarps - 1) / kFillWarps);
    k_bin_perm<<<nb, 256, 0, st>>>(n, D.key, D.rank, D.cell_start, D.perm);
    if (P.fp64)
      k_cell_fill<IO, true><<<nf, 32 * kFillWarps, 0, st>>>(pos, q, A, D.cell_start, D.atoms, D.gfrac, D.gbase,
                                                            D.perm, P.ncell);
    else
      k_cell_fill<IO, false><<<nf, 32 * kFillWarps, 0, st>>>(pos, q, A, D.cell_start, D.atoms, D.gfrac, D.gbase,
                                                             D.perm, P.ncell);
  }
  P.launches += 2 + (n > 0 ? 3 : 0);
  return cudaGetLastError();
}

struct BinBatch {
  BatchTable<BinKArgs<double>> atoms;  // count and perm: 256 atoms per block
  BatchTable<BinKArgs<double>> cells;  // cell fill: kFillWarps cells per block
  BatchTable<ScanKArgs> scan;          // cell sums and scan: kScanChunk cells per block
};

cudaError_t bin_batch_build(const std::vector<BatchRep>& reps, BinBatch** out) {
  *out = nullptr;
  BinBatch* b = new (std::nothrow) BinBatch();
  if (!b) return cudaErrorMemoryAllocation;
  std::vector<BinKArgs<double>> ka;
  std::vector<ScanKArgs> sa;
  std::vector<int> kb, cb, sb;
  for (const BatchRep& r : reps) {
    Plan& P = *r.plan;
    DeviceBuffers& D = P.d;
    BinKArgs<double> a;
    a.pos = r.pos;
    a.q = r.q;
    a.n = (int)r.n;
    a.A = bin_args(P);
    a.count = D.count;
    a.key = D.key;
    a.rank = D.rank;
    a.status = D.status;
    a.cell_start = D.cell_start;
    a.atoms = D.atoms;
    a.gfrac = D.gfrac;
    a.gbase = D.gbase;
    a.perm = D.perm;
    a.ncell = P.ncell;
    ka.push_back(a);
    kb.push_back((int)((r.n + 255) / 256));
    cb.push_back(r.n > 0 ? (P.ncell + kFillWarps - 1) / kFillWarps : 0);
    sa.push_back(ScanKArgs{D.count, P.ncell, D.csum, D.cell_start});
    sb.push_back((P.ncell + kScanChunk - 1) / kScanChunk);
  }
  cudaError_t e = make_table(b->atoms, ka, kb);
  if (e == cudaSuccess) e = make_table(b->cells, ka, cb);
  if (e == cudaSuccess) e = make_table(b->scan, sa, sb);
  if (e != cudaSuccess) {
    bin_batch_free(b);
    return e;
  }
  *out = b;
  return cudaSuccess;
}

cudaError_t bin_batch_launch(BinBatch* b, cudaStream_t st) {
  if (b->atoms.total > 0)
    kb_bin_count<double, false><<<b->atoms.total, 256, 0, st>>>(b->atoms.args, b->atoms.first, b->atoms.nrep);
  kb_cell_sums<<<b->scan.total, 1024, 0, st>>>(b->scan.args, b->scan.first, b->scan.nrep);
  kb_cell_scan<<<b->scan.total, 1024, 0, st>>>(b->scan.args, b->scan.first, b->scan.nrep);
  if (b->atoms.total > 0)
    kb_bin_perm<<<b->atoms.total, 256, 0, st>>>(b->atoms.args, b->atoms.first, b->atoms.nrep);
  if (b->cells.total > 0)
    kb_cell_fill<double, false><<<b->cells.total, 32 * kFillWarps, 0, st>>>(b->cells.args, b->cells.first,
                                                                             b->cells.nrep);
  return cudaGetLastError();
}

void bin_batch_free(BinBatch* b) {
  if (!b) return;
  b->atoms.release();
  b->cells.release();
  b->scan.release();
  delete b;
}

template cudaError_t launch_binning<double>(Plan&, int64_t, const double*, const double*, cudaStream_t);
template cudaError_t launch_binning<float>(Plan&, int64_t, const float*, const float*, cudaStream_t);

}  // namespace msm
