// fft.cu -- the lattice cutoff of a periodic level as a cyclic convolution.
//
// On a periodic grid the lattice cutoff of level k (the step "lattice
// cutoff" of Sec. "Multilevel Summation Method", with g^k of Eq. msmgrid),
//   u^k_mu = sum_nu g^k(r_mu, r_nu) q^k_nu  over |r_mu - r_nu| < 2^(k+1) a,
// is the cyclic convolution u = K * q of the level's charges with the folded
// kernel K[n] = sum over the images of the taps n (mod M) of 2^-k G0(n): the
// same finite sum, so its discrete Fourier transform is the product of the
// transforms, u = IDFT(DFT(K) DFT(q)).  The kernel's transform K^ (real, as
// K is even) is computed once per plan and level in FP64 and stored with the
// 1/N of the inverse folded in; each evaluation then costs five passes over
// the level's grid instead of (taps) multiply-adds per point:
//   x forward (reading the FP64 charges), y forward, z forward with the
//   product by K^ and z inverse fused (the z line stays in shared memory),
//   y inverse, x inverse (writing the real part as the potential).
// Each pass is one launch over every lattice level of a plan (or of every
// replica of a batch), a table of per-level arguments mapping blocks to
// levels.  The 1-D transforms are mixed-radix Stockham FFTs (radices 4, 2,
// 3, 5, 7: every periodic grid size m 2^j with m <= 8) run in shared memory,
// a block taking L lines at once; along y and z the L lines are L
// consecutive x positions, so that every global access is a coalesced row
// segment, and the lines sit at an odd pitch so that those row segments
// land in distinct banks.  Twiddles are tabulated per stage on the host in
// FP64; index arithmetic divides by multiply and shift.  T = float on the
// mixed plan (the grids there are FP32), double on the FP64 plan.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "msm_internal.h"

namespace msm {

namespace {

constexpr int kFftThreads = 256;
constexpr int kFftBatch = 4;      // global loads a thread issues together
constexpr int kRoots = 7;          // the seventh roots of unity after the stage tables (radix 7)
constexpr size_t kFftSmem = 48 * 1024;  // line buffers per block, the budget lines_per_block aims for

template <typename T>
struct Cx {
  T x, y;
};

template <typename T>
__device__ __forceinline__ Cx<T> cmul(Cx<T> a, Cx<T> b) {
  return Cx<T>{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T>
__device__ __forceinline__ Cx<T> cadd(Cx<T> a, Cx<T> b) {
  return Cx<T>{a.x + b.x, a.y + b.y};
}
template <typename T>
__device__ __forceinline__ Cx<T> csub(Cx<T> a, Cx<T> b) {
  return Cx<T>{a.x - b.x, a.y - b.y};
}
// s i z with s = +1 or -1
template <typename T>
__device__ __forceinline__ Cx<T> cmuli(Cx<T> z, T s) {
  return Cx<T>{-s * z.y, s * z.x};
}
// the conjugate when s > 0 (the inverse transform's twiddles)
template <typename T>
__device__ __forceinline__ Cx<T> conj_if(Cx<T> z, T s) {
  return Cx<T>{z.x, s > 0 ? -z.y : z.y};
}

// Sizes are n = c 2^s with c odd and a product of 3, 5 and 7, so that
// x / n = (x >> s) / c: a shift, then a division by a constant for the usual
// c (1, 3, 5, 7: every periodic grid size m 2^j with m <= 8) and a plain
// division otherwise.
__device__ __forceinline__ int div_c(int x, int c) {
  return c == 1 ? x : c == 3 ? x / 3 : c == 5 ? x / 5 : c == 7 ? x / 7 : x / c;
}

// One axis's line transform (host-built): length n = c 2^s, stages with
// their radices (radix 4 and 2 first, then 3, 5, 7).
struct FftAxisDesc {
  int n, c, s;                    // n = c 2^s, c odd
  int nst;                        // stages
  unsigned long long radix_code;  // radix of stage st in bits 5 st .. 5 st + 4
};

// Small DFTs in place on v[0..R-1]; s = -1 forward, +1 inverse.
template <typename T>
__device__ __forceinline__ void dft2(Cx<T>* v) {
  const Cx<T> a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}
template <typename T>
__device__ __forceinline__ void dft4(Cx<T>* v, T s) {
  const Cx<T> a = v[0], b = v[1], c = v[2], d = v[3];
  const Cx<T> t0 = cadd(a, c), t1 = csub(a, c), t2 = cadd(b, d), t3 = cmuli(csub(b, d), s);
  v[0] = cadd(t0, t2);
  v[2] = csub(t0, t2);
  v[1] = cadd(t1, t3);
  v[3] = csub(t1, t3);
}
template <typename T>
__device__ __forceinline__ void dft3(Cx<T>* v, T s) {
  const T h = (T)0.86602540378443864676;  // sin(2 pi / 3)
  const Cx<T> a = v[0], b = v[1], c = v[2];
  const Cx<T> t = cadd(b, c);
  const Cx<T> m = Cx<T>{a.x - (T)0.5 * t.x, a.y - (T)0.5 * t.y};
  const Cx<T> d = cmuli(csub(b, c), s * h);
  v[0] = cadd(a, t);
  v[1] = cadd(m, d);
  v[2] = csub(m, d);
}
template <typename T>
__device__ __forceinline__ void dft5(Cx<T>* v, T s) {
  const T c1 = (T)0.30901699437494742410, c2 = (T)-0.80901699437494742410;  // cos(2 pi/5), cos(4 pi/5)
  const T s1 = (T)0.95105651629515357212, s2 = (T)0.58778525229247312917;   // sin(2 pi/5), sin(4 pi/5)
  const Cx<T> a = v[0];
  const Cx<T> t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]), t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
  const Cx<T> m1 = Cx<T>{a.x + c1 * t1.x + c2 * t2.x, a.y + c1 * t1.y + c2 * t2.y};
  const Cx<T> m2 = Cx<T>{a.x + c2 * t1.x + c1 * t2.x, a.y + c2 * t1.y + c1 * t2.y};
  const Cx<T> d1 = cmuli(Cx<T>{s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y}, s);
  const Cx<T> d2 = cmuli(Cx<T>{s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y}, s);
  v[0] = cadd(a, cadd(t1, t2));
  v[1] = cadd(m1, d1);
  v[4] = csub(m1, d1);
  v[2] = cadd(m2, d2);
  v[3] = csub(m2, d2);
}
// 16 points as 4 x 4: for each r2 a size-4 DFT over r1 of v[4 r1 + r2],
// times W16^(r2 k1), then for each k1 a size-4 DFT over r2; output k1 + 4 k2.
// W16^q = exp(-2 pi i q / 16) for the q = r2 k1 that occur (conjugated for
// the inverse).
template <typename T>
__device__ __forceinline__ void dft16(Cx<T>* v, T s) {
  const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173;  // cos, sin (pi / 8)
  const T h = (T)0.70710678118654752440;                                   // cos (pi / 4)
  Cx<T> t[16];
#pragma unroll
  for (int r2 = 0; r2 < 4; ++r2) {
    Cx<T> a[4] = {v[r2], v[4 + r2], v[8 + r2], v[12 + r2]};
    dft4(a, s);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) t[4 * r2 + k1] = a[k1];
  }
  // W16^(r2 k1): (1), (r2 = 1) q = 1, 2, 3; (r2 = 2) q = 2, 4, 6; (r2 = 3) q = 3, 6, 9
  const Cx<T> w1 = Cx<T>{c1, s * s1}, w2 = Cx<T>{h, s * h}, w3 = Cx<T>{s1, s * c1};
  const Cx<T> w6 = Cx<T>{-h, s * h}, w9 = Cx<T>{-c1, -s * s1};
  t[5] = cmul(t[5], w1);
  t[6] = cmul(t[6], w2);
  t[7] = cmul(t[7], w3);
  t[9] = cmul(t[9], w2);
  t[10] = cmuli(t[10], s);  // W16^4 = s i
  t[11] = cmul(t[11], w6);
  t[13] = cmul(t[13], w3);
  t[14] = cmul(t[14], w6);
  t[15] = cmul(t[15], w9);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    Cx<T> a[4] = {t[k1], t[4 + k1], t[8 + k1], t[12 + k1]};
    dft4(a, s);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = a[k2];
  }
}
// a prime radix R by the definition: V_k = sum_r v_r z^(r k mod R), z the
// R-th roots of unity in root[0..R-1] (conjugated for the inverse)
template <typename T, int R>
__device__ __forceinline__ void dft_prime(Cx<T>* v, const Cx<T>* root, T s) {
  Cx<T> o[R];
#pragma unroll
  for (int k = 0; k < R; ++k) {
    Cx<T> acc = v[0];
#pragma unroll
    for (int r = 1; r < R; ++r) acc = cadd(acc, cmul(v[r], conj_if(root[(r * k) % R], s)));
    o[k] = acc;
  }
#pragma unroll
  for (int k = 0; k < R; ++k) v[k] = o[k];
}

// Element e of a line sits at e + e / 16 (one spare slot after every 16
// complex values, 128 bytes): a warp's strided Stockham writes, 16 j + r for a
// radix-16 stage or 4 j + r for a radix-4 one, then fall on distinct bank
// pairs instead of one or four.
__host__ __device__ __forceinline__ int pad(int e) { return e + (e >> 4); }

// One Stockham stage of radix R over the L lines of X into Y (line pitch P):
// butterfly j = g Ns + k of a line reads X[j + r m] (m = n / R), multiplies
// element r by w^(r k) (w = exp(-2 pi i / (Ns R)), from the stage's table
// ws[(r - 1) Ns + k]), applies the size-R DFT and writes Y[g Ns R + k + r Ns].
// Ns = cNs 2^sNs; m = cm 2^sm (cNs, cm odd); the block's L = 2^sL lines.
template <typename T, int R>
__device__ __forceinline__ void fft_stage(const Cx<T>* X, Cx<T>* Y, int sL, int n, int P, int sNs, int cNs, int cm,
                                          int sm, const Cx<T>* ws, const Cx<T>* root, T s) {
  const int m = n / R, Ns = cNs << sNs;
  for (int b = threadIdx.x; b < (m << sL); b += blockDim.x) {
    const int line = div_c(b >> sm, cm), j = b - line * m;
    const int g = div_c(j >> sNs, cNs), k = j - g * Ns;
    const Cx<T>* x = X + line * P;
    Cx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = x[pad(j + r * m)];
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(v[r], conj_if(ws[(r - 1) * Ns + k], s));
    }
    if (R == 16) dft16(v, s);
    else if (R == 4) dft4(v, s);
    else if (R == 2) dft2(v);
    else if (R == 3) dft3(v, s);
    else if (R == 5) dft5(v, s);
    else dft_prime<T, R>(v, root, s);
    Cx<T>* y = Y + line * P;
    const int o = g * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) y[pad(o + r * Ns)] = v[r];
  }
}

// Transforms the 2^sL lines held in X (line l at X + l P) with Y as scratch,
// all threads of the block; returns the buffer holding the result.  w: the
// axis's stage tables (stage with Ns at w + Ns - 1) and its roots at w + n - 1.
template <typename T>
__device__ __forceinline__ Cx<T>* fft_lines(Cx<T>* X, Cx<T>* Y, int sL, int P, int n, int c, int sn, int nst,
                                            unsigned long long radix_code, const Cx<T>* w, T s) {
  const Cx<T>* root = w + n - 1;
  int sNs = 0, cNs = 1;  // the sub-transform size so far, Ns = cNs 2^sNs
#pragma unroll 1
  for (int st = 0; st < nst; ++st) {
    const int R = (int)((radix_code >> (5 * st)) & 31u);
    const Cx<T>* ws = w + (cNs << sNs) - 1;
    // m = n / R = cm 2^sm: c 2^(sn-4), c 2^(sn-2), c 2^(sn-1), or (c / R) 2^sn for an odd radix
    switch (R) {
      case 16: fft_stage<T, 16>(X, Y, sL, n, P, sNs, cNs, c, sn - 4, ws, root, s); sNs += 4; break;
      case 4: fft_stage<T, 4>(X, Y, sL, n, P, sNs, cNs, c, sn - 2, ws, root, s); sNs += 2; break;
      case 2: fft_stage<T, 2>(X, Y, sL, n, P, sNs, cNs, c, sn - 1, ws, root, s); sNs += 1; break;
      case 3: fft_stage<T, 3>(X, Y, sL, n, P, sNs, cNs, c / 3, sn, ws, root, s); cNs *= 3; break;
      case 5: fft_stage<T, 5>(X, Y, sL, n, P, sNs, cNs, c / 5, sn, ws, root, s); cNs *= 5; break;
      default: fft_stage<T, 7>(X, Y, sL, n, P, sNs, cNs, c / 7, sn, ws, root, s); cNs *= 7; break;
    }
    __syncthreads();
    Cx<T>* t = X;
    X = Y;
    Y = t;
  }
  return X;
}

// Arguments of one pass over one level's grid.
template <typename T>
struct FftPassArgs {
  int n[3];
  int axis;              // 0 (x), 1 (y), 2 (z)
  int sL;                // lines per block L = 2^sL
  int groups_per_row;    // axis 1, 2: x-groups of L lines per row of the other dimension
  FftAxisDesc D;
  const Cx<T>* tw;       // this axis's stage tables and roots (n - 1 + kRoots entries)
  Cx<T>* buf;            // the level's complex grid
  const double* qin;     // x forward: the FP64 charges (real input)
  T* uout;               // x inverse: the potential (real output)
  const T* khat;         // z pass: the kernel's transform (real), scaled
};

// Line pitch in shared memory: the padded line, made odd, so that the L lines
// of a y or z pass, loaded one grid row segment at a time, fall in distinct
// banks.
__host__ __device__ __forceinline__ int line_pitch(int n) { return (pad(n - 1) + 1) | 1; }

// MODE: 0 x forward from real FP64 input, 1 forward (any axis), 2 z forward
// x K^ x z inverse, 3 inverse (y), 4 x inverse to real output.  The block's
// descriptor fields are read once into registers.
template <typename T, int MODE>
__device__ __forceinline__ void fft_pass_body(const FftPassArgs<T>* __restrict__ Ap, int blk) {
  extern __shared__ __align__(16) unsigned char fft_smem[];
  const int ax = Ap->axis, sL = Ap->sL, gpr = Ap->groups_per_row;
  const int n0 = Ap->n[0], n1 = Ap->n[1], n2 = Ap->n[2];
  const int n = Ap->D.n, c = Ap->D.c, sn = Ap->D.s, nst = Ap->D.nst;
  const unsigned long long radix_code = Ap->D.radix_code;
  const Cx<T>* tw = Ap->tw;
  Cx<T>* buf = Ap->buf;
  const int L = 1 << sL, P = line_pitch(n);
  Cx<T>* X = reinterpret_cast<Cx<T>*>(fft_smem);
  Cx<T>* Y = X + L * P;
  Cx<T>* w = Y + L * P;
  for (int i = threadIdx.x; i < n - 1 + kRoots; i += blockDim.x) w[i] = tw[i];
  // the block's lines: element e of line l at global offset base + l * ls + e * es
  long long base, ls, es;
  int nl;  // valid lines
  if (ax == 0) {
    base = (long long)blk * L * n0;
    ls = n0;
    es = 1;
    nl = min(L, n1 * n2 - blk * L);
  } else {
    const int g = blk % gpr, other = blk / gpr;  // other: z (axis 1) or y (axis 2)
    const int x0 = g * L;
    nl = min(L, n0 - x0);
    ls = 1;
    if (ax == 1) {
      base = (long long)other * n1 * n0 + x0;
      es = n0;
    } else {
      base = (long long)other * n0 + x0;
      es = (long long)n0 * n1;
    }
  }
  // load (consecutive threads on consecutive global addresses): axis 0 takes
  // t = l n + e, the others t = e L + l; kFftBatch loads per thread are issued
  // before their shared-memory stores, so that they are in flight together
  const int total = n << sL;
  for (int t0 = threadIdx.x; t0 < total; t0 += kFftBatch * blockDim.x) {
    Cx<T> v[kFftBatch];
    int at[kFftBatch];
#pragma unroll
    for (int u = 0; u < kFftBatch; ++u) {
      const int t = t0 + u * (int)blockDim.x;
      v[u] = Cx<T>{T(0), T(0)};
      at[u] = -1;
      if (t < total) {
        int l, e;
        if (ax == 0) {
          l = div_c(t >> sn, c);
          e = t - l * n;
        } else {
          e = t >> sL;
          l = t & (L - 1);
        }
        at[u] = l * P + pad(e);
        if (l < nl) {
          const long long o = base + l * ls + e * es;
          if (MODE == 0) v[u].x = (T)Ap->qin[o];
          else v[u] = buf[o];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kFftBatch; ++u)
      if (at[u] >= 0) X[at[u]] = v[u];
  }
  __syncthreads();
  const T s = (MODE == 3 || MODE == 4) ? T(1) : T(-1);
  Cx<T>* R = fft_lines(X, Y, sL, P, n, c, sn, nst, radix_code, w, s);
  if (MODE == 2) {  // product by K^ at this line's points, then the inverse along z
    const T* khat = Ap->khat;
    for (int t0 = threadIdx.x; t0 < total; t0 += kFftBatch * blockDim.x) {
      T kh[kFftBatch];
#pragma unroll
      for (int u = 0; u < kFftBatch; ++u) {
        const int t = t0 + u * (int)blockDim.x, e = t >> sL, l = t & (L - 1);
        kh[u] = (t < total && l < nl) ? khat[base + l * ls + e * es] : T(0);
      }
#pragma unroll
      for (int u = 0; u < kFftBatch; ++u) {
        const int t = t0 + u * (int)blockDim.x, e = t >> sL, l = t & (L - 1);
        if (t < total && l < nl) {
          R[l * P + pad(e)].x *= kh[u];
          R[l * P + pad(e)].y *= kh[u];
        }
      }
    }
    __syncthreads();
    R = fft_lines(R, R == X ? Y : X, sL, P, n, c, sn, nst, radix_code, w, T(1));
  }
  T* uout = Ap->uout;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    int l, e;
    if (ax == 0) {
      l = div_c(t >> sn, c);
      e = t - l * n;
    } else {
      e = t >> sL;
      l = t & (L - 1);
    }
    if (l < nl) {
      const long long o = base + l * ls + e * es;
      if (MODE == 4) uout[o] = R[l * P + pad(e)].x;
      else buf[o] = R[l * P + pad(e)];
    }
  }
}

// One pass over a table of levels (one plan's, or every replica's): block b
// belongs to the item whose range of blocks holds it.
template <typename T, int MODE>
__global__ void __launch_bounds__(kFftThreads, sizeof(T) == 4 ? 4 : 2) k_fft_pass(const FftPassArgs<T>* __restrict__ tab,
                                                          const int* __restrict__ first, int nitems) {
  const int r = batch_rep(first, nitems, blockIdx.x);
  fft_pass_body<T, MODE>(tab + r, (int)blockIdx.x - __ldg(first + r));
}

// n = c 2^s with c a product of 3, 5 and 7: stages radix 16 (while 16
// divides the power of two, with radix16: the FP32 form, whose 16 values a
// thread keeps in registers), radix 4 (while 4 divides what is left), one
// radix 2 if one factor 2 is left, then the factors of c (3s, 5s, 7s).
// Returns false for any other n or more than 12 stages.
bool factorize(int n, FftAxisDesc& D, bool radix16) {
  D = FftAxisDesc{n, 1, 0, 0, 0ull};
  if (n < 1) return false;
  int p = n;
  while ((p & 1) == 0) {
    p >>= 1;
    D.s++;
  }
  D.c = p;
  int s = D.s;
  auto push = [&](int r) {
    if (D.nst < 12) D.radix_code |= (unsigned long long)r << (5 * D.nst);
    D.nst++;
  };
  if (radix16)
    for (; s >= 4; s -= 4) push(16);
  for (; s >= 2; s -= 2) push(4);
  if (s == 1) push(2);
  for (int r : {3, 5, 7})
    while (p % r == 0) {
      push(r);
      p /= r;
    }
  return p == 1 && D.nst <= 12;
}

// Lines per block: the largest power of two up to 16 whose two line buffers
// stay within the shared-memory budget (at least one line); returns log2.
template <typename T>
int lines_per_block_log2(int n) {
  const size_t per = 2 * (size_t)line_pitch(n) * sizeof(Cx<T>);
  int sL = 4;
  while (sL > 0 && ((size_t)1 << sL) * per > kFftSmem) --sL;
  return sL;
}

template <typename T>
size_t pass_smem(int n, int sL) {
  return (2 * ((size_t)1 << sL) * line_pitch(n) + n - 1 + kRoots) * sizeof(Cx<T>);
}

template <typename T>
FftPassArgs<T> pass_args(const int dims[3], int axis, const void* tw, void* buf, const void* khat) {
  FftPassArgs<T> A;
  for (int d = 0; d < 3; ++d) A.n[d] = dims[d];
  const int n = dims[axis];
  A.axis = axis;
  A.sL = lines_per_block_log2<T>(n);
  A.groups_per_row = (dims[0] + (1 << A.sL) - 1) >> A.sL;
  factorize(n, A.D, sizeof(T) == sizeof(float));
  A.tw = reinterpret_cast<const Cx<T>*>(tw);
  A.buf = reinterpret_cast<Cx<T>*>(buf);
  A.qin = nullptr;
  A.uout = nullptr;
  A.khat = reinterpret_cast<const T*>(khat);
  return A;
}

template <typename T>
int pass_blocks(const FftPassArgs<T>& A) {
  if (A.axis == 0) return (A.n[1] * A.n[2] + (1 << A.sL) - 1) >> A.sL;
  const int other = A.axis == 1 ? A.n[2] : A.n[1];
  return A.groups_per_row * other;
}

template <typename T, int MODE>
void run_pass(const BatchTable<FftPassArgs<T>>& t, cudaStream_t st) {
  if (t.total > 0) k_fft_pass<T, MODE><<<t.total, kFftThreads, t.smem, st>>>(t.args, t.first, t.nrep);
}

// The twiddle table of one axis of length n, FP64: the stage tables
// exp(-2 pi i r k / (Ns R)) at (Ns - 1) + (r - 1) Ns + k, then the seventh
// roots of unity exp(-2 pi i q / 7).
std::vector<double> twiddles(int n, bool radix16) {
  FftAxisDesc D;
  factorize(n, D, radix16);
  std::vector<double> tw(2 * (size_t)(n - 1 + kRoots), 0.0);
  int Ns = 1;
  for (int st = 0; st < D.nst; ++st) {
    const int R = (int)((D.radix_code >> (5 * st)) & 31u);
    for (int r = 1; r < R; ++r)
      for (int k = 0; k < Ns; ++k) {
        const size_t i = (size_t)(Ns - 1) + (size_t)(r - 1) * Ns + k;
        const double a = -2.0 * M_PI * (double)(r * k) / (double)(Ns * R);
        tw[2 * i] = std::cos(a);
        tw[2 * i + 1] = std::sin(a);
      }
    Ns *= R;
  }
  for (int q = 0; q < kRoots; ++q) {
    const size_t i = (size_t)(n - 1) + q;
    tw[2 * i] = std::cos(-2.0 * M_PI * q / kRoots);
    tw[2 * i + 1] = std::sin(-2.0 * M_PI * q / kRoots);
  }
  return tw;
}

// The kernel's transform, FP64: the real part of the forward transform of
// the folded kernel, times scale (the level factor and 1/N).
__global__ void k_take_real(const Cx<double>* __restrict__ src, double scale, float* __restrict__ dstf,
                            double* __restrict__ dstd, int64_t count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const double v = scale * src[i].x;
  if (dstf) dstf[i] = (float)v;
  if (dstd) dstd[i] = v;
}

}  // namespace

struct FftBatch {
  bool fp64 = false;
  BatchTable<FftPassArgs<float>> f[5];
  BatchTable<FftPassArgs<double>> d[5];
};

template <typename T>
static cudaError_t set_pass_attributes() {
  cudaError_t e = cudaSuccess;
  auto set = [&](const void* f) {
    const cudaError_t r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (r != cudaSuccess) e = r;
  };
  set((const void*)k_fft_pass<T, 0>);
  set((const void*)k_fft_pass<T, 1>);
  set((const void*)k_fft_pass<T, 2>);
  set((const void*)k_fft_pass<T, 3>);
  set((const void*)k_fft_pass<T, 4>);
  return e;
}

cudaError_t configure_fft_kernels() {
  cudaError_t e = set_pass_attributes<float>();
  if (e == cudaSuccess) e = set_pass_attributes<double>();
  return e;
}

bool fft_size_ok(int n) {
  FftAxisDesc D;
  return n <= 4096 && factorize(n, D, false) && factorize(n, D, true);
}

// Builds level k's tables: twiddles per axis (in the plan's precision) and
// K^ from the host kernel grid K (FP64, folded, M0 x M1 x M2, x fastest),
// computed with FP64 passes in work (16 bytes per point of the level).
cudaError_t fft_build_level(Plan& P, int k, const std::vector<double>& K, void* work) {
  FftLevel& F = P.fftl[k];
  for (int d = 0; d < 3; ++d) F.n[d] = P.n[k][d];
  const int64_t N = (int64_t)F.n[0] * F.n[1] * F.n[2];
  cudaError_t e = cudaSuccess;
  void* tw64[3] = {nullptr, nullptr, nullptr};
  for (int d = 0; d < 3 && e == cudaSuccess; ++d) {
    // FP64 passes (K^ here, and the FP64 plan's) take radix 4 at most; the
    // FP32 form also radix 16, with its own stage tables
    const std::vector<double> tw = twiddles(F.n[d], false);
    e = cudaMalloc(&tw64[d], sizeof(double) * tw.size());
    if (e == cudaSuccess) e = cudaMemcpy(tw64[d], tw.data(), sizeof(double) * tw.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) break;
    if (P.fp64) {
      e = cudaMalloc(&F.tw[d], sizeof(double) * tw.size());
      if (e == cudaSuccess) e = cudaMemcpy(F.tw[d], tw.data(), sizeof(double) * tw.size(), cudaMemcpyHostToDevice);
    } else {
      const std::vector<double> tw16 = twiddles(F.n[d], true);
      const std::vector<float> twf(tw16.begin(), tw16.end());
      e = cudaMalloc(&F.tw[d], sizeof(float) * twf.size());
      if (e == cudaSuccess) e = cudaMemcpy(F.tw[d], twf.data(), sizeof(float) * twf.size(), cudaMemcpyHostToDevice);
    }
  }
  if (e == cudaSuccess) e = cudaMalloc(&F.khat, (P.fp64 ? sizeof(double) : sizeof(float)) * (size_t)N);
  double* kd = nullptr;
  if (e == cudaSuccess) e = cudaMalloc((void**)&kd, sizeof(double) * (size_t)N);
  if (e == cudaSuccess) e = cudaMemcpy(kd, K.data(), sizeof(double) * (size_t)N, cudaMemcpyHostToDevice);
  BatchTable<FftPassArgs<double>> t[3];
  for (int d = 0; d < 3 && e == cudaSuccess; ++d) {  // forward along x (real input), y, z
    FftPassArgs<double> A = pass_args<double>(F.n, d, tw64[d], work, nullptr);
    if (d == 0) A.qin = kd;
    e = make_table(t[d], std::vector<FftPassArgs<double>>{A}, std::vector<int>{pass_blocks(A)},
                   pass_smem<double>(F.n[d], A.sL));
  }
  if (e == cudaSuccess) {
    run_pass<double, 0>(t[0], 0);
    run_pass<double, 1>(t[1], 0);
    run_pass<double, 1>(t[2], 0);
    const double scale = std::ldexp(1.0, -k) / (double)N;
    k_take_real<<<(unsigned)((N + 255) / 256), 256>>>((const Cx<double>*)work, scale,
                                                      P.fp64 ? nullptr : (float*)F.khat,
                                                      P.fp64 ? (double*)F.khat : nullptr, N);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  for (auto& x : t) x.release();
  if (kd) cudaFree(kd);
  for (int d = 0; d < 3; ++d)
    if (tw64[d]) cudaFree(tw64[d]);
  return e;
}

void fft_free_level(FftLevel& F) {
  for (int d = 0; d < 3; ++d)
    if (F.tw[d]) cudaFree(F.tw[d]);
  if (F.khat) cudaFree(F.khat);
  F = FftLevel();
}

template <typename T>
static cudaError_t build_tables(const std::vector<FftBatchItem>& items, BatchTable<FftPassArgs<T>>* tab) {
  const int axis_of[5] = {0, 1, 2, 1, 0};
  cudaError_t e = cudaSuccess;
  for (int p = 0; p < 5 && e == cudaSuccess; ++p) {
    std::vector<FftPassArgs<T>> args;
    std::vector<int> blocks;
    size_t sm = 0;
    for (const FftBatchItem& it : items) {
      const int ax = axis_of[p];
      FftPassArgs<T> A = pass_args<T>(it.F->n, ax, it.F->tw[ax], it.work, it.F->khat);
      if (p == 0) A.qin = it.q;
      if (p == 4) A.uout = (T*)it.u;
      args.push_back(A);
      blocks.push_back(pass_blocks(A));
      sm = std::max(sm, pass_smem<T>(A.D.n, A.sL));
    }
    e = make_table(tab[p], args, blocks, sm);
  }
  return e;
}

cudaError_t fft_batch_build(const std::vector<FftBatchItem>& items, bool fp64, FftBatch** out) {
  *out = nullptr;
  FftBatch* b = new (std::nothrow) FftBatch();
  if (!b) return cudaErrorMemoryAllocation;
  b->fp64 = fp64;
  const cudaError_t e = fp64 ? build_tables<double>(items, b->d) : build_tables<float>(items, b->f);
  if (e != cudaSuccess) {
    fft_batch_free(b);
    return e;
  }
  *out = b;
  return cudaSuccess;
}

template <typename T>
static void launch_tables(const BatchTable<FftPassArgs<T>>* t, cudaStream_t st) {
  run_pass<T, 0>(t[0], st);
  run_pass<T, 1>(t[1], st);
  run_pass<T, 2>(t[2], st);
  run_pass<T, 3>(t[3], st);
  run_pass<T, 4>(t[4], st);
}

cudaError_t fft_batch_launch(const FftBatch* b, cudaStream_t st) {
  if (b->fp64) launch_tables<double>(b->d, st);
  else launch_tables<float>(b->f, st);
  return cudaGetLastError();
}

void fft_batch_free(FftBatch* b) {
  if (!b) return;
  for (auto& t : b->f) t.release();
  for (auto& t : b->d) t.release();
  delete b;
}

}  // namespace msm
