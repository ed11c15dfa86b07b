// msm_internal.h -- plan layout and kernel launchers of the GB300 MSM library.
// Not part of the public ABI (include/msm.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/msm.h"

namespace msm {

constexpr int kMaxLevels = 16;
constexpr int kSeg = 8;           // taps per stencil segment (x direction)
constexpr int kMaxCellOffsets = 125;

// Status bits posted by kernels (atomicOr) and decoded by msm_status.
constexpr int kStatusOutside = 1;
constexpr int kStatusNonfinite = 2;
constexpr int kStatusTimeout = 4;

template <typename T>
struct alignas(4 * sizeof(T)) R4 {
  T x, y, z, w;
};

// One x-run of the level stencil: taps (dx0 + j, dy, dz), j = 0..kSeg-1,
// with coefficients g[j] (zero past the end of the run).
template <typename T>
struct Segment {
  int dy, dx0;
  T g[kSeg];
};

// A run over two adjacent stencil rows, for packed FP32x2 FMAs: g[j] =
// (tap (dx0 + j, dy, dz), tap (dx0 + j, dy - 1, dz)), the coefficients that
// one input row applies to the two output rows y and y + 1 it feeds.
struct alignas(16) Segment2 {
  float2 g[kSeg];  // first, so that it loads as four 16-byte words
  int dy, dx0;
};

// Per-precision device tables and buffers.
struct DeviceBuffers {
  // binning / sorting
  int* key = nullptr;          // [cap]  cell of each atom (input order)
  int* rank = nullptr;         // [cap]  its place inside the cell
  int* perm = nullptr;         // [cap]  sorted slot -> input index
  int* count = nullptr;        // [ncell] atoms per cell (zero between evaluations)
  int* csum = nullptr;         // [ncell / 4096 + 1] per-chunk sums of count
  int* cell_start = nullptr;   // [ncell + 1]
  // sorted atoms (type T = float or double, selected by precision)
  void* atoms = nullptr;       // R4<T>[cap]: cell-local x, y, z and q
  void* gfrac = nullptr;       // R4<T>[cap]: fractional grid offsets (0..1) and q
  int4* gbase = nullptr;       // [cap]: first level-0 index of the basis support per dim
  // per-atom results in sorted order
  void* phis = nullptr;        // T[cap]  short-range potential
  void* fs = nullptr;          // R4<T>[cap] short-range force (x, y, z), spare (w)
  void* glong = nullptr;       // R4<T>[cap] long-range gradient (x, y, z) and long-range potential (w)
  // grids, one per level: charges q^k in FP64, potentials u^k in T
  void* gq[kMaxLevels] = {};
  void* gu[kMaxLevels] = {};
  // adjoint grids
  void* aq[kMaxLevels] = {};
  void* au[kMaxLevels] = {};
  // lattice partial sums of levels split over several blocks: [nsplit][points] in T
  void* lparts = nullptr;
  // complex work grid of the FFT lattice (the largest convolved level, FP64 complex)
  void* fft_work = nullptr;
  // separable restriction / prolongation temporaries (each as large as level 0, in doubles)
  void* tmp[2] = {nullptr, nullptr};
  // top level (always FP64)
  double* topK = nullptr;      // periodic: [M^3] circulant; open: [(2M-1)^3] Toeplitz
  double* topq = nullptr;
  double* topu = nullptr;
  // level stencil
  void* seg = nullptr;         // Segment<T>[nseg]
  void* seg2 = nullptr;        // Segment2[nseg] (mixed precision only, instead of seg)
  int* seg_start = nullptr;    // [2*Ez+2]: segments of plane dz live in [start[dz+Ez], start[dz+Ez+1])
  // neighbour cell offsets (x, y, z) of the pair kernel
  int4* cell_off = nullptr;    // [noff]
  void* cell_shift = nullptr;  // R4<T>[noff]: offset times cell width, in the plan's precision
  int4* cell_rows = nullptr;   // [nrows]: (dy, dz, xlo, xhi) rows of neighbour cell offsets
  // reductions and status
  double* partial = nullptr;   // per-block energy partials
  double* scalars = nullptr;   // [8] scratch scalars (0: backward scale; 1, 2..7: MD energy and record when none is kept)
  double* md_partial = nullptr;  // [4 * kMdBlocks] per-block kinetic energy and momentum of the MD loop
  int* md_step = nullptr;        // [1] record counter of MD steps replayed from a graph
  int* status = nullptr;
  // host-path staging (msm_eval_host)
  double* hpos = nullptr;
  double* hq = nullptr;
  double* hphi = nullptr;
  double* hforce = nullptr;
  double* henergy = nullptr;
  int* hstatus = nullptr;  // pinned host copy of the status word, read after the call's one sync
};

// The lattice cutoff of one periodic level as an FFT convolution (fft.cu):
// the level's dimensions, twiddle tables per axis and the kernel's transform
// (real, with the level factor 2^-k and the inverse's 1/N), in the plan's
// precision.
struct FftLevel {
  int n[3] = {0, 0, 0};
  void* tw[3] = {nullptr, nullptr, nullptr};
  void* khat = nullptr;
};
// The five passes' argument tables over a list of levels (fft.cu).
struct FftBatch;

struct Plan {
  msm_params P;
  bool fp64 = false;
  int S = 2, W = 4;            // basis half support, taps per dimension
  int levels = 1;
  double h[3];                 // finest spacing
  int lo[kMaxLevels][3];
  int n[kMaxLevels][3];
  // short-range cells
  int nc[3];
  double cw[3];
  int ncell = 1;
  int noff = 0;
  int nrows = 0;
  // anterpolation patches: blocks of ablk^3 cells, patches of apd^3 points
  int ablk = 1, apd = 1;
  int ablk_batch = 1, apd_batch = 1;  // the same for the batched launches (at least as large)
  // lattice: blocks per SM to aim for when splitting a small level's planes,
  // and the warp tile of the FP32 kernel (0 x 0: the default)
  int lattice_waves = 8;
  int lattice_txn = 0, lattice_tyn = 0;
  // mixed pair kernel: targets culled together (8: clusters; 32: a cell's warp)
  int pair_targets = 32;
  // mixed pair kernel: targets in runs of 32 consecutive sorted atoms (true) or one cell per warp
  bool pair_runs = false;
  // batched graphs: restriction and prolongation chains as persistent launches
  int batch_persistent = 0;
  // lattice cutoff of periodic levels as an FFT convolution (fft.cu)
  bool lattice_fft = false;
  bool stencil_fits = true;  // the stencil kernel's shared-memory window holds this plan's stencil
  int64_t tmp_elems = 0;     // FP64 elements of each of the two temporaries tmp[0], tmp[1]
  FftLevel fftl[kMaxLevels];
  FftBatch* fftb[2] = {nullptr, nullptr};  // every lattice level: the forward sweep's grids, the adjoint's
  // smoothing constants
  double gamma0 = 0.0;         // gamma(0)
  // level stencil
  int E[3] = {0, 0, 0};        // largest |dx|, |dy|, |dz| of a tap
  int nseg = 0;
  double stencil_taps = 0.0;   // number of taps (for work accounting)
  // top level
  int top_table_dims[3];
  // workspace
  int64_t cap = 0;
  int nblk_partial = 0;
  DeviceBuffers d;
  // concurrency: the grid passes of a forward evaluation run on `side` (a
  // plan-owned stream of the highest priority) while the pair sums run on the
  // caller's stream; fork and join are event waits
  bool overlap = true;
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // state
  cudaStream_t last_stream = nullptr;
  int64_t last_n = -1;
  // id of the forward pass whose per-atom terms the buffers hold (0: none);
  // every forward, and every replay of a captured forward, takes the next id
  int64_t forward_id = 0;
  int64_t next_id = 0;
  // damping of Wolf summation when it is the MD force (msm_set_wolf_alpha)
  double wolf_alpha = 0.0;
  int host_status = 0;
  // diagnostics: stage event pairs (pool reused across reads), launch count
  struct StageRec {
    int stage;
    cudaEvent_t a, b;
  };
  bool profiling = false;
  std::vector<StageRec> recs;
  size_t nrec = 0;
  int64_t launches = 0;
  int64_t evals = 0;
};

// ---- batches of independent systems (one launch per stage over all replicas) ----
// A batched launch numbers the blocks of all replicas consecutively; first[r]
// is the first block of replica r (first[nrep] = total) and every block finds
// its replica by binary search and reads that replica's kernel arguments from
// a table in device memory.
#ifdef __CUDACC__
__device__ __forceinline__ int batch_rep(const int* __restrict__ first, int nrep, int b) {
  int lo = 0, hi = nrep - 1;  // largest r with first[r] <= b (replicas without blocks are skipped)
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(first + mid) <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}
#endif

// A table of per-replica kernel arguments and block offsets in device memory.
template <typename A>
struct BatchTable {
  A* args = nullptr;
  int* first = nullptr;
  int nrep = 0;
  int total = 0;       // blocks over all replicas
  size_t smem = 0;     // dynamic shared memory per block (the largest over the replicas)
  void release() {
    if (args) cudaFree(args);
    if (first) cudaFree(first);
    args = nullptr;
    first = nullptr;
  }
};

// Uploads per-replica arguments and block counts (synchronous; batch set-up only).
template <typename A>
cudaError_t make_table(BatchTable<A>& t, const std::vector<A>& args, const std::vector<int>& blocks, size_t smem = 0) {
  t.release();
  t.nrep = (int)args.size();
  std::vector<int> first(args.size() + 1, 0);
  for (size_t r = 0; r < args.size(); ++r) first[r + 1] = first[r] + blocks[r];
  t.total = first.back();
  t.smem = smem;
  cudaError_t e = cudaMalloc((void**)&t.args, sizeof(A) * (args.empty() ? 1 : args.size()));
  if (e == cudaSuccess) e = cudaMalloc((void**)&t.first, sizeof(int) * first.size());
  if (e == cudaSuccess && !args.empty()) e = cudaMemcpy(t.args, args.data(), sizeof(A) * args.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(t.first, first.data(), sizeof(int) * first.size(), cudaMemcpyHostToDevice);
  return e;
}

// One replica of a batch: its plan and its slices of the caller's arrays
// (device pointers; outputs may be NULL where the batch entry point allows).
struct BatchRep {
  Plan* plan;
  int64_t n;
  const double* pos;
  const double* q;
  double* energy;
  double* phi;
  double* force;
  const double* grad_energy;
  double* grad_pos;
  double* grad_q;
};

// Batched stages, each a set of launches over all replicas on one stream.
// build() uploads the tables (synchronous, allocates); launch() only
// enqueues kernels.  The replicas must be mixed-precision plans of one
// interpolation order and one splitting.
struct BinBatch;
struct PairBatch;
struct GridBatch;
cudaError_t bin_batch_build(const std::vector<BatchRep>& reps, BinBatch** out);
cudaError_t bin_batch_launch(BinBatch* b, cudaStream_t st);
void bin_batch_free(BinBatch* b);
cudaError_t pair_batch_build(const std::vector<BatchRep>& reps, PairBatch** out);
cudaError_t pair_batch_launch(PairBatch* b, cudaStream_t st);
void pair_batch_free(PairBatch* b);
// The grid passes: anterpolation and the sweep through the levels, then
// interpolation with assembly (forward: phi, F and the energies; backward,
// built only when every replica has grad_energy: dL/dq and dL/dr).
cudaError_t grid_batch_build(const std::vector<BatchRep>& reps, bool backward, GridBatch** out);
// The sweep in two parts: the front (anterpolation into the fixed-point
// grids and their conversion to the level-0 charges of the forward and, with
// backward, of the adjoint) and the level chain of one direction
// (restriction, lattice cutoff, top level, prolongation).  The adjoint's
// chain has its own temporaries, so it may run concurrently with the
// forward's unless the chains are persistent (one grid barrier word).
cudaError_t grid_batch_front(GridBatch* b, bool backward, cudaStream_t st);
cudaError_t grid_batch_levels(GridBatch* b, int dir, cudaStream_t st);
bool grid_batch_persistent(const GridBatch* b);
cudaError_t grid_batch_interp(GridBatch* b, bool backward, cudaStream_t st);
void grid_batch_free(GridBatch* b);

// ---- host helpers (plan.cpp) ----
int validate_params(const msm_params* p);  // host only, no CUDA calls
int plan_geometry(const msm_params* p, Plan* P);  // validation and grid geometry only (host, no CUDA calls)
int validate_tuning(const msm_tuning* t);  // host only, no CUDA calls
int build_plan(const msm_params* p, const msm_tuning* t, Plan* plan);
void free_plan(Plan* plan);
int64_t grid_points(const Plan& P, int k);

// ---- launchers (.cu files); all asynchronous on stream ----
// binning: keys, stable radix sort by cell, cell_start, gather of sorted atoms
template <typename IO>  // IO = double or float (caller's position and charge type)
cudaError_t launch_binning(Plan& P, int64_t n, const IO* pos, const IO* q, cudaStream_t s);
// short-range pair sums (phis, fs.xyz)
cudaError_t launch_short_range(Plan& P, int64_t n, cudaStream_t s);
// the cutoff method: Coulomb pair sums within the cutoff (phis, fs.xyz); Wolf
// summation: its damped shifted-force pair sums; and the assembly of phi
// (minus self_c q_i: 0 for the cutoff method, 2 c_s for Wolf), F and E
cudaError_t launch_cutoff_pairs(Plan& P, int64_t n, cudaStream_t s);
cudaError_t launch_wolf_pairs(Plan& P, int64_t n, double alpha, cudaStream_t s);
template <typename OUT>
cudaError_t launch_cutoff_assemble(Plan& P, int64_t n, double* energy, OUT* phi, OUT* force, cudaStream_t s,
                                   double self_c = 0.0);
// grid passes: anterpolation (charges q_i * scale, scale from device or 1)
cudaError_t launch_anterpolate(Plan& P, int64_t n, void* grid0, const double* dscale, double factor,
                               cudaStream_t s);
// the adjoint's level-0 charges: factor * dscale[0] times the forward's
cudaError_t launch_scale_grid(Plan& P, const void* src, void* dst, const double* dscale, double factor,
                              cudaStream_t s);
cudaError_t launch_restrict(Plan& P, int k, const void* fine, void* coarse, cudaStream_t s);
// Velocity Verlet around the MSM force: the two half steps of one MD step
// and the per-step record (potential, kinetic, total energy, momentum).
constexpr int kMdBlocks = 1024;  // blocks (and partials) of the MD kernels
cudaError_t launch_md_drift(Plan& P, int64_t n, double* pos, double* vel, const double* force,
                            const double* inv_mass, double dt, cudaStream_t s);
// counter: NULL, or a device step counter that places the record at
// record + 6 * counter and advances (steps replayed from a graph)
cudaError_t launch_md_kick(Plan& P, int64_t n, double* vel, const double* force, const double* inv_mass, double dt,
                           const double* potential, double* record, int* counter, cudaStream_t s);
// The parareal correction of one time point (uses P's box and MD partials):
// lam = gnew + (f - g), g = gnew, change[0..1] = largest position and
// velocity change of lam against its previous value.
cudaError_t launch_parareal_correct(Plan& P, int64_t n, const double* gnew_pos, const double* gnew_vel,
                                    const double* f_pos, const double* f_vel, double* g_pos, double* g_vel,
                                    double* lam_pos, double* lam_vel, double* change, cudaStream_t s);

// Whether the level stencil's window fits the lattice kernel's shared memory
// (a stencil of half-width E holds about (2 E)^2 window points per plane).
bool lattice_fits(const Plan& P);
// blocks sharing one brick's input planes at level k, and the elements of the
// plan's split-partial buffer (largest nsplit x points over the split levels)
int lattice_nsplit(const Plan& P, int k);
void lattice_tile_of(const Plan& P, int k, int& txn, int& tyn);
bool lattice_tile_fits(const Plan& P, int txn, int tyn);  // the tile's staging window fits shared memory
int64_t lattice_parts_elems(const Plan& P);
cudaError_t launch_lattice(Plan& P, int k, const void* qk, void* uk, cudaStream_t s);
// the FFT form (fft.cu): tables per level, the convolution, one-time attributes
bool fft_size_ok(int n);
cudaError_t fft_build_level(Plan& P, int k, const std::vector<double>& K, void* work);
void fft_free_level(FftLevel& F);
cudaError_t configure_fft_kernels();
// One launch per pass over every listed level (of one plan, or of every
// replica of a batch).  Each item is one level: its tables, its FP64
// charges, its potential (FP32, or FP64 with fp64) and a complex workspace
// of its size in that precision.
struct FftBatchItem {
  const FftLevel* F;
  const double* q;
  void* u;
  void* work;
};
cudaError_t fft_batch_build(const std::vector<FftBatchItem>& items, bool fp64, FftBatch** out);
cudaError_t fft_batch_launch(const FftBatch* b, cudaStream_t s);
void fft_batch_free(FftBatch* b);
cudaError_t launch_top(Plan& P, const void* qt, void* ut, cudaStream_t s);
cudaError_t launch_prolong(Plan& P, int k, const void* coarse, void* fine, cudaStream_t s);
// interpolation of u^0 at the atoms and assembly of E, phi, F (forward) in two
// launches: the grid gather (u_long and its gradient per atom, needs only
// u^0) and the assembly with the pair sums (phi, F, E; OUT = caller's type)
cudaError_t launch_interp_gather(Plan& P, int64_t n, cudaStream_t s);
template <typename OUT>
cudaError_t launch_interp_assemble(Plan& P, int64_t n, double* energy, OUT* phi, OUT* force, cudaStream_t s);
// adjoint: interpolation of the adjoint grid and assembly of dL/dq, dL/dr
template <typename OUT>
cudaError_t launch_interp_backward(Plan& P, int64_t n, const double* gE, OUT* grad_pos, OUT* grad_q,
                                   cudaStream_t s);
// one-time kernel attributes (called once per process before the first launch)
cudaError_t configure_kernels();
// grid copy to double (debug)
cudaError_t launch_grid_to_double(Plan& P, const void* src, double* dst, int64_t count, bool is_double,
                                  cudaStream_t s);

}  // namespace msm
