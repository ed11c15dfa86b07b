// capi.cu -- the extern "C" entry points declared in include/msm.h.
// Each evaluation is a fixed sequence of kernel launches (no host
// synchronisation, no allocation), in the order of the method: binning,
// short-range pairs, anterpolation, restriction and lattice cutoff per level,
// top level, prolongation, interpolation and assembly.  The grid passes may
// run on a plan-owned stream forked from and joined back onto the caller's.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "msm_internal.h"

using namespace msm;

struct msm_plan {
  Plan p;
};

namespace {

int decode_status(int bits) {
  if (bits & kStatusNonfinite) return MSM_ERR_NONFINITE;
  if (bits & kStatusOutside) return MSM_ERR_ATOM_OUTSIDE_BOX;
  if (bits & kStatusTimeout) return MSM_ERR_TIMEOUT;
  return MSM_OK;
}

// Runs one stage launcher; with profiling on, brackets it with an event pair
// from the plan's pool (events only: no synchronisation).
template <typename F>
cudaError_t stage(Plan& P, int which, cudaStream_t st, F&& launch) {
  if (!P.profiling) return launch();
  if (P.nrec == P.recs.size()) {
    Plan::StageRec r;
    r.stage = which;
    if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess)
      return cudaErrorMemoryAllocation;
    P.recs.push_back(r);
  }
  Plan::StageRec& r = P.recs[P.nrec++];
  r.stage = which;
  cudaEventRecord(r.a, st);
  cudaError_t e = launch();
  cudaEventRecord(r.b, st);
  return e;
}

// The grid sweep shared by the forward pass and its adjoint (dir 0: the
// grids gq/gu, 1: aq/au): starting from the level-0 charges in q[0], fills
// q[1..l-1] by restriction, u[k] by the lattice cutoff and the top level,
// then prolongates u down to level 0.  The FFT form of the lattice cutoff
// takes every level in one set of launches, after the last restriction.
cudaError_t grid_sweep(Plan& P, int dir, cudaStream_t st) {
  void* const* q = dir ? P.d.aq : P.d.gq;
  void* const* u = dir ? P.d.au : P.d.gu;
  cudaError_t e = cudaSuccess;
  int l = P.levels;
  for (int k = 0; k + 1 < l && e == cudaSuccess; ++k) {
    e = stage(P, MSM_STAGE_RESTRICTION, st, [&] { return launch_restrict(P, k, q[k], q[k + 1], st); });
    if (e == cudaSuccess && !P.lattice_fft)
      e = stage(P, MSM_STAGE_LATTICE, st, [&] { return launch_lattice(P, k, q[k], u[k], st); });
  }
  if (e == cudaSuccess && P.lattice_fft)
    e = stage(P, MSM_STAGE_LATTICE, st, [&] {
      P.launches += 5;
      return fft_batch_launch(P.fftb[dir], st);
    });
  if (e == cudaSuccess) e = stage(P, MSM_STAGE_TOP, st, [&] { return launch_top(P, q[l - 1], u[l - 1], st); });
  for (int k = l - 2; k >= 0 && e == cudaSuccess; --k)
    e = stage(P, MSM_STAGE_PROLONGATION, st, [&] { return launch_prolong(P, k, u[k + 1], u[k], st); });
  return e;
}

// IO = the caller's type of positions, charges and per-atom outputs
// After binning, the pair sums and the grid passes (anterpolation through
// prolongation) depend only on the binned atoms, so with overlap on they run
// concurrently: the grid passes on the plan's high-priority side stream (its
// chain of small, latency-bound launches gets the SMs first), the pair sums on
// the caller's stream filling the rest; the caller's stream waits for the grid
// before interpolation.  Fork and join are event waits, so a stream capture of
// st takes the side stream in and the graph gets two parallel branches.
template <typename IO>
int forward(Plan& P, int64_t n, const IO* pos, const IO* q, double* energy, IO* phi, IO* force, cudaStream_t st) {
  cudaError_t e = stage(P, MSM_STAGE_BINNING, st, [&] { return launch_binning(P, n, pos, q, st); });
  cudaStream_t gs = st;
  if (e == cudaSuccess && P.overlap) {
    gs = P.side;
    e = cudaEventRecord(P.ev_fork, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(gs, P.ev_fork, 0);
  }
  if (e == cudaSuccess)
    e = stage(P, MSM_STAGE_ANTERPOLATION, gs,
              [&] { return launch_anterpolate(P, n, P.d.gq[0], nullptr, 1.0, gs); });
  if (e == cudaSuccess) e = stage(P, MSM_STAGE_SHORT_RANGE, st, [&] { return launch_short_range(P, n, st); });
  if (e == cudaSuccess) e = grid_sweep(P, 0, gs);
  // the grid gather needs only u^0, so it runs on the grid's stream, under
  // the pair sums; the assembly waits for both
  if (e == cudaSuccess) e = stage(P, MSM_STAGE_INTERPOLATION, gs, [&] { return launch_interp_gather(P, n, gs); });
  if (e == cudaSuccess && gs != st) {
    e = cudaEventRecord(P.ev_join, gs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, P.ev_join, 0);
  }
  if (e == cudaSuccess)
    e = stage(P, MSM_STAGE_INTERPOLATION, st,
              [&] { return launch_interp_assemble(P, n, energy, phi, force, st); });
  if (e != cudaSuccess) return MSM_ERR_CUDA;
  P.last_stream = st;
  P.last_n = n;
  P.forward_id = ++P.next_id;
  P.evals += 1;
  return MSM_OK;
}

// forward_id: the id the caller's forward pass was given (msm_forward_id);
// 0 accepts whatever forward the plan holds (the batched adjoints).
template <typename IO>
int backward(Plan& P, int64_t forward_id, const double* grad_energy, IO* grad_pos, IO* grad_q, cudaStream_t st) {
  if (P.last_n < 0 || P.forward_id == 0) return MSM_ERR_NO_FORWARD;  // no MSM forward in the plan's buffers
  if (forward_id != 0 && forward_id != P.forward_id) return MSM_ERR_STALE_FORWARD;
  int64_t n = P.last_n;
  // adjoint of u_long = A^T M A q with respect to its inputs: anterpolate the
  // adjoint of u_long (1/2 dL/dE q_i), sweep the (symmetric) grid operator,
  // and interpolate the result back to the atoms.  The anterpolation of
  // 1/2 dL/dE q_i is 1/2 dL/dE times the forward's level-0 charge grid (the
  // same atoms and weights, kept in gq[0] until the next forward), so the
  // adjoint's grid is that one scaled; the potential is recomputed by the
  // sweep.  On the mixed path the result equals a fresh anterpolation bit
  // for bit (the fixed-point sum and the power-of-two unit are exact).
  cudaError_t e = stage(P, MSM_STAGE_ANTERPOLATION, st,
                        [&] { return launch_scale_grid(P, P.d.gq[0], P.d.aq[0], grad_energy, 0.5, st); });
  if (e == cudaSuccess) e = grid_sweep(P, 1, st);
  if (e == cudaSuccess)
    e = stage(P, MSM_STAGE_INTERPOLATION, st,
              [&] { return launch_interp_backward(P, n, grad_energy, grad_pos, grad_q, st); });
  if (e != cudaSuccess) return MSM_ERR_CUDA;
  P.last_stream = st;
  return MSM_OK;
}

// ---- batches: replicas forked over a pool of streams, joined on the caller's ----
constexpr int kPoolStreams = 16;

struct StreamPool {
  int device = -1;
  cudaEvent_t fork = nullptr;
  cudaStream_t s[kPoolStreams] = {};
  cudaEvent_t done[kPoolStreams] = {};
};

std::mutex g_pool_mu;
StreamPool g_pools[8];

cudaError_t pool_for_device(StreamPool** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 8) return cudaErrorInvalidDevice;
  StreamPool& P = g_pools[dev];
  if (P.device != dev) {
    e = cudaEventCreateWithFlags(&P.fork, cudaEventDisableTiming);
    for (int k = 0; k < kPoolStreams && e == cudaSuccess; ++k) {
      e = cudaStreamCreateWithFlags(&P.s[k], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P.done[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return e;
    P.device = dev;
  }
  *out = &P;
  return cudaSuccess;
}

int check_batch(const msm_handle* plans, int nrep, const int64_t* offsets) {
  if (!plans || nrep < 1 || !offsets || offsets[0] != 0) return MSM_ERR_INVALID_ARG;
  for (int r = 0; r < nrep; ++r) {
    if (!plans[r]) return MSM_ERR_INVALID_ARG;
    int64_t n = offsets[r + 1] - offsets[r];
    if (n < 0) return MSM_ERR_INVALID_ARG;
    if (n > plans[r]->p.cap) return MSM_ERR_TOO_MANY_ATOMS;
    for (int s = 0; s < r; ++s)
      if (plans[s] == plans[r]) return MSM_ERR_INVALID_ARG;  // a plan's workspace serves one replica
  }
  return MSM_OK;
}

// Runs body(r, stream) for every replica on the pool, forked from and joined
// back onto st (events only; capturable).
template <typename F>
int fork_join(int nrep, cudaStream_t st, F&& body) {
  std::lock_guard<std::mutex> lock(g_pool_mu);
  StreamPool* pool = nullptr;
  if (pool_for_device(&pool) != cudaSuccess) return MSM_ERR_CUDA;
  const int K = nrep < kPoolStreams ? nrep : kPoolStreams;
  if (cudaEventRecord(pool->fork, st) != cudaSuccess) return MSM_ERR_CUDA;
  for (int k = 0; k < K; ++k)
    if (cudaStreamWaitEvent(pool->s[k], pool->fork, 0) != cudaSuccess) return MSM_ERR_CUDA;
  int rc = MSM_OK;
  for (int r = 0; r < nrep && rc == MSM_OK; ++r) rc = body(r, pool->s[r % K]);
  for (int k = 0; k < K; ++k) {
    if (cudaEventRecord(pool->done[k], pool->s[k]) != cudaSuccess) return MSM_ERR_CUDA;
    if (cudaStreamWaitEvent(st, pool->done[k], 0) != cudaSuccess) return MSM_ERR_CUDA;
  }
  return rc;
}

int batch_forward(const msm_handle* plans, int nrep, const int64_t* off, const double* pos, const double* q,
                  double* energies, double* phi, double* force, cudaStream_t st) {
  return fork_join(nrep, st, [&](int r, cudaStream_t s) {
    Plan& P = plans[r]->p;
    int64_t o = off[r], n = off[r + 1] - off[r];
    return forward(P, n, pos + 3 * o, q + o, energies + r, phi ? phi + o : nullptr, force ? force + 3 * o : nullptr,
                   s);
  });
}

int batch_backward(const msm_handle* plans, int nrep, const int64_t* off, const double* grad_energies,
                   double* grad_pos, double* grad_q, cudaStream_t st) {
  return fork_join(nrep, st, [&](int r, cudaStream_t s) {
    Plan& P = plans[r]->p;
    int64_t o = off[r];
    if (P.last_n != off[r + 1] - off[r]) return (int)MSM_ERR_NO_FORWARD;
    return backward(P, 0, grad_energies + r, grad_pos ? grad_pos + 3 * o : nullptr, grad_q ? grad_q + o : nullptr,
                    s);
  });
}

// The cutoff method's evaluation (binning, the pair kernel with the Coulomb
// pair function, assembly): no grid passes.
int cutoff_forward(Plan& P, int64_t n, const double* pos, const double* q, double* energy, double* phi, double* force,
                   cudaStream_t st) {
  P.last_n = -1;  // the per-atom buffers no longer hold an MSM forward pass
  P.forward_id = 0;
  cudaError_t e = stage(P, MSM_STAGE_BINNING, st, [&] { return launch_binning(P, n, pos, q, st); });
  if (e == cudaSuccess) e = stage(P, MSM_STAGE_SHORT_RANGE, st, [&] { return launch_cutoff_pairs(P, n, st); });
  if (e == cudaSuccess)
    e = stage(P, MSM_STAGE_INTERPOLATION, st, [&] { return launch_cutoff_assemble(P, n, energy, phi, force, st); });
  if (e != cudaSuccess) return MSM_ERR_CUDA;
  P.last_stream = st;
  P.evals += 1;
  return MSM_OK;
}

// Wolf summation (damped, shifted force, damping alpha, cutoff a): the plan's
// binning, the pair kernel with the Wolf pair function, and the assembly with
// the self term phi_i -= 2 c_s q_i, c_s = erfc(alpha a)/(2a) + alpha/sqrt(pi).
template <typename IO>
int wolf_forward(Plan& P, double alpha, int64_t n, const IO* pos, const IO* q, double* energy, IO* phi, IO* force,
                 cudaStream_t st) {
  P.last_n = -1;  // the per-atom buffers no longer hold an MSM forward pass
  P.forward_id = 0;
  const double a = P.P.cutoff;
  const double self_c = 2.0 * (std::erfc(alpha * a) / (2.0 * a) + alpha / std::sqrt(M_PI));
  cudaError_t e = stage(P, MSM_STAGE_BINNING, st, [&] { return launch_binning(P, n, pos, q, st); });
  if (e == cudaSuccess) e = stage(P, MSM_STAGE_SHORT_RANGE, st, [&] { return launch_wolf_pairs(P, n, alpha, st); });
  if (e == cudaSuccess)
    e = stage(P, MSM_STAGE_INTERPOLATION, st,
              [&] { return launch_cutoff_assemble(P, n, energy, phi, force, st, self_c); });
  if (e != cudaSuccess) return MSM_ERR_CUDA;
  P.last_stream = st;
  P.evals += 1;
  return MSM_OK;
}

// Energy and force at pos by MSM, the cutoff method or Wolf summation.
int md_force(Plan& P, int method, int64_t n, const double* pos, const double* q, double* energy, double* force,
             cudaStream_t st) {
  if (method == MSM_MD_CUTOFF) return cutoff_forward(P, n, pos, q, energy, nullptr, force, st);
  if (method == MSM_MD_WOLF) return wolf_forward(P, P.wolf_alpha, n, pos, q, energy, (double*)nullptr, force, st);
  return forward(P, n, pos, q, energy, (double*)nullptr, force, st);
}

bool valid_method(int m) { return m == MSM_MD_MSM || m == MSM_MD_CUTOFF || m == MSM_MD_WOLF; }

// One velocity Verlet step (drift, force, kick).  rec: this step's record or
// NULL; with a step counter rec is the base of the records and the kick's
// record kernel places and advances (steps replayed from a graph).
int md_step(Plan& P, int method, int64_t n, double* pos, double* vel, double* force, const double* inv_mass,
            const double* q, double dt, double* rec, int* counter, cudaStream_t st) {
  double* u = (rec && !counter) ? rec : P.d.scalars + 1;  // the step's energy
  if (launch_md_drift(P, n, pos, vel, force, inv_mass, dt, st) != cudaSuccess) return MSM_ERR_CUDA;
  int rc = md_force(P, method, n, pos, q, u, force, st);
  if (rc != MSM_OK) return rc;
  if (launch_md_kick(P, n, vel, force, inv_mass, dt, u, rec ? rec : P.d.scalars + 2, rec ? counter : nullptr, st) !=
      cudaSuccess)
    return MSM_ERR_CUDA;
  return MSM_OK;
}

// nsteps of velocity Verlet; with init_force the force at the starting
// positions is evaluated first.
int md_loop(Plan& P, int method, int64_t n, double* pos, double* vel, double* force, const double* inv_mass,
            const double* q, double dt, int nsteps, bool init_force, double* records, cudaStream_t st) {
  if (init_force) {
    int rc = md_force(P, method, n, pos, q, P.d.scalars + 1, force, st);
    if (rc != MSM_OK) return rc;
  }
  for (int s = 0; s < nsteps; ++s) {
    int rc = md_step(P, method, n, pos, vel, force, inv_mass, q, dt, records ? records + 6 * (size_t)s : nullptr,
                     nullptr, st);
    if (rc != MSM_OK) return rc;
  }
  P.last_stream = st;
  return MSM_OK;
}

// msm_md_run replays one captured step from a CUDA graph on systems this
// small (their steps are launch-bound), and launches eagerly otherwise or
// when the caller's stream is itself being captured.
constexpr int64_t kMdGraphMaxAtoms = 262144;
constexpr int kMdGraphMinSteps = 16;  // enough steps to repay capturing and instantiating the graph

// Captures body(stream) on a private stream into an instantiated graph whose
// kernel nodes keep the priorities of the streams they were captured from.
template <typename F>
int capture_graph(F&& body, cudaGraphExec_t* out) {
  *out = nullptr;
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return MSM_ERR_CUDA;
  int rc = MSM_OK;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    rc = MSM_ERR_CUDA;
  } else {
    rc = body(cs);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cs, &g);  // always end the capture
    if (rc == MSM_OK && e != cudaSuccess) rc = MSM_ERR_CUDA;
    if (rc == MSM_OK && cudaGraphInstantiateWithFlags(out, g, cudaGraphInstantiateFlagUseNodePriority) != cudaSuccess)
      rc = MSM_ERR_CUDA;
    if (g) cudaGraphDestroy(g);
  }
  cudaStreamDestroy(cs);
  return rc;
}

std::once_flag g_config_once;
cudaError_t g_config_err = cudaSuccess;

}  // namespace

struct msm_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // batched form: the argument tables of the batched stages and the stream
  // that carries the grid passes during the capture
  BinBatch* bin = nullptr;
  PairBatch* pair = nullptr;
  GridBatch* grid = nullptr;
  cudaStream_t side = nullptr, side2 = nullptr;  // the forward's and the adjoint's grid passes
  cudaEvent_t fork = nullptr, join = nullptr, front = nullptr, join2 = nullptr;
  // the plans whose buffers a replay refills (each replay is a new forward)
  std::vector<Plan*> plans;
};

namespace {

// The batched form needs one kernel family for every replica: mixed
// precision, one interpolation order, one splitting; and its lattice runs by
// FFT when every plan took that form, else by the stencil, which every plan's
// stencil must then fit.
bool batchable(const msm_handle* plans, int nrep) {
  bool all_fft = true, all_fit = true;
  for (int r = 0; r < nrep; ++r) {
    const Plan& P = plans[r]->p;
    if (P.fp64 || P.P.order != plans[0]->p.P.order || P.P.splitting != plans[0]->p.P.splitting) return false;
    all_fft = all_fft && P.lattice_fft;
    all_fit = all_fit && P.stencil_fits;
  }
  return all_fft || all_fit;
}

// Builds the argument tables of the batched stages (synchronous; allocates).
int batch_tables(msm_graph* g, const msm_handle* plans, int nrep, const int64_t* off, const double* pos,
                 const double* q, double* energies, double* phi, double* force, const double* grad_energies,
                 double* grad_pos, double* grad_q) {
  std::vector<BatchRep> reps;
  for (int r = 0; r < nrep; ++r) {
    const int64_t o = off[r];
    BatchRep b;
    b.plan = &plans[r]->p;
    b.n = off[r + 1] - o;
    b.pos = pos + 3 * o;
    b.q = q + o;
    b.energy = energies + r;
    b.phi = phi ? phi + o : nullptr;
    b.force = force ? force + 3 * o : nullptr;
    b.grad_energy = grad_energies ? grad_energies + r : nullptr;
    b.grad_pos = grad_pos ? grad_pos + 3 * o : nullptr;
    b.grad_q = grad_q ? grad_q + o : nullptr;
    reps.push_back(b);
  }
  int least = 0, greatest = 0;
  if (bin_batch_build(reps, &g->bin) != cudaSuccess || pair_batch_build(reps, &g->pair) != cudaSuccess ||
      grid_batch_build(reps, grad_energies != nullptr, &g->grid) != cudaSuccess ||
      cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
      cudaStreamCreateWithPriority(&g->side, cudaStreamNonBlocking, greatest) != cudaSuccess ||
      cudaStreamCreateWithPriority(&g->side2, cudaStreamNonBlocking, greatest) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->front, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->join2, cudaEventDisableTiming) != cudaSuccess)
    return MSM_ERR_CUDA;
  for (int r = 0; r < nrep; ++r) plans[r]->p.last_n = off[r + 1] - off[r];
  return MSM_OK;
}

// The batched forward (and adjoint) on cs: binning of every replica, then the
// pair sums of every replica on cs concurrently with the grid passes of every
// replica on the high-priority side stream, then interpolation; each stage is
// one launch over all replicas.  The adjoint's grid passes need only the
// binned atoms and the anterpolated charges (not the forward's pair sums or
// potentials), so after the shared anterpolation they run on a second side
// stream beside the forward's (each direction has its own temporaries); the
// adjoint's interpolation waits for them.  Persistent chains share one grid
// barrier, so with them the adjoint's passes follow the forward's on cs.
int batch_fused(msm_graph* g, cudaStream_t cs, bool backward) {
  const bool side_adjoint = backward && !grid_batch_persistent(g->grid);
  cudaError_t e = bin_batch_launch(g->bin, cs);
  if (e == cudaSuccess) e = cudaEventRecord(g->fork, cs);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(g->side, g->fork, 0);
  if (e == cudaSuccess) e = grid_batch_front(g->grid, backward, g->side);
  if (e == cudaSuccess && side_adjoint) {
    e = cudaEventRecord(g->front, g->side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(g->side2, g->front, 0);
    if (e == cudaSuccess) e = grid_batch_levels(g->grid, 1, g->side2);
    if (e == cudaSuccess) e = cudaEventRecord(g->join2, g->side2);
  }
  if (e == cudaSuccess) e = grid_batch_levels(g->grid, 0, g->side);
  if (e == cudaSuccess) e = cudaEventRecord(g->join, g->side);
  if (e == cudaSuccess) e = pair_batch_launch(g->pair, cs);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, g->join, 0);
  if (e == cudaSuccess) e = grid_batch_interp(g->grid, false, cs);
  if (e == cudaSuccess && backward) {
    if (side_adjoint) e = cudaStreamWaitEvent(cs, g->join2, 0);
    else e = grid_batch_levels(g->grid, 1, cs);
  }
  if (e == cudaSuccess && backward) e = grid_batch_interp(g->grid, true, cs);
  return e == cudaSuccess ? MSM_OK : MSM_ERR_CUDA;
}

}  // namespace

extern "C" {

int msm_create(const msm_params* params, msm_handle* out) { return msm_create_tuned(params, nullptr, out); }

int msm_create_tuned(const msm_params* params, const msm_tuning* tuning, msm_handle* out) {
  if (!params || !out) return MSM_ERR_INVALID_ARG;
  *out = nullptr;
  int vrc = validate_params(params);
  if (vrc == MSM_OK) vrc = validate_tuning(tuning);
  if (vrc != MSM_OK) return vrc;
  std::call_once(g_config_once, [] { g_config_err = configure_kernels(); });
  if (g_config_err != cudaSuccess) return MSM_ERR_CUDA;
  msm_plan* h = new (std::nothrow) msm_plan();
  if (!h) return MSM_ERR_OOM;
  int rc = build_plan(params, tuning, &h->p);
  if (rc != MSM_OK) {
    free_plan(&h->p);
    delete h;
    return rc;
  }
  *out = h;
  return MSM_OK;
}

void msm_destroy(msm_handle h) {
  if (!h) return;
  cudaDeviceSynchronize();
  for (auto& r : h->p.recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  free_plan(&h->p);
  delete h;
}

int msm_geometry(const msm_params* params, double h_eff[3], int* levels, int* dims, int* lo) {
  if (!params) return MSM_ERR_INVALID_ARG;
  Plan P;  // host fields only: nothing is allocated
  const int rc = plan_geometry(params, &P);
  if (rc != MSM_OK) return rc;
  if (h_eff)
    for (int d = 0; d < 3; ++d) h_eff[d] = P.h[d];
  if (levels) *levels = P.levels;
  for (int k = 0; k < P.levels; ++k)
    for (int d = 0; d < 3; ++d) {
      if (dims) dims[3 * k + d] = P.n[k][d];
      if (lo) lo[3 * k + d] = P.lo[k][d];
    }
  return MSM_OK;
}

int msm_query(msm_handle h, double h_eff[3], int* levels, int* dims, int* lo) {
  if (!h) return MSM_ERR_INVALID_ARG;
  const Plan& P = h->p;
  if (h_eff)
    for (int d = 0; d < 3; ++d) h_eff[d] = P.h[d];
  if (levels) *levels = P.levels;
  for (int k = 0; k < P.levels; ++k)
    for (int d = 0; d < 3; ++d) {
      if (dims) dims[3 * k + d] = P.n[k][d];
      if (lo) lo[3 * k + d] = P.lo[k][d];
    }
  return MSM_OK;
}

int msm_lattice_method(msm_handle h, int* method) {
  if (!h || !method) return MSM_ERR_INVALID_ARG;
  *method = h->p.lattice_fft ? 2 : 1;
  return MSM_OK;
}

int msm_eval(msm_handle h, int64_t n, const double* pos, const double* q, double* energy, double* phi,
             double* force, void* stream) {
  if (!h || n < 0 || !energy || (n > 0 && (!pos || !q))) return MSM_ERR_INVALID_ARG;
  Plan& P = h->p;
  if (n > P.cap) return MSM_ERR_TOO_MANY_ATOMS;
  return forward(P, n, pos, q, energy, phi, force, (cudaStream_t)stream);
}

int msm_cutoff_eval(msm_handle h, int64_t n, const double* pos, const double* q, double* energy, double* phi,
                    double* force, void* stream) {
  if (!h || n < 0 || !energy || (n > 0 && (!pos || !q))) return MSM_ERR_INVALID_ARG;
  Plan& P = h->p;
  if (n > P.cap) return MSM_ERR_TOO_MANY_ATOMS;
  return cutoff_forward(P, n, pos, q, energy, phi, force, (cudaStream_t)stream);
}

int msm_wolf_eval(msm_handle h, double alpha, int64_t n, const double* pos, const double* q, double* energy,
                  double* phi, double* force, void* stream) {
  if (!h || n < 0 || !energy || (n > 0 && (!pos || !q)) || !(alpha >= 0.0) || !std::isfinite(alpha))
    return MSM_ERR_INVALID_ARG;
  Plan& P = h->p;
  if (n > P.cap) return MSM_ERR_TOO_MANY_ATOMS;
  return wolf_forward(P, alpha, n, pos, q, energy, phi, force, (cudaStream_t)stream);
}

int msm_set_wolf_alpha(msm_handle h, double alpha) {
  if (!h || !(alpha >= 0.0) || !std::isfinite(alpha)) return MSM_ERR_INVALID_ARG;
  h->p.wolf_alpha = alpha;
  return MSM_OK;
}

int msm_md_run(msm_handle h, int64_t n, double* pos, double* vel, double* force, const double* inv_mass,
               const double* q, double dt, int nsteps, int method, double* records, void* stream) {
  if (!h || n < 0 || nsteps < 0 || !std::isfinite(dt)) return MSM_ERR_INVALID_ARG;
  if (!valid_method(method)) return MSM_ERR_INVALID_ARG;
  if (n > 0 && (!pos || !vel || !force || !inv_mass || !q)) return MSM_ERR_INVALID_ARG;
  Plan& P = h->p;
  if (n > P.cap) return MSM_ERR_TOO_MANY_ATOMS;
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return MSM_ERR_CUDA;
  if (cap != cudaStreamCaptureStatusNone || nsteps < kMdGraphMinSteps || n > kMdGraphMaxAtoms)
    return md_loop(P, method, n, pos, vel, force, inv_mass, q, dt, nsteps, false, records, st);
  if (records && cudaMemsetAsync(P.d.md_step, 0, sizeof(int), st) != cudaSuccess) return MSM_ERR_CUDA;
  cudaGraphExec_t g = nullptr;
  int rc = capture_graph(
      [&](cudaStream_t cs) {
        return md_step(P, method, n, pos, vel, force, inv_mass, q, dt, records, P.d.md_step, cs);
      },
      &g);
  P.last_stream = st;
  for (int s = 0; s < nsteps && rc == MSM_OK; ++s)
    if (cudaGraphLaunch(g, st) != cudaSuccess) rc = MSM_ERR_CUDA;
  if (g) cudaGraphExecDestroy(g);  // freed once its launches complete
  return rc;
}

int msm_md_run_batch(const msm_handle* plans, int nrep, const int64_t* offsets, double* pos, double* vel,
                     double* force, const double* inv_mass, const double* q, double dt, int nsteps, int method,
                     double* records, void* stream) {
  int rc = check_batch(plans, nrep, offsets);
  if (rc != MSM_OK) return rc;
  if (nsteps < 0 || !std::isfinite(dt) || !valid_method(method))
    return MSM_ERR_INVALID_ARG;
  if (offsets[nrep] > 0 && (!pos || !vel || !force || !inv_mass || !q)) return MSM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int64_t nmax = 0;
  for (int r = 0; r < nrep; ++r) nmax = std::max(nmax, offsets[r + 1] - offsets[r]);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return MSM_ERR_CUDA;
  if (cap != cudaStreamCaptureStatusNone || nsteps < kMdGraphMinSteps || nmax > kMdGraphMaxAtoms)
    return fork_join(nrep, st, [&](int r, cudaStream_t s) {
      const int64_t o = offsets[r], n = offsets[r + 1] - offsets[r];
      return md_loop(plans[r]->p, method, n, pos + 3 * o, vel + 3 * o, force + 3 * o, inv_mass + o, q + o, dt,
                     nsteps, false, records ? records + 6 * (size_t)nsteps * r : nullptr, s);
    });
  // small replicas: one step of all of them captured into a graph and replayed
  for (int r = 0; r < nrep && records; ++r)
    if (cudaMemsetAsync(plans[r]->p.d.md_step, 0, sizeof(int), st) != cudaSuccess) return MSM_ERR_CUDA;
  cudaGraphExec_t g = nullptr;
  rc = capture_graph(
      [&](cudaStream_t cs) {
        return fork_join(nrep, cs, [&](int r, cudaStream_t s) {
          const int64_t o = offsets[r], n = offsets[r + 1] - offsets[r];
          Plan& P = plans[r]->p;
          return md_step(P, method, n, pos + 3 * o, vel + 3 * o, force + 3 * o, inv_mass + o, q + o, dt,
                         records ? records + 6 * (size_t)nsteps * r : nullptr, P.d.md_step, s);
        });
      },
      &g);
  for (int r = 0; r < nrep; ++r) plans[r]->p.last_stream = st;
  for (int s = 0; s < nsteps && rc == MSM_OK; ++s)
    if (cudaGraphLaunch(g, st) != cudaSuccess) rc = MSM_ERR_CUDA;
  if (g) cudaGraphExecDestroy(g);
  return rc;
}

int64_t msm_parareal_workspace(int64_t n, int window) {
  if (n < 0 || window < 1 || window > MSM_PARAREAL_MAX_WINDOW) return -1;
  return (int64_t)sizeof(double) * (3 * n * (5 * (int64_t)window + 3) + 2 * (int64_t)window);
}

int msm_parareal(const msm_handle* fine, msm_handle coarse, int64_t n, const double* pos0, const double* vel0,
                 const double* inv_mass, const double* q, int window, double dt_fine, int steps_fine,
                 double dt_coarse, int steps_coarse, int coarse_method, int max_iter, double tol, double* lam_pos,
                 double* lam_vel, void* workspace, int* iterations, double* change, void* stream) {
  if (!fine || !coarse || n < 0 || window < 1 || window > MSM_PARAREAL_MAX_WINDOW) return MSM_ERR_INVALID_ARG;
  if (!valid_method(coarse_method)) return MSM_ERR_INVALID_ARG;
  if (!std::isfinite(dt_fine) || !std::isfinite(dt_coarse) || steps_fine < 0 || steps_coarse < 0 || max_iter < 0 ||
      !(tol >= 0.0) || !std::isfinite(tol))
    return MSM_ERR_INVALID_ARG;
  if (!workspace || !lam_pos || !lam_vel || (n > 0 && (!pos0 || !vel0 || !inv_mass || !q))) return MSM_ERR_INVALID_ARG;
  for (int r = 0; r < window; ++r) {
    if (!fine[r]) return MSM_ERR_INVALID_ARG;
    if (n > fine[r]->p.cap) return MSM_ERR_TOO_MANY_ATOMS;
    for (int s = 0; s < r; ++s)
      if (fine[s] == fine[r]) return MSM_ERR_INVALID_ARG;  // the fine propagations run concurrently
  }
  if (n > coarse->p.cap) return MSM_ERR_TOO_MANY_ATOMS;
  if (iterations) *iterations = 0;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t N3 = 3 * (size_t)n, B3 = sizeof(double) * N3;
  double* ws = (double*)workspace;
  double *fpos = ws, *fvel = fpos + window * N3, *gpos = fvel + window * N3, *gvel = gpos + window * N3;
  double *fforce = gvel + window * N3, *cpos = fforce + window * N3, *cvel = cpos + N3, *cforce = cvel + N3;
  double* chg = cforce + N3;  // [window][2]
  Plan& C = coarse->p;
  auto lp = [&](int k) { return lam_pos + k * N3; };
  auto lv = [&](int k) { return lam_vel + k * N3; };
  auto cp = [&](double* dst, const double* src, cudaStream_t s) {
    return B3 == 0 || cudaMemcpyAsync(dst, src, B3, cudaMemcpyDeviceToDevice, s) == cudaSuccess;
  };
  // G from time point k: the coarse state (cpos, cvel) after steps_coarse steps
  auto coarse_from = [&](int k, cudaStream_t s) {
    if (!cp(cpos, lp(k), s) || !cp(cvel, lv(k), s)) return (int)MSM_ERR_CUDA;
    return md_loop(C, coarse_method, n, cpos, cvel, cforce, inv_mass, q, dt_coarse, steps_coarse, true, nullptr, s);
  };
  // lambda_0 = the initial state; iteration 0 is one coarse sweep
  if (!cp(lp(0), pos0, st) || !cp(lv(0), vel0, st)) return MSM_ERR_CUDA;
  for (int k = 0; k < window; ++k) {
    int rc = coarse_from(k, st);
    if (rc != MSM_OK) return rc;
    if (!cp(gpos + k * N3, cpos, st) || !cp(gvel + k * N3, cvel, st) || !cp(lp(k + 1), cpos, st) ||
        !cp(lv(k + 1), cvel, st))
      return MSM_ERR_CUDA;
  }
  const double span = dt_fine * steps_fine;  // Delta T: velocity changes are weighed by it
  // One iteration: F from every time point of the window, concurrently (one
  // plan each), then the sequential coarse sweep with the correction.  On a
  // small system that is thousands of short launches, so it is captured once
  // into a CUDA graph and replayed.
  auto iteration = [&](cudaStream_t s) {
    int rc = fork_join(window, s, [&](int r, cudaStream_t fs) {
      if (!cp(fpos + r * N3, lp(r), fs) || !cp(fvel + r * N3, lv(r), fs)) return (int)MSM_ERR_CUDA;
      return md_loop(fine[r]->p, MSM_MD_MSM, n, fpos + r * N3, fvel + r * N3, fforce + r * N3, inv_mass, q, dt_fine,
                     steps_fine, true, nullptr, fs);
    });
    for (int k = 0; k < window && rc == MSM_OK; ++k) {
      rc = coarse_from(k, s);
      if (rc == MSM_OK && launch_parareal_correct(C, n, cpos, cvel, fpos + k * N3, fvel + k * N3, gpos + k * N3,
                                                  gvel + k * N3, lp(k + 1), lv(k + 1), chg + 2 * k, s) != cudaSuccess)
        rc = MSM_ERR_CUDA;
    }
    return rc;
  };
  cudaGraphExec_t graph = nullptr;
  int rc = max_iter > 0 ? capture_graph(iteration, &graph) : MSM_OK;
  for (int r = 0; r < window; ++r) fine[r]->p.last_stream = st;  // not the capture's streams
  C.last_stream = st;
  std::vector<double> h(2 * (size_t)window);
  for (int it = 0; it < max_iter && rc == MSM_OK; ++it) {
    if (cudaGraphLaunch(graph, st) != cudaSuccess ||
        cudaMemcpyAsync(h.data(), chg, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      rc = MSM_ERR_CUDA;
      break;
    }
    double dr = 0.0, dv = 0.0;
    for (int k = 0; k < window; ++k) {
      dr = std::max(dr, h[2 * k]);
      dv = std::max(dv, h[2 * k + 1]);
    }
    if (change) {
      change[2 * it] = dr;
      change[2 * it + 1] = dv;
    }
    if (iterations) *iterations = it + 1;
    if (dr <= tol && dv * std::fabs(span) <= tol) break;
  }
  if (graph) cudaGraphExecDestroy(graph);
  return rc;
}

int msm_eval_backward(msm_handle h, int64_t forward_id, const double* grad_energy, double* grad_pos, double* grad_q,
                      void* stream) {
  if (!h || !grad_energy || forward_id <= 0) return MSM_ERR_INVALID_ARG;
  return backward(h->p, forward_id, grad_energy, grad_pos, grad_q, (cudaStream_t)stream);
}

int msm_forward_id(msm_handle h, int64_t* forward_id) {
  if (!h || !forward_id) return MSM_ERR_INVALID_ARG;
  *forward_id = h->p.forward_id;
  return MSM_OK;
}

int msm_eval_f32io(msm_handle h, int64_t n, const float* pos, const float* q, double* energy, float* phi,
                   float* force, void* stream) {
  if (!h || n < 0 || !energy || (n > 0 && (!pos || !q))) return MSM_ERR_INVALID_ARG;
  Plan& P = h->p;
  if (n > P.cap) return MSM_ERR_TOO_MANY_ATOMS;
  return forward(P, n, pos, q, energy, phi, force, (cudaStream_t)stream);
}

int msm_eval_backward_f32io(msm_handle h, int64_t forward_id, const double* grad_energy, float* grad_pos,
                            float* grad_q, void* stream) {
  if (!h || !grad_energy || forward_id <= 0) return MSM_ERR_INVALID_ARG;
  return backward(h->p, forward_id, grad_energy, grad_pos, grad_q, (cudaStream_t)stream);
}

int msm_eval_batch(const msm_handle* plans, int nrep, const int64_t* offsets, const double* pos, const double* q,
                   double* energies, double* phi, double* force, void* stream) {
  int rc = check_batch(plans, nrep, offsets);
  if (rc != MSM_OK) return rc;
  if (!energies || (offsets[nrep] > 0 && (!pos || !q))) return MSM_ERR_INVALID_ARG;
  return batch_forward(plans, nrep, offsets, pos, q, energies, phi, force, (cudaStream_t)stream);
}

int msm_eval_backward_batch(const msm_handle* plans, int nrep, const int64_t* offsets, const double* grad_energies,
                            double* grad_pos, double* grad_q, void* stream) {
  int rc = check_batch(plans, nrep, offsets);
  if (rc != MSM_OK) return rc;
  if (!grad_energies) return MSM_ERR_INVALID_ARG;
  return batch_backward(plans, nrep, offsets, grad_energies, grad_pos, grad_q, (cudaStream_t)stream);
}

int msm_batch_graph_create(const msm_handle* plans, int nrep, const int64_t* offsets, const double* pos,
                           const double* q, double* energies, double* phi, double* force,
                           const double* grad_energies, double* grad_pos, double* grad_q, msm_graph_handle* out) {
  if (!out) return MSM_ERR_INVALID_ARG;
  *out = nullptr;
  int rc = check_batch(plans, nrep, offsets);
  if (rc != MSM_OK) return rc;
  if (!energies || (offsets[nrep] > 0 && (!pos || !q))) return MSM_ERR_INVALID_ARG;
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return MSM_ERR_CUDA;
  msm_graph* g = new (std::nothrow) msm_graph();
  if (!g) {
    cudaStreamDestroy(cs);
    return MSM_ERR_OOM;
  }
  // one replica gains nothing from the batched tables: it is captured on the
  // single-system path (its compile-time lattice tile, its own patch size)
  const bool fused = nrep > 1 && batchable(plans, nrep);
  rc = fused ? batch_tables(g, plans, nrep, offsets, pos, q, energies, phi, force, grad_energies, grad_pos, grad_q)
             : MSM_OK;
  if (rc == MSM_OK && cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = MSM_ERR_CUDA;
  if (rc == MSM_OK) {
    if (fused) {
      rc = batch_fused(g, cs, grad_energies != nullptr);
    } else {
      rc = batch_forward(plans, nrep, offsets, pos, q, energies, phi, force, cs);
      if (rc == MSM_OK && grad_energies)
        rc = batch_backward(plans, nrep, offsets, grad_energies, grad_pos, grad_q, cs);
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &graph);  // always end the capture
    if (rc == MSM_OK && e != cudaSuccess) rc = MSM_ERR_CUDA;
    g->graph = graph;
    // node priorities: the grid passes keep the precedence of the plan's
    // high-priority side stream they were captured from
    if (rc == MSM_OK && cudaGraphInstantiateWithFlags(&g->exec, graph, cudaGraphInstantiateFlagUseNodePriority) !=
                            cudaSuccess)
      rc = MSM_ERR_CUDA;
  }
  cudaStreamDestroy(cs);
  for (int r = 0; r < nrep; ++r) {
    plans[r]->p.last_stream = nullptr;  // not the destroyed capture stream
    g->plans.push_back(&plans[r]->p);
  }
  if (rc != MSM_OK) {
    msm_graph_destroy(g);
    return rc;
  }
  *out = g;
  return MSM_OK;
}

int msm_graph_launch(msm_graph_handle g, void* stream) {
  if (!g || !g->exec) return MSM_ERR_INVALID_ARG;
  if (cudaGraphLaunch(g->exec, (cudaStream_t)stream) != cudaSuccess) return MSM_ERR_CUDA;
  // the replay refilled every plan's buffers: a later adjoint of an earlier
  // forward id must be refused
  for (Plan* P : g->plans) P->forward_id = ++P->next_id;
  return MSM_OK;
}

void msm_graph_destroy(msm_graph_handle g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->bin || g->pair || g->grid) cudaDeviceSynchronize();  // the tables may be in use by a launched graph
  bin_batch_free(g->bin);
  pair_batch_free(g->pair);
  grid_batch_free(g->grid);
  if (g->side) cudaStreamDestroy(g->side);
  if (g->side2) cudaStreamDestroy(g->side2);
  if (g->fork) cudaEventDestroy(g->fork);
  if (g->join) cudaEventDestroy(g->join);
  if (g->front) cudaEventDestroy(g->front);
  if (g->join2) cudaEventDestroy(g->join2);
  delete g;
}

int msm_eval_host(msm_handle h, int64_t n, const double* pos, const double* q, double* energy, double* phi,
                  double* force, void* stream) {
  if (!h || n < 0 || !energy || (n > 0 && (!pos || !q))) return MSM_ERR_INVALID_ARG;
  Plan& P = h->p;
  if (n > P.cap) return MSM_ERR_TOO_MANY_ATOMS;
  DeviceBuffers& D = P.d;
  if (!D.hpos) {  // staging buffers for the host-buffer entry point, made on first use
    cudaError_t e = cudaMalloc((void**)&D.hpos, sizeof(double) * 3 * P.cap);
    if (e == cudaSuccess) e = cudaMalloc((void**)&D.hq, sizeof(double) * P.cap);
    if (e == cudaSuccess) e = cudaMalloc((void**)&D.hphi, sizeof(double) * P.cap);
    if (e == cudaSuccess) e = cudaMalloc((void**)&D.hforce, sizeof(double) * 3 * P.cap);
    if (e == cudaSuccess) e = cudaMalloc((void**)&D.henergy, sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&D.hstatus, sizeof(int));
    if (e != cudaSuccess) return MSM_ERR_OOM;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (n > 0) {
    if (cudaMemcpyAsync(D.hpos, pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(D.hq, q, sizeof(double) * n, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return MSM_ERR_CUDA;
  }
  int rc = forward(P, n, D.hpos, D.hq, D.henergy, phi ? D.hphi : nullptr, force ? D.hforce : nullptr, st);
  if (rc != MSM_OK) return rc;
  if (cudaMemcpyAsync(energy, D.henergy, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return MSM_ERR_CUDA;
  if (phi && n > 0 && cudaMemcpyAsync(phi, D.hphi, sizeof(double) * n, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return MSM_ERR_CUDA;
  if (force && n > 0 &&
      cudaMemcpyAsync(force, D.hforce, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return MSM_ERR_CUDA;
  // the status word comes back with the results: one synchronisation of the
  // stream instead of a device-wide one and a blocking copy
  if (cudaMemcpyAsync(D.hstatus, P.d.status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return MSM_ERR_CUDA;
  const int bits = *D.hstatus;
  if (bits && cudaMemset(P.d.status, 0, sizeof(int)) != cudaSuccess) return MSM_ERR_CUDA;
  return decode_status(bits);
}

int msm_status(msm_handle h) {
  if (!h) return MSM_ERR_INVALID_ARG;
  Plan& P = h->p;
  if (cudaDeviceSynchronize() != cudaSuccess) return MSM_ERR_CUDA;
  int bits = 0;
  if (cudaMemcpy(&bits, P.d.status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return MSM_ERR_CUDA;
  if (bits && cudaMemset(P.d.status, 0, sizeof(int)) != cudaSuccess) return MSM_ERR_CUDA;
  return decode_status(bits);
}

int msm_debug_grid(msm_handle h, int level, int which, double* host_out) {
  if (!h || !host_out || level < 0 || which < 0 || which > 1) return MSM_ERR_INVALID_ARG;
  Plan& P = h->p;
  if (level >= P.levels) return MSM_ERR_INVALID_ARG;
  int64_t np = grid_points(P, level);
  double* tmp = nullptr;
  if (cudaMalloc((void**)&tmp, sizeof(double) * np) != cudaSuccess) return MSM_ERR_OOM;
  cudaStream_t st = P.last_stream;
  const void* src = which == 0 ? P.d.gq[level] : P.d.gu[level];
  cudaError_t e = launch_grid_to_double(P, src, tmp, np, which == 0, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemcpy(host_out, tmp, sizeof(double) * np, cudaMemcpyDeviceToHost);
  cudaFree(tmp);
  return e == cudaSuccess ? MSM_OK : MSM_ERR_CUDA;
}

int msm_set_overlap(msm_handle h, int enable) {
  if (!h) return MSM_ERR_INVALID_ARG;
  h->p.overlap = enable != 0;
  return MSM_OK;
}

int msm_profile(msm_handle h, int enable) {
  if (!h) return MSM_ERR_INVALID_ARG;
  h->p.profiling = enable != 0;
  return MSM_OK;
}

int msm_profile_read(msm_handle h, double* ms, int64_t* launches, int64_t* evals) {
  if (!h) return MSM_ERR_INVALID_ARG;
  Plan& P = h->p;
  double acc[MSM_NSTAGES] = {0};
  for (size_t i = 0; i < P.nrec; ++i) {
    Plan::StageRec& r = P.recs[i];
    float t = 0.f;
    if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess)
      return MSM_ERR_CUDA;
    if (r.stage >= 0 && r.stage < MSM_NSTAGES) acc[r.stage] += t;
  }
  if (ms)
    for (int s = 0; s < MSM_NSTAGES; ++s) ms[s] = acc[s];
  if (launches) *launches = P.launches;
  if (evals) *evals = P.evals;
  P.nrec = 0;
  P.launches = 0;
  P.evals = 0;
  return MSM_OK;
}

const char* msm_stage_name(int s) {
  static const char* names[MSM_NSTAGES] = {"binning", "short_range", "anterpolation", "restriction",
                                           "lattice_cutoff", "top_level", "prolongation",
                                           "interpolation"};
  return (s >= 0 && s < MSM_NSTAGES) ? names[s] : "?";
}

const char* msm_strerror(int code) {
  switch (code) {
    case MSM_OK: return "ok";
    case MSM_ERR_INVALID_ARG: return "invalid argument";
    case MSM_ERR_UNSUPPORTED: return "unsupported configuration";
    case MSM_ERR_CUTOFF_GT_HALF_BOX: return "cutoff larger than half the periodic box";
    case MSM_ERR_ATOM_OUTSIDE_BOX: return "atom outside the open box";
    case MSM_ERR_NONFINITE: return "non-finite position or charge";
    case MSM_ERR_OOM: return "device allocation failed";
    case MSM_ERR_CUDA: return "CUDA error";
    case MSM_ERR_TIMEOUT: return "bounded device wait gave up";
    case MSM_ERR_TOO_MANY_ATOMS: return "more atoms than the plan's capacity";
    case MSM_ERR_NO_FORWARD: return "backward before forward";
    case MSM_ERR_STALE_FORWARD: return "the plan holds a later forward pass than the one named";
    default: return "unknown error";
  }
}

}  // extern "C"
