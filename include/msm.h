/*
 * msm.h -- C ABI of the GB300 multilevel summation (MSM) library.
 *
 * One call evaluates Coulomb electrostatics of N point charges by the
 * multilevel summation method of the thesis proposal "Large-Scale Molecular
 * Dynamics Simulations for Highly Parallel Infrastructures" (Pazurikova,
 * 2014), Sec. "Multilevel Summation Method": the kernel 1/r is split as
 * g* + g^0 + ... + g^{l-1} (Eq. msmgrid) with the Taylor smoothing gamma;
 * the short-range part g* is summed over atom pairs within the cutoff a; the
 * rest goes through anterpolation, restriction, a lattice cutoff per level,
 * an all-pairs top level, prolongation and interpolation; the potential is
 * U_i = k_c (u_i^short + u_i^long) and the forces are F_i = -dU/dr_i
 * (Sec. "Simulation loop").  Around that evaluation: its adjoint, batches of
 * independent systems, the cutoff method (the parareal section's coarse
 * propagator), velocity Verlet molecular dynamics and one parareal window.
 *
 * Conventions shared by every entry point:
 *   - Units are the caller's: positions in the unit of box/cutoff/spacing
 *     (Angstrom in the tests), charges in e; energies come out in
 *     coulomb_k * charge^2 / length.
 *   - Device pointers are CUDA device addresses on the current device.
 *     Arrays are dense, C order: pos and force are [n][3] (x, y, z of one
 *     atom adjacent), q and phi are [n].
 *   - The caller owns every input and output buffer; the plan owns its
 *     workspace (sorted atoms, grids, tables) and frees it in msm_destroy.
 *   - Evaluation calls are asynchronous on the given CUDA stream (NULL = the
 *     legacy default stream) and never synchronise the host (msm_eval_host,
 *     msm_parareal, msm_status and msm_debug_grid do, as documented).  msm_eval may
 *     fork part of its work onto a plan-owned stream and joins it back onto
 *     the given stream before returning control of the results (events
 *     only; see msm_set_overlap).  Errors that can
 *     only be seen on the device (an atom outside an open box, a non-finite
 *     input) are posted to a device status word that msm_status reads.
 *   - A plan is not thread-safe: calls on one plan must be ordered (one
 *     stream, or the caller's own synchronisation).
 *   - Every function returns MSM_OK (0) or a negative MSM_ERR_* code.
 */
#ifndef MSM_GB300_H
#define MSM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MSM_OK 0
#define MSM_ERR_INVALID_ARG (-1)        /* bad parameter, NULL pointer, n < 0 */
#define MSM_ERR_UNSUPPORTED (-2)        /* valid but not built (e.g. box too small for the cell walk) */
#define MSM_ERR_CUTOFF_GT_HALF_BOX (-3) /* periodic box with a > L/2 (minimum image fails) */
#define MSM_ERR_ATOM_OUTSIDE_BOX (-4)   /* open box: an atom outside [0, L] (device-detected) */
#define MSM_ERR_NONFINITE (-5)          /* NaN/Inf position or charge (device-detected) */
#define MSM_ERR_OOM (-6)                /* device allocation failed */
#define MSM_ERR_CUDA (-7)               /* a CUDA runtime call failed */
#define MSM_ERR_TIMEOUT (-8)            /* a bounded device wait gave up (the persistent batch chains) */
#define MSM_ERR_TOO_MANY_ATOMS (-9)     /* n > max_atoms of the plan */
#define MSM_ERR_NO_FORWARD (-10)        /* backward called before a forward on this plan */
#define MSM_ERR_STALE_FORWARD (-11)     /* backward of a forward whose buffers a later forward reused */

#define MSM_FP64 0  /* every step in double precision */
#define MSM_MIXED 1 /* pairs and grids in FP32 with compensated sums; top level and energy in FP64 */

typedef struct msm_plan* msm_handle;

/* Parameters of one MSM configuration (Sec. "Multilevel Summation Method"). */
typedef struct {
  double box[3];    /* box edges L_x, L_y, L_z; open boxes require 0 <= x <= L per coordinate */
  int periodic;     /* 1: periodic in x, y and z; 0: open boundaries */
  double cutoff;    /* a: cutoff of the short-range kernel g*; level k reaches 2^(k+1) a */
  double spacing;   /* h: finest grid spacing (periodic: an upper bound, h_eff = L/M0 <= h) */
  int levels;       /* l: number of grids; 0 picks it (top grid <= 8 points per dimension) */
  int order;        /* p: interpolation degree, 3 (cubic, C1) or 5 (quintic, C1) */
  int splitting;    /* m: Taylor smoothing order of gamma, 1 (C1), 2 (C2, printed), 3 (C3) */
  int precision;    /* MSM_FP64 or MSM_MIXED */
  double coulomb_k; /* prefactor k_c (1/(4 pi eps0) in caller units); 1.0 gives e^2/length */
  int64_t max_atoms;/* capacity of the plan's workspace */
} msm_params;

/* Tile shapes of a plan (0 in a field keeps its default).  They change
 * speed, never results beyond floating-point summation order.
 *   cell_fill     target atoms per short-range cell at the plan's capacity
 *                 density (default 24; cells are at least a/2 wide)
 *   patch_cells   short-range cells per side of the shared-memory patch blocks
 *                 of anterpolation and interpolation (default: 4, lowered to
 *                 3 or 2 on a mixed-precision plan evaluated alone while fewer
 *                 than 152 patch blocks cover its box, and lower still where
 *                 the patch would not fit shared memory; batched launches
 *                 keep the largest patch that fits)
 *   lattice_waves blocks per SM the lattice cutoff aims for when it splits the
 *                 stencil planes of a small level over several blocks (default 8)
 *   pair_targets  mixed-precision pair kernel: 32 culls sources against
 *                 the bounding box of up to 32 atoms of a cell, one target
 *                 per lane (the default); 8 against clusters of 8 spatially
 *                 consecutive atoms of a cell (fewer pairs, more culling
 *                 work: measured slower on water)
 *   pair_runs     mixed-precision pair kernel with pair_targets 32: 1 a
 *                 warp takes 32 consecutive atoms of the sorted order as its
 *                 targets (runs across the cells of a row, which binning
 *                 sorts by x), 2 a warp takes one cell's atoms; 0 the
 *                 default, 1 on plans of at least 16,384 cells and 2 below.
 *                 Runs need at least seven cells along x on a periodic plan
 *                 and fall back to cells otherwise
 *   lattice_txn, lattice_tyn  warp tile of the mixed-precision lattice
 *                 kernel: txn lanes of 8 x outputs by tyn lanes of two rows,
 *                 txn * tyn <= 32 (default 4 x 8 on a single system; batched
 *                 launches pick a tile per level size); both 0 or both set
 *   batch_persistent  1: in a batched graph (msm_batch_graph_create, taken
 *                 from the first replica's plan) the restriction and the
 *                 prolongation of each grid sweep run as one cooperative
 *                 launch each, the co-resident blocks meeting at a bounded
 *                 grid barrier between passes (a wait that gives up posts
 *                 MSM_ERR_TIMEOUT to that plan's status), instead of one
 *                 launch per pass (0, the default)
 *   lattice_method  the lattice cutoff of a periodic plan: 1 the direct
 *                 stencil sum over staged shared-memory bricks, 2 the same
 *                 cyclic convolution by FFT (five passes over the levels'
 *                 grids; the kernel's transform computed in FP64 when the
 *                 plan is built) where every lattice level's sizes are c 2^s
 *                 with c a product of 3, 5 and 7, up to 4096; 0 the default,
 *                 2 (measured faster on every periodic workload).  Open
 *                 plans use the stencil; a batched graph takes the FFT when
 *                 every replica's plan did; msm_lattice_method reports the
 *                 form a plan took.
 * Ranges: cell_fill 0..256, patch_cells 0..4, lattice_waves 0..64,
 * pair_targets 0, 8 or 32, batch_persistent 0 or 1, lattice_method 0..2, pair_runs 0..2,
 * lattice_txn and lattice_tyn 0..32 with
 * txn * tyn <= 32 and a staging window that fits shared memory; anything else
 * is INVALID_ARG (checked on the host before any device call; the window
 * check, which needs the plan's stencil, at msm_create_tuned). */
typedef struct {
  int cell_fill;
  int patch_cells;
  int lattice_waves;
  int pair_targets;
  int lattice_txn;
  int lattice_tyn;
  int batch_persistent;
  int lattice_method;
  int pair_runs;
} msm_tuning;

/* Builds a plan: validates params, fixes the grid geometry, builds the
 * level stencil and the top-level kernel (FP64, host) and allocates device
 * workspace for max_atoms atoms on the current device.  Synchronous.
 * UNSUPPORTED also covers a level stencil too wide for the stencil lattice
 * kernel's shared-memory window, 2a/h beyond about 65 grid spacings
 * (MSM_MIXED) or 27 (MSM_FP64) (the usual range is 4 to 10), on a plan that
 * would run that kernel: open plans, lattice_method = 1, or periodic sizes
 * the FFT does not take.  A periodic plan in FFT form has no such limit.
 * Errors: INVALID_ARG, UNSUPPORTED, CUTOFF_GT_HALF_BOX, OOM, CUDA. */
int msm_create(const msm_params* params, msm_handle* out);

/* msm_create with explicit tile shapes (tuning may be NULL: defaults).
 * Errors as msm_create; INVALID_ARG for negative or out-of-range fields. */
int msm_create_tuned(const msm_params* params, const msm_tuning* tuning, msm_handle* out);

/* Frees the plan and its device workspace (synchronises the device). */
void msm_destroy(msm_handle h);

/* Grid geometry of the plan (Sec. "Multilevel Summation Method": level k
 * has spacing 2^k h and nodal basis functions Phi((x - x_mu^k) / (2^k h)) on
 * its points; how many points and where the grids start is not printed and
 * follows the plan's reading of it): h_eff[3] (finest spacing per
 * dimension), the level count, and for level k the point counts
 * dims[3k..3k+2] and the first absolute index lo[3k..3k+2] (0 for periodic
 * grids; grid point i of level k sits at i * 2^k * h_eff).  dims and lo may
 * be NULL, else hold 3*levels ints.  Host only; Errors: INVALID_ARG. */
int msm_query(msm_handle h, double h_eff[3], int* levels, int* dims, int* lo);

/* *method = the lattice-cutoff form plan h evaluates with: 1 the stencil
 * sum, 2 the FFT convolution (msm_tuning.lattice_method).
 * Errors: INVALID_ARG (null handle or pointer). */
int msm_lattice_method(msm_handle h, int* method);

/* The grid geometry msm_create would give these parameters, as msm_query
 * reports it, computed on the host alone: no device call, no allocation (it
 * runs without a GPU).  Errors: those of msm_create's parameter checks. */
int msm_geometry(const msm_params* params, double h_eff[3], int* levels, int* dims, int* lo);

/* One energy+force evaluation (the forward pass): the short-range sum of
 * g* over pairs within a (Eq. msmgrid) and the six steps of the long-range
 * part in the order of Sec. "Multilevel Summation Method" (anterpolation;
 * restriction and lattice cutoff per level; top level; prolongation;
 * interpolation), U_i = k_c (u_i^short + u_i^long), and the forces
 * F_i = -dU/dr_i of Sec. "Simulation loop".
 *   pos    [n][3] double, device; periodic positions may lie anywhere (they are
 *          folded into the box), open ones must lie in [0, L].
 *   q      [n] double, device.
 *   energy [1] double, device: E = 1/2 sum_i q_i phi_i.
 *   phi    [n] double, device or NULL: phi_i = dE/dq_i.
 *   force  [n][3] double, device or NULL: F_i = -dE/dr_i.
 * The plan keeps the sorted atoms and per-atom grid terms of this call for a
 * following msm_eval_backward.  Errors: INVALID_ARG, TOO_MANY_ATOMS, CUDA;
 * ATOM_OUTSIDE_BOX and NONFINITE later through msm_status. */
int msm_eval(msm_handle h, int64_t n, const double* pos, const double* q, double* energy,
             double* phi, double* force, void* cuda_stream);

/* The cutoff method (the simplest coarse propagator G of the parareal
 * section, paragraph "Cutoff Method": the Coulomb law summed only over atoms
 * within a constant cutoff, farther pairs neglected), on this plan's box,
 * cutoff a, precision and coulomb_k:
 *   phi_i = k_c sum_{j != i, r_ij < a} q_j / r_ij (minimum image when
 *   periodic), F_i = -dE/dr_i inside the cutoff, E = 1/2 sum_i q_i phi_i.
 * Arguments, layouts and errors as msm_eval; uses the plan's binning and pair
 * kernel (no grid passes).  A following msm_eval_backward returns
 * NO_FORWARD. */
int msm_cutoff_eval(msm_handle h, int64_t n, const double* pos, const double* q, double* energy,
                    double* phi, double* force, void* cuda_stream);

/* Wolf summation (Wolf, Keblinski, Phillpot and Eggebrecht, J. Chem. Phys.
 * 110, 8254 (1999)), the other coarse function G the proposal lists for the
 * parareal method (Sec. "Proposed Solutions"; the thesis prints no formula),
 * in its damped, shifted-force form (pair potential and force both vanish at
 * the cutoff; the force-shifted variant of Fennell and Gezelter, J. Chem.
 * Phys. 124, 234104 (2006)), on this plan's box, cutoff R = a, precision and
 * coulomb_k:
 *   v(r)  = erfc(alpha r)/r - erfc(alpha R)/R + c1 (r - R) for r < R, else 0,
 *           c1 = erfc(alpha R)/R^2 + (2 alpha/sqrt(pi)) exp(-alpha^2 R^2)/R;
 *   phi_i = k_c [sum_{j != i} q_j v(r_ij) - 2 c_s q_i],
 *           c_s = erfc(alpha R)/(2R) + alpha/sqrt(pi);
 *   E = 1/2 sum_i q_i phi_i,  F_i = -dE/dr_i (minimum image when periodic).
 * alpha >= 0 in inverse length units (alpha = 0: the shifted-force Coulomb
 * cutoff; about 2.4/R is usual).  Arguments, layouts and errors as msm_eval,
 * plus INVALID_ARG for a negative or non-finite alpha; uses the plan's
 * binning and pair kernel (no grid passes).  A following msm_eval_backward
 * returns NO_FORWARD. */
int msm_wolf_eval(msm_handle h, double alpha, int64_t n, const double* pos, const double* q, double* energy,
                  double* phi, double* force, void* cuda_stream);

/* The damping alpha that the MSM_MD_WOLF force of the MD and parareal entry
 * points uses on this plan (default 2.4 / cutoff).  Host only.
 * Errors: INVALID_ARG (negative or non-finite alpha). */
int msm_set_wolf_alpha(msm_handle h, double alpha);

/* Force methods of the MD entry points. */
#define MSM_MD_MSM 0    /* the MSM evaluation (msm_eval) */
#define MSM_MD_CUTOFF 1 /* the cutoff method (msm_cutoff_eval) */
#define MSM_MD_WOLF 2   /* Wolf summation (msm_wolf_eval with the plan's msm_set_wolf_alpha) */

/* Molecular dynamics: nsteps steps of the velocity Verlet scheme (Sec.
 * "Molecular Dynamics", the velocity Verlet equations), each one
 *   v += (dt/2) F inv_mass;  r += dt v  (periodic boxes wrap r into [0, L));
 *   F = force at the new r (method: MSM_MD_MSM, one msm_eval; MSM_MD_CUTOFF,
 *   one msm_cutoff_eval; MSM_MD_WOLF, one msm_wolf_eval with the plan's
 *   damping);  v += (dt/2) F inv_mass.
 *   pos      [n][3] double, device, in/out: r(t0) in, r(t0 + nsteps dt) out.
 *   vel      [n][3] double, device, in/out.
 *   force    [n][3] double, device, in/out: must hold F(r(t0)) of the same
 *            method on entry (from msm_eval / msm_cutoff_eval, or from the
 *            previous call); holds F at the final r.
 *   inv_mass [n] double, device: 1/m_i; 0 fixes the atom (no kick, and it
 *            carries no kinetic energy or momentum).
 *   q        [n] double, device.
 *   records  [nsteps][6] double, device or NULL: per step, after its second
 *            half kick, {potential E, kinetic 1/2 sum m v^2, total, and the
 *            momentum sum m v (x, y, z)}, each reduced in a fixed order.
 * Units are the caller's: the kick is F * inv_mass * dt, so coulomb_k, the
 * masses and dt must be consistent.  Asynchronous on cuda_stream and
 * capturable in a CUDA graph (3 + one evaluation's launches per step).  On
 * systems of at most 262,144 atoms, with nsteps >= 16 and cuda_stream not
 * being captured, one step is captured into a CUDA graph and replayed
 * nsteps times (small systems' steps are bound by launch latency).
 * Errors: INVALID_ARG (n < 0, nsteps < 0, non-finite dt, unknown method,
 * missing buffers), TOO_MANY_ATOMS, CUDA; ATOM_OUTSIDE_BOX (an atom left an
 * open box) and NONFINITE later through msm_status. */
int msm_md_run(msm_handle h, int64_t n, double* pos, double* vel, double* force, const double* inv_mass,
               const double* q, double dt, int nsteps, int method, double* records, void* cuda_stream);

/* msm_md_run for nrep independent systems, replica r holding atoms
 * offsets[r] .. offsets[r+1]-1 of every per-atom array and evaluated by
 * plans[r] (distinct plans); records, when given, is [nrep][nsteps][6].  The
 * replicas run concurrently on a pool of streams forked from cuda_stream
 * and joined back (events only; capturable); when no replica exceeds
 * 262,144 atoms (and nsteps >= 16, cuda_stream not being captured) one step
 * of all replicas is captured into a CUDA graph and replayed, as in
 * msm_md_run.  Errors as msm_eval_batch and msm_md_run. */
int msm_md_run_batch(const msm_handle* plans, int nrep, const int64_t* offsets, double* pos, double* vel,
                     double* force, const double* inv_mass, const double* q, double dt, int nsteps, int method,
                     double* records, void* cuda_stream);

/* Parareal integration of one window (Sec. "Parareal Method", Eq. parareal):
 * time points T_k = T_0 + k dT, k = 0..window, with dT = steps_fine dt_fine;
 * the fine propagator F is steps_fine velocity Verlet steps of dt_fine with
 * the MSM force (fine[k] evaluates the propagation from T_k; the window's
 * propagations run concurrently, one plan each), the coarse propagator G
 * steps_coarse steps of dt_coarse with the force coarse_method of plan
 * coarse (MSM_MD_CUTOFF: the cutoff method, the section's "Cutoff Method";
 * MSM_MD_WOLF: Wolf summation; MSM_MD_MSM: MSM with the coarse plan's own
 * cutoff and grid, the "shorter cutoff" and "coarse grid" options); coarse may be one of fine[].  Each
 * propagation starts by evaluating the force at its starting positions.  Iteration 0 is the coarse sweep lambda_{k+1} =
 * G(lambda_k); each further iteration computes F(lambda_k) for every k, then
 * sweeps lambda_{k+1} = G(lambda_k new) + F(lambda_k old) - G(lambda_k old),
 * positions through the minimum image of F - G and wrapped when periodic.
 * It stops after max_iter iterations or once the largest change of a
 * position, and of a velocity times dT, is at most tol (A).  After
 * `window` iterations the result is the sequential fine trajectory.
 *   pos0, vel0 [n][3], inv_mass [n], q [n]: device, the state at T_0.
 *   lam_pos, lam_vel [window+1][n][3] double, device, out: lambda_0..window.
 *   workspace  device, msm_parareal_workspace(n, window) bytes.
 *   iterations host int or NULL: iterations run (not counting the sweep).
 *   change     host double [max_iter][2] or NULL: per iteration the largest
 *              position change (A) and velocity change.
 * One iteration (the window's fine propagations and the corrected coarse
 * sweep) is captured once into a CUDA graph and replayed.
 * Synchronous: reads the change back after each iteration.  window is 1 to
 * MSM_PARAREAL_MAX_WINDOW.  Errors: INVALID_ARG (also an unknown coarse_method),
 * TOO_MANY_ATOMS, CUDA. */
#define MSM_PARAREAL_MAX_WINDOW 64
int64_t msm_parareal_workspace(int64_t n, int window);
int msm_parareal(const msm_handle* fine, msm_handle coarse, int64_t n, const double* pos0, const double* vel0,
                 const double* inv_mass, const double* q, int window, double dt_fine, int steps_fine,
                 double dt_coarse, int steps_coarse, int coarse_method, int max_iter, double tol, double* lam_pos,
                 double* lam_vel, void* workspace, int* iterations, double* change, void* cuda_stream);

/* Adjoint of one forward pass (the reverse mode of the whole evaluation:
 * Sec. "Multilevel Summation Method", the six steps of the algorithm taken
 * backwards, with F_i = -dU/dr_i of Sec. "Simulation loop").
 *   forward_id  the id msm_forward_id returned right after that forward
 *               pass (msm_eval, msm_eval_f32io, msm_eval_host, a batch or
 *               a graph replay); it must still be the plan's latest forward.
 *   grad_energy dL/dE, [1] double, device.
 *   grad_pos    dL/dr, [n][3] double, device or NULL.
 *   grad_q      dL/dq, [n] double, device or NULL.
 * The long-range part is evaluated by the transposed grid passes
 * (interpolation^T = anterpolation, prolongation^T = restriction, the
 * symmetric lattice and top kernels): the anterpolated adjoint charges are
 * the forward's level-0 charge grid times dL/dE / 2 (the same atoms and
 * weights), from which the sweep rebuilds the adjoint level-0 potential
 * instead of storing any forward potential; the short-range part reuses the
 * per-atom pair sums the forward pass kept.  Asynchronous on cuda_stream.
 * Errors: INVALID_ARG (also forward_id <= 0), NO_FORWARD (no MSM forward on
 * this plan, or the last evaluation was msm_cutoff_eval or msm_wolf_eval),
 * STALE_FORWARD (a later forward has reused the buffers: run the forward
 * again), CUDA. */
int msm_eval_backward(msm_handle h, int64_t forward_id, const double* grad_energy, double* grad_pos,
                      double* grad_q, void* cuda_stream);

/* The id of the plan's latest forward pass (0 when there is none, or after
 * msm_cutoff_eval): ids grow by one with every forward of the plan, and each
 * msm_graph_launch gives every plan of the graph a new one.  Host only.
 * Errors: INVALID_ARG.  (No counterpart in the paper: bookkeeping of the
 * adjoint, above.) */
int msm_forward_id(msm_handle h, int64_t* forward_id);

/* msm_eval with FP32 positions, charges and per-atom outputs (device):
 *   pos [n][3] float, q [n] float, phi [n] float or NULL, force [n][3] float
 *   or NULL; energy stays [1] double.
 * The plan's precision decides the arithmetic exactly as for msm_eval; FP32
 * inputs only skip the FP64 reads, and on a mixed plan the results match
 * msm_eval on the same (float-representable) inputs to FP32 rounding.
 * Errors as msm_eval.  (Interface from the same input/output definition,
 * Sec. "Multilevel Summation Method": charges q_i and positions r_i in, the
 * potential and the forces F_i = -dU/dr_i out.) */
int msm_eval_f32io(msm_handle h, int64_t n, const float* pos, const float* q, double* energy,
                   float* phi, float* force, void* cuda_stream);

/* msm_eval_backward with FP32 outputs grad_pos [n][3] and grad_q [n]
 * (grad_energy stays [1] double).  Follows either msm_eval or
 * msm_eval_f32io.  Errors as msm_eval_backward. */
int msm_eval_backward_f32io(msm_handle h, int64_t forward_id, const double* grad_energy, float* grad_pos,
                            float* grad_q, void* cuda_stream);

/* Same as msm_eval with HOST buffers: copies pos and q to the device, runs
 * the evaluation on the stream, copies energy (and phi/force when non-NULL)
 * back and synchronises the stream before returning.  Pinned host memory
 * makes the copies asynchronous to the host thread; pageable memory works.
 * Device-detected errors are returned directly. */
int msm_eval_host(msm_handle h, int64_t n, const double* pos, const double* q, double* energy,
                  double* phi, double* force, void* cuda_stream);

/* ---- batches of independent systems (replicas) ----
 * Each replica is one evaluation of Sec. "Multilevel Summation Method" as
 * msm_eval; evaluating independent systems side by side is the sampling use
 * of the method (no formula of its own in the paper; the parareal section
 * likewise runs the propagations of a window concurrently).
 * Replica r uses plans[r] (its own box, geometry and workspace; a plan may
 * appear only once in a batch) and the atoms offsets[r] .. offsets[r+1]-1 of
 * the concatenated arrays pos [N][3] and q [N] (device), N = offsets[nrep]
 * (host array of nrep+1 int64, offsets[0] = 0).  energies [nrep] (device)
 * receives one energy per replica; phi [N] and force [N][3] (device, either
 * NULL) the per-atom results in the input order.  The replicas are forked
 * over a pool of library-owned streams and joined back onto cuda_stream with
 * events, so independent small systems run concurrently; the call is
 * asynchronous and can be captured into a CUDA graph.
 * Errors: INVALID_ARG, TOO_MANY_ATOMS, CUDA. */
int msm_eval_batch(const msm_handle* plans, int nrep, const int64_t* offsets, const double* pos, const double* q,
                   double* energies, double* phi, double* force, void* cuda_stream);

/* Adjoint of the latest forward of every plan (msm_eval_batch, or each
 * plan's own last msm_eval on these atoms): grad_energies [nrep] (device) ->
 * grad_pos [N][3], grad_q [N] (device, either NULL), per replica as
 * msm_eval_backward (Sec. "Multilevel Summation Method" taken backwards).
 * No forward id is checked: the caller orders its batch calls.
 * Errors: INVALID_ARG, TOO_MANY_ATOMS, NO_FORWARD, CUDA. */
int msm_eval_backward_batch(const msm_handle* plans, int nrep, const int64_t* offsets, const double* grad_energies,
                            double* grad_pos, double* grad_q, void* cuda_stream);

/* A batched forward (and, when grad_energies is not NULL, its adjoint)
 * captured once into an instantiated CUDA graph on the given buffers; every
 * msm_graph_launch replays all kernels of all replicas with one launch.  When
 * there are several replicas and every plan is MSM_MIXED with one
 * interpolation order and one splitting, each stage is a single kernel launch
 * over all replicas (a block finds its replica in a table of per-replica
 * arguments built here), the pair sums of all replicas running concurrently
 * with their grid passes; otherwise the replicas' own launch sequences are
 * forked over library streams.  With nrep = 1 this is the graph form of one
 * plan's msm_eval (small systems lose most of their launch overhead).  Kernel
 * nodes keep the priority of the stream they were captured from.  The
 * buffers and plans must outlive the graph; inputs may change between
 * replays (same sizes).  Creating the graph uploads the tables (synchronous)
 * and runs no kernel.  Errors: INVALID_ARG, TOO_MANY_ATOMS, OOM, CUDA. */
typedef struct msm_graph* msm_graph_handle;
int msm_batch_graph_create(const msm_handle* plans, int nrep, const int64_t* offsets, const double* pos,
                           const double* q, double* energies, double* phi, double* force,
                           const double* grad_energies, double* grad_pos, double* grad_q, msm_graph_handle* out);
int msm_graph_launch(msm_graph_handle g, void* cuda_stream);
void msm_graph_destroy(msm_graph_handle g);

/* Synchronises the device and returns the first device-posted error of this
 * plan since the previous msm_status call (or MSM_OK), then clears it.
 * Device-posted errors: ATOM_OUTSIDE_BOX, NONFINITE.  (No counterpart in the
 * paper: error reporting of the asynchronous evaluation.) */
int msm_status(msm_handle h);

/* Copies one grid of the last evaluation to HOST memory, as doubles in the
 * layout [dims_z][dims_y][dims_x] of msm_query: which = 0 the charges q^k,
 * which = 1 the potential u^k (after prolongation; level l-1: top level).
 * Synchronous.  For tests and diagnostics. */
int msm_debug_grid(msm_handle h, int level, int which, double* host_out);

/* Stages of one evaluation, in launch order (for msm_profile_read). */
#define MSM_STAGE_BINNING 0       /* cell keys, radix sort, cell starts, gather */
#define MSM_STAGE_SHORT_RANGE 1   /* g* pair sums */
#define MSM_STAGE_ANTERPOLATION 2
#define MSM_STAGE_RESTRICTION 3   /* all levels */
#define MSM_STAGE_LATTICE 4       /* lattice cutoff, all levels */
#define MSM_STAGE_TOP 5
#define MSM_STAGE_PROLONGATION 6  /* all levels */
#define MSM_STAGE_INTERPOLATION 7 /* interpolation, assembly, energy reduction */
#define MSM_NSTAGES 8

/* Concurrency of the forward pass (on by default): after binning, the grid
 * passes (anterpolation through prolongation) run on a stream the plan owns,
 * created at the device's highest priority, concurrently with the short-range
 * pair sums on the caller's stream; the caller's stream waits (event) for the
 * grid before interpolation.  Fork and join are event waits, so a stream
 * capture of the caller's stream takes both branches.  enable = 0 runs every
 * stage on the caller's stream, one after another (stage timings then
 * measure each kernel alone).  Results agree either way up to the rounding
 * order of the atomic sums (the same as between two runs).
 * Errors: INVALID_ARG. */
int msm_set_overlap(msm_handle h, int enable);

/* Diagnostics: enable != 0 makes every following msm_eval and
 * msm_eval_backward record a CUDA event pair around each stage on its stream
 * (events only, no synchronisation).  Disabling keeps what was recorded. */
int msm_profile(msm_handle h, int enable);

/* Synchronises the recorded events and returns, since the previous read:
 * ms[MSM_NSTAGES] the summed device time of each stage (may be NULL),
 * *launches the number of kernels and memset nodes the library enqueued and
 * *evals the number of evaluations (either may be NULL); then resets. */
int msm_profile_read(msm_handle h, double* ms, int64_t* launches, int64_t* evals);

/* Name of a stage (e.g. "short_range"); "?" when out of range. */
const char* msm_stage_name(int stage);

/* Energy E = 1/2 sum_i q_i phi_i from per-atom charges q[n] and potentials
 * phi[n] (double, device), written to energy[1] (double, device), computed in
 * FP64 with a fixed two-pass reduction -- the same reduction msm_eval ends
 * with, for callers that must not allocate device memory (an engine whose
 * pool owns all device memory, or a step loop that cannot afford cudaMalloc,
 * which may synchronise the device).  The paper has no counterpart.
 *   - Allocates nothing: its scratch (one partial sum per 256 atoms) is a
 *     file-scope device array of 65,536 doubles (512 KiB) that every GPU
 *     loading the library holds until the process exits; n is therefore
 *     limited to 16,777,216 atoms, larger n returns MSM_ERR_TOO_MANY_ATOMS.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *   - Every call shares the one array: calls that overlap on the GPU (on
 *     different streams, or from several threads) race.  Each call writes
 *     every partial it reads, so nothing has to be cleared between calls.
 *   - Asynchronous on cuda_stream; no plan is needed.
 * Errors: INVALID_ARG, TOO_MANY_ATOMS, CUDA. */
int msm_energy_noalloc(int64_t n, const double* q, const double* phi, double* energy, void* cuda_stream);

/* Human-readable name of an MSM_ERR_* code. */
const char* msm_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* MSM_GB300_H */
