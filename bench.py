"""Benchmark: MSM energy+force evaluations per second on the 1,066,628-atom
periodic water box (216.8 A, 0.15 M NaCl; a = 12 A, h = 2.5 A, quintic C1
basis, C2 Taylor smoothing), mixed precision, with the plain FP64 GPU path
measured beside it and the FP64 CPU oracle as the reference arm.

One step = one whole evaluation (binning, short-range pairs, anterpolation,
restriction + lattice cutoff on every level, top level, prolongation,
interpolation + energy) on inputs already resident in HBM.  The L2 cache is
flushed (a 512 MB write) between timed steps, outside the timed events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank evaluates its own replica (the single-system
path does not shard); rank 0 prints one JSON line.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth import WORKLOADS  # noqa: E402

METRIC = "MSM energy+force evals/sec at 1.07M atoms (mixed precision; FP64 GPU path beside it)"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK = {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}
N_SM, FP32_LANES, FP64_FMA_PER_SM_CLK = 152, 128, 2


def load_peaks():
    if os.path.exists(PEAKS_FILE):
        p = json.load(open(PEAKS_FILE))
        return p, "measured"
    return FALLBACK, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


# FP32 flop of one evaluation of the short-range pair function with the C2
# splitting (FMA = 2 flop, as in the measured peak): difference 3, r^2 5
# (1 mul + 2 FMA), rsqrt 1, gamma polynomial in r^2 4 (2 FMA), 1/r - gamma/a
# 1, potential accumulate 2, force factor 6 (1/r^2 1, the FMA to 1/r^3 plus
# the derivative polynomial 2, that polynomial's FMA 2, times q_j 1), force
# accumulate 6 (3 FMA): 28.  The clamp of r^2 at a^2 is not counted.
PAIR_FLOP = 28.0


def work_model(plan, n, box, cutoff, order):
    """Algorithmic work per evaluation: each stage's flops and the fewest bytes
    it must move.  The short range counts the method's pairs once (half
    pairs, N (4/3) pi a^3 rho / 2 at the box's mean density) times one pair
    evaluation; evaluating each pair from both atoms is the kernel's choice,
    not the method's work."""
    V = box ** 3
    rho = n / V
    pairs = 0.5 * n * (4.0 / 3.0) * math.pi * cutoff ** 3 * rho   # unordered pairs within a
    W3 = (order + 1) ** 3
    pts = [d[0] * d[1] * d[2] for d in plan.dims]
    lat_pts = sum(pts[:-1])
    if getattr(plan, "lattice_method", "stencil") == "fft":
        # the same convolution by FFT: a complex 3-D transform each way (5 N log2 N
        # flop each, the usual count) and the product by the real K^ (2 N); the
        # fewest bytes are the FP64 charges in and the FP32 potential out (12 per
        # point); the five passes move 80 bytes per point (FP32 complex grid read
        # and written each pass, K^ once, q in, u out)
        fft_flop = sum(10.0 * p * math.log2(p) + 2.0 * p for p in pts[:-1])
        lattice = {"flop": fft_flop, "bytes": 12.0 * lat_pts, "pass_bytes": 80.0 * lat_pts,
                   "units": "%d points, FFT convolution (10 N log2 N + 2 N flop per level)" % lat_pts}
    else:
        taps = plan_taps(plan)
        lattice = {"flop": 2.0 * taps * lat_pts, "bytes": 12.0 * lat_pts,
                   "units": "%d points x %d taps" % (lat_pts, taps)}
    return {
        "short_range": {"flop": PAIR_FLOP * pairs, "bytes": 36.0 * n, "pairs": pairs,
                        "units": "%.4g pairs within a (each counted once) x %g flop" % (pairs, PAIR_FLOP)},
        "lattice_cutoff": lattice,
        "anterpolation": {"flop": 3.0 * W3 * n, "bytes": 32.0 * n + 8.0 * pts[0]},
        "interpolation": {"flop": 8.0 * W3 * n, "bytes": 68.0 * n + 4.0 * pts[0]},
        "binning": {"flop": 0.0, "bytes": 32.0 * n + 4 * 8.0 * n * 2 + 64.0 * n},
    }


def recorded_traffic():
    """DRAM bytes per launch from the committed ncu capture (profiles/roofline_traffic.json),
    for each stage whose kernel source is unchanged since the capture; None otherwise."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    if not os.path.exists(path):
        return {}
    rec = json.load(open(path))
    out = {}
    for stage, k in rec.get("kernels", {}).items():
        src = os.path.join(ROOT, k["source"])
        if os.path.exists(src) and hashlib.sha256(open(src, "rb").read()).hexdigest() == k["sha256"]:
            out[stage] = k["dram_bytes_per_launch"]
    return out


def plan_taps(plan):
    h = plan.h_eff
    a = plan.params.cutoff
    E = [int(math.ceil(2 * a / h[d])) for d in range(3)]
    cnt = 0
    for dz in range(-E[2], E[2] + 1):
        for dy in range(-E[1], E[1] + 1):
            for dx in range(-E[0], E[0] + 1):
                if (dx * h[0]) ** 2 + (dy * h[1]) ** 2 + (dz * h[2]) ** 2 < (2 * a) ** 2:
                    cnt += 1
    return cnt


def run_reference(args):
    """Reference arm: the FP64 CPU oracle, as it stands, on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    import oracle as O
    w = WORKLOADS[args.workload]
    pos, q = w.make()
    P = O.Params(box=(w.box,) * 3, periodic=w.periodic, cutoff=w.cutoff, spacing=w.spacing,
                 levels=w.levels, order=w.order, split=w.split)
    O.lib()
    cores = os.cpu_count()
    times = []
    # each step is one whole evaluation; steps stop once 150 s are spent so the
    # run ends within a few minutes whatever --steps asks
    for _ in range(max(1, args.steps)):
        t0 = time.perf_counter()
        O.msm(P, pos, q)
        times.append(time.perf_counter() - t0)
        if sum(times) > 150.0:
            break
    v = len(times) / sum(times)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "evals/s", "n_gpus": args.gpus,
        "steps": len(times), "warmup": 0, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": args.workload, "atoms": w.n_atoms},
        "cpu_baseline": {"value": v, "unit": "evals/s", "cores": cores, "kind": "oracle",
                         "sample": "%d whole evaluation(s) of the %d-atom system" % (len(times), w.n_atoms)},
        "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def cpu_baseline(w, budget_s=30.0):
    """One whole oracle evaluation of the same system on the host cores;
    returns (the baseline entry, the oracle's result)."""
    import oracle as O
    pos, q = w.make()
    P = O.Params(box=(w.box,) * 3, periodic=w.periodic, cutoff=w.cutoff, spacing=w.spacing,
                 levels=w.levels, order=w.order, split=w.split)
    O.lib()
    t0 = time.perf_counter()
    ref = O.msm(P, pos, q)
    t = time.perf_counter() - t0
    return ({"value": 1.0 / t, "unit": "evals/s", "cores": os.cpu_count(), "kind": "oracle",
             "sample": "1 whole evaluation of the %d-atom system (%.1f s)" % (w.n_atoms, t)}, ref)


def errors_vs(E, phi, F, ref):
    """Energy relative error, force and potential rel-RMS, and the worst atom's
    force error over the RMS force, against a reference (numpy arrays)."""
    import numpy as np
    dF = np.sqrt(((F - ref["F"]) ** 2).sum(1))
    sF = float(np.sqrt((ref["F"] ** 2).sum(1).mean()))
    return {"energy_rel": abs(E - ref["E"]) / abs(ref["E"]),
            "force_rel_rms": float(np.sqrt(((F - ref["F"]) ** 2).sum() / (ref["F"] ** 2).sum())),
            "phi_rel_rms": float(np.sqrt(((phi - ref["phi"]) ** 2).sum() / (ref["phi"] ** 2).sum())),
            "force_worst_atom_over_rms": float(dF.max() / sF)}


def config_errors(dev):
    """The two small configurations against the FP64 oracle, every atom: the
    3,000-atom open water box (cubic, C1; also against the direct Coulomb
    sum, the method's own error) and the 23,558-atom periodic box (cubic,
    C2, net +2 e), both GPU paths, with their evaluations per second (back
    to back, eager and replayed from a one-plan graph; inputs stay in L2 at
    this size)."""
    import torch
    import oracle as O
    from paper_1402_7216_gb300 import MSM
    out = {}
    for name in ("water3k_open", "water23k"):
        w = WORKLOADS[name]
        pos, q = w.make()
        P = O.Params(box=(w.box,) * 3, periodic=w.periodic, cutoff=w.cutoff, spacing=w.spacing,
                     levels=w.levels, order=w.order, split=w.split)
        ref = O.msm(P, pos, q)
        e = {"atoms": len(q)}
        tp, tq = torch.tensor(pos, device=dev), torch.tensor(q, device=dev)
        stream = torch.cuda.current_stream()

        def rate(fn, steps=50):
            for _ in range(5):
                fn()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(steps):
                fn()
            b.record(stream)
            torch.cuda.synchronize()
            return steps / (a.elapsed_time(b) * 1e-3)
        for precision in ("mixed", "fp64"):
            plan = MSM(box=w.box, periodic=w.periodic, cutoff=w.cutoff, spacing=w.spacing, levels=w.levels,
                       order=w.order, splitting=w.split, precision=precision, max_atoms=len(q))
            E, phi, F = plan.eval(tp, tq)
            torch.cuda.synchronize()
            plan.check_status()
            e[precision] = errors_vs(E.item(), phi.cpu().numpy(), F.cpu().numpy(), ref)
            # evaluations per second on this small system: eager launches, and the
            # one-plan CUDA graph (launch latency dominates at this size)
            e[precision]["evals_per_s_eager"] = rate(lambda: plan.eval(tp, tq, out=(E, phi, F)))
            g = plan.graph(tp, tq, E.reshape(1), phi, F)
            e[precision]["evals_per_s_graph"] = rate(g.launch)
            g.close()
            plan.check_status()
            plan.close()
        if not w.periodic:
            d = O.direct_sum(pos, q)
            e["oracle_vs_direct_sum"] = errors_vs(ref["E"], ref["phi"], ref["F"], d)
        out[name] = e
    return out


def bench_large(dev, args):
    """The 4.1M-atom box (340 A, a = 10, h = 1.5 -> 240^3, quintic, 5 levels),
    mixed precision: forward (E, phi, F) and adjoint (dE/dr, dE/dq; the
    adjoint rebuilds the level-0 potential instead of storing it) timed with
    CUDA events, the device memory they hold, and both against the FP64 GPU
    path (the host oracle cannot afford a full evaluation at this size)."""
    import torch
    from paper_1402_7216_gb300 import MSM
    w = WORKLOADS["water4m"]
    pos_h, q_h = w.make()
    n = len(q_h)
    pos, q = torch.tensor(pos_h, device=dev), torch.tensor(q_h, device=dev)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats(dev)
    free0 = torch.cuda.mem_get_info(dev)[0]
    # the lattice form (FFT or stencil) and, for the stencil, the warp tile of
    # the finest grid, and the pair kernel's target grouping, from the
    # project's autotuner, timed on forward + adjoint
    from paper_1402_7216_gb300.autotune import TILES, autotune
    tuning, tune_ms = autotune(pos, q, w.box, True, w.cutoff, w.spacing, levels=w.levels, order=w.order,
                               splitting=w.split, precision="mixed", reps=3,
                               search=[("lattice_method", [1]), ("pair_runs", [1, 2]), ("lattice_tile", TILES)],
                               backward=True)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(dev)[0]
    plan = MSM(box=w.box, periodic=True, cutoff=w.cutoff, spacing=w.spacing, levels=w.levels, order=w.order,
               splitting=w.split, precision="mixed", max_atoms=n, tuning=tuning)
    workspace = free0 - torch.cuda.mem_get_info(dev)[0]
    E = torch.empty((), dtype=torch.float64, device=dev)
    phi = torch.empty(n, dtype=torch.float64, device=dev)
    F = torch.empty((n, 3), dtype=torch.float64, device=dev)
    gE = torch.ones((), dtype=torch.float64, device=dev)
    for _ in range(2):
        plan.eval(pos, q, out=(E, phi, F))
        gp, gq = plan.backward(gE)
    torch.cuda.synchronize()
    steps = max(3, args.steps // 5)
    tf, tb = [], []
    for _ in range(steps):
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record(stream)
        plan.eval(pos, q, out=(E, phi, F))
        b.record(stream)
        gp, gq = plan.backward(gE)
        c.record(stream)
        torch.cuda.synchronize()
        tf.append(a.elapsed_time(b))
        tb.append(b.elapsed_time(c))
    plan.check_status()
    peak_torch = torch.cuda.max_memory_allocated(dev)
    Em, phim, Fm, gpm, gqm = E.item(), phi.cpu().numpy(), F.cpu().numpy(), gp.cpu().numpy(), gq.cpu().numpy()
    plan.close()
    plan64 = MSM(box=w.box, periodic=True, cutoff=w.cutoff, spacing=w.spacing, levels=w.levels, order=w.order,
                 splitting=w.split, precision="fp64", max_atoms=n)
    E64, phi64, F64 = plan64.eval(pos, q)
    gp64, gq64 = plan64.backward(gE)
    torch.cuda.synchronize()
    plan64.check_status()
    ref = {"E": E64.item(), "phi": phi64.cpu().numpy(), "F": F64.cpu().numpy()}
    import numpy as np
    err = errors_vs(Em, phim, Fm, ref)
    err["adjoint_dE_dr_rel_rms"] = float(np.sqrt(((gpm - gp64.cpu().numpy()) ** 2).sum() /
                                                 (gp64.cpu().numpy() ** 2).sum()))
    err["adjoint_dE_dq_rel_rms"] = float(np.sqrt(((gqm - gq64.cpu().numpy()) ** 2).sum() /
                                                 (gq64.cpu().numpy() ** 2).sum()))
    plan64.close()
    fm, bm = sorted(tf)[len(tf) // 2], sorted(tb)[len(tb) // 2]
    return {"workload": "water4m: periodic 340 A, 1,364,300 waters + 3,550 Na+ + 3,550 Cl- (%d atoms); a=10, h=1.5 "
                        "(240^3), quintic, C2, 5 levels, mixed" % n,
            "metric": "energy+force+adjoint evaluations per second", "value": 1e3 / (fm + bm),
            "unit": "evals/s", "forward_ms": fm, "backward_ms": bm, "steps": steps,
            "device_memory_GB": {"plan_workspace": workspace / 1e9, "caller_tensors_peak": peak_torch / 1e9,
                                 "budget": 180.0},
            "tuning": tuning, "autotune_ms": {k: (round(v, 3) if isinstance(v, float) else v)
                                              for k, v in tune_ms.items()},
            "mixed_vs_fp64_gpu": err,
            "timing": "CUDA events around each forward and each adjoint (inputs and grids exceed L2)"}


def bench_batch(dev, args, n_rep=64):
    """The 64-replica batch; under torchrun each rank takes its share of the
    replicas (balanced by atoms, no collective on the data path) and the
    job's time per batch is the slowest rank's."""
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1402_7216_gb300 import MSM, MSMBatch
    from paper_1402_7216_gb300.shard import max_over_ranks, shard_replicas
    from synth import replica_boxes
    from paper_1402_7216_gb300.autotune import autotune_batch
    reps_all = replica_boxes(n_rep)
    world = dist.get_world_size() if dist.is_initialized() else 1
    rank = dist.get_rank() if dist.is_initialized() else 0
    mine = shard_replicas([len(q) for (_, _, q) in reps_all], world)[rank]
    reps = [reps_all[i] for i in mine]
    n_rep_all, n_rep = n_rep, len(reps)
    counts = [len(q) for (_, _, q) in reps]
    n = sum(counts)
    pos = torch.tensor(np.vstack([p for (_, p, _) in reps]), device=dev)
    q = torch.tensor(np.concatenate([qq for (_, _, qq) in reps]), device=dev)
    # tile shapes from the project's autotuner (timed on the batch graph): the
    # fields every replica shares, and a lattice tile per finest-grid size
    tunings, tuning, tune_ms = autotune_batch([L for (L, _, _) in reps], pos, q, counts, cutoff=10.0, spacing=2.0,
                                              order=3, splitting=2, reps=3)
    plans = [MSM(box=L, periodic=True, cutoff=10.0, spacing=2.0, order=3, splitting=2, precision="mixed",
                 max_atoms=len(q), tuning=t) for (L, _, q), t in zip(reps, tunings)]
    E = torch.zeros(n_rep, dtype=torch.float64, device=dev)
    F = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    phi = torch.zeros(n, dtype=torch.float64, device=dev)
    gE = torch.ones(n_rep, dtype=torch.float64, device=dev)
    gp = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    gq = torch.zeros(n, dtype=torch.float64, device=dev)
    batch = MSMBatch(plans)
    graph = batch.graph(pos, q, counts, E, phi, F, gE, gp, gq)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        graph.launch()
    torch.cuda.synchronize()
    steps = max(5, args.steps // 5)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for a, b in ev:
        flush.fill_(1.0)
        a.record(stream)
        graph.launch()
        b.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = [a.elapsed_time(b) for a, b in ev]
    # the same work as separate calls on one stream (no graph, no fork)
    seq = []
    for _ in range(3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(1.0)
        a.record(stream)
        o = 0
        for r, p in enumerate(plans):
            c = counts[r]
            p.eval(pos[o:o + c], q[o:o + c], want_phi=False, want_force=False)
            p.backward(gE[r], want_pos=True, want_q=True)
            o += c
        b.record(stream)
        torch.cuda.synchronize()
        seq.append(a.elapsed_time(b))
    for p in plans:
        p.check_status()
    # three replicas (smallest, median, largest) of the last replay against
    # the FP64 oracle, every atom
    import oracle as O
    graph.launch()
    torch.cuda.synchronize()
    Eh, phih, Fh = E.cpu().numpy(), phi.cpu().numpy(), F.cpu().numpy()
    order = sorted(range(n_rep), key=lambda r: counts[r])
    off = np.concatenate([[0], np.cumsum(counts)])
    rep_err = {}
    for r in (order[0], order[n_rep // 2], order[-1]):
        L, p_r, q_r = reps[r]
        ref = O.msm(O.Params(box=(L,) * 3, periodic=True, cutoff=10.0, spacing=2.0, order=3, split=2), p_r, q_r)
        rep_err["replica_%d_%d_atoms" % (mine[r], counts[r])] = errors_vs(
            float(Eh[r]), phih[off[r]:off[r + 1]], Fh[off[r]:off[r + 1]], ref)
    graph.close()
    t = max_over_ranks(sum(ms) / len(ms), device=dev)
    return {"metric": "replica energy+force+adjoint evaluations per second (one graph launch = all replicas)",
            "value": n_rep_all / (t * 1e-3), "unit": "replica-evals/s", "replicas": n_rep_all,
            "replicas_per_rank": n_rep, "atoms_total": sum(len(q) for (_, _, q) in reps_all),
            "atoms_min": min(len(q) for (_, _, q) in reps_all), "atoms_max": max(len(q) for (_, _, q) in reps_all),
            "ms_per_batch": t, "steps": steps,
            "ms_per_batch_sequential_calls": min(seq), "tuning": tuning,
            "errors_vs_oracle": rep_err,
            "autotune_ms": {k: (round(v, 4) if isinstance(v, float) else v) for k, v in tune_ms.items()},
            "config": "periodic water boxes at 0.1 atoms/A^3, a=10, h=2.0, cubic, C2, mixed precision, "
                      "forward + adjoint, one CUDA graph (each stage one launch over all replicas), "
                      "autotuned tile shapes, L2 flushed between steps"}


def parareal_timings(args, w, plan, pos, q, n, dev, stream, flush, f_ms, E_mix, F_mix):
    """The parareal section's coarse propagators G on the same system: the
    cutoff method (Coulomb law within a) and MSM with a shorter cutoff or a
    coarser grid, each timed against the MSM evaluation (F, f_ms per eval)."""
    import torch
    from paper_1402_7216_gb300 import MSM
    # the cutoff method on the same system and cutoff (the parareal section's
    # coarse propagator G): its evaluation time against MSM's (F)
    E_c = torch.empty((), dtype=torch.float64, device=dev)
    phi_c = torch.empty(n, dtype=torch.float64, device=dev)
    F_c = torch.empty((n, 3), dtype=torch.float64, device=dev)
    for _ in range(3):
        plan.cutoff_eval(pos, q, out=(E_c, phi_c, F_c))
    torch.cuda.synchronize()
    ms_g = []
    for _ in range(max(3, args.steps // 4)):
        flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plan.cutoff_eval(pos, q, out=(E_c, phi_c, F_c))
        b.record(stream)
        torch.cuda.synchronize()
        ms_g.append(a.elapsed_time(b))
    plan.check_status()
    g_ms = sorted(ms_g)[len(ms_g) // 2]
    cutoff_G = {"metric": "cutoff-method energy+force evals/sec on the same system (Coulomb law within a = %g A)"
                          % w.cutoff, "value": 1e3 / g_ms, "unit": "evals/s", "ms_per_eval": g_ms,
                "msm_ms_per_eval": f_ms, "ratio_F_over_G": f_ms / g_ms,
                "paper_ratio_estimate": {"value": 60, "basis": "operation counts, MSM a=12, h=2, h*=1 A, C2, "
                                                              "cubic against a 12 A cutoff (no hardware)"},
                "energy_cutoff_vs_msm_rel": abs(E_c.item() - E_mix) / abs(E_mix)}
    # Wolf summation (damped, shifted force, alpha = 0.2/A, R = a): the
    # section's other coarse function, timed the same way
    alpha_w = 0.2
    for _ in range(3):
        plan.wolf_eval(pos, q, alpha_w, out=(E_c, phi_c, F_c))
    torch.cuda.synchronize()
    ms_w = []
    for _ in range(max(3, args.steps // 4)):
        flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plan.wolf_eval(pos, q, alpha_w, out=(E_c, phi_c, F_c))
        b.record(stream)
        torch.cuda.synchronize()
        ms_w.append(a.elapsed_time(b))
    plan.check_status()
    w_ms = sorted(ms_w)[len(ms_w) // 2]
    dFw = float(torch.sqrt(((F_c - F_mix) ** 2).sum() / (F_mix ** 2).sum()))
    wolf_G = {"metric": "Wolf-summation energy+force evals/sec on the same system (damped shifted force, "
                                  "alpha = %g /A, R = a = %g A)" % (alpha_w, w.cutoff),
                        "value": 1e3 / w_ms, "unit": "evals/s", "ms_per_eval": w_ms, "ratio_F_over_G": f_ms / w_ms,
                        "energy_wolf_vs_msm_rel": abs(E_c.item() - E_mix) / abs(E_mix), "force_rel_rms_vs_F": dFw}
    plan.eval(pos, q)  # leave the plan holding an MSM forward pass

    # MSM itself as the coarse propagator (the parareal section's "shorter
    # cutoff" and "coarse grid" options): time, F/G and the force error
    # against the fine configuration
    def g_variant(cutoff, spacing):
        pg = MSM(box=w.box, periodic=w.periodic, cutoff=cutoff, spacing=spacing, levels=0, order=w.order,
                 splitting=w.split, precision="mixed", max_atoms=n)
        Eg, _, Fg = pg.eval(pos, q)
        for _ in range(2):
            pg.eval(pos, q)
        torch.cuda.synchronize()
        tg = []
        for _ in range(max(3, args.steps // 4)):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pg.eval(pos, q, out=(Eg, None, Fg))
            b.record(stream)
            torch.cuda.synchronize()
            tg.append(a.elapsed_time(b))
        pg.check_status()
        gm = sorted(tg)[len(tg) // 2]
        dF = float(torch.sqrt(((Fg - F_mix) ** 2).sum() / (F_mix ** 2).sum()))
        out = {"cutoff_A": cutoff, "spacing_A": spacing, "h_eff_A": pg.h_eff[0], "grid0": pg.dims[0],
               "ms_per_eval": gm, "ratio_F_over_G": f_ms / gm, "force_rel_rms_vs_F": dF,
               "energy_rel_vs_F": abs(Eg.item() - E_mix) / abs(E_mix)}
        pg.close()
        return out
    msm_G = {"shorter_cutoff": g_variant(0.5 * w.cutoff, w.spacing),
             "coarser_grid": g_variant(w.cutoff, 4.0 * w.spacing),
             "paper_estimates": "shorter cutoff (6 vs 12 A): at most 7x theoretical speed-up, force error "
                                "1-5 % from 8 A (Hardy); coarser grid: little gain, the work depends mainly on a"}
    return cutoff_G, msm_G, wolf_G


def md_timing(args, plan, pos, q, n, stream, f_ms):
    """Velocity Verlet steps around the MSM force (msm_md_run) on the same
    system: one call runs every timed step back to back; its working set
    (positions, velocities, forces, sorted atoms, grid coordinates, about
    160 MB) is larger than L2, so no flush is needed between its steps."""
    import torch
    r = pos.clone()
    v = torch.zeros_like(r)
    inv_mass = torch.full((n,), 1.0 / 18.0, dtype=torch.float64, device=r.device)
    F, _ = plan.md_run(r, v, inv_mass, q, 1e-3, 3)  # evaluates F(r) first
    torch.cuda.synchronize()
    steps = max(10, args.steps // 2)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    _, rec = plan.md_run(r, v, inv_mass, q, 1e-3, steps, force=F)
    b.record(stream)
    torch.cuda.synchronize()
    plan.check_status()
    ms = a.elapsed_time(b) / steps
    return {"metric": "velocity Verlet MD steps/sec on the same system (one msm_md_run call of %d steps)" % steps,
            "value": 1e3 / ms, "unit": "steps/s", "ms_per_step": ms, "msm_ms_per_eval": f_ms,
            "integrator_overhead_ms": ms - f_ms, "records_finite": bool(torch.isfinite(rec).all().item())}


def parareal_window_timing(coarse_method="cutoff", coarse_cutoff=10.0, window=8, steps_fine=10, dt_fine=0.05,
                           steps_coarse=2, dt_coarse=0.25, tol=1e-4):
    """One parareal window (msm_parareal) on a 23,558-ion one-component
    plasma in the 62.2 A periodic box of the 23,558-atom configuration (a =
    10 A, h = 2 A, cubic, mixed precision; unit masses, kT = 0.05 in
    e^2/A): its wall time against the sequential fine run over the same
    time span, the iterations it needs to tol and each iteration's change.
    The fine propagations of a window run concurrently, one plan each."""
    import torch
    from paper_1402_7216_gb300 import MSM, parareal
    from synth import make_ion_system
    L, n = 62.2, 23558
    pos, q, im, vel = make_ion_system(L, n, seed=61, kind="plasma", dmin=2.0)
    dev = torch.device("cuda", torch.cuda.current_device())
    tp, tv, ti, tq = (torch.tensor(a, device=dev) for a in (pos, vel, im, q))

    def mk():
        return MSM(box=L, periodic=True, cutoff=10.0, spacing=2.0, order=3, splitting=2, precision="mixed",
                   max_atoms=n)
    fine = [mk() for _ in range(window)]
    coarse = MSM(box=L, periodic=True, cutoff=coarse_cutoff, spacing=2.0, order=3, splitting=2, precision="mixed",
                 max_atoms=n)
    stream = torch.cuda.current_stream()
    # sequential fine run over window * steps_fine steps
    sp, sv = tp.clone(), tv.clone()
    fine[0].md_run(tp.clone(), tv.clone(), ti, tq, dt_fine, 2)   # warm-up
    F, _ = fine[0].md_run(sp, sv, ti, tq, dt_fine, 0)            # the force at the start
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    fine[0].md_run(sp, sv, ti, tq, dt_fine, window * steps_fine, force=F, records=False)
    b.record(stream)
    torch.cuda.synchronize()
    t_seq = a.elapsed_time(b)
    parareal(fine, coarse, tp, tv, ti, tq, window, dt_fine, steps_fine, dt_coarse, steps_coarse, 1, 0.0,
             coarse_method=coarse_method)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lp, lv, iters, ch = parareal(fine, coarse, tp, tv, ti, tq, window, dt_fine, steps_fine, dt_coarse,
                                 steps_coarse, window, tol, coarse_method=coarse_method)
    t_par = 1e3 * (time.perf_counter() - t0)
    d = lp[window] - sp
    err = float((d - L * torch.round(d / L)).abs().max())
    for p in fine + [coarse]:
        p.close()
    return {"workload": "plasma23k: 23,558 ions (+1 e, unit mass) in the 62.2 A periodic box, a=10, h=2, cubic, "
                        "mixed; kT=0.05 e^2/A",
            "window": window, "fine": "%d steps x dt %g (MSM)" % (steps_fine, dt_fine),
            "coarse": "%d steps x dt %g (%s, a=%g A)" % (steps_coarse, dt_coarse,
                                                         {"cutoff": "cutoff method", "msm": "MSM",
                                                          "wolf": "Wolf summation, alpha = 2.4/a"}[coarse_method],
                                                         coarse_cutoff),
            "tol_A": tol, "iterations": iters, "change_per_iteration": [[float(x) for x in c] for c in ch],
            "ms_parareal": t_par, "ms_sequential_fine": t_seq, "speedup": t_seq / t_par,
            "final_point_vs_sequential_A": err,
            "timing": "parareal: host wall clock of the synchronous call; sequential: CUDA events"}


def load_fma_probe():
    """bench's FP32 FMA probe library (fma_probe.cu, built beside this file)."""
    import ctypes
    from __graft_entry__ import build_fma_probe
    L = ctypes.CDLL(build_fma_probe())
    L.fma_probe.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    L.fma_probe.restype = ctypes.c_int
    return L


def fma_probe(dev, iters=1 << 16, blocks=152 * 8):
    """Measured FP32 FMA throughput (fma_probe.cu): packed two-lane and
    scalar FMA chains over every SM, median of 5 timed launches, TFLOP/s."""
    import ctypes
    import torch
    L = load_fma_probe()
    out = torch.empty(blocks * 256, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    res = {}
    for packed in (1, 0):
        def launch():
            rc = L.fma_probe(packed, iters, blocks, ctypes.c_void_p(out.data_ptr()),
                             ctypes.c_void_p(stream.cuda_stream))
            if rc != 0:
                raise RuntimeError("fma_probe failed: %d" % rc)
        for _ in range(3):
            launch()
        ts = []
        for _ in range(5):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            launch()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        ms = sorted(ts)[2]
        res["packed" if packed else "scalar"] = blocks * 256 * iters * 32 / (ms * 1e-3) / 1e12
    res["finite"] = bool(torch.isfinite(out).all().item())
    return res


def run_profile_case(args):
    """One section of the bench alone on cuda:0 (for ncu captures)."""
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    if args.profile_case == "batch":
        out = bench_batch(dev, args)
    elif args.profile_case == "large":
        out = bench_large(dev, args)
    else:
        from paper_1402_7216_gb300 import MSM
        w = WORKLOADS[args.workload]
        pos_h, q_h = w.make()
        pos, q = torch.tensor(pos_h, device=dev), torch.tensor(q_h, device=dev)
        plan = MSM(box=w.box, periodic=w.periodic, cutoff=w.cutoff, spacing=w.spacing, levels=w.levels,
                   order=w.order, splitting=w.split, precision="mixed", max_atoms=len(q_h),
                   tuning=json.loads(args.tuning) if args.tuning else None)
        plan.set_overlap(False)
        for _ in range(args.warmup + args.steps):
            plan.eval(pos, q, want_phi=False, want_force=False)
        torch.cuda.synchronize()
        plan.check_status()
        out = {"workload": args.workload, "evaluations": args.warmup + args.steps, "lattice": plan.lattice_method,
               "levels": plan.levels, "dims": plan.dims, "tuning": plan.tuning}
    print(json.dumps({"profile_case": args.profile_case, "result": out}, default=str))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="water1m")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-parareal", action="store_true", help="skip the coarse-propagator timings")
    ap.add_argument("--no-md", action="store_true", help="skip the velocity Verlet timing")
    ap.add_argument("--no-large", action="store_true", help="skip the 4.1M-atom forward + adjoint timing")
    ap.add_argument("--profile-case", choices=["evals", "batch", "large"],
                    help="run one section alone and print its JSON (the commands the ncu summaries in profiles/ "
                         "use): 'evals' builds the benchmark system's default plan and runs --warmup then --steps "
                         "plain evaluations; 'batch' the 64-replica batch; 'large' the 4.1M-atom box")
    ap.add_argument("--tuning", default=None,
                    help="msm_tuning fields as JSON for --profile-case evals (e.g. the autotuner's choice)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_case:
        return run_profile_case(args)

    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1402_7216_gb300 import MSM

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    w = WORKLOADS[args.workload]
    pos_h, q_h = w.make()
    n = len(q_h)
    pos = torch.tensor(pos_h, device=dev)
    q = torch.tensor(q_h, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def make(precision):
        return MSM(box=w.box, periodic=w.periodic, cutoff=w.cutoff, spacing=w.spacing, levels=w.levels,
                   order=w.order, splitting=w.split, precision=precision, max_atoms=n)

    def timed(plan, steps, warmup, profile=False):
        E = torch.empty((), dtype=torch.float64, device=dev)
        phi = torch.empty(n, dtype=torch.float64, device=dev)
        F = torch.empty((n, 3), dtype=torch.float64, device=dev)
        for _ in range(warmup):
            plan.eval(pos, q, out=(E, phi, F))
        torch.cuda.synchronize()
        plan.check_status()
        plan.profile_read()
        if profile:
            plan.profile(True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        for a, b in ev:
            flush.fill_(1.0)                     # L2 flush, outside the timed events
            a.record(stream)
            plan.eval(pos, q, out=(E, phi, F))
            b.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        plan.profile(False)
        ms = [a.elapsed_time(b) for a, b in ev]
        prof = plan.profile_read()
        plan.check_status()
        return ms, prof, (E.item(), phi, F)

    # mixed precision (the headline), with the tile shapes of the project's
    # autotuner (each candidate timed on this system's own evaluations)
    from paper_1402_7216_gb300.autotune import autotune
    head_tuning, head_tune_ms = autotune(pos, q, w.box, w.periodic, w.cutoff, w.spacing, levels=w.levels,
                                         order=w.order, splitting=w.split, precision="mixed", reps=5)
    plan = MSM(box=w.box, periodic=w.periodic, cutoff=w.cutoff, spacing=w.spacing, levels=w.levels,
               order=w.order, splitting=w.split, precision="mixed", max_atoms=n, tuning=head_tuning)
    clocks = ClockSampler(local)
    clocks.start()
    ms, (stage_ms, launches, evals), (E_mix, phi_mix, F_mix) = timed(plan, args.steps, max(3, args.warmup), True)
    clk = clocks.stop()
    tot = sum(ms)
    if world > 1:
        t = torch.tensor([tot], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot = t.item()
    value = world * args.steps / (tot / 1e3)

    # the same evaluation with every stage in turn on one stream (no overlap):
    # per-kernel times without the concurrent grid passes, for context
    plan.set_overlap(False)
    ms_iso, (stage_iso, _, evals_iso), _ = timed(plan, max(3, args.steps // 4), 2, True)
    plan.set_overlap(True)

    cutoff_G = msm_G = wolf_G = md = None
    f_ms = sorted(ms)[len(ms) // 2]
    if not args.no_parareal:
        cutoff_G, msm_G, wolf_G = parareal_timings(args, w, plan, pos, q, n, dev, stream, flush, f_ms, E_mix, F_mix)
    if not args.no_md:
        md = md_timing(args, plan, pos, q, n, stream, f_ms)
    pr_window = None
    if not args.no_parareal:
        pr_window = [parareal_window_timing("cutoff", 10.0), parareal_window_timing("msm", 5.0),
                     parareal_window_timing("wolf", 10.0)]

    # end to end through the host-buffer entry point (pinned host memory):
    # positions and charges in, energy, potentials and forces out, every step
    pos_pin = torch.tensor(pos_h).pin_memory()
    q_pin = torch.tensor(q_h).pin_memory()
    host_out = (torch.empty((), dtype=torch.float64).pin_memory(), torch.empty(n, dtype=torch.float64).pin_memory(),
                torch.empty((n, 3), dtype=torch.float64).pin_memory())
    for _ in range(2):
        plan.eval_host(pos_pin, q_pin, out=host_out)
    torch.cuda.synchronize()
    e2e_t = []
    for _ in range(max(3, args.steps // 3)):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.eval_host(pos_pin, q_pin, out=host_out)
        e2e_t.append(time.perf_counter() - t0)
    e2e_tot = sum(e2e_t)
    if world > 1:
        t = torch.tensor([e2e_tot], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_tot = t.item()
    e2e_value = world * len(e2e_t) / e2e_tot

    # plain FP64 GPU path at the same parameters, and the mixed path's error against it
    fp64 = None
    if not args.no_fp64:
        plan64 = make("fp64")
        ms64, prof64, (E64, phi64, F64) = timed(plan64, max(3, args.steps // 6), 2, True)
        fp64 = {"value": len(ms64) / (sum(ms64) / 1e3), "unit": "evals/s",
                "ms_per_step": sum(ms64) / len(ms64),
                "stage_ms": {k: v / prof64[2] for k, v in prof64[0].items()}}
        Fm, Fd = F_mix.double(), F64.double()
        fp64["mixed_vs_fp64"] = {
            "energy_rel": abs(E_mix - E64) / abs(E64),
            "force_rel_rms": float(torch.sqrt(((Fm - Fd) ** 2).sum() / (Fd ** 2).sum())),
            "phi_rel_rms": float(torch.sqrt(((phi_mix - phi64) ** 2).sum() / (phi64 ** 2).sum()))}
        plan64.close()

    # batched replicas: 64 periodic water boxes, N log-uniform in [5k, 50k] at
    # 0.1 atoms/A^3, a = 10, h = 2.0, cubic, mixed precision; forward + adjoint
    # of all replicas replayed from one captured CUDA graph
    batched = None
    if not args.no_batch:
        batched = bench_batch(dev, args)
    large = None
    if not args.no_large and world == 1:
        large = bench_large(dev, args)
    cfg_err = None
    if not args.no_cpu_baseline and world == 1:
        cfg_err = config_errors(dev)

    if rank != 0:
        return
    peaks, peak_kind = load_peaks()
    hbm = peaks.get("hbm_gbs", FALLBACK["hbm_gbs"])
    sm_max = peaks.get("sm_max_mhz", FALLBACK["sm_max_mhz"])
    fp32_derived = N_SM * FP32_LANES * 2 * sm_max * 1e6 / 1e12    # TFLOP/s, FMA = 2 flop
    probe = fma_probe(dev)
    fp32_peak = max(probe["packed"], probe["scalar"])              # measured: the ALU kernels' denominator
    per_eval = {k: v / evals for k, v in stage_ms.items()}
    model = work_model(plan, n, w.box, w.cutoff, w.order)
    kernels = {}
    for k, v in per_eval.items():
        e = {"ms": v}
        if k in model and v > 0:
            e["gflop_s"] = model[k]["flop"] / (v * 1e-3) / 1e9
            e["hbm_gb_s_algorithmic"] = model[k]["bytes"] / (v * 1e-3) / 1e9
            e["frac_fp32_peak"] = e["gflop_s"] / (fp32_peak * 1e3)
            e["frac_hbm_peak"] = e["hbm_gb_s_algorithmic"] / hbm
        kernels[k] = e
    traffic = recorded_traffic()
    for k, e in kernels.items():
        if k in traffic:
            e["dram_bytes_ncu"] = traffic[k]
    per_iso = {k: v / evals_iso for k, v in stage_iso.items()}

    def roofline(stage_times, note):
        dom = max(stage_times, key=stage_times.get)
        if dom in ("short_range", "lattice_cutoff", "anterpolation", "interpolation"):
            ach = model[dom]["flop"] / (stage_times[dom] * 1e-3) / 1e12
            return {"kernel": dom, "bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                    "frac": ach / fp32_peak, "traffic": traffic.get(dom),
                    "peak_source": "FP32 FMA throughput measured by fma_probe.cu in this run (packed %.1f, "
                                   "scalar %.1f TFLOP/s); nominal %d SMs x %d lanes x 2 flop x %.0f MHz (%s "
                                   "sm_max_mhz) = %.1f" % (probe["packed"], probe["scalar"], N_SM, FP32_LANES,
                                                           sm_max, peak_kind, fp32_derived),
                    "work_per_launch": model[dom].get("units"), "timing": note}
        ach = model.get(dom, {"bytes": 0})["bytes"] / (stage_times[dom] * 1e-3) / 1e9
        return {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm, "traffic": traffic.get(dom), "timing": note}
    roof = roofline(per_eval, "live: CUDA events on the kernel's stream in the timed region, where the grid "
                              "passes run concurrently on the plan's side stream")
    roof_iso = roofline(per_iso, "isolated: the same evaluation with every stage in turn on one stream")
    out = {
        "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": tot / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (pairs, grids) + f64 (top level, energy)",
        "data": "synthetic",
        "config": {"workload": args.workload, "atoms": n, "box_A": w.box, "cutoff_A": w.cutoff,
                   "spacing_A": w.spacing, "h_eff_A": plan.h_eff[0], "order": w.order,
                   "splitting": w.split, "levels": plan.levels, "grid0": plan.dims[0],
                   "precision": "mixed", "l2": "flushed between timed steps (512 MB write)",
                   "tuning": head_tuning,
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "e2e": {"value": e2e_value, "unit": "evals/s", "h2d_bytes_per_step": 32 * n,
                "d2h_bytes_per_step": 32 * n + 8,
                "api": "msm_eval_host (pinned host buffers): positions and charges in; energy, potentials and "
                       "forces out"},
        "gpu_launches": launches,
        "roofline": roof,
        "roofline_isolated": roof_iso,
        "fp32_peak": {"measured_tflops": fp32_peak, "packed_tflops": probe["packed"], "scalar_tflops": probe["scalar"],
                      "nominal_tflops": fp32_derived, "probe_outputs_finite": probe["finite"]},
        "kernels_ms_per_eval": kernels,
        "kernels_ms_isolated": {k: round(v, 5) for k, v in per_iso.items()},
        "autotune_ms": {k: (round(v, 4) if isinstance(v, float) else v) for k, v in head_tune_ms.items()},
        "ms_per_step_serial": sum(ms_iso) / len(ms_iso),
        "fp64_gpu_path": fp64,
        "batched_replicas": batched,
        "water4m_forward_adjoint": large,
        "parareal_G_cutoff": cutoff_G,
        "parareal_G_msm": msm_G,
        "parareal_G_wolf": wolf_G,
        "md_velocity_verlet": md,
        "parareal_window": pr_window,
        "clocks": clk,
        "energy": E_mix,
    }
    if not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"], ref = cpu_baseline(w)
        # every atom of the headline system against the FP64 oracle (its
        # whole evaluation above): the mixed path and the FP64 GPU path
        out["errors_vs_oracle"] = {"mixed": errors_vs(E_mix, phi_mix.cpu().numpy(), F_mix.cpu().numpy(), ref),
                                   "atoms_compared": n, "other_configs": cfg_err}
        if fp64 is not None:
            out["errors_vs_oracle"]["fp64_gpu"] = errors_vs(E64, phi64.cpu().numpy(), F64.cpu().numpy(), ref)
    print(json.dumps(out))
    plan.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
