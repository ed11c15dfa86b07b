"""Autotuner for the tile shapes of an MSM plan (``msm_tuning`` of the C ABI).

The tunables change speed, never results beyond summation order:
  pair_targets   targets the pair kernel culls together: 32 (a cell's warp)
                 or 8 (clusters of 8 consecutive atoms)
  pair_runs      with 32: a warp's targets are one cell's atoms (2) or 32
                 consecutive atoms of an x-sorted cell row (1); the default
                 takes runs on plans of at least 16,384 cells
  cell_fill      target atoms per short-range cell (pair-kernel lane use vs
                 candidate volume)
  patch_cells    cells per side of the anterpolation/interpolation patch blocks
  lattice_waves  blocks per SM the lattice aims for on small levels
  batch_persistent  batched graphs: restriction and prolongation chains as
                 one cooperative launch each (1) or one launch per pass (0)
  lattice_method periodic plans: the lattice cutoff by FFT (the default) or
                 by the direct stencil (1, the candidate); the stencil's own
                 fields (lattice_waves, lattice_tile) are searched only when
                 it wins
  lattice_tile   warp tile (txn, tyn) of the lattice kernel on the finest
                 level: txn lanes of 8 x outputs by tyn lanes of 2 rows
                 (msm_tuning.lattice_txn / lattice_tyn)
A coordinate search times each candidate with CUDA events on the caller's own
inputs (evaluations on the caller's stream, warm-up excluded) and keeps a
change only when it is faster by MARGIN (1 %).  Batches search the shared fields on
the captured batch graph, then, with the stencil, one lattice tile per finest-grid size: the
replicas with the same level-0 grid share a tile, since the best tile
depends on how the grid's rows and columns fill a warp.  Results are cached
in a JSON file keyed by the plan parameters and the atom counts
(``MSM_AUTOTUNE_CACHE``, default ``~/.cache/msm_gb300/autotune.json``).
"""
import json
import os

import torch

from . import MSM

# A candidate replaces the best so far only when it is faster by this fraction:
# repeated timings of one configuration agree to ~0.2 % (CUDA events, medians).
MARGIN = 0.01

# (txn, tyn) lattice warp tiles: 32 x 16 outputs (the default) and shapes that
# fit small or flat grids better
TILES = [(4, 8), (2, 8), (4, 4), (8, 4), (2, 16), (8, 2), (1, 16)]
SEARCH = [("lattice_method", [1]), ("pair_targets", [32, 8]), ("pair_runs", [1, 2]), ("cell_fill", [20, 24, 28, 32]),
          ("patch_cells", [2, 3, 4]), ("lattice_waves", [4, 8, 16]), ("lattice_tile", TILES)]
# fields that only the stencil form of the lattice cutoff reads
STENCIL_ONLY = ("lattice_waves", "lattice_tile")


def uses_stencil(cand, periodic=True):
    """Whether a candidate runs the stencil lattice (open plans always do)."""
    return (not periodic) or int(cand.get("lattice_method", 0)) == 1


def tuning_fields(cand):
    """The msm_tuning fields of a candidate (lattice_tile -> lattice_txn, lattice_tyn)."""
    t = {k: v for k, v in cand.items() if k != "lattice_tile"}
    if "lattice_tile" in cand:
        t["lattice_txn"], t["lattice_tyn"] = (int(x) for x in cand["lattice_tile"])
    return t


def _label(cand):
    return ",".join("%s=%s" % (k, "x".join(map(str, v)) if isinstance(v, (list, tuple)) else v)
                    for k, v in sorted(cand.items()))


def cache_path():
    return os.environ.get("MSM_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "msm_gb300", "autotune.json"))


def cache_key(box, periodic, cutoff, spacing, levels, order, splitting, precision, n, backward=False):
    b = box if hasattr(box, "__len__") else (box, box, box)
    return "v3|box=%.4f,%.4f,%.4f|per=%d|a=%.4f|h=%.4f|l=%d|p=%d|m=%d|%s|n=%d|bwd=%d" % (
        b[0], b[1], b[2], int(bool(periodic)), cutoff, spacing, levels, order, splitting, precision, n,
        int(bool(backward)))


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, data):
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def time_plan(plan, pos, q, reps=5, warmup=2, backward=False):
    """Median CUDA-event time (ms) of one evaluation (and its adjoint)."""
    stream = torch.cuda.current_stream()
    g = torch.ones((), dtype=torch.float64, device=pos.device)

    def once():
        plan.eval(pos, q, want_phi=False, want_force=False)
        if backward:
            plan.backward(g)
    for _ in range(warmup):
        once()
    ms = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        once()
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    plan.check_status()
    ms.sort()
    return ms[len(ms) // 2]


def _coordinate_search(run, search, start=None, times=None, skip=None):
    """Tries each field's values in turn from the best so far; skip(field,
    best) -> True leaves a field out (it cannot change the timing)."""
    best = dict(start or {})
    times = {} if times is None else times
    best_ms = run(best)
    times[_label(best) or "default"] = best_ms
    for field, values in search:
        if skip is not None and skip(field, best):
            continue
        for v in values:
            cand = dict(best)
            cand[field] = list(v) if isinstance(v, tuple) else v
            label = _label(cand)
            if label in times:
                continue
            try:
                ms = run(cand)
            except Exception as e:  # a tile whose window does not fit this plan: not a candidate
                times[label] = "rejected: %s" % e
                continue
            times[label] = ms
            if ms < best_ms * (1.0 - MARGIN):  # keep a change only when it is clearly faster
                best, best_ms = cand, ms
    return best, best_ms, times


def autotune(pos, q, box, periodic, cutoff, spacing, levels=0, order=3, splitting=2, precision="mixed",
             reps=5, use_cache=True, search=SEARCH, backward=False):
    """Returns (tuning dict for MSM(tuning=...), {candidate: ms}) for this
    system; backward=True times each evaluation together with its adjoint."""
    n = int(q.shape[0])
    key = cache_key(box, periodic, cutoff, spacing, levels, order, splitting, precision, n, backward)
    path = cache_path()
    if use_cache:
        hit = _load(path).get(key)
        if hit:
            return tuning_fields(hit["tuning"]), {"cached": hit.get("ms"), "choice": hit["tuning"]}

    def run(cand):
        plan = MSM(box=box, periodic=periodic, cutoff=cutoff, spacing=spacing, levels=levels, order=order,
                   splitting=splitting, precision=precision, max_atoms=n, tuning=tuning_fields(cand))
        try:
            return time_plan(plan, pos, q, reps, backward=backward)
        finally:
            plan.close()

    best, best_ms, times = _coordinate_search(
        run, search, skip=lambda field, b: (field in STENCIL_ONLY and not uses_stencil(b, periodic)) or
        (field == "lattice_method" and not periodic))
    if use_cache:
        data = _load(path)
        data[key] = {"tuning": best, "ms": best_ms}
        _store(path, data)
    times["choice"] = best
    return tuning_fields(best), times


def tuned_plan(pos, q, box, periodic, cutoff, spacing, **kw):
    """An MSM plan with the autotuned tile shapes for this system."""
    kw2 = {k: kw[k] for k in ("levels", "order", "splitting", "precision") if k in kw}
    tuning, _ = autotune(pos, q, box, periodic, cutoff, spacing, **kw2)
    return MSM(box=box, periodic=periodic, cutoff=cutoff, spacing=spacing, max_atoms=int(q.shape[0]),
               tuning=tuning, **kw2)


# Batches: timed on the captured batch graph (forward + adjoint), the form
# msm_batch_graph_create runs.
SEARCH_BATCH = [("lattice_method", [1]), ("pair_targets", [32, 8]), ("pair_runs", [1, 2]), ("batch_persistent", [0, 1]),
                ("lattice_waves", [8, 16]), ("patch_cells", [3, 4]), ("cell_fill", [20, 24])]
TILES_BATCH = [(4, 8), (2, 8), (4, 4), (8, 4), (2, 16), (1, 16)]


def time_graph(graph, reps=5, warmup=2):
    """Median CUDA-event time (ms) of one replay of a batch graph."""
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        graph.launch()
    ms = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        graph.launch()
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    ms.sort()
    return ms[len(ms) // 2]


def batch_key(boxes, counts, cutoff, spacing, order, splitting, precision):
    import hashlib
    h = hashlib.sha1(repr((list(map(float, boxes)), list(map(int, counts)))).encode()).hexdigest()[:16]
    return "batch4|%s|a=%.4f|h=%.4f|p=%d|m=%d|%s" % (h, cutoff, spacing, order, splitting, precision)


def autotune_batch(boxes, pos, q, counts, cutoff, spacing, order=3, splitting=2, precision="mixed", reps=5,
                   use_cache=True, search=SEARCH_BATCH, tiles=TILES_BATCH):
    """Tunes a batch of periodic boxes (edges `boxes`, atoms `counts`,
    concatenated `pos`, `q` on the device) on its batch graph with the
    adjoint: first the fields every replica shares, then (when the stencil lattice
    wins) a lattice tile per finest-grid size.  Returns (per-replica tuning dicts, summary
    {"shared": ..., "lattice_tile_by_grid0": {M0: [txn, tyn]}}, {candidate:
    ms}); cached like autotune()."""
    from . import MSMBatch
    key = batch_key(boxes, counts, cutoff, spacing, order, splitting, precision)
    path = cache_path()
    n, nrep = int(q.shape[0]), len(counts)
    dev = q.device
    mk = dict(periodic=True, cutoff=cutoff, spacing=spacing, order=order, splitting=splitting, precision=precision)
    # the finest grid of every replica (host geometry of a default plan)
    grid0 = []
    for L, c in zip(boxes, counts):
        p = MSM(box=L, max_atoms=int(c), **mk)
        grid0.append(int(p.dims[0][0]))
        p.close()

    def per_replica(shared, by_grid):
        out = []
        for g in grid0:
            cand = dict(shared)
            if str(g) in by_grid:
                cand["lattice_tile"] = by_grid[str(g)]
            out.append(tuning_fields(cand))
        return out

    if use_cache:
        hit = _load(path).get(key)
        if hit:
            summ = hit["summary"]
            return per_replica(summ["shared"], summ["lattice_tile_by_grid0"]), summ, {"cached": hit.get("ms")}
    E = torch.zeros(nrep, dtype=torch.float64, device=dev)
    F = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    gE = torch.ones(nrep, dtype=torch.float64, device=dev)
    gp = torch.zeros((n, 3), dtype=torch.float64, device=dev)

    def run_all(tunings):
        plans = [MSM(box=L, max_atoms=int(c), tuning=t, **mk) for L, c, t in zip(boxes, counts, tunings)]
        try:
            g = MSMBatch(plans).graph(pos, q, counts, E, None, F, gE, gp, None)
            try:
                return time_graph(g, reps)
            finally:
                g.close()
        finally:
            for p in plans:
                p.close()

    shared, best_ms, times = _coordinate_search(
        lambda cand: run_all(per_replica(cand, {})), search,
        skip=lambda field, b: field in STENCIL_ONLY and not uses_stencil(b))
    by_grid = {}
    tile_grids = sorted(set(grid0), reverse=True) if uses_stencil(shared) else []
    for g in tile_grids:  # the largest grids first: they carry the most lattice work
        def run_tile(cand, g=g):
            trial = dict(by_grid)
            if "lattice_tile" in cand:
                trial[str(g)] = cand["lattice_tile"]
            return run_all(per_replica(shared, trial))
        t_times = {}
        best_t, ms_t, _ = _coordinate_search(run_tile, [("lattice_tile", tiles)], times=t_times)
        for k, v in t_times.items():
            times["grid0=%d|%s" % (g, k)] = v
        if "lattice_tile" in best_t and ms_t < best_ms:
            by_grid[str(g)] = best_t["lattice_tile"]
            best_ms = ms_t
    summary = {"shared": shared, "lattice_tile_by_grid0": by_grid, "grid0_sizes": sorted(set(grid0)),
               "ms": best_ms}
    if use_cache:
        data = _load(path)
        data[key] = {"summary": summary, "ms": best_ms}
        _store(path, data)
    return per_replica(shared, by_grid), summary, times
