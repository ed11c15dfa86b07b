"""Autotuner for the tile shapes of an MSM plan (``msm_tuning`` of the C ABI).

The tunables change speed, never results beyond summation order:
  cell_fill      target atoms per short-range cell (pair-kernel lane use vs
                 candidate volume)
  patch_cells    cells per side of the anterpolation/interpolation patch blocks
  lattice_waves  blocks per SM the lattice aims for on small levels
A coordinate search times each candidate with CUDA events on the caller's own
inputs (evaluations on the caller's stream, warm-up excluded) and keeps the
fastest.  Results are cached in a JSON file keyed by the plan parameters and
the atom count (``MSM_AUTOTUNE_CACHE``, default ``~/.cache/msm_gb300/autotune.json``).
"""
import json
import os

import torch

from . import MSM

SEARCH = [("cell_fill", [20, 24, 28, 32]), ("patch_cells", [2, 3, 4]), ("lattice_waves", [4, 8, 16])]


def cache_path():
    return os.environ.get("MSM_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "msm_gb300", "autotune.json"))


def cache_key(box, periodic, cutoff, spacing, levels, order, splitting, precision, n):
    b = box if hasattr(box, "__len__") else (box, box, box)
    return "box=%.4f,%.4f,%.4f|per=%d|a=%.4f|h=%.4f|l=%d|p=%d|m=%d|%s|n=%d" % (
        b[0], b[1], b[2], int(bool(periodic)), cutoff, spacing, levels, order, splitting, precision, n)


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


def time_plan(plan, pos, q, reps=5, warmup=2):
    """Median CUDA-event time (ms) of one evaluation."""
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        plan.eval(pos, q, want_phi=False, want_force=False)
    ms = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plan.eval(pos, q, want_phi=False, want_force=False)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    plan.check_status()
    ms.sort()
    return ms[len(ms) // 2]


def autotune(pos, q, box, periodic, cutoff, spacing, levels=0, order=3, splitting=2, precision="mixed",
             reps=5, use_cache=True, search=SEARCH):
    """Returns (tuning dict, {candidate: ms}) for this system; cached."""
    n = int(q.shape[0])
    key = cache_key(box, periodic, cutoff, spacing, levels, order, splitting, precision, n)
    path = cache_path()
    if use_cache:
        hit = _load(path).get(key)
        if hit:
            return dict(hit["tuning"]), {"cached": hit.get("ms")}
    best, times = {}, {}

    def run(t):
        plan = MSM(box=box, periodic=periodic, cutoff=cutoff, spacing=spacing, levels=levels, order=order,
                   splitting=splitting, precision=precision, max_atoms=n, tuning=t)
        try:
            return time_plan(plan, pos, q, reps)
        finally:
            plan.close()

    best_ms = run(best)
    times["default"] = best_ms
    for field, values in search:
        for v in values:
            cand = dict(best)
            cand[field] = v
            label = ",".join("%s=%d" % kv for kv in sorted(cand.items()))
            if label in times:
                continue
            ms = run(cand)
            times[label] = ms
            if ms < best_ms * 0.98:  # keep a change only when it is clearly faster
                best, best_ms = cand, ms
    if use_cache:
        data = _load(path)
        data[key] = {"tuning": best, "ms": best_ms}
        _store(path, data)
    return best, times


def tuned_plan(pos, q, box, periodic, cutoff, spacing, **kw):
    """An MSM plan with the autotuned tile shapes for this system."""
    kw2 = {k: kw[k] for k in ("levels", "order", "splitting", "precision") if k in kw}
    tuning, _ = autotune(pos, q, box, periodic, cutoff, spacing, **kw2)
    return MSM(box=box, periodic=periodic, cutoff=cutoff, spacing=spacing, max_atoms=int(q.shape[0]),
               tuning=tuning, **kw2)


# Batches: one tuning shared by every replica, timed on the captured batch
# graph (forward + adjoint), the form msm_batch_graph_create runs.
SEARCH_BATCH = [("lattice_waves", [8, 16]), ("patch_cells", [3, 4]), ("cell_fill", [20, 24])]


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
    return "batch|%s|a=%.4f|h=%.4f|p=%d|m=%d|%s" % (h, cutoff, spacing, order, splitting, precision)


def autotune_batch(boxes, pos, q, counts, cutoff, spacing, order=3, splitting=2, precision="mixed", reps=5,
                   use_cache=True, search=SEARCH_BATCH):
    """Returns (tuning dict, {candidate: ms}) for a batch of periodic boxes
    (edges `boxes`, atoms `counts`, concatenated `pos`, `q` on the device),
    timing the batch graph with the adjoint; cached like autotune()."""
    from . import MSMBatch
    key = batch_key(boxes, counts, cutoff, spacing, order, splitting, precision)
    path = cache_path()
    if use_cache:
        hit = _load(path).get(key)
        if hit:
            return dict(hit["tuning"]), {"cached": hit.get("ms")}
    n, nrep = int(q.shape[0]), len(counts)
    dev = q.device
    E = torch.zeros(nrep, dtype=torch.float64, device=dev)
    F = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    gE = torch.ones(nrep, dtype=torch.float64, device=dev)
    gp = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    best, times = {}, {}

    def run(t):
        plans = [MSM(box=L, periodic=True, cutoff=cutoff, spacing=spacing, order=order, splitting=splitting,
                     precision=precision, max_atoms=int(c), tuning=t) for L, c in zip(boxes, counts)]
        g = MSMBatch(plans).graph(pos, q, counts, E, None, F, gE, gp, None)
        try:
            return time_graph(g, reps)
        finally:
            g.close()
            for p in plans:
                p.close()

    best_ms = run(best)
    times["default"] = best_ms
    for field, values in search:
        for v in values:
            cand = dict(best)
            cand[field] = v
            label = ",".join("%s=%d" % kv for kv in sorted(cand.items()))
            if label in times:
                continue
            ms = run(cand)
            times[label] = ms
            if ms < best_ms * 0.98:
                best, best_ms = cand, ms
    if use_cache:
        data = _load(path)
        data[key] = {"tuning": best, "ms": best_ms}
        _store(path, data)
    return best, times
