"""GB300-native multilevel summation (MSM) energy+force evaluation.

Thin Python binding over the C ABI of ``include/msm.h``: every step of an
evaluation runs in the CUDA kernels of ``libmsm_gb300.so``; PyTorch only
provides device memory and the stream.  The method follows Sec. "Multilevel
Summation Method" of the thesis proposal "Large-Scale Molecular Dynamics
Simulations for Highly Parallel Infrastructures" (Pazurikova, 2014).

    plan = MSM(box=(62.2,)*3, periodic=True, cutoff=10.0, spacing=2.0, order=3)
    E, phi, F = plan.eval(pos, q)        # pos [N,3], q [N]: float64 CUDA tensors
    E = MSMEnergy.apply(pos, q, plan)    # differentiable: dE/dpos = -F, dE/dq = phi
"""
import ctypes as C

import torch

from . import _capi
from ._capi import MSMError, MSM_FP64, MSM_MIXED  # noqa: F401

__all__ = ["MSM", "MSMBatch", "BatchGraph", "MSMEnergy", "MSMError", "MSM_FP64", "MSM_MIXED", "lib", "parareal",
           "MD_METHODS"]

MD_METHODS = {"msm": 0, "cutoff": 1, "wolf": 2}  # MSM_MD_MSM, MSM_MD_CUTOFF, MSM_MD_WOLF


def lib():
    return _capi.load()


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(None)


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


class MSM:
    """One MSM configuration (plan) on the current CUDA device.

    box: edges (L_x, L_y, L_z); periodic: bool; cutoff: a; spacing: h;
    levels: l (0 = automatic); order: 3 cubic / 5 quintic; splitting: Taylor
    order m of gamma (1, 2, 3); precision: "fp64" or "mixed"; coulomb_k:
    prefactor; max_atoms: capacity of the workspace; tuning: optional tile
    shapes and methods, any of the fields of msm_tuning in include/msm.h
    ({"cell_fill", "patch_cells", "lattice_waves", "pair_targets", "lattice_txn",
    "lattice_tyn", "batch_persistent", "lattice_method"}; see autotune.py).
    After construction, lattice_method says which lattice-cutoff form the
    plan took ("stencil" or "fft").
    """

    def __init__(self, box, periodic, cutoff, spacing, levels=0, order=3, splitting=2,
                 precision="mixed", coulomb_k=1.0, max_atoms=1 << 20, tuning=None):
        L = lib()
        p = _capi.MSMParams()
        b = box if hasattr(box, "__len__") else (box, box, box)
        for d in range(3):
            p.box[d] = float(b[d])
        p.periodic = int(bool(periodic))
        p.cutoff = float(cutoff)
        p.spacing = float(spacing)
        p.levels = int(levels)
        p.order = int(order)
        p.splitting = int(splitting)
        p.precision = {"fp64": MSM_FP64, "mixed": MSM_MIXED}[precision]
        p.coulomb_k = float(coulomb_k)
        p.max_atoms = int(max_atoms)
        self.params = p
        self.precision = precision
        self._h = C.c_void_p()
        self._last_n = None
        self.tuning = dict(tuning or {})
        t = _capi.MSMTuning(*[int(self.tuning.get(k, 0)) for k, _ in _capi.MSMTuning._fields_])
        _capi.check(L.msm_create_tuned(C.byref(p), C.byref(t), C.byref(self._h)), "msm_create_tuned")
        heff = (C.c_double * 3)()
        nl = C.c_int()
        dims = (C.c_int * (3 * _capi.MAX_LEVELS))()
        lo = (C.c_int * (3 * _capi.MAX_LEVELS))()
        _capi.check(L.msm_query(self._h, heff, C.byref(nl), dims, lo), "msm_query")
        self.h_eff = tuple(heff)
        self.levels = nl.value
        self.dims = [tuple(dims[3 * k:3 * k + 3]) for k in range(self.levels)]
        self.lo = [tuple(lo[3 * k:3 * k + 3]) for k in range(self.levels)]
        lm = C.c_int()
        _capi.check(L.msm_lattice_method(self._h, C.byref(lm)), "msm_lattice_method")
        self.lattice_method = {1: "stencil", 2: "fft"}[lm.value]

    def close(self):
        if self._h:
            lib().msm_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _check_inputs(pos, q):
        if not (pos.is_cuda and q.is_cuda):
            raise ValueError("pos and q must be CUDA tensors")
        if pos.dtype != q.dtype or pos.dtype not in (torch.float64, torch.float32):
            raise ValueError("pos and q must both be float64 (msm_eval) or both float32 (msm_eval_f32io)")
        if pos.dim() != 2 or pos.shape[1] != 3 or q.shape != (pos.shape[0],):
            raise ValueError("pos must be [N,3] and q [N]")
        return pos.contiguous(), q.contiguous()

    def eval(self, pos, q, want_phi=True, want_force=True, stream=None, out=None):
        """Forward pass: returns (E [0-d] float64, phi [N] or None, F [N,3] or
        None).  float64 inputs go through msm_eval, float32 inputs through
        msm_eval_f32io (phi and F then come back as float32)."""
        pos, q = self._check_inputs(pos, q)
        n = pos.shape[0]
        io = pos.dtype
        if out is None:
            E = torch.empty((), dtype=torch.float64, device=pos.device)
            phi = torch.empty(n, dtype=io, device=pos.device) if want_phi else None
            F = torch.empty((n, 3), dtype=io, device=pos.device) if want_force else None
        else:
            E, phi, F = out
        fn = lib().msm_eval if io == torch.float64 else lib().msm_eval_f32io
        rc = fn(self._h, n, _ptr(pos), _ptr(q), _ptr(E), _ptr(phi), _ptr(F), _stream(stream))
        _capi.check(rc, "msm_eval" if io == torch.float64 else "msm_eval_f32io")
        self._last_n = n
        self._last_io = io
        return E, phi, F

    def cutoff_eval(self, pos, q, want_phi=True, want_force=True, stream=None, out=None):
        """msm_cutoff_eval: the cutoff method (Coulomb law within this plan's
        cutoff only; the parareal coarse propagator) on float64 device
        inputs; returns (E, phi or None, F or None)."""
        pos, q = self._check_inputs(pos, q)
        if pos.dtype != torch.float64:
            raise ValueError("cutoff_eval takes float64 pos and q")
        n = pos.shape[0]
        if out is None:
            E = torch.empty((), dtype=torch.float64, device=pos.device)
            phi = torch.empty(n, dtype=torch.float64, device=pos.device) if want_phi else None
            F = torch.empty((n, 3), dtype=torch.float64, device=pos.device) if want_force else None
        else:
            E, phi, F = out
        rc = lib().msm_cutoff_eval(self._h, n, _ptr(pos), _ptr(q), _ptr(E), _ptr(phi), _ptr(F), _stream(stream))
        _capi.check(rc, "msm_cutoff_eval")
        self._last_n = None
        return E, phi, F

    def wolf_eval(self, pos, q, alpha, want_phi=True, want_force=True, stream=None, out=None):
        """msm_wolf_eval: Wolf summation (damped, shifted force, damping alpha,
        cutoff = this plan's) on float64 device inputs; returns (E, phi or
        None, F or None)."""
        pos, q = self._check_inputs(pos, q)
        if pos.dtype != torch.float64:
            raise ValueError("wolf_eval takes float64 pos and q")
        n = pos.shape[0]
        if out is None:
            E = torch.empty((), dtype=torch.float64, device=pos.device)
            phi = torch.empty(n, dtype=torch.float64, device=pos.device) if want_phi else None
            F = torch.empty((n, 3), dtype=torch.float64, device=pos.device) if want_force else None
        else:
            E, phi, F = out
        rc = lib().msm_wolf_eval(self._h, float(alpha), n, _ptr(pos), _ptr(q), _ptr(E), _ptr(phi), _ptr(F),
                                 _stream(stream))
        _capi.check(rc, "msm_wolf_eval")
        self._last_n = None
        return E, phi, F

    def set_wolf_alpha(self, alpha):
        """msm_set_wolf_alpha: the damping of the "wolf" MD force on this plan."""
        _capi.check(lib().msm_set_wolf_alpha(self._h, float(alpha)), "msm_set_wolf_alpha")

    def md_run(self, pos, vel, inv_mass, q, dt, nsteps, force=None, records=True, stream=None, method="msm"):
        """msm_md_run: nsteps velocity Verlet steps around the MSM force
        (method "msm") or the cutoff method's ("cutoff"), in place on float64
        device tensors pos [N,3], vel [N,3] and force [N,3] (F at pos by the
        same method; None evaluates it first).  Returns (force, records) with
        records [nsteps, 6] = (potential, kinetic, total, momentum x, y, z)
        per step, or None when records is False."""
        if method not in MD_METHODS:
            raise ValueError("method must be one of %s" % sorted(MD_METHODS))
        if not pos.is_contiguous():
            raise ValueError("md_run updates pos in place: it must be contiguous")
        pos, q = self._check_inputs(pos, q)
        if pos.dtype != torch.float64:
            raise ValueError("md_run takes float64 pos and q")
        checks = [("vel", vel, pos.shape), ("inv_mass", inv_mass, q.shape)]
        if force is not None:
            checks.append(("force", force, pos.shape))
        for name, t, shape in checks:
            if t.dtype != torch.float64 or t.device != pos.device or tuple(t.shape) != tuple(shape) \
                    or not t.is_contiguous():
                raise ValueError("%s must be a contiguous float64 tensor of shape %s on %s"
                                 % (name, tuple(shape), pos.device))
        n = pos.shape[0]
        if force is None:
            if method == "wolf":
                raise ValueError("md_run with method 'wolf' needs the starting force (wolf_eval with the plan's alpha)")
            ev = self.eval if method == "msm" else self.cutoff_eval
            _, _, force = ev(pos, q, want_phi=False, stream=stream)
        rec = torch.empty((max(int(nsteps), 0), 6), dtype=torch.float64, device=pos.device) if records else None
        rc = lib().msm_md_run(self._h, n, _ptr(pos), _ptr(vel), _ptr(force), _ptr(inv_mass), _ptr(q), float(dt),
                              int(nsteps), MD_METHODS[method], _ptr(rec), _stream(stream))
        _capi.check(rc, "msm_md_run")
        if nsteps > 0 or force is None:
            self._last_n = n if method == "msm" else None
            self._last_io = torch.float64
        return force, rec

    def graph(self, pos, q, energy, phi=None, force=None, grad_energy=None, grad_pos=None, grad_q=None):
        """msm_batch_graph_create with this plan alone: msm_eval (and, with
        grad_energy, msm_eval_backward) on these float64 buffers captured into
        a CUDA graph; energy and grad_energy are 1-element tensors.  Returns
        a BatchGraph (launch() replays it)."""
        return MSMBatch([self]).graph(pos, q, [pos.shape[0]], energy, phi, force, grad_energy, grad_pos, grad_q)

    def eval_f32io(self, pos, q, want_phi=True, want_force=True, stream=None, out=None):
        """msm_eval_f32io: eval with float32 positions, charges and outputs."""
        if pos.dtype != torch.float32 or q.dtype != torch.float32:
            raise ValueError("eval_f32io takes float32 pos and q")
        return self.eval(pos, q, want_phi, want_force, stream, out)

    def forward_id(self):
        """msm_forward_id: the id of this plan's latest forward pass (0: none)."""
        fid = C.c_int64()
        _capi.check(lib().msm_forward_id(self._h, C.byref(fid)), "msm_forward_id")
        return fid.value

    def backward(self, grad_E, want_pos=True, want_q=True, stream=None, dtype=None, forward_id=None):
        """Adjoint of a forward pass: returns (dL/dpos [N,3], dL/dq [N]) in the
        last eval's input type (or `dtype`: float64 -> msm_eval_backward,
        float32 -> msm_eval_backward_f32io).  forward_id names the forward
        (its forward_id() right after it ran; default: the plan's latest);
        MSMError STALE_FORWARD (-11) when a later forward reused the plan's
        buffers."""
        n = self._last_n
        if n is None:
            raise MSMError(-10, "msm_eval_backward")
        fid = self.forward_id() if forward_id is None else int(forward_id)
        if fid == 0:
            raise MSMError(-10, "msm_eval_backward")
        io = dtype or getattr(self, "_last_io", torch.float64)
        dev = grad_E.device
        gp = torch.empty((n, 3), dtype=io, device=dev) if want_pos else None
        gq = torch.empty(n, dtype=io, device=dev) if want_q else None
        g = grad_E.to(torch.float64).reshape(()).contiguous()
        fn = lib().msm_eval_backward if io == torch.float64 else lib().msm_eval_backward_f32io
        rc = fn(self._h, fid, _ptr(g), _ptr(gp), _ptr(gq), _stream(stream))
        _capi.check(rc, "msm_eval_backward" if io == torch.float64 else "msm_eval_backward_f32io")
        return gp, gq

    def eval_host(self, pos, q, want_phi=False, want_force=False, stream=None, out=None):
        """End-to-end call with HOST (CPU) buffers: copies in, evaluates,
        copies the energy (and phi/F when asked) out, synchronises.  out:
        optional (E [0-d], phi [N] or None, F [N,3] or None) float64 CPU
        tensors to fill (pinned ones make the copies asynchronous)."""
        if pos.is_cuda or q.is_cuda:
            raise ValueError("eval_host takes CPU tensors")
        pos = pos.to(torch.float64).contiguous()
        q = q.to(torch.float64).contiguous()
        n = pos.shape[0]
        if out is None:
            E = torch.empty((), dtype=torch.float64, pin_memory=pos.is_pinned())
            phi = torch.empty(n, dtype=torch.float64, pin_memory=pos.is_pinned()) if want_phi else None
            F = torch.empty((n, 3), dtype=torch.float64, pin_memory=pos.is_pinned()) if want_force else None
        else:
            E, phi, F = out
            for t in (E, phi, F):
                if t is not None and (t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous()):
                    raise ValueError("eval_host outputs must be contiguous float64 CPU tensors")
        rc = lib().msm_eval_host(self._h, n, _ptr(pos), _ptr(q), _ptr(E), _ptr(phi), _ptr(F),
                                 _stream(stream))
        _capi.check(rc, "msm_eval_host")
        self._last_n = n
        self._last_io = torch.float64
        return E, phi, F

    def set_overlap(self, enable=True):
        """Runs the grid passes concurrently with the pair sums (default) or,
        with enable=False, every stage in turn on the caller's stream."""
        _capi.check(lib().msm_set_overlap(self._h, int(bool(enable))), "msm_set_overlap")

    def profile(self, enable=True):
        """Records per-stage CUDA events around every following evaluation."""
        _capi.check(lib().msm_profile(self._h, int(bool(enable))), "msm_profile")

    def profile_read(self):
        """Returns ({stage: ms}, launches, evals) accumulated since the last read."""
        ms = (C.c_double * _capi.NSTAGES)()
        nl, ne = C.c_int64(), C.c_int64()
        _capi.check(lib().msm_profile_read(self._h, ms, C.byref(nl), C.byref(ne)), "msm_profile_read")
        names = [lib().msm_stage_name(i).decode() for i in range(_capi.NSTAGES)]
        return dict(zip(names, list(ms))), nl.value, ne.value

    def status(self):
        return lib().msm_status(self._h)

    def check_status(self):
        _capi.check(self.status(), "device status")

    def debug_grid(self, level, which):
        """Copy of a grid of the last evaluation (which: 'q' or 'u'), as a
        float64 CPU tensor [nz, ny, nx]."""
        import numpy as np
        nx, ny, nz = self.dims[level]
        out = np.zeros((nz, ny, nx))
        rc = lib().msm_debug_grid(self._h, int(level), {"q": 0, "u": 1}[which],
                                  out.ctypes.data_as(C.POINTER(C.c_double)))
        _capi.check(rc, "msm_debug_grid")
        return out


class MSMBatch:
    """Independent systems (replicas) evaluated together: replica r uses
    plans[r] and the atoms offsets[r]..offsets[r+1]-1 of concatenated pos/q."""

    def __init__(self, plans):
        self.plans = list(plans)
        self._arr = (C.c_void_p * len(self.plans))(*[p._h.value for p in self.plans])

    def _offsets(self, counts):
        off = [0]
        for c in counts:
            off.append(off[-1] + int(c))
        return (C.c_int64 * len(off))(*off), off[-1]

    def eval(self, pos, q, counts, want_phi=True, want_force=True, stream=None, out=None):
        """Returns (energies [nrep], phi [N] or None, F [N,3] or None)."""
        offs, n = self._offsets(counts)
        dev = pos.device
        if out is None:
            E = torch.empty(len(self.plans), dtype=torch.float64, device=dev)
            phi = torch.empty(n, dtype=torch.float64, device=dev) if want_phi else None
            F = torch.empty((n, 3), dtype=torch.float64, device=dev) if want_force else None
        else:
            E, phi, F = out
        rc = lib().msm_eval_batch(self._arr, len(self.plans), offs, _ptr(pos), _ptr(q), _ptr(E), _ptr(phi),
                                  _ptr(F), _stream(stream))
        _capi.check(rc, "msm_eval_batch")
        for p, c in zip(self.plans, counts):
            p._last_n = int(c)
        return E, phi, F

    def backward(self, grad_energies, counts, want_pos=True, want_q=True, stream=None):
        offs, n = self._offsets(counts)
        dev = grad_energies.device
        gp = torch.empty((n, 3), dtype=torch.float64, device=dev) if want_pos else None
        gq = torch.empty(n, dtype=torch.float64, device=dev) if want_q else None
        g = grad_energies.to(torch.float64).contiguous()
        rc = lib().msm_eval_backward_batch(self._arr, len(self.plans), offs, _ptr(g), _ptr(gp), _ptr(gq),
                                           _stream(stream))
        _capi.check(rc, "msm_eval_backward_batch")
        return gp, gq

    def md_run(self, pos, vel, force, inv_mass, q, counts, dt, nsteps, method="msm", records=True, stream=None):
        """msm_md_run_batch: nsteps velocity Verlet steps of every replica, in
        place on the concatenated float64 device tensors pos, vel and force
        (force: F at pos of each replica by the same method).  Returns the
        records [nrep, nsteps, 6] or None."""
        offs, n = self._offsets(counts)
        rec = (torch.empty((len(self.plans), max(int(nsteps), 0), 6), dtype=torch.float64, device=pos.device)
               if records else None)
        rc = lib().msm_md_run_batch(self._arr, len(self.plans), offs, _ptr(pos), _ptr(vel), _ptr(force),
                                    _ptr(inv_mass), _ptr(q), float(dt), int(nsteps), MD_METHODS[method], _ptr(rec),
                                    _stream(stream))
        _capi.check(rc, "msm_md_run_batch")
        for p, c in zip(self.plans, counts):
            p._last_n = int(c) if method == "msm" else None
        return rec

    def graph(self, pos, q, counts, energies, phi=None, force=None, grad_energies=None, grad_pos=None,
              grad_q=None):
        """Captures the batched forward (+ adjoint when grad_energies is given)
        on these buffers into a CUDA graph; returns a BatchGraph."""
        offs, _ = self._offsets(counts)
        h = C.c_void_p()
        rc = lib().msm_batch_graph_create(self._arr, len(self.plans), offs, _ptr(pos), _ptr(q), _ptr(energies),
                                          _ptr(phi), _ptr(force), _ptr(grad_energies), _ptr(grad_pos),
                                          _ptr(grad_q), C.byref(h))
        _capi.check(rc, "msm_batch_graph_create")
        return BatchGraph(h, keep=(pos, q, energies, phi, force, grad_energies, grad_pos, grad_q, self))


class BatchGraph:
    """An instantiated CUDA graph of a batched evaluation."""

    def __init__(self, h, keep):
        self._h = h
        self._keep = keep  # the captured buffers must outlive the graph

    def launch(self, stream=None):
        _capi.check(lib().msm_graph_launch(self._h, _stream(stream)), "msm_graph_launch")

    def close(self):
        if self._h:
            lib().msm_graph_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def parareal(fine, coarse, pos0, vel0, inv_mass, q, window, dt_fine, steps_fine, dt_coarse, steps_coarse,
             max_iter, tol, stream=None, coarse_method="cutoff"):
    """msm_parareal: one parareal window (Eq. parareal) with F = steps_fine
    velocity Verlet steps of dt_fine on the MSM force (fine: `window`
    distinct plans, run concurrently) and G = steps_coarse steps of dt_coarse
    on plan coarse's cutoff method (coarse_method "cutoff") or its MSM
    ("msm").  Returns (lam_pos [window+1, N, 3],
    lam_vel [window+1, N, 3], iterations, change [iterations, 2]) with the
    largest position and velocity change of each iteration."""
    import numpy as np
    fine = list(fine)
    if len(fine) != window:
        raise ValueError("one fine plan per time point of the window")
    n = pos0.shape[0]
    dev = pos0.device
    for name, t, shape in (("pos0", pos0, (n, 3)), ("vel0", vel0, (n, 3)), ("inv_mass", inv_mass, (n,)),
                           ("q", q, (n,))):
        if t.dtype != torch.float64 or t.device != dev or tuple(t.shape) != shape or not t.is_contiguous():
            raise ValueError("%s must be a contiguous float64 tensor of shape %s on %s" % (name, shape, dev))
    nbytes = lib().msm_parareal_workspace(n, int(window))
    if nbytes < 0:
        raise ValueError("window must be 1..64")
    ws = torch.empty(max(nbytes, 8), dtype=torch.uint8, device=dev)
    lam_pos = torch.empty((window + 1, n, 3), dtype=torch.float64, device=dev)
    lam_vel = torch.empty_like(lam_pos)
    arr = (C.c_void_p * window)(*[p._h.value for p in fine])
    iters = C.c_int(0)
    change = np.zeros((max(int(max_iter), 1), 2))
    rc = lib().msm_parareal(arr, coarse._h, n, _ptr(pos0), _ptr(vel0), _ptr(inv_mass), _ptr(q), int(window),
                            float(dt_fine), int(steps_fine), float(dt_coarse), int(steps_coarse),
                            MD_METHODS[coarse_method], int(max_iter),
                            float(tol), _ptr(lam_pos), _ptr(lam_vel), _ptr(ws), C.byref(iters),
                            change.ctypes.data_as(C.c_void_p), _stream(stream))
    _capi.check(rc, "msm_parareal")
    for p in fine:
        p._last_n = n
    coarse._last_n = None
    return lam_pos, lam_vel, iters.value, change[:iters.value]


class MSMEnergy(torch.autograd.Function):
    """E(pos, q) with a hand-written adjoint: backward runs the transposed
    grid passes of the library (msm_eval_backward).

    The adjoint reuses the per-atom terms the plan's buffers keep from the
    forward pass.  Each forward records its forward id; when a later forward
    on the same plan (another apply, or any eval) has reused the buffers,
    the backward re-runs this forward on its saved inputs first, so the
    gradient is always that of this call's inputs."""

    @staticmethod
    def forward(ctx, pos, q, plan):
        pos_d, q_d = pos.detach(), q.detach()
        E, _, _ = plan.eval(pos_d, q_d, want_phi=False, want_force=False)
        ctx.plan = plan
        ctx.forward_id = plan.forward_id()
        ctx.save_for_backward(pos_d, q_d)
        return E

    @staticmethod
    def backward(ctx, grad_E):
        plan = ctx.plan
        pos, q = ctx.saved_tensors
        kw = dict(want_pos=ctx.needs_input_grad[0], want_q=ctx.needs_input_grad[1])
        if plan.forward_id() != ctx.forward_id:
            # the buffers hold a later forward: recompute this one
            plan.eval(pos, q, want_phi=False, want_force=False)
            ctx.forward_id = plan.forward_id()
        gp, gq = plan.backward(grad_E, forward_id=ctx.forward_id, **kw)
        return gp, gq, None
