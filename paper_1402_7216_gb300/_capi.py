"""ctypes declarations of the C ABI in include/msm.h (argument marshalling only).

The shared library is built in-tree (``paper_1402_7216_gb300/build.py``); if it
is missing this module raises instead of falling back to anything else.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmsm_gb300.so")

MSM_OK = 0
ERRORS = {
    -1: "MSM_ERR_INVALID_ARG", -2: "MSM_ERR_UNSUPPORTED", -3: "MSM_ERR_CUTOFF_GT_HALF_BOX",
    -4: "MSM_ERR_ATOM_OUTSIDE_BOX", -5: "MSM_ERR_NONFINITE", -6: "MSM_ERR_OOM", -7: "MSM_ERR_CUDA",
    -8: "MSM_ERR_TIMEOUT", -9: "MSM_ERR_TOO_MANY_ATOMS", -10: "MSM_ERR_NO_FORWARD",
    -11: "MSM_ERR_STALE_FORWARD",
}
MSM_FP64, MSM_MIXED = 0, 1
MAX_LEVELS = 16


class MSMParams(C.Structure):
    _fields_ = [("box", C.c_double * 3), ("periodic", C.c_int), ("cutoff", C.c_double),
                ("spacing", C.c_double), ("levels", C.c_int), ("order", C.c_int),
                ("splitting", C.c_int), ("precision", C.c_int), ("coulomb_k", C.c_double),
                ("max_atoms", C.c_int64)]


class MSMTuning(C.Structure):
    _fields_ = [("cell_fill", C.c_int), ("patch_cells", C.c_int), ("lattice_waves", C.c_int),
                ("pair_targets", C.c_int), ("lattice_txn", C.c_int), ("lattice_tyn", C.c_int),
                ("batch_persistent", C.c_int), ("lattice_method", C.c_int), ("pair_runs", C.c_int)]


class MSMError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__("%s%s (%d)" % (what + ": " if what else "", ERRORS.get(code, "unknown"), code))


_lib = None
_D = C.POINTER(C.c_double)
EXPORTS = ["msm_create", "msm_create_tuned", "msm_destroy", "msm_query", "msm_geometry", "msm_eval", "msm_cutoff_eval",
           "msm_wolf_eval", "msm_set_wolf_alpha", "msm_md_run", "msm_md_run_batch",
           "msm_parareal_workspace", "msm_parareal",
           "msm_eval_backward", "msm_forward_id", "msm_lattice_method",
           "msm_eval_f32io", "msm_eval_backward_f32io",
           "msm_eval_host", "msm_status", "msm_debug_grid", "msm_set_overlap", "msm_profile", "msm_profile_read",
           "msm_stage_name", "msm_energy_noalloc", "msm_eval_batch", "msm_eval_backward_batch",
           "msm_batch_graph_create", "msm_graph_launch", "msm_graph_destroy", "msm_strerror"]
NSTAGES = 8


def load(path=LIB_PATH):
    """Loads the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libmsm_gb300.so is not built (run __graft_entry__.build() or "
                          "python paper_1402_7216_gb300/build.py); there is no fallback")
    L = C.CDLL(path)
    vp = C.c_void_p
    L.msm_create.argtypes = [C.POINTER(MSMParams), C.POINTER(vp)]
    L.msm_create.restype = C.c_int
    L.msm_create_tuned.argtypes = [C.POINTER(MSMParams), C.POINTER(MSMTuning), C.POINTER(vp)]
    L.msm_create_tuned.restype = C.c_int
    L.msm_destroy.argtypes = [vp]
    L.msm_destroy.restype = None
    L.msm_query.argtypes = [vp, _D, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.msm_query.restype = C.c_int
    L.msm_geometry.argtypes = [C.POINTER(MSMParams), _D, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.msm_geometry.restype = C.c_int
    L.msm_eval.argtypes = [vp, C.c_int64, vp, vp, vp, vp, vp, vp]
    L.msm_eval.restype = C.c_int
    L.msm_cutoff_eval.argtypes = [vp, C.c_int64, vp, vp, vp, vp, vp, vp]
    L.msm_cutoff_eval.restype = C.c_int
    L.msm_wolf_eval.argtypes = [vp, C.c_double, C.c_int64, vp, vp, vp, vp, vp, vp]
    L.msm_wolf_eval.restype = C.c_int
    L.msm_set_wolf_alpha.argtypes = [vp, C.c_double]
    L.msm_set_wolf_alpha.restype = C.c_int
    L.msm_md_run.argtypes = [vp, C.c_int64, vp, vp, vp, vp, vp, C.c_double, C.c_int, C.c_int, vp, vp]
    L.msm_md_run.restype = C.c_int
    L.msm_md_run_batch.argtypes = [vp, C.c_int, vp, vp, vp, vp, vp, vp, C.c_double, C.c_int, C.c_int, vp, vp]
    L.msm_md_run_batch.restype = C.c_int
    L.msm_parareal_workspace.argtypes = [C.c_int64, C.c_int]
    L.msm_parareal_workspace.restype = C.c_int64
    L.msm_parareal.argtypes = [vp, vp, C.c_int64, vp, vp, vp, vp, C.c_int, C.c_double, C.c_int, C.c_double, C.c_int,
                               C.c_int, C.c_int, C.c_double, vp, vp, vp, vp, vp, vp]
    L.msm_parareal.restype = C.c_int
    L.msm_eval_backward.argtypes = [vp, C.c_int64, vp, vp, vp, vp]
    L.msm_eval_backward.restype = C.c_int
    L.msm_forward_id.argtypes = [vp, C.POINTER(C.c_int64)]
    L.msm_forward_id.restype = C.c_int
    L.msm_lattice_method.argtypes = [vp, C.POINTER(C.c_int)]
    L.msm_lattice_method.restype = C.c_int
    L.msm_eval_f32io.argtypes = [vp, C.c_int64, vp, vp, vp, vp, vp, vp]
    L.msm_eval_f32io.restype = C.c_int
    L.msm_eval_backward_f32io.argtypes = [vp, C.c_int64, vp, vp, vp, vp]
    L.msm_eval_backward_f32io.restype = C.c_int
    L.msm_eval_host.argtypes = [vp, C.c_int64, vp, vp, vp, vp, vp, vp]
    L.msm_eval_host.restype = C.c_int
    L.msm_status.argtypes = [vp]
    L.msm_status.restype = C.c_int
    L.msm_debug_grid.argtypes = [vp, C.c_int, C.c_int, _D]
    L.msm_debug_grid.restype = C.c_int
    L.msm_set_overlap.argtypes = [vp, C.c_int]
    L.msm_set_overlap.restype = C.c_int
    L.msm_profile.argtypes = [vp, C.c_int]
    L.msm_profile.restype = C.c_int
    L.msm_profile_read.argtypes = [vp, _D, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    L.msm_profile_read.restype = C.c_int
    L.msm_stage_name.argtypes = [C.c_int]
    L.msm_stage_name.restype = C.c_char_p
    L.msm_eval_batch.argtypes = [vp, C.c_int, vp, vp, vp, vp, vp, vp, vp]
    L.msm_eval_batch.restype = C.c_int
    L.msm_eval_backward_batch.argtypes = [vp, C.c_int, vp, vp, vp, vp, vp]
    L.msm_eval_backward_batch.restype = C.c_int
    L.msm_batch_graph_create.argtypes = [vp, C.c_int, vp, vp, vp, vp, vp, vp, vp, vp, vp, C.POINTER(vp)]
    L.msm_batch_graph_create.restype = C.c_int
    L.msm_graph_launch.argtypes = [vp, vp]
    L.msm_graph_launch.restype = C.c_int
    L.msm_graph_destroy.argtypes = [vp]
    L.msm_graph_destroy.restype = None
    L.msm_energy_noalloc.argtypes = [C.c_int64, vp, vp, vp, vp]
    L.msm_energy_noalloc.restype = C.c_int
    L.msm_strerror.argtypes = [C.c_int]
    L.msm_strerror.restype = C.c_char_p
    _lib = L
    return L


def check(code, what=""):
    if code != MSM_OK:
        raise MSMError(code, what)
