"""ctypes binding of ``libtrinity.so`` (declared in include/trinity.h).

Argument marshalling only: every step of the forward model runs inside the library.
Loading fails loudly if the library has not been built; there is no fallback.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtrinity.so")

OK, W_NOT_CONVERGED = 0, 1
STATUS = {0: "OK", 1: "W_NOT_CONVERGED", -1: "E_INVALID", -2: "E_OOM", -3: "E_CUDA",
          -4: "E_STATE", -5: "E_TIMEOUT", -6: "E_UNSUPPORTED"}

c_int, c_double, c_size_t, c_void_p = ctypes.c_int, ctypes.c_double, ctypes.c_size_t, ctypes.c_void_p
P_double = ctypes.POINTER(ctypes.c_double)
P_int = ctypes.POINTER(ctypes.c_int)
P_float = ctypes.POINTER(ctypes.c_float)


class GridDesc(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("nz", c_int), ("h_mm", c_double),
                ("nside", c_int), ("courant", c_double), ("n_ref", c_double),
                ("boundary", c_int), ("precision", c_int), ("tol", c_double),
                ("max_iters", c_int), ("nside_scatter", c_int)]


class SourceDesc(ctypes.Structure):
    _fields_ = [("face", c_int), ("u_mm", c_double), ("v_mm", c_double),
                ("half_angle_deg", c_double), ("pulse_steps", c_int), ("energy", c_double)]


class DetectorDesc(ctypes.Structure):
    _fields_ = [("face", c_int), ("u_mm", c_double), ("v_mm", c_double), ("radius_mm", c_double),
                ("half_angle_deg", c_double)]


class Request(ctypes.Structure):
    _fields_ = [("grid", GridDesc), ("mua", c_void_p), ("mus", c_void_p), ("n", c_void_p),
                ("g", c_double), ("source", SourceDesc), ("n_detectors", c_int),
                ("detectors", ctypes.POINTER(DetectorDesc)), ("bin_ps", c_double),
                ("nbins", c_int), ("nsteps", c_int), ("fresnel", c_int)]


# name -> (restype, argtypes)
SIGNATURES = {
    "trinity_footprint_bytes": (c_size_t, [ctypes.POINTER(GridDesc)]),
    "trinity_create_grid": (c_int, [ctypes.POINTER(GridDesc), c_void_p, ctypes.POINTER(c_void_p)]),
    "trinity_set_optics": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_double, c_int]),
    "trinity_set_optics_uniform": (c_int, [c_void_p, c_double, c_double, c_double, c_double]),
    "trinity_set_fresnel": (c_int, [c_void_p, c_int]),
    "trinity_set_exact_solve": (c_int, [c_void_p, c_int]),
    "trinity_exact_classes": (c_int, [c_void_p, P_int]),
    "trinity_exact_form": (c_int, [c_void_p, P_int]),
    "trinity_set_warm_start": (c_int, [c_void_p, c_int]),
    "trinity_interface_count": (c_int, [c_void_p, P_int]),
    "trinity_interface_entries": (c_int, [c_int, c_int, c_int, c_int, c_double, c_int, c_void_p,
                                          c_void_p, c_void_p, c_void_p, c_void_p, c_size_t,
                                          ctypes.POINTER(c_size_t)]),
    "trinity_set_source": (c_int, [c_void_p, c_int, c_double, c_double, c_double, c_int, c_double]),
    "trinity_add_detector": (c_int, [c_void_p, c_int, c_double, c_double, c_double, c_double, P_int]),
    "trinity_set_bins": (c_int, [c_void_p, c_double, c_int]),
    "trinity_set_initial_state": (c_int, [c_void_p, c_void_p, c_void_p, c_int]),
    "trinity_step": (c_int, [c_void_p, c_int, P_int]),
    "trinity_run": (c_int, [c_void_p, c_int]),
    "trinity_sync": (c_int, [c_void_p]),
    "trinity_profile_steps": (c_int, [c_void_p, c_int, P_double]),
    "trinity_read_detectors": (c_int, [c_void_p, P_double, c_size_t]),
    "trinity_read_energy": (c_int, [c_void_p, P_double, P_double, P_double, P_double, c_size_t]),
    "trinity_kernels_per_step": (c_int, [c_void_p, P_int]),
    "trinity_sweep_form": (c_int, [c_void_p, P_int]),
    "trinity_set_sweep_tma": (c_int, [c_void_p, c_int]),
    "trinity_read_iterations": (c_int, [c_void_p, P_int, P_double, c_size_t]),
    "trinity_read_executed_iterations": (c_int, [c_void_p, P_double, c_size_t]),
    "trinity_read_field": (c_int, [c_void_p, c_int, c_int, c_void_p, c_size_t, c_int]),
    "trinity_steps_done": (c_int, [c_void_p, P_int]),
    "trinity_reset": (c_int, [c_void_p]),
    "trinity_last_error": (ctypes.c_char_p, [c_void_p]),
    "trinity_destroy": (None, [c_void_p]),
    "trinity_tc_selftest": (c_int, [c_int, c_void_p, c_void_p, c_void_p]),
    "trinity_adjoint_footprint_bytes": (c_size_t, [ctypes.POINTER(GridDesc), c_int, c_int, c_int, c_int]),
    "trinity_run_checkpointed": (c_int, [c_void_p, c_int, c_int]),
    "trinity_adjoint": (c_int, [c_void_p, c_void_p, c_size_t, c_void_p, c_void_p, c_int]),
    "trinity_adjoint_profile": (c_int, [c_void_p, c_void_p, c_size_t, c_void_p, c_void_p, c_int, P_double]),
    "trinity_source_iteration_noalloc": (c_int, [c_int, c_int] + [c_void_p] * 7 +
                                         [c_double, c_int, P_int, c_void_p]),
    "trinity_serve_create": (c_int, [c_size_t, c_int, c_int, ctypes.POINTER(c_void_p)]),
    "trinity_serve_submit": (c_int, [c_void_p, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
    "trinity_serve_poll": (c_int, [c_void_p, ctypes.c_uint64, P_int, P_double, c_size_t, P_double]),
    "trinity_serve_wait": (c_int, [c_void_p, ctypes.c_uint64, c_double]),
    "trinity_serve_cancel": (c_int, [c_void_p, ctypes.c_uint64]),
    "trinity_serve_stats": (c_int, [c_void_p, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                    P_int, ctypes.POINTER(c_size_t)]),
    "trinity_serve_destroy": (None, [c_void_p]),
    "trinity_healpix_dirs": (c_int, [c_int, P_double, c_size_t]),
    "trinity_phase_matrix": (c_int, [c_int, c_double, P_double, c_size_t, P_double]),
    "trinity_lattice_tables": (c_int, [c_int, c_int, c_int, c_int, c_double, c_int,
                                       ctypes.POINTER(ctypes.c_int32), P_double,
                                       ctypes.POINTER(ctypes.c_int8), c_size_t]),
    "trinity_cone_weights": (c_int, [c_int, c_int, c_double, c_int, P_double, c_size_t]),
    "trinity_parent_map": (c_int, [c_int, c_int, P_int, c_size_t]),
}

_lib = None


def load():
    """Load the library (once).  Raises if it is missing: build it with build.py first."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libtrinity.so is not built (run paper_2105_01028_gb300/build.py); "
                           "there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class TrinityError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status
