"""ctypes view of include/hopf.h.  Loads the in-tree libhopf_gb300.so."""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhopf_gb300.so")

c_int, c_double, c_void_p = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
P_double = ctypes.POINTER(c_double)
P_int = ctypes.POINTER(c_int)


class HopfProblem(ctypes.Structure):
    _fields_ = [("n", c_int), ("m", c_int), ("A", P_double), ("B", P_double), ("ctrl_kind", c_int),
                ("radius", c_double), ("half_widths", P_double), ("W", P_double)]


class HopfOpts(ctypes.Structure):
    _fields_ = [("rule", c_int), ("N", c_int), ("max_iter", c_int), ("gap_every", c_int),
                ("precision", c_int), ("host_io", c_int), ("tau", c_double), ("sigma_scale", c_double),
                ("tol_gap", c_double), ("t_max", c_double), ("tol_T", c_double), ("profile", c_int),
                ("accel", c_int), ("park_iters", c_int), ("newton", c_int),
                ("kernel", c_int), ("variables", c_int), ("max_steps", c_int),
                ("adaptive", c_int)]


class HopfMlp(ctypes.Structure):
    _fields_ = [("n_in", c_int), ("hidden", c_int), ("n_out", c_int), ("w", c_void_p), ("w_bf16", c_void_p),
                ("adam_m", c_void_p), ("adam_v", c_void_p), ("x_shift", c_void_p), ("x_scale", c_void_p),
                ("y_shift", c_void_p), ("y_scale", c_void_p), ("use_tc", c_int)]


class HopfStacked(ctypes.Structure):
    _fields_ = [("base", HopfProblem), ("copies", c_int), ("W_blocks", P_double)]


EXPORTS = ("hopf_default_opts", "hopf_value", "hopf_value_stacked", "hopf_time_to_reach", "hopf_trajectory",
           "hopf_status_string", "hopf_last_error", "hopf_release_workspace", "hopf_last_profile",
           "hopf_value_noalloc", "hopf_mlp_param_count", "hopf_mlp_sync", "hopf_mlp_forward",
           "hopf_mlp_loss_grad", "hopf_mlp_adam", "hopf_value_warm", "hopf_tc_selftest", "hopf_node_table")

_lib = None


def load(path=LIB_PATH):
    """Load the CUDA library (once).  Raises if it is missing: there is no
    fallback implementation."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} not found: build it with `python -m paper_1712_08226_gb300.build`")
    lib = ctypes.CDLL(path)
    PP, PO = ctypes.POINTER(HopfProblem), ctypes.POINTER(HopfOpts)
    lib.hopf_default_opts.argtypes = [PO]
    lib.hopf_default_opts.restype = None
    lib.hopf_value.argtypes = [PP, PO, c_int, c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p,
                               c_void_p, c_void_p, c_void_p, c_void_p]
    lib.hopf_value.restype = c_int
    lib.hopf_value_stacked.argtypes = [ctypes.POINTER(HopfStacked)] + lib.hopf_value.argtypes[1:]
    lib.hopf_value_stacked.restype = c_int
    lib.hopf_time_to_reach.argtypes = [PP, PO, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                       c_void_p, c_void_p, c_void_p, P_int, c_void_p]
    lib.hopf_time_to_reach.restype = c_int
    lib.hopf_trajectory.argtypes = [PP, PO, c_int, c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p,
                                    c_void_p]
    lib.hopf_trajectory.restype = c_int
    lib.hopf_status_string.argtypes = [c_int]
    lib.hopf_status_string.restype = ctypes.c_char_p
    lib.hopf_last_error.argtypes = []
    lib.hopf_last_error.restype = ctypes.c_char_p
    lib.hopf_release_workspace.argtypes = []
    lib.hopf_release_workspace.restype = c_int
    lib.hopf_last_profile.argtypes = [P_double, P_double]
    lib.hopf_last_profile.restype = c_int
    lib.hopf_node_table.argtypes = [PP, PO, c_double, c_void_p, c_void_p, c_void_p]
    lib.hopf_node_table.restype = c_int
    lib.hopf_value_noalloc.argtypes = lib.hopf_value.argtypes
    lib.hopf_value_noalloc.restype = c_int
    PM = ctypes.POINTER(HopfMlp)
    lib.hopf_mlp_param_count.argtypes = [c_int, c_int, c_int]
    lib.hopf_mlp_param_count.restype = ctypes.c_longlong
    lib.hopf_mlp_sync.argtypes = [PM, c_void_p]
    lib.hopf_mlp_sync.restype = c_int
    lib.hopf_mlp_forward.argtypes = [PM, c_int, c_void_p, c_void_p, c_void_p]
    lib.hopf_mlp_forward.restype = c_int
    lib.hopf_mlp_loss_grad.argtypes = [PM, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
    lib.hopf_mlp_loss_grad.restype = c_int
    lib.hopf_mlp_adam.argtypes = [PM, c_void_p, c_int, c_double, c_double, c_double, c_double, c_void_p]
    lib.hopf_mlp_adam.restype = c_int
    lib.hopf_value_warm.argtypes = [PP, PO, PM, c_int, c_void_p, c_void_p, c_int, c_int, c_void_p, c_void_p,
                                    c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
    lib.hopf_value_warm.restype = c_int
    lib.hopf_tc_selftest.argtypes = [c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
    lib.hopf_tc_selftest.restype = c_int
    _lib = lib
    return lib
