"""ctypes binding of libaderdg.so (include/aderdg.h): argument marshalling only.

Every computation happens in the CUDA library; this module only converts
Python arguments to C types and C status codes to exceptions.  Loading fails
loudly if the library has not been built.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libaderdg.so")

ADG_OK = 0
ADG_EINVAL = 1
ADG_ENOMEM = 2
ADG_ECUDA = 3
ADG_ENONFINITE = 4
ADG_ETIMEOUT = 5
ADG_ESTATE = 6
ADG_EUNSUPPORTED = 7

ADG_BC_PERIODIC = 0
ADG_BC_WALL = 1
ADG_BC_EXCHANGE = 2
ADG_BC_WALL_EXCHANGE = 3
ADG_BC_EXCHANGE_WALL = 4
ADG_BC_NOSLIP = 5
ADG_BC_ANALYTIC = 6
ADG_FIELD_NONE = 0
ADG_FIELD_TAYLOR_GREEN = 1
ADG_FIELD_ABC = 2
ADG_SRC_NONE = 0
ADG_SRC_STEADY = 1
ADG_SRC_PAPER = 2
ADG_PREC_FP64 = 0
ADG_PREC_MIXED = 1
ADG_PREC_MIXED_TF32 = 2
ADG_PREC_MIXED_BF16X3 = 3
ADG_TV_RHO = 0
ADG_TV_THETA = 1
ADG_SCEN_STEADY = 0
ADG_SCEN_COSINE = 1
ADG_SCEN_TWO_BUBBLES = 2
ADG_SCEN_BACKGROUND = 3
ADG_SCEN_PAPER = 4
ADG_SCEN_TAYLOR_GREEN = 5
ADG_SCEN_CAVITY = 6
ADG_SCEN_ABC = 7
ADG_MAX_DEGREE_3D = 4
ADG_COPY_HOST_ASYNC = 2
ADG_NOALLOC_SCRATCH_BYTES = 32 << 20

STATUS_NAMES = {1: "ADG_EINVAL", 2: "ADG_ENOMEM", 3: "ADG_ECUDA", 4: "ADG_ENONFINITE",
                5: "ADG_ETIMEOUT", 6: "ADG_ESTATE", 7: "ADG_EUNSUPPORTED"}


class MeshDesc(ctypes.Structure):
    _fields_ = [("degree", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("x0", ctypes.c_double), ("y0", ctypes.c_double),
                ("Lx", ctypes.c_double), ("Ly", ctypes.c_double),
                ("bc_x", ctypes.c_int), ("bc_y", ctypes.c_int),
                ("gamma", ctypes.c_double), ("Pr", ctypes.c_double),
                ("R", ctypes.c_double), ("mu", ctypes.c_double),
                ("gravity", ctypes.c_int), ("g", ctypes.c_double),
                ("p0", ctypes.c_double), ("theta0", ctypes.c_double),
                ("source", ctypes.c_int), ("src_a", ctypes.c_double),
                ("src_L", ctypes.c_double), ("src_U", ctypes.c_double),
                ("src_p", ctypes.c_double), ("precision", ctypes.c_int),
                ("device", ctypes.c_int), ("max_levels", ctypes.c_int),
                ("lid_u", ctypes.c_double), ("bc_field", ctypes.c_int)]


class Scenario(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("A", ctypes.c_double), ("a", ctypes.c_double),
                ("xc", ctypes.c_double), ("zc", ctypes.c_double)]


class AdgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_S = ctypes.c_size_t

# name -> (restype, argtypes); the list of symbols include/aderdg.h declares
SIGNATURES = {
    "adg_create_mesh": (_I, [ctypes.POINTER(MeshDesc), ctypes.POINTER(_P)]),
    "adg_destroy_mesh": (None, [_P]),
    "adg_state_count": (_S, [_P]),
    "adg_set_state": (_I, [_P, _P, _S, _I, _P]),
    "adg_get_state": (_I, [_P, _P, _S, _I, _P]),
    "adg_state_ptr": (_P, [_P]),
    "adg_set_time": (_I, [_P, _D]),
    "adg_get_time": (_D, [_P]),
    "adg_init_scenario": (_I, [_P, ctypes.POINTER(Scenario), _P]),
    "adg_predictor": (_I, [_P, _D, _P]),
    "adg_corrector": (_I, [_P, _D, _P]),
    "adg_step": (_I, [_P, _D, _P]),
    "adg_step_lts": (_I, [_P, _D, ctypes.POINTER(_D), _P]),
    "adg_stable_dt": (_I, [_P, _D, ctypes.POINTER(_D), _P]),
    "adg_tv_indicator": (_I, [_P, _I, _D, _D, _P, _P, _P, _P]),
    "adg_fv_create": (_I, [ctypes.POINTER(MeshDesc), ctypes.POINTER(_P)]),
    "adg_fv_destroy": (None, [_P]),
    "adg_fv_state_count": (_S, [_P]),
    "adg_fv_set_state": (_I, [_P, _P, _S, _I, _P]),
    "adg_fv_get_state": (_I, [_P, _P, _S, _I, _P]),
    "adg_fv_init_scenario": (_I, [_P, _P, _P]),
    "adg_fv_step": (_I, [_P, _D, _P]),
    "adg_fv_stable_dt": (_I, [_P, _D, _P, _P]),
    "adg3_create": (_I, [ctypes.POINTER(MeshDesc), _I, _D, _D, _I, ctypes.POINTER(_P)]),
    "adg3_destroy": (None, [_P]),
    "adg3_state_count": (_S, [_P]),
    "adg3_set_state": (_I, [_P, _P, _S, _I, _P]),
    "adg3_get_state": (_I, [_P, _P, _S, _I, _P]),
    "adg3_set_time": (_I, [_P, _D]),
    "adg3_get_time": (_D, [_P]),
    "adg3_init_scenario": (_I, [_P, _P, _P]),
    "adg3_step": (_I, [_P, _D, _I, _P]),
    "adg3_stable_dt": (_I, [_P, _D, _P, _P]),
    "adg_step_tv": (_I, [_P, _D, _I, _D, _D, _P, _P, _P, _P]),
    "adg_check_finite": (_I, [_P, _P]),
    "adg_step_adjoint": (_I, [_P, _D, _P, _P, _P, _P]),
    "adg_theta_to_state": (_I, [_P, _P, _P, _P]),
    "adg_theta_to_state_adjoint": (_I, [_P, _P, _P, _P, _P]),
    "adg_state_to_theta": (_I, [_P, _P, _P, _P]),
    "adg_probe_objective": (_I, [_P, _P, _I, _P, _P, _P, _P, _P, _P]),
    "adg_get_boundary_traces": (_I, [_P, _P, _P, _P]),
    "adg_set_halo_traces": (_I, [_P, _P, _P, _P]),
    "adg_tv_flags": (_I, [_P, _P, _D, _D, _D, _D, _D, _P, _P]),
    "adg_batch_create": (_I, [ctypes.POINTER(_P), _I, ctypes.POINTER(_P)]),
    "adg_batch_step": (_I, [_P, ctypes.POINTER(_D), _I, _P]),
    "adg_batch_info": (_I, [_P, ctypes.POINTER(_I), _I]),
    "adg_batch_set_candidate": (_I, [_P, _I]),
    "adg_batch_destroy": (None, [_P]),
    "adg_step_noalloc": (_I, [ctypes.POINTER(MeshDesc), _P, _S, _D, _P]),
    "adg_leaf_count": (_S, [_P]),
    "adg_leaf_info": (_I, [_P, _P, _S]),
    "adg_adapt": (_I, [_P, _P, _P, _P]),
    "adg_last_error": (ctypes.c_char_p, []),
}

_lib = None


def lib():
    """Load libaderdg.so once; raise if it is missing (no fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libaderdg.so not built ({LIB_PATH}); run "
                               "`python -m paper_1905_05524_gb300.build` first")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(code):
    if code != ADG_OK:
        msg = lib().adg_last_error().decode(errors="replace")
        raise AdgError(code, msg)
    return code
