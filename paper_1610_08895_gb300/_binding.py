"""ctypes binding of the C ABI in include/pd.h (argument marshalling only).

Every function here forwards to the CUDA library ``_lib/libpdgb.so``; nothing
computes on the host. If the library is missing, loading raises
``ExtensionMissing`` -- there is no fallback path.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libpdgb.so")

PD_OK, PD_EINVAL, PD_ENOMEM, PD_ECUDA, PD_ETIMEOUT, PD_ENOTCONV, PD_ENOTSUP = range(7)
PD_F32, PD_F64 = 0, 1
PD_G_ON_THE_FLY, PD_G_CSR = 0, 1
STATUS_NAMES = {0: "PD_OK", 1: "PD_EINVAL", 2: "PD_ENOMEM", 3: "PD_ECUDA", 4: "PD_ETIMEOUT",
                5: "PD_ENOTCONV", 6: "PD_ENOTSUP"}


class ExtensionMissing(RuntimeError):
    """The compiled CUDA library is not present (run __graft_entry__.build())."""


class PDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class PdPlanDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("osf", ctypes.c_int32),
                ("nvis", ctypes.c_int64), ("uv", ctypes.c_void_p), ("nblocks", ctypes.c_int32),
                ("block_of_vis", ctypes.c_void_p), ("kernel_width", ctypes.c_int32),
                ("kb_beta", ctypes.c_double), ("nbases", ctypes.c_int32), ("basis_ids", ctypes.c_void_p),
                ("levels", ctypes.c_int32), ("precision", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("g_mode", ctypes.c_int32), ("dde_width", ctypes.c_int32), ("dde_kernels", ctypes.c_void_p)]


class PdParams(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("sigma", ctypes.c_double), ("varsigma", ctypes.c_double),
                ("kappa", ctypes.c_double), ("psi_norm", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("p_block", ctypes.c_void_p), ("p_basis", ctypes.c_void_p), ("adaptive", ctypes.c_int32),
                ("adapt_n", ctypes.c_double), ("adapt_p_min", ctypes.c_double),
                ("adapt_p_max", ctypes.c_double), ("use_graph", ctypes.c_int32), ("profile", ctypes.c_int32),
                ("adapt_exact", ctypes.c_int32), ("per_block", ctypes.c_int32),
                ("sparsity_weights", ctypes.c_void_p)]


_lib = None
_VP = ctypes.c_void_p
_SIGS = {
    "pd_plan_create": ([ctypes.POINTER(PdPlanDesc), ctypes.POINTER(_VP)], ctypes.c_int),
    "pd_plan_destroy": ([_VP], ctypes.c_int),
    "pd_plan_autotune": ([ctypes.POINTER(PdPlanDesc), _VP, ctypes.c_int32, ctypes.c_int32, _VP, _VP, _VP],
                         ctypes.c_int),
    "pd_last_error": ([], ctypes.c_char_p),
    "pd_plan_info": ([_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "pd_daubechies_filter": ([ctypes.c_int32, _VP], ctypes.c_int),
    "pd_apply_phi": ([_VP, _VP, _VP, ctypes.c_int32, _VP], ctypes.c_int),
    "pd_apply_phi_adj": ([_VP, _VP, _VP, ctypes.c_int32, _VP], ctypes.c_int),
    "pd_apply_psi_adj": ([_VP, _VP, _VP, _VP], ctypes.c_int),
    "pd_sara_weights": ([_VP, _VP, ctypes.c_double, _VP, _VP], ctypes.c_int),
    "pd_apply_psi": ([_VP, _VP, _VP, _VP], ctypes.c_int),
    "pd_apply_psi_adj_noalloc": ([_VP, _VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _VP, ctypes.c_int32,
                                  ctypes.c_int32, _VP], ctypes.c_int),
    "pd_operator_norms": ([_VP, _VP, ctypes.c_int32, ctypes.c_double, _VP, _VP, _VP, _VP], ctypes.c_int),
    "pd_state_create": ([_VP, ctypes.POINTER(_VP)], ctypes.c_int),
    "pd_state_destroy": ([_VP], ctypes.c_int),
    "pd_state_set_data": ([_VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "pd_state_set_start": ([_VP, _VP, _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "pd_iterate": ([_VP, _VP, ctypes.POINTER(PdParams), ctypes.c_int32, _VP], ctypes.c_int),
    "pd_synthesis_iterate": ([_VP, _VP, ctypes.POINTER(PdParams), ctypes.c_int32, _VP], ctypes.c_int),
    "pd_iterate_dual": ([_VP, _VP, ctypes.POINTER(PdParams), _VP], ctypes.c_int),
    "pd_iterate_primal": ([_VP, _VP, ctypes.POINTER(PdParams), _VP, _VP], ctypes.c_int),
    "pd_state_u": ([_VP, ctypes.POINTER(_VP), _VP], ctypes.c_int),
    "pd_state_get_x": ([_VP, _VP, _VP], ctypes.c_int),
    "pd_state_get_x_tilde": ([_VP, _VP, _VP], ctypes.c_int),
    "pd_state_get_s": ([_VP, _VP, _VP], ctypes.c_int),
    "pd_state_get_v": ([_VP, _VP, _VP, _VP], ctypes.c_int),
    "pd_state_report": ([_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "pd_state_bytes": ([_VP], ctypes.c_size_t),
    "pd_state_profile": ([_VP, _VP, _VP, ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
    "pd_phase_name": ([ctypes.c_int32], ctypes.c_char_p),
    "pd_state_save": ([_VP, _VP, _VP, _VP], ctypes.c_int),
    "pd_state_load": ([_VP, _VP, _VP, _VP], ctypes.c_int),
}


def exported_symbols():
    """Names of the C ABI functions this binding declares."""
    return sorted(_SIGS)


def load():
    """Load the CUDA library (once). Raises ExtensionMissing if it was not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ExtensionMissing(f"CUDA library not built: {LIB_PATH} is missing; run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (args, res) in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def check(status, where=""):
    if status != PD_OK:
        msg = load().pd_last_error().decode()
        raise PDError(status, f"{where}: {msg}" if where else msg)
    return status


def call(name, *args):
    """Call a C ABI function by name and raise PDError on a non-OK status."""
    return check(getattr(load(), name)(*args), name)
