"""ctypes declarations of the C ABI in include/lbm.h (argument marshalling
only).  Loading fails loudly when the compiled library is missing: there is
no CPU fallback."""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblbm.so")

LBM_OK, LBM_EINVAL, LBM_EDEGREE, LBM_ENOMEM, LBM_ECUDA = 0, -1, -2, -3, -4
LBM_ENONFINITE, LBM_ETIMEOUT, LBM_ENOTCONV, LBM_ENOTSUP = -5, -6, -7, -8
LBM_FP64, LBM_FP32, LBM_FP16, LBM_BF16 = 0, 1, 2, 3
LBM_MAX_V = 128

c_int_p = ctypes.POINTER(ctypes.c_int)
c_double_p = ctypes.POINTER(ctypes.c_double)
c_long_p = ctypes.POINTER(ctypes.c_long)
c_size_p = ctypes.POINTER(ctypes.c_size_t)


class lbm_dvm(ctypes.Structure):
    _fields_ = [("D", ctypes.c_int), ("V", ctypes.c_int), ("e", c_int_p),
                ("w", c_double_p), ("c", ctypes.c_double)]


# name -> (restype, argtypes), in the order of include/lbm.h
SIGNATURES = {
    "lbm_dvm_expand": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, c_int_p, c_int_p, c_double_p,
                                      ctypes.c_int, c_int_p, c_double_p, c_int_p]),
    "lbm_dvm_marginal_xz": (ctypes.c_int, [ctypes.c_int, c_int_p, c_double_p, ctypes.c_int,
                                           c_int_p, c_double_p, c_int_p]),
    "lbm_dvm_quadrature_order": (ctypes.c_int, [ctypes.POINTER(lbm_dvm), c_int_p]),
    "lbm_dvm_solve_weights": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, c_int_p, ctypes.c_double,
                                             ctypes.c_int, c_double_p, c_int_p]),
    "lbm_dvm_find_c": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, c_int_p, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_double, c_double_p]),
    "lbm_dvm_nontrivial_moments": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, c_int_p,
                                                  c_int_p]),
    "lbm_dvm_augment": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, c_int_p, ctypes.c_double,
                                       ctypes.c_int, ctypes.c_int, c_int_p, c_double_p,
                                       c_double_p]),
    "lbm_workspace_bytes": (ctypes.c_int, [ctypes.POINTER(lbm_dvm), ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, c_size_p]),
    "lbm_create": (ctypes.c_int, [ctypes.POINTER(lbm_dvm), ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                  ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "lbm_create_in": (ctypes.c_int, [ctypes.POINTER(lbm_dvm), ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_size_t, ctypes.POINTER(ctypes.c_void_p)]),
    "lbm_destroy": (None, [ctypes.c_void_p]),
    "lbm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "lbm_init": (ctypes.c_int, [ctypes.c_void_p, c_double_p]),
    "lbm_init_device": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "lbm_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_long]),
    "lbm_average": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_long, ctypes.c_long]),
    "lbm_fma_rate": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "lbm_set_resident": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "lbm_resident_ctas": (ctypes.c_int, [ctypes.c_void_p, c_int_p]),
    "lbm_run_to_steady": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_long,
                                         ctypes.c_long, c_long_p, c_double_p]),
    "lbm_moments": (ctypes.c_int, [ctypes.c_void_p, c_double_p, c_double_p, c_double_p]),
    "lbm_mass_flow": (ctypes.c_int, [ctypes.c_void_p, c_double_p, c_double_p]),
    "lbm_slip_velocity": (ctypes.c_int, [ctypes.c_void_p, c_double_p]),
    "lbm_status": (ctypes.c_int, [ctypes.c_void_p]),
    "lbm_knudsen_layer": (ctypes.c_int, [ctypes.c_void_p, c_double_p]),
    "lbm_steps_done": (ctypes.c_int, [ctypes.c_void_p, c_long_p]),
    "lbm_populations": (ctypes.c_int, [ctypes.c_void_p, c_double_p]),
    "lbm_state_bytes": (ctypes.c_int, [ctypes.c_void_p, c_size_p]),
    "lbm_get_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "lbm_set_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "lbm_engine_solve_bytes": (ctypes.c_int, [ctypes.POINTER(lbm_dvm), ctypes.c_int, ctypes.c_int,
                                              ctypes.c_int, c_size_p]),
    "lbm_engine_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                         ctypes.c_size_t, ctypes.c_void_p,
                                         ctypes.POINTER(ctypes.c_void_p)]),
    "lbm_engine_destroy": (None, [ctypes.c_void_p]),
    "lbm_engine_add": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(lbm_dvm), ctypes.c_int,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_double, c_double_p, c_int_p]),
    "lbm_engine_remove": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "lbm_engine_set_chunk": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "lbm_engine_set_resident": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "lbm_engine_paths": (ctypes.c_int, [ctypes.c_void_p, c_int_p, c_int_p]),
    "lbm_engine_state_bytes": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_size_t)]),
    "lbm_engine_get_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                            ctypes.c_size_t]),
    "lbm_engine_set_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                            ctypes.c_size_t]),
    "lbm_engine_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, c_double_p]),
    "lbm_engine_launch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "lbm_engine_wait": (ctypes.c_int, [ctypes.c_void_p, c_double_p]),
    "lbm_engine_autotune": (ctypes.c_int, [ctypes.c_void_p, c_double_p]),
    "lbm_engine_set_schedule": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_int, ctypes.c_int, ctypes.c_double]),
    "lbm_engine_get_schedule": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, c_int_p, c_int_p,
                                               c_int_p, c_double_p]),
    "lbm_engine_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, c_long_p, c_int_p]),
    "lbm_engine_moments": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, c_double_p, c_double_p,
                                          c_double_p]),
    "lbm_engine_free_bytes": (ctypes.c_int, [ctypes.c_void_p, c_size_p]),
    "lbm_observables_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                                               ctypes.c_void_p]),
}

_lib = None


def lib():
    """The loaded liblbm.so with every signature declared."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"CUDA library {LIB_PATH} is missing: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'` "
                "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class LBMError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        msg = lib().lbm_strerror(code).decode()
        super().__init__(f"{where}: {msg} ({code})" if where else f"{msg} ({code})")


def check(code, where=""):
    if code != LBM_OK:
        raise LBMError(code, where)
    return code
