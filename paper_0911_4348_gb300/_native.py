"""ctypes loader for libfedvr_negf.so with the C ABI of include/fedvr_negf.h.

The library is built in-tree by ``paper_0911_4348_gb300.build``. Loading
fails loudly if it is missing: there is no fallback implementation.
"""

from __future__ import annotations

import ctypes as C
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libfedvr_negf.so")

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_vp = C.c_void_p

# name -> (restype, argtypes); every function declared in include/fedvr_negf.h
SIGNATURES = {
    "fedvr_create": (C.c_int, [C.POINTER(_vp), _vp]),
    "fedvr_destroy": (None, [_vp]),
    "fedvr_last_error": (C.c_char_p, [_vp]),
    "build_fedvr": (C.c_int, [_vp, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int, _ip]),
    "set_potential": (C.c_int, [_vp, C.c_int, _dp, _dp, C.c_double, C.c_double, C.c_int, _dp]),
    "fedvr_get_basis": (C.c_int, [_vp, _dp, _dp, _ip, _ip]),
    "fedvr_get_gll": (C.c_int, [_vp, _dp, _dp]),
    "fedvr_get_operators": (C.c_int, [_vp, _dp, _dp, _dp, _dp]),
    "solve_hf": (C.c_int, [_vp, C.c_double, C.c_double, C.c_int, _dp, _dp]),
    "fedvr_get_hf": (C.c_int, [_vp, _dp, _dp, _dp, _dp]),
    "fedvr_density": (C.c_int, [_vp, C.c_int, _dp]),
    "solve_2b": (C.c_int, [_vp, C.c_double, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int,
                           C.c_int, C.c_int, _vp, _vp, _vp, _dp, _dp, _ip]),
    "fedvr_2b_prepare": (C.c_int, [_vp, C.c_double, C.c_int, C.c_int, C.c_int]),
    "fedvr_2b_step": (C.c_int, [_vp, C.c_double, _vp, C.c_int, _dp, _dp, _dp]),
    "fedvr_2b_read": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp]),
    "fedvr_stage_times": (C.c_int, [_vp, _dp, _ip]),
    "fedvr_use_graphs": (C.c_int, [_vp, C.c_int, _ip]),
    "fedvr_conv1_splits": (C.c_int, [_vp, C.c_int, _ip]),
    "fedvr_set_quadrature": (C.c_int, [_vp, C.c_int]),
    "fedvr_set_mu": (C.c_int, [_vp, C.c_double]),
    "fedvr_set_initial_sigma": (C.c_int, [_vp, _vp, C.c_int, C.c_int, C.c_int]),
    "fedvr_get_history": (C.c_int, [_vp, _dp, C.c_int, _ip]),
    "solve_2b_batched": (C.c_int, [C.POINTER(_vp), C.c_int, _dp, _ip, _ip, C.c_double, C.c_double,
                                   C.c_int, C.c_int, _dp, _dp, _ip]),
    "fedvr_batch_create": (C.c_int, [C.POINTER(_vp), C.POINTER(_vp), C.c_int, _dp, _ip, _ip,
                                     C.c_int]),
    "fedvr_batch_step": (C.c_int, [_vp, C.c_double, C.c_double, _ip, _dp, _dp, _dp]),
    "fedvr_batch_destroy": (None, [_vp]),
    "fedvr_mlp_create": (C.c_int, [C.POINTER(_vp), C.c_int, C.c_int, C.c_ulonglong, _vp]),
    "fedvr_mlp_destroy": (None, [_vp]),
    "fedvr_mlp_last_error": (C.c_char_p, [_vp]),
    "fedvr_mlp_num_params": (C.c_int, [_vp, C.POINTER(C.c_long)]),
    "fedvr_mlp_get_params": (C.c_int, [_vp, C.POINTER(C.c_float), C.c_long]),
    "fedvr_mlp_set_params": (C.c_int, [_vp, C.POINTER(C.c_float), C.c_long]),
    "fedvr_mlp_loss_grad": (C.c_int, [_vp, _vp, _vp, C.c_int, C.POINTER(C.c_float), _dp]),
    "fedvr_mlp_forward": (C.c_int, [_vp, _vp, C.c_int, _vp, C.c_int]),
    "fedvr_mlp_collect": (C.c_int, [_vp, _vp, C.c_double, C.c_int, C.c_int, C.c_double, C.c_double,
                                    C.c_int, _ip]),
    "fedvr_mlp_train": (C.c_int, [_vp, C.c_int, C.c_int, C.c_double, _dp]),
    "fedvr_mlp_rows": (C.c_int, [_vp, C.POINTER(C.c_long)]),
    "fedvr_mlp_get_rows": (C.c_int, [_vp, C.c_long, C.c_long, C.POINTER(C.c_float),
                                     C.POINTER(C.c_float)]),
    "fedvr_warm_start": (C.c_int, [_vp, _vp, C.c_double, C.c_int, C.c_int, C.c_int]),
    "fedvr_power_mesh": (C.c_int, [_vp, C.c_double, C.c_int, C.c_int, _vp, _vp, _vp, _vp, _vp,
                                   _vp]),
    "fedvr_sigma2": (C.c_int, [_vp, C.c_int, C.c_int, C.c_double, _vp, _vp, _vp, C.c_int]),
    "fedvr_sigma2_noalloc": (C.c_int, [C.c_int, C.c_int, C.c_double, _vp, _vp, _vp, _vp]),
    "fedvr_conv_sigma_g": (C.c_int, [_vp, C.c_int, C.c_double, C.c_int, C.c_int, _vp, _vp, _vp,
                                     _vp, C.c_int]),
    "fedvr_conv_g0": (C.c_int, [_vp, C.c_int, C.c_double, C.c_int, C.c_int, _vp, _vp, C.c_double,
                                _vp, _vp, C.c_int]),
    "fedvr_selftest_wait": (C.c_int, [_vp, C.c_int, C.c_double]),
    "fedvr_kbe_propagate": (C.c_int, [_vp, C.c_double, C.c_int, C.c_int, C.c_int, _dp, _dp, _dp,
                                      _dp, _dp]),
    "fedvr_kbe_get_block": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, _dp]),
    "fedvr_kbe_stats": (C.c_int, [_vp, _dp]),
    "fedvr_set_self_energy": (C.c_int, [_vp, C.c_int, C.c_double, C.c_double, C.c_int]),
    "fedvr_gw_last_inner": (C.c_int, [_vp, _ip]),
    "fedvr_sigma_gw": (C.c_int, [_vp, C.c_int, C.c_double, C.c_int, C.c_int, C.c_double, _vp, _vp,
                                 _vp, _vp, C.c_int, C.c_double, C.c_double, C.c_int, _ip]),
    "fedvr_sigma_tmatrix": (C.c_int, [_vp, C.c_int, C.c_double, C.c_int, C.c_int, C.c_double,
                                      _vp, _vp, _vp, _vp, C.c_int, C.c_double, C.c_double,
                                      C.c_int, _ip]),
}

_lib = None


def lib() -> C.CDLL:
    """Load the library once and declare every signature."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; "
                "g.build()'` (nvcc, sm_103a). There is no CPU fallback.")
        handle = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib
