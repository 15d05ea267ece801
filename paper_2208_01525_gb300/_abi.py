"""ctypes mirror of include/u1u1.h (argument marshalling only).

The shared library is built in-tree by ``paper_2208_01525_gb300.build``;
loading fails loudly when it is missing.  There is no fallback path: every
step of the computation runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libu1u1.so")

U1U1_OK = 0
ERRORS = {
    -1: "INVALID_ARG", -2: "BAD_BUFFER", -3: "OUT_OF_MEMORY", -4: "CUDA", -5: "TIMEOUT",
    -6: "NAN", -7: "NOT_SUPPORTED", -8: "STATE", -9: "IO",
}
FP32, FP64 = 0, 1
NOALLOC_MAX_SITES = 16777216
NPOS, NMOM = 10, 10
NFIELDS = NPOS + NMOM
KERNEL_AUTO, KERNEL_SIMPLE, KERNEL_TILED = 0, 1, 2
ENS_PERSISTENT, ENS_PER_STEP, ENS_UNBATCHED = 0, 1, 2


class U1U1Error(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"u1u1 error {ERRORS.get(code, code)}: {msg}")
        self.code = code


class CParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("dx", ctypes.c_double), ("deta", ctypes.c_double), ("eta0", ctypes.c_double),
        ("m", ctypes.c_double), ("eta_ref", ctypes.c_double), ("beta", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("lambda_p", ctypes.c_double), ("lambda_q", ctypes.c_double),
        ("e_p", ctypes.c_double), ("e_q", ctypes.c_double),
        ("sigma_p", ctypes.c_double), ("sigma_q", ctypes.c_double),
        ("kappa", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("precision", ctypes.c_int),
    ]


class CBuffers(ctypes.Structure):
    _fields_ = [("pos", (ctypes.c_void_p * NPOS) * 2), ("mom", ctypes.c_void_p * NMOM)]


class CStrings(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64), ("eta", ctypes.c_double),
        ("n_p", ctypes.c_int64), ("n_q", ctypes.c_int64),
        ("nonzero_p", ctypes.c_int64), ("nonzero_q", ctypes.c_int64),
        ("n_pq_plaq", ctypes.c_int64), ("n_pq_cell", ctypes.c_int64), ("n_pq_cell_q", ctypes.c_int64),
        ("n_flagged", ctypes.c_int64),
        ("max_abs_w", ctypes.c_int32), ("overlap_tol", ctypes.c_int32),
        ("n_w2_p", ctypes.c_int64), ("n_w2_q", ctypes.c_int64),
        ("n_cells_ge4_p", ctypes.c_int64), ("n_cells_ge4_q", ctypes.c_int64),
        ("L_p", ctypes.c_double), ("L_q", ctypes.c_double), ("L_pq", ctypes.c_double),
        ("xi_p", ctypes.c_double), ("xi_q", ctypes.c_double), ("xi_pq", ctypes.c_double),
        ("xi_w", ctypes.c_double), ("f_total", ctypes.c_double), ("f_p", ctypes.c_double),
    ]


class CSegments(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64), ("overlap_tol", ctypes.c_int32), ("min_cells", ctypes.c_int32),
        ("n_cells", ctypes.c_int64), ("n_components", ctypes.c_int64), ("n_segments", ctypes.c_int64),
        ("largest", ctypes.c_int64), ("L_pq", ctypes.c_double), ("l_pq", ctypes.c_double),
        ("xi_pq", ctypes.c_double),
    ]


_DIAG_DOUBLES_1 = ["eta", "a", "kin_p", "kin_q", "grad_p", "grad_q", "el_p", "el_q", "mag_p", "mag_q",
                   "pot", "vint", "pot_p", "pot_q", "lag", "energy", "rl_num", "rl_den", "rpq_num", "rpq_den",
                   "lag_total", "energy_total", "xi_l", "lag_p", "lag_q", "xi_l_p", "xi_l_q",
                   "R_l", "v2_l", "R_pq", "v2_pq"]
_DIAG_DOUBLES_2 = ["gauss_sum_p", "gauss_sum_q", "charge_sum_p", "charge_sum_q", "gauss_max_p",
                   "gauss_max_q", "gauss_rel_p", "gauss_rel_q", "phi_min_p", "phi_max_p",
                   "phi_min_q", "phi_max_q"]


class CDiag(ctypes.Structure):
    _fields_ = ([("n", ctypes.c_int64)] + [(k, ctypes.c_double) for k in _DIAG_DOUBLES_1]
                + [("has_gauss", ctypes.c_int32)] + [(k, ctypes.c_double) for k in _DIAG_DOUBLES_2]
                + [("nan_count", ctypes.c_int64)])


def struct_to_dict(s) -> dict:
    return {name: getattr(s, name) for name, _ in s._fields_}


# every function of the header: name -> (restype, argtypes)
_P = ctypes.POINTER
_vp = ctypes.c_void_p
PROTOTYPES = {
    "u1u1_version": (ctypes.c_char_p, []),
    "u1u1_last_error": (ctypes.c_char_p, []),
    "u1u1_params_default": (ctypes.c_int, [_P(CParams)]),
    "u1u1_check_params": (ctypes.c_int, [_P(CParams)]),
    "u1u1_coefficients": (ctypes.c_int, [_P(CParams), ctypes.c_int64, _P(ctypes.c_double)]),
    "u1u1_field_bytes": (ctypes.c_size_t, [_P(CParams)]),
    "u1u1_abi_sizes": (None, [_P(ctypes.c_size_t)]),
    "u1u1_init_lattice": (ctypes.c_int, [_P(CParams), _P(CBuffers), _vp, _P(_vp)]),
    "u1u1_attach_lattice": (ctypes.c_int, [_P(CParams), _P(CBuffers), ctypes.c_int64, ctypes.c_int, _P(_vp)]),
    "u1u1_destroy": (None, [_vp]),
    "u1u1_current": (ctypes.c_int, [_vp, _P(ctypes.c_int64), _P(ctypes.c_int)]),
    "u1u1_step": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp]),
    "u1u1_set_overlap_tol": (ctypes.c_int, [_vp, ctypes.c_int]),
    "u1u1_cool": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_int, _vp]),
    "u1u1_set_params": (ctypes.c_int, [_vp, _P(CParams), ctypes.c_int64]),
    "u1u1_detect_strings": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp, _P(CStrings), _vp]),
    "u1u1_diagnostics": (ctypes.c_int, [_vp, _P(CDiag), _vp]),
    "u1u1_pq_segments": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp, _P(CSegments), _vp]),
    "u1u1_read_records": (ctypes.c_int, [_vp, _P(CStrings), _P(CDiag), ctypes.c_int, _P(ctypes.c_int),
                                         _P(ctypes.c_int64), _vp]),
    "u1u1_upload_state": (ctypes.c_int, [_vp, _P(_vp), _vp]),
    "u1u1_download_state": (ctypes.c_int, [_vp, _P(_vp), _vp]),
    "u1u1_host_span_mapped": (ctypes.c_int, [_vp, ctypes.c_size_t, _P(ctypes.c_int)]),
    "u1u1_save": (ctypes.c_int, [_vp, ctypes.c_char_p, _vp]),
    "u1u1_load": (ctypes.c_int, [_vp, ctypes.c_char_p, _vp]),
    "u1u1_set_kernel": (ctypes.c_int, [_vp, ctypes.c_int]),
    "u1u1_set_tile_waves": (ctypes.c_int, [_vp, ctypes.c_int]),
    "u1u1_inject_copy_timeout": (ctypes.c_int, [ctypes.c_int, ctypes.c_int64]),
    "u1u1_inject_alloc_failure": (ctypes.c_int, [ctypes.c_int]),
    "u1u1_live_allocations": (ctypes.c_int, [_P(ctypes.c_int64), _P(ctypes.c_int64)]),
    "u1u1_set_alloc_guard": (ctypes.c_int, [ctypes.c_int64]),
    "u1u1_check_alloc_guards": (ctypes.c_int, [_P(ctypes.c_int64)]),
    "u1u1_inject_guard_damage": (ctypes.c_int, []),
    "u1u1_get_kernel": (ctypes.c_int, [_vp, _P(ctypes.c_int)]),
    "u1u1_autotune": (ctypes.c_int, [_vp, ctypes.c_char_p, _P(ctypes.c_int), _P(ctypes.c_int), _vp]),
    "u1u1_eval_link_phase": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int64, _vp]),
    "u1u1_eval_link_phase64": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int64, _vp]),
    "u1u1_eval_edge_phase": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int64, _vp]),
    "u1u1_fp64_fma_rate": (ctypes.c_int, [_P(ctypes.c_double), _vp]),
    "u1u1_ensemble_create": (ctypes.c_int, [_P(CParams), ctypes.c_int, _P(CBuffers), ctypes.c_int, _vp, _P(_vp)]),
    "u1u1_ensemble_run": (ctypes.c_int, [_vp, _P(ctypes.c_int), ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp]),
    "u1u1_ensemble_lattice": (ctypes.c_int, [_vp, ctypes.c_int, _P(_vp)]),
    "u1u1_ensemble_status": (ctypes.c_int, [_vp, _P(ctypes.c_int), _vp]),
    "u1u1_ensemble_set_wait_limit": (ctypes.c_int, [_vp, ctypes.c_int64]),
    "u1u1_ensemble_inject_unreachable_wait": (ctypes.c_int, [_vp, ctypes.c_int]),
    "u1u1_ensemble_destroy": (None, [_vp]),
    "u1u1_ensemble_autotune": (ctypes.c_int, [_vp, ctypes.c_int, _P(ctypes.c_int), _P(ctypes.c_int), _vp]),
    "u1u1_ensemble_set_tuning": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp]),
    "u1u1_ensemble_get_tuning": (ctypes.c_int, [_vp, _P(ctypes.c_int), _P(ctypes.c_int)]),
    "u1u1_detect_strings_noalloc": (ctypes.c_int, [_P(CParams), _P(_vp), ctypes.c_int64, ctypes.c_int,
                                                   _P(CStrings), _vp]),
}

_lib = None


def lib():
    """Load libu1u1.so (building it first if the sources are newer)."""
    global _lib
    if _lib is None:
        from . import build as _build
        if not _build.up_to_date():
            _build.build()
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libu1u1.so missing at {LIB_PATH}; run paper_2208_01525_gb300.build")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in PROTOTYPES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(rc: int) -> None:
    if rc != U1U1_OK:
        msg = lib().u1u1_last_error().decode(errors="replace")
        raise U1U1Error(rc, msg)
