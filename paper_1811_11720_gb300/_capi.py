"""ctypes declarations mirroring include/qmc_gb300.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libqmc_gb300.so")

QMC_MAX_DIM = 16
QMC_MAX_SHIFTS = 1024
QMC_MAX_TERMS = 512
QMC_NOALLOC_SCRATCH_BYTES = 8 << 20

STATUS = {
    0: "QMC_OK", -1: "QMC_ERR_ARG", -2: "QMC_ERR_DIM", -3: "QMC_ERR_N", -4: "QMC_ERR_GENVEC",
    -5: "QMC_ERR_M", -6: "QMC_ERR_FIT_PARAMS", -7: "QMC_ERR_INTEGRAND", -8: "QMC_ERR_TRANSFORM",
    -9: "QMC_ERR_CUDA", -10: "QMC_ERR_WORKSPACE", -11: "QMC_ERR_NONFINITE", -12: "QMC_ERR_RANGE",
    -13: "QMC_ERR_NO_DEVICE",
}
QMC_ERR_NONFINITE = -11

FAMILY = {"oscillatory": 1, "product_peak": 2, "corner_peak": 3, "gaussian": 4, "c0": 5,
          "discontinuous": 6, "monomial": 10, "trig": 11, "feynman": 20, "sector": 21}
TRANSFORM = {"none": 0, "baker": 1, "korobov": 2, "sidi": 3}
ERRORMODE = {"all": 0, "largest": 1}


class qmc_c64(C.Structure):
    _fields_ = [("re", C.c_double), ("im", C.c_double)]


class qmc_result(C.Structure):
    _fields_ = [("integral", qmc_c64), ("error", qmc_c64), ("n", C.c_uint64), ("m", C.c_uint64),
                ("iterations", C.c_uint64), ("evaluations", C.c_uint64),
                ("nonfinite", C.c_uint64), ("signfail", C.c_uint64)]


class qmc_integrand(C.Structure):
    _fields_ = [("family", C.c_int), ("dim", C.c_int),
                ("c", C.c_void_p), ("w", C.c_void_p), ("h", C.c_void_p),
                ("nu", C.c_int), ("nf", C.c_int),
                ("ucoef", C.c_void_p), ("fcoef", C.c_void_p),
                ("uexp", C.c_void_p), ("fexp", C.c_void_p),
                ("pa", C.c_double), ("pb", C.c_double), ("lambda_", C.c_double)]


class qmc_transform(C.Structure):
    _fields_ = [("kind", C.c_int), ("r0", C.c_int), ("r1", C.c_int)]


class qmc_genvec_table(C.Structure):
    _fields_ = [("n", C.c_void_p), ("z", C.c_void_p), ("s_max", C.c_int), ("count", C.c_int)]


class qmc_rule(C.Structure):
    _fields_ = [("n", C.c_uint64), ("dim", C.c_int), ("z", C.c_uint64 * QMC_MAX_DIM),
                ("m", C.c_uint64), ("shifts", C.c_void_p), ("transform", qmc_transform),
                ("fit", C.c_void_p)]


class qmc_batch_item(C.Structure):
    _fields_ = [("f", qmc_integrand), ("rule", qmc_rule), ("i_begin", C.c_uint64),
                ("i_end", C.c_uint64)]


class qmc_batch_config(C.Structure):
    _fields_ = [("streams_per_block", C.c_int), ("points_per_stream", C.c_uint32)]


class qmc_server_config(C.Structure):
    _fields_ = [("memory_budget", C.c_size_t), ("max_slots", C.c_int), ("m", C.c_uint64),
                ("transform", qmc_transform), ("step_evaluations", C.c_uint64)]


class qmc_fit_opts(C.Structure):
    _fields_ = [("enabled", C.c_int), ("evaluateminn", C.c_uint64), ("bins", C.c_int),
                ("maxiter", C.c_int), ("xtol", C.c_double), ("gtol", C.c_double),
                ("ftol", C.c_double), ("stepsize", C.c_int)]


class qmc_options(C.Structure):
    _fields_ = [("epsrel", C.c_double), ("epsabs", C.c_double), ("maxeval", C.c_uint64),
                ("errormode", C.c_int)]


# name -> (restype, argtypes)
_P = C.POINTER
PROTOTYPES = {
    "qmc_strerror": (C.c_char_p, [C.c_int]),
    "qmc_abi_version": (C.c_int, []),
    "qmc_get_next_n": (C.c_int, [_P(qmc_genvec_table), C.c_uint64, _P(C.c_uint64)]),
    "qmc_make_shifts": (C.c_int, [C.c_uint64, C.c_uint64, C.c_int, C.c_void_p]),
    "qmc_points": (C.c_int, [_P(qmc_rule), C.c_uint64, C.c_uint64, C.c_void_p, C.c_void_p]),
    "qmc_sums_workspace_bytes": (C.c_size_t, [_P(qmc_rule), C.c_int, C.c_uint64, C.c_uint64]),
    "qmc_sums": (C.c_int, [_P(qmc_integrand), _P(qmc_rule), C.c_uint64, C.c_uint64, C.c_void_p,
                           C.c_size_t, C.c_void_p, C.c_void_p, C.c_void_p]),
    "qmc_sums_noalloc": (C.c_int, [_P(qmc_integrand), _P(qmc_rule), C.c_uint64, C.c_uint64,
                                   C.c_void_p, C.c_void_p, C.c_void_p]),
    "qmc_finalize": (C.c_int, [C.c_void_p, C.c_uint64, C.c_uint64, C.c_int, C.c_void_p,
                               C.c_void_p, C.c_void_p]),
    "qmc_evaluate": (C.c_int, [_P(qmc_integrand), C.c_uint64, C.c_void_p, C.c_int, C.c_void_p,
                               C.c_uint64, C.c_uint64, C.c_void_p, C.c_void_p]),
    "qmc_histogram_workspace_bytes": (C.c_size_t, [C.c_uint64, C.c_int, C.c_int]),
    "qmc_histogram": (C.c_int, [_P(qmc_integrand), C.c_uint64, C.c_void_p, C.c_int, C.c_void_p,
                                C.c_int, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "qmc_fit_polysingular": (C.c_int, [C.c_void_p, C.c_int, C.c_int, _P(qmc_fit_opts), C.c_void_p]),
    "qmc_batch_workspace_bytes": (C.c_size_t, [_P(qmc_batch_item), C.c_int, _P(qmc_batch_config)]),
    "qmc_batch_sums": (C.c_int, [_P(qmc_batch_item), C.c_int, _P(qmc_batch_config), C.c_void_p,
                                 C.c_size_t, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "qmc_batch_autotune": (C.c_int, [_P(qmc_batch_item), C.c_int, C.c_void_p, C.c_size_t,
                                     C.c_void_p, C.c_void_p, _P(qmc_batch_config)]),
    "qmc_batch_plan_create": (C.c_int, [_P(qmc_batch_item), C.c_int, _P(qmc_batch_config),
                                        C.c_void_p, C.c_size_t, C.c_void_p, _P(C.c_void_p)]),
    "qmc_batch_plan_run": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "qmc_batch_plan_destroy": (None, [C.c_void_p]),
    "qmc_server_create": (C.c_int, [_P(qmc_genvec_table), _P(qmc_server_config), C.c_void_p,
                                    _P(C.c_void_p)]),
    "qmc_server_destroy": (None, [C.c_void_p]),
    "qmc_server_submit": (C.c_int, [C.c_void_p, _P(qmc_integrand), C.c_double, C.c_double,
                                    C.c_uint64, C.c_uint64, C.c_uint64, _P(C.c_uint64)]),
    "qmc_server_step": (C.c_int, [C.c_void_p, _P(C.c_int)]),
    "qmc_server_status": (C.c_int, [C.c_void_p, C.c_uint64, _P(C.c_int), _P(qmc_result),
                                    _P(C.c_double)]),
    "qmc_server_counts": (C.c_int, [C.c_void_p, _P(C.c_int), _P(C.c_int), _P(C.c_size_t)]),
    "qmc_server_completed": (C.c_int, [C.c_void_p, _P(C.c_uint64), C.c_int, _P(C.c_int)]),
    "qmc_sums_tile_count": (C.c_int, [C.c_uint64, C.c_uint64, _P(C.c_uint64), _P(C.c_uint64)]),
    "qmc_sums_tiles": (C.c_int, [_P(qmc_integrand), _P(qmc_rule), C.c_uint64, C.c_uint64,
                                 C.c_uint64, C.c_uint64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "qmc_reduce_tiles": (C.c_int, [C.c_void_p, C.c_uint64, C.c_uint64, C.c_int, C.c_void_p,
                                   C.c_void_p]),
    "qmc_merge_sums": (C.c_int, [C.c_void_p, C.c_uint64, C.c_uint64, C.c_void_p]),
    "qmc_probe_units": (C.c_int, [C.c_int, C.c_uint32, C.c_void_p, _P(C.c_double), C.c_void_p]),
    "qmc_cbc_device_bytes": (C.c_size_t, [C.c_uint64]),
    "qmc_cbc_korobov": (C.c_int, [C.c_uint64, C.c_int, C.c_double, C.c_double, _P(C.c_uint64),
                                  _P(C.c_double), C.c_void_p]),
    "qmc_integrate": (C.c_int, [_P(qmc_integrand), _P(qmc_genvec_table), C.c_uint64, C.c_uint64,
                                qmc_transform, _P(qmc_fit_opts), C.c_uint64, _P(qmc_options),
                                C.c_void_p, _P(qmc_result)]),
}


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load the compiled library.  Raises if it has not been built: there is no fallback."""
    if not os.path.exists(path):
        raise ImportError(
            f"libqmc_gb300.so not found at {path}; build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc, sm_103a)")
    lib = C.CDLL(path)
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib
