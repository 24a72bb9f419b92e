"""ctypes declarations of libpmcmc (include/pmcmc.h).  Marshalling only: no arithmetic here."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpmcmc.so")

# enums (values of include/pmcmc.h)
PMCMC_OK, PMCMC_NOT_CONVERGED = 0, 1
PMCMC_EINVAL, PMCMC_ENOMEM, PMCMC_ECUDA, PMCMC_ETIMEOUT, PMCMC_ENAN, PMCMC_EUNSUPPORTED = (
    -1, -2, -3, -4, -5, -6)
STATUS_NAMES = {0: "OK", 1: "NOT_CONVERGED", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA",
                -4: "ETIMEOUT", -5: "ENAN", -6: "EUNSUPPORTED"}
SAMPLERS = {"mala": 0, "hmc": 1, "hmc_par_leapfrog": 2, "gibbs": 3}
TARGETS = {"gaussian": 0, "logreg": 1, "banana": 2, "schools": 3}
JACS = {"dense": 0, "diag": 1, "block2": 2, "diag_hutch": 3, "zero": 4}
PRECISIONS = {"f64": 0, "f32": 1, "f32_scan_bf16": 2}
ENGINES = {"auto": 0, "simt": 1}


class pmcmc_target(C.Structure):
    _fields_ = [("kind", C.c_int), ("D", C.c_int), ("N", C.c_int),
                ("mean", C.c_void_p), ("prec", C.c_void_p), ("X", C.c_void_p),
                ("y", C.c_void_p), ("prior_scale", C.c_double), ("Q", C.c_void_p)]


class pmcmc_options(C.Structure):
    _fields_ = [("sampler", C.c_int), ("step", C.c_double), ("leapfrog_L", C.c_int),
                ("jac", C.c_int), ("precision", C.c_int), ("atol", C.c_double),
                ("rtol", C.c_double), ("max_iters", C.c_int), ("damping", C.c_double),
                ("clip", C.c_int), ("gate_grad", C.c_int), ("seed", C.c_ulonglong),
                ("chain_id", C.c_uint), ("spin_limit", C.c_int),
                ("engine", C.c_int), ("seq_after", C.c_int), ("window", C.c_int)]


class pmcmc_result(C.Structure):
    _fields_ = [("iters", C.c_int), ("status", C.c_int), ("max_residual", C.c_double),
                ("accept_rate", C.c_double), ("min_margin", C.c_double),
                ("nonfinite_resets", C.c_int), ("elapsed_ms", C.c_float), ("sequential", C.c_int)]


class pmcmc_chain_desc(C.Structure):
    _fields_ = [("target", pmcmc_target), ("sampler", C.c_int), ("step", C.c_double),
                ("leapfrog_L", C.c_int), ("T", C.c_int), ("s0", C.c_void_p),
                ("xi", C.c_void_p), ("u", C.c_void_p), ("s_out", C.c_void_p)]


class pmcmc_profile(C.Structure):
    _fields_ = [("launches", C.c_longlong), ("eval_launches", C.c_longlong),
                ("eval_ms", C.c_double), ("jac_launches", C.c_longlong), ("jac_ms", C.c_double),
                ("scan_launches", C.c_longlong), ("scan_ms", C.c_double)]


EXPORTS = [
    "pmcmc_options_default", "pmcmc_create", "pmcmc_destroy", "pmcmc_last_error",
    "pmcmc_gen_noise", "pmcmc_solve", "pmcmc_seq_solve", "pmcmc_linearize", "pmcmc_scan",
    "pmcmc_adjoint", "pmcmc_solve_batched", "pmcmc_profile_enable", "pmcmc_profile_get",
    "pmcmc_scan_noalloc", "pmcmc_seq_solve_batched", "pmcmc_scan_plan",
]

_lib = None


def load(path: str = LIB_PATH):
    """Load libpmcmc.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with "
                           "`python -m paper_2508_18413_gb300.build` (the CUDA path has no "
                           "fallback)")
    lib = C.CDLL(path)
    vp, i, d, st = C.c_void_p, C.c_int, C.c_double, C.c_int
    lib.pmcmc_options_default.argtypes = [C.POINTER(pmcmc_options)]
    lib.pmcmc_options_default.restype = None
    lib.pmcmc_create.argtypes = [C.POINTER(vp), i]
    lib.pmcmc_create.restype = st
    lib.pmcmc_destroy.argtypes = [vp]
    lib.pmcmc_destroy.restype = st
    lib.pmcmc_last_error.argtypes = [vp]
    lib.pmcmc_last_error.restype = C.c_char_p
    lib.pmcmc_gen_noise.argtypes = [vp, C.c_ulonglong, C.c_uint, i, i, i, vp, vp, vp]
    lib.pmcmc_gen_noise.restype = st
    lib.pmcmc_solve.argtypes = [vp, C.POINTER(pmcmc_target), C.POINTER(pmcmc_options), i, vp,
                                vp, vp, vp, vp, C.POINTER(pmcmc_result), vp]
    lib.pmcmc_solve.restype = st
    lib.pmcmc_solve_async.argtypes = [vp, C.POINTER(pmcmc_target), C.POINTER(pmcmc_options), i,
                                      vp, vp, vp, vp, vp, vp, vp]
    lib.pmcmc_solve_async.restype = st
    lib.pmcmc_seq_solve.argtypes = [vp, C.POINTER(pmcmc_target), C.POINTER(pmcmc_options), i,
                                    vp, vp, vp, vp, vp, vp]
    lib.pmcmc_seq_solve.restype = st
    lib.pmcmc_linearize.argtypes = [vp, C.POINTER(pmcmc_target), C.POINTER(pmcmc_options), i,
                                    vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.pmcmc_linearize.restype = st
    lib.pmcmc_scan.argtypes = [vp, i, i, i, i, vp, vp, vp, vp]
    lib.pmcmc_scan.restype = st
    lib.pmcmc_adjoint.argtypes = [vp, C.POINTER(pmcmc_target), C.POINTER(pmcmc_options), i, vp,
                                  vp, vp, vp, vp, vp, C.c_size_t, vp, C.POINTER(d), vp]
    lib.pmcmc_adjoint.restype = st
    lib.pmcmc_solve_batched.argtypes = [vp, i, C.POINTER(pmcmc_chain_desc),
                                        C.POINTER(pmcmc_options), C.POINTER(pmcmc_result), vp]
    lib.pmcmc_solve_batched.restype = st
    lib.pmcmc_seq_solve_batched.argtypes = [vp, i, C.POINTER(pmcmc_chain_desc),
                                            C.POINTER(pmcmc_options), vp]
    lib.pmcmc_seq_solve_batched.restype = st
    lib.pmcmc_scan_noalloc.argtypes = [i, i, i, vp, vp, vp, vp]
    lib.pmcmc_scan_noalloc.restype = st
    ip = C.POINTER(C.c_int)
    lib.pmcmc_scan_plan.argtypes = [i, i, i, i, ip, ip, ip, ip]
    lib.pmcmc_scan_plan.restype = st
    lib.pmcmc_profile_enable.argtypes = [vp, i]
    lib.pmcmc_profile_enable.restype = st
    lib.pmcmc_profile_get.argtypes = [vp, C.POINTER(pmcmc_profile)]
    lib.pmcmc_profile_get.restype = st
    _lib = lib
    return lib
