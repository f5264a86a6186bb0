"""ctypes binding of the C ABI in include/pkasp.h (argument marshalling only).

Every function here has the name of the C entry point it calls. The shared library is
built in-tree by ``paper_1204_2586_gb300.build``; if it is missing, ``load()`` raises:
there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpkasp.so")

PKASP_OK, PKASP_EINVAL, PKASP_EMESH, PKASP_ENOMEM, PKASP_ENOTCONV, PKASP_EBREAKDOWN, \
    PKASP_ECUDA, PKASP_ESTATE = range(8)
ERROR_NAMES = {0: "OK", 1: "EINVAL", 2: "EMESH", 3: "ENOMEM", 4: "ENOTCONV", 5: "EBREAKDOWN",
               6: "ECUDA", 7: "ESTATE"}
MODE_ADDITIVE, MODE_MULTIPLICATIVE = 0, 1
SMOOTHER_SGS, SMOOTHER_L1JACOBI = 0, 1
PREC_FP64, PREC_FP32 = 0, 1
KRYLOV_CG, KRYLOV_FGMRES = 0, 1
SOURCE_NONE, SOURCE_SINE, SOURCE_NODAL = 0, 1, 2
MAX_LEVELS, MAX_COLS = 25, 64


class pkasp_options(C.Structure):
    _fields_ = [("theta", C.c_double), ("mode", C.c_int), ("smoother", C.c_int),
                ("level_smoother", C.c_int), ("coarse_size", C.c_int), ("max_levels", C.c_int),
                ("seed", C.c_uint64), ("tol", C.c_double), ("max_iter", C.c_int),
                ("flexible", C.c_int), ("precond_precision", C.c_int), ("use_graph", C.c_int),
                ("spmv_threads", C.c_int), ("smoother_layout", C.c_int), ("krylov", C.c_int),
                ("restart", C.c_int), ("interp_pmax", C.c_int), ("interp_trunc", C.c_int),
                ("interp_cc", C.c_int), ("l2_persist", C.c_int)]


class pkasp_info(C.Structure):
    _fields_ = [("n_h", C.c_int64), ("n_H", C.c_int64), ("nnz_h", C.c_int64), ("nnz_H", C.c_int64),
                ("nnz_pi", C.c_int64), ("n_all", C.c_int64), ("n_tets", C.c_int64),
                ("n_verts", C.c_int64), ("k", C.c_int), ("levels", C.c_int),
                ("fine_colours", C.c_int), ("coarse_rows", C.c_int),
                ("level_rows", C.c_int64 * MAX_LEVELS), ("level_nnz", C.c_int64 * MAX_LEVELS),
                ("level_colours", C.c_int * MAX_LEVELS), ("op_complexity", C.c_double),
                ("setup_ms", C.c_double), ("assemble_ms", C.c_double),
                ("spmv_layout", C.c_int), ("smoother_layout", C.c_int),
                ("block_width", C.c_int), ("block_group", C.c_int), ("block_lanes", C.c_int),
                ("l2_persist_bytes", C.c_int64)]


class pkasp_stats(C.Structure):
    _fields_ = [("ncols", C.c_int), ("iters", C.c_int * MAX_COLS), ("status", C.c_int * MAX_COLS),
                ("true_rel", C.c_double * MAX_COLS), ("hist_host", C.POINTER(C.c_double)),
                ("hist_cap", C.c_int), ("hist_len", C.c_int), ("restarts", C.c_int),
                ("solve_ms", C.c_float), ("kernel_launches", C.c_int64)]


_lib = None
vp = C.c_void_p
i64 = C.c_int64
PI64 = C.POINTER(C.c_int64)
PI32 = C.POINTER(C.c_int32)
PF64 = C.POINTER(C.c_double)

# (name, restype, argtypes) for every entry point of include/pkasp.h
SIGNATURES = [
    ("pkasp_default_options", None, [C.POINTER(pkasp_options)]),
    ("pkasp_last_error", C.c_int, [C.c_char_p, C.c_size_t]),
    ("pkasp_assemble", C.c_int, [vp, i64, vp, i64, C.c_int, vp, C.c_int, vp, C.POINTER(vp)]),
    ("pkasp_problem_info", C.c_int, [vp, C.POINTER(pkasp_info)]),
    ("pkasp_get_dofmap", C.c_int, [vp, vp, vp]),
    ("pkasp_get_rhs", C.c_int, [vp, vp, vp]),
    ("pkasp_set_kappa", C.c_int, [vp, vp, vp]),
    ("pkasp_setup", C.c_int, [vp, C.POINTER(pkasp_options), vp]),
    ("pkasp_solve", C.c_int, [vp, vp, vp, C.c_int, i64, C.POINTER(pkasp_stats), vp]),
    ("pkasp_solve_from_zero", C.c_int, [vp, vp, vp, C.c_int, i64, C.POINTER(pkasp_stats), vp]),
    ("pkasp_solve_adjoint", C.c_int, [vp, vp, vp, C.c_int, i64, C.POINTER(pkasp_stats), vp]),
    ("pkasp_grad_kappa", C.c_int, [vp, vp, vp, C.c_int, i64, vp, vp]),
    ("pkasp_destroy", C.c_int, [vp]),
    ("pkasp_spmv", C.c_int, [vp, vp, vp, vp]),
    ("pkasp_apply_prec", C.c_int, [vp, vp, vp, vp]),
    ("pkasp_apply_smoother", C.c_int, [vp, vp, vp, vp]),
    ("pkasp_apply_vcycle", C.c_int, [vp, vp, vp, vp]),
    ("pkasp_get_matrix", C.c_int, [vp, C.c_int, PI64, PI64, PI64, vp, vp, vp]),
    ("pkasp_get_colours", C.c_int, [vp, C.c_int, vp, C.POINTER(C.c_int)]),
    ("pkasp_get_splitting", C.c_int, [vp, C.c_int, vp, vp]),
    ("pkasp_pmis", C.c_int, [i64, vp, vp, vp, C.c_uint64, vp, vp]),
    ("pkasp_pmis_noalloc", C.c_int, [i64, vp, vp, vp, C.c_uint64, vp, vp]),
    ("pkasp_dofmap_host", C.c_int, [vp, i64, vp, i64, C.c_int, vp, vp, vp, vp, vp, vp, vp, vp]),
    ("pkasp_nodes_host", C.c_int, [vp, i64, vp, i64, C.c_int, PI64, vp]),
    ("pkasp_reference_tensors", C.c_int, [C.c_int, vp]),
    ("pkasp_stokes_blocks_host", C.c_int, [vp, i64, vp, i64, C.c_int, vp, vp, vp, vp, vp, vp, vp]),
    ("pkasp_time_kernel", C.c_int, [vp, C.c_int, C.c_int, C.POINTER(C.c_float), vp]),
    ("pkasp_stokes_setup", C.c_int, [vp, C.c_int, vp]),
    ("pkasp_stokes_sizes", C.c_int, [vp, vp]),
    ("pkasp_stokes_apply", C.c_int, [vp, vp, vp, vp]),
    ("pkasp_stokes_apply_prec", C.c_int, [vp, vp, vp, vp]),
    ("pkasp_stokes_solve", C.c_int, [vp, vp, vp, C.POINTER(pkasp_stats), vp]),
]


class PkaspError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


def load():
    """Load libpkasp.so (built in-tree). Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run paper_1204_2586_gb300.build.build() first")
    L = C.CDLL(LIB_PATH)
    for name, res, args in SIGNATURES:
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def last_error() -> str:
    buf = C.create_string_buffer(1024)
    load().pkasp_last_error(buf, 1024)
    return buf.value.decode(errors="replace")


def check(rc: int):
    if rc != PKASP_OK:
        raise PkaspError(rc, last_error())
    return rc


def default_options(**kw) -> pkasp_options:
    o = pkasp_options()
    load().pkasp_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def __getattr__(name):
    # pkasp_* names resolve to the raw C entry points
    if name.startswith("pkasp_"):
        return getattr(load(), name)
    raise AttributeError(name)
