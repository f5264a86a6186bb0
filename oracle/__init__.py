"""Python access to the plain FP64 CPU oracle (``pk_oracle.c``).

TEST INFRASTRUCTURE ONLY. The oracle exists to check the CUDA library: only the
test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package. The solver package never imports it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pk_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
i8p = np.ctypeslib.ndpointer(np.int8, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so products round as written)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fPIC",
             "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class OOpts(C.Structure):
    _fields_ = [("theta", C.c_double), ("mode", C.c_int), ("smoother", C.c_int),
                ("level_smoother", C.c_int), ("coarse_size", C.c_int),
                ("max_levels", C.c_int), ("seed", C.c_uint64), ("tol", C.c_double),
                ("max_iter", C.c_int), ("flexible", C.c_int), ("krylov", C.c_int),
                ("restart", C.c_int), ("interp_pmax", C.c_int), ("interp_trunc", C.c_int),
                ("interp_cc", C.c_int)]


def lib():
    global _lib
    if _lib is not None:
        return _lib
    L = C.CDLL(build())
    vp = C.c_void_p
    L.orc_problem_create.restype = vp
    L.orc_problem_create.argtypes = [C.c_int64, f64p, C.c_int64, i32p, C.c_int, f64p,
                                     C.c_int, C.c_int]
    L.orc_problem_free.argtypes = [vp]
    L.orc_problem_sizes.argtypes = [vp, i64p]
    L.orc_problem_matrix.restype = vp
    L.orc_problem_matrix.argtypes = [vp, C.c_int]
    L.orc_problem_rhs.argtypes = [vp, f64p]
    L.orc_problem_dofs.argtypes = [vp, i64p, f64p]
    L.orc_problem_elem_dofs.argtypes = [vp, i32p]
    L.orc_set_kappa.argtypes = [vp, f64p]
    L.orc_set_source_nodal.restype = C.c_int
    L.orc_set_source_nodal.argtypes = [vp, f64p]
    L.orc_problem_nodes.restype = None
    L.orc_problem_nodes.argtypes = [vp, f64p]
    L.orc_csr_info.argtypes = [vp, i64p]
    L.orc_csr_copy.argtypes = [vp, i64p, i32p, f64p]
    L.orc_csr_free.argtypes = [vp]
    L.orc_csr_new.restype = vp
    L.orc_csr_new.argtypes = [C.c_int64, C.c_int64, C.c_int64, i64p, i32p, f64p]
    L.orc_nloc.restype = C.c_int
    L.orc_ref_nodes.argtypes = [C.c_int, i32p]
    L.orc_ref_tensor.argtypes = [C.c_int, f64p]
    L.orc_basis_eval.argtypes = [C.c_int, f64p, f64p]
    L.orc_gm_rule.restype = C.c_int
    L.orc_gm_rule.argtypes = [C.c_int, f64p, f64p, C.c_int]
    L.orc_element_stiffness.argtypes = [C.c_int, f64p, C.c_double, f64p]
    L.orc_colour_jp.restype = C.c_int
    L.orc_colour_jp.argtypes = [C.c_int64, i64p, i32p, C.c_uint64, i32p]
    L.orc_strength.argtypes = [vp, C.c_double, u8p]
    L.orc_pmis.argtypes = [vp, u8p, C.c_uint64, i8p]
    L.orc_extpi.restype = vp
    L.orc_extpi.argtypes = [vp, u8p, i8p, C.c_int]
    L.orc_truncate.restype = vp
    L.orc_truncate.argtypes = [vp, C.c_double, C.c_int]
    L.orc_transpose.restype = vp
    L.orc_transpose.argtypes = [vp]
    L.orc_spgemm.restype = vp
    L.orc_spgemm.argtypes = [vp, vp]
    L.orc_rap.restype = vp
    L.orc_rap.argtypes = [vp, vp]
    L.orc_spmv.argtypes = [vp, f64p, f64p]
    L.orc_sgs.argtypes = [vp, i32p, C.c_int, f64p, f64p]
    L.orc_setup.restype = C.c_int
    L.orc_setup.argtypes = [vp, C.POINTER(OOpts)]
    L.orc_set_max_iter.restype = C.c_int
    L.orc_set_max_iter.argtypes = [vp, C.c_int]
    L.orc_levels.restype = C.c_int
    L.orc_levels.argtypes = [vp]
    L.orc_level_matrix.restype = vp
    L.orc_level_matrix.argtypes = [vp, C.c_int, C.c_int]
    L.orc_level_info.argtypes = [vp, C.c_int, i64p]
    L.orc_level_cf.argtypes = [vp, C.c_int, i8p]
    L.orc_level_strong.argtypes = [vp, C.c_int, u8p]
    L.orc_level_colour.argtypes = [vp, C.c_int, i32p]
    L.orc_fine_colour.argtypes = [vp, i32p]
    L.orc_apply_prec.argtypes = [vp, f64p, f64p]
    L.orc_vcycle.argtypes = [vp, f64p, f64p]
    L.orc_smoother.argtypes = [vp, f64p, f64p]
    L.orc_solve.restype = C.c_int
    L.orc_solve.argtypes = [vp, f64p, f64p, f64p, C.c_int, C.POINTER(C.c_int),
                            C.POINTER(C.c_double)]
    L.orc_grad_kappa.argtypes = [vp, f64p, f64p, f64p]
    L.orc_stokes_create.restype = vp
    L.orc_stokes_create.argtypes = [vp, vp, C.c_int]
    L.orc_stokes_free.argtypes = [vp]
    L.orc_stokes_sizes.argtypes = [vp, i64p]
    L.orc_stokes_matrix.restype = vp
    L.orc_stokes_matrix.argtypes = [vp, C.c_int]
    L.orc_stokes_apply.argtypes = [vp, f64p, f64p]
    L.orc_stokes_prec.argtypes = [vp, f64p, f64p]
    L.orc_stokes_solve.restype = C.c_int
    L.orc_stokes_solve.argtypes = [vp, f64p, f64p, C.c_int, C.c_double, C.c_int, f64p, C.c_int,
                                   C.POINTER(C.c_int), C.POINTER(C.c_double)]
    L.orc_l2_error_sine.restype = C.c_double
    L.orc_l2_error_sine.argtypes = [vp, f64p]
    _lib = L
    return L


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


class CSR:
    """A CSR matrix copied out of (or into) the oracle."""

    def __init__(self, ptr, col, val, shape):
        self.ptr, self.col, self.val, self.shape = ptr, col, val, shape

    @classmethod
    def from_handle(cls, h):
        L = lib()
        info = np.zeros(3, np.int64)
        L.orc_csr_info(h, info)
        n, m, nnz = (int(v) for v in info)
        ptr = np.zeros(n + 1, np.int64)
        col = np.zeros(max(nnz, 1), np.int32)
        val = np.zeros(max(nnz, 1), np.float64)
        L.orc_csr_copy(h, ptr, col, val)
        return cls(ptr, col[:nnz].copy(), val[:nnz].copy(), (n, m))

    @classmethod
    def from_scipy(cls, a):
        a = a.tocsr()
        a.sort_indices()
        return cls(_i64(a.indptr), _i32(a.indices), _f64(a.data), a.shape)

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val.copy(), self.col.copy(), self.ptr.copy()),
                             shape=self.shape)

    def handle(self):
        """A new oracle-owned copy; free with :func:`free_csr`."""
        col = self.col if self.col.size else np.zeros(1, np.int32)
        val = self.val if self.val.size else np.zeros(1, np.float64)
        return lib().orc_csr_new(self.shape[0], self.shape[1], self.col.size, self.ptr,
                                 col, val)

    @property
    def nnz(self):
        return int(self.col.size)


def free_csr(h):
    lib().orc_csr_free(h)


def _take(h):
    """Copy an oracle-allocated matrix out and free it."""
    out = CSR.from_handle(h)
    free_csr(h)
    return out


# ---- stand-alone pieces on plain CSR ----------------------------------------------
def nloc(k):
    return int(lib().orc_nloc(k))


def ref_nodes(k):
    m = np.zeros((nloc(k), 4), np.int32)
    lib().orc_ref_nodes(k, m)
    return m


def ref_tensor(k):
    n = nloc(k)
    S = np.zeros((4, 4, n, n))
    lib().orc_ref_tensor(k, S)
    return S


def basis_eval(k, lam4):
    phi = np.zeros(nloc(k))
    lib().orc_basis_eval(k, _f64(lam4), phi)
    return phi


def gm_rule(s):
    cap = 4096
    lam = np.zeros((cap, 4))
    w = np.zeros(cap)
    q = lib().orc_gm_rule(s, lam, w, cap)
    return lam[:q].copy(), w[:q].copy()


def element_stiffness(k, x4x3, kappa=1.0):
    n = nloc(k)
    K = np.zeros((n, n))
    lib().orc_element_stiffness(k, _f64(x4x3).ravel(), float(kappa), K)
    return K


def colour_jp(a: CSR, stream: int):
    c = np.zeros(a.shape[0], np.int32)
    col = a.col if a.col.size else np.zeros(1, np.int32)
    nc = lib().orc_colour_jp(a.shape[0], a.ptr, col, stream, c)
    return c, int(nc)


def truncate(p: CSR, tf: float, pmax: int) -> CSR:
    """Interpolation truncation (drop small weights, keep the largest, keep row sums)."""
    h = p.handle()
    try:
        return _take(lib().orc_truncate(h, float(tf), int(pmax)))
    finally:
        free_csr(h)


def strength(a: CSR, theta: float):
    h = a.handle()
    s = np.zeros(max(a.nnz, 1), np.uint8)
    lib().orc_strength(h, theta, s)
    free_csr(h)
    return s[: a.nnz].copy()


def pmis(a: CSR, strong, stream: int):
    h = a.handle()
    cf = np.zeros(a.shape[0], np.int8)
    s = np.ascontiguousarray(strong, dtype=np.uint8)
    if s.size == 0:
        s = np.zeros(1, np.uint8)
    lib().orc_pmis(h, s, stream, cf)
    free_csr(h)
    return cf


def extpi(a: CSR, strong, cf, cc=0):
    """Extended+i interpolation; cc=1 gives the "+cc" form."""
    h = a.handle()
    s = np.ascontiguousarray(strong, dtype=np.uint8)
    if s.size == 0:
        s = np.zeros(1, np.uint8)
    out = _take(lib().orc_extpi(h, s, np.ascontiguousarray(cf, dtype=np.int8), int(cc)))
    free_csr(h)
    return out


def rap(a: CSR, p: CSR):
    ha, hp = a.handle(), p.handle()
    out = _take(lib().orc_rap(ha, hp))
    free_csr(ha)
    free_csr(hp)
    return out


def sgs(a: CSR, colour, ncolour, r):
    h = a.handle()
    z = np.zeros(a.shape[0])
    lib().orc_sgs(h, _i32(colour), int(ncolour), _f64(r), z)
    free_csr(h)
    return z


def stream_colour(seed: int, m: int) -> int:
    """Hash stream of the colouring of matrix m (0: A_h, 1+l: AMG level l)."""
    return (seed * 64 + m) & (2 ** 64 - 1)


def stream_pmis(seed: int, level: int) -> int:
    return (seed * 64 + 32 + level) & (2 ** 64 - 1)


SOURCE_NONE, SOURCE_SINE = 0, 1


def default_opts(**kw) -> OOpts:
    o = OOpts(theta=0.25, mode=0, smoother=0, level_smoother=0, coarse_size=256,
              max_levels=25, seed=0, tol=1e-8, max_iter=500, flexible=0, krylov=0, restart=30,
              interp_pmax=0, interp_trunc=0, interp_cc=0)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Problem:
    """Assembled P_k problem in the oracle: DOF map, A_h, A_H, I_P and the load."""

    def __init__(self, xyz, tets, k, kappa=None, source=SOURCE_SINE, dirichlet=True):
        L = lib()
        xyz = _f64(xyz)
        tets = _i32(tets)
        self.nt = tets.shape[0]
        kap = _f64(np.ones(self.nt) if kappa is None else kappa)
        self.k = k
        self.h = L.orc_problem_create(xyz.shape[0], xyz.ravel(), self.nt, tets.ravel(), k, kap,
                                      source, 1 if dirichlet else 0)
        if not self.h:
            raise ValueError("oracle could not build the problem")
        s = np.zeros(8, np.int64)
        L.orc_problem_sizes(self.h, s)
        self.nh, self.nH, self.nnz_h, self.nnz_H, self.nnz_pi, self.nall, self.nedge, self.nface = (
            int(v) for v in s)
        self.opts = None

    def __del__(self):
        h = getattr(self, "h", None)
        if h and _lib is not None:
            _lib.orc_problem_free(h)
            self.h = None

    def matrix(self, which):
        """0: A_h, 1: A_H, 2: I_P."""
        return CSR.from_handle(lib().orc_problem_matrix(self.h, which))

    def rhs(self):
        b = np.zeros(self.nh)
        lib().orc_problem_rhs(self.h, b)
        return b

    def dofs(self):
        a = np.zeros(self.nh, np.int64)
        x = np.zeros((self.nh, 3))
        lib().orc_problem_dofs(self.h, a, x)
        return a, x

    def elem_dofs(self):
        e = np.zeros((self.nt, nloc(self.k)), np.int32)
        lib().orc_problem_elem_dofs(self.h, e)
        return e

    def set_kappa(self, kappa):
        lib().orc_set_kappa(self.h, _f64(kappa))
        self.opts = None

    def nodes(self):
        """Coordinates [n_all, 3] of every P_k node in the all-node numbering."""
        x = np.zeros((self.nall, 3))
        lib().orc_problem_nodes(self.h, x)
        return x

    def set_source_nodal(self, f_all):
        """Load from a caller's f given at all n_all P_k nodes (its nodal interpolant)."""
        f = _f64(f_all)
        if f.shape != (self.nall,):
            raise ValueError("f_all must hold one value per P_k node (n_all)")
        lib().orc_set_source_nodal(self.h, f)

    def setup(self, **kw):
        o = default_opts(**kw)
        rc = lib().orc_setup(self.h, C.byref(o))
        if rc != 0:
            raise RuntimeError(f"oracle setup failed ({rc})")
        self.opts = o
        return self

    def set_max_iter(self, max_iter):
        """Iteration cap of later solves, keeping the preconditioner: a solve stopped
        after j iterations returns the iterate x_j."""
        if lib().orc_set_max_iter(self.h, int(max_iter)) != 0:
            raise RuntimeError("set_max_iter needs a setup and max_iter >= 1")

    def levels(self):
        return int(lib().orc_levels(self.h))

    def level(self, l):
        L = lib()
        info = np.zeros(4, np.int64)
        L.orc_level_info(self.h, l, info)
        n, nnz, ncol, nc = (int(v) for v in info)
        A = CSR.from_handle(L.orc_level_matrix(self.h, l, 0))
        out = dict(A=A, ncolour=ncol)
        c = np.zeros(n, np.int32)
        L.orc_level_colour(self.h, l, c)
        out["colour"] = c
        if nc >= 0:
            out["P"] = CSR.from_handle(L.orc_level_matrix(self.h, l, 1))
            cf = np.zeros(n, np.int8)
            L.orc_level_cf(self.h, l, cf)
            out["cf"] = cf
            st = np.zeros(max(nnz, 1), np.uint8)
            L.orc_level_strong(self.h, l, st)
            out["strong"] = st[:nnz].copy()
        return out

    def fine_colour(self):
        c = np.zeros(self.nh, np.int32)
        lib().orc_fine_colour(self.h, c)
        return c

    def apply_prec(self, r):
        z = np.zeros(self.nh)
        lib().orc_apply_prec(self.h, _f64(r), z)
        return z

    def smoother(self, r):
        z = np.zeros(self.nh)
        lib().orc_smoother(self.h, _f64(r), z)
        return z

    def vcycle(self, b):
        """One V-cycle on level 0 of the hierarchy (A_H, or A_h in plain AMG mode)."""
        info = np.zeros(4, np.int64)
        lib().orc_level_info(self.h, 0, info)
        b = _f64(b)
        if b.shape[0] != int(info[0]):
            raise ValueError("vcycle input must have the size of level 0")
        x = np.zeros(int(info[0]))
        lib().orc_vcycle(self.h, b, x)
        return x

    def solve(self, b=None, x0=None, hist_cap=1024):
        b = self.rhs() if b is None else _f64(b)
        x = np.zeros(self.nh) if x0 is None else _f64(x0).copy()
        hist = np.zeros(hist_cap)
        it = C.c_int(0)
        tr = C.c_double(0)
        st = lib().orc_solve(self.h, b, x, hist, hist_cap, C.byref(it), C.byref(tr))
        n = min(it.value + 1, hist_cap)
        return dict(x=x, status=int(st), iters=int(it.value), hist=hist[:n].copy(),
                    true_rel=float(tr.value))

    def grad_kappa(self, u, lam):
        g = np.zeros(self.nt)
        lib().orc_grad_kappa(self.h, _f64(u), _f64(lam), g)
        return g

    def l2_error_sine(self, u):
        return float(lib().orc_l2_error_sine(self.h, _f64(u)))


class Stokes:
    """Taylor-Hood P_k - P_{k-1} Stokes system (Sec. 5) over two oracle problems on one
    mesh: ``u`` of degree k with Dirichlet nodes removed (set up: its auxiliary-space
    preconditioner approximates A^{-1}) and ``p`` of degree k-1 created with
    ``dirichlet=False``. Unknowns: 3 velocity components (component-major), then p."""

    def __init__(self, u: "Problem", p: "Problem", mp_iters: int = 10):
        self.u, self.p = u, p
        h = lib().orc_stokes_create(u.h, p.h, int(mp_iters))
        if not h:
            raise ValueError("Stokes needs a degree-k Dirichlet velocity problem and a degree-(k-1) "
                             "pressure problem without Dirichlet nodes on the same mesh")
        self.h = h
        sz = np.zeros(3, np.int64)
        lib().orc_stokes_sizes(h, sz)
        self.nh, self.np, self.n = (int(v) for v in sz)

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_stokes_free(self.h)
            self.h = None

    def matrix(self, which):
        """0: B (n_p x 3 n_h), 1: B^T, 2: M_p."""
        return CSR.from_handle(lib().orc_stokes_matrix(self.h, which))

    def apply(self, x):
        y = np.zeros(self.n)
        lib().orc_stokes_apply(self.h, _f64(x), y)
        return y

    def prec(self, r):
        z = np.zeros(self.n)
        lib().orc_stokes_prec(self.h, _f64(r), z)
        return z

    def solve(self, b, x0=None, restart=30, tol=1e-8, max_iter=1000, hist_cap=2048):
        x = np.zeros(self.n) if x0 is None else _f64(x0).copy()
        hist = np.zeros(hist_cap)
        it = C.c_int(0)
        tr = C.c_double(0)
        st = lib().orc_stokes_solve(self.h, _f64(b), x, int(restart), float(tol), int(max_iter), hist,
                                    hist_cap, C.byref(it), C.byref(tr))
        n = min(it.value + 1, hist_cap)
        return dict(x=x, status=int(st), iters=int(it.value), hist=hist[:n].copy(), true_rel=float(tr.value))
