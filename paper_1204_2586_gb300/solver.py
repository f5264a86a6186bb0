"""Python-side handle over the C ABI: device buffers and streams come from PyTorch,
every computation runs in libpkasp's CUDA kernels."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L


def _ptr(t) -> int:
    return t.data_ptr()


def _row_stride(a) -> int:
    """Elements between consecutive rows of a [n] or [n, ncols] array (the ABI's ld);
    columns must be adjacent."""
    if hasattr(a, "stride") and callable(a.stride):
        st = a.stride()
    else:
        st = tuple(s // a.itemsize for s in a.strides)
    if a.ndim == 1:
        return st[0]  # one column of a wider block is a strided vector
    if a.shape[1] > 1 and st[1] != 1:
        raise ValueError("columns of a multi-RHS block must be adjacent (stride 1)")
    return st[0]


def _f64_arg(a):
    """(keep-alive object, pointer) of a float64 array for a host-or-device argument: a
    CUDA tensor is passed as its device pointer, anything else as contiguous host data."""
    import torch

    if isinstance(a, torch.Tensor):
        t = a.detach().to(torch.float64).contiguous()
        if t.is_cuda:
            return t, t.data_ptr()
        a = t.numpy()
    h = np.ascontiguousarray(a, dtype=np.float64)
    return h, h.ctypes.data


def _stream(stream=None):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Problem:
    """An assembled P_k problem (Eq. 7 of Lee, Leng & Zhang) living on the GPU."""

    def __init__(self, xyz, tets, k, kappa=None, source=L.SOURCE_SINE, f_nodal=None):
        """kappa: [nt] (host array or CUDA tensor, default 1); f_nodal: the source f at
        every P_k node ([n_all], the order of :func:`nodes_host`; host array or CUDA
        tensor), which selects PKASP_SOURCE_NODAL."""
        import torch

        lib = L.load()
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        tets = np.ascontiguousarray(tets, dtype=np.int32)
        nt = tets.shape[0]
        kap, kp = _f64_arg(np.ones(nt) if kappa is None else kappa)
        fn, fp = (None, None) if f_nodal is None else _f64_arg(f_nodal)
        if f_nodal is not None:
            source = L.SOURCE_NODAL
        torch.cuda.init()
        h = C.c_void_p()
        L.check(lib.pkasp_assemble(xyz.ctypes.data, xyz.shape[0], tets.ctypes.data, nt, k,
                                   kp, source, fp, C.byref(h)))
        self.h = h
        self.k = k
        self.nt = nt
        inf = self._info()
        self.nh = int(inf.n_h)
        self.nH = int(inf.n_H)
        self.opts = None

    @property
    def info(self):
        """pkasp_info of the problem as it is now (sizes, hierarchy, autotuned layouts)."""
        return self._info()

    def _info(self):
        inf = L.pkasp_info()
        L.check(L.load().pkasp_problem_info(self.h, C.byref(inf)))
        return inf

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            L.load().pkasp_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- data access ----------------------------------------------------------
    def rhs(self, stream=None):
        import torch

        b = torch.empty(self.nh, dtype=torch.float64, device="cuda")
        L.check(L.load().pkasp_get_rhs(self.h, _ptr(b), _stream(stream)))
        return b

    def dofmap(self):
        a = np.zeros(self.nh, np.int64)
        x = np.zeros((self.nh, 3))
        L.check(L.load().pkasp_get_dofmap(self.h, a.ctypes.data, x.ctypes.data))
        return a, x

    def matrix(self, which):
        """Host copy (ptr, col, val, shape): 0 A_h, 1 A_H, 2 I_P, 3+2l A_l, 4+2l P_l."""
        lib = L.load()
        n, m, nnz = C.c_int64(), C.c_int64(), C.c_int64()
        L.check(lib.pkasp_get_matrix(self.h, which, C.byref(n), C.byref(m), C.byref(nnz), None, None, None))
        ptr = np.zeros(n.value + 1, np.int64)
        col = np.zeros(max(nnz.value, 1), np.int32)
        val = np.zeros(max(nnz.value, 1), np.float64)
        L.check(lib.pkasp_get_matrix(self.h, which, None, None, None, ptr.ctypes.data, col.ctypes.data,
                                     val.ctypes.data))
        return ptr, col[: nnz.value], val[: nnz.value], (n.value, m.value)

    def colours(self, level=-1):
        n = self.nh if level < 0 else int(self.info.level_rows[level])
        c = np.zeros(n, np.int32)
        nc = C.c_int()
        L.check(L.load().pkasp_get_colours(self.h, level, c.ctypes.data, C.byref(nc)))
        return c, nc.value

    def splitting(self, level):
        n = int(self.info.level_rows[level])
        nnz = int(self.info.level_nnz[level])
        cf = np.zeros(n, np.int8)
        st = np.zeros(max(nnz, 1), np.uint8)
        L.check(L.load().pkasp_get_splitting(self.h, level, cf.ctypes.data, st.ctypes.data))
        return cf, st[:nnz]

    def set_kappa(self, kappa, stream=None):
        """kappa: [nt] host array or CUDA tensor (a device tensor is passed as it is)."""
        kap, kp = _f64_arg(kappa)
        L.check(L.load().pkasp_set_kappa(self.h, kp, _stream(stream)))
        self.opts = None

    # ---- setup / solve ----------------------------------------------------------
    def setup(self, stream=None, **kw):
        o = L.default_options(**kw)
        L.check(L.load().pkasp_setup(self.h, C.byref(o), _stream(stream)))
        self.opts = o
        return self

    def solve(self, b, x=None, hist_cap=0, stream=None, raise_on_fail=True, from_zero=False):
        """Solve A_h x = b; b, x are CUDA tensors [n_h] or [n_h, ncols] (or host arrays).
        from_zero: start from x0 = 0 without reading x (pkasp_solve_from_zero).
        Returns (x, stats dict)."""
        import torch

        if x is None:
            x = torch.zeros_like(b) if isinstance(b, torch.Tensor) else np.zeros_like(b)
        ncols = 1 if b.ndim == 1 else b.shape[1]
        ld = _row_stride(x)
        if _row_stride(b) != ld:
            raise ValueError("b and x must share one row stride (ld)")
        st = L.pkasp_stats()
        hist = None
        if hist_cap > 0:
            hist = np.zeros(hist_cap * ncols)
            st.hist_host = hist.ctypes.data_as(C.POINTER(C.c_double))
            st.hist_cap = hist_cap
        bp = _ptr(b) if isinstance(b, torch.Tensor) else b.ctypes.data
        xp = _ptr(x) if isinstance(x, torch.Tensor) else x.ctypes.data
        fn = L.load().pkasp_solve_from_zero if from_zero else L.load().pkasp_solve
        rc = fn(self.h, bp, xp, ncols, ld, C.byref(st), _stream(stream))
        if rc not in (L.PKASP_OK, L.PKASP_ENOTCONV, L.PKASP_EBREAKDOWN) or (rc != L.PKASP_OK and raise_on_fail):
            L.check(rc)
        out = dict(rc=rc, iters=list(st.iters[:ncols]), status=list(st.status[:ncols]),
                   true_rel=list(st.true_rel[:ncols]), restarts=st.restarts, solve_ms=st.solve_ms,
                   kernel_launches=int(st.kernel_launches))
        if hist is not None:
            out["hist"] = hist.reshape(hist_cap, ncols)[: st.hist_len].copy()
        return x, out

    def solve_adjoint(self, g, lam=None, hist_cap=0, stream=None):
        """Adjoint solve A_h^T lambda = g (A_h is symmetric: same operator and
        preconditioner, through pkasp_solve_adjoint). Returns (lambda, stats)."""
        import torch

        if lam is None:
            lam = torch.zeros_like(g)
        ncols = 1 if g.ndim == 1 else g.shape[1]
        ld = _row_stride(lam)
        if _row_stride(g) != ld:
            raise ValueError("g and lam must share one row stride (ld)")
        st = L.pkasp_stats()
        L.check(L.load().pkasp_solve_adjoint(self.h, _ptr(g), _ptr(lam), ncols, ld, C.byref(st),
                                             _stream(stream)))
        return lam, dict(iters=list(st.iters[:ncols]), status=list(st.status[:ncols]),
                         true_rel=list(st.true_rel[:ncols]), kernel_launches=int(st.kernel_launches))

    # ---- Stokes (Taylor-Hood P_k - P_{k-1}) ---------------------------------------
    def stokes_setup(self, mp_iters=10, stream=None):
        """B = -div_h, B^T, M_p and the block preconditioner; needs setup() first."""
        L.check(L.load().pkasp_stokes_setup(self.h, int(mp_iters), _stream(stream)))
        sz = np.zeros(5, np.int64)
        L.check(L.load().pkasp_stokes_sizes(self.h, sz.ctypes.data))
        self.stokes_nh, self.stokes_np, self.stokes_n = int(sz[0]), int(sz[1]), int(sz[2])
        return self

    def stokes_apply(self, x, stream=None):
        import torch

        y = torch.empty_like(x)
        L.check(L.load().pkasp_stokes_apply(self.h, _ptr(x), _ptr(y), _stream(stream)))
        return y

    def stokes_prec(self, r, stream=None):
        import torch

        z = torch.empty_like(r)
        L.check(L.load().pkasp_stokes_apply_prec(self.h, _ptr(r), _ptr(z), _stream(stream)))
        return z

    def stokes_solve(self, b, x=None, hist_cap=0, stream=None, raise_on_fail=True):
        """FGMRES with Q_t on F x = b (CUDA tensors of n = 3 n_h + n_p entries)."""
        import torch

        if x is None:
            x = torch.zeros_like(b)
        st = L.pkasp_stats()
        hist = None
        if hist_cap > 0:
            hist = np.zeros(hist_cap)
            st.hist_host = hist.ctypes.data_as(C.POINTER(C.c_double))
            st.hist_cap = hist_cap
        rc = L.load().pkasp_stokes_solve(self.h, _ptr(b), _ptr(x), C.byref(st), _stream(stream))
        if rc not in (L.PKASP_OK, L.PKASP_ENOTCONV) or (rc != L.PKASP_OK and raise_on_fail):
            L.check(rc)
        out = dict(rc=rc, iters=st.iters[0], status=st.status[0], true_rel=st.true_rel[0],
                   restarts=st.restarts, solve_ms=st.solve_ms, kernel_launches=int(st.kernel_launches))
        if hist is not None:
            out["hist"] = hist[: st.hist_len].copy()
        return x, out

    def spmv(self, x, stream=None):
        import torch

        y = torch.empty_like(x)
        L.check(L.load().pkasp_spmv(self.h, _ptr(x), _ptr(y), _stream(stream)))
        return y

    def apply_prec(self, r, stream=None):
        import torch

        z = torch.empty_like(r)
        L.check(L.load().pkasp_apply_prec(self.h, _ptr(r), _ptr(z), _stream(stream)))
        return z

    def apply_smoother(self, r, stream=None):
        import torch

        z = torch.empty_like(r)
        L.check(L.load().pkasp_apply_smoother(self.h, _ptr(r), _ptr(z), _stream(stream)))
        return z

    def apply_vcycle(self, b, stream=None):
        import torch

        x = torch.empty_like(b)
        L.check(L.load().pkasp_apply_vcycle(self.h, _ptr(b), _ptr(x), _stream(stream)))
        return x

    def grad_kappa(self, u, lam, stream=None):
        """dL/dkappa_e = -sum_c lambda_{c,e}^T Khat_e u_{c,e} for u, lam CUDA tensors [n_h]
        or [n_h, ncols] (one row stride); the column sum runs in the library."""
        import torch

        ncols = 1 if u.ndim == 1 else u.shape[1]
        ld = _row_stride(u)
        if _row_stride(lam) != ld or lam.shape != u.shape:
            raise ValueError("u and lam must have one shape and row stride")
        g = torch.empty(self.nt, dtype=torch.float64, device=u.device)
        L.check(L.load().pkasp_grad_kappa(self.h, _ptr(u), _ptr(lam), ncols, ld, _ptr(g), _stream(stream)))
        return g

    def time_kernel(self, which, reps=20, stream=None):
        ms = C.c_float()
        L.check(L.load().pkasp_time_kernel(self.h, which, reps, C.byref(ms), _stream(stream)))
        return ms.value


def pmis(ptr, col, strong, stream_id, stream=None):
    """PMIS C/F splitting on the GPU for a caller-supplied strength graph (CUDA tensors)."""
    import torch

    n = ptr.numel() - 1
    cf = torch.empty(n, dtype=torch.int8, device=ptr.device)
    L.check(L.load().pkasp_pmis(n, _ptr(ptr), _ptr(col), _ptr(strong), stream_id, _ptr(cf), _stream(stream)))
    return cf


def dofmap_host(xyz, tets, k):
    """Host-only DOF map of the library: dict with dof_all, elem_dof, A_h pattern, I_P."""
    lib = L.load()
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    nt = tets.shape[0]
    sz = np.zeros(6, np.int64)
    L.check(lib.pkasp_dofmap_host(xyz.ctypes.data, xyz.shape[0], tets.ctypes.data, nt, k, sz.ctypes.data,
                                  None, None, None, None, None, None, None))
    n_all, nh, nH, nnz_h, nnz_H, nnz_pi = (int(v) for v in sz)
    nl = (k + 1) * (k + 2) * (k + 3) // 6
    dof_all = np.zeros(nh, np.int64)
    elem = np.zeros((nt, nl), np.int32)
    ap = np.zeros(nh + 1, np.int64)
    ac = np.zeros(max(nnz_h, 1), np.int32)
    pp = np.zeros(nh + 1, np.int64)
    pc = np.zeros(max(nnz_pi, 1), np.int32)
    pv = np.zeros(max(nnz_pi, 1), np.float64)
    L.check(lib.pkasp_dofmap_host(xyz.ctypes.data, xyz.shape[0], tets.ctypes.data, nt, k, sz.ctypes.data,
                                  dof_all.ctypes.data, elem.ctypes.data, ap.ctypes.data, ac.ctypes.data,
                                  pp.ctypes.data, pc.ctypes.data, pv.ctypes.data))
    return dict(n_all=n_all, nh=nh, nH=nH, nnz_H=nnz_H, dof_all=dof_all, elem_dof=elem,
                ah_ptr=ap, ah_col=ac[:nnz_h], pi_ptr=pp, pi_col=pc[:nnz_pi], pi_val=pv[:nnz_pi])


def nodes_host(xyz, tets, k):
    """Coordinates [n_all, 3] of every P_k node of a mesh, in the node numbering of the
    library (the order of a nodal source f_nodal)."""
    lib = L.load()
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    n = C.c_int64()
    L.check(lib.pkasp_nodes_host(xyz.ctypes.data, xyz.shape[0], tets.ctypes.data, tets.shape[0], k,
                                 C.byref(n), None))
    X = np.zeros((n.value, 3))
    L.check(lib.pkasp_nodes_host(xyz.ctypes.data, xyz.shape[0], tets.ctypes.data, tets.shape[0], k,
                                 C.byref(n), X.ctypes.data))
    return X


def stokes_blocks_host(xyz, tets, k):
    """Host-only Taylor-Hood blocks of the library (B = -div_h, M_p): dict with n_h, n_p and
    CSR arrays b_ptr/b_col/b_val, m_ptr/m_col/m_val."""
    lib = L.load()
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    nt = tets.shape[0]
    sz = np.zeros(4, np.int64)
    L.check(lib.pkasp_stokes_blocks_host(xyz.ctypes.data, xyz.shape[0], tets.ctypes.data, nt, k, sz.ctypes.data,
                                         None, None, None, None, None, None))
    nh, npr, nb, nm = (int(v) for v in sz)
    out = dict(n_h=nh, n_p=npr, b_ptr=np.zeros(npr + 1, np.int64), b_col=np.zeros(max(nb, 1), np.int32),
               b_val=np.zeros(max(nb, 1)), m_ptr=np.zeros(npr + 1, np.int64), m_col=np.zeros(max(nm, 1), np.int32),
               m_val=np.zeros(max(nm, 1)))
    L.check(lib.pkasp_stokes_blocks_host(xyz.ctypes.data, xyz.shape[0], tets.ctypes.data, nt, k, sz.ctypes.data,
                                         out["b_ptr"].ctypes.data, out["b_col"].ctypes.data,
                                         out["b_val"].ctypes.data, out["m_ptr"].ctypes.data,
                                         out["m_col"].ctypes.data, out["m_val"].ctypes.data))
    for key, m in (("b_col", nb), ("b_val", nb), ("m_col", nm), ("m_val", nm)):
        out[key] = out[key][:m]
    return out


def reference_tensors(k):
    nl = (k + 1) * (k + 2) * (k + 3) // 6
    S = np.zeros((4, 4, nl, nl))
    L.check(L.load().pkasp_reference_tensors(k, S.ctypes.data))
    return S
