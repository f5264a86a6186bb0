"""CPU checks of the CUDA library's host side: it loads, exports every entry point that
include/pkasp.h declares, and its host logic (DOF numbering, sparsity patterns, I_P,
reference tensors, argument validation) agrees with the oracle. No GPU call is made."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1204_2586_gb300 import _lib as L
from paper_1204_2586_gb300 import build as B
from paper_1204_2586_gb300.inputs import kappa_lognormal, kuhn_mesh
from paper_1204_2586_gb300.solver import dofmap_host, reference_tensors

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pkasp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pkasp_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    bound = {s[0] for s in L.SIGNATURES}
    assert set(names) == bound


def test_struct_layouts_match_header(lib):
    # the defaults written by the library land in the right fields
    o = L.default_options()
    assert o.theta == 0.25 and o.coarse_size == 256 and o.max_levels == 25
    assert o.tol == 1e-8 and o.max_iter == 500 and o.use_graph == 1
    # sizes and field offsets as the C compiler lays them out from the header
    import subprocess
    import tempfile
    checks = []
    for st, fields in ((L.pkasp_options, L.pkasp_options._fields_), (L.pkasp_info, L.pkasp_info._fields_),
                       (L.pkasp_stats, L.pkasp_stats._fields_)):
        name = st.__name__
        checks.append((f"sizeof({name})", C.sizeof(st)))
        for f in fields:
            checks.append((f"offsetof({name}, {f[0]})", getattr(st, f[0]).offset))
    prog = '#include <stdio.h>\n#include <stddef.h>\n#include "pkasp.h"\nint main(void){\n'
    prog += "".join(f'printf("%zu\\n", (size_t){c});\n' for c, _ in checks) + "return 0;}\n"
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "l.c"), os.path.join(d, "l")
        open(src, "w").write(prog)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe])
        got = [int(v) for v in subprocess.check_output([exe]).split()]
    assert got == [v for _, v in checks]


@pytest.mark.parametrize("k,n", [(1, 3), (2, 3), (3, 2), (4, 2), (2, 4)])
def test_dofmap_matches_oracle(lib, oracle_mod, k, n):
    xyz, t = kuhn_mesh(n, 0.2, 0)
    D = dofmap_host(xyz, t, k)
    P = oracle_mod.Problem(xyz, t, k, source=0)
    dof_all, _ = P.dofs()
    assert D["nh"] == P.nh and D["nH"] == P.nH and D["n_all"] == P.nall
    assert np.array_equal(D["dof_all"], dof_all)
    assert np.array_equal(D["elem_dof"], P.elem_dofs())
    A = P.matrix(0)
    assert np.array_equal(D["ah_ptr"], A.ptr) and np.array_equal(D["ah_col"], A.col)
    assert D["nnz_H"] == P.nnz_H
    Pi = P.matrix(2)
    assert np.array_equal(D["pi_ptr"], Pi.ptr) and np.array_equal(D["pi_col"], Pi.col)
    assert np.array_equal(D["pi_val"], Pi.val)


@pytest.mark.parametrize("k,n", [(1, 3), (2, 3), (3, 2), (4, 2)])
def test_nodes_match_oracle(lib, oracle_mod, k, n):
    """Coordinates of every P_k node in the library's node numbering (the order of a
    nodal source) against the oracle's, bit-exact (both form sum_a m_a v_a / k in the
    same order), and against the unknowns' coordinates of the DOF map."""
    from paper_1204_2586_gb300.solver import nodes_host

    xyz, t = kuhn_mesh(n, 0.2, 0)
    X = nodes_host(xyz, t, k)
    P = oracle_mod.Problem(xyz, t, k, source=0)
    assert X.shape == (P.nall, 3)
    assert np.array_equal(X, P.nodes())
    dof_all, dx = P.dofs()
    assert np.array_equal(X[dof_all], dx)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_reference_tensors_match_oracle(lib, oracle_mod, k):
    """The library integrates by Grundmann-Moeller quadrature, the oracle by exact
    monomial integrals: two routes to the same tensors."""
    S = reference_tensors(k)
    So = oracle_mod.ref_tensor(k)
    assert np.allclose(S, So, rtol=0, atol=1e-12 * np.abs(So).max())


@pytest.mark.parametrize("k,n,ks", [(2, 3, None), (3, 2, 1), (4, 2, None)])
def test_stokes_blocks_match_oracle(lib, oracle_mod, k, n, ks):
    """The Taylor-Hood blocks the library assembles on the host (B = -div_h, M_p; Sec. 5)
    against the oracle's: patterns bit-exact, values within 1e-12 of the largest entry.
    (Independent routes: quadrature reference tensors and a pressure-node incidence in
    the library; the oracle's own element integrals and assembly.)"""
    from paper_1204_2586_gb300.solver import stokes_blocks_host

    xyz, t = kuhn_mesh(n, 0.2, 0)
    kap = None if ks is None else kappa_lognormal(t.shape[0], ks)
    S = stokes_blocks_host(xyz, t, k)
    Ou = oracle_mod.Problem(xyz, t, k, kap)
    Ou.setup()
    Op = oracle_mod.Problem(xyz, t, k - 1, dirichlet=False)
    OS = oracle_mod.Stokes(Ou, Op, 10)
    assert (S["n_h"], S["n_p"]) == (OS.nh, OS.np)
    for pre, which in (("b", 0), ("m", 2)):
        o = OS.matrix(which)
        assert np.array_equal(S[pre + "_ptr"], o.ptr) and np.array_equal(S[pre + "_col"], o.col)
        assert np.abs(S[pre + "_val"] - o.val).max() <= 1e-12 * np.abs(o.val).max()


def test_host_argument_errors(lib):
    xyz, t = kuhn_mesh(2, 0.2, 0)
    sz = np.zeros(6, np.int64)
    rc = lib.pkasp_dofmap_host(xyz.ctypes.data, xyz.shape[0], t.ctypes.data, t.shape[0], 7, sz.ctypes.data,
                               None, None, None, None, None, None, None)
    assert rc == L.PKASP_EINVAL
    bad = t.copy()
    bad[3, 2] = xyz.shape[0] + 5
    rc = lib.pkasp_dofmap_host(xyz.ctypes.data, xyz.shape[0], bad.ctypes.data, t.shape[0], 2, sz.ctypes.data,
                               None, None, None, None, None, None, None)
    assert rc == L.PKASP_EMESH
    assert "out of range" in L.last_error()
    h = C.c_void_p()
    kap = np.ones(t.shape[0])
    rc = lib.pkasp_assemble(xyz.ctypes.data, xyz.shape[0], bad.ctypes.data, t.shape[0], 2, kap.ctypes.data, 1,
                            None, C.byref(h))
    assert rc == L.PKASP_EMESH and not h.value
    rc = lib.pkasp_assemble(xyz.ctypes.data, xyz.shape[0], t.ctypes.data, t.shape[0], 0, kap.ctypes.data, 1,
                            None, C.byref(h))
    assert rc == L.PKASP_EINVAL
    # a nodal source needs its values, and values need the nodal source
    f = np.ones(1000)
    rc = lib.pkasp_assemble(xyz.ctypes.data, xyz.shape[0], t.ctypes.data, t.shape[0], 2, kap.ctypes.data,
                            L.SOURCE_NODAL, None, C.byref(h))
    assert rc == L.PKASP_EINVAL and "f_nodal" in L.last_error()
    rc = lib.pkasp_assemble(xyz.ctypes.data, xyz.shape[0], t.ctypes.data, t.shape[0], 2, kap.ctypes.data,
                            L.SOURCE_SINE, f.ctypes.data, C.byref(h))
    assert rc == L.PKASP_EINVAL and not h.value
    rc = lib.pkasp_grad_kappa(None, None, None, 1, 1, None, None)
    assert rc == L.PKASP_EINVAL
    n = C.c_int64()
    rc = lib.pkasp_nodes_host(xyz.ctypes.data, xyz.shape[0], bad.ctypes.data, t.shape[0], 2, C.byref(n), None)
    assert rc == L.PKASP_EMESH
    rc = lib.pkasp_solve(None, None, None, 1, 1, None, None)
    assert rc == L.PKASP_EINVAL
    rc = lib.pkasp_solve_from_zero(None, None, None, 1, 1, None, None)
    assert rc == L.PKASP_EINVAL
    s4 = np.zeros(4, np.int64)
    rc = lib.pkasp_stokes_blocks_host(xyz.ctypes.data, xyz.shape[0], t.ctypes.data, t.shape[0], 1, s4.ctypes.data,
                                      None, None, None, None, None, None)
    assert rc == L.PKASP_EINVAL  # Taylor-Hood needs k >= 2
    rc = lib.pkasp_stokes_blocks_host(xyz.ctypes.data, xyz.shape[0], bad.ctypes.data, t.shape[0], 2,
                                      s4.ctypes.data, None, None, None, None, None, None)
    assert rc == L.PKASP_EMESH


def test_no_cpu_fallback_in_package():
    """The solver package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_1204_2586_gb300")
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            src = open(os.path.join(pkg, f)).read()
            assert "import oracle" not in src and "from oracle" not in src, f
