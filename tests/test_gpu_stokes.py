"""GPU parity of the Taylor-Hood P_k - P_{k-1} Stokes system (Sec. 5) against the oracle:
the blocks B = -div_h, B^T, M_p (pattern bit-exact, values 1e-12), the operator F, the
block upper-triangular preconditioner Q_t, and FGMRES with Q_t (step counts +-1,
residual histories within 1e-10 ||r_0||, velocity within 1e-8, pressure within 1e-8 up
to the constant F leaves free)."""
import numpy as np
import pytest

from paper_1204_2586_gb300.inputs import kappa_lognormal, kuhn_mesh, rhs_normal

pytestmark = pytest.mark.gpu

MP_ITERS = 10


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1204_2586_gb300 import build

    build.build()
    return torch


CASES = {"p2p1_n4": (2, 4, None), "p3p2_n3_lognormal": (3, 3, 1), "p4p3_n2": (4, 2, None)}


@pytest.fixture(scope="module", params=list(CASES))
def stokes(request, torch_cuda, oracle_mod):
    from paper_1204_2586_gb300 import Problem

    k, n, ks = CASES[request.param]
    xyz, t = kuhn_mesh(n, 0.2, 0)
    kap = None if ks is None else kappa_lognormal(t.shape[0], ks)
    G = Problem(xyz, t, k, kap)
    G.setup()
    G.stokes_setup(MP_ITERS)
    Ou = oracle_mod.Problem(xyz, t, k, kap)
    Ou.setup()
    Op = oracle_mod.Problem(xyz, t, k - 1, dirichlet=False)
    OS = oracle_mod.Stokes(Ou, Op, MP_ITERS)
    yield G, OS
    G.close()


def _close(a, b, rtol):
    err = np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)
    assert err <= rtol, err


def test_stokes_blocks(stokes):
    G, OS = stokes
    assert (G.stokes_nh, G.stokes_np, G.stokes_n) == (OS.nh, OS.np, OS.n)
    for which, ow in ((-1, 0), (-2, 1), (-3, 2)):
        ptr, col, val, shape = G.matrix(which)
        o = OS.matrix(ow)
        assert shape == o.shape
        assert np.array_equal(ptr, o.ptr) and np.array_equal(col, o.col)
        _close(val, o.val, 1e-12)


def test_stokes_operator_and_preconditioner(stokes, torch_cuda):
    torch = torch_cuda
    G, OS = stokes
    rng = np.random.default_rng(4)
    x = rng.standard_normal(OS.n)
    _close(G.stokes_apply(torch.tensor(x, device="cuda")).cpu().numpy(), OS.apply(x), 1e-12)
    r = rng.standard_normal(OS.n)
    _close(G.stokes_prec(torch.tensor(r, device="cuda")).cpu().numpy(), OS.prec(r), 1e-10)


@pytest.mark.parametrize("graph", [1, 0])
def test_stokes_fgmres(stokes, torch_cuda, graph):
    torch = torch_cuda
    G, OS = stokes
    G.setup(use_graph=graph)  # a new setup discards the Stokes data
    G.stokes_setup(MP_ITERS)
    b = np.concatenate([rhs_normal(3 * OS.nh, 1, 2)[:, 0], np.zeros(OS.np)])
    ref = OS.solve(b, restart=30, tol=1e-8, max_iter=500)
    assert ref["status"] == 0
    x, st = G.stokes_solve(torch.tensor(b, device="cuda"), hist_cap=600)
    assert st["status"] == 0 and st["true_rel"] <= 1e-8
    assert abs(st["iters"] - ref["iters"]) <= 1, (st["iters"], ref["iters"])
    h = st["hist"]
    m = min(len(h), len(ref["hist"]))
    assert (np.abs(h[:m] - ref["hist"][:m]) / ref["hist"][0]).max() <= 1e-10
    xs, xo = x.cpu().numpy(), ref["x"]
    nu = 3 * OS.nh
    assert np.linalg.norm(xs[:nu] - xo[:nu]) <= 1e-8 * np.linalg.norm(xo[:nu])
    ps, po = xs[nu:] - xs[nu:].mean(), xo[nu:] - xo[nu:].mean()
    assert np.linalg.norm(ps - po) <= 1e-8 * np.linalg.norm(po)


def test_stokes_errors(torch_cuda):
    torch = torch_cuda
    from paper_1204_2586_gb300 import PkaspError, Problem
    from paper_1204_2586_gb300 import _lib as L

    xyz, t = kuhn_mesh(2, 0.2, 0)
    G = Problem(xyz, t, 2)
    with pytest.raises(PkaspError) as e:
        G.stokes_setup()  # before setup
    assert e.value.code == L.PKASP_ESTATE
    G.setup()
    with pytest.raises(PkaspError) as e:
        G.stokes_solve(torch.zeros(10, dtype=torch.float64, device="cuda"))
    assert e.value.code == L.PKASP_ESTATE
    with pytest.raises(PkaspError) as e:
        G.stokes_setup(0)
    assert e.value.code == L.PKASP_EINVAL
    G.close()
    P1 = Problem(*kuhn_mesh(3, 0.2, 0), 1)
    P1.setup()
    with pytest.raises(PkaspError) as e:
        P1.stokes_setup()
    assert e.value.code == L.PKASP_EINVAL
    P1.close()
