"""GPU parity of the multi-RHS PCG (several independent right-hand sides in one blocked
solve) against the oracle, one oracle solve per column, through the C ABI.

Each column is the iteration of Algorithm 2.1's preconditioner inside CG on its own:
per-column iteration counts within +-1 of the oracle, residual histories within 1e-10
of ||r_0||, solutions within 1e-8. Columns must not influence one another: a column's
result is bitwise the same whatever the other columns of the block hold."""
import numpy as np
import pytest

from paper_1204_2586_gb300.inputs import kappa_lognormal, kuhn_mesh, rhs_normal

pytestmark = pytest.mark.gpu

RTOL_ITER = 1e-10


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1204_2586_gb300 import build

    build.build()
    return torch


CASES = {"p2_n8": (2, 8, None), "p3_n5_lognormal": (3, 5, 1)}


@pytest.fixture(scope="module", params=list(CASES))
def pair(request, torch_cuda, oracle_mod):
    from paper_1204_2586_gb300 import Problem

    k, n, ks = CASES[request.param]
    xyz, t = kuhn_mesh(n, 0.2, 0)
    kap = np.ones(t.shape[0]) if ks is None else kappa_lognormal(t.shape[0], ks)
    G = Problem(xyz, t, k, kap)
    O = oracle_mod.Problem(xyz, t, k, kap)
    yield request.param, G, O
    G.close()


def _setup_both(G, O, **kw):
    G.setup(**kw)
    O.setup(**{k: v for k, v in kw.items() if k in ("mode", "smoother", "level_smoother", "tol", "max_iter")})


def _check_column(st, c, ref, x, hist_tol=RTOL_ITER):
    assert st["status"][c] == 0
    assert abs(st["iters"][c] - ref["iters"]) <= 1, (c, st["iters"][c], ref["iters"])
    h = st["hist"][:, c]
    m = min(st["iters"][c] + 1, len(ref["hist"]))
    dev = np.abs(h[:m] - ref["hist"][:m]) / ref["hist"][0]
    assert dev.max() <= hist_tol, (c, dev.max())
    assert st["true_rel"][c] <= 1e-8
    xo = ref["x"]
    assert np.linalg.norm(x - xo) <= 1e-8 * np.linalg.norm(xo)


@pytest.mark.parametrize("mode,graph", [(0, 1), (0, 0), (1, 1), (2, 1)])
def test_columns_match_oracle(pair, torch_cuda, mode, graph):
    torch = torch_cuda
    _, G, O = pair
    _setup_both(G, O, mode=mode, use_graph=graph)
    B = rhs_normal(G.nh, 5, 2)  # 5 columns: a block of 8 with 3 padding columns
    X0 = np.zeros_like(B)
    X0[:, 3] = rhs_normal(G.nh, 1, 7)[:, 0]  # one column starts from a nonzero guess
    x, st = G.solve(torch.tensor(B, device="cuda"), torch.tensor(X0, device="cuda"), hist_cap=600)
    x = x.cpu().numpy()
    assert st["rc"] == 0
    for c in range(5):
        ref = O.solve(B[:, c], X0[:, c])
        assert ref["status"] == 0
        _check_column(st, c, ref, x[:, c])


def test_columns_are_independent_bitwise(pair, torch_cuda):
    torch = torch_cuda
    _, G, O = pair
    G.setup(spmv_threads=4)
    B = rhs_normal(G.nh, 6, 3)
    a = torch.tensor(np.ascontiguousarray(B[:, [0, 1, 2]]), device="cuda")
    b = torch.tensor(np.ascontiguousarray(B[:, [0, 3, 4]]), device="cuda")
    c = torch.tensor(np.ascontiguousarray(B[:, [5, 0, 4]] * np.array([1.0, 1.0, 0.0])), device="cuda")  # a zero column
    xa, sa = G.solve(a, hist_cap=600)
    xb, sb = G.solve(b, hist_cap=600)
    xc, sc = G.solve(c, hist_cap=600)
    assert torch.equal(xa[:, 0], xb[:, 0]) and torch.equal(xa[:, 0], xc[:, 1])
    assert sa["iters"][0] == sb["iters"][0] == sc["iters"][1]
    assert np.array_equal(sa["hist"][:, 0], sb["hist"][:, 0])
    # the zero right-hand side: no iteration, solution stays zero, status OK
    assert sc["iters"][2] == 0 and sc["status"][2] == 0
    assert torch.count_nonzero(xc[:, 2]).item() == 0
    # and repeating a solve gives the same bits (fixed-grid reductions)
    xa2, _ = G.solve(a, hist_cap=600)
    assert torch.equal(xa, xa2)


def test_graph_equals_eager_bitwise(pair, torch_cuda):
    torch = torch_cuda
    _, G, O = pair
    B = torch.tensor(rhs_normal(G.nh, 4, 5), device="cuda")
    outs = []
    for graph in (1, 0):
        G.setup(use_graph=graph, spmv_threads=4)
        outs.append(G.solve(B, hist_cap=600))
    assert torch.equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1]["hist"], outs[1][1]["hist"])


def test_leading_dimension_and_host_buffers(pair, torch_cuda):
    """b and x as views with ld > ncols, in host memory; same bits as a dense device block
    of the same width."""
    torch = torch_cuda
    _, G, O = pair
    G.setup()
    B = rhs_normal(G.nh, 3, 11)
    xd, sd = G.solve(torch.tensor(B, device="cuda"))
    wide_b = np.zeros((G.nh, 7))
    wide_b[:, :3] = B
    wide_x = np.full((G.nh, 7), 5.0)
    wide_x[:, :3] = 0.0
    xh, sh = G.solve(wide_b[:, :3], wide_x[:, :3])
    assert sd["iters"] == sh["iters"]
    assert np.array_equal(xd.cpu().numpy(), wide_x[:, :3])
    assert np.all(wide_x[:, 3:] == 5.0)  # columns beyond ncols untouched


@pytest.mark.parametrize("ncols", [2, 9, 17, 33, 48, 64])
def test_block_widths(pair, torch_cuda, ncols):
    """Every block width (4, 16, 32, 48, 64 and the padded ones) against the oracle on two
    sampled columns."""
    torch = torch_cuda
    _, G, O = pair
    _setup_both(G, O)
    B = rhs_normal(G.nh, ncols, 13)
    x, st = G.solve(torch.tensor(B, device="cuda"), hist_cap=600)
    x = x.cpu().numpy()
    assert all(s == 0 for s in st["status"])
    for c in sorted({0, ncols - 1}):
        _check_column(st, c, O.solve(B[:, c]), x[:, c])


def test_fp32_preconditioner_columns(pair, torch_cuda):
    """FP32 preconditioner with FP64 flexible CG on a block: every column reaches 1e-8;
    the error against the FP64 oracle solution is stated by the bound."""
    torch = torch_cuda
    _, G, O = pair
    G.setup(precond_precision=1)
    O.setup()
    B = rhs_normal(G.nh, 8, 17)
    x, st = G.solve(torch.tensor(B, device="cuda"))
    x = x.cpu().numpy()
    for c in range(8):
        ref = O.solve(B[:, c])
        assert st["status"][c] == 0 and st["true_rel"][c] <= 1e-8
        assert abs(st["iters"][c] - ref["iters"]) <= 3
        err = np.linalg.norm(x[:, c] - ref["x"]) / np.linalg.norm(ref["x"])
        assert err <= 1e-4, err


def test_not_converged_columns_report(pair, torch_cuda):
    torch = torch_cuda
    _, G, O = pair
    G.setup(max_iter=3)
    from paper_1204_2586_gb300 import _lib as L

    B = torch.tensor(rhs_normal(G.nh, 4, 19), device="cuda")
    _, st = G.solve(B, raise_on_fail=False)
    assert st["rc"] == L.PKASP_ENOTCONV
    assert st["iters"] == [3] * 4 and st["status"] == [L.PKASP_ENOTCONV] * 4
    G.setup()


def test_adjoint_block_equals_forward(pair, torch_cuda):
    torch = torch_cuda
    _, G, O = pair
    G.setup()
    B = torch.tensor(rhs_normal(G.nh, 2, 23), device="cuda")
    x, _ = G.solve(B)
    lam, _ = G.solve_adjoint(B)
    assert torch.equal(x, lam)


def test_too_many_columns_rejected(pair, torch_cuda):
    torch = torch_cuda
    _, G, O = pair
    G.setup()
    from paper_1204_2586_gb300 import PkaspError
    from paper_1204_2586_gb300 import _lib as L

    with pytest.raises(PkaspError) as e:
        G.solve(torch.zeros(G.nh, 65, dtype=torch.float64, device="cuda"))
    assert e.value.code == L.PKASP_EINVAL
