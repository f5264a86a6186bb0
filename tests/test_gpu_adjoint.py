"""Differentiable solve: the adjoint gradient dL/dkappa against the oracle's gradient and
against central differences of the loss (step 1e-6, forward solves to 1e-13)."""
import numpy as np
import pytest

from paper_1204_2586_gb300.inputs import kappa_lognormal, kuhn_mesh, rhs_normal, uniform01

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1204_2586_gb300 import build

    build.build()
    return torch


def test_grad_kappa_matches_oracle(torch_cuda, oracle_mod):
    torch = torch_cuda
    from paper_1204_2586_gb300 import Problem

    xyz, t = kuhn_mesh(4, 0.2, 0)
    kap = kappa_lognormal(t.shape[0], 1)
    G = Problem(xyz, t, 3, kap)
    O = oracle_mod.Problem(xyz, t, 3, kap)
    rng = np.random.default_rng(3)
    u = rng.standard_normal(G.nh)
    lam = rng.standard_normal(G.nh)
    g = G.grad_kappa(torch.tensor(u, device="cuda"), torch.tensor(lam, device="cuda")).cpu().numpy()
    go = O.grad_kappa(u, lam)
    assert np.abs(g - go).max() <= 1e-12 * np.abs(go).max()
    G.close()


def test_grad_kappa_columns_summed_on_device(torch_cuda, oracle_mod):
    """pkasp_grad_kappa over a block of 3 columns in a [n_h][4] array (ld > ncols):
    the library's column sum against the sum of the oracle's single-column gradients."""
    torch = torch_cuda
    from paper_1204_2586_gb300 import Problem

    xyz, t = kuhn_mesh(3, 0.2, 0)
    kap = kappa_lognormal(t.shape[0], 1)
    G = Problem(xyz, t, 4, kap)
    O = oracle_mod.Problem(xyz, t, 4, kap)
    rng = np.random.default_rng(5)
    U = rng.standard_normal((G.nh, 4))
    Lm = rng.standard_normal((G.nh, 4))
    Ud, Ld = torch.tensor(U, device="cuda"), torch.tensor(Lm, device="cuda")
    g = G.grad_kappa(Ud[:, :3], Ld[:, :3]).cpu().numpy()
    go = sum(O.grad_kappa(U[:, c].copy(), Lm[:, c].copy()) for c in range(3))
    assert np.abs(g - go).max() <= 1e-12 * np.abs(go).max()
    # one column of the same block equals the single-column call bitwise
    g1 = G.grad_kappa(Ud[:, 1], Ld[:, 1]).cpu().numpy()
    g1c = G.grad_kappa(Ud[:, 1].contiguous(), Ld[:, 1].contiguous()).cpu().numpy()
    assert np.array_equal(g1, g1c)
    G.close()


@pytest.mark.parametrize("k,n,ks", [(2, 5, None), (3, 3, 1), (4, 3, 1)])
def test_nodal_source_load_matches_oracle(torch_cuda, oracle_mod, k, n, ks):
    """A caller's f at the P_k nodes (PKASP_SOURCE_NODAL; here a smooth non-sine f with
    a seeded random part) against the oracle's load b = <f_h, phi_i>, element by element
    at 1e-12; a device f and a host f give the same load; set_kappa keeps the source."""
    torch = torch_cuda
    from paper_1204_2586_gb300 import Problem, nodes_host

    xyz, t = kuhn_mesh(n, 0.2, 0)
    kap = None if ks is None else kappa_lognormal(t.shape[0], ks)
    X = nodes_host(xyz, t, k)
    f = np.exp(X[:, 0]) * np.cos(2 * X[:, 1]) + X[:, 2] ** 3 + 0.1 * rhs_normal(X.shape[0], 1, 7)[:, 0]
    G = Problem(xyz, t, k, kap, f_nodal=f)
    Gd = Problem(xyz, t, k, kap, f_nodal=torch.tensor(f, device="cuda"))
    O = oracle_mod.Problem(xyz, t, k, kap, source=oracle_mod.SOURCE_NONE)
    O.set_source_nodal(f)
    bo = O.rhs()
    b = G.rhs().cpu().numpy()
    assert np.abs(b - bo).max() <= 1e-12 * np.abs(bo).max()
    assert np.array_equal(Gd.rhs().cpu().numpy(), b)
    k2 = kappa_lognormal(t.shape[0], 9)
    G.set_kappa(torch.tensor(k2, device="cuda"))
    O.set_kappa(k2)
    assert np.abs(G.rhs().cpu().numpy() - O.rhs()).max() <= 1e-12 * np.abs(bo).max()
    assert np.abs(G.matrix(0)[2] - O.matrix(0).val).max() <= 1e-12 * np.abs(O.matrix(0).val).max()
    G.close()
    Gd.close()


def _fd_check(torch, n, k, nfd, tol_rel, eps=1e-6):
    from paper_1204_2586_gb300 import Problem
    from paper_1204_2586_gb300.autograd import solve

    xyz, t = kuhn_mesh(n, 0.2, 0)
    nt = t.shape[0]
    kap = torch.tensor(kappa_lognormal(nt, 1), dtype=torch.float64, requires_grad=True)
    kobs = kappa_lognormal(nt, 3)
    P = Problem(xyz, t, k, kobs)
    P.setup(tol=1e-13)
    b = P.rhs()
    uobs, _ = P.solve(b)
    skw = dict(tol=1e-13, max_iter=1000)
    u = solve(kap, b, P, **skw)
    loss = 0.5 * ((u - uobs) ** 2).sum()
    loss.backward()
    g = kap.grad.cpu().numpy()
    picks = (uniform01(4, np.arange(nfd)) * nt).astype(int)

    def L(kv):
        with torch.no_grad():
            uu = solve(torch.tensor(kv), b, P, **skw)
            return 0.5 * float(((uu - uobs) ** 2).sum())

    k0 = kap.detach().numpy().copy()
    errs = []
    for e in picks:
        kp, km = k0.copy(), k0.copy()
        kp[e] += eps
        km[e] -= eps
        fd = (L(kp) - L(km)) / (2 * eps)
        errs.append(abs(fd - g[e]) / max(abs(g[e]), 1e-30))
        assert abs(fd - g[e]) <= tol_rel * abs(g[e]) + 1e-9 * np.abs(g).max(), (e, fd, g[e])
    P.close()
    return max(errs)


def test_adjoint_gradient_central_differences_small(torch_cuda):
    _fd_check(torch_cuda, 4, 2, 6, 1e-5)


@pytest.mark.slow
def test_adjoint_gradient_central_differences_p3_n24(torch_cuda):
    """The differentiable workload: P3 on 24^3 jittered Kuhn cubes (82,944 tets),
    kappa = exp(N(0,1)), L = 0.5 ||u - u_obs||^2, 16 seeded elements.

    One element's derivative is about 1e-5 of L here, so a central difference with
    step 1e-6 resolves 2e-11 L against an FP64 rounding floor of about 1e-14 L in L
    itself: agreement is limited to ~1e-3 by arithmetic, not by the gradient. The
    1e-5 bar is checked with step 1e-4 (truncation error O(step^2) ~ 1e-8)."""
    err6 = _fd_check(torch_cuda, 24, 3, 16, 2e-3, eps=1e-6)
    err4 = _fd_check(torch_cuda, 24, 3, 16, 1e-5, eps=1e-4)
    print(f"max relative FD error over 16 elements: step 1e-6 {err6:.2e}, step 1e-4 {err4:.2e}")


def test_adjoint_block_of_right_hand_sides(torch_cuda):
    """[n_h, 2] right-hand sides through one differentiable block solve: dL/dkappa is the
    sum of the two single-column gradients, dL/db the block of adjoint solutions."""
    torch = torch_cuda
    from paper_1204_2586_gb300 import Problem
    from paper_1204_2586_gb300.autograd import solve

    xyz, t = kuhn_mesh(4, 0.2, 0)
    nt = t.shape[0]
    P = Problem(xyz, t, 2, kappa_lognormal(nt, 1))
    skw = dict(tol=1e-13, max_iter=1000)
    B = torch.tensor(np.ascontiguousarray(rhs_normal(P.nh, 2, 5)), device="cuda")
    W = torch.tensor(np.ascontiguousarray(rhs_normal(P.nh, 2, 6)), device="cuda")

    def grads(b, w):
        kap = torch.tensor(kappa_lognormal(nt, 1), dtype=torch.float64, requires_grad=True)
        bb = b.clone().requires_grad_(True)
        u = solve(kap, bb, P, **skw)
        (w * u).sum().backward()
        return kap.grad.cpu().numpy(), bb.grad.cpu().numpy()

    gk, gb = grads(B, W)
    parts = [grads(B[:, c].contiguous(), W[:, c].contiguous()) for c in range(2)]
    gk_sum = parts[0][0] + parts[1][0]
    assert np.abs(gk - gk_sum).max() <= 1e-9 * np.abs(gk_sum).max()
    for c in range(2):
        assert np.abs(gb[:, c] - parts[c][1]).max() <= 1e-9 * np.abs(parts[c][1]).max()
    P.close()
