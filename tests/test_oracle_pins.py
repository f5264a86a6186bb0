"""Pins of the CPU oracle against facts fixed by the paper and by the mathematics:
closed forms, invariants, special cases and brute force on tiny inputs.

None of these tests re-types an oracle formula: each checks the oracle through a
different route (symbolic integration, dense linear algebra, a sequential algorithm
proven equivalent to the parallel one, convergence rates of the PDE solution).
"""
import itertools
import math

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from paper_1204_2586_gb300.inputs import kappa_lognormal, kuhn_mesh, splitmix64

pytestmark = pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")


def _mesh(n, seed=0):
    return kuhn_mesh(n, 0.2, seed)


# ---------------------------------------------------------------------------------
# Quadrature (load vector of Eq. 7): Grundmann-Moeller exactness on monomials
# ---------------------------------------------------------------------------------
@pytest.mark.parametrize("s", [0, 1, 2, 3, 4, 5])
def test_gm_rule_exact_to_degree(oracle_mod, s):
    lam, w = oracle_mod.gm_rule(s)
    assert np.isclose(w.sum(), 1.0 / 6.0, rtol=0, atol=1e-14)
    d = 2 * s + 1
    for deg in range(d + 1):
        for a in itertools.product(range(deg + 1), repeat=4):
            if sum(a) != deg:
                continue
            exact = math.prod(math.factorial(x) for x in a) / math.factorial(deg + 3)
            got = np.sum(w * np.prod(lam ** np.array(a), axis=1))
            assert abs(got - exact) <= 1e-13 * max(1.0, exact) + 1e-16, (s, a)
    # and the degree claim is sharp for s >= 1: some monomial of degree d+1 is missed
    if s >= 1:
        a = (d + 1, 0, 0, 0)
        exact = math.factorial(d + 1) / math.factorial(d + 4)
        got = np.sum(w * lam[:, 0] ** (d + 1))
        assert abs(got - exact) > 1e-12 * exact


# ---------------------------------------------------------------------------------
# P_k basis (Sec. 2): nodal (Kronecker) property and partition of unity
# ---------------------------------------------------------------------------------
@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_basis_nodal_and_partition(oracle_mod, k):
    nodes = oracle_mod.ref_nodes(k)
    assert nodes.shape[0] == (k + 1) * (k + 2) * (k + 3) // 6
    assert np.all(nodes.sum(1) == k)
    for n, m in enumerate(nodes):
        phi = oracle_mod.basis_eval(k, m / k)
        e = np.zeros(len(nodes))
        e[n] = 1
        assert np.allclose(phi, e, atol=1e-13)
    rng = np.random.default_rng(0)
    for _ in range(5):
        lam = rng.dirichlet(np.ones(4))
        assert abs(oracle_mod.basis_eval(k, lam).sum() - 1.0) < 1e-13


# ---------------------------------------------------------------------------------
# Element stiffness (Eq. 7) against an independent symbolic computation: Cartesian
# monomial basis from the Vandermonde matrix on the reference tetrahedron, exact
# integrals by sympy, affine map to a random physical tetrahedron.
# ---------------------------------------------------------------------------------
def _sympy_stiffness(k, X, nodes):
    sympy = pytest.importorskip("sympy")
    x, y, z = sympy.symbols("x y z")
    monos = [x ** a * y ** b * z ** c for a in range(k + 1) for b in range(k + 1 - a)
             for c in range(k + 1 - a - b)]
    vhat = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]
    pts = [tuple(sympy.Rational(sum(int(m[a]) * vhat[a][c] for a in range(4)), k)
                 for c in range(3)) for m in nodes]
    V = sympy.Matrix([[mo.subs({x: p[0], y: p[1], z: p[2]}) for mo in monos] for p in pts])
    Cm = V.inv()  # phi_n = sum_c Cm[c, n] mono_c
    basis = [sum(Cm[c, n] * monos[c] for c in range(len(monos))) for n in range(len(pts))]
    grads = [[sympy.diff(b, v) for v in (x, y, z)] for b in basis]
    J = np.array([X[1] - X[0], X[2] - X[0], X[3] - X[0]]).T
    Jit = np.linalg.inv(J).T
    det = np.linalg.det(J)
    cache = {}

    def integ(expr):
        expr = sympy.expand(expr)
        if expr == 0:
            return 0.0
        key = sympy.srepr(expr)
        if key not in cache:
            cache[key] = float(sympy.integrate(expr, (z, 0, 1 - x - y), (y, 0, 1 - x), (x, 0, 1)))
        return cache[key]

    n = len(basis)
    # M[p,q][m,n] = int dphi_m/dxi_p dphi_n/dxi_q over the reference tet
    M = np.zeros((3, 3, n, n))
    for p in range(3):
        for q in range(3):
            for a in range(n):
                for b in range(a, n):
                    v = integ(grads[a][p] * grads[b][q])
                    M[p, q, a, b] = v
                    M[q, p, b, a] = v
    K = np.zeros((n, n))
    G = Jit.T @ Jit  # grad_x phi = J^{-T} grad_xi phi
    for p in range(3):
        for q in range(3):
            K += G[p, q] * M[p, q]
    return K * det


@pytest.mark.parametrize("k", [1, 2, 3])
def test_element_stiffness_vs_symbolic(oracle_mod, k):
    rng = np.random.default_rng(k)
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float) + 0.2 * rng.standard_normal((4, 3))
    if np.linalg.det(np.array([X[1] - X[0], X[2] - X[0], X[3] - X[0]]).T) < 0:
        X[[2, 3]] = X[[3, 2]]
    K = oracle_mod.element_stiffness(k, X, 1.7)
    Ks = 1.7 * _sympy_stiffness(k, X, oracle_mod.ref_nodes(k))
    assert np.allclose(K, Ks, rtol=1e-12, atol=1e-12 * np.abs(Ks).max())


# ---------------------------------------------------------------------------------
# Assembled operators (Sec. 2)
# ---------------------------------------------------------------------------------
@pytest.mark.parametrize("k", [2, 3, 4])
def test_neumann_matrix_zero_row_sums_and_symmetry(oracle_mod, k):
    xyz, t = _mesh(3)
    kap = kappa_lognormal(t.shape[0], 1)
    P = oracle_mod.Problem(xyz, t, k, kap, dirichlet=False)
    A = P.matrix(0).to_scipy()
    assert P.nh == P.nall
    rs = np.abs(A @ np.ones(P.nh))
    assert rs.max() <= 1e-12 * abs(A).max()
    assert abs(A - A.T).max() <= 1e-13 * abs(A).max()
    AH = P.matrix(1).to_scipy()
    assert (np.abs(AH @ np.ones(P.nH))).max() <= 1e-12 * abs(AH).max()


@pytest.mark.parametrize("k", [2, 3, 4])
def test_dirichlet_matrix_spd(oracle_mod, k):
    xyz, t = _mesh(2)
    P = oracle_mod.Problem(xyz, t, k)
    A = P.matrix(0).to_scipy().toarray()
    assert np.allclose(A, A.T, atol=1e-14 * np.abs(A).max())
    np.linalg.cholesky(A)  # raises if not positive definite


@pytest.mark.parametrize("k", [2, 3, 4])
def test_galerkin_identity(oracle_mod, k):
    """A_H = I_R A_h I_P (Sec. 2, after Eq. 10) with element-wise kappa."""
    xyz, t = _mesh(3)
    kap = kappa_lognormal(t.shape[0], 1)
    for dirichlet in (True, False):
        P = oracle_mod.Problem(xyz, t, k, kap, dirichlet=dirichlet)
        A = P.matrix(0).to_scipy()
        AH = P.matrix(1).to_scipy()
        Pi = P.matrix(2).to_scipy()
        G = (Pi.T @ A @ Pi).toarray()
        assert np.abs(G - AH.toarray()).max() <= 1e-13 * np.abs(AH).max()


@pytest.mark.parametrize("k", [2, 3, 4])
def test_pi_reproduces_affine_functions(oracle_mod, k):
    """c_j^i = psi_j(x_i^h) (Eq. 10): I_P maps P1 nodal values of an affine function to
    its P_k nodal values, exactly, on the full space."""
    xyz, t = _mesh(3)
    P = oracle_mod.Problem(xyz, t, k, dirichlet=False)
    Pi = P.matrix(2).to_scipy()
    _, dx = P.dofs()
    assert np.allclose(Pi @ np.ones(P.nH), 1.0, atol=1e-14)
    for coef in ([1.0, -2.0, 0.5, 3.0], [0.0, 1.0, 1.0, 1.0]):
        g = lambda X: coef[0] + X @ np.array(coef[1:])  # noqa: E731
        assert np.allclose(Pi @ g(xyz), g(dx), atol=1e-13)
    vals = Pi.data
    assert np.all(np.isin(np.round(vals * k), np.arange(1, k + 1)))
    assert np.allclose(vals * k, np.round(vals * k), atol=1e-15)


def test_kuhn_sizes_match_closed_form(oracle_mod):
    """Interior DOF count of P_k on n^3 Kuhn cubes is (kn-1)^3; P1 count (n-1)^3."""
    for k, n in [(2, 4), (3, 3), (4, 2)]:
        xyz, t = _mesh(n)
        P = oracle_mod.Problem(xyz, t, k)
        assert P.nh == (k * n - 1) ** 3
        assert P.nH == (n - 1) ** 3
        assert P.nall == (k * n + 1) ** 3


def _monomial(p):
    return lambda X: X[:, 0] ** p[0] * X[:, 1] ** p[1] * X[:, 2] ** p[2]


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_nodal_load_integrates_products_exactly(oracle_mod, k):
    """Load from a caller's f given at the P_k nodes: b_i = <f_h, phi_i> with f_h the
    nodal interpolant (Sec. 2). Without Dirichlet removal every node is an unknown, and
    for polynomials f, g of degree <= k the interpolants are exact, so
    b(f) . g(nodes) = int_{[0,1]^3} f g = prod_c 1 / (a_c + d_c + 1) for monomials
    x^a, x^d (a closed form; the jittered mesh still tiles the unit cube exactly). A
    wrong quadrature weight, basis function or node index changes these integrals."""
    xyz, t = _mesh(3, seed=5)
    O = oracle_mod.Problem(xyz, t, k, source=oracle_mod.SOURCE_NONE, dirichlet=False)
    X = O.nodes()
    dof_all, dx = O.dofs()
    assert O.nh == O.nall
    assert np.array_equal(X[dof_all], dx)
    exps = [p for p in itertools.product(range(k + 1), repeat=3) if sum(p) <= k]
    rng = np.random.default_rng(k)
    picks = [exps[i] for i in rng.choice(len(exps), size=min(6, len(exps)), replace=False)]
    for a in picks:
        O.set_source_nodal(_monomial(a)(X))
        b = O.rhs()
        for d in picks:
            want = np.prod([1.0 / (a[c] + d[c] + 1) for c in range(3)])
            got = b @ _monomial(d)(X[dof_all])
            assert abs(got - want) <= 1e-13 * max(1.0, abs(want)), (a, d, got, want)


def test_nodal_load_of_the_sine_interpolant_converges(oracle_mod):
    """With Dirichlet removal, the load of the nodal interpolant of the manufactured f
    approaches the quadrature load of f itself at the interpolation order: the
    difference b_nodal - b_sine integrates (I_k f - f) phi_i, so its size relative to b
    falls by about 2^{k+1} when h halves (k = 2: ratio >= 6)."""
    errs = []
    for n in (4, 8):
        xyz, t = kuhn_mesh(n, 0.2, 0)
        O = oracle_mod.Problem(xyz, t, 2)
        b_sine = O.rhs()
        X = O.nodes()
        O.set_source_nodal(3 * np.pi ** 2 * np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1]) *
                           np.sin(np.pi * X[:, 2]))
        b_nod = O.rhs()
        errs.append(np.abs(b_nod - b_sine).max() / np.abs(b_sine).max())
    assert errs[0] / errs[1] >= 6.0, errs


@pytest.mark.slow
@pytest.mark.parametrize("k", [2, 3, 4])
def test_manufactured_solution_rate(oracle_mod, k):
    """u = sin(pi x) sin(pi y) sin(pi z): the L2 error of the P_k solution converges at
    O(h^{k+1}); measured between n = 4 and n = 8 on jittered meshes."""
    errs = []
    for n in (4, 8):
        xyz, t = _mesh(n)
        P = oracle_mod.Problem(xyz, t, k)
        A = P.matrix(0).to_scipy().tocsc()
        u = spla.spsolve(A, P.rhs())
        errs.append(P.l2_error_sine(u))
    rate = math.log2(errs[0] / errs[1])
    assert rate >= k + 0.8, (errs, rate)


# ---------------------------------------------------------------------------------
# Colouring: Jones-Plassmann with fixed priorities (degree, hash, -index) equals the
# sequential greedy colouring in decreasing priority order.
# ---------------------------------------------------------------------------------
def _greedy_colouring(A, stream):
    n = A.shape[0]
    h = splitmix64(stream, np.arange(n))
    deg = [int(np.sum(A.indices[A.indptr[i]:A.indptr[i + 1]] != i)) for i in range(n)]
    order = sorted(range(n), key=lambda i: (-deg[i], -int(h[i]), i))
    col = -np.ones(n, int)
    for i in order:
        nb = A.indices[A.indptr[i]:A.indptr[i + 1]]
        used = {col[j] for j in nb if j != i and col[j] >= 0}
        c = 0
        while c in used:
            c += 1
        col[i] = c
    return col


@pytest.mark.parametrize("k,n", [(2, 3), (3, 2), (1, 5)])
def test_colouring_equals_sequential_greedy(oracle_mod, k, n):
    xyz, t = _mesh(n)
    P = oracle_mod.Problem(xyz, t, max(k, 2))
    A = P.matrix(0 if k > 1 else 1)
    stream = oracle_mod.stream_colour(7, 0)
    c, nc = oracle_mod.colour_jp(A, stream)
    S = A.to_scipy()
    assert np.array_equal(c, _greedy_colouring(S, stream))
    assert nc == c.max() + 1
    r, cc = S.nonzero()
    off = r != cc
    assert np.all(c[r[off]] != c[cc[off]])


# ---------------------------------------------------------------------------------
# Smoothers
# ---------------------------------------------------------------------------------
def test_sgs_closed_form(oracle_mod):
    """One forward plus one backward multicolour GS sweep from zero is
    (D+U)^{-1} D (D+L)^{-1} r in the colour-sorted ordering; it is symmetric."""
    xyz, t = _mesh(2)
    P = oracle_mod.Problem(xyz, t, 3, kappa_lognormal(t.shape[0], 1))
    A = P.matrix(0)
    c, nc = oracle_mod.colour_jp(A, 123)
    perm = np.lexsort((np.arange(len(c)), c))
    Ad = A.to_scipy().toarray()[np.ix_(perm, perm)]
    D = np.diag(np.diag(Ad))
    Lo = np.tril(Ad, -1)
    Up = np.triu(Ad, 1)
    rng = np.random.default_rng(0)
    r = rng.standard_normal(P.nh)
    y = sla.solve_triangular(D + Lo, r[perm], lower=True)
    zp = sla.solve_triangular(D + Up, D @ y, lower=False)
    z = oracle_mod.sgs(A, c, nc, r)
    assert np.allclose(z[perm], zp, rtol=1e-12, atol=1e-12 * np.abs(zp).max())
    s = rng.standard_normal(P.nh)
    zs = oracle_mod.sgs(A, c, nc, s)
    assert abs(s @ z - r @ zs) <= 1e-12 * abs(s @ z)


def test_l1_jacobi_closed_form(oracle_mod):
    xyz, t = _mesh(2)
    P = oracle_mod.Problem(xyz, t, 2)
    P.setup(smoother=1)
    A = P.matrix(0).to_scipy()
    r = np.random.default_rng(1).standard_normal(P.nh)
    d = np.asarray(abs(A).sum(axis=1)).ravel()
    assert np.allclose(P.smoother(r), r / d, rtol=1e-15)


# ---------------------------------------------------------------------------------
# AMG pieces
# ---------------------------------------------------------------------------------
def _p1_matrix(oracle_mod, n=6, dirichlet=True, seed=0):
    xyz, t = kuhn_mesh(n, 0.2, seed)
    P = oracle_mod.Problem(xyz, t, 2, kappa_lognormal(t.shape[0], 1), dirichlet=dirichlet)
    return P.matrix(1)


def test_strength_definition(oracle_mod):
    """Sec. 6.2: j strong for i iff -a_ij > theta max_{k != i}(-a_ik)."""
    A = _p1_matrix(oracle_mod)
    for theta in (0.25, 0.5, 0.8):
        s = oracle_mod.strength(A, theta)
        S = A.to_scipy()
        for i in range(S.shape[0]):
            lo, hi = S.indptr[i], S.indptr[i + 1]
            cols, vals = S.indices[lo:hi], S.data[lo:hi]
            off = cols != i
            mx = (-vals[off]).max()
            want = off & (-vals > theta * mx) if mx > 0 else np.zeros_like(off)
            assert np.array_equal(s[lo:hi].astype(bool), want)


def _sequential_pmis(S, strong, stream):
    """PMIS with fixed measures equals this sequential rule: visit points in decreasing
    (|S_i^T|, hash, i); an undecided point becomes C and every undecided point that
    strongly depends on it becomes F."""
    n = S.shape[0]
    Sg = sp.csr_matrix((strong.astype(float), S.indices.copy(), S.indptr.copy()), shape=S.shape)
    Sg.eliminate_zeros()
    mu = np.asarray((Sg != 0).sum(axis=0)).ravel()
    deg = np.diff(Sg.indptr)
    h = splitmix64(stream, np.arange(n))
    cf = np.zeros(n, int)
    cf[(deg == 0) & (mu == 0)] = -1
    ST = Sg.T.tocsr()
    order = sorted(range(n), key=lambda i: (-int(mu[i]), -int(h[i]), -i))
    for i in order:
        if cf[i] != 0:
            continue
        cf[i] = 1
        for j in ST.indices[ST.indptr[i]:ST.indptr[i + 1]]:  # j depends on i
            if cf[j] == 0:
                cf[j] = -1
    return cf


@pytest.mark.parametrize("theta", [0.25, 0.6])
def test_pmis_equals_sequential_rule(oracle_mod, theta):
    A = _p1_matrix(oracle_mod, 7)
    s = oracle_mod.strength(A, theta)
    stream = oracle_mod.stream_pmis(3, 0)
    cf = oracle_mod.pmis(A, s, stream)
    assert np.array_equal(cf, _sequential_pmis(A.to_scipy(), s, stream))
    # validity: every F point with a strong dependency depends on some C point unless
    # it was isolated; no two C points depend strongly on each other
    S = A.to_scipy()
    rows = np.repeat(np.arange(S.shape[0]), np.diff(S.indptr))
    st = s.astype(bool)
    for i in np.nonzero(cf == -1)[0]:
        dep = S.indices[S.indptr[i]:S.indptr[i + 1]][st[S.indptr[i]:S.indptr[i + 1]]]
        if dep.size:
            assert np.any(cf[dep] == 1)
    pairs = set(zip(rows[st], S.indices[st]))
    for (i, j) in pairs:
        if cf[i] == 1 and cf[j] == 1:
            assert (j, i) not in pairs


def test_extpi_preserves_constants_and_pattern(oracle_mod):
    """On a zero-row-sum matrix extended+i interpolation reproduces constants exactly,
    and row i's columns are C_i^s plus the strong C points of F_i^s."""
    A = _p1_matrix(oracle_mod, 6, dirichlet=False)
    s = oracle_mod.strength(A, 0.25)
    cf = oracle_mod.pmis(A, s, 11)
    Pm = oracle_mod.extpi(A, s, cf)
    Ps = Pm.to_scipy()
    nc = int((cf == 1).sum())
    assert Ps.shape == (A.shape[0], nc)
    rs = np.asarray(Ps.sum(axis=1)).ravel()
    has = np.diff(Ps.indptr) > 0
    assert np.allclose(rs[has], 1.0, atol=1e-12)
    S = A.to_scipy()
    Sb = sp.csr_matrix((s.astype(float), S.indices.copy(), S.indptr.copy()), shape=S.shape)
    Sb.eliminate_zeros()
    Cm = sp.diags((cf == 1).astype(float))
    Fm = sp.diags((cf == -1).astype(float))
    reach = (Sb @ Cm + Sb @ Fm @ Sb @ Cm).tocsr()
    cidx = np.cumsum(cf == 1) - 1
    for i in np.nonzero(cf == -1)[0]:
        want = sorted(set(cidx[reach.indices[reach.indptr[i]:reach.indptr[i + 1]]]))
        got = list(Ps.indices[Ps.indptr[i]:Ps.indptr[i + 1]])
        assert got == want
    for i in np.nonzero(cf == 1)[0]:
        assert list(Ps.indices[Ps.indptr[i]:Ps.indptr[i + 1]]) == [cidx[i]]
        assert Ps.data[Ps.indptr[i]] == 1.0


def _entries_csr(oracle_mod, n, entries):
    """CSR matrix of n rows from {(i, j): a_ij} (only the listed entries are stored),
    with strong flags from the set of (i, j) pairs marked strong."""
    rows = [[] for _ in range(n)]
    for (i, j), v in entries.items():
        rows[i].append((j, v))
    ptr, col, val = [0], [], []
    for r in rows:
        r.sort()
        col += [j for j, _ in r]
        val += [v for _, v in r]
        ptr.append(len(col))
    return oracle_mod.CSR(np.array(ptr, np.int64), np.array(col, np.int32), np.array(val), (n, n))


def _extpi_rows(oracle_mod, n, entries, strong_pairs, cf, cc=0):
    A = _entries_csr(oracle_mod, n, entries)
    s = np.array([1 if (i, int(A.col[e])) in strong_pairs else 0
                  for i in range(n) for e in range(A.ptr[i], A.ptr[i + 1])], np.uint8)
    P = oracle_mod.extpi(A, s, np.array(cf, np.int8), cc=cc)
    return {i: dict(zip(P.col[P.ptr[i]:P.ptr[i + 1]].tolist(), P.val[P.ptr[i]:P.ptr[i + 1]].tolist()))
            for i in range(n)}


def test_extpi_hand_weights_1d_cffc(oracle_mod):
    """Extended+i weights computed by hand on the 1D Laplacian tridiag(-1, 2, -1) with the
    splitting C F F C (every off-diagonal strong). For F point 1: C_1^s = {0}, F_1^s = {2},
    C_2^s = {3}, so Chat_1 = {0, 3}; abar_2l = a_2l (all negative, a_22 > 0);
    d_2 = abar_21 + abar_23 = -2; atil_11 = 2 + (-1)(-1)/(-2) = 3/2;
    w_10 = -(-1 + 0)/(3/2) = 2/3, w_13 = -(0 + (-1)(-1)/(-2))/(3/2) = 1/3: the linear
    interpolant between the two C points, as the distance-two reach of ext+i promises.
    Point 2 mirrors it (1/3, 2/3). C points inject."""
    e = {(0, 0): 2.0, (0, 1): -1.0, (1, 0): -1.0, (1, 1): 2.0, (1, 2): -1.0,
         (2, 1): -1.0, (2, 2): 2.0, (2, 3): -1.0, (3, 2): -1.0, (3, 3): 2.0}
    strong = {p for p in e if p[0] != p[1]}
    P = _extpi_rows(oracle_mod, 4, e, strong, [1, -1, -1, 1])
    assert P[0] == {0: 1.0} and P[3] == {1: 1.0}
    assert P[1].keys() == {0, 1} and P[2].keys() == {0, 1}
    assert abs(P[1][0] - 2 / 3) <= 1e-15 and abs(P[1][1] - 1 / 3) <= 1e-15
    assert abs(P[2][0] - 1 / 3) <= 1e-15 and abs(P[2][1] - 2 / 3) <= 1e-15


def test_extpi_hand_weights_sign_filter(oracle_mod):
    """The abar filter of extended+i: a connection a_kl of an F neighbour k whose sign
    equals that of a_kk is dropped. Points: 0 F, 1 F, 2 C, 3 C; row 0: a_00 = 4,
    a_01 = -2 (strong F), a_02 = -1 (strong C); row 1: a_11 = 5, a_10 = -2 (strong),
    a_12 = +1 (positive, weak), a_13 = -2 (strong C). Chat_0 = {2} u C_1^s = {2, 3}.
    abar_10 = -2, abar_12 = 0 (filtered), abar_13 = -2, so d_1 = 0 - 2 - 2 = -4;
    atil_00 = 4 + (-2)(-2)/(-4) = 3; w_02 = -(-1 + 0)/3 = 1/3;
    w_03 = -(0 + (-2)(-2)/(-4))/3 = 1/3. Without the filter the weights would be 1/8
    and 1/2."""
    e = {(0, 0): 4.0, (0, 1): -2.0, (0, 2): -1.0,
         (1, 0): -2.0, (1, 1): 5.0, (1, 2): 1.0, (1, 3): -2.0,
         (2, 0): -1.0, (2, 1): 1.0, (2, 2): 3.0, (3, 1): -2.0, (3, 3): 3.0}
    strong = {(0, 1), (0, 2), (1, 0), (1, 3), (2, 0), (3, 1)}
    P = _extpi_rows(oracle_mod, 4, e, strong, [-1, -1, 1, 1])
    assert P[0].keys() == {0, 1}
    assert abs(P[0][0] - 1 / 3) <= 1e-15 and abs(P[0][1] - 1 / 3) <= 1e-15
    # F point 1: C_1^s = {3}, F_1^s = {0}, C_0^s = {2}: Chat_1 = {2, 3};
    # abar_0l: abar_01 = -2, abar_02 = -1, d_0 = abar_01 + abar_02 = -3;
    # atil_11 = 5 + (-2)(-2)/(-3) = 11/3; the weak a_12 = +1 is in Chat_1, so
    # w_12 = -(1 + (-2)(-1)/(-3))/(11/3) = -(1/3)/(11/3) = -1/11;
    # w_13 = -(-2 + 0)/(11/3) = 6/11
    assert P[1].keys() == {0, 1}
    assert abs(P[1][0] + 1 / 11) <= 1e-15 and abs(P[1][1] - 6 / 11) <= 1e-15


def test_extpi_hand_weights_zero_denominator_lumped(oracle_mod):
    """A strong F neighbour k whose denominator d_k = sum over Chat_i u {i} of abar_kl
    is zero is lumped into the diagonal: atil_ii += a_ik. Points: 0 F, 1 F, 2 C, 3 F;
    row 0: a_00 = 4, a_01 = -2 (strong F), a_02 = -1 (strong C); row 1: a_11 = 3,
    a_10 = +1 (filtered: same sign as a_11), a_13 = -1 (an F point outside Chat_0).
    Chat_0 = {2} (k = 1 has no strong C point), d_1 = abar_10 + abar_12 = 0 + 0 = 0,
    atil_00 = 4 + (-2) = 2, w_02 = -(-1)/2 = 1/2 (dropping k instead would give 1/4).
    Point 3 has no strong C point within distance two: an empty row."""
    e = {(0, 0): 4.0, (0, 1): -2.0, (0, 2): -1.0,
         (1, 0): 1.0, (1, 1): 3.0, (1, 3): -1.0,
         (2, 0): -1.0, (2, 2): 2.0, (3, 1): -1.0, (3, 3): 2.0}
    strong = {(0, 1), (0, 2), (1, 3), (2, 0), (3, 1)}
    P = _extpi_rows(oracle_mod, 4, e, strong, [-1, -1, 1, -1])
    assert P[0] == {0: 0.5}
    assert P[3] == {}


def test_extpi_cc_hand_weights(oracle_mod):
    """The "+cc" rule by hand: points 0 F, 1 F, 2 C, 3 C; row 0: a_00 = 4, a_01 = -1,
    a_02 = -2; row 1: a_11 = 4, a_10 = -1, a_12 = -1, a_13 = -2; all strong. F neighbour
    1 shares the strong C point 2 with 0, so under +cc it adds nothing: Chat_0 = {2},
    d_1 = abar_10 + abar_12 = -2, atil_00 = 4 + (-1)(-1)/(-2) = 7/2,
    w_02 = -(-2 + (-1)(-1)/(-2))/(7/2) = 5/7. Plain extended+i takes Chat_0 = {2, 3},
    d_1 = -4, atil_00 = 15/4, w_02 = 3/5, w_03 = 2/15."""
    e = {(0, 0): 4.0, (0, 1): -1.0, (0, 2): -2.0,
         (1, 0): -1.0, (1, 1): 4.0, (1, 2): -1.0, (1, 3): -2.0,
         (2, 0): -2.0, (2, 1): -1.0, (2, 2): 4.0, (3, 1): -2.0, (3, 3): 4.0}
    strong = {p for p in e if p[0] != p[1]}
    cf = [-1, -1, 1, 1]
    Pc = _extpi_rows(oracle_mod, 4, e, strong, cf, cc=1)
    assert Pc[0].keys() == {0} and abs(Pc[0][0] - 5 / 7) <= 1e-15
    P0 = _extpi_rows(oracle_mod, 4, e, strong, cf, cc=0)
    assert P0[0].keys() == {0, 1}
    assert abs(P0[0][0] - 3 / 5) <= 1e-15 and abs(P0[0][1] - 2 / 15) <= 1e-15


@pytest.mark.parametrize("theta", [0.25, 0.5])
def test_extpi_cc_pattern_constants_and_agreement(oracle_mod, theta):
    """Extended+i+cc (Sec. 1, Sec. 6.1): row i interpolates from C_i^s and the strong C
    points of those strong F neighbours k that share no strong C point with i (sets
    built here from the strength graph); constants are reproduced on a zero-row-sum
    matrix (every F row's weights sum to 1); rows where no F
    neighbour shares a C point equal the extended+i rows bitwise; and the rule removes
    entries on this matrix."""
    A = _p1_matrix(oracle_mod, 6, dirichlet=False)
    s = oracle_mod.strength(A, theta)
    cf = oracle_mod.pmis(A, s, 11)
    P0 = oracle_mod.extpi(A, s, cf).to_scipy()
    Pc = oracle_mod.extpi(A, s, cf, cc=1).to_scipy()
    S = A.to_scipy()
    st = s.astype(bool)
    cidx = np.cumsum(cf == 1) - 1

    def strong_nb(i):
        cols = S.indices[S.indptr[i]:S.indptr[i + 1]]
        return [int(j) for j in cols[st[S.indptr[i]:S.indptr[i + 1]]] if j != i]

    removed = 0
    for i in np.nonzero(cf == -1)[0]:
        ci = {j for j in strong_nb(i) if cf[j] == 1}
        want, shared_any = set(ci), False
        for k in strong_nb(i):
            if cf[k] != -1:
                continue
            ck = {j for j in strong_nb(k) if cf[j] == 1}
            if ck & ci:
                shared_any = True
            else:
                want |= ck
        got = Pc.indices[Pc.indptr[i]:Pc.indptr[i + 1]]
        assert sorted(got.tolist()) == sorted(cidx[j] for j in want)
        w = Pc.data[Pc.indptr[i]:Pc.indptr[i + 1]]
        if len(w):
            assert abs(w.sum() - 1.0) <= 1e-12
        r0 = slice(P0.indptr[i], P0.indptr[i + 1])
        if not shared_any:
            assert np.array_equal(P0.indices[r0], got) and np.array_equal(P0.data[r0], w)
        removed += (P0.indptr[i + 1] - P0.indptr[i]) - len(got)
    assert removed > 0
    for i in np.nonzero(cf == 1)[0]:
        assert list(Pc.indices[Pc.indptr[i]:Pc.indptr[i + 1]]) == [cidx[i]]


def test_extpi_cc_hierarchy_converges_with_lower_complexity(oracle_mod):
    """The aux-space solve with the +cc hierarchy reaches 1e-8, and the P1 hierarchy's
    operator complexity is no larger than with extended+i."""
    xyz, t = _mesh(6)
    P = oracle_mod.Problem(xyz, t, 2, kappa_lognormal(t.shape[0], 1))
    out = {}
    for cc in (0, 1):
        P.setup(coarse_size=20, interp_cc=cc)
        ref = P.solve()
        assert ref["status"] == 0
        out[cc] = sum(P.level(l)["A"].nnz for l in range(P.levels()))
    assert out[1] <= out[0]


@pytest.mark.parametrize("tf,pmax", [(0.0, 0), (0.2, 0), (0.0, 3), (0.3, 4)])
def test_interpolation_truncation_properties(oracle_mod, tf, pmax):
    """Truncation keeps what its definition fixes: no row longer than pmax; every kept
    |w| >= tf max|w| of its row; no dropped weight larger in magnitude than a kept one
    unless the factor dropped it; row sums unchanged (so constants stay reproduced on a
    zero-row-sum matrix); tf = 0, pmax = 0 is the identity."""
    A = _p1_matrix(oracle_mod, 6, dirichlet=False)
    s = oracle_mod.strength(A, 0.25)
    cf = oracle_mod.pmis(A, s, 11)
    P0 = oracle_mod.extpi(A, s, cf).to_scipy()
    Pt = oracle_mod.truncate(oracle_mod.CSR.from_scipy(P0), tf, pmax).to_scipy()
    assert Pt.shape == P0.shape
    if tf == 0.0 and pmax == 0:
        assert (abs(Pt - P0)).max() == 0.0
        return
    assert np.allclose(np.asarray(Pt.sum(axis=1)).ravel(), np.asarray(P0.sum(axis=1)).ravel(), atol=1e-12)
    has = np.diff(P0.indptr) > 0
    assert np.allclose(np.asarray(Pt.sum(axis=1)).ravel()[has], 1.0, atol=1e-12)
    for i in range(P0.shape[0]):
        c0 = P0.indices[P0.indptr[i]:P0.indptr[i + 1]]
        w0 = P0.data[P0.indptr[i]:P0.indptr[i + 1]]
        ct = set(Pt.indices[Pt.indptr[i]:Pt.indptr[i + 1]].tolist())
        if pmax:
            assert len(ct) <= pmax
        if len(w0) == 0:
            continue
        mx = np.abs(w0).max()
        kept = [abs(w) for c, w in zip(c0, w0) if c in ct]
        dropped = [abs(w) for c, w in zip(c0, w0) if c not in ct and abs(w) >= tf * mx]
        assert all(k >= tf * mx for k in kept)
        if kept and dropped:
            assert max(dropped) <= min(kept)


def test_truncation_lowers_operator_complexity_and_converges(oracle_mod):
    xyz, t = _mesh(6)
    P = oracle_mod.Problem(xyz, t, 2, kappa_lognormal(t.shape[0], 1))
    cop, its = [], []
    for pmax in (0, 4, 2):
        P.setup(coarse_size=20, interp_pmax=pmax)
        nnz = [P.level(l)["A"].nnz for l in range(P.levels())]
        cop.append(sum(nnz) / nnz[0])
        out = P.solve()
        assert out["status"] == 0
        its.append(out["iters"])
    assert cop[1] <= cop[0] + 1e-12 and cop[2] <= cop[1] + 1e-12, cop


def test_rap_matches_dense_product(oracle_mod):
    A = _p1_matrix(oracle_mod, 6)
    s = oracle_mod.strength(A, 0.25)
    cf = oracle_mod.pmis(A, s, 5)
    Pm = oracle_mod.extpi(A, s, cf)
    Ac = oracle_mod.rap(A, Pm)
    D = Pm.to_scipy().toarray()
    want = D.T @ A.to_scipy().toarray() @ D
    got = Ac.to_scipy().toarray()
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()
    # structural pattern: every product term appears
    pat = (abs(Pm.to_scipy()).T @ abs(A.to_scipy()) @ abs(Pm.to_scipy())).tocsr()
    assert np.array_equal(pat.indptr, Ac.ptr)


# ---------------------------------------------------------------------------------
# Preconditioner and solver
# ---------------------------------------------------------------------------------
def _dense_ops(P):
    A = P.matrix(0).to_scipy().toarray()
    Pi = P.matrix(2).to_scipy().toarray()
    AH = P.matrix(1).to_scipy().toarray()
    return A, Pi, AH


@pytest.mark.parametrize("mode", [0, 1])
def test_two_level_closed_form(oracle_mod, mode):
    """With the exact coarse solve (one AMG level), the additive preconditioner is
    S_sgs + I_P A_H^{-1} I_R, and the multiplicative one (Algorithm 2.1 with
    pre-smoothing) has error operator (I - S_b A)(I - I_P A_H^{-1} I_R A)(I - S_f A)."""
    xyz, t = _mesh(3)
    P = oracle_mod.Problem(xyz, t, 2, kappa_lognormal(t.shape[0], 1))
    P.setup(mode=mode, coarse_size=10 ** 6)
    assert P.levels() == 1
    A, Pi, AH = _dense_ops(P)
    c = P.fine_colour()
    perm = np.lexsort((np.arange(len(c)), c))
    inv = np.argsort(perm)
    Ap = A[np.ix_(perm, perm)]
    D = np.diag(np.diag(Ap))
    Sf = np.linalg.inv(D + np.tril(Ap, -1))[np.ix_(inv, inv)]
    Sb = np.linalg.inv(D + np.triu(Ap, 1))[np.ix_(inv, inv)]
    Cc = Pi @ np.linalg.solve(AH, Pi.T)
    n = A.shape[0]
    I = np.eye(n)
    Bm = np.column_stack([P.apply_prec(I[:, j]) for j in range(n)])
    if mode == 0:
        want = Sb @ D[np.ix_(inv, inv)] @ Sf + Cc
        assert np.abs(Bm - want).max() <= 1e-11 * np.abs(want).max()
    else:
        E = (I - Sb @ A) @ (I - Cc @ A) @ (I - Sf @ A)
        assert np.abs((I - Bm @ A) - E).max() <= 1e-11
    assert np.abs(Bm - Bm.T).max() <= 1e-11 * np.abs(Bm).max()
    assert np.linalg.eigvalsh(0.5 * (Bm + Bm.T)).min() > 0


@pytest.mark.parametrize("lsm", [0, 1])
def test_plain_amg_two_level_closed_form(oracle_mod, lsm):
    """Plain AMG on A_h (the comparison method), two levels with the exact coarse solve:
    one V(1,1)-cycle has error operator (I - S_b A)(I - P A_c^{-1} P^T A)(I - S_f A)
    with A_c = P^T A P, S_f / S_b the forward / backward multicolour GS of level 0 in its
    colour order (lsm = 0) or the l1-Jacobi step D_l1^{-1} (lsm = 1)."""
    xyz, t = _mesh(3)
    P = oracle_mod.Problem(xyz, t, 2, kappa_lognormal(t.shape[0], 1))
    P.setup(mode=2, level_smoother=lsm, max_levels=2, coarse_size=1)
    assert P.levels() == 2
    A = P.matrix(0).to_scipy().toarray()
    L0 = P.level(0)
    assert np.array_equal(L0["A"].ptr, P.matrix(0).ptr)  # level 0 is A_h itself
    Pm = L0["P"].to_scipy().toarray()
    n = A.shape[0]
    I = np.eye(n)
    if lsm == 0:
        c = L0["colour"]
        perm = np.lexsort((np.arange(n), c))
        inv = np.argsort(perm)
        Ap = A[np.ix_(perm, perm)]
        D = np.diag(np.diag(Ap))
        Sf = np.linalg.inv(D + np.tril(Ap, -1))[np.ix_(inv, inv)]
        Sb = np.linalg.inv(D + np.triu(Ap, 1))[np.ix_(inv, inv)]
    else:
        Sf = Sb = np.diag(1.0 / np.abs(A).sum(axis=1))
    Ac = Pm.T @ A @ Pm
    E = (I - Sb @ A) @ (I - Pm @ np.linalg.solve(Ac, Pm.T @ A)) @ (I - Sf @ A)
    Bm = np.column_stack([P.apply_prec(I[:, j]) for j in range(n)])
    assert np.abs((I - Bm @ A) - E).max() <= 1e-10


def test_plain_amg_pcg_reaches_dense_solution(oracle_mod):
    xyz, t = _mesh(3)
    P = oracle_mod.Problem(xyz, t, 3, kappa_lognormal(t.shape[0], 1))
    P.setup(mode=2, coarse_size=20, tol=1e-12)
    assert P.levels() >= 3
    out = P.solve()
    assert out["status"] == 0
    A = P.matrix(0).to_scipy().toarray()
    u = np.linalg.solve(A, P.rhs())
    assert np.linalg.norm(out["x"] - u) <= 1e-9 * np.linalg.norm(u)


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("lsm", [0, 1])
def test_multilevel_preconditioner_symmetric_positive(oracle_mod, mode, lsm):
    xyz, t = _mesh(5)
    P = oracle_mod.Problem(xyz, t, 2, kappa_lognormal(t.shape[0], 1))
    P.setup(mode=mode, level_smoother=lsm, coarse_size=8)
    assert P.levels() >= 2
    rng = np.random.default_rng(2)
    x, y = rng.standard_normal(P.nh), rng.standard_normal(P.nh)
    bx, by = P.apply_prec(x), P.apply_prec(y)
    assert abs(y @ bx - x @ by) <= 1e-12 * abs(y @ bx)
    assert x @ bx > 0
    # the V-cycle on its own is symmetric too (level 0: A_H, or A_h in plain AMG mode)
    n0 = P.nh if mode == 2 else P.nH
    u, v = rng.standard_normal(n0), rng.standard_normal(n0)
    assert abs(v @ P.vcycle(u) - u @ P.vcycle(v)) <= 1e-12 * abs(v @ P.vcycle(u))


@pytest.mark.parametrize("k", [2, 3, 4])
def test_pcg_reaches_dense_solution(oracle_mod, k):
    xyz, t = _mesh(2)
    P = oracle_mod.Problem(xyz, t, k, kappa_lognormal(t.shape[0], 1))
    P.setup(tol=1e-13)
    out = P.solve()
    assert out["status"] == 0
    A = P.matrix(0).to_scipy().toarray()
    u = np.linalg.solve(A, P.rhs())
    assert np.linalg.norm(out["x"] - u) <= 1e-10 * np.linalg.norm(u)
    assert out["true_rel"] <= 1e-13 * 1.01


def test_fcg_matches_pcg_with_fixed_preconditioner(oracle_mod):
    """With a fixed SPD preconditioner the flexible beta equals the standard one in exact
    arithmetic, so the two iterations coincide up to rounding."""
    xyz, t = _mesh(4)
    P = oracle_mod.Problem(xyz, t, 3)
    P.setup(flexible=0)
    a = P.solve()
    P.setup(flexible=1)
    b = P.solve()
    assert a["iters"] == b["iters"]
    assert np.allclose(a["hist"], b["hist"], rtol=1e-6)


# ---------------------------------------------------------------------------------
# FGMRES (the outer iteration of Sec. 6.2)
# ---------------------------------------------------------------------------------
@pytest.mark.parametrize("mode", [0, 1])
def test_fgmres_minimal_residual_over_explicit_krylov_space(oracle_mod, mode):
    """With a fixed preconditioner B, FGMRES is right-preconditioned GMRES: after k steps
    ||b - A x_k|| is the minimum of ||r_0 - A B K c|| over c, K = [r_0, ABr_0, ...,
    (AB)^{k-1} r_0]. The oracle's residual estimates must equal that minimum computed by
    dense least squares on the explicit Krylov matrix (B assembled column by column)."""
    xyz, t = _mesh(3)
    P = oracle_mod.Problem(xyz, t, 2, kappa_lognormal(t.shape[0], 1))
    P.setup(mode=mode, coarse_size=8, krylov=1, restart=30, tol=1e-14, max_iter=8)
    A = P.matrix(0).to_scipy().toarray()
    n = A.shape[0]
    B = np.column_stack([P.apply_prec(np.eye(n)[:, j]) for j in range(n)])
    b = P.rhs()
    out = P.solve(b)
    AB = A @ B
    K = [b / np.linalg.norm(b)]
    for _ in range(7):
        v = AB @ K[-1]
        K.append(v / np.linalg.norm(v))
    for k in range(1, 8):
        Kk = np.column_stack(K[:k])
        c, *_ = np.linalg.lstsq(AB @ Kk, b, rcond=None)
        rmin = np.linalg.norm(b - AB @ Kk @ c)
        assert abs(out["hist"][k] - rmin) <= 1e-7 * np.linalg.norm(b), (k, out["hist"][k], rmin)
    # and the history is non-increasing (minimal residual over nested spaces)
    assert np.all(np.diff(out["hist"][: out["iters"] + 1]) <= 1e-14 * np.linalg.norm(b))


@pytest.mark.parametrize("k_stop", [3, 7])
def test_fgmres_estimate_is_the_true_residual(oracle_mod, k_stop):
    """|g_{k+1}| of the Givens-rotated least-squares problem is ||b - A x_k|| for the
    x_k that the cycle's triangular solve produces: stop after k steps and compare with
    the true residual of the returned x."""
    xyz, t = _mesh(4)
    P = oracle_mod.Problem(xyz, t, 3)
    P.setup(krylov=1, restart=30, max_iter=k_stop)
    out = P.solve()
    assert out["iters"] == k_stop and out["status"] != 0
    r0 = out["hist"][0]
    assert abs(out["true_rel"] * r0 - out["hist"][k_stop]) <= 1e-9 * r0


@pytest.mark.parametrize("k", [2, 3])
def test_fgmres_reaches_dense_solution_with_restarts(oracle_mod, k):
    xyz, t = _mesh(3)
    P = oracle_mod.Problem(xyz, t, k, kappa_lognormal(t.shape[0], 1))
    A = P.matrix(0).to_scipy().toarray()
    u = np.linalg.solve(A, P.rhs())
    iters = {}
    for m in (30, 3):
        P.setup(krylov=1, restart=m, tol=1e-12, max_iter=400)
        out = P.solve()
        assert out["status"] == 0 and out["true_rel"] <= 1e-12 * 1.01
        assert np.linalg.norm(out["x"] - u) <= 1e-9 * np.linalg.norm(u)
        iters[m] = out["iters"]
    # restarting throws the Krylov space away: never fewer steps
    assert iters[3] >= iters[30]


def test_fgmres_multiplicative_mode_iterations_flat_in_h(oracle_mod):
    """The paper's setting (Sec. 6.2: FGMRES, one multilevel cycle, Algorithm 2.1 with
    pre-smoothing): iteration counts stay flat as h halves (Theorem 4.2)."""
    its = []
    for n in (4, 8):
        xyz, t = _mesh(n)
        P = oracle_mod.Problem(xyz, t, 2)
        P.setup(mode=1, krylov=1, tol=1e-6)
        out = P.solve()
        assert out["status"] == 0
        its.append(out["iters"])
    assert its[1] <= its[0] + 2, its


@pytest.mark.slow
def test_iterations_independent_of_h(oracle_mod):
    """Theorem 4.2: the two-level convergence rate is bounded independently of h."""
    its = {}
    for mode in (0, 1):
        for n in (4, 8, 16):
            xyz, t = _mesh(n)
            P = oracle_mod.Problem(xyz, t, 2)
            P.setup(mode=mode)
            out = P.solve()
            assert out["status"] == 0
            its[(mode, n)] = out["iters"]
        vals = [its[(mode, n)] for n in (4, 8, 16)]
        assert max(vals) - min(vals) <= 4, its


def test_theta_robustness(oracle_mod):
    """Tables 2-4: the auxiliary-space method is nearly insensitive to theta."""
    xyz, t = _mesh(6)
    P = oracle_mod.Problem(xyz, t, 3)
    its = []
    for theta in (0.2, 0.4, 0.6, 0.8):
        P.setup(theta=theta, mode=1)
        out = P.solve()
        assert out["status"] == 0
        its.append(out["iters"])
    assert max(its) - min(its) <= 3, its


# ---------------------------------------------------------------------------------
# Stokes, Taylor-Hood P_k - P_{k-1} (Sec. 5)
# ---------------------------------------------------------------------------------
def _stokes(oracle_mod, k, n, setup=True, **kw):
    xyz, t = _mesh(n)
    U = oracle_mod.Problem(xyz, t, k)
    if setup:
        U.setup(**kw)
    Pp = oracle_mod.Problem(xyz, t, k - 1, dirichlet=False)
    return xyz, t, U, Pp, oracle_mod.Stokes(U, Pp)


@pytest.mark.parametrize("k", [2, 3, 4])
def test_stokes_gradient_of_linear_pressure(oracle_mod, k):
    """B = -div_h: for the pressure q = x_c (exact in P_{k-1}), integration by parts with
    phi = 0 on the boundary gives (B^T q)_{(d, v)} = delta_cd int phi_v. int phi_v is
    computed here by Grundmann-Moeller quadrature of the basis on every element."""
    xyz, t, U, Pp, S = _stokes(oracle_mod, k, 2, setup=False)
    BT = S.matrix(1).to_scipy()
    _, pxyz = Pp.dofs()
    lam, w = oracle_mod.gm_rule(k)
    phi = np.array([oracle_mod.basis_eval(k, l) for l in lam])  # [q, nloc]
    ref = 6.0 * (w @ phi)  # (1/|T|) int phi_m; the rule's weights sum to the reference volume 1/6
    ed = U.elem_dofs()
    integ = np.zeros(S.nh)
    for e in range(t.shape[0]):
        X = xyz[t[e]]
        vol = abs(np.linalg.det((X[1:] - X[0]).T)) / 6.0
        for m in range(ed.shape[1]):
            if ed[e, m] >= 0:
                integ[ed[e, m]] += vol * ref[m]
    for c in range(3):
        y = BT @ pxyz[:, c]
        for d in range(3):
            want = integ if d == c else np.zeros(S.nh)
            assert np.abs(y[d * S.nh:(d + 1) * S.nh] - want).max() <= 1e-12 * np.abs(integ).max(), (c, d)


@pytest.mark.parametrize("k", [2, 3, 4])
def test_stokes_pressure_mass_matrix_integrates_exactly(oracle_mod, k):
    _, _, _, Pp, S = _stokes(oracle_mod, k, 2, setup=False)
    M = S.matrix(2).to_scipy()
    _, pxyz = Pp.dofs()
    one = np.ones(S.np)
    assert abs(one @ M @ one - 1.0) <= 1e-13            # |unit cube|
    assert abs(pxyz[:, 0] @ M @ pxyz[:, 0] - 1.0 / 3.0) <= 1e-13  # int x^2
    assert abs(pxyz[:, 0] @ M @ pxyz[:, 1] - 0.25) <= 1e-13      # int x y
    assert (abs(M - M.T)).max() <= 1e-15


@pytest.mark.parametrize("k", [2, 3])
def test_stokes_solve_matches_dense_solution(oracle_mod, k):
    """F x = b with b_p = 0 is consistent (F is singular only in the constant pressure):
    FGMRES with Q_t reaches the dense least-squares solution; velocity exactly, pressure
    up to a constant; the discrete velocity is divergence free (B u = 0)."""
    _, _, U, Pp, S = _stokes(oracle_mod, k, 2, coarse_size=5)
    rng = np.random.default_rng(3)
    b = np.concatenate([rng.standard_normal(3 * S.nh), np.zeros(S.np)])
    out = S.solve(b, tol=1e-12, max_iter=500)
    assert out["status"] == 0
    A = U.matrix(0).to_scipy().toarray()
    B = S.matrix(0).to_scipy().toarray()
    F = np.block([[sla.block_diag(A, A, A), B.T], [B, np.zeros((S.np, S.np))]])
    xd, *_ = np.linalg.lstsq(F, b, rcond=None)
    nu = 3 * S.nh
    u, p = out["x"][:nu], out["x"][nu:]
    assert np.linalg.norm(u - xd[:nu]) <= 1e-9 * np.linalg.norm(xd[:nu])
    dp = (p - p.mean()) - (xd[nu:] - xd[nu:].mean())
    assert np.linalg.norm(dp) <= 1e-8 * np.linalg.norm(xd[nu:] - xd[nu:].mean())
    assert np.linalg.norm(B @ u) <= 1e-10 * np.linalg.norm(b)


def test_stokes_iterations_flat_in_h(oracle_mod):
    """Q_t with one auxiliary-space cycle per velocity component (Sec. 6.3: the iteration
    count does not grow with the number of unknowns)."""
    its = []
    for n in (3, 6):
        _, _, U, Pp, S = _stokes(oracle_mod, 2, n, coarse_size=20)
        b = np.concatenate([np.random.default_rng(1).standard_normal(3 * S.nh), np.zeros(S.np)])
        out = S.solve(b, tol=1e-8, restart=30, max_iter=500)
        assert out["status"] == 0
        its.append(out["iters"])
    assert its[1] <= its[0] + 4, its


def test_adjoint_gradient_matches_central_differences(oracle_mod):
    """dL/dkappa_e = -lambda_e^T Khat_e u_e with A lambda = u - u_obs, against central
    differences of L = 0.5 ||u - u_obs||^2 computed with direct solves."""
    xyz, t = _mesh(2)
    kap = kappa_lognormal(t.shape[0], 1)
    kobs = kappa_lognormal(t.shape[0], 3)
    P = oracle_mod.Problem(xyz, t, 2, kap)
    Q = oracle_mod.Problem(xyz, t, 2, kobs)
    uobs = spla.spsolve(Q.matrix(0).to_scipy().tocsc(), Q.rhs())

    def loss(kv):
        P.set_kappa(kv)
        u = spla.spsolve(P.matrix(0).to_scipy().tocsc(), P.rhs())
        return 0.5 * np.sum((u - uobs) ** 2), u

    L0, u = loss(kap)
    A = P.matrix(0).to_scipy().tocsc()
    lam = spla.spsolve(A, u - uobs)
    g = P.grad_kappa(u, lam)
    eps = 1e-6
    for e in [0, 5, 17, 40]:
        kp, km = kap.copy(), kap.copy()
        kp[e] += eps
        km[e] -= eps
        fd = (loss(kp)[0] - loss(km)[0]) / (2 * eps)
        assert abs(fd - g[e]) <= 1e-6 * max(abs(g).max(), 1e-30), (e, fd, g[e])
