"""Pins of the FP64 CPU oracle against facts fixed outside the oracle itself.

Each test checks one oracle function against a closed form, a textbook/library
routine, an invariant of the mathematics, a brute-force evaluation or a number the
paper prints, chosen so that a plausible slip (dropped term, wrong sign, transposed
operand, wrong index) fails at least one of them.
"""
from fractions import Fraction
from math import factorial

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
import workloads as wl

GOLDEN = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden")


def _ref_integrals():
    out = {}
    for line in open(f"{GOLDEN}/reference_integrals.txt"):
        if line.startswith("#") or not line.strip():
            continue
        d, p, kind, val = line.split()
        out[(int(d), int(p), kind)] = float(Fraction(val))
    return out


def _node_kind(alpha):
    nz = int(np.count_nonzero(alpha))
    return {1: "vertex", 2: "edge", 3: "face", 4: "cell"}[nz]


# ---------------------------------------------------------------------------
# Reference element: Lagrange basis and quadrature
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (2, 3), (3, 1), (3, 2), (3, 3)])
def test_basis_is_nodal_and_partition_of_unity(dim, p):
    """phi_i(x_j) = delta_ij at the lattice nodes (definition of the nodal basis,
    Sec. 2.2/3.1), sum_i phi_i = 1 and sum_i grad phi_i = 0 anywhere."""
    alpha = oracle.ref_nodes(dim, p)
    xi = alpha[:, 1:] / p
    val, _ = oracle.ref_basis(dim, p, xi)
    np.testing.assert_allclose(val, np.eye(len(alpha)), atol=1e-12)
    rng = np.random.default_rng(1)
    pts = rng.dirichlet(np.ones(dim + 1), size=7)[:, 1:]
    v, g = oracle.ref_basis(dim, p, pts)
    np.testing.assert_allclose(v.sum(axis=1), 1.0, atol=1e-12)
    np.testing.assert_allclose(g.sum(axis=1), 0.0, atol=1e-10)


@pytest.mark.parametrize("dim,p", [(2, 2), (2, 3), (3, 2)])
def test_basis_gradient_matches_finite_differences(dim, p):
    rng = np.random.default_rng(2)
    pts = rng.dirichlet(np.ones(dim + 1), size=3)[:, 1:] * 0.8 + 0.05
    _, g = oracle.ref_basis(dim, p, pts)
    h = 1e-6
    for d in range(dim):
        e = np.zeros(dim)
        e[d] = h
        vp, _ = oracle.ref_basis(dim, p, pts + e)
        vm, _ = oracle.ref_basis(dim, p, pts - e)
        np.testing.assert_allclose(g[:, :, d], (vp - vm) / (2 * h), atol=1e-8)


@pytest.mark.parametrize("dim,q", [(2, 3), (2, 4), (3, 3), (3, 4)])
def test_quadrature_exact_on_monomials(dim, q):
    """int_ref xi^a = a1! ... ad! / (|a| + d)! (textbook Dirichlet integral) for every
    monomial up to the rule's degree (2q-2 in 2D, 2q-3 in 3D for the collapsed rule)."""
    pts, wts = oracle.simplex_rule(dim, q)
    np.testing.assert_allclose(wts.sum(), 1.0 / factorial(dim), rtol=1e-14)
    deg = 2 * q - 2 if dim == 2 else 2 * q - 3
    import itertools
    for a in itertools.product(range(deg + 1), repeat=dim):
        if sum(a) > deg:
            continue
        exact = np.prod([factorial(x) for x in a]) / factorial(sum(a) + dim)
        approx = np.sum(wts * np.prod(pts ** np.array(a), axis=1))
        assert abs(approx - exact) <= 1e-14, (a, approx, exact)


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (2, 3), (3, 1), (3, 2)])
def test_basis_integrals_match_closed_form(dim, p):
    """int_K eta_m / |K| equals the closed forms of tests/golden/reference_integrals.txt."""
    table = _ref_integrals()
    alpha = oracle.ref_nodes(dim, p)
    pts, wts = oracle.simplex_rule(dim, 5)
    v, _ = oracle.ref_basis(dim, p, pts)
    ints = (wts[:, None] * v).sum(axis=0) * factorial(dim)   # divide by |ref| = 1/d!
    for m, a in enumerate(alpha):
        assert abs(ints[m] - table[(dim, p, _node_kind(a))]) < 1e-14


# ---------------------------------------------------------------------------
# Trilinear form T, stiffness, mass, interpolation
# ---------------------------------------------------------------------------

def _two_triangle_mesh():
    coords = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    cells = np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int32)
    return wl.Mesh(2, coords, cells, np.zeros(4, dtype=np.uint8))


def _closed_form_T(mesh, P, deg):
    """T_imk = sum_K iota^K_m grad lambda_i . grad lambda_k |K| with iota from the table
    and gradients from the 2x2 (3x3) geometry solve -- no quadrature involved."""
    table = _ref_integrals()
    alpha = oracle.ref_nodes(mesh.dim, deg)
    c2d = P.cell2dof(0)
    T = {}
    for c, cell in enumerate(mesh.cells):
        X = mesh.coords[cell]
        B = (X[1:] - X[0]).T
        vol = abs(np.linalg.det(B)) / factorial(mesh.dim)
        G = np.vstack([-np.ones(mesh.dim), np.eye(mesh.dim)]) @ np.linalg.inv(B)  # rows: grad lambda_a
        for a in range(mesh.dim + 1):
            for b in range(mesh.dim + 1):
                for m in range(len(alpha)):
                    key = (cell[a], c2d[c, m], cell[b])
                    T[key] = T.get(key, 0.0) + table[(mesh.dim, deg, _node_kind(alpha[m]))] * vol * G[a] @ G[b]
    return T


@pytest.mark.parametrize("deg", [1, 2, 3])
def test_T_two_triangles_brute_force_vs_closed_form(deg):
    """All entries of T on the 2-element mesh (P1/P2 gives 4 x 9 x 4) by the oracle's
    quadrature equal the closed form, for two different rule sizes."""
    mesh = _two_triangle_mesh()
    for q in (4, 7):
        P = oracle.Problem(mesh, a=("pow", 2.0), a_deg=deg, qpts=q)
        I, M, K, V = P.T_coo()
        ref = _closed_form_T(mesh, P, deg)
        got = {(i, m, k): v for i, m, k, v in zip(I, M, K, V)}
        assert set(got) == set(ref)
        for key in ref:
            assert abs(got[key] - ref[key]) < 1e-14, (key, got[key], ref[key])
    if deg == 2:
        # 2 cells x (3 x 6 x 3) local entries, minus the 2 x 3 x 2 keys on the shared edge
        assert P.nw == 9 and len(V) == 2 * 54 - 12


@pytest.mark.parametrize("deg", [1, 2, 3])
def test_T_invariants(deg):
    """sum_m T_imk = A_ik (partition of unity of W); sum_i T = sum_k T = 0 (sum of P1
    gradients vanishes); T_imk = T_kmi (symmetric bilinear gradient form)."""
    mesh = wl.unit_square_mesh(6)
    P = oracle.Problem(mesh, a=("pow", 2.0), a_deg=deg)
    I, M, K, V = P.T_coo()
    n, nw = P.n, P.nw
    A = sp.coo_matrix((V, (I, K)), shape=(n, n)).tocsr()
    # textbook: P1 stiffness on the SW-NE triangulated square grid is the 5-point stencil
    A5 = sp.lil_matrix((n, n))
    m1 = 7
    for j in range(m1):
        for i in range(m1):
            v = i + m1 * j
            A5[v, v] = 0.0
            for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                ii, jj = i + di, j + dj
                if 0 <= ii < m1 and 0 <= jj < m1:
                    A5[v, ii + m1 * jj] = -1.0
                    A5[v, v] += 1.0 if (0 < i < m1 - 1 and 0 < j < m1 - 1) else 0.0
    interior = np.array([(0 < v % m1 < m1 - 1) and (0 < v // m1 < m1 - 1) for v in range(n)])
    Ad = A.toarray()
    A5d = A5.toarray()
    for v in np.where(interior)[0]:
        A5d[v, v] = 4.0
        np.testing.assert_allclose(Ad[v], A5d[v], atol=1e-13)
    key = lambda i, m, k: (i * nw + m) * n + k
    Tm = dict(zip(key(I, M, K), V))
    for i, m, k, v in zip(I, M, K, V):
        assert abs(Tm.get(key(k, m, i), 0.0) - v) < 1e-14
    sum_i = np.zeros((nw, n))
    np.add.at(sum_i, (M, K), V)
    sum_k = np.zeros((n, nw))
    np.add.at(sum_k, (I, M), V)
    assert np.abs(sum_i).max() < 1e-13 and np.abs(sum_k).max() < 1e-13


@pytest.mark.parametrize("dim", [2, 3])
def test_mass_matrix_closed_form(dim):
    """P1-P1 mass M_ij = |K| (1 + delta_ij) / ((d+1)(d+2)) per element; sum M = |Omega| = 1."""
    mesh = wl.unit_square_mesh(3) if dim == 2 else wl.unit_cube_mesh(2)
    P = oracle.Problem(mesh, a=None, a_deg=1, c=("exp",), c_deg=1, gamma=1.0)
    I, J, V = P.M_coo()
    M = sp.coo_matrix((V, (I, J)), shape=(P.n, P.n)).toarray()
    ref = np.zeros_like(M)
    for cell in mesh.cells:
        X = mesh.coords[cell]
        vol = abs(np.linalg.det((X[1:] - X[0]).T)) / factorial(dim)
        for a in cell:
            for b in cell:
                ref[a, b] += vol * (1 + (a == b)) / ((dim + 1) * (dim + 2))
    np.testing.assert_allclose(M, ref, atol=1e-15)
    assert abs(M.sum() - 1.0) < 1e-13


@pytest.mark.parametrize("dim,deg", [(2, 2), (2, 3), (3, 2), (3, 3)])
def test_interpolation_reproduces_linear_functions(dim, deg):
    """(Pi u)_m = u_h(x_m) (Sec. 3.2): exact for u linear; rows sum to 1."""
    mesh = wl.unit_square_mesh(4) if dim == 2 else wl.unit_cube_mesh(2)
    P = oracle.Problem(mesh, a=("pow", 2.0), a_deg=deg)
    Pi = P.Pi(0)
    xw = P.space_coords(0)
    coef = np.array([0.3, -1.2, 0.7, 2.1])[: dim + 1]
    u = coef[0] + mesh.coords @ coef[1:]
    np.testing.assert_allclose(Pi @ u, coef[0] + xw @ coef[1:], atol=1e-13)
    np.testing.assert_allclose(np.asarray(Pi.sum(axis=1)).ravel(), 1.0, atol=1e-13)


@pytest.mark.parametrize("label", ["SGA", "EGFEM_P2", "EGFEM_P3", "GFEM"])
def test_table1_sizes(label):
    """Unknown counts of Table 1 (Sec. 5.3) on the 64 x 64 triangulated square: the P1
    space plus, for the group methods, the W space of the substituted nonlinearity."""
    rows = [l.split() for l in open(f"{GOLDEN}/table1_sizes.txt") if l.strip() and not l.startswith("#")]
    row = next(r for r in rows if r[0] == label)
    n, wdeg, size = int(row[1]), int(row[2]), int(row[3])
    mesh = wl.unit_square_mesh(n)
    if wdeg == 0:
        assert mesh.n_nodes == size
        return
    P = oracle.Problem(mesh, a=("pow", 2.0), a_deg=wdeg, cells=np.array([0], dtype=np.int32))
    assert mesh.n_nodes + P.nw == size


def test_table1_quadrature_space_size():
    """I_4 of Table 1: one unknown per quadrature point of a 6-point rule per triangle."""
    rows = [l.split() for l in open(f"{GOLDEN}/table1_sizes.txt") if l.strip() and not l.startswith("#")]
    row = next(r for r in rows if r[0] == "EGFEM_I4")
    mesh = wl.unit_square_mesh(int(row[1]))
    assert mesh.n_nodes + 6 * mesh.n_cells == int(row[3])


# ---------------------------------------------------------------------------
# EGFEM vs SGA (Case 1 exactness), residual forms, Jacobians
# ---------------------------------------------------------------------------

def _rand_u(mesh, seed, scale=1.0):
    return wl.random_vector(mesh.n_nodes, seed, scale) * (1 - mesh.dirichlet)


@pytest.mark.parametrize("p,deg", [(2.0, 2), (3.0, 3)])
def test_case1_egfem_equals_sga_residual_and_jacobian(p, deg):
    """Case 1 (Sec. 3.1, Example 3.1): u^p with u in P1 lies in P_p, so EGFEM with W = P_p
    reproduces SGA exactly (Sec. 5: 'numerically equivalent to the standard Galerkin approach')."""
    mesh = wl.unit_square_mesh(8)
    P = oracle.Problem(mesh, a=("pow", p), a_deg=deg, qpts=5)
    b = P.load_vector(wl.mms_source)
    u = _rand_u(mesh, 3)
    r_e, r_s = P.residual(u, b, method="egfem"), P.residual(u, b, method="sga")
    assert np.linalg.norm(r_e - r_s) <= 1e-12 * np.linalg.norm(r_s)
    J_e, J_s = P.jacobian(u, "egfem"), P.jacobian(u, "sga")
    assert abs(J_e - J_s).max() <= 1e-12 * abs(J_s).max()


def test_gfem_is_not_exact():
    """Case 2 (Sec. 3.1): GFEM (W = V = P1) only approximates u^2, so it must differ from
    SGA -- this gives the exactness test above its power."""
    mesh = wl.unit_square_mesh(8)
    P = oracle.Problem(mesh, a=("pow", 2.0), a_deg=1)
    u = _rand_u(mesh, 3)
    b = np.zeros(mesh.n_nodes)
    r_e, r_s = P.residual(u, b, method="egfem"), P.residual(u, b, method="sga")
    assert np.linalg.norm(r_e - r_s) > 1e-3 * np.linalg.norm(r_s)


def test_residual_plain_and_difference_forms_agree():
    mesh = wl.unit_square_mesh(10)
    P = oracle.Problem(mesh, a=("pow", 2.0), a_deg=2)
    b = P.load_vector(wl.mms_source)
    u = _rand_u(mesh, 4)
    for method in ("egfem", "sga"):
        r1, r2 = P.residual(u, b, method=method), P.residual(u, b, method=method, form="diff")
        assert np.linalg.norm(r1 - r2) <= 1e-13 * np.linalg.norm(r1)


@pytest.mark.parametrize("method", ["egfem", "sga"])
@pytest.mark.parametrize("case", ["u2_p2", "u3_p3", "bratu_p1"])
def test_jacobian_matches_central_differences(method, case):
    """J columns equal (r(u + h e_l) - r(u - h e_l)) / 2h, h = 1e-6."""
    if case == "bratu_p1":
        mesh = wl.unit_cube_mesh(3)
        P = oracle.Problem(mesh, a=None, a_deg=1, c=("exp",), c_deg=1, gamma=-2.0)
    else:
        mesh = wl.unit_square_mesh(5)
        P = oracle.Problem(mesh, a=("pow", 2.0 if case == "u2_p2" else 3.0), a_deg=2 if case == "u2_p2" else 3)
    u = _rand_u(mesh, 5, 0.8)
    b = np.zeros(mesh.n_nodes)
    J = P.jacobian(u, method).toarray()
    h = 1e-6
    free = np.where(mesh.dirichlet == 0)[0]
    for l in free[:: max(1, len(free) // 12)]:
        e = np.zeros(mesh.n_nodes)
        e[l] = h
        col = (P.residual(u + e, b, method=method) - P.residual(u - e, b, method=method)) / (2 * h)
        np.testing.assert_allclose(J[free, l], col[free], atol=1e-7 * max(1.0, np.abs(J).max()))


# ---------------------------------------------------------------------------
# Linear solvers
# ---------------------------------------------------------------------------

def test_band_solve_matches_lapack():
    """Banded LU with partial pivoting vs LAPACK gbsv (scipy.linalg.solve_banded)."""
    rng = np.random.default_rng(7)
    n, kl, ku = 60, 4, 3
    A = np.zeros((n, n))
    for i in range(n):
        for j in range(max(0, i - kl), min(n, i + ku + 1)):
            A[i, j] = rng.standard_normal()
    rhs = rng.standard_normal(n)
    ab = np.zeros((kl + ku + 1, n))
    for i in range(n):
        for j in range(max(0, i - kl), min(n, i + ku + 1)):
            ab[ku + i - j, j] = A[i, j]
    ref = sla.solve_banded((kl, ku), ab, rhs)
    got = oracle.band_solve(sp.csr_matrix(A), rhs)
    np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-12)


def test_bicgstab_matches_direct_solve():
    mesh = wl.unit_square_mesh(12)
    P = oracle.Problem(mesh, a=("pow", 2.0), a_deg=2)
    J = P.jacobian(_rand_u(mesh, 8, 0.5), "egfem")
    rhs = wl.random_vector(mesh.n_nodes, 9)
    ref = spla.spsolve(J.tocsc(), rhs)
    x, st, its, rr = oracle.bicgstab(J, rhs, rtol=1e-13)
    assert st == 0 and its > 5
    np.testing.assert_allclose(x, ref, rtol=1e-9, atol=1e-11)


# ---------------------------------------------------------------------------
# Newton: Case-1 iterates, manufactured-solution rates, Bratu
# ---------------------------------------------------------------------------

def test_newton_iterates_egfem_equal_sga_on_32x32():
    """Same Newton iterates for EGFEM (w = u^2 in P2) and SGA on the 32 x 32 grid."""
    mesh = wl.unit_square_mesh(32)
    P = oracle.Problem(mesh, a=("pow", 2.0), a_deg=2)
    b = P.load_vector(wl.mms_source)
    ue, he, ie, _ = P.newton(b, method="egfem", rtol=1e-13, keep_iterates=True)
    us, hs, is_, _ = P.newton(b, method="sga", rtol=1e-13, keep_iterates=True)
    assert len(he) == len(hs) and len(he) <= 8
    for a, c in zip(ie[1:], is_[1:]):
        assert np.linalg.norm(a - c) <= 1e-12 * np.linalg.norm(c)
    assert he[-1] <= 1e-13 * he[0]


def _errors(mesh, u):
    """L2 and H1-seminorm errors of the P1 function u against sin(pi x) sin(pi y),
    by a 6x6 collapsed Gauss rule per triangle (test-side arithmetic)."""
    pts, wts = oracle.simplex_rule(2, 6)
    l2 = h1 = 0.0
    X = mesh.coords[mesh.cells]              # [nc, 3, 2]
    U = u[mesh.cells]                        # [nc, 3]
    B = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]], axis=2)   # columns
    det = np.abs(np.linalg.det(B))
    lam = np.stack([1 - pts.sum(1), pts[:, 0], pts[:, 1]], axis=1)  # [nq, 3]
    xq = np.einsum("qa,cad->cqd", lam, X)
    uh = np.einsum("qa,ca->cq", lam, U)
    G = np.einsum("ab,cbd->cad", np.array([[-1.0, -1.0], [1.0, 0.0], [0.0, 1.0]]), np.linalg.inv(B))
    guh = np.einsum("ca,cad->cd", U, G)
    ex = wl.mms_exact(xq[..., 0], xq[..., 1])
    gx, gy = wl.mms_exact_grad(xq[..., 0], xq[..., 1])
    l2 = np.sum(det[:, None] * wts[None] * (uh - ex) ** 2)
    h1 = np.sum(det[:, None] * wts[None] * ((guh[:, None, 0] - gx) ** 2 + (guh[:, None, 1] - gy) ** 2))
    return np.sqrt(l2), np.sqrt(h1)


def test_manufactured_solution_convergence_rates():
    """P1 Newton solutions of -div((1+u^2) grad u) = f converge at O(h^2) in L2 and O(h)
    in H1 (method of manufactured solutions, Sec. 5)."""
    errs = []
    for n in (8, 16, 32, 64):
        mesh = wl.unit_square_mesh(n)
        P = oracle.Problem(mesh, a=("pow", 2.0), a_deg=2)
        b = P.load_vector(wl.mms_source)
        u, _, _, _ = P.newton(b, rtol=1e-12)
        errs.append(_errors(mesh, u))
    e = np.array(errs)
    rates = np.log2(e[:-1] / e[1:])
    assert np.all(np.abs(rates[:, 0] - 2.0) < 0.1), rates
    assert np.all(np.abs(rates[:, 1] - 1.0) < 0.1), rates


def test_bratu_limits_and_gfem_rate():
    """Bratu -lap u = lambda e^u: lambda = 0 with f = 0 gives u = 0; lambda = 2 converges;
    lambda = 12 lies above the critical value (about 9.9 on the cube) and Newton from 0
    fails; the GFEM (W = P1, Case 2) solution differs from SGA by O(h^2)."""
    mesh = wl.unit_cube_mesh(4)
    P0 = oracle.Problem(mesh, a=None, a_deg=1, c=("exp",), c_deg=1, gamma=0.0)
    u, hist, _, _ = P0.newton(np.zeros(mesh.n_nodes))
    assert np.abs(u).max() == 0.0
    diffs = []
    for n in (4, 8, 16):
        mesh = wl.unit_cube_mesh(n)
        P = oracle.Problem(mesh, a=None, a_deg=1, c=("exp",), c_deg=1, gamma=-2.0, qpts=4)
        ue, he, _, _ = P.newton(np.zeros(mesh.n_nodes), method="egfem", rtol=1e-12, solver="lu" if n < 16 else "bicgstab")
        us, hs, _, _ = P.newton(np.zeros(mesh.n_nodes), method="sga", rtol=1e-12, solver="lu" if n < 16 else "bicgstab")
        assert ue.max() > 0.01
        diffs.append(np.abs(ue - us).max())
    rates = np.log2(np.array(diffs[:-1]) / np.array(diffs[1:]))
    assert np.all(rates > 1.7), (diffs, rates)
    mesh = wl.unit_cube_mesh(4)
    P = oracle.Problem(mesh, a=None, a_deg=1, c=("exp",), c_deg=1, gamma=-12.0)
    with pytest.raises(RuntimeError):
        P.newton(np.zeros(mesh.n_nodes), maxit=30)


# ---------------------------------------------------------------------------
# Adjoint
# ---------------------------------------------------------------------------

def test_adjoint_linear_special_case():
    """With no nonlinearity the Jacobian is the stiffness matrix and lambda solves
    A^T lambda = u - u_d exactly (direct sparse solve)."""
    mesh = wl.unit_square_mesh(10)
    P = oracle.Problem(mesh, a=None, a_deg=1)
    b = P.load_vector(wl.mms_source)
    u, _, _, _ = P.newton(b)
    ud = wl.adjoint_target()(mesh.coords[:, 0], mesh.coords[:, 1])
    g = (u - ud) * (1 - mesh.dirichlet)
    lam, _ = P.adjoint(u, g)
    A = P.jacobian(u, "egfem").tocsc()
    np.testing.assert_allclose(lam, spla.spsolve(A.T.tocsc(), g), rtol=1e-10, atol=1e-14)


def test_adjoint_gradients_match_central_differences():
    """dJ/db_i = lambda_i and dJ/dkappa_m = -sum lambda_i T_imk u_k for
    J = 0.5 ||u - u_d||^2, against central differences (h = 1e-6) of re-solved Newton."""
    mesh = wl.unit_square_mesh(8)
    P = oracle.Problem(mesh, a=("pow", 2.0), a_deg=2)
    kappa = np.ones(P.nw)
    P.set_kappa_field(kappa)
    b = P.load_vector(wl.mms_source)
    ud = wl.adjoint_target()(mesh.coords[:, 0], mesh.coords[:, 1])

    def J_of(bb, kk):
        P.set_kappa_field(kk)
        u, _, _, _ = P.newton(bb, rtol=1e-14, maxit=60)
        return 0.5 * np.sum((u - ud) ** 2 * (1 - mesh.dirichlet)), u

    J0, u = J_of(b, kappa)
    lam, gk = P.adjoint(u, (u - ud) * (1 - mesh.dirichlet))
    h = 1e-6
    free = np.where(mesh.dirichlet == 0)[0]
    for i in free[::9]:
        e = np.zeros(mesh.n_nodes)
        e[i] = h
        fd = (J_of(b + e, kappa)[0] - J_of(b - e, kappa)[0]) / (2 * h)
        assert abs(fd - lam[i]) <= 1e-6 * max(1e-3, abs(lam[i])), (i, fd, lam[i])
    for m in range(0, P.nw, 37):
        e = np.zeros(P.nw)
        e[m] = h
        fd = (J_of(b, kappa + e)[0] - J_of(b, kappa - e)[0]) / (2 * h)
        assert abs(fd - gk[m]) <= 1e-6 * max(1e-4, abs(gk[m])), (m, fd, gk[m])


# ---------------------------------------------------------------------------------------
# Picard iteration (Sec. 4, Example 4.1): the frozen-coefficient matrix A(u) = T .2 a(u)
# ---------------------------------------------------------------------------------------

def test_picard_matrix_reproduces_the_residual():
    """A(u) u - b is the plain-form residual on free rows (r = sum T_imk a_m u_k - b), and A(u)
    is the Newton Jacobian without its g' block: for a constant coefficient they coincide."""
    mesh = wl.unit_square_mesh(7)
    P = oracle.Problem(mesh, a=("pow", 2.0), a_deg=2)
    u = wl.random_vector(mesh.n_nodes, 11, 0.7) * (1 - mesh.dirichlet)
    b = wl.random_vector(mesh.n_nodes, 12) * (1 - mesh.dirichlet)
    A = P.jacobian(u, method="picard")
    r = P.residual(u, b, form="plain")
    free = mesh.dirichlet == 0
    assert np.abs((A @ u - b)[free] - r[free]).max() <= 1e-13 * np.abs(r).max()
    J = P.jacobian(u)
    assert abs(J - A).max() > 1e-3                      # the g' block is there in Newton
    Pc = oracle.Problem(mesh, a=None, a_deg=1, kappa=2.5)
    assert abs(Pc.jacobian(u) - Pc.jacobian(u, method="picard")).max() <= 1e-14


def test_picard_and_newton_reach_the_same_solution():
    """Both iterations converge to the one discrete solution; Picard linearly (more steps,
    residual ratios bounded away from zero), Newton quadratically."""
    mesh = wl.unit_square_mesh(12)
    P = oracle.Problem(mesh, a=("pow", 2.0), a_deg=2)
    b = P.load_vector(wl.mms_source) * (1 - mesh.dirichlet)
    un, hn, _, _ = P.newton(b, rtol=1e-12)
    up, hp, _, _ = P.newton(b, rtol=1e-12, iteration="picard", maxit=200)
    assert np.linalg.norm(up - un) <= 1e-10 * np.linalg.norm(un)
    assert len(hp) > len(hn) + 2
    ratios = hp[2:] / hp[1:-1]
    assert ratios.max() < 0.9 and np.median(ratios) > 1e-3


def test_picard_solves_a_linear_problem_in_one_step():
    """With a constant coefficient the Picard matrix is the stiffness matrix: one exact step."""
    mesh = wl.unit_square_mesh(9)
    P = oracle.Problem(mesh, a=None, a_deg=1, kappa=1.7)
    b = P.load_vector(wl.mms_source) * (1 - mesh.dirichlet)
    u, h, _, _ = P.newton(b, rtol=1e-13, iteration="picard")
    assert len(h) == 2 and h[-1] <= 1e-13 * h[0]


# ---------------------------------------------------------------------------------------
# Gradient nonlinearities with W = P0 (Sec. 5, p-Laplace and minimal surface examples)
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("q,shift", [(-0.5, 1.0), (0.25, 0.3), (-0.25, 0.05)])
def test_gradient_nonlinearity_egfem_p0_equals_sga(q, shift):
    """For P1 u the gradient is constant per cell, so EGFEM with a P0 W space (the tensor path:
    T_iKk, nodal g(||grad u_K||^2)) equals the standard Galerkin approach (the quadrature path)
    exactly -- the equivalence the paper reports for these examples."""
    mesh = wl.unit_square_mesh(7)
    P = oracle.Problem(mesh, a=("gradpow", q, shift), a_deg=0, kappa=0.4)
    u = wl.random_vector(mesh.n_nodes, 31, 0.8)
    b = wl.random_vector(mesh.n_nodes, 32)
    re, rs = P.residual(u, b, form="plain"), P.residual(u, b, method="sga", form="plain")
    assert np.abs(re - rs).max() <= 1e-13 * np.abs(re).max()
    Je, Js = P.jacobian(u), P.jacobian(u, method="sga")
    assert abs(Je - Js).max() <= 1e-13 * abs(Je).max()


def test_gradient_nonlinearity_jacobian_matches_finite_differences():
    mesh = wl.unit_square_mesh(6)
    P = oracle.Problem(mesh, a=("gradpow", -0.5, 1.0), a_deg=0, kappa=0.0)
    u = wl.random_vector(mesh.n_nodes, 41, 0.9)
    b = wl.random_vector(mesh.n_nodes, 42)
    J = P.jacobian(u).toarray()
    free = np.where(mesh.dirichlet == 0)[0]
    h = 1e-6
    for l in free[::3]:
        e = np.zeros(mesh.n_nodes)
        e[l] = h
        fd = (P.residual(u + e, b, form="plain") - P.residual(u - e, b, form="plain")) / (2 * h)
        assert np.abs(fd[free] - J[free, l]).max() <= 1e-8 * max(1.0, np.abs(J).max())


def test_constant_gradient_coefficient_is_the_stiffness_matrix():
    """With exponent 0 the coefficient is the constant scale * 1: the Jacobian is that multiple
    of the Poisson stiffness matrix (no derivative term)."""
    mesh = wl.unit_square_mesh(5)
    u = wl.random_vector(mesh.n_nodes, 51, 0.5)
    A = oracle.Problem(mesh, a=("gradpow", 0.0, 2.0), a_deg=0, a_scale=1.5, kappa=0.0).jacobian(u)
    S = oracle.Problem(mesh, a=None, a_deg=1, kappa=1.5).jacobian(u)
    assert abs(A - S).max() <= 1e-13


def test_minimal_surface_manufactured_solution_converges_at_second_order():
    """Minimal surface on the unit square with u_D = x y (x + y) and the manufactured source:
    the nodal RMS error falls by about 4 per mesh halving (P1, O(h^2))."""
    errs = []
    for n in (8, 16, 32):
        mesh = wl.unit_square_mesh(n)
        P = oracle.Problem(mesh, a=("gradpow", -0.5, 1.0), a_deg=0, kappa=0.0)
        ue = wl.minsurf_exact(mesh.coords[:, 0], mesh.coords[:, 1])
        b = P.load_vector(wl.minsurf_source) * (1 - mesh.dirichlet)
        u, _, _, _ = P.newton(b, u0=ue, uD=ue * mesh.dirichlet, rtol=1e-8)
        errs.append(np.sqrt(np.mean((u - ue) ** 2)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates.min() > 1.8, (errs, rates)


def test_p_laplace_disk_closed_form_second_order():
    """p-Laplace, p = 3/2, d = 1 on the unit disk with u = 0 on its boundary (Sec. 5): the
    Picard iteration with W = P0 reaches the closed-form solution at O(h^2) in the nodal RMS
    error (a = ||grad u||^(p-2), regularised by a 1e-12 shift of ||grad u||^2), and Newton
    from the interpolated exact solution reaches the same discrete solution."""
    p = 1.5
    errs = []
    for n in (4, 8, 16):
        mesh = wl.unit_disk_mesh(n)
        ue = wl.plaplace_disk_exact(mesh.coords[:, 0], mesh.coords[:, 1], p)
        P = oracle.Problem(mesh, a=("gradpow", (p - 2) / 2, 1e-12), a_deg=0, kappa=0.0)
        b = P.load_vector(lambda x, y: np.ones_like(x)) * (1 - mesh.dirichlet)
        u, h, _, _ = P.newton(b, rtol=1e-10, iteration="picard", maxit=200)
        assert h[-1] <= 1e-10 * h[0]
        errs.append(np.sqrt(np.mean((u - ue) ** 2)))
        if n == 8:
            un, hn, _, _ = P.newton(b, u0=ue * (1 - mesh.dirichlet), rtol=1e-10)
            assert len(hn) <= 6 and np.abs(un - u).max() <= 1e-9
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates.min() > 1.8 and errs[-1] < 5e-5, (errs, rates)


def test_unit_disk_mesh_is_a_conforming_triangulation():
    """The disk generator: 6 n^2 positively oriented cells, every interior edge shared by two
    cells, the boundary ring on the circle, and the area tending to pi at O(h^2)."""
    from collections import Counter
    for n in (1, 3, 8):
        m = wl.unit_disk_mesh(n)
        assert m.n_cells == 6 * n * n and m.n_nodes == 1 + 3 * n * (n + 1)
        c = m.coords[m.cells]
        det = (c[:, 1, 0] - c[:, 0, 0]) * (c[:, 2, 1] - c[:, 0, 1]) - (c[:, 1, 1] - c[:, 0, 1]) * (c[:, 2, 0] - c[:, 0, 0])
        assert det.min() > 0
        edges = Counter(tuple(sorted((t[a], t[b]))) for t in m.cells for a, b in ((0, 1), (1, 2), (2, 0)))
        bnd = {e for e, k in edges.items() if k == 1}
        assert set(edges.values()) <= {1, 2} and len(bnd) == 6 * n
        assert all(m.dirichlet[v] for e in bnd for v in e)
        assert np.allclose(np.hypot(*m.coords[m.dirichlet == 1].T), 1.0)
        # inscribed 6n-gon: area (6n/2) sin(2 pi / 6n)
        assert abs(det.sum() / 2 - 3 * n * np.sin(2 * np.pi / (6 * n))) <= 1e-12


# ---------------------------------------------------------------------------------------
# Quadrature spaces I_k (Sec. 3.1, Case 3)
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("dim,k", [(2, 1), (2, 2), (2, 3), (2, 4), (3, 1), (3, 2), (3, 3)])
def test_symmetric_rule_is_exact_to_its_degree_and_no_further(dim, k):
    """The rule behind I_k integrates every monomial of degree <= k over the reference simplex
    exactly (int xi^alpha = alpha! / (|alpha| + d)!) and misses one of degree k + 1."""
    import itertools
    import math
    p, w = oracle.sym_rule(dim, k)
    assert np.all(p >= 0) and np.all(p.sum(axis=1) <= 1)
    worst = {}
    for deg in range(k + 2):
        for al in itertools.product(range(deg + 1), repeat=dim):
            if sum(al) != deg:
                continue
            exact = np.prod([math.factorial(a) for a in al]) / math.factorial(deg + dim)
            err = abs(np.sum(w * np.prod(p ** np.array(al), axis=1)) - exact)
            worst[deg] = max(worst.get(deg, 0.0), err)
    assert max(worst[d] for d in range(k + 1)) <= 1e-15
    assert worst[k + 1] > 1e-6


def test_table1_quadrature_space_size():
    """Table 1: on the 64 x 64 grid the EGFEM with I_4 has 53377 unknowns (4225 P1 nodes plus
    six rule points on each of the 8192 triangles)."""
    mesh = wl.unit_square_mesh(64)
    P = oracle.Problem(mesh, a=None, a_deg=1, c=("pow", 3.0), c_deg=4, c_space="quad", gamma=1.0)
    assert mesh.n_nodes + P.nc_space == 53377


@pytest.mark.parametrize("dim,k", [(2, 1), (2, 2), (2, 3), (2, 4), (3, 1), (3, 2), (3, 3)])
def test_quadrature_space_reproduces_sga_with_the_same_rule(dim, k):
    """Case 3's claim: with W = I_k for both the coefficient and the reaction, the EGFEM
    residual and Jacobian equal those of the standard Galerkin approach integrated by the same
    rule (to rounding), for any nonlinearity."""
    mesh = wl.unit_square_mesh(5) if dim == 2 else wl.unit_cube_mesh(2)
    kw = dict(a=("pow", 3.0), a_deg=k, a_space="quad", c=("exp",), c_deg=k, c_space="quad", gamma=0.7,
              kappa=0.5, rule=k)
    P = oracle.Problem(mesh, **kw)
    assert P.nw == P.nc_space == mesh.n_cells * len(oracle.sym_rule(dim, k)[1])
    u = wl.random_vector(mesh.n_nodes, 61, 0.8)
    b = wl.random_vector(mesh.n_nodes, 62)
    re, rs = P.residual(u, b, form="plain"), P.residual(u, b, method="sga", form="plain")
    assert np.abs(re - rs).max() <= 1e-13 * np.abs(rs).max()
    Je, Js = P.jacobian(u), P.jacobian(u, method="sga")
    assert abs(Je - Js).max() <= 1e-13 * abs(Js).max()


def test_quadrature_and_lagrange_spaces_agree_where_both_are_exact():
    """c = u^2 with u in P1: W_c = P2 holds it exactly, and I_3 integrates u^2 phi_i exactly,
    so both EGFEM residuals equal the exactly integrated one; likewise a = 1 + u^2 with
    W_a = P2 and W_a = I_2 (the integrand a(u) grad phi_k . grad phi_i is quadratic)."""
    mesh = wl.unit_square_mesh(6)
    u = wl.random_vector(mesh.n_nodes, 71, 0.9)
    b = wl.random_vector(mesh.n_nodes, 72)
    base = dict(a=("pow", 2.0), kappa=1.0, c=("pow", 2.0), gamma=1.3)
    r_lag = oracle.Problem(mesh, a_deg=2, c_deg=2, **base).residual(u, b)
    r_quad = oracle.Problem(mesh, a_deg=2, a_space="quad", c_deg=3, c_space="quad", **base).residual(u, b)
    r_sga = oracle.Problem(mesh, a_deg=2, c_deg=2, qpts=4, **base).residual(u, b, method="sga")
    scale = np.abs(r_sga).max()
    assert np.abs(r_lag - r_sga).max() <= 1e-13 * scale
    assert np.abs(r_quad - r_sga).max() <= 1e-13 * scale


def test_i1_equals_p0_for_the_gradient_coefficient():
    """For P1 u the gradient is constant per cell, so I_1 (one point, weight |K|) and P0 give
    the same residual and Jacobian (Sec. 5 uses both for the p-Laplace and minimal surface)."""
    mesh = wl.unit_square_mesh(6)
    u = wl.random_vector(mesh.n_nodes, 81, 0.7)
    b = wl.random_vector(mesh.n_nodes, 82)
    P0 = oracle.Problem(mesh, a=("gradpow", -0.5, 1.0), a_deg=0, kappa=0.0)
    I1 = oracle.Problem(mesh, a=("gradpow", -0.5, 1.0), a_deg=1, a_space="quad", kappa=0.0)
    assert np.abs(P0.residual(u, b) - I1.residual(u, b)).max() <= 1e-14
    assert abs(P0.jacobian(u) - I1.jacobian(u)).max() <= 1e-14


# ---------------------------------------------------------------------------------------
# Reaction EGFEM with higher-order W_c: the superconductivity example (Sec. 5, Table 1)
# ---------------------------------------------------------------------------------------

def _supercond(mesh, nu, **w):
    """Decomposition (b): nu K u + M u + M^c c with c = u^3 on W_c (kappa = nu, sigma = 1)."""
    return oracle.Problem(mesh, a=None, a_deg=1, kappa=nu, c=("pow", 3.0), gamma=1.0, sigma=1.0, **w)


def test_laplacian_of_the_superconductivity_solution():
    """The manufactured source's closed-form Laplacian against central differences."""
    rng = np.random.Generator(np.random.PCG64(5))
    x, y = rng.uniform(0.1, 0.9, 20), rng.uniform(0.1, 0.9, 20)
    h = 1e-4
    u = wl.supercond_exact
    lap_fd = (u(x + h, y) + u(x - h, y) + u(x, y + h) + u(x, y - h) - 4 * u(x, y)) / h ** 2
    lap = (u(x, y) ** 3 + u(x, y) - wl.supercond_source(x, y, 1.0))   # = lap u for nu = 1
    assert np.abs(lap - lap_fd).max() <= 1e-5 * np.abs(lap).max()


@pytest.mark.parametrize("space", ["p3", "p2", "i4"])
def test_superconductivity_egfem_reproduces_sga(space):
    """c = u^3 with u in P1 is a cubic on every cell: P3 W_c holds it exactly (Case 1) and I_4
    integrates u^3 phi_i exactly (Case 3), so both EGFEM variants of Table 1 equal the standard
    Galerkin approach; P2 W_c only interpolates c (Case 2) and differs from it."""
    mesh = wl.unit_square_mesh(6)
    u = wl.random_vector(mesh.n_nodes, 91, 0.8)
    b = wl.random_vector(mesh.n_nodes, 92) * 1e-3
    kw = {"p3": dict(c_deg=3), "p2": dict(c_deg=2), "i4": dict(c_deg=4, c_space="quad")}[space]
    P = _supercond(mesh, 0.01, **kw)
    S = _supercond(mesh, 0.01, c_deg=3)
    r, rs = P.residual(u, b), S.residual(u, b, method="sga")
    if space in ("p3", "i4"):
        assert np.abs(r - rs).max() <= 1e-13 * np.abs(rs).max()
        assert abs(P.jacobian(u) - S.jacobian(u, method="sga")).max() <= 1e-13 * abs(S.jacobian(u, method="sga")).max()
    else:
        assert np.abs(r - rs).max() > 1e-10 * np.abs(rs).max()


def test_sigma_term_is_the_p1_mass_matrix():
    """sigma M u with M_ab = |K| (1 + delta_ab) / 12 per triangle (closed form of int phi_a phi_b)."""
    mesh = wl.unit_square_mesh(4)
    P = oracle.Problem(mesh, a=None, a_deg=1, kappa=0.0, sigma=2.5)
    u = wl.random_vector(mesh.n_nodes, 93)
    M = np.zeros((mesh.n_nodes, mesh.n_nodes))
    for cell in mesh.cells:
        X = mesh.coords[cell]
        e1, e2 = X[1] - X[0], X[2] - X[0]
        area = 0.5 * abs(e1[0] * e2[1] - e1[1] * e2[0])
        for a in range(3):
            for b2 in range(3):
                M[cell[a], cell[b2]] += area * (2.0 if a == b2 else 1.0) / 12.0
    free = mesh.dirichlet == 0
    r = P.residual(u, np.zeros(mesh.n_nodes))
    assert np.abs(r[free] - 2.5 * (M @ u)[free]).max() <= 1e-15


@pytest.mark.parametrize("space", ["p3", "i4"])
def test_superconductivity_manufactured_solution_second_order(space):
    kw = {"p3": dict(c_deg=3), "i4": dict(c_deg=4, c_space="quad")}[space]
    errs = []
    for n in (8, 16, 32):
        mesh = wl.unit_square_mesh(n)
        P = _supercond(mesh, 1.0, **kw)
        ue = wl.supercond_exact(mesh.coords[:, 0], mesh.coords[:, 1])
        b = P.load_vector(lambda x, y: wl.supercond_source(x, y, 1.0)) * (1 - mesh.dirichlet)
        uD = ue * mesh.dirichlet
        u, h, _, _ = P.newton(b, u0=uD, uD=uD, rtol=1e-11)
        errs.append(np.sqrt(np.mean((u - ue) ** 2)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates.min() > 1.8, (errs, rates)


@pytest.mark.parametrize("space", ["p2", "i4"])
def test_superconductivity_decomposition_a_reproduces_sga(space):
    """Decomposition (a): nu K u + M3 : (u x c~) with c~ = u^2 + 1, written as sigma M u (the +1)
    plus the product reaction int c u phi_i with c = u^2.  P2 holds u^2 exactly and I_4 integrates
    u^3 phi_i exactly, so both equal the standard Galerkin approach, and the residual equals that
    of decomposition (b) (nu K u + M u + M^c u^3 on P3)."""
    mesh = wl.unit_square_mesh(6)
    u = wl.random_vector(mesh.n_nodes, 95, 0.8)
    b = wl.random_vector(mesh.n_nodes, 96) * 1e-3
    kw = dict(c_deg=2) if space == "p2" else dict(c_deg=4, c_space="quad")
    A = oracle.Problem(mesh, a=None, a_deg=1, kappa=0.01, c=("pow", 2.0), gamma=1.0, sigma=1.0, c_product=True, **kw)
    rs = A.residual(u, b, method="sga")
    assert np.abs(A.residual(u, b) - rs).max() <= 1e-13 * np.abs(rs).max()
    Js = A.jacobian(u, method="sga")
    assert abs(A.jacobian(u) - Js).max() <= 1e-13 * abs(Js).max()
    B = _supercond(mesh, 0.01, c_deg=3)
    assert np.abs(B.residual(u, b) - A.residual(u, b)).max() <= 1e-13 * np.abs(rs).max()


def test_product_reaction_jacobian_matches_finite_differences():
    """Case 2 (exp interpolated in P2) for the product form: the Jacobian against central
    differences of the residual (both terms of d(c u)/du)."""
    mesh = wl.unit_square_mesh(5)
    P = oracle.Problem(mesh, a=None, a_deg=1, kappa=0.5, c=("exp",), c_deg=2, gamma=0.7, c_product=True)
    u = wl.random_vector(mesh.n_nodes, 97, 0.8)
    b = wl.random_vector(mesh.n_nodes, 98)
    J = P.jacobian(u).toarray()
    free = np.where(mesh.dirichlet == 0)[0]
    h = 1e-6
    for l in free[::2]:
        e = np.zeros(mesh.n_nodes)
        e[l] = h
        fd = (P.residual(u + e, b) - P.residual(u - e, b)) / (2 * h)
        assert np.abs(fd[free] - J[free, l]).max() <= 1e-8 * max(1.0, np.abs(J).max())
