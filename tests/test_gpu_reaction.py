"""GPU checks of reaction EGFEM with higher-order W_c (Lagrange P2/P3, I_k) and the linear
reaction sigma M u, in the element-local operator: residual and Jacobian against the oracle,
and the superconductivity example (Sec. 5, Table 1, decomposition (b): nu K u + M u + M^c c,
c = u^3) solved with W_c = P3 and I_4 against the oracle's standard Galerkin solution, which both
reproduce exactly."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import workloads as wl

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2005_06193_gb300 as P
    return P


def cuda(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _jac(h, u, n):
    rp, cl = h.pattern()
    vals = torch.empty(h.sizes.jac_nnz, device="cuda", dtype=torch.float64)
    h.jacobian(cuda(u), vals)
    torch.cuda.synchronize()
    return sp.csr_matrix((vals.cpu().numpy(), cl.cpu().numpy(), rp.cpu().numpy()), shape=(n, n))


# (dim, W_c degree, reaction kind, sigma, coefficient)
CASES = [(2, 2, ("pow", 3), 0.0, None), (2, 3, ("pow", 3), 1.3, None), (2, 3, ("exp",), 0.0, ("pow", 2)),
         (3, 2, ("pow", 2), 0.7, None), (3, 2, ("exp",), 0.0, ("pow", 2)), (2, 1, ("exp",), 0.9, None)]


@pytest.mark.parametrize("dim,deg,c,sigma,a", CASES)
def test_reaction_space_residual_and_jacobian_parity(P, dim, deg, c, sigma, a):
    mesh = wl.unit_square_mesh(10) if dim == 2 else wl.unit_cube_mesh(3)
    orc = oracle.Problem(mesh, a=(a[0], float(a[1])) if a else None, a_deg=2 if a else 1,
                         c=(c[0], float(c[1])) if len(c) > 1 else c, c_deg=deg, gamma=0.8, kappa=0.6, sigma=sigma)
    h = P.Handle(mesh, P.make_problem(a=a, a_degree=2 if a else 1, c=c, c_degree=deg, gamma=0.8, kappa=0.6,
                                      sigma=sigma), P.default_options(op=P.OP_MATRIX_FREE))
    if deg > 1:
        assert h.sizes.n_wc == orc.nc_space
    b = wl.random_vector(mesh.n_nodes, 3) * (1 - mesh.dirichlet)
    u = wl.random_vector(mesh.n_nodes, 4, 0.8)
    r = torch.empty(mesh.n_nodes, device="cuda", dtype=torch.float64)
    h.residual(cuda(u), cuda(b), r)
    torch.cuda.synchronize()
    assert rel(r.cpu().numpy(), orc.residual(u, b)) <= 1e-12
    A, Ao = _jac(h, u, mesh.n_nodes), orc.jacobian(u)
    assert abs(A - Ao).max() <= 1e-12 * abs(Ao).max()


def test_reaction_space_picard_matrix_keeps_the_linear_term(P):
    mesh = wl.unit_square_mesh(10)
    orc = oracle.Problem(mesh, a=None, a_deg=1, c=("pow", 3.0), c_deg=3, gamma=1.0, kappa=0.01, sigma=1.0)
    h = P.Handle(mesh, P.make_problem(a=None, a_degree=1, c=("pow", 3), c_degree=3, gamma=1.0, kappa=0.01, sigma=1.0),
                 P.default_options(op=P.OP_MATRIX_FREE, iteration=P.ITER_PICARD))
    u = wl.random_vector(mesh.n_nodes, 8, 0.8)
    A, Ao = _jac(h, u, mesh.n_nodes), orc.jacobian(u, method="picard")
    assert abs(A - Ao).max() <= 1e-12 * abs(Ao).max()


@pytest.mark.parametrize("space,nu,prec", [("p3", 1.0, "fp64"), ("i4", 1.0, "fp64"), ("p3", 1e-2, "fp64"),
                                           ("i4", 1e-2, "mixed")])
def test_superconductivity_newton_matches_sga(P, space, nu, prec):
    """Decomposition (b) on the 32 x 32 grid: W_c = P3 and I_4 both reproduce the standard
    Galerkin discretisation (c = u^3 is cubic per cell), so the library's Newton solution equals
    the oracle's SGA solution."""
    mesh = wl.unit_square_mesh(32)
    x, y = mesh.coords[:, 0], mesh.coords[:, 1]
    ue = wl.supercond_exact(x, y)
    uD = ue * mesh.dirichlet
    sga = oracle.Problem(mesh, a=None, a_deg=1, kappa=nu, c=("pow", 3.0), c_deg=3, gamma=1.0, sigma=1.0)
    b = sga.load_vector(lambda xx, yy: wl.supercond_source(xx, yy, nu)) * (1 - mesh.dirichlet)
    u_sga, _, _, _ = sga.newton(b, u0=uD, uD=uD, method="sga", rtol=1e-13)
    deg, cs = (3, "lagrange") if space == "p3" else (4, "quad")
    mixed = prec == "mixed"
    h = P.Handle(mesh, P.make_problem(a=None, a_degree=1, kappa=nu, c=("pow", 3), c_degree=deg, c_space=cs,
                                      gamma=1.0, sigma=1.0),
                 P.default_options(op=P.OP_MATRIX_FREE, newton_rtol=1e-10 if mixed else 1e-13,
                                   precision=P.PREC_MIXED if mixed else P.PREC_FP64))
    u = cuda(uD)
    st = h.newton_solve(u, cuda(b + uD))
    torch.cuda.synchronize()
    assert st.status == 0
    assert rel(u.cpu().numpy(), u_sga) <= (1e-8 if mixed else 1e-11)


# product reaction gamma int c u phi_i (decomposition (a)): (dim, W_c degree, space, kind)
PRODUCT = [(2, 1, "lagrange", ("exp",)), (2, 2, "lagrange", ("pow", 2)), (2, 4, "quad", ("pow", 2)),
           (3, 2, "lagrange", ("exp",)), (3, 3, "quad", ("pow", 2))]


@pytest.mark.parametrize("iteration", ["newton", "picard"])
@pytest.mark.parametrize("dim,deg,space,c", PRODUCT)
def test_product_reaction_parity(P, dim, deg, space, c, iteration):
    mesh = wl.unit_square_mesh(9) if dim == 2 else wl.unit_cube_mesh(3)
    orc = oracle.Problem(mesh, a=None, a_deg=1, c=(c[0], float(c[1])) if len(c) > 1 else c, c_deg=deg, c_space=space,
                         gamma=0.9, kappa=0.3, sigma=0.5, c_product=True)
    h = P.Handle(mesh, P.make_problem(a=None, a_degree=1, c=c, c_degree=deg, c_space=space, gamma=0.9, kappa=0.3,
                                      sigma=0.5, c_product=True),
                 P.default_options(op=P.OP_MATRIX_FREE, iteration=P.ITER_PICARD if iteration == "picard" else P.ITER_NEWTON))
    b = wl.random_vector(mesh.n_nodes, 13) * (1 - mesh.dirichlet)
    u = wl.random_vector(mesh.n_nodes, 14, 0.8)
    r = torch.empty(mesh.n_nodes, device="cuda", dtype=torch.float64)
    h.residual(cuda(u), cuda(b), r)
    torch.cuda.synchronize()
    assert rel(r.cpu().numpy(), orc.residual(u, b)) <= 1e-12
    A, Ao = _jac(h, u, mesh.n_nodes), orc.jacobian(u, method="picard" if iteration == "picard" else "egfem")
    assert abs(A - Ao).max() <= 1e-12 * abs(Ao).max()


@pytest.mark.parametrize("space,nu", [("p2", 1.0), ("i4", 1.0), ("p2", 1e-2)])
def test_superconductivity_decomposition_a_newton_matches_sga(P, space, nu):
    """Decomposition (a) on the 32 x 32 grid: sigma M u plus the product reaction with c = u^2 on
    P2 or I_4 reproduces the standard Galerkin discretisation of -nu lap u + u^3 + u = d."""
    mesh = wl.unit_square_mesh(32)
    ue = wl.supercond_exact(mesh.coords[:, 0], mesh.coords[:, 1])
    uD = ue * mesh.dirichlet
    sga = oracle.Problem(mesh, a=None, a_deg=1, kappa=nu, c=("pow", 3.0), c_deg=3, gamma=1.0, sigma=1.0)
    b = sga.load_vector(lambda xx, yy: wl.supercond_source(xx, yy, nu)) * (1 - mesh.dirichlet)
    u_sga, _, _, _ = sga.newton(b, u0=uD, uD=uD, method="sga", rtol=1e-13)
    deg, cs = (2, "lagrange") if space == "p2" else (4, "quad")
    h = P.Handle(mesh, P.make_problem(a=None, a_degree=1, kappa=nu, c=("pow", 2), c_degree=deg, c_space=cs, gamma=1.0,
                                      sigma=1.0, c_product=True),
                 P.default_options(op=P.OP_MATRIX_FREE, newton_rtol=1e-13))
    u = cuda(uD)
    st = h.newton_solve(u, cuda(b + uD))
    torch.cuda.synchronize()
    assert st.status == 0
    assert rel(u.cpu().numpy(), u_sga) <= 1e-11
