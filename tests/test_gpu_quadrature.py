"""GPU checks of the quadrature spaces I_k (Sec. 3.1, Case 3) in the element-local operator:
residual and Jacobian against the oracle's EGFEM with the same spaces (which equals the standard
Galerkin approach under that rule), and the quadratic example's Newton solution (Sec. 5,
-lap u + u^2 = d with W_c = I_3) against the oracle's I_3 and P2 solutions."""
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


CASES = [(2, k) for k in (1, 2, 3, 4)] + [(3, k) for k in (1, 2, 3)]


def _pair(P, dim, k, **opt):
    mesh = wl.unit_square_mesh(11) if dim == 2 else wl.unit_cube_mesh(4)
    orc = oracle.Problem(mesh, a=("pow", 2.0), a_deg=k, a_space="quad", c=("exp",), c_deg=k, c_space="quad",
                         gamma=0.6, kappa=0.8)
    h = P.Handle(mesh, P.make_problem(a=("pow", 2), a_degree=k, a_space="quad", c=("exp",), c_degree=k,
                                      c_space="quad", gamma=0.6, kappa=0.8),
                 P.default_options(op=P.OP_MATRIX_FREE, **opt))
    return mesh, orc, h


@pytest.mark.parametrize("dim,k", CASES)
def test_quadrature_space_residual_and_jacobian_parity(P, dim, k):
    mesh, orc, h = _pair(P, dim, k)
    assert h.sizes.n_wa == h.sizes.n_wc == orc.nw
    b = wl.random_vector(mesh.n_nodes, 5) * (1 - mesh.dirichlet)
    u = wl.random_vector(mesh.n_nodes, 6, 0.8)
    r = torch.empty(mesh.n_nodes, device="cuda", dtype=torch.float64)
    h.residual(cuda(u), cuda(b), r)
    torch.cuda.synchronize()
    assert rel(r.cpu().numpy(), orc.residual(u, b)) <= 1e-12
    rp, cl = h.pattern()
    vals = torch.empty(h.sizes.jac_nnz, device="cuda", dtype=torch.float64)
    h.jacobian(cuda(u), vals)
    torch.cuda.synchronize()
    A = sp.csr_matrix((vals.cpu().numpy(), cl.cpu().numpy(), rp.cpu().numpy()), shape=(mesh.n_nodes, mesh.n_nodes))
    Ao = orc.jacobian(u)
    assert abs(A - Ao).max() <= 1e-12 * abs(Ao).max()


def test_quadrature_space_picard_matrix_parity(P):
    mesh, orc, h = _pair(P, 2, 4, iteration=P.ITER_PICARD)
    u = wl.random_vector(mesh.n_nodes, 7, 0.8)
    rp, cl = h.pattern()
    vals = torch.empty(h.sizes.jac_nnz, device="cuda", dtype=torch.float64)
    h.jacobian(cuda(u), vals)
    torch.cuda.synchronize()
    A = sp.csr_matrix((vals.cpu().numpy(), cl.cpu().numpy(), rp.cpu().numpy()), shape=(mesh.n_nodes, mesh.n_nodes))
    Ao = orc.jacobian(u, method="picard")
    assert abs(A - Ao).max() <= 1e-12 * abs(Ao).max()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_quadratic_example_newton_with_i3(P, prec):
    """-lap u + u^2 = d, u = x y (x + y) on the boundary and manufactured d (Sec. 5): the
    library's solution with W_c = I_3 equals the oracle's with I_3 and with P2 (both represent
    the u^2 term exactly), and is O(h^2) from the exact solution."""
    mesh = wl.unit_square_mesh(32)
    x, y = mesh.coords[:, 0], mesh.coords[:, 1]
    ue = wl.minsurf_exact(x, y)
    uD = ue * mesh.dirichlet
    kw = dict(a=None, a_deg=1, kappa=1.0, c=("pow", 2.0), gamma=1.0)
    o3 = oracle.Problem(mesh, c_deg=3, c_space="quad", **kw)
    o2 = oracle.Problem(mesh, c_deg=2, **kw)
    b = o2.load_vector(wl.quadratic_source) * (1 - mesh.dirichlet)
    u3, _, _, _ = o3.newton(b, u0=uD, uD=uD, rtol=1e-13)
    u2, _, _, _ = o2.newton(b, u0=uD, uD=uD, rtol=1e-13)
    assert rel(u3, u2) <= 1e-12
    mixed = prec == "mixed"
    h = P.Handle(mesh, P.make_problem(a=None, a_degree=1, kappa=1.0, c=("pow", 2), c_degree=3, c_space="quad", gamma=1.0),
                 P.default_options(op=P.OP_MATRIX_FREE, newton_rtol=1e-10 if mixed else 1e-13,
                                   precision=P.PREC_MIXED if mixed else P.PREC_FP64))
    u = cuda(uD)
    st = h.newton_solve(u, cuda(b + uD))
    torch.cuda.synchronize()
    assert st.status == 0
    un = u.cpu().numpy()
    tol = 1e-8 if mixed else 1e-11
    assert rel(un, u3) <= tol and rel(un, u2) <= tol
    assert np.sqrt(np.mean((un - ue) ** 2)) <= 1e-4


def test_gradient_coefficient_on_i1_equals_p0(P):
    """I_1 and P0 carry the same cell gradient: the minimal-surface residual agrees (Sec. 5)."""
    mesh = wl.unit_square_mesh(12)
    u = wl.random_vector(mesh.n_nodes, 9, 0.7)
    b = wl.random_vector(mesh.n_nodes, 10) * (1 - mesh.dirichlet)
    out = []
    for deg, space in ((0, "lagrange"), (1, "quad")):
        h = P.Handle(mesh, P.make_problem(a=("gradpow", -0.5, 1.0), a_degree=deg, a_space=space, kappa=0.0),
                     P.default_options(op=P.OP_MATRIX_FREE))
        r = torch.empty(mesh.n_nodes, device="cuda", dtype=torch.float64)
        h.residual(cuda(u), cuda(b), r)
        torch.cuda.synchronize()
        out.append(r.cpu().numpy())
    assert np.abs(out[0] - out[1]).max() <= 1e-14 * np.abs(out[0]).max()
