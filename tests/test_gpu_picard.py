"""GPU checks of the Picard iteration (Sec. 4, Example 4.1): the frozen-coefficient matrix
T .2 a(u) against the oracle's, and Picard solutions against the oracle's Picard and Newton
solutions (one discrete solution)."""
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


@pytest.mark.parametrize("op", ["csf", "mf"])
def test_picard_matrix_parity(P, op):
    mesh = wl.unit_square_mesh(13)
    orc = oracle.Problem(mesh, a=("pow", 2.0), a_deg=2)
    h = P.Handle(mesh, P.make_problem(a=("pow", 2), a_degree=2),
                 P.default_options(iteration=P.ITER_PICARD, op=P.OP_MATRIX_FREE if op == "mf" else P.OP_CSF))
    u = wl.random_vector(mesh.n_nodes, 21, 0.6) * (1 - mesh.dirichlet)
    rp, cl = h.pattern()
    vals = torch.empty(h.sizes.jac_nnz, device="cuda", dtype=torch.float64)
    h.jacobian(cuda(u), vals)
    torch.cuda.synchronize()
    A = sp.csr_matrix((vals.cpu().numpy(), cl.cpu().numpy(), rp.cpu().numpy()), shape=(mesh.n_nodes, mesh.n_nodes))
    Ao = orc.jacobian(u, method="picard")
    assert abs(A - Ao).max() <= 1e-12 * abs(Ao).max()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_picard_solution_equals_newton_and_oracle(P, prec):
    mesh = wl.unit_square_mesh(24)
    orc = oracle.Problem(mesh, a=("pow", 2.0), a_deg=2)
    b = orc.load_vector(wl.mms_source) * (1 - mesh.dirichlet)
    u_pic, hist_pic, _, _ = orc.newton(b, rtol=1e-13, iteration="picard", maxit=200)
    u_new, _, _, _ = orc.newton(b, rtol=1e-13)
    assert rel(u_pic, u_new) <= 1e-11
    opts = P.default_options(iteration=P.ITER_PICARD, newton_maxit=200,
                             newton_rtol=1e-13 if prec == "fp64" else 1e-10,
                             precision=P.PREC_MIXED if prec == "mixed" else P.PREC_FP64)
    h = P.Handle(mesh, P.make_problem(a=("pow", 2), a_degree=2), opts)
    u = torch.zeros(mesh.n_nodes, device="cuda", dtype=torch.float64)
    st = h.newton_solve(u, cuda(b))
    torch.cuda.synchronize()
    assert st.status == 0
    assert st.newton_iters > 5                     # linear convergence: many more steps than Newton
    tol = 1e-11 if prec == "fp64" else 1e-6
    assert rel(u.cpu().numpy(), u_pic) <= tol
    assert rel(u.cpu().numpy(), u_new) <= tol


def test_picard_bratu_reaction_on_the_right_hand_side(P):
    """Bratu (GFEM, exp in P1): Picard keeps the reaction explicit and reaches Newton's solution."""
    mesh = wl.unit_cube_mesh(5)
    orc = oracle.Problem(mesh, a=None, a_deg=1, c=("exp",), c_deg=1, gamma=-2.0)
    b = np.zeros(mesh.n_nodes)
    u_new, _, _, _ = orc.newton(b, rtol=1e-13)
    h = P.Handle(mesh, P.make_problem(a=None, a_degree=1, c=("exp",), c_degree=1, gamma=-2.0),
                 P.default_options(iteration=P.ITER_PICARD, newton_maxit=200, newton_rtol=1e-13))
    u = torch.zeros(mesh.n_nodes, device="cuda", dtype=torch.float64)
    st = h.newton_solve(u, cuda(b))
    torch.cuda.synchronize()
    assert st.status == 0
    assert rel(u.cpu().numpy(), u_new) <= 1e-11
