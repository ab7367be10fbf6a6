"""GPU checks on high-valence meshes: a centre vertex with 20 or 48 neighbours takes the 32- and
64-column variants of the row kernels (fused, mixed and element-local), whose blocks are smaller
so their shared arrays stay below the static limit.  Residual, Jacobian and the Newton solution
against the oracle."""
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


@pytest.mark.parametrize("op,prec", [("csf", "fp64"), ("csf", "mixed"), ("mf", "fp64")])
@pytest.mark.parametrize("k", [20, 48])
def test_high_valence_parity_and_solve(P, k, op, prec):
    mesh = wl.fan_mesh(k)
    orc = oracle.Problem(mesh, a=("pow", 2.0), a_deg=2, c=("exp",), c_deg=1, gamma=0.5)
    h = P.Handle(mesh, P.make_problem(a=("pow", 2), a_degree=2, c=("exp",), c_degree=1, gamma=0.5),
                 P.default_options(op=P.OP_MATRIX_FREE if op == "mf" else P.OP_CSF, newton_rtol=1e-12,
                                   precision=P.PREC_MIXED if prec == "mixed" else P.PREC_FP64))
    u = wl.random_vector(mesh.n_nodes, 3, 0.7)
    b = np.where(mesh.dirichlet == 0, 1.0, 0.0)
    if prec == "fp64":
        r = torch.empty(mesh.n_nodes, device="cuda", dtype=torch.float64)
        h.residual(cuda(u), cuda(b), r)
        rp, cl = h.pattern()
        vals = torch.empty(h.sizes.jac_nnz, device="cuda", dtype=torch.float64)
        h.jacobian(cuda(u), vals)
        torch.cuda.synchronize()
        assert rel(r.cpu().numpy(), orc.residual(u, b)) <= 1e-12
        A = sp.csr_matrix((vals.cpu().numpy(), cl.cpu().numpy(), rp.cpu().numpy()), shape=(mesh.n_nodes, mesh.n_nodes))
        Ao = orc.jacobian(u)
        assert abs(A - Ao).max() <= 1e-12 * abs(Ao).max()
    u_orc, _, _, _ = orc.newton(b, rtol=1e-13)
    x = torch.zeros(mesh.n_nodes, device="cuda", dtype=torch.float64)
    st = h.newton_solve(x, cuda(b))
    torch.cuda.synchronize()
    assert st.status == 0
    assert rel(x.cpu().numpy(), u_orc) <= (1e-8 if prec == "mixed" else 1e-11)
