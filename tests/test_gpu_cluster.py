"""GPU checks of the cluster BiCGStab solve (one thread-block cluster, the Krylov vectors in
distributed shared memory): for every cluster size and both precisions (FP64; double-float
vectors with the FP32 operator), the Newton solution equals the oracle's and the grid-wide
persistent solve's (FP64: with the same number of Newton steps)."""
import numpy as np
import pytest

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


@pytest.fixture(scope="module")
def case():
    mesh = wl.unit_square_mesh(40)
    orc = oracle.Problem(mesh, a=("pow", 2.0), a_deg=2)
    b = orc.load_vector(wl.mms_source) * (1 - mesh.dirichlet)
    u_orc, _, _, _ = orc.newton(b, rtol=1e-13)
    return mesh, b, u_orc


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("cluster", [1, 2, 4, 8, 16, 0])
def test_cluster_solve_matches_oracle_and_grid_solve(P, case, cluster, prec):
    mesh, b, u_orc = case
    prob = P.make_problem(a=("pow", 2), a_degree=2)
    mixed = prec == "mixed"
    out = {}
    for name, c in (("cluster", cluster), ("grid", -1)):
        h = P.Handle(mesh, prob, P.default_options(newton_rtol=1e-10 if mixed else 1e-13, krylov_cluster=c,
                                                   precision=P.PREC_MIXED if mixed else P.PREC_FP64))
        u = torch.zeros(mesh.n_nodes, device="cuda", dtype=torch.float64)
        st = h.newton_solve(u, cuda(b))
        torch.cuda.synchronize()
        assert st.status == 0, (name, st.status)
        out[name] = (u.cpu().numpy(), st.newton_iters)
        kernels = {p["name"] for p in h.profile_kernels(u, cuda(b), reps=1)}
        assert ("kry_cluster" in kernels) == (name == "cluster"), kernels
        h.close()
    tol = 1e-8 if mixed else 1e-11
    assert rel(out["cluster"][0], u_orc) <= tol
    assert rel(out["cluster"][0], out["grid"][0]) <= tol
    if not mixed:
        assert out["cluster"][1] == out["grid"][1]


def test_cluster_solve_too_large_falls_back_to_the_grid_solve(P):
    """16 x 3904 rows is the most a cluster holds: a 300 x 300 grid (90 601 rows) uses the
    grid-wide solve even when a cluster is asked for."""
    mesh = wl.unit_square_mesh(300)
    h = P.Handle(mesh, P.make_problem(a=None, a_degree=1), P.default_options(krylov_cluster=16))
    u = torch.zeros(mesh.n_nodes, device="cuda", dtype=torch.float64)
    d = torch.ones(mesh.n_nodes, device="cuda", dtype=torch.float64) * cuda(1.0 - mesh.dirichlet)
    kernels = {p["name"] for p in h.profile_kernels(u, d, reps=1)}
    assert ("kry_window" in kernels or "kry_persistent" in kernels) and "kry_cluster" not in kernels


def test_cluster_solve_adjoint_matches_oracle(P):
    mesh = wl.unit_square_mesh(24)
    orc = oracle.Problem(mesh, a=("pow", 2.0), a_deg=2)
    b = orc.load_vector(wl.mms_source) * (1 - mesh.dirichlet)
    u_orc, _, _, _ = orc.newton(b, rtol=1e-13)
    g = wl.random_vector(mesh.n_nodes, 17) * (1 - mesh.dirichlet)
    lam_orc, _ = orc.adjoint(u_orc, g)
    h = P.Handle(mesh, P.make_problem(a=("pow", 2), a_degree=2), P.default_options(krylov_cluster=4))
    lam = torch.empty(mesh.n_nodes, device="cuda", dtype=torch.float64)
    h.adjoint(cuda(u_orc), cuda(g), lam)
    torch.cuda.synchronize()
    assert rel(lam.cpu().numpy(), lam_orc) <= 1e-10
