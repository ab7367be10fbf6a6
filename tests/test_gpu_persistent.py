"""GPU checks of the persistent (cooperative, grid-barrier) BiCGStab solve against the
graph-captured iteration kernels and the oracle, and of the barrier's bounded wait."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

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


def test_grid_barrier_passes_when_every_block_arrives(P):
    ok, err = P.selftest_grid_barrier(8, 8, 1000.0)
    assert ok == [1] * 8 and err == 0


def test_grid_barrier_wait_runs_out_and_reports(P):
    """Two of four blocks never arrive (a flag nothing sets): the two waiting blocks give up
    after 20 ms, raise the error word, and the context stays usable."""
    ok, err = P.selftest_grid_barrier(4, 2, 20.0)
    assert ok == [0, 0, -1, -1] and err == 1
    ok, err = P.selftest_grid_barrier(4, 4, 1000.0)
    assert ok == [1] * 4 and err == 0


def _setup(P, n, **opt):
    mesh = wl.unit_square_mesh(n)
    orc = oracle.Problem(mesh, a=("pow", 2), a_deg=2)
    h = P.Handle(mesh, P.make_problem(a=("pow", 2), a_degree=2), P.default_options(**opt))
    return mesh, orc, h


@pytest.mark.parametrize("persistent", [1, 0])
def test_bicgstab_persistent_and_graph_solve_the_same_system(P, persistent):
    mesh, orc, h = _setup(P, 40, krylov_persistent=persistent)
    u = wl.random_vector(mesh.n_nodes, 5, 0.5) * (1 - mesh.dirichlet)
    rp, cl = h.pattern()
    vals = torch.empty(h.sizes.jac_nnz, device="cuda", dtype=torch.float64)
    h.jacobian(cuda(u), vals)
    torch.cuda.synchronize()
    J = sp.csr_matrix((vals.cpu().numpy(), cl.cpu().numpy(), rp.cpu().numpy()), shape=(mesh.n_nodes, mesh.n_nodes))
    # the library's Jacobian is the oracle's (checked elementwise elsewhere)
    assert abs(J - orc.jacobian(u)).max() <= 1e-12 * abs(J).max()
    rhs = wl.random_vector(mesh.n_nodes, 7)
    sol = torch.zeros(mesh.n_nodes, device="cuda", dtype=torch.float64)
    its = h.bicgstab(vals, cuda(rhs), sol, rtol=1e-12)
    torch.cuda.synchronize()
    ref = spla.spsolve(J.tocsc(), rhs)
    assert its > 10
    assert rel(sol.cpu().numpy(), ref) <= 1e-9


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("persistent", [1, 0])
def test_newton_parity_both_krylov_drivers(P, prec, persistent):
    mesh, orc, h = _setup(P, 48, krylov_persistent=persistent, newton_rtol=1e-13 if prec == "fp64" else 1e-10,
                          precision=P.PREC_MIXED if prec == "mixed" else P.PREC_FP64)
    b = orc.load_vector(wl.mms_source) * (1 - mesh.dirichlet)
    u_ref, _, _, _ = orc.newton(b, rtol=1e-13)
    u = torch.zeros(mesh.n_nodes, device="cuda", dtype=torch.float64)
    st = h.newton_solve(u, cuda(b))
    torch.cuda.synchronize()
    assert st.status == 0
    assert st.fp64_rescues == 0
    if prec == "fp64":
        assert st.res_final <= 1e-13 * st.res0
        assert rel(u.cpu().numpy(), u_ref) <= 1e-11
    else:
        assert st.res_final <= 1e-10 * st.res0
        assert rel(u.cpu().numpy(), u_ref) <= 1e-6
    # one kernel per BiCGStab solve on the persistent driver
    if persistent:
        assert st.kernel_launches < 20 * st.newton_iters + 10


def test_single_system_grid_solve_with_ragged_tiles(P):
    """The grid-wide persistent solve on 40 401 rows: about 250 row tiles, fewer than the
    resident grid, the last one short; every block sums all partials itself.  The solution of
    J x = b equals a direct solve."""
    mesh, orc, h = _setup(P, 200, krylov_cluster=-1)
    u = wl.random_vector(mesh.n_nodes, 15, 0.5) * (1 - mesh.dirichlet)
    rp, cl = h.pattern()
    vals = torch.empty(h.sizes.jac_nnz, device="cuda", dtype=torch.float64)
    h.jacobian(cuda(u), vals)
    torch.cuda.synchronize()
    J = sp.csr_matrix((vals.cpu().numpy(), cl.cpu().numpy(), rp.cpu().numpy()), shape=(mesh.n_nodes, mesh.n_nodes))
    rhs = wl.random_vector(mesh.n_nodes, 16)
    sol = torch.zeros(mesh.n_nodes, device="cuda", dtype=torch.float64)
    its = h.bicgstab(vals, cuda(rhs), sol, rtol=1e-12)
    torch.cuda.synchronize()
    ref = spla.spsolve(J.tocsc(), rhs)
    assert its > 100
    assert rel(sol.cpu().numpy(), ref) <= 1e-8


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batched_solve_with_many_tiles_per_instance(P, prec):
    """Two instances cut into hundreds of tiles each (the batched solve's per-system sums run
    over many tiles per lane) and a small third one: every instance's Newton solution equals
    the single-system solve of that instance."""
    ns = (150, 190, 12)
    meshes = [wl.unit_square_mesh(n) for n in ns]
    prob = P.make_problem(a=("pow", 2), a_degree=2)
    mixed = prec == "mixed"
    opts = dict(newton_rtol=1e-12 if not mixed else 1e-10, precision=P.PREC_MIXED if mixed else P.PREC_FP64)
    loads = [oracle.Problem(m, a=("pow", 2), a_deg=2).load_vector(wl.mms_source) * (1 - m.dirichlet) for m in meshes]
    hb = P.BatchHandle(meshes, prob, P.default_options(**opts))
    d = hb.scatter(loads)
    u = torch.zeros_like(d)
    st = hb.batch_newton_solve(u, d)
    torch.cuda.synchronize()
    got = hb.gather(u, [m.n_nodes for m in meshes])
    for b, (m, ld) in enumerate(zip(meshes, loads)):
        assert st[b].status == 0, b
        h = P.Handle(m, prob, P.default_options(newton_rtol=1e-12))
        ub = torch.zeros(m.n_nodes, device="cuda", dtype=torch.float64)
        s1 = h.newton_solve(ub, cuda(ld))
        torch.cuda.synchronize()
        assert s1.status == 0
        assert rel(got[b], ub.cpu().numpy()) <= (1e-8 if mixed else 1e-10), b
        h.close()
    hb.close()
