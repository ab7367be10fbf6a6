"""GPU edge cases: a zero source (the solve ends before its first step), meshes with no or one
free node, the smallest ragged sizes (far fewer rows than one 32-row slice), and a batch that
mixes such tiny instances with larger ones -- each against the oracle, for both Krylov drivers
and both precisions."""
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


DRIVERS = [("fp64", 0), ("fp64", -1), ("mixed", 0)]   # (precision, krylov_cluster: 0 auto, -1 grid)


def _opts(P, prec, cluster, **kw):
    return P.default_options(precision=P.PREC_MIXED if prec == "mixed" else P.PREC_FP64, krylov_cluster=cluster, **kw)


@pytest.mark.parametrize("prec,cluster", DRIVERS)
def test_zero_source_returns_zero_without_a_step(P, prec, cluster):
    mesh = wl.unit_square_mesh(12)
    h = P.Handle(mesh, P.make_problem(a=("pow", 2), a_degree=2), _opts(P, prec, cluster))
    u = torch.zeros(mesh.n_nodes, device="cuda", dtype=torch.float64)
    st = h.newton_solve(u, torch.zeros_like(u))
    torch.cuda.synchronize()
    assert st.status == 0 and st.newton_iters == 0
    assert float(torch.abs(u).max()) == 0.0


@pytest.mark.parametrize("prec,cluster", DRIVERS)
@pytest.mark.parametrize("n", [1, 2, 3])
def test_tiny_meshes_match_oracle(P, n, prec, cluster):
    """n = 1: every node on the boundary (the solve only imposes the boundary data); n = 2: one
    free node; n = 3: four.  Boundary data u_D = x y (x + y), the quadratic example's source."""
    mesh = wl.unit_square_mesh(n)
    x, y = mesh.coords[:, 0], mesh.coords[:, 1]
    uD = wl.minsurf_exact(x, y) * mesh.dirichlet
    orc = oracle.Problem(mesh, a=("pow", 2.0), a_deg=2)
    b = orc.load_vector(wl.quadratic_source) * (1 - mesh.dirichlet)
    u_orc, _, _, _ = orc.newton(b, u0=uD, uD=uD, rtol=1e-13)
    h = P.Handle(mesh, P.make_problem(a=("pow", 2), a_degree=2),
                 _opts(P, prec, cluster, newton_rtol=1e-10 if prec == "mixed" else 1e-13))
    u = cuda(uD)
    st = h.newton_solve(u, cuda(b + uD))
    torch.cuda.synchronize()
    assert st.status == 0
    assert rel(u.cpu().numpy(), u_orc) <= (1e-8 if prec == "mixed" else 1e-11)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_with_tiny_and_larger_instances(P, prec):
    sizes = [1, 9, 2, 17, 3]
    meshes = [wl.unit_square_mesh(n) for n in sizes]
    loads, refs = [], []
    for mesh in meshes:
        orc = oracle.Problem(mesh, a=("pow", 2.0), a_deg=2)
        b = orc.load_vector(wl.mms_source) * (1 - mesh.dirichlet)
        u_ref, _, _, _ = orc.newton(b, rtol=1e-13)
        loads.append(b)
        refs.append(u_ref)
    h = P.BatchHandle(meshes, P.make_problem(a=("pow", 2), a_degree=2),
                      _opts(P, prec, 0, newton_rtol=1e-10 if prec == "mixed" else 1e-13))
    d = h.scatter(loads)
    u = torch.zeros_like(d)
    stats = h.batch_newton_solve(u, d)
    torch.cuda.synchronize()
    for b, (sol, ref) in enumerate(zip(h.gather(u, [m.n_nodes for m in meshes]), refs)):
        assert stats[b].status == 0, b
        if np.linalg.norm(ref) == 0.0:
            assert np.abs(sol).max() == 0.0
        else:
            assert rel(sol, ref) <= (1e-8 if prec == "mixed" else 1e-11), b
