"""GPU checks of the graph-resident Newton loop (a conditional WHILE node in one CUDA graph;
option newton_graph), batched and for one system: with the graph required (newton_graph = 2)
every solution equals the oracle's and the host loop's, with the same Newton step counts (for
one system the same Krylov counts step by step); a second call reuses the graph; Picard runs in
it too; and steps that fail the sufficient-decrease test are halved inside the graph exactly as
the host loop halves them."""
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


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def batch():
    inst = wl.batch_instances(count=5, seed=7, n_lo=6, n_hi=24)
    meshes = [wl.unit_square_mesh(n) for n, _ in inst]
    loads, refs = [], []
    for (n, src), mesh in zip(inst, meshes):
        orc = oracle.Problem(mesh, a=("pow", 3.0), a_deg=3)
        b = orc.load_vector(src) * (1 - mesh.dirichlet)
        u_ref, _, _, _ = orc.newton(b, rtol=1e-13)
        loads.append(b)
        refs.append(u_ref)
    return meshes, loads, refs


def _solve(P, meshes, loads, graph, prec, **kw):
    opts = P.default_options(newton_graph=graph, newton_rtol=1e-13 if prec == "fp64" else 1e-10,
                             precision=P.PREC_MIXED if prec == "mixed" else P.PREC_FP64, **kw)
    h = P.BatchHandle(meshes, P.make_problem(a=("pow", 3), a_degree=3), opts)
    d = h.scatter(loads)
    u = torch.zeros_like(d)
    stats = h.batch_newton_solve(u, d)
    torch.cuda.synchronize()
    return h, d, u, stats


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_graph_newton_matches_host_loop_and_oracle(P, batch, prec):
    meshes, loads, refs = batch
    sizes = [m.n_nodes for m in meshes]
    hg, dg, ug, sg = _solve(P, meshes, loads, 2, prec)
    hh, dh, uh, sh = _solve(P, meshes, loads, 0, prec)
    tol = 1e-11 if prec == "fp64" else 1e-6
    for b, (x, y, ref) in enumerate(zip(hg.gather(ug, sizes), hh.gather(uh, sizes), refs)):
        assert sg[b].status == 0 and sh[b].status == 0, b
        assert rel(x, ref) <= tol and rel(y, ref) <= tol, b
        assert sg[b].newton_iters == sh[b].newton_iters, b
        for s_ in (sg[b], sh[b]):   # every Krylov iteration is counted once, in its step
            assert s_.krylov_iters == sum(s_.krylov_hist[:s_.newton_iters]), b
    # a second call with the same tensors runs the captured graph again
    ug.zero_()
    sg2 = hg.batch_newton_solve(ug, dg)
    torch.cuda.synchronize()
    for b, (x, ref) in enumerate(zip(hg.gather(ug, sizes), refs)):
        assert sg2[b].status == 0 and rel(x, ref) <= tol, b


def test_graph_picard_matches_oracle(P, batch):
    meshes, loads, refs = batch
    h, d, u, st = _solve(P, meshes, loads, 2, "fp64", iteration=P.ITER_PICARD, newton_maxit=300)
    hn, dn, un, sn = _solve(P, meshes, loads, 2, "fp64", eta_max=1e-2)   # Newton with Picard's forcing cap
    for b, (x, ref) in enumerate(zip(h.gather(u, [m.n_nodes for m in meshes]), refs)):
        assert st[b].status == 0, b
        assert st[b].newton_iters >= sn[b].newton_iters, b   # linear convergence: no fewer steps
        assert rel(x, ref) <= 1e-10, b


@pytest.mark.parametrize("graph", [2, 0])
def test_batched_steps_that_need_damping(P, graph):
    """Minimal surface from the boundary data (full Newton steps overshoot there): the step
    halving (in the graph, or in the host loop) brings every instance to the oracle's discrete
    solution."""
    meshes = [wl.unit_square_mesh(n) for n in (24, 32)]
    loads, refs, starts = [], [], []
    for mesh in meshes:
        orc = oracle.Problem(mesh, a=("gradpow", -0.5, 1.0), a_deg=0, kappa=0.0)
        x, y = mesh.coords[:, 0], mesh.coords[:, 1]
        ue = wl.minsurf_exact(x, y)
        uD = ue * mesh.dirichlet
        b = orc.load_vector(wl.minsurf_source) * (1 - mesh.dirichlet)
        u_ref, _, _, _ = orc.newton(b, u0=ue + 0.2 * np.sin(np.pi * x) * np.sin(np.pi * y), uD=uD, rtol=1e-12)
        loads.append(b + uD)
        refs.append(u_ref)
        starts.append(uD)
    h = P.BatchHandle(meshes, P.make_problem(a=("gradpow", -0.5, 1.0), a_degree=0, kappa=0.0),
                      P.default_options(op=P.OP_MATRIX_FREE, newton_graph=graph, newton_rtol=1e-12))
    d = h.scatter(loads)
    u = h.scatter(starts)
    st = h.batch_newton_solve(u, d)
    torch.cuda.synchronize()
    for b, (x, ref) in enumerate(zip(h.gather(u, [m.n_nodes for m in meshes]), refs)):
        assert st[b].status == 0, b
        assert rel(x, ref) <= 1e-10, b
        assert st[b].krylov_iters == sum(st[b].krylov_hist[:st[b].newton_iters]), b


@pytest.mark.parametrize("prec,cluster", [("fp64", 0), ("fp64", -1), ("mixed", 0), ("mixed", -1)])
def test_single_system_graph_newton_matches_host_loop(P, prec, cluster):
    """egfem_newton_solve with the graph loop required equals the host loop (the same Newton
    steps with the same Krylov counts and residual norms: both run the same kernels) and the
    oracle, for the cluster and the grid-wide BiCGStab and both precisions.  From u = 0 the
    first full step of this problem fails the sufficient-decrease test, so the halving runs
    too."""
    mesh = wl.unit_square_mesh(40)
    orc = oracle.Problem(mesh, a=("pow", 2.0), a_deg=2)
    b = orc.load_vector(wl.mms_source) * (1 - mesh.dirichlet)
    u_ref, _, _, _ = orc.newton(b, rtol=1e-13)
    mixed = prec == "mixed"
    out = []
    for graph in (2, 0):
        h = P.Handle(mesh, P.make_problem(a=("pow", 2), a_degree=2),
                     P.default_options(newton_graph=graph, krylov_cluster=cluster, newton_rtol=1e-10 if mixed else 1e-13,
                                       precision=P.PREC_MIXED if mixed else P.PREC_FP64))
        u = torch.zeros(mesh.n_nodes, device="cuda", dtype=torch.float64)
        d = torch.tensor(b, device="cuda", dtype=torch.float64)
        st = h.newton_solve(u, d)
        u2 = torch.zeros_like(u)
        st2 = h.newton_solve(u2, d) if graph == 2 else st   # a second call reuses the captured graph
        torch.cuda.synchronize()
        assert st.status == 0 and st2.status == 0
        out.append((u.cpu().numpy(), st))
        assert st.krylov_iters == sum(st.krylov_hist[:st.newton_iters])
        if graph == 2:
            assert np.array_equal(u.cpu().numpy(), u2.cpu().numpy())
        h.close()
    tol = 1e-8 if mixed else 1e-11
    assert rel(out[0][0], u_ref) <= tol and rel(out[1][0], u_ref) <= tol
    sg, sh = out[0][1], out[1][1]
    k = sg.newton_iters
    assert k == sh.newton_iters and sg.krylov_iters == sh.krylov_iters
    assert list(sg.krylov_hist[:k]) == list(sh.krylov_hist[:k])
    assert np.allclose(sg.res_hist[:k], sh.res_hist[:k], rtol=1e-12, atol=0.0)
    assert sg.fp64_rescues == sh.fp64_rescues


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_single_system_graph_damped_steps_match_host_loop(P, prec):
    """Minimal surface from the boundary data: the graph's halvings reproduce the host loop's
    iteration step by step, and both reach the oracle's discrete solution."""
    mesh = wl.unit_square_mesh(32)
    orc = oracle.Problem(mesh, a=("gradpow", -0.5, 1.0), a_deg=0, kappa=0.0)
    x, y = mesh.coords[:, 0], mesh.coords[:, 1]
    ue = wl.minsurf_exact(x, y)
    uD = ue * mesh.dirichlet
    b = orc.load_vector(wl.minsurf_source) * (1 - mesh.dirichlet)
    u_ref, _, _, _ = orc.newton(b, u0=ue + 0.2 * np.sin(np.pi * x) * np.sin(np.pi * y), uD=uD, rtol=1e-12)
    mixed = prec == "mixed"
    res = []
    for graph in (2, 0):
        h = P.Handle(mesh, P.make_problem(a=("gradpow", -0.5, 1.0), a_degree=0, kappa=0.0),
                     P.default_options(op=P.OP_MATRIX_FREE, newton_graph=graph, newton_rtol=1e-10 if mixed else 1e-12,
                                       precision=P.PREC_MIXED if mixed else P.PREC_FP64))
        u = torch.tensor(uD, device="cuda", dtype=torch.float64)
        st = h.newton_solve(u, torch.tensor(b + uD, device="cuda", dtype=torch.float64))
        torch.cuda.synchronize()
        assert st.status == 0
        assert rel(u.cpu().numpy(), u_ref) <= (1e-8 if mixed else 1e-10)
        assert st.krylov_iters == sum(st.krylov_hist[:st.newton_iters])
        res.append(st)
        h.close()
    k = res[0].newton_iters
    assert k == res[1].newton_iters and list(res[0].krylov_hist[:k]) == list(res[1].krylov_hist[:k])
