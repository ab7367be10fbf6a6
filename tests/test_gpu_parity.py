"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (FP64 path): kernel outputs on identical inputs agree to 1e-12 relative
(2-norm over the vector, or max-norm over the Jacobian values); converged Newton
solutions agree to 1e-11 relative on grids whose condition number keeps the FP64
solution error far below that.  Mixed precision (FP32 operator and Krylov, FP64
residual and update): the solution agrees with the FP64 oracle to 1e-6 relative.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2005_06193_gb300 as P
    return P


def cuda(x, dtype=torch.float64):
    return torch.tensor(np.asarray(x), device="cuda", dtype=dtype)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def gpu_jacobian(h, u):
    rp, cl = h.pattern()
    vals = torch.empty(h.sizes.jac_nnz, device="cuda", dtype=torch.float64)
    h.jacobian(u, vals)
    torch.cuda.synchronize()
    n = h.sizes.jac_rows
    return sp.csr_matrix((vals.cpu().numpy(), cl.cpu().numpy(), rp.cpu().numpy()), shape=(n, n))


def match_w(oc, lc):
    key = lambda c: [tuple(np.round(x, 12)) for x in c]
    lk = {k: i for i, k in enumerate(key(lc))}
    return np.array([lk[k] for k in key(oc)])


CASES = {
    # name: (mesh factory, oracle kwargs, library problem kwargs)
    "u2_p2_2d": (lambda: wl.unit_square_mesh(32), dict(a=("pow", 2.0), a_deg=2), dict(a=("pow", 2), a_degree=2)),
    "u2_p2_ragged": (lambda: wl.unit_square_mesh(13), dict(a=("pow", 2.0), a_deg=2), dict(a=("pow", 2), a_degree=2)),
    "u3_p3_2d": (lambda: wl.unit_square_mesh(17), dict(a=("pow", 3.0), a_deg=3), dict(a=("pow", 3), a_degree=3)),
    "u2_p1_gfem": (lambda: wl.unit_square_mesh(9), dict(a=("pow", 2.0), a_deg=1), dict(a=("pow", 2), a_degree=1)),
    "u2_p2_3d": (lambda: wl.unit_cube_mesh(5), dict(a=("pow", 2.0), a_deg=2), dict(a=("pow", 2), a_degree=2)),
    "bratu_3d": (lambda: wl.unit_cube_mesh(8), dict(a=None, a_deg=1, c=("exp",), c_deg=1, gamma=-2.0),
                 dict(a=None, a_degree=1, c=("exp",), c_degree=1, gamma=-2.0)),
}


def _source(mesh, name):
    if CASES[name][1].get("c") is not None:
        return lambda *x: 0.0 * x[0]
    return wl.mms_source if mesh.dim == 2 else wl.smooth_source_3d


def _setup(P, name, **opt):
    mk, okw, pkw = CASES[name]
    mesh = mk()
    orc = oracle.Problem(mesh, **okw)
    h = P.Handle(mesh, P.make_problem(**pkw), P.default_options(**opt))
    return mesh, orc, h


OPS = ["csf", "mf"]


@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("name", list(CASES))
def test_residual_parity(P, name, op):
    mesh, orc, h = _setup(P, name, op=P.OP_MATRIX_FREE if op == "mf" else P.OP_CSF)
    b = orc.load_vector(_source(mesh, name)) * (1 - mesh.dirichlet)
    for seed, scale in ((1, 1.0), (2, 0.3)):
        u = wl.random_vector(mesh.n_nodes, seed, scale) * (1 - mesh.dirichlet)
        r = torch.empty(mesh.n_nodes, device="cuda", dtype=torch.float64)
        h.residual(cuda(u), cuda(b), r)
        torch.cuda.synchronize()
        ref = orc.residual(u, b)
        assert rel(r.cpu().numpy(), ref) <= 1e-12
    # u = 0: the residual is -b on free rows
    r0 = torch.empty(mesh.n_nodes, device="cuda", dtype=torch.float64)
    h.residual(torch.zeros(mesh.n_nodes, device="cuda", dtype=torch.float64), cuda(b), r0)
    torch.cuda.synchronize()
    assert rel(r0.cpu().numpy(), orc.residual(np.zeros(mesh.n_nodes), b)) <= 1e-12


@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("name", list(CASES))
def test_jacobian_parity(P, name, op):
    mesh, orc, h = _setup(P, name, op=P.OP_MATRIX_FREE if op == "mf" else P.OP_CSF)
    u = wl.random_vector(mesh.n_nodes, 3, 0.8) * (1 - mesh.dirichlet)
    J = gpu_jacobian(h, cuda(u))
    Jo = orc.jacobian(u)
    diff = abs(J - Jo)
    assert diff.max() <= 1e-12 * abs(Jo).max()
    # every stored value belongs to the P1 adjacency; no oracle value outside it is nonzero
    extra = Jo - Jo.multiply(J != 0)
    assert abs(extra).max() <= 1e-13 * abs(Jo).max()


@pytest.mark.parametrize("name", ["u2_p2_2d", "u3_p3_2d", "u2_p2_3d"])
def test_pointwise_parity(P, name):
    mesh, orc, h = _setup(P, name)
    u = wl.random_vector(mesh.n_nodes, 4, 1.0)
    w = torch.empty(h.sizes.n_wa, device="cuda", dtype=torch.float64)
    wp = torch.empty_like(w)
    h.pointwise(cuda(u), w, wp)
    torch.cuda.synchronize()
    ow, owp, _, _ = orc.pointwise(u)
    perm = match_w(orc.space_coords(0), h.w_coords(0))
    assert rel(w.cpu().numpy()[perm], ow) <= 1e-13
    assert rel(wp.cpu().numpy()[perm], owp) <= 1e-13


def test_spmv_and_bicgstab_parity(P):
    mesh, orc, h = _setup(P, "u2_p2_2d")
    u = wl.random_vector(mesh.n_nodes, 5, 0.5) * (1 - mesh.dirichlet)
    J = gpu_jacobian(h, cuda(u))
    vals = cuda(J.data)
    x = wl.random_vector(mesh.n_nodes, 6)
    y = torch.empty(mesh.n_nodes, device="cuda", dtype=torch.float64)
    h.spmv(vals, cuda(x), y)
    torch.cuda.synchronize()
    assert rel(y.cpu().numpy(), J @ x) <= 1e-14
    rhs = wl.random_vector(mesh.n_nodes, 7)
    sol = torch.zeros(mesh.n_nodes, device="cuda", dtype=torch.float64)
    its = h.bicgstab(vals, cuda(rhs), sol, rtol=1e-12)
    ref = spla.spsolve(J.tocsc(), rhs)
    assert its > 10
    assert rel(sol.cpu().numpy(), ref) <= 1e-9
    xo, st, _, _ = oracle.bicgstab(J, rhs, rtol=1e-12)
    assert rel(sol.cpu().numpy(), xo) <= 1e-9


@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("name", ["u2_p2_2d", "u2_p2_ragged", "u3_p3_2d", "u2_p2_3d", "bratu_3d"])
def test_newton_solution_parity_fp64(P, name, op):
    mesh, orc, h = _setup(P, name, newton_rtol=1e-13, op=P.OP_MATRIX_FREE if op == "mf" else P.OP_CSF)
    b = orc.load_vector(_source(mesh, name)) * (1 - mesh.dirichlet)
    u_ref, hist, _, _ = orc.newton(b, rtol=1e-13, solver="lu" if mesh.n_nodes < 20000 else "bicgstab")
    u = torch.zeros(mesh.n_nodes, device="cuda", dtype=torch.float64)
    st = h.newton_solve(u, cuda(b))
    torch.cuda.synchronize()
    assert st.status == 0 and st.res_final <= 1e-13 * st.res0
    if name == "bratu_3d":
        assert u_ref.max() > 0.01
    assert rel(u.cpu().numpy(), u_ref) <= 1e-11


def test_newton_default_tolerance_and_egfem_equals_sga(P):
    """32 x 32, w = u^2 in P2: the GPU EGFEM solution at the default 1e-10 target is the
    SGA (standard Galerkin) solution of the oracle up to that tolerance (Case 1)."""
    mesh, orc, h = _setup(P, "u2_p2_2d")
    b = orc.load_vector(wl.mms_source) * (1 - mesh.dirichlet)
    u = torch.zeros(mesh.n_nodes, device="cuda", dtype=torch.float64)
    st = h.newton_solve(u, cuda(b))
    torch.cuda.synchronize()
    un = u.cpu().numpy()
    assert st.res_final <= 1e-10 * st.res0
    r_sga = orc.residual(un, b, method="sga", form="diff")
    assert np.linalg.norm(r_sga * (1 - mesh.dirichlet)) <= 1.5e-10 * np.linalg.norm(b)
    u_sga, _, _, _ = orc.newton(b, method="sga", rtol=1e-13)
    assert rel(un, u_sga) <= 1e-8


@pytest.mark.parametrize("name", ["u2_p2_2d", "bratu_3d"])
def test_newton_mixed_precision(P, name):
    mesh, orc, h = _setup(P, name, precision=P.PREC_MIXED)
    b = orc.load_vector(_source(mesh, name)) * (1 - mesh.dirichlet)
    u_ref, _, _, _ = orc.newton(b, rtol=1e-13)
    u = torch.zeros(mesh.n_nodes, device="cuda", dtype=torch.float64)
    st = h.newton_solve(u, cuda(b))
    torch.cuda.synchronize()
    un = u.cpu().numpy()
    assert st.status == 0 and st.res_final <= 1e-10 * st.res0
    # the FP64 residual of the oracle confirms the target
    free = 1 - mesh.dirichlet
    r0 = np.linalg.norm(orc.residual(np.zeros(mesh.n_nodes), b, form="diff") * free)
    assert np.linalg.norm(orc.residual(un, b, form="diff") * free) <= 1.5e-10 * r0
    assert rel(un, u_ref) <= 1e-6


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_adjoint_parity(P, prec):
    mesh, orc, h = _setup(P, "u2_p2_ragged", newton_rtol=1e-13, precision=P.PREC_MIXED if prec == "mixed" else P.PREC_FP64)
    b = orc.load_vector(wl.mms_source) * (1 - mesh.dirichlet)
    u_ref, _, _, _ = orc.newton(b, rtol=1e-14)
    ud = wl.adjoint_target()(mesh.coords[:, 0], mesh.coords[:, 1])
    g = (u_ref - ud) * (1 - mesh.dirichlet)
    orc.set_kappa_field(np.ones(orc.nw))
    lam_ref, gk_ref = orc.adjoint(u_ref, g)
    lam = torch.zeros(mesh.n_nodes, device="cuda", dtype=torch.float64)
    gk = torch.zeros(h.sizes.n_wa, device="cuda", dtype=torch.float64)
    h.adjoint(cuda(u_ref), cuda(g), lam, gk)
    torch.cuda.synchronize()
    assert rel(lam.cpu().numpy(), lam_ref) <= 1e-10
    perm = match_w(orc.space_coords(0), h.w_coords(0))
    assert rel(gk.cpu().numpy()[perm], gk_ref) <= 1e-10


def test_load_cellwise_matches_oracle_quadrature(P):
    mesh = wl.unit_square_mesh(32)
    h = P.Handle(mesh, P.make_problem())
    orc = oracle.Problem(mesh, a=("pow", 2.0), a_deg=2)
    f = wl.random_vector(mesh.n_cells, 11)
    d = torch.empty(mesh.n_nodes, device="cuda", dtype=torch.float64)
    h.load_cellwise(cuda(f), d)
    torch.cuda.synchronize()
    ref = orc.load_vector_cellwise(f) * (1 - mesh.dirichlet)
    assert rel(d.cpu().numpy(), ref) <= 1e-13
    lam = wl.random_vector(mesh.n_nodes, 12)
    g = torch.empty(mesh.n_cells, device="cuda", dtype=torch.float64)
    h.load_cellwise_transpose(cuda(lam), g)
    torch.cuda.synchronize()
    # transpose identity: <d(f), lam> = <f, g(lam)>
    assert abs(np.dot(d.cpu().numpy(), lam) - np.dot(f, g.cpu().numpy())) <= 1e-12 * abs(np.dot(f, g.cpu().numpy()))


def test_full_size_1024_residual_on_sampled_rows(P):
    """1024 x 1024 grid (1.05 M P1, 4.2 M P2 nodes): the GPU residual and Jacobian rows
    equal the oracle's on sampled rows (oracle assembles only the cells around them)."""
    n = 1024
    mesh = wl.unit_square_mesh(n)
    h = P.Handle(mesh, P.make_problem(a=("pow", 2), a_degree=2))
    rng = np.random.default_rng(0)
    rows = np.unique(np.concatenate([rng.integers(0, mesh.n_nodes, 300), [0, 1, n, n + 1, n + 2, mesh.n_nodes - 1]]))
    cellmask = np.isin(mesh.cells, rows).any(axis=1)
    orc = oracle.Problem(mesh, a=("pow", 2.0), a_deg=2, cells=np.where(cellmask)[0].astype(np.int32))
    u = wl.random_vector(mesh.n_nodes, 13) * (1 - mesh.dirichlet)
    b = wl.random_vector(mesh.n_nodes, 14, 1e-5) * (1 - mesh.dirichlet)
    r = torch.empty(mesh.n_nodes, device="cuda", dtype=torch.float64)
    h.residual(cuda(u), cuda(b), r)
    J = gpu_jacobian(h, cuda(u))
    torch.cuda.synchronize()
    ref = orc.residual(u, b)
    assert rel(r.cpu().numpy()[rows], ref[rows]) <= 1e-12
    Jo = orc.jacobian(u)
    for i in rows[:60]:
        a, o = J.getrow(i).toarray().ravel(), Jo.getrow(i).toarray().ravel()
        assert np.abs(a - o).max() <= 1e-12 * np.abs(o).max()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batched_newton_matches_single_instance_oracle(P, prec, persistent=1):
    """Four instances of uneven size (w = u^3 in P3 and different sine sources) solved in
    one batched call; each equals the oracle's own Newton solution of that instance."""
    inst = wl.batch_instances(count=4, seed=3, n_lo=6, n_hi=21)
    meshes = [wl.unit_square_mesh(n) for n, _ in inst]
    loads, refs = [], []
    for (n, src), mesh in zip(inst, meshes):
        orc = oracle.Problem(mesh, a=("pow", 3.0), a_deg=3)
        b = orc.load_vector(src) * (1 - mesh.dirichlet)
        u_ref, _, _, _ = orc.newton(b, rtol=1e-13)
        loads.append(b)
        refs.append(u_ref)
    opts = P.default_options(newton_rtol=1e-13 if prec == "fp64" else 1e-10,
                             precision=P.PREC_MIXED if prec == "mixed" else P.PREC_FP64, krylov_persistent=persistent)
    h = P.BatchHandle(meshes, P.make_problem(a=("pow", 3), a_degree=3), opts)
    d = h.scatter(loads)
    u = torch.zeros_like(d)
    stats = h.batch_newton_solve(u, d)
    torch.cuda.synchronize()
    sols = h.gather(u, [m.n_nodes for m in meshes])
    for b, (sol, ref) in enumerate(zip(sols, refs)):
        assert stats[b].status == 0
        assert rel(sol, ref) <= (1e-11 if prec == "fp64" else 1e-6), b


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batched_newton_graph_driver(P, prec):
    """The same batch through the graph-captured iteration kernels (krylov_persistent = 0)."""
    test_batched_newton_matches_single_instance_oracle(P, prec, persistent=0)


def _adjoint_setup(P, n, grid, thetas, prec="fp64", rtol=1e-13):
    mesh = wl.unit_square_mesh(n)
    pc = wl.param_cell_of_cells(mesh, grid)
    ud = wl.adjoint_target()(mesh.coords[:, 0], mesh.coords[:, 1])
    opts = P.default_options(newton_rtol=rtol, precision=P.PREC_MIXED if prec == "mixed" else P.PREC_FP64)
    return mesh, pc, ud, opts


def _objective(P, h, theta, pc, ud, free, kappa=None):
    from paper_2005_06193_gb300 import autograd as ag
    f_cell = theta.reshape(-1)[pc]
    d = ag.load_cellwise(f_cell, h)
    u = ag.newton_solve(d, kappa, h)
    return 0.5 * torch.sum(((u - ud) * free) ** 2), u


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_autograd_adjoint_matches_central_differences_and_oracle(P, prec):
    """Gradient of j = 0.5 ||u - u_d||^2 with respect to a 4 x 4 piecewise-constant source
    theta and the W-space coefficient kappa, through torch.autograd and the CUDA adjoint,
    against central differences (h = 1e-6) of FP64 re-solves (1e-5 relative + 1e-9 absolute:
    the re-solves' own 1e-14 tolerance bounds the difference quotients to ~2e-10 absolute) and
    against the oracle's FP64 adjoint at the same solution (1e-10 relative)."""
    mesh, pc, ud_np, opts = _adjoint_setup(P, 16, 4, None, prec)
    h = P.Handle(mesh, P.make_problem(a=("pow", 2), a_degree=2), opts)
    hf = P.Handle(mesh, P.make_problem(a=("pow", 2), a_degree=2), P.default_options(newton_rtol=1e-14))
    free = cuda(1.0 - mesh.dirichlet)
    ud = cuda(ud_np)
    pc_t = torch.tensor(pc, device="cuda", dtype=torch.int64)
    theta = cuda(wl.adjoint_theta(7, 4)).requires_grad_(True)
    kappa = torch.ones(h.sizes.n_wa, device="cuda", dtype=torch.float64, requires_grad=True)
    J, u = _objective(P, h, theta, pc_t, ud, free, kappa)
    J.backward()
    gt, gk = theta.grad.detach().cpu().numpy().ravel(), kappa.grad.detach().cpu().numpy()

    def J_at(th, ka):
        with torch.no_grad():
            return float(_objective(P, hf, th, pc_t, ud, free, ka)[0])

    eps = 1e-6
    for p in (0, 5, 10, 15):
        e = torch.zeros(16, device="cuda", dtype=torch.float64)
        e[p] = eps
        th0 = theta.detach().reshape(-1)
        fd = (J_at((th0 + e).reshape(4, 4), kappa.detach()) - J_at((th0 - e).reshape(4, 4), kappa.detach())) / (2 * eps)
        assert abs(fd - gt[p]) <= 1e-5 * abs(gt[p]) + 1e-9, (p, fd, gt[p])
    for m in (100, 400, 700):
        e = torch.zeros_like(kappa)
        e[m] = eps
        fd = (J_at(theta.detach(), kappa.detach() + e) - J_at(theta.detach(), kappa.detach() - e)) / (2 * eps)
        assert abs(fd - gk[m]) <= 1e-5 * abs(gk[m]) + 1e-9, (m, fd, gk[m])
    # oracle adjoint at the GPU solution: dj/db = lambda, dj/df_K = sum_i lambda_i int_K phi_i
    orc = oracle.Problem(mesh, a=("pow", 2.0), a_deg=2)
    un = u.detach().cpu().numpy()
    g = (un - ud_np) * (1 - mesh.dirichlet)
    orc.set_kappa_field(np.ones(orc.nw))
    lam, gk_ref = orc.adjoint(un, g)
    gf = np.zeros(mesh.n_cells)
    for c in range(mesh.n_cells):
        e = np.zeros(mesh.n_cells)
        e[c] = 1.0
        gf[c] = np.dot(orc.load_vector_cellwise(e) * (1 - mesh.dirichlet), lam)
    gt_ref = np.bincount(pc, weights=gf, minlength=16)
    assert rel(gt, gt_ref) <= (1e-10 if prec == "fp64" else 1e-7)
    perm = match_w(orc.space_coords(0), h.w_coords(0))
    assert rel(gk[perm], gk_ref) <= (1e-10 if prec == "fp64" else 1e-7)


def test_autograd_interleaved_forwards_use_their_own_kappa(P):
    """Two forwards on ONE handle with different kappa fields, then both backwards (the
    second first): each gradient equals the gradient from a handle that saw only its own
    forward (1e-12 relative).  A forward with kappa=None after a kappa field runs with the
    handle's constant kappa again."""
    mesh, pc, ud_np, opts = _adjoint_setup(P, 12, 4, None)
    prob = P.make_problem(a=("pow", 2), a_degree=2)
    h = P.Handle(mesh, prob, opts)
    free, ud = cuda(1.0 - mesh.dirichlet), cuda(ud_np)
    pc_t = torch.tensor(pc, device="cuda", dtype=torch.int64)
    theta0 = cuda(wl.adjoint_theta(3, 4))
    kappas = [1.0 + 0.5 * torch.rand(h.sizes.n_wa, device="cuda", dtype=torch.float64, generator=torch.Generator(
        device="cuda").manual_seed(s)) for s in (1, 2)]

    def grads(handle, ka):
        th = theta0.clone().requires_grad_(True)
        k = ka.clone().requires_grad_(True)
        J, _ = _objective(P, handle, th, pc_t, ud, free, k)
        return J, th, k

    runs = [grads(h, ka) for ka in kappas]          # both forwards first
    for J, _, _ in reversed(runs):                  # then the backwards, last forward first
        J.backward()
    for (J, th, k), ka in zip(runs, kappas):
        hs = P.Handle(mesh, prob, opts)
        Js, ths, ks = grads(hs, ka)
        Js.backward()
        assert rel(th.grad.cpu().numpy(), ths.grad.cpu().numpy()) <= 1e-12
        assert rel(k.grad.cpu().numpy(), ks.grad.cpu().numpy()) <= 1e-12
        hs.close()
    # kappa=None after a field: the constant kappa (= 1) again, as on a fresh handle
    from paper_2005_06193_gb300 import autograd as ag
    d = ag.load_cellwise(theta0.reshape(-1)[pc_t], h)
    u_none = ag.newton_solve(d, None, h)
    hf = P.Handle(mesh, prob, opts)
    u_fresh = ag.newton_solve(ag.load_cellwise(theta0.reshape(-1)[pc_t], hf), None, hf)
    assert rel(u_none.detach().cpu().numpy(), u_fresh.detach().cpu().numpy()) <= 1e-12
    h.close()
    hf.close()


def test_batched_adjoint_gradients_equal_single_instance(P):
    """Three instances on one mesh with different theta: the batched forward solve and the
    block-diagonal adjoint give each instance the gradient of its own single solve."""
    from paper_2005_06193_gb300 import autograd as ag
    n, grid = 12, 4
    mesh = wl.unit_square_mesh(n)
    pc = torch.tensor(wl.param_cell_of_cells(mesh, grid), device="cuda", dtype=torch.int64)
    ud = cuda(wl.adjoint_target()(mesh.coords[:, 0], mesh.coords[:, 1]))
    free = cuda(1.0 - mesh.dirichlet)
    prob = P.make_problem(a=("pow", 2), a_degree=2)
    opts = P.default_options(newton_rtol=1e-13)
    hb = P.BatchHandle([mesh] * 3, prob, opts)
    thetas = [cuda(wl.adjoint_theta(b, grid)).requires_grad_(True) for b in range(3)]
    off = hb.offsets
    # batch: cell sources concatenated in instance order (the union keeps each mesh's cells)
    f_all = torch.cat([t.reshape(-1)[pc] for t in thetas])
    d = ag.load_cellwise(f_all, hb)
    u = ag.newton_solve(d, None, hb)
    J = sum(0.5 * torch.sum(((u[off[b]:off[b] + mesh.n_nodes] - ud) * free) ** 2) for b in range(3))
    J.backward()
    hs = P.Handle(mesh, prob, opts)
    for b in range(3):
        t = thetas[b].detach().clone().requires_grad_(True)
        Jb, _ = _objective(P, hs, t, pc, ud, free)
        Jb.backward()
        assert rel(thetas[b].grad.cpu().numpy(), t.grad.cpu().numpy()) <= 1e-9, b


def test_bratu_64_cube_mixed_precision_full_size(P):
    """64^3 cube, 6 Kuhn tetrahedra per cube (274,625 nodes, 1,572,864 tets), Bratu
    -lap u = 2 e^u with e^u interpolated in P1: the mixed solve (FP32 operator and Krylov,
    FP64 residual) reaches the 1e-10 FP64 residual target, its residual rows equal the
    oracle's on sampled rows, and it agrees with the FP64 solve to 1e-6."""
    mesh = wl.unit_cube_mesh(64)
    prob = P.make_problem(a=None, a_degree=1, c=("exp",), c_degree=1, gamma=-2.0)
    d = torch.zeros(mesh.n_nodes, device="cuda", dtype=torch.float64)
    sols = {}
    for prec in ("fp64", "mixed"):
        h = P.Handle(mesh, prob, P.default_options(precision=P.PREC_MIXED if prec == "mixed" else P.PREC_FP64))
        u = torch.zeros_like(d)
        st = h.newton_solve(u, d)
        torch.cuda.synchronize()
        assert st.status == 0 and st.res_final <= 1e-10 * st.res0
        sols[prec] = (u.cpu().numpy(), st, h)
    um, stm, hm = sols["mixed"]
    uf = sols["fp64"][0]
    # a Kuhn mesh's tiles have halos of about nine tiles: the five-barrier kernel is used
    assert "kry_persistent" in {p["name"] for p in sols["fp64"][2].profile_kernels(cuda(uf), d, reps=1)}
    err = rel(um, uf)
    assert err <= 1e-6, err
    assert um.max() > 0.05
    rng = np.random.default_rng(1)
    rows = np.unique(rng.integers(0, mesh.n_nodes, 150))
    cellmask = np.isin(mesh.cells, rows).any(axis=1)
    orc = oracle.Problem(mesh, a=None, a_deg=1, c=("exp",), c_deg=1, gamma=-2.0, qpts=3,
                         cells=np.where(cellmask)[0].astype(np.int32))
    r = torch.empty_like(d)
    hm.residual(cuda(um), d, r)
    torch.cuda.synchronize()
    ro = orc.residual(um, np.zeros(mesh.n_nodes), form="diff")
    rg = r.cpu().numpy()
    scale = stm.res0 / np.sqrt(mesh.n_nodes)
    assert np.abs(rg[rows] - ro[rows]).max() <= 1e-12 * max(scale, np.abs(ro[rows]).max())

