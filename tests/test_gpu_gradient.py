"""GPU checks of the gradient coefficient a = kappa + scale (shift + ||grad u||^2)^q with a P0
W space (Sec. 5, the p-Laplace and minimal-surface examples): residual and Jacobian against
the oracle's, the Picard matrix, and Newton solutions against the oracle's (one discrete
solution), in FP64 and mixed precision."""
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


# (mesh, exponent q, shift, scale, kappa): minimal surface (q = -1/2, shift 1), a regularised
# p-Laplacian with p = 3 (q = 1/2), a shear-thinning exponent in 3D (these three take the
# square-root path of the power) and two exponents with 4q not an integer (the general power)
CASES = {
    "minsurf_2d": (lambda: wl.unit_square_mesh(13), -0.5, 1.0, 1.0, 0.0),
    "plap3_2d": (lambda: wl.unit_square_mesh(11), 0.5, 0.05, 1.0, 0.0),
    "shear_3d": (lambda: wl.unit_cube_mesh(4), -0.25, 0.3, 2.0, 0.4),
    "general_q_2d": (lambda: wl.unit_square_mesh(9), 0.3, 0.2, 1.5, 0.1),   # 4q not an integer: pow
    "general_q_3d": (lambda: wl.unit_cube_mesh(3), -0.7, 0.5, 1.0, 0.2),
}


def _setup(P, name, **opt):
    mk, q, shift, scale, kappa = CASES[name]
    mesh = mk()
    orc = oracle.Problem(mesh, a=("gradpow", q, shift), a_deg=0, a_scale=scale, kappa=kappa)
    h = P.Handle(mesh, P.make_problem(a=("gradpow", q, shift), a_degree=0, a_scale=scale, kappa=kappa),
                 P.default_options(op=P.OP_MATRIX_FREE, **opt))
    return mesh, orc, h


@pytest.mark.parametrize("name", list(CASES))
def test_gradient_residual_parity(P, name):
    mesh, orc, h = _setup(P, name)
    b = wl.random_vector(mesh.n_nodes, 7) * (1 - mesh.dirichlet)
    for seed, s in ((1, 1.0), (2, 0.2)):
        u = wl.random_vector(mesh.n_nodes, seed, s)           # boundary values too
        r = torch.empty(mesh.n_nodes, device="cuda", dtype=torch.float64)
        h.residual(cuda(u), cuda(b), r)
        torch.cuda.synchronize()
        assert rel(r.cpu().numpy(), orc.residual(u, b)) <= 1e-12
    # u = 0: a constant coefficient scale * shift^q, so r = -b on free rows
    r0 = torch.empty(mesh.n_nodes, device="cuda", dtype=torch.float64)
    h.residual(torch.zeros(mesh.n_nodes, device="cuda", dtype=torch.float64), cuda(b), r0)
    torch.cuda.synchronize()
    assert rel(r0.cpu().numpy(), orc.residual(np.zeros(mesh.n_nodes), b)) <= 1e-12


@pytest.mark.parametrize("iteration", ["newton", "picard"])
@pytest.mark.parametrize("name", list(CASES))
def test_gradient_jacobian_parity(P, name, iteration):
    it = P.ITER_PICARD if iteration == "picard" else P.ITER_NEWTON
    mesh, orc, h = _setup(P, name, iteration=it)
    u = wl.random_vector(mesh.n_nodes, 11, 0.7)
    rp, cl = h.pattern()
    vals = torch.empty(h.sizes.jac_nnz, device="cuda", dtype=torch.float64)
    h.jacobian(cuda(u), vals)
    torch.cuda.synchronize()
    A = sp.csr_matrix((vals.cpu().numpy(), cl.cpu().numpy(), rp.cpu().numpy()), shape=(mesh.n_nodes, mesh.n_nodes))
    Ao = orc.jacobian(u, method="picard" if iteration == "picard" else "egfem")
    assert abs(A - Ao).max() <= 1e-12 * abs(Ao).max()
    if iteration == "newton":
        # the gradient coefficient's Jacobian is symmetric on the free block
        free = np.where(mesh.dirichlet == 0)[0]
        Af = A[free][:, free]
        assert abs(Af - Af.T).max() <= 1e-12 * abs(Af).max()


def test_gradient_coefficient_w_space_is_p0(P):
    mesh, _, h = _setup(P, "minsurf_2d")
    assert h.sizes.n_wa == mesh.n_cells
    c = h.w_coords(0)
    nv = mesh.dim + 1
    ref = mesh.coords[mesh.cells].sum(axis=1) / nv
    assert np.abs(c - ref).max() <= 1e-15
    with pytest.raises(P.EgfemError) as e:
        h.pointwise(torch.zeros(mesh.n_nodes, device="cuda", dtype=torch.float64))
    assert e.value.status == 10


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_minimal_surface_newton_matches_oracle(P, prec):
    """Minimal surface with u_D = x y (x + y) and the manufactured source: the library's
    Newton solution equals the oracle's discrete solution and is O(h^2) from the exact one."""
    mesh = wl.unit_square_mesh(32)
    orc = oracle.Problem(mesh, a=("gradpow", -0.5, 1.0), a_deg=0, kappa=0.0)
    ue = wl.minsurf_exact(mesh.coords[:, 0], mesh.coords[:, 1])
    b = orc.load_vector(wl.minsurf_source) * (1 - mesh.dirichlet)
    uD = ue * mesh.dirichlet
    # start from the boundary data with a smooth interior bump (not the exact solution)
    x, y = mesh.coords[:, 0], mesh.coords[:, 1]
    u0 = ue + 0.2 * np.sin(np.pi * x) * np.sin(np.pi * y)
    u_orc, _, _, _ = orc.newton(b, u0=u0, uD=uD, rtol=1e-12)
    opts = P.default_options(op=P.OP_MATRIX_FREE, newton_rtol=1e-12 if prec == "fp64" else 1e-10,
                             precision=P.PREC_MIXED if prec == "mixed" else P.PREC_FP64)
    h = P.Handle(mesh, P.make_problem(a=("gradpow", -0.5, 1.0), a_degree=0, kappa=0.0), opts)
    u = cuda(u0)
    st = h.newton_solve(u, cuda(b + uD))
    torch.cuda.synchronize()
    assert st.status == 0
    un = u.cpu().numpy()
    assert rel(un, u_orc) <= (1e-11 if prec == "fp64" else 1e-8)
    assert np.sqrt(np.mean((un - ue) ** 2)) <= 1e-3


def test_p_laplace_3d_newton_matches_oracle(P):
    mesh = wl.unit_cube_mesh(5)
    orc = oracle.Problem(mesh, a=("gradpow", 0.5, 0.1), a_deg=0, kappa=0.0)
    b = orc.load_vector(wl.smooth_source_3d) * (1 - mesh.dirichlet)
    u_orc, _, _, _ = orc.newton(b, rtol=1e-12)
    h = P.Handle(mesh, P.make_problem(a=("gradpow", 0.5, 0.1), a_degree=0, kappa=0.0),
                 P.default_options(op=P.OP_MATRIX_FREE, newton_rtol=1e-12))
    u = torch.zeros(mesh.n_nodes, device="cuda", dtype=torch.float64)
    st = h.newton_solve(u, cuda(b))
    torch.cuda.synchronize()
    assert st.status == 0
    assert rel(u.cpu().numpy(), u_orc) <= 1e-11


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_p_laplace_disk_picard_matches_oracle_and_closed_form(P, prec):
    """p = 3/2 on the unit disk (Sec. 5): the library's Picard iteration from u = 0 reaches
    the oracle's Picard solution, and Newton from the interpolated closed form the same one."""
    p, n = 1.5, 16
    mesh = wl.unit_disk_mesh(n)
    ue = wl.plaplace_disk_exact(mesh.coords[:, 0], mesh.coords[:, 1], p)
    q = (p - 2) / 2
    orc = oracle.Problem(mesh, a=("gradpow", q, 1e-12), a_deg=0, kappa=0.0)
    b = orc.load_vector(lambda x, y: np.ones_like(x)) * (1 - mesh.dirichlet)
    u_orc, _, _, _ = orc.newton(b, rtol=1e-12, iteration="picard", maxit=300)
    mixed = prec == "mixed"
    prob = P.make_problem(a=("gradpow", q, 1e-12), a_degree=0, kappa=0.0)
    base = dict(op=P.OP_MATRIX_FREE, precision=P.PREC_MIXED if mixed else P.PREC_FP64)
    h = P.Handle(mesh, prob, P.default_options(iteration=P.ITER_PICARD, newton_maxit=300,
                                               newton_rtol=1e-10 if mixed else 1e-12, **base))
    u = torch.zeros(mesh.n_nodes, device="cuda", dtype=torch.float64)
    st = h.newton_solve(u, cuda(b))
    torch.cuda.synchronize()
    assert st.status == 0 and st.newton_iters > 10
    tol = 1e-8 if mixed else 1e-10
    assert rel(u.cpu().numpy(), u_orc) <= tol
    assert np.sqrt(np.mean((u.cpu().numpy() - ue) ** 2)) <= 5e-5
    hn = P.Handle(mesh, prob, P.default_options(newton_rtol=1e-10, eta_max=1e-2, **base))   # tight early solves
    un = cuda(ue * (1 - mesh.dirichlet))
    st = hn.newton_solve(un, cuda(b))
    torch.cuda.synchronize()
    assert st.status == 0 and st.newton_iters <= 8
    assert rel(un.cpu().numpy(), u_orc) <= tol
