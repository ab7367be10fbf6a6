"""Batches of one mesh (egfem_options.batch_share): the tensor T and the reaction entries are
stored once and every instance reads that copy, its W indices offset per instance and node
kind.  The shared handle must give the results of the per-instance copies (batch_share = 0)
bit for bit in the tensor action (residual, Jacobian), the same Newton solutions and adjoint
gradients, and each instance must still equal the oracle's single-instance residual.

Tolerances: residual and Jacobian values are compared exactly (the same arithmetic in the
same order per row); Newton solutions to 1e-12 relative (FP64) and 1e-9 (mixed), adjoint
gradients (accumulated with atomics in an unspecified order) to 1e-12 relative; the oracle
residual to 1e-12 relative as in the other parity tests.
"""
import dataclasses

import numpy as np
import pytest

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


CASES = {
    # name: (mesh factory, oracle kwargs, library problem kwargs); the P3 case has vertex,
    # third-point and face W nodes, the reaction case a second W space (W_c = P1)
    "u2_p2_ragged": (lambda: wl.unit_square_mesh(13), dict(a=("pow", 2.0), a_deg=2), dict(a=("pow", 2), a_degree=2)),
    "u3_p3_2d": (lambda: wl.unit_square_mesh(17), dict(a=("pow", 3.0), a_deg=3), dict(a=("pow", 3), a_degree=3)),
    "u2_p2_reaction": (lambda: wl.unit_square_mesh(16),
                       dict(a=("pow", 2.0), a_deg=2, c=("exp",), c_deg=1, gamma=-1.0),
                       dict(a=("pow", 2), a_degree=2, c=("exp",), c_degree=1, gamma=-1.0)),
    "u2_p2_3d": (lambda: wl.unit_cube_mesh(4), dict(a=("pow", 2.0), a_deg=2), dict(a=("pow", 2), a_degree=2)),
}
K = 5


def _pair(P, mesh, pkw, **opt):
    prob = P.make_problem(**pkw)
    hs = P.BatchHandle([mesh] * K, prob, P.default_options(**opt))
    hu = P.BatchHandle([mesh] * K, prob, P.default_options(batch_share=0, **opt))
    return hs, hu


def _jacobian(h, u):
    vals = torch.empty(h.sizes.jac_nnz, device="cuda", dtype=torch.float64)
    h.jacobian(u, vals)
    return vals


@pytest.mark.parametrize("name", list(CASES))
def test_shared_tensor_equals_per_instance_copies(P, name):
    mk, okw, pkw = CASES[name]
    mesh = mk()
    hs, hu = _pair(P, mesh, pkw)
    bs, ks = hs.tensor_storage()
    bu, ku = hu.tensor_storage()
    assert ks == K and ku == 0
    assert bs * K == bu and bs > 0
    assert np.array_equal(hs.offsets, hu.offsets) and hs.sizes.n_wa == hu.sizes.n_wa
    free = 1 - mesh.dirichlet
    us = [wl.random_vector(mesh.n_nodes, 10 + b, 0.3 + 0.2 * b) * free for b in range(K)]
    orc = oracle.Problem(mesh, **okw)
    src = wl.mms_source if mesh.dim == 2 else wl.smooth_source_3d
    b0 = orc.load_vector(src) * free
    ds = [b0 * (1.0 + 0.25 * b) for b in range(K)]
    u, d = hs.scatter(us), hs.scatter(ds)
    r_s, r_u = torch.empty_like(u), torch.empty_like(u)
    hs.residual(u, d, r_s)
    hu.residual(u, d, r_u)
    torch.cuda.synchronize()
    assert torch.equal(r_s, r_u)
    rs = hs.gather(r_s, [mesh.n_nodes] * K)
    for b in range(K):
        assert rel(rs[b], orc.residual(us[b], ds[b])) <= 1e-12, b
    assert torch.equal(_jacobian(hs, u), _jacobian(hu, u))
    # a coefficient field kappa over the union's W_a nodes: every instance reads its own part
    kappa = cuda(1.0 + 0.5 * wl.random_vector(hs.sizes.n_wa, 7, 1.0) ** 2)
    hs.set_kappa(kappa)
    hu.set_kappa(kappa)
    hs.residual(u, d, r_s)
    hu.residual(u, d, r_u)
    torch.cuda.synchronize()
    assert torch.equal(r_s, r_u)
    assert torch.equal(_jacobian(hs, u), _jacobian(hu, u))
    hs.close()
    hu.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_shared_tensor_batched_newton(P, prec):
    """Five P3 instances of one mesh with different sources: the batched Newton solve on the
    shared tensor gives the solutions of the per-instance copies, and each the oracle's."""
    mesh = wl.unit_square_mesh(17)
    free = 1 - mesh.dirichlet
    inst = wl.batch_instances(count=K, seed=5, n_lo=17, n_hi=17)
    orc = oracle.Problem(mesh, a=("pow", 3.0), a_deg=3)
    loads = [orc.load_vector(src) * free for _, src in inst]
    opt = dict(newton_rtol=1e-13 if prec == "fp64" else 1e-10,
               precision=P.PREC_MIXED if prec == "mixed" else P.PREC_FP64)
    hs, hu = _pair(P, mesh, dict(a=("pow", 3), a_degree=3), **opt)
    sols = []
    for h in (hs, hu):
        d = h.scatter(loads)
        u = torch.zeros_like(d)
        st = h.batch_newton_solve(u, d)
        torch.cuda.synchronize()
        assert all(s.status == 0 for s in st)
        sols.append(h.gather(u, [mesh.n_nodes] * K))
    for b in range(K):
        assert rel(sols[0][b], sols[1][b]) <= (1e-12 if prec == "fp64" else 1e-9), b
        u_ref, _, _, _ = orc.newton(loads[b], rtol=1e-13)
        assert rel(sols[0][b], u_ref) <= (1e-11 if prec == "fp64" else 1e-6), b
    hs.close()
    hu.close()


def test_shared_tensor_adjoint_kappa_gradient(P):
    """The adjoint and the kappa gradient (one atomic scatter per fibre into the union's W_a
    field) on the shared tensor equal those of the per-instance copies."""
    mesh = wl.unit_square_mesh(14)
    free = 1 - mesh.dirichlet
    hs, hu = _pair(P, mesh, dict(a=("pow", 2), a_degree=2), newton_rtol=1e-13)
    orc = oracle.Problem(mesh, a=("pow", 2.0), a_deg=2)
    b0 = orc.load_vector(wl.mms_source) * free
    out = []
    for h in (hs, hu):
        d = h.scatter([b0 * (1.0 + 0.5 * b) for b in range(K)])
        u = torch.zeros_like(d)
        h.batch_newton_solve(u, d)
        g = h.scatter([wl.random_vector(mesh.n_nodes, 20 + b, 1.0) * free for b in range(K)])
        lam = torch.empty_like(u)
        gk = torch.empty(h.sizes.n_wa, device="cuda", dtype=torch.float64)
        h.adjoint(u, g, lam, gk)
        torch.cuda.synchronize()
        out.append((u.cpu().numpy(), lam.cpu().numpy(), gk.cpu().numpy()))
    for a, b in zip(out[0], out[1]):
        assert rel(a, b) <= 1e-12
    hs.close()
    hu.close()


def test_batches_of_different_meshes_keep_their_copies(P):
    """Instances that differ in anything (here one Dirichlet flag) are not shared, and a
    single-instance batch has nothing to share."""
    mesh = wl.unit_square_mesh(12)
    other = dataclasses.replace(mesh, dirichlet=mesh.dirichlet.copy())
    other.dirichlet[np.flatnonzero(mesh.dirichlet)[0]] = 0
    prob = P.make_problem(a=("pow", 2), a_degree=2)
    h = P.BatchHandle([mesh, mesh, other], prob)
    assert h.tensor_storage()[1] == 0
    h.close()
    h1 = P.BatchHandle([mesh], prob)
    assert h1.tensor_storage()[1] == 0
    h1.close()


def test_shared_tensor_profile_counts_bytes_once(P):
    """The tensor action's algorithmic bytes count the shared tensor once (its operations
    once per instance)."""
    mesh = wl.unit_square_mesh(40)
    hs, hu = _pair(P, mesh, dict(a=("pow", 2), a_degree=2))
    free = 1 - mesh.dirichlet
    u = hs.scatter([wl.random_vector(mesh.n_nodes, 3, 0.5) * free] * K)
    d = torch.zeros_like(u)
    ps = {p["name"]: p for p in hs.profile_kernels(u, d, reps=2)}
    pu = {p["name"]: p for p in hu.profile_kernels(u, d, reps=2)}
    assert ps["csf_fused"]["flops"] == pu["csf_fused"]["flops"]
    bs, _ = hs.tensor_storage()
    assert pu["csf_fused"]["bytes"] - ps["csf_fused"]["bytes"] == pytest.approx((K - 1) * bs, rel=1e-12)
    hs.close()
    hu.close()


@pytest.mark.parametrize("n,k", [(4, 3), (4, 40), (9, 17)])
def test_shared_tensor_small_instances_many_copies(P, n, k):
    """Instances of one slice (a 4 x 4 grid: 25 nodes in 32 rows) and many copies: the tensor
    action's blocks then cover fewer rows than a block holds and take the instances in turn; the
    residual and Jacobian still equal those of the per-instance copies bit for bit and the oracle's
    per instance."""
    mesh = wl.unit_square_mesh(n)
    prob = P.make_problem(a=("pow", 3), a_degree=3)
    hs = P.BatchHandle([mesh] * k, prob, P.default_options())
    hu = P.BatchHandle([mesh] * k, prob, P.default_options(batch_share=0))
    assert hs.tensor_storage()[1] == k and hu.tensor_storage()[1] == 0
    free = 1 - mesh.dirichlet
    us = [wl.random_vector(mesh.n_nodes, 100 + b, 0.6) * free for b in range(k)]
    ds = [wl.random_vector(mesh.n_nodes, 300 + b, 1.0) * free for b in range(k)]
    u, d = hs.scatter(us), hs.scatter(ds)
    r_s, r_u = torch.empty_like(u), torch.empty_like(u)
    hs.residual(u, d, r_s)
    hu.residual(u, d, r_u)
    torch.cuda.synchronize()
    assert torch.equal(r_s, r_u)
    assert torch.equal(_jacobian(hs, u), _jacobian(hu, u))
    orc = oracle.Problem(mesh, a=("pow", 3.0), a_deg=3)
    rs = hs.gather(r_s, [mesh.n_nodes] * k)
    for b in (0, k // 2, k - 1):
        assert rel(rs[b], orc.residual(us[b], ds[b])) <= 1e-12, b
    hs.close()
    hu.close()
