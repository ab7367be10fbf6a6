"""The allocation-free residual-norm entry point, egfem_free_norm2_noalloc.

Callers that cannot allocate device memory when they need the Newton convergence number
(an application that reserves all device memory for its own pool, or a real-time loop
that cannot afford cudaMalloc's implicit synchronisation) call this entry point: its
scratch is a static device array.  This file runs last (pytest collects files in name
order), so a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_noalloc_norm_equals_newton_initial_residual_norm_twice():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2005_06193_gb300 as P
    assert torch.cuda.is_available()
    mesh = wl.unit_square_mesh(32)
    cen = wl.cell_centroids(mesh)
    h = P.Handle(mesh, P.make_problem(a=("pow", 2), a_degree=2), P.default_options(newton_maxit=0))
    f = torch.tensor(wl.mms_source(cen[:, 0], cen[:, 1]), device="cuda", dtype=torch.float64)
    d = torch.empty(mesh.n_nodes, device="cuda", dtype=torch.float64)
    h.load_cellwise(f, d)
    u = torch.tensor(wl.random_vector(mesh.n_nodes, 21, 0.5) * (1 - mesh.dirichlet), device="cuda", dtype=torch.float64)
    # existing entry point: with newton_maxit = 0 the solve only evaluates ||r(u0)|| over free rows
    st = h.newton_solve(u, d, check=False)
    r = torch.empty_like(u)
    h.residual(u, d, r)
    dirichlet = torch.tensor(mesh.dirichlet, device="cuda", dtype=torch.uint8)
    out = torch.full((1,), -1.0, device="cuda", dtype=torch.float64)
    L = P.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    vals = []
    for _ in range(2):
        status = L.egfem_free_norm2_noalloc(mesh.n_nodes, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(dirichlet.data_ptr()),
                                           ctypes.c_void_p(out.data_ptr()), stream)
        assert status == 0, L.egfem_last_error()
        torch.cuda.synchronize()
        vals.append(float(out.item()))
        out.fill_(-1.0)
    assert st.res0 > 0
    # independent check: the host's sum over the copied-back residual's free rows
    rn = r.cpu().numpy()
    host = float(np.sum(rn[mesh.dirichlet == 0] ** 2))
    for v in vals:
        assert abs(v - host) <= 1e-12 * host
        assert abs(np.sqrt(v) - st.res0) <= 1e-12 * st.res0
    assert vals[0] == vals[1]


def test_noalloc_norm_rejects_sizes_beyond_its_scratch():
    import paper_2005_06193_gb300 as P
    small = torch.zeros(4, device="cuda", dtype=torch.float64)
    mask = torch.zeros(4, device="cuda", dtype=torch.uint8)
    L = P.lib()
    # checked on the host before any launch: the buffers are never read
    status = L.egfem_free_norm2_noalloc(8192 * 16384 + 1, ctypes.c_void_p(small.data_ptr()), ctypes.c_void_p(mask.data_ptr()),
                                       ctypes.c_void_p(small.data_ptr()), None)
    assert status == 1
    assert b"static scratch" in L.egfem_last_error()
