"""CPU-only checks of the CUDA library: the C ABI loads and exports every declared
symbol, and its host-side offline assembly (W numbering, stored CSF tensor) matches
the oracle's independent quadrature.  No GPU code runs here."""
import os
import re

import numpy as np
import pytest

import oracle
import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def egf():
    import __graft_entry__
    __graft_entry__.build_library()
    import paper_2005_06193_gb300 as P
    return P


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "egfem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(egfem_[a-z_0-9]+)\s*\(", src)))


def test_abi_exports_every_declared_symbol(egf):
    names = _declared_functions()
    assert len(names) >= 19
    L = egf.lib()
    for n in names:
        assert hasattr(L, n), n
    assert L.egfem_status_string(0) == b"EGFEM_OK"
    assert L.egfem_status_string(6) == b"EGFEM_ERR_BREAKDOWN"


def _match_w(oc, lc):
    """permutation p with lc[p[j]] == oc[j] (coordinates rounded to 1e-12)"""
    key = lambda c: [tuple(np.round(x, 12)) for x in c]
    lk = {k: i for i, k in enumerate(key(lc))}
    return np.array([lk[k] for k in key(oc)])


@pytest.mark.parametrize("dim,n,deg", [(2, 5, 1), (2, 5, 2), (2, 5, 3), (3, 2, 1), (3, 2, 2), (3, 2, 3)])
def test_stored_tensor_matches_oracle_quadrature(egf, dim, n, deg):
    """Every stored T_imk (off-diagonal leaves plus the per-fibre diagonal) equals the
    oracle's quadrature value, and every oracle entry not stored is zero to rounding."""
    mesh = wl.unit_square_mesh(n) if dim == 2 else wl.unit_cube_mesh(n)
    I, M, K, V, Wc = egf.inspect_tensor(mesh, egf.make_problem(a=("pow", 2), a_degree=deg))
    P = oracle.Problem(mesh, a=("pow", 2.0), a_deg=deg, qpts=5)
    oI, oM, oK, oV = P.T_coo()
    perm = _match_w(P.space_coords(0), Wc)          # oracle m -> library m
    assert len(perm) == len(Wc)
    scale = np.abs(oV).max()
    orc = {(i, perm[m], k): v for i, m, k, v in zip(oI, oM, oK, oV) if not mesh.dirichlet[i]}
    lib = {(i, m, k): v for i, m, k, v in zip(I, M, K, V)}
    assert not any(mesh.dirichlet[i] for (i, _, _) in lib)
    for key, v in lib.items():
        assert abs(orc.get(key, 0.0) - v) <= 1e-13 * scale, (key, v, orc.get(key))
    for key, v in orc.items():
        if key not in lib:
            assert abs(v) <= 1e-13 * scale, (key, v)


def test_stored_tensor_has_exact_zero_row_sums(egf):
    mesh = wl.unit_square_mesh(7)
    I, M, K, V, _ = egf.inspect_tensor(mesh, egf.make_problem(a=("pow", 2), a_degree=2))
    s = {}
    for i, m, v in zip(I, M, V):
        s[(i, m)] = s.get((i, m), 0.0) + v
    assert max(abs(x) for x in s.values()) <= 1e-15


def test_constant_coefficient_stores_the_stiffness(egf):
    """Without a coefficient nonlinearity the stored form is kappa-free stiffness A."""
    mesh = wl.unit_cube_mesh(3)
    I, M, K, V, _ = egf.inspect_tensor(mesh, egf.make_problem(a=None, a_degree=1, c=("exp",), c_degree=1, gamma=-2.0))
    assert np.all(M == -1)
    P = oracle.Problem(mesh, a=None, a_deg=1)
    oI, oM, oK, oV = P.T_coo()
    A = {}
    for i, k, v in zip(oI, oK, oV):
        if not mesh.dirichlet[i]:
            A[(i, k)] = A.get((i, k), 0.0) + v
    lib = {(i, k): v for i, k, v in zip(I, K, V)}
    for key, v in A.items():
        assert abs(lib.get(key, 0.0) - v) <= 1e-14, key


def test_table1_w_space_sizes_match(egf):
    """Library W numbering reproduces the P2/P3 counts of Table 1 on the 64 x 64 grid."""
    mesh = wl.unit_square_mesh(64)
    for deg, size in ((2, 20866), (3, 41474)):
        _, _, _, _, W = egf.inspect_tensor(mesh, egf.make_problem(a=("pow", 2), a_degree=deg))
        assert mesh.n_nodes + len(W) == size


@pytest.mark.parametrize("bad", ["index", "degenerate", "repeat"])
def test_malformed_mesh_is_rejected(egf, bad):
    mesh = wl.unit_square_mesh(3)
    cells = mesh.cells.copy()
    coords = mesh.coords.copy()
    if bad == "index":
        cells[4, 1] = mesh.n_nodes + 5
    elif bad == "repeat":
        cells[2, 2] = cells[2, 0]
    else:
        coords[cells[3, 1]] = coords[cells[3, 0]]
    m2 = wl.Mesh(2, coords, cells, mesh.dirichlet)
    with pytest.raises(egf.EgfemError) as e:
        egf.inspect_tensor(m2, egf.make_problem())
    assert e.value.status == 2


def test_bad_problem_is_rejected(egf):
    mesh = wl.unit_square_mesh(3)
    with pytest.raises(egf.EgfemError) as e:
        egf.inspect_tensor(mesh, egf.make_problem(a_degree=4))
    assert e.value.status == 1


def test_barrier_selftest_rejects_bad_sizes_without_a_gpu(egf):
    """Argument checks of the grid-barrier self-test happen before any CUDA call."""
    L = egf.lib()
    import ctypes
    ok = (ctypes.c_int32 * 4)()
    for blocks, arrive, wait in [(0, 0, 10.0), (65, 1, 10.0), (4, 5, 10.0), (4, 2, 0.0), (4, 2, 5000.0)]:
        assert L.egfem_selftest_grid_barrier(blocks, arrive, wait, ok, None) == 1
    assert L.egfem_selftest_grid_barrier(4, 2, 10.0, None, None) == 1


@pytest.mark.parametrize("dim,n", [(2, 5), (3, 2)])
def test_p0_form_of_the_gradient_coefficient_matches_oracle_quadrature(egf, dim, n):
    """With W_a = P0 (gradient coefficient) the form the element-local operator reads per cell,
    T_iKk = S^K_ik, equals the oracle's quadrature of int eta_K grad phi_k . grad phi_i."""
    mesh = wl.unit_square_mesh(n) if dim == 2 else wl.unit_cube_mesh(n)
    I, M, K, V, Wc = egf.inspect_tensor(mesh, egf.make_problem(a=("gradpow", -0.5, 1.0), a_degree=0))
    assert len(Wc) == mesh.n_cells
    P = oracle.Problem(mesh, a=("gradpow", -0.5, 1.0), a_deg=0)
    oI, oM, oK, oV = P.T_coo()
    perm = _match_w(P.space_coords(0), Wc)
    scale = np.abs(oV).max()
    orc = {(i, perm[m], k): v for i, m, k, v in zip(oI, oM, oK, oV) if not mesh.dirichlet[i]}
    lib = {}
    for i, m, k, v in zip(I, M, K, V):
        lib[(i, m, k)] = lib.get((i, m, k), 0.0) + v
    assert not any(mesh.dirichlet[i] for (i, _, _) in lib)
    assert set(lib) == set(orc)
    for key, v in lib.items():
        assert abs(orc[key] - v) <= 1e-13 * scale, (key, v, orc[key])


def test_bad_gradient_coefficient_is_rejected_before_any_cuda_call(egf):
    """Build-time checks of the gradient coefficient return before the library touches a
    device: W_a must be P0, the operator element-local, (shift + s)^q finite at s = 0, and
    the reaction may not take the gradient kind."""
    import ctypes
    mesh = wl.unit_square_mesh(3)
    m, keep = egf.egfem._mesh_struct(mesh)
    mf = egf.default_options(op=egf.OP_MATRIX_FREE)
    cases = [(egf.make_problem(a=("gradpow", -0.5, 1.0), a_degree=0), egf.default_options(op=egf.OP_CSF), 10),
             (egf.make_problem(a=("gradpow", -0.5, 1.0), a_degree=1), mf, 1),
             (egf.make_problem(a=("gradpow", 0.5, 0.0), a_degree=0), mf, 1),
             (egf.make_problem(a=("gradpow", -0.5, -1.0), a_degree=0), mf, 1),
             (egf.make_problem(a=None, c=("gradpow", 1.0, 1.0), c_degree=1), mf, 1)]
    for prob, opts, want in cases:
        h = ctypes.c_void_p()
        assert egf.lib().egfem_build(ctypes.byref(m), ctypes.byref(prob), ctypes.byref(opts), ctypes.byref(h)) == want
        assert not h.value
    del keep


@pytest.mark.parametrize("dim,n,k", [(2, 4, 1), (2, 4, 2), (2, 4, 3), (2, 4, 4), (3, 2, 1), (3, 2, 2), (3, 2, 3)])
def test_quadrature_space_form_matches_oracle(egf, dim, n, k):
    """W_a = I_k: the form the element-local operator applies, T_ilk = w_l S^K_ik / |K|, and the
    node coordinates (the rule's points on every cell) equal the oracle's, whose rule is pinned
    by its exactness; the library's rule table is written independently."""
    mesh = wl.unit_square_mesh(n) if dim == 2 else wl.unit_cube_mesh(n)
    I, M, K, V, Wc = egf.inspect_tensor(mesh, egf.make_problem(a=("pow", 2), a_degree=k, a_space="quad"))
    P = oracle.Problem(mesh, a=("pow", 2.0), a_deg=k, a_space="quad")
    assert len(Wc) == P.nw == mesh.n_cells * len(oracle.sym_rule(dim, k)[1])
    oI, oM, oK, oV = P.T_coo()
    perm = _match_w(P.space_coords(0), Wc)
    scale = np.abs(oV).max()
    orc = {(i, perm[m], kk): v for i, m, kk, v in zip(oI, oM, oK, oV) if not mesh.dirichlet[i]}
    lib = {}
    for i, m, kk, v in zip(I, M, K, V):
        lib[(i, m, kk)] = lib.get((i, m, kk), 0.0) + v
    assert set(lib) == set(orc)
    for key, v in lib.items():
        assert abs(orc[key] - v) <= 1e-13 * scale, (key, v, orc[key])


def test_table1_quadrature_space_size_in_the_library(egf):
    """Table 1: the EGFEM with I_4 on the 64 x 64 grid has 4225 + 6 x 8192 = 53377 unknowns."""
    mesh = wl.unit_square_mesh(64)
    _, _, _, _, W = egf.inspect_tensor(mesh, egf.make_problem(a=("pow", 2), a_degree=4, a_space="quad"))
    assert mesh.n_nodes + len(W) == 53377


def test_bad_quadrature_space_is_rejected_before_any_cuda_call(egf):
    import ctypes
    mesh = wl.unit_cube_mesh(2)
    m, keep = egf.egfem._mesh_struct(mesh)
    mf = egf.default_options(op=egf.OP_MATRIX_FREE)
    cases = [(egf.make_problem(a=("pow", 2), a_degree=4, a_space="quad"), mf, 1),       # no degree-4 tetrahedron rule
             (egf.make_problem(a=("pow", 2), a_degree=2, a_space="quad"), egf.default_options(op=egf.OP_CSF), 10),
             (egf.make_problem(a=None, c=("pow", 2), c_degree=0, c_space="quad", gamma=1.0), mf, 1)]
    for prob, opts, want in cases:
        h = ctypes.c_void_p()
        assert egf.lib().egfem_build(ctypes.byref(m), ctypes.byref(prob), ctypes.byref(opts), ctypes.byref(h)) == want
        assert not h.value
    bad = egf.make_problem()
    bad.a_space = 7
    h = ctypes.c_void_p()
    assert egf.lib().egfem_build(ctypes.byref(m), ctypes.byref(bad), ctypes.byref(mf), ctypes.byref(h)) == 1
    del keep


def test_empty_mesh_is_rejected(egf):
    """A mesh without nodes or cells is an invalid argument, reported before any device work."""
    import numpy as np
    empty = wl.Mesh(2, np.zeros((0, 2)), np.zeros((0, 3), dtype=np.int32), np.zeros(0, dtype=np.uint8))
    with pytest.raises(egf.EgfemError) as e:
        egf.inspect_tensor(empty, egf.make_problem())
    assert e.value.status == 1


def test_default_options_leave_the_choices_to_the_library(egf):
    """The defaults the C library fills in (no GPU needed): the forcing-term cap 0 (the library
    picks 0.9 for Newton, 1e-2 for Picard), Newton iteration, FP64, the CSF operator, the
    persistent Krylov driver, the cluster solve where it fits and the graph Newton loop on."""
    o = egf.default_options()
    assert o.eta_max == 0.0 and o.eta_min == 1e-12
    assert o.newton_rtol == 1e-10 and o.newton_maxit == 50 and o.krylov_maxit == 100000
    assert o.iteration == egf.ITER_NEWTON and o.precision == egf.PREC_FP64 and o.op == egf.OP_CSF
    assert o.krylov_persistent == 1 and o.krylov_cluster == 0 and o.newton_graph == 1 and o.fixed_eta == 0
    # keyword overrides reach the structure
    o2 = egf.default_options(eta_max=0.3, iteration=egf.ITER_PICARD)
    assert o2.eta_max == 0.3 and o2.iteration == egf.ITER_PICARD


def _union(mesh, k):
    """k copies of one mesh laid out as a batch lays out its instances: each copy's nodes padded to
    whole 32-row slices with isolated Dirichlet nodes (no cells)."""
    rows = -(-mesh.n_nodes // 32) * 32
    X = np.zeros((k * rows, mesh.dim))
    cells = np.concatenate([mesh.cells + b * rows for b in range(k)]).astype(np.int32)
    dirichlet = np.ones(k * rows, dtype=np.uint8)
    for b in range(k):
        X[b * rows:b * rows + mesh.n_nodes] = mesh.coords
        dirichlet[b * rows:b * rows + mesh.n_nodes] = mesh.dirichlet
    return wl.Mesh(mesh.dim, X, cells, dirichlet), rows


@pytest.mark.parametrize("dim,n,deg", [(2, 7, 2), (2, 6, 3), (3, 2, 2)])
def test_union_of_one_mesh_is_instance_affine(egf, dim, n, deg):
    """The premise of the shared-tensor batch: in the disjoint union of k copies of one mesh, copy
    b's stored tensor is copy 0's, entry by entry in stored order, with rows and columns shifted by
    b x (padded rows) and every W index shifted by b times one stride per node kind (the W nodes
    are numbered kind by kind, copy after copy inside each kind)."""
    mesh = wl.unit_square_mesh(n) if dim == 2 else wl.unit_cube_mesh(n)
    k = 3
    U, rows = _union(mesh, k)
    I, M, K, V, W = egf.inspect_tensor(U, egf.make_problem(a=("pow", 2), a_degree=deg))
    grp = [np.flatnonzero((I >= b * rows) & (I < (b + 1) * rows)) for b in range(k)]
    assert len(grp[0]) > 0 and all(len(g) == len(grp[0]) for g in grp)
    i0, m0, k0, v0 = I[grp[0]], M[grp[0]], K[grp[0]], V[grp[0]]
    strides = set()
    for b in range(1, k):
        g = grp[b]
        assert np.array_equal(I[g] - b * rows, i0)
        assert np.array_equal(K[g] - b * rows, k0)
        assert np.array_equal(V[g], v0)   # the same tensor values, bit for bit
        assert np.array_equal(M[g] < 0, m0 < 0)
        w = m0 >= 0
        dm = M[g][w] - m0[w]
        assert np.all(dm % b == 0)
        assert np.array_equal(W[M[g][w]], W[m0[w]])   # the same W node of the copy
        strides.add(tuple(sorted(set((dm // b).tolist()))))
    # one stride per node kind that the tensor holds, the same for every copy: on triangles the P2
    # vertex functions integrate to zero, so T holds edge nodes only (one stride); P3 on triangles
    # and P2 on tetrahedra hold vertices too (and P3 face nodes)
    assert len(strides) == 1
    assert len(next(iter(strides))) == {(2, 2): 1, (2, 3): 3, (3, 2): 2}[(dim, deg)]
