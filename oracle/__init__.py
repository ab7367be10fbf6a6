"""FP64 CPU oracle for the EGFEM Newton hot path -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl
reference`` legs of ``bench.py`` may import this package.  It never imports the CUDA
library and the CUDA library never imports it; the two share nothing but the seeded
inputs of ``workloads.py``.

The arithmetic lives in ``egfem_oracle.c`` (plain C loops, FP64); this module only
compiles it (gcc, no vendor tools) and marshals numpy arrays.  What each function
computes, with the paper passage it follows:

* ``Problem.residual(method="sga")``   -- standard Galerkin residual, re-integrated by
  quadrature at every call (Sec. 2.1 discrete problem, Sec. 4 SGA root).
* ``Problem.residual(method="egfem")`` -- EGFEM residual from the precomputed trilinear
  form T_imk = int eta_m grad phi_k . grad phi_i and M_im = int eta_m phi_i, with the
  nonlinearity evaluated pointwise at the W nodes, a = kappa + g(Pi u)
  (Sec. 3.1 nodal coefficients, Sec. 3.2 interpolation operators, Sec. 3.3 multilinear
  forms, Sec. 4 EGFEM root).
* ``Problem.jacobian``                 -- SGA Jacobian by quadrature, or the EGFEM
  Jacobian of Sec. 4 with the identity blocks of the augmented system eliminated.
* ``Problem.newton``                   -- Newton's method (Sec. 4) with banded LU
  (the direct solve of Sec. 5) or Jacobi BiCGStab.
* ``Problem.adjoint``                  -- implicit-function adjoint of a functional of
  the converged solution (the repeated forward/backward solves that Sec. 6 names for
  optimal control).

Parity pins for every function live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np
import scipy.sparse as sp

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "egfem_oracle.c")
_LIBPATH = os.path.join(_HERE, "_build", "liborc.so")
_LOCK = threading.Lock()
_LIB = None

G_NONE, G_POW, G_EXP, G_GRADPOW = 0, 1, 2, 3
FORM_PLAIN, FORM_DIFF = 0, 1

_c_dp = ctypes.POINTER(ctypes.c_double)
_c_ip = ctypes.POINTER(ctypes.c_int)
_c_lp = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags only, OpenMP for the BiCGStab loops) into
    oracle/_build/liborc.so."""
    os.makedirs(os.path.dirname(_LIBPATH), exist_ok=True)
    if force or not os.path.exists(_LIBPATH) or os.path.getmtime(_LIBPATH) < os.path.getmtime(_SRC):
        tmp = _LIBPATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-fopenmp", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIBPATH)
    return _LIBPATH


class _Spec(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nv", ctypes.c_int), ("nc", ctypes.c_int),
                ("X", _c_dp), ("cells", _c_ip), ("dir", ctypes.POINTER(ctypes.c_ubyte)),
                ("a_kind", ctypes.c_int), ("a_p", ctypes.c_double), ("a_scale", ctypes.c_double), ("a_deg", ctypes.c_int),
                ("c_kind", ctypes.c_int), ("c_p", ctypes.c_double), ("c_scale", ctypes.c_double), ("c_deg", ctypes.c_int),
                ("gamma", ctypes.c_double), ("kappa", ctypes.c_double), ("qpts", ctypes.c_int),
                ("a_shift", ctypes.c_double), ("a_quad", ctypes.c_int), ("c_quad", ctypes.c_int),
                ("rule", ctypes.c_int), ("sigma", ctypes.c_double), ("c_product", ctypes.c_int)]


def lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            L = ctypes.CDLL(build())
            L.orc_create.restype = ctypes.c_void_p
            L.orc_create.argtypes = [ctypes.POINTER(_Spec), _c_ip, ctypes.c_int]
            L.orc_destroy.argtypes = [ctypes.c_void_p]
            L.orc_set_kappa_field.argtypes = [ctypes.c_void_p, _c_dp]
            for f in ("orc_space_size", "orc_space_nloc"):
                getattr(L, f).argtypes = [ctypes.c_void_p, ctypes.c_int]
                getattr(L, f).restype = ctypes.c_int
            L.orc_space_coords.argtypes = [ctypes.c_void_p, ctypes.c_int, _c_dp]
            L.orc_space_cell2dof.argtypes = [ctypes.c_void_p, ctypes.c_int, _c_ip]
            L.orc_coo_size.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.orc_coo_size.restype = ctypes.c_int64
            L.orc_coo_export.argtypes = [ctypes.c_void_p, ctypes.c_int, _c_lp, _c_lp, _c_lp, _c_dp]
            L.orc_num_qpts.argtypes = [ctypes.c_void_p]
            L.orc_num_qpts.restype = ctypes.c_int
            L.orc_ref_rule.argtypes = [ctypes.c_void_p, _c_dp, _c_dp]
            L.orc_ref_basis.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _c_dp, _c_dp, _c_dp]
            L.orc_ref_basis.restype = ctypes.c_int
            L.orc_ref_nodes.argtypes = [ctypes.c_int, ctypes.c_int, _c_ip]
            L.orc_simplex_rule.argtypes = [ctypes.c_int, ctypes.c_int, _c_dp, _c_dp]
            L.orc_simplex_rule.restype = ctypes.c_int
            L.orc_sym_rule.argtypes = [ctypes.c_int, ctypes.c_int, _c_dp, _c_dp]
            L.orc_sym_rule.restype = ctypes.c_int
            L.orc_pointwise.argtypes = [ctypes.c_void_p, _c_dp, _c_dp, _c_dp, _c_dp, _c_dp]
            for f in ("orc_egfem_residual", "orc_sga_residual"):
                getattr(L, f).argtypes = [ctypes.c_void_p, _c_dp, _c_dp, _c_dp, ctypes.c_int, _c_dp]
            for f in ("orc_egfem_jacobian", "orc_sga_jacobian", "orc_picard_matrix"):
                getattr(L, f).argtypes = [ctypes.c_void_p, _c_dp, ctypes.c_int64, _c_lp, _c_lp, _c_dp]
                getattr(L, f).restype = ctypes.c_int64
            L.orc_quad_points.argtypes = [ctypes.c_void_p, _c_dp]
            L.orc_load_vector.argtypes = [ctypes.c_void_p, _c_dp, _c_dp]
            L.orc_band_solve.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64, _c_lp, _c_lp, _c_dp, _c_dp]
            L.orc_band_solve.restype = ctypes.c_int
            L.orc_bicgstab.argtypes = [ctypes.c_int, ctypes.c_int64, _c_lp, _c_lp, _c_dp, _c_dp, _c_dp,
                                       ctypes.c_double, ctypes.c_int, _c_ip, _c_dp]
            L.orc_bicgstab.restype = ctypes.c_int
            L.orc_set_threads.argtypes = [ctypes.c_int]
            L.orc_get_threads.restype = ctypes.c_int
            L.orc_newton.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _c_dp, _c_dp, _c_dp,
                                     ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_int, _c_dp, _c_dp, _c_ip]
            L.orc_newton.restype = ctypes.c_int
            L.orc_adjoint.argtypes = [ctypes.c_void_p, _c_dp, _c_dp, ctypes.c_int, ctypes.c_double, _c_dp, _c_dp]
            L.orc_adjoint.restype = ctypes.c_int
            _LIB = L
    return _LIB


def _dp(a):
    return None if a is None else a.ctypes.data_as(_c_dp)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


_KIND = {None: G_NONE, "none": G_NONE, "pow": G_POW, "exp": G_EXP, "gradpow": G_GRADPOW}


class Problem:
    """One discretised problem  -div((kappa + w) grad u) + gamma c + sigma u = d,  u = u_D on Gamma.

    w = a_scale * g_a(Pi_a u) lives in the Lagrange space of degree ``a_deg``;
    c = c_scale * g_c(Pi_c u) in the space of degree ``c_deg``.  ``g`` is
    ``("pow", p)`` -> s^p or ``("exp",)`` -> e^s.  ``a_space="quad"`` (``c_space``) makes
    W the quadrature space I_k of Sec. 3.1, Case 3 with k = ``a_deg`` (``c_deg``): one node
    per point of the symmetric degree-k rule on every cell.  ``rule=k`` makes every integral
    (the standard Galerkin approach, the load vector and the Lagrange-space tensors) use that
    same rule instead of the collapsed Gauss rule of ``qpts`` points.  ``sigma`` adds the linear
    reaction sigma * int u phi_i (P1 mass matrix).  ``c_product=True`` makes the reaction
    gamma * int c u phi_i (the trilinear mass form M3 : (u x c), decomposition (a) of the
    superconductivity example) instead of gamma * int c phi_i.  ``cells`` restricts the tensor
    assembly (and the SGA integrals) to a subset of cells, so that single rows of a
    large problem can be evaluated exactly: a row is complete when every cell that
    contains its vertex is in the subset.
    """

    def __init__(self, mesh, *, a=("pow", 2.0), a_scale=1.0, a_deg=2, c=None, c_scale=1.0, c_deg=1,
                 gamma=0.0, kappa=1.0, qpts=4, cells=None, a_space="lagrange", c_space="lagrange", rule=0,
                 sigma=0.0, c_product=False):
        self.mesh = mesh
        self._X = np.ascontiguousarray(mesh.coords, dtype=np.float64)
        self._cells = np.ascontiguousarray(mesh.cells, dtype=np.int32)
        self._dir = np.ascontiguousarray(mesh.dirichlet, dtype=np.uint8)
        s = _Spec()
        s.dim, s.nv, s.nc = mesh.dim, mesh.n_nodes, mesh.n_cells
        s.X = self._X.ctypes.data_as(_c_dp)
        s.cells = self._cells.ctypes.data_as(_c_ip)
        s.dir = self._dir.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))
        s.a_kind = _KIND[a[0] if a else None]
        s.a_p = float(a[1]) if a and len(a) > 1 else 1.0
        s.a_shift = float(a[2]) if a and a[0] == "gradpow" and len(a) > 2 else 0.0
        s.a_scale, s.a_deg = float(a_scale), int(a_deg)
        s.c_kind = _KIND[c[0] if c else None]
        s.c_p = float(c[1]) if c and len(c) > 1 else 1.0
        s.c_scale, s.c_deg = float(c_scale), int(c_deg)
        s.gamma, s.kappa, s.qpts = float(gamma), float(kappa), int(qpts)
        s.a_quad, s.c_quad, s.rule = int(a_space == "quad"), int(c_space == "quad"), int(rule)
        s.sigma = float(sigma)
        s.c_product = int(bool(c_product))
        self._spec = s
        self._sel = None if cells is None else np.ascontiguousarray(cells, dtype=np.int32)
        L = lib()
        self._h = L.orc_create(ctypes.byref(s), None if self._sel is None else self._sel.ctypes.data_as(_c_ip),
                               0 if self._sel is None else len(self._sel))
        if not self._h:
            raise ValueError("oracle: no symmetric rule of that degree (triangle 1..4, tetrahedron 1..3)")
        self.n = mesh.n_nodes
        self.nw = L.orc_space_size(self._h, 0)
        self.nc_space = L.orc_space_size(self._h, 1)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    # --- introspection ---
    def space_coords(self, which=0):
        n = lib().orc_space_size(self._h, which)
        out = np.empty((n, self.mesh.dim))
        lib().orc_space_coords(self._h, which, _dp(out))
        return out

    def cell2dof(self, which=0):
        nl = lib().orc_space_nloc(self._h, which)
        out = np.empty((self.mesh.n_cells, nl), dtype=np.int32)
        lib().orc_space_cell2dof(self._h, which, out.ctypes.data_as(_c_ip))
        return out

    def _coo(self, which):
        L = lib()
        n = L.orc_coo_size(self._h, which)
        I, J, K = (np.empty(n, dtype=np.int64) for _ in range(3))
        V = np.empty(n)
        L.orc_coo_export(self._h, which, I.ctypes.data_as(_c_lp), J.ctypes.data_as(_c_lp), K.ctypes.data_as(_c_lp), _dp(V))
        return I, J, K, V

    def T_coo(self):
        """(i, m, k, T_imk) for the assembled cells, sorted, duplicates summed."""
        return self._coo(0)

    def M_coo(self):
        I, J, _, V = self._coo(1)
        return I, J, V

    def Pi(self, which=0):
        I, J, _, V = self._coo(2 if which == 0 else 3)
        n = self.nw if which == 0 else self.nc_space
        return sp.csr_matrix((V, (I, J)), shape=(n, self.n))

    def set_kappa_field(self, kappa):
        self._kappa = _f64(kappa)
        lib().orc_set_kappa_field(self._h, _dp(self._kappa))

    # --- quadrature / load ---
    def quad_points(self):
        nq = lib().orc_num_qpts(self._h)
        out = np.empty((self.mesh.n_cells * nq, self.mesh.dim))
        lib().orc_quad_points(self._h, _dp(out))
        return out

    def load_vector(self, f):
        """b_i = int f phi_i by the oracle's quadrature; f is a callable f(x, y[, z])."""
        xq = self.quad_points()
        fq = _f64(f(*[xq[:, d] for d in range(self.mesh.dim)]))
        b = np.empty(self.n)
        lib().orc_load_vector(self._h, _dp(fq), _dp(b))
        return b

    def load_vector_cellwise(self, f_cell):
        """b_i for f constant on each cell (f_cell[c]), by the same quadrature."""
        nq = lib().orc_num_qpts(self._h)
        fq = np.repeat(_f64(f_cell), nq)
        b = np.empty(self.n)
        lib().orc_load_vector(self._h, _dp(fq), _dp(b))
        return b

    # --- nonlinear operators ---
    def pointwise(self, u):
        u = _f64(u)
        w, wp = np.empty(self.nw), np.empty(self.nw)
        c, cp = np.empty(self.nc_space), np.empty(self.nc_space)
        lib().orc_pointwise(self._h, _dp(u), _dp(w), _dp(wp), _dp(c), _dp(cp))
        return w, wp, c, cp

    def residual(self, u, b=None, uD=None, method="egfem", form="plain"):
        u, b, uD = _f64(u), _f64(b), _f64(uD)
        r = np.empty(self.n)
        f = lib().orc_egfem_residual if method == "egfem" else lib().orc_sga_residual
        f(self._h, _dp(u), _dp(b), _dp(uD), FORM_DIFF if form == "diff" else FORM_PLAIN, _dp(r))
        return r

    def jacobian(self, u, method="egfem"):
        """Newton Jacobian (method "egfem" or "sga"), or the Picard iteration matrix T .2 a(u)
        (method "picard"; Sec. 4, Example 4.1), with Dirichlet rows/columns handled."""
        u = _f64(u)
        f = {"egfem": lib().orc_egfem_jacobian, "sga": lib().orc_sga_jacobian, "picard": lib().orc_picard_matrix}[method]
        n = f(self._h, _dp(u), 0, None, None, None)
        I, L = np.empty(n, dtype=np.int64), np.empty(n, dtype=np.int64)
        V = np.empty(n)
        f(self._h, _dp(u), n, I.ctypes.data_as(_c_lp), L.ctypes.data_as(_c_lp), _dp(V))
        return sp.csr_matrix((V, (I, L)), shape=(self.n, self.n))

    def newton(self, b, u0=None, uD=None, method="egfem", solver="lu", rtol=1e-10, maxit=50, ktol=1e-12,
               form="diff", keep_iterates=False, iteration="newton"):
        """Newton's method from u0 (default 0) -- or, with iteration="picard" (EGFEM only), the
        Picard iteration with the frozen-coefficient matrix (Sec. 4, Example 4.1).  Returns
        (u, residual_history, iterates, krylov_iters)."""
        u = np.zeros(self.n) if u0 is None else _f64(u0).copy()
        b, uD = _f64(b), _f64(uD)
        hist = np.zeros(maxit + 1)
        its = np.zeros((maxit + 1) * self.n) if keep_iterates else None
        ktot = ctypes.c_int(0)
        code = 2 if iteration == "picard" else (0 if method == "egfem" else 1)
        k = lib().orc_newton(self._h, code, 0 if solver == "lu" else 1, _dp(b), _dp(uD),
                             _dp(u), float(rtol), int(maxit), float(ktol), FORM_DIFF if form == "diff" else FORM_PLAIN,
                             _dp(hist), _dp(its), ctypes.byref(ktot))
        if k < 0:
            raise RuntimeError(f"oracle Newton failed with code {k}")
        iterates = its.reshape(maxit + 1, self.n)[: k + 1] if keep_iterates else None
        return u, hist[: k + 1], iterates, ktot.value

    def adjoint(self, u, dJdu, solver="lu", ktol=1e-13):
        """lambda solving J^T lambda = dJdu (free rows; 0 on Dirichlet rows) and
        dJ/dkappa_m = -sum_{i,k} lambda_i T_imk u_k.  dJ/db = lambda."""
        u, g = _f64(u), _f64(dJdu)
        lam, gk = np.empty(self.n), np.empty(self.nw)
        st = lib().orc_adjoint(self._h, _dp(u), _dp(g), 0 if solver == "lu" else 1, float(ktol), _dp(lam), _dp(gk))
        if st != 0:
            raise RuntimeError(f"oracle adjoint solve failed with code {st}")
        return lam, gk


# --- reference-element and solver probes (used by the pin tests) ---

def ref_basis(dim, p, xi):
    xi = np.ascontiguousarray(np.atleast_2d(xi), dtype=np.float64)
    npts = xi.shape[0]
    nb = {0: 1, 1: dim + 1, 2: (dim + 1) * (dim + 2) // 2, 3: (dim + 1) * (dim + 2) * (dim + 3) // 6}[p]
    val, grad = np.empty((npts, nb)), np.empty((npts, nb, dim))
    lib().orc_ref_basis(dim, p, npts, _dp(xi), _dp(val), _dp(grad))
    return val, grad


def ref_nodes(dim, p):
    nb = {0: 1, 1: dim + 1, 2: (dim + 1) * (dim + 2) // 2, 3: (dim + 1) * (dim + 2) * (dim + 3) // 6}[p]
    out = np.empty((nb, dim + 1), dtype=np.int32)
    lib().orc_ref_nodes(dim, p, out.ctypes.data_as(_c_ip))
    return out


def simplex_rule(dim, q):
    pts, wts = np.empty(q ** dim * dim), np.empty(q ** dim)
    n = lib().orc_simplex_rule(dim, q, _dp(pts), _dp(wts))
    return pts[: n * dim].reshape(n, dim), wts[:n]


def sym_rule(dim, k):
    """The symmetric degree-k rule behind I_k: reference points [n, dim] and weights (sum 1/d!)."""
    pts, wts = np.empty(16 * dim), np.empty(16)
    n = lib().orc_sym_rule(dim, k, _dp(pts), _dp(wts))
    if n < 0:
        raise ValueError(f"no symmetric rule of degree {k} in {dim}D")
    return pts[: n * dim].reshape(n, dim), wts[:n]


def band_solve(A, rhs):
    """Banded LU with partial pivoting on a scipy sparse matrix A."""
    A = sp.coo_matrix(A)
    I, L = A.row.astype(np.int64), A.col.astype(np.int64)
    V = A.data.astype(np.float64)
    kl = int(max(0, (I - L).max())) if len(I) else 0
    ku = int(max(0, (L - I).max())) if len(I) else 0
    x = _f64(rhs).copy()
    st = lib().orc_band_solve(A.shape[0], kl, ku, len(I), I.ctypes.data_as(_c_lp), L.ctypes.data_as(_c_lp), _dp(V), _dp(x))
    if st != 0:
        raise RuntimeError(f"band solve failed with code {st}")
    return x


def set_threads(n: int) -> int:
    """Use n OpenMP threads in the oracle's BiCGStab (its results do not depend on n); returns
    the thread count now in effect."""
    lib().orc_set_threads(int(n))
    return int(lib().orc_get_threads())


def get_threads() -> int:
    return int(lib().orc_get_threads())


def bicgstab(A, rhs, rtol=1e-12, maxit=100000, x0=None):
    A = sp.coo_matrix(A)
    order = np.lexsort((A.col, A.row))
    I, L = A.row[order].astype(np.int64), A.col[order].astype(np.int64)
    V = A.data[order].astype(np.float64)
    x = np.zeros(A.shape[0]) if x0 is None else _f64(x0).copy()
    b = _f64(rhs)
    its, rr = ctypes.c_int(0), ctypes.c_double(0)
    st = lib().orc_bicgstab(A.shape[0], len(I), I.ctypes.data_as(_c_lp), L.ctypes.data_as(_c_lp), _dp(V), _dp(b), _dp(x),
                            float(rtol), int(maxit), ctypes.byref(its), ctypes.byref(rr))
    return x, st, its.value, rr.value
