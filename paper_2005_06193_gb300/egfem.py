"""Thin Python binding of the C ABI in include/egfem.h (argument marshalling only).

Every step of the hot path runs in the CUDA library ``_build/libegfem.so``; this module
converts torch tensors to device pointers and the current torch stream to a
``cudaStream_t``, and raises on any non-OK status.  There is no CPU fallback: if the
library is missing or cannot load, importing the binding's entry points fails.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libegfem.so")

G_NONE, G_POW, G_EXP, G_GRADPOW = 0, 1, 2, 3
W_LAGRANGE, W_QUADRATURE = 0, 1
PREC_FP64, PREC_MIXED = 0, 1
OP_CSF, OP_MATRIX_FREE = 0, 1
ITER_NEWTON, ITER_PICARD = 0, 1
HIST = 64

STATUS = {0: "EGFEM_OK", 1: "EGFEM_ERR_INVALID_ARG", 2: "EGFEM_ERR_MESH", 3: "EGFEM_ERR_CUDA", 4: "EGFEM_ERR_OOM",
          5: "EGFEM_ERR_NOT_CONVERGED", 6: "EGFEM_ERR_BREAKDOWN", 7: "EGFEM_ERR_SINGULAR", 8: "EGFEM_ERR_NONFINITE",
          9: "EGFEM_ERR_TIMEOUT", 10: "EGFEM_ERR_UNSUPPORTED"}


class EgfemError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}" + (f" ({detail})" if detail else ""))


class Mesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("n_nodes", ctypes.c_int64), ("n_cells", ctypes.c_int64),
                ("coords", ctypes.POINTER(ctypes.c_double)), ("cells", ctypes.POINTER(ctypes.c_int32)),
                ("dirichlet", ctypes.POINTER(ctypes.c_uint8))]


class Problem(ctypes.Structure):
    _fields_ = [("a_kind", ctypes.c_int32), ("a_p", ctypes.c_double), ("a_scale", ctypes.c_double),
                ("a_degree", ctypes.c_int32), ("c_kind", ctypes.c_int32), ("c_p", ctypes.c_double),
                ("c_scale", ctypes.c_double), ("c_degree", ctypes.c_int32), ("gamma", ctypes.c_double),
                ("kappa", ctypes.c_double), ("a_shift", ctypes.c_double), ("a_space", ctypes.c_int32),
                ("c_space", ctypes.c_int32), ("sigma", ctypes.c_double), ("c_product", ctypes.c_int32)]


class Options(ctypes.Structure):
    _fields_ = [("newton_rtol", ctypes.c_double), ("newton_atol", ctypes.c_double), ("newton_maxit", ctypes.c_int32),
                ("eta_max", ctypes.c_double), ("eta_min", ctypes.c_double), ("krylov_maxit", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("op", ctypes.c_int32), ("graph_chunk", ctypes.c_int32),
                ("fixed_eta", ctypes.c_int32), ("krylov_persistent", ctypes.c_int32), ("iteration", ctypes.c_int32),
                ("krylov_block_rows", ctypes.c_int32), ("krylov_cluster", ctypes.c_int32),
                ("newton_graph", ctypes.c_int32), ("batch_share", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("newton_iters", ctypes.c_int32), ("krylov_iters", ctypes.c_int64),
                ("res0", ctypes.c_double), ("res_final", ctypes.c_double), ("res_hist", ctypes.c_double * HIST),
                ("krylov_hist", ctypes.c_int32 * HIST), ("solve_ms", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64), ("fp64_rescues", ctypes.c_int32)]

    def as_dict(self) -> dict:
        k = min(self.newton_iters, HIST)
        return {"status": STATUS.get(self.status, self.status), "newton_iters": self.newton_iters,
                "krylov_iters": int(self.krylov_iters), "res0": self.res0, "res_final": self.res_final,
                "res_hist": list(self.res_hist[:k]), "krylov_hist": list(self.krylov_hist[:k]),
                "solve_ms": self.solve_ms, "kernel_launches": int(self.kernel_launches),
                "fp64_rescues": self.fp64_rescues}


PROF_MAX = 8


class Profile(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int32), ("name", (ctypes.c_char * 24) * PROF_MAX), ("ms", ctypes.c_double * PROF_MAX),
                ("bytes", ctypes.c_double * PROF_MAX), ("flops", ctypes.c_double * PROF_MAX),
                ("fp64", ctypes.c_int32 * PROF_MAX)]

    def as_list(self) -> list:
        return [{"name": self.name[k].value.decode(), "ms": self.ms[k], "bytes": self.bytes[k], "flops": self.flops[k],
                 "fp64": bool(self.fp64[k])} for k in range(self.count)]


_lib = None
_P = ctypes.c_void_p
_DP = ctypes.c_void_p   # device pointers travel as plain addresses


def lib() -> ctypes.CDLL:
    """Load libegfem.so (built by paper_2005_06193_gb300._build).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library {LIB_PATH} is missing: run __graft_entry__.build() (nvcc, sm_103a)")
    L = ctypes.CDLL(LIB_PATH)
    S = ctypes.c_int
    sig = {
        "egfem_default_options": (None, [ctypes.POINTER(Options)]),
        "egfem_build": (S, [ctypes.POINTER(Mesh), ctypes.POINTER(Problem), ctypes.POINTER(Options), ctypes.POINTER(_P)]),
        "egfem_destroy": (None, [_P]),
        "egfem_set_options": (S, [_P, ctypes.POINTER(Options)]),
        "egfem_sizes": (S, [_P] + [ctypes.POINTER(ctypes.c_int64)] * 5),
        "egfem_w_coords": (S, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]),
        "egfem_tensor_storage": (S, [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)]),
        "egfem_jacobian_pattern": (S, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P)]),
        "egfem_set_kappa": (S, [_P, _DP, _P]),
        "egfem_pointwise": (S, [_P, _DP, _DP, _DP, _P]),
        "egfem_residual": (S, [_P, _DP, _DP, _DP, _P]),
        "egfem_jacobian": (S, [_P, _DP, _DP, _P]),
        "egfem_spmv": (S, [_P, _DP, _DP, _DP, _P]),
        "egfem_bicgstab": (S, [_P, _DP, _DP, _DP, ctypes.c_double, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), _P]),
        "egfem_newton_solve": (S, [_P, _DP, _DP, ctypes.POINTER(Stats), _P]),
        "egfem_adjoint": (S, [_P, _DP, _DP, _DP, _DP, ctypes.POINTER(Stats), _P]),
        "egfem_load_cellwise": (S, [_P, _DP, _DP, _P]),
        "egfem_batch_build": (S, [ctypes.c_int32, ctypes.POINTER(Mesh), ctypes.POINTER(Problem), ctypes.POINTER(Options),
                                  ctypes.POINTER(_P)]),
        "egfem_batch_layout": (S, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)]),
        "egfem_batch_newton_solve": (S, [_P, _DP, _DP, _P, _P]),
        "egfem_profile_kernels": (S, [_P, _DP, _DP, ctypes.c_int32, ctypes.POINTER(Profile), _P]),
        "egfem_load_cellwise_transpose": (S, [_P, _DP, _DP, _P]),
        "egfem_inspect_tensor": (S, [ctypes.POINTER(Mesh), ctypes.POINTER(Problem), ctypes.POINTER(ctypes.c_int64),
                                     _P, _P, _P, _P, ctypes.POINTER(ctypes.c_int64), _P]),
        "egfem_free_norm2_noalloc": (S, [ctypes.c_int64, _DP, _DP, _DP, _P]),
        "egfem_selftest_grid_barrier": (S, [ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                            ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
        "egfem_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "egfem_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(status: int, where: str):
    if status != 0:
        detail = lib().egfem_last_error().decode(errors="replace")
        raise EgfemError(status, where, detail)


def default_options(**kw) -> Options:
    o = Options()
    lib().egfem_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp64": PREC_FP64, "mixed": PREC_MIXED}[v]
        setattr(o, k, v)
    return o


def selftest_grid_barrier(blocks: int, arrive: int, wait_ms: float):
    """Run the bounded grid-barrier self-test; returns (per-block outcome list, error word)."""
    ok = (ctypes.c_int32 * blocks)()
    err = ctypes.c_int32(0)
    _check(lib().egfem_selftest_grid_barrier(blocks, arrive, wait_ms, ok, ctypes.byref(err)), "selftest_grid_barrier")
    return list(ok), err.value


def make_problem(a=("pow", 2), a_degree=2, a_scale=1.0, c=None, c_degree=1, c_scale=1.0, gamma=0.0, kappa=1.0,
                 a_space="lagrange", c_space="lagrange", sigma=0.0, c_product=False) -> Problem:
    """a = (kind, exponent[, shift]): ("pow", p), ("exp",), ("gradpow", q, shift) for the gradient
    coefficient (shift + |grad u|^2)^q (with a_degree=0); c likewise for the reaction.
    a_space / c_space = "quad" selects the quadrature space I_k with k = a_degree / c_degree;
    sigma adds the linear reaction sigma * int u phi_i; c_product makes the reaction
    gamma * int c u phi_i (trilinear mass form) instead of gamma * int c phi_i."""
    spaces = {"lagrange": W_LAGRANGE, "quad": W_QUADRATURE}
    kinds = {None: G_NONE, "none": G_NONE, "pow": G_POW, "exp": G_EXP, "gradpow": G_GRADPOW}
    p = Problem()
    p.a_kind = kinds[a[0] if a else None]
    p.a_p = float(a[1]) if a and len(a) > 1 else 1.0
    p.a_shift = float(a[2]) if a and a[0] == "gradpow" and len(a) > 2 else 0.0
    p.a_scale, p.a_degree = float(a_scale), int(a_degree)
    p.c_kind = kinds[c[0] if c else None]
    p.c_p = float(c[1]) if c and len(c) > 1 else 1.0
    p.c_scale, p.c_degree = float(c_scale), int(c_degree)
    p.gamma, p.kappa = float(gamma), float(kappa)
    p.a_space, p.c_space = spaces[a_space], spaces[c_space]
    p.sigma = float(sigma)
    p.c_product = int(bool(c_product))
    return p


def _mesh_struct(mesh):
    coords = np.ascontiguousarray(mesh.coords, dtype=np.float64)
    cells = np.ascontiguousarray(mesh.cells, dtype=np.int32)
    dirichlet = np.ascontiguousarray(mesh.dirichlet, dtype=np.uint8)
    m = Mesh()
    m.dim, m.n_nodes, m.n_cells = mesh.dim, coords.shape[0], cells.shape[0]
    m.coords = coords.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    m.cells = cells.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    m.dirichlet = dirichlet.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    return m, (coords, cells, dirichlet)


def inspect_tensor(mesh, problem: Problem):
    """Host-only: the stored trilinear form as COO (i, m, k, T_imk) and the W_a node
    coordinates; runs no GPU code."""
    m, keep = _mesh_struct(mesh)
    n, nw = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(lib().egfem_inspect_tensor(ctypes.byref(m), ctypes.byref(problem), ctypes.byref(n), None, None, None, None,
                                      ctypes.byref(nw), None), "egfem_inspect_tensor")
    I, M, K = (np.empty(n.value, dtype=np.int64) for _ in range(3))
    V = np.empty(n.value)
    W = np.empty((nw.value, mesh.dim))
    _check(lib().egfem_inspect_tensor(ctypes.byref(m), ctypes.byref(problem), ctypes.byref(n), I.ctypes.data,
                                      M.ctypes.data, K.ctypes.data, V.ctypes.data, ctypes.byref(nw), W.ctypes.data),
           "egfem_inspect_tensor")
    del keep
    return I, M, K, V, W


def _ptr(t):
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise TypeError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


@dataclass
class Sizes:
    n_nodes: int
    n_wa: int
    n_wc: int
    jac_rows: int
    jac_nnz: int


class Handle:
    """An assembled EGFEM operator on the current CUDA device (egfem_build)."""

    def __init__(self, mesh, problem: Problem, options: Options | None = None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("egfem: a CUDA device is required (no CPU fallback)")
        m, keep = _mesh_struct(mesh)
        self._h = _P()
        self.options = options or default_options()
        _check(lib().egfem_build(ctypes.byref(m), ctypes.byref(problem), ctypes.byref(self.options), ctypes.byref(self._h)),
               "egfem_build")
        del keep
        self.problem = problem
        self.dim = mesh.dim
        vals = [ctypes.c_int64() for _ in range(5)]
        _check(lib().egfem_sizes(self._h, *[ctypes.byref(v) for v in vals]), "egfem_sizes")
        self.sizes = Sizes(*[v.value for v in vals])
        self.device = torch.device("cuda", torch.cuda.current_device())

    def close(self):
        if getattr(self, "_h", None):
            lib().egfem_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- inspection ---
    def tensor_storage(self):
        """(device bytes of the stored tensor and reaction entries, instances sharing them or 0)"""
        b, k = ctypes.c_int64(0), ctypes.c_int32(0)
        _check(lib().egfem_tensor_storage(self._h, ctypes.byref(b), ctypes.byref(k)), "egfem_tensor_storage")
        return b.value, k.value

    def w_coords(self, which=0) -> np.ndarray:
        n = self.sizes.n_wa if which == 0 else self.sizes.n_wc
        out = np.empty((n, self.dim))
        _check(lib().egfem_w_coords(self._h, which, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "egfem_w_coords")
        return out

    def pattern(self):
        """(rowptr, cols) of the Jacobian as int32 CUDA tensors (copies of the handle's arrays)."""
        rp, cl = _P(), _P()
        _check(lib().egfem_jacobian_pattern(self._h, ctypes.byref(rp), ctypes.byref(cl)), "egfem_jacobian_pattern")
        n, nnz = self.sizes.jac_rows, self.sizes.jac_nnz
        return _wrap_device(rp.value, (n + 1,), "<i4").clone(), _wrap_device(cl.value, (nnz,), "<i4").clone()

    # --- hot path ---
    def set_kappa(self, kappa=None, stream=None):
        _check(lib().egfem_set_kappa(self._h, _ptr(kappa), _stream(stream)), "egfem_set_kappa")

    def pointwise(self, u, w=None, wprime=None, stream=None):
        _check(lib().egfem_pointwise(self._h, _ptr(u), _ptr(w), _ptr(wprime), _stream(stream)), "egfem_pointwise")
        return w, wprime

    def residual(self, u, d, r, stream=None):
        _check(lib().egfem_residual(self._h, _ptr(u), _ptr(d), _ptr(r), _stream(stream)), "egfem_residual")
        return r

    def jacobian(self, u, vals, stream=None):
        _check(lib().egfem_jacobian(self._h, _ptr(u), _ptr(vals), _stream(stream)), "egfem_jacobian")
        return vals

    def spmv(self, vals, x, y, stream=None):
        _check(lib().egfem_spmv(self._h, _ptr(vals), _ptr(x), _ptr(y), _stream(stream)), "egfem_spmv")
        return y

    def bicgstab(self, vals, rhs, x, rtol=1e-10, maxit=100000, stream=None) -> int:
        it = ctypes.c_int32(0)
        _check(lib().egfem_bicgstab(self._h, _ptr(vals), _ptr(rhs), _ptr(x), float(rtol), int(maxit), ctypes.byref(it),
                                    _stream(stream)), "egfem_bicgstab")
        return it.value

    def newton_solve(self, u, d, stream=None, check=True) -> Stats:
        st = Stats()
        status = lib().egfem_newton_solve(self._h, _ptr(u), _ptr(d), ctypes.byref(st), _stream(stream))
        if check:
            _check(status, "egfem_newton_solve")
        return st

    def adjoint(self, u, dJdu, lam, grad_kappa=None, stream=None) -> Stats:
        st = Stats()
        _check(lib().egfem_adjoint(self._h, _ptr(u), _ptr(dJdu), _ptr(lam), _ptr(grad_kappa), ctypes.byref(st),
                                   _stream(stream)), "egfem_adjoint")
        return st

    def profile_kernels(self, u, d, reps=20, stream=None) -> list:
        prof = Profile()
        _check(lib().egfem_profile_kernels(self._h, _ptr(u), _ptr(d), int(reps), ctypes.byref(prof), _stream(stream)),
               "egfem_profile_kernels")
        return prof.as_list()

    def load_cellwise(self, f, d, stream=None):
        _check(lib().egfem_load_cellwise(self._h, _ptr(f), _ptr(d), _stream(stream)), "egfem_load_cellwise")
        return d

    def load_cellwise_transpose(self, lam, g, stream=None):
        _check(lib().egfem_load_cellwise_transpose(self._h, _ptr(lam), _ptr(g), _stream(stream)),
               "egfem_load_cellwise_transpose")
        return g

    def set_options(self, options: Options):
        _check(lib().egfem_set_options(self._h, ctypes.byref(options)), "egfem_set_options")
        self.options = options


class _DeviceArray:
    """A raw device allocation exposed through __cuda_array_interface__ (zero copy)."""

    def __init__(self, ptr: int, shape: tuple, typestr: str):
        self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr, "data": (int(ptr), False), "version": 3,
                                         "strides": None}


def _wrap_device(ptr: int, shape: tuple, typestr: str):
    import torch
    return torch.as_tensor(_DeviceArray(ptr, shape, typestr), device="cuda")


class BatchHandle(Handle):
    """Many instances as one block-diagonal operator (egfem_batch_build).  Instance b
    owns rows offsets[b]:offsets[b+1] of every batch vector (padded to 32 rows)."""

    def __init__(self, meshes, problem: Problem, options: Options | None = None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("egfem: a CUDA device is required (no CPU fallback)")
        structs, keep = [], []
        for m in meshes:
            st, k = _mesh_struct(m)
            structs.append(st)
            keep.append(k)
        arr = (Mesh * len(structs))(*structs)
        self._h = _P()
        self.options = options or default_options()
        _check(lib().egfem_batch_build(len(structs), arr, ctypes.byref(problem), ctypes.byref(self.options),
                                       ctypes.byref(self._h)), "egfem_batch_build")
        del keep
        self.problem = problem
        self.dim = meshes[0].dim
        vals = [ctypes.c_int64() for _ in range(5)]
        _check(lib().egfem_sizes(self._h, *[ctypes.byref(v) for v in vals]), "egfem_sizes")
        self.sizes = Sizes(*[v.value for v in vals])
        self.device = torch.device("cuda", torch.cuda.current_device())
        cnt = ctypes.c_int32(0)
        _check(lib().egfem_batch_layout(self._h, ctypes.byref(cnt), None), "egfem_batch_layout")
        off = np.zeros(cnt.value + 1, dtype=np.int64)
        _check(lib().egfem_batch_layout(self._h, ctypes.byref(cnt), off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))),
               "egfem_batch_layout")
        self.count = cnt.value
        self.offsets = off

    def scatter(self, parts, dtype=None):
        """Concatenate per-instance host arrays into one padded batch tensor on the device."""
        import torch
        out = np.zeros(self.offsets[-1])
        for b, p in enumerate(parts):
            out[self.offsets[b]:self.offsets[b] + len(p)] = p
        return torch.tensor(out, device=self.device, dtype=dtype or torch.float64)

    def gather(self, t, sizes):
        a = t.detach().cpu().numpy()
        return [a[self.offsets[b]:self.offsets[b] + sizes[b]] for b in range(self.count)]

    def batch_newton_solve(self, u, d, stream=None, check=True):
        st = (Stats * self.count)()
        status = lib().egfem_batch_newton_solve(self._h, _ptr(u), _ptr(d), st, _stream(stream))
        if check:
            _check(status, "egfem_batch_newton_solve")
        return list(st)
