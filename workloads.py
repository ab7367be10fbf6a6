"""Seeded synthetic inputs for the EGFEM Newton hot path.

This module is shared by the CPU oracle (``oracle/``), the CUDA library's tests and
``bench.py``.  It holds *input data only*: meshes (coordinates, connectivity,
Dirichlet masks), closed-form source functions and exact solutions chosen by the
method of manufactured solutions (Sec. 5, quadratic example), and the seeded random
parameters of the batched and adjoint workloads.  It contains none of the method's
arithmetic: no basis function, quadrature rule, tensor, interpolation operator or
solver lives here.

Mesh conventions (the paper uses Gmsh meshes "refined through splitting", Sec. 5;
structured generators stand in for them):

* 2D: the n x n unit-square grid, vertex (i, j) at (i/n, j/n) numbered i + (n+1) j.
  Every grid cell is split along its SW->NE diagonal into the triangles
  [(i,j), (i+1,j), (i+1,j+1)] and [(i,j), (i+1,j+1), (i,j+1)].
* 3D: the n^3 unit-cube grid, vertex (i, j, k) numbered i + (n+1)(j + (n+1) k).
  Every cube is split into the 6 Kuhn (Freudenthal) tetrahedra that share the
  (0,0,0)->(1,1,1) diagonal, one per permutation of the three axes.

The Dirichlet boundary is the whole boundary (homogeneous data, except the minimal-surface
example, whose boundary values are those of its exact solution).
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np


@dataclass
class Mesh:
    """A conforming simplicial mesh (host arrays)."""

    dim: int
    coords: np.ndarray     # float64 [n_nodes, dim]
    cells: np.ndarray      # int32   [n_cells, dim + 1]
    dirichlet: np.ndarray  # uint8   [n_nodes], 1 on the Dirichlet boundary

    @property
    def n_nodes(self) -> int:
        return int(self.coords.shape[0])

    @property
    def n_cells(self) -> int:
        return int(self.cells.shape[0])


def unit_square_mesh(n: int) -> Mesh:
    """n x n structured grid of the unit square, 2 triangles per cell (2 n^2 total)."""
    if n < 1:
        raise ValueError("n must be >= 1")
    m = n + 1
    jj, ii = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    coords = np.stack([ii.ravel() / n, jj.ravel() / n], axis=1).astype(np.float64)
    cj, ci = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    v00 = (ci + m * cj).ravel()
    v10 = v00 + 1
    v11 = v00 + 1 + m
    v01 = v00 + m
    t1 = np.stack([v00, v10, v11], axis=1)
    t2 = np.stack([v00, v11, v01], axis=1)
    cells = np.stack([t1, t2], axis=1).reshape(-1, 3).astype(np.int32)
    x, y = ii.ravel(), jj.ravel()
    dirichlet = ((x == 0) | (x == n) | (y == 0) | (y == n)).astype(np.uint8)
    return Mesh(2, coords, cells, dirichlet)


def unit_cube_mesh(n: int) -> Mesh:
    """n^3 structured grid of the unit cube, 6 Kuhn tetrahedra per cube (6 n^3 total)."""
    if n < 1:
        raise ValueError("n must be >= 1")
    m = n + 1
    kk, jj, ii = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    coords = np.stack([ii.ravel() / n, jj.ravel() / n, kk.ravel() / n], axis=1).astype(np.float64)
    ck, cj, ci = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    base = (ci + m * (cj + m * ck)).ravel()
    step = [1, m, m * m]
    tets = []
    for perm in itertools.permutations(range(3)):
        a = base
        b = a + step[perm[0]]
        c = b + step[perm[1]]
        d = c + step[perm[2]]
        tets.append(np.stack([a, b, c, d], axis=1))
    cells = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)
    x, y, z = ii.ravel(), jj.ravel(), kk.ravel()
    dirichlet = ((x == 0) | (x == n) | (y == 0) | (y == n) | (z == 0) | (z == n)).astype(np.uint8)
    return Mesh(3, coords, cells, dirichlet)


def unit_disk_mesh(n: int) -> Mesh:
    """Unit disk (the p-Laplace example's domain, Sec. 5) as n concentric rings: ring k
    (k = 1..n) holds 6k vertices at radius k/n and angles 2 pi j / (6k), j = 0..6k-1;
    vertex 0 is the centre and ring k starts at index 1 + 3k(k-1).  The band between rings
    k-1 and k is zipped by angle into 6(2k-1) triangles, 6 n^2 in all.  The Dirichlet
    boundary is the outer ring (its vertices lie on the circle)."""
    if n < 1:
        raise ValueError("n must be >= 1")
    pts = [np.zeros((1, 2))]
    starts = [0]
    for k in range(1, n + 1):
        t = 2.0 * np.pi * np.arange(6 * k) / (6 * k)
        starts.append(1 + 3 * k * (k - 1))
        pts.append(np.stack([k / n * np.cos(t), k / n * np.sin(t)], axis=1))
    coords = np.concatenate(pts).astype(np.float64)
    cells = []
    for k in range(1, n + 1):
        nin, nout = max(1, 6 * (k - 1)), 6 * k
        inner = [starts[k - 1] + j for j in range(nin)] if k > 1 else [0]
        outer = [starts[k] + j for j in range(nout)]
        if k == 1:
            cells += [[0, outer[j], outer[(j + 1) % nout]] for j in range(nout)]
            continue
        # zipper: advance along whichever ring's next vertex comes first in angle (exact
        # rational comparison (j+1)/nin vs (l+1)/nout of the fractions of a turn)
        i = l = 0
        while i < nin or l < nout:
            if l < nout and (i == nin or (l + 1) * nin <= (i + 1) * nout):
                cells.append([inner[i % nin], outer[l], outer[(l + 1) % nout]])
                l += 1
            else:
                cells.append([inner[i], outer[l % nout], inner[(i + 1) % nin]])
                i += 1
    cells = np.array(cells, dtype=np.int32)
    # counter-clockwise orientation (the library and the oracle take |det|; kept tidy)
    a, b, c = coords[cells[:, 0]], coords[cells[:, 1]], coords[cells[:, 2]]
    det = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
    cells[det < 0] = cells[det < 0][:, [0, 2, 1]]
    dirichlet = np.zeros(coords.shape[0], dtype=np.uint8)
    dirichlet[starts[n]:] = 1
    return Mesh(2, coords, cells, dirichlet)


def fan_mesh(k: int) -> Mesh:
    """A high-valence test mesh: a centre vertex, a free ring of k vertices at radius 1/2 and a
    Dirichlet ring of k vertices at radius 1, with k centre triangles and 2k between the rings.
    The centre has k neighbours, so k > 31 exercises the 64-column row kernels."""
    if k < 3:
        raise ValueError("k must be >= 3")
    t = 2.0 * np.pi * np.arange(k) / k
    coords = np.concatenate([np.zeros((1, 2)), 0.5 * np.stack([np.cos(t), np.sin(t)], 1),
                             np.stack([np.cos(t + np.pi / k), np.sin(t + np.pi / k)], 1)]).astype(np.float64)
    cells = []
    for j in range(k):
        a, b = 1 + j, 1 + (j + 1) % k            # inner ring
        c, d = 1 + k + j, 1 + k + (j + 1) % k    # outer ring
        cells += [[0, a, b], [a, c, b], [b, c, d]]
    dirichlet = np.zeros(coords.shape[0], dtype=np.uint8)
    dirichlet[1 + k:] = 1
    return Mesh(2, coords, np.array(cells, dtype=np.int32), dirichlet)


def plaplace_disk_exact(x: np.ndarray, y: np.ndarray, p: float) -> np.ndarray:
    """The closed-form solution of -div(|grad u|^(p-2) grad u) = 1 on the unit disk with u = 0
    on its boundary (Sec. 5, p-Laplace example): 2^(-1/(p-1)) (p-1)/p (1 - |x|^(p/(p-1)))."""
    r = np.sqrt(x * x + y * y)
    return 2.0 ** (-1.0 / (p - 1.0)) * (p - 1.0) / p * (1.0 - r ** (p / (p - 1.0)))


# ---------------------------------------------------------------------------
# Manufactured solution for -div((1 + u^2) grad u) = f on the unit square.
# With u = sin(pi x) sin(pi y):  -div((1+u^2) grad u) = -(1+u^2) lap u - 2 u |grad u|^2,
# lap u = -2 pi^2 u and |grad u|^2 = pi^2 (cos^2(pi x) sin^2(pi y) + sin^2(pi x) cos^2(pi y)).
# ---------------------------------------------------------------------------

def mms_exact(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    return np.sin(np.pi * x) * np.sin(np.pi * y)


def mms_exact_grad(x: np.ndarray, y: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    return (np.pi * np.cos(np.pi * x) * np.sin(np.pi * y),
            np.pi * np.sin(np.pi * x) * np.cos(np.pi * y))


def mms_source(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """f for -div((1+u^2) grad u) = f with exact solution sin(pi x) sin(pi y)."""
    u = mms_exact(x, y)
    gx, gy = mms_exact_grad(x, y)
    return 2.0 * np.pi ** 2 * u * (1.0 + u * u) - 2.0 * u * (gx * gx + gy * gy)


def mms_source_cubic(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """f for -div((1+u^3) grad u) = f with exact solution sin(pi x) sin(pi y)."""
    u = mms_exact(x, y)
    gx, gy = mms_exact_grad(x, y)
    return 2.0 * np.pi ** 2 * u * (1.0 + u ** 3) - 3.0 * u * u * (gx * gx + gy * gy)


def minsurf_exact(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """The minimal-surface example's boundary data and exact solution, u = x y (x + y)
    (Sec. 5, minimal surface equation on the unit square)."""
    return x * y * (x + y)


def minsurf_source(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """d = -div(grad u / sqrt(1 + |grad u|^2)) for u = minsurf_exact (manufactured source):
    with q = grad u, H its Hessian and Q = 1 + |q|^2, div(q / sqrt(Q)) = lap(u) / sqrt(Q)
    - q^T H q / Q^(3/2)."""
    ux, uy = 2.0 * x * y + y * y, x * x + 2.0 * x * y
    uxx, uxy, uyy = 2.0 * y, 2.0 * x + 2.0 * y, 2.0 * x
    Q = 1.0 + ux * ux + uy * uy
    qhq = ux * ux * uxx + 2.0 * ux * uy * uxy + uy * uy * uyy
    return -((uxx + uyy) / np.sqrt(Q) - qhq / Q ** 1.5)


def quadratic_source(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """d for -lap u + u^2 = d with exact solution u = x y (x + y) (Sec. 5, quadratic example):
    -lap u = -2 (x + y) and u^2 = x^2 y^2 (x + y)^2."""
    return -2.0 * (x + y) + (x * y * (x + y)) ** 2


def supercond_exact(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """The superconductivity example's boundary data and exact solution (Sec. 5, simplified
    Ginzburg-Landau model): u = sin(2 pi x) sin(2 pi y) exp(2 x) / 6."""
    return np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y) * np.exp(2 * x) / 6.0


def supercond_source(x: np.ndarray, y: np.ndarray, nu: float) -> np.ndarray:
    """d = -nu lap u + u^3 + u for u = supercond_exact (manufactured source): with
    f(x) = sin(2 pi x) e^(2x), f'' = (4 - 4 pi^2) sin(2 pi x) e^(2x) + 8 pi cos(2 pi x) e^(2x), so
    lap u = e^(2x) sin(2 pi y) ((4 - 8 pi^2) sin(2 pi x) + 8 pi cos(2 pi x)) / 6."""
    u = supercond_exact(x, y)
    lap = np.exp(2 * x) * np.sin(2 * np.pi * y) * ((4 - 8 * np.pi ** 2) * np.sin(2 * np.pi * x)
                                                    + 8 * np.pi * np.cos(2 * np.pi * x)) / 6.0
    return -nu * lap + u ** 3 + u


def smooth_source_3d(x: np.ndarray, y: np.ndarray, z: np.ndarray) -> np.ndarray:
    """A smooth 3D source, 10 sin(pi x) sin(pi y) sin(pi z) (test input for 3D cases)."""
    return 10.0 * np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)


# ---------------------------------------------------------------------------
# Batched workload: 256 instances of -div((1 + u^3) grad u) = f_b, u in P1, w in P3.
# ---------------------------------------------------------------------------

@dataclass
class SineSource:
    """f(x, y) = sum_j A_j sin(p_j pi x) sin(q_j pi y)."""

    amps: np.ndarray
    p: np.ndarray
    q: np.ndarray

    def __call__(self, x: np.ndarray, y: np.ndarray) -> np.ndarray:
        out = np.zeros(np.broadcast(x, y).shape)
        for a, p, q in zip(self.amps, self.p, self.q):
            out = out + a * np.sin(p * np.pi * x) * np.sin(q * np.pi * y)
        return out


def batch_instances(count: int = 256, seed: int = 0, n_lo: int = 64, n_hi: int = 512,
                    modes: int = 8) -> list[tuple[int, SineSource]]:
    """Seeded (side length, source) pairs: n_b ~ U{n_lo..n_hi}, 8 sine modes,
    amplitudes ~ U(-1, 1), (p, q) ~ U{1..4}^2 (numpy PCG64, one stream)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        n = int(n_lo + rng.integers(0, n_hi - n_lo + 1))
        amps = rng.uniform(-1.0, 1.0, size=modes)
        p = rng.integers(1, 5, size=modes)
        q = rng.integers(1, 5, size=modes)
        out.append((n, SineSource(amps, p, q)))
    return out


# ---------------------------------------------------------------------------
# Adjoint workload: 64 instances on the 512 x 512 grid, source f = theta piecewise
# constant on a 16 x 16 grid of parameter cells, J = 0.5 ||u - u_d||^2 (nodal).
# ---------------------------------------------------------------------------

def adjoint_theta(index: int, grid: int = 16) -> np.ndarray:
    """theta_b ~ N(0, 1)^{grid x grid}, seeded by the instance index b."""
    rng = np.random.Generator(np.random.PCG64(index))
    return rng.standard_normal((grid, grid))


@dataclass
class TargetField:
    """u_d(x, y) = 0.1 sum_j c_j sin(p_j pi x) sin(q_j pi y)."""

    c: np.ndarray
    p: np.ndarray
    q: np.ndarray

    def __call__(self, x: np.ndarray, y: np.ndarray) -> np.ndarray:
        out = np.zeros(np.broadcast(x, y).shape)
        for c, p, q in zip(self.c, self.p, self.q):
            out = out + 0.1 * c * np.sin(p * np.pi * x) * np.sin(q * np.pi * y)
        return out


def adjoint_target(seed: int = 12345, modes: int = 4) -> TargetField:
    rng = np.random.Generator(np.random.PCG64(seed))
    c = rng.standard_normal(modes)
    p = rng.integers(1, 4, size=modes)
    q = rng.integers(1, 4, size=modes)
    return TargetField(c, p, q)


def param_cell_of_cells(mesh: Mesh, grid: int = 16) -> np.ndarray:
    """Index (row-major, y outer) of the grid x grid parameter cell that contains each
    mesh cell, located by the cell's vertex average.  The structured meshes align with
    the parameter grid whenever n is a multiple of grid."""
    cen = mesh.coords[mesh.cells].mean(axis=1)
    ix = np.minimum((cen[:, 0] * grid).astype(np.int64), grid - 1)
    iy = np.minimum((cen[:, 1] * grid).astype(np.int64), grid - 1)
    return (ix + grid * iy).astype(np.int32)


def cell_centroids(mesh: Mesh) -> np.ndarray:
    return mesh.coords[mesh.cells].mean(axis=1)


def random_vector(n: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """Seeded U(-scale, scale) vector (test inputs for the residual/Jacobian kernels)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-scale, scale, size=n)
