"""Seeded synthetic inputs for the additive-MG MPCG solver.

This module produces the *data* of Algorithm 1 (the matrix A, the right-hand
side b and an initial guess) for the model problem of Section 1: the diffusion
equation -div(K grad u) = f on the unit square or cube with homogeneous
Dirichlet data, discretised by Q1 finite elements on a uniform structured grid
(Eq. 1 and the FEM paragraph that follows it).  It holds none of the solver's
arithmetic (no transfers, smoothers, Galerkin products or Krylov steps); both
the CUDA path and the CPU oracle take their inputs from here.

Stencil format (the one the C-ABI's ``mg_operator`` carries)
-------------------------------------------------------------
A grid with ``N`` nodes per side (boundary included) has ``n1 = N - 2``
interior nodes per side and ``n = n1**d`` unknowns, numbered
lexicographically with x fastest.  The operator is a float64 array of shape
``(3**d, n)``: plane ``s`` holds, for every row, the coefficient that couples
the row's node to the node at offset ``(dx, dy[, dz])`` with
``s = (dx+1) + 3*(dy+1) [+ 9*(dz+1)]``.  Couplings to Dirichlet (boundary)
nodes are eliminated, so their entries are zero.

Randomness
----------
All random numbers come from splitmix64 (Steele, Lea, Flood 2014), with uniform
doubles built from the top 53 bits and normals by the Box-Muller transform, so
the arrays are identical on every platform and numpy version.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int) -> np.ndarray:
    """The first ``count`` outputs of splitmix64 started from state ``seed``."""
    with np.errstate(over="ignore"):
        state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + np.arange(1, count + 1, dtype=np.uint64) * _GOLDEN
        z = state
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, count: int) -> np.ndarray:
    """``count`` doubles uniform in [0, 1) (53-bit resolution)."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, count: int) -> np.ndarray:
    """``count`` standard normal doubles by the Box-Muller transform."""
    m = (count + 1) // 2
    u = uniform(seed, 2 * m)
    u1 = 1.0 - u[0::2]                     # (0, 1]: log is finite
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * m)
    out[0::2] = rad * np.cos(2.0 * np.pi * u2)
    out[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return out[:count]


# ---------------------------------------------------------------------------
# grids
# ---------------------------------------------------------------------------

def nodes_for_levels(levels: int) -> int:
    """Nodes per side of the finest grid of a ``levels``-grid hierarchy whose
    coarsest grid has 5 nodes per side (uniform refinement halves h)."""
    if levels < 1:
        raise ValueError("levels must be >= 1")
    return 4 * 2 ** (levels - 1) + 1


def levels_for_nodes(nodes: int) -> int:
    """Inverse of :func:`nodes_for_levels`; raises if ``nodes`` is not of that form."""
    q = nodes - 1
    if q < 4 or q & (q - 1):
        raise ValueError(f"{nodes} nodes per side is not 4*2^k+1")
    return int(math.log2(q)) - 1


def _offsets(dim: int):
    """All stencil offsets in plane order (x fastest), as tuples (dx, dy[, dz])."""
    out = []
    for s in range(3 ** dim):
        out.append(tuple((s // 3 ** k) % 3 - 1 for k in range(dim)))
    return out


def plane_index(offset) -> int:
    """Plane number of a stencil offset (dx, dy[, dz])."""
    return sum((o + 1) * 3 ** k for k, o in enumerate(offset))


# ---------------------------------------------------------------------------
# Q1 element matrices
# ---------------------------------------------------------------------------

def _q1_1d(h: float):
    k1 = np.array([[1.0, -1.0], [-1.0, 1.0]]) / h
    m1 = np.array([[2.0, 1.0], [1.0, 2.0]]) * (h / 6.0)
    return k1, m1


def q1_stiffness(dim: int, h: float, kdiag=None) -> np.ndarray:
    """Q1 element stiffness matrix of -div(K grad u) with K = diag(kdiag) on a
    cube element of side h.  Local nodes are numbered by their corner bits
    (x fastest).  Built from 1D P1 factors: sum_a k_a (x)_b (a==b ? K1 : M1)."""
    kdiag = np.ones(dim) if kdiag is None else np.asarray(kdiag, dtype=np.float64)
    k1, m1 = _q1_1d(h)
    nl = 2 ** dim
    ke = np.zeros((nl, nl))
    for a in range(nl):
        for b in range(nl):
            tot = 0.0
            for axis in range(dim):
                prod = kdiag[axis]
                for ax2 in range(dim):
                    ia, ib = (a >> ax2) & 1, (b >> ax2) & 1
                    prod *= (k1 if ax2 == axis else m1)[ia, ib]
                tot += prod
            ke[a, b] = tot
    return ke


def q1_mass(dim: int, h: float) -> np.ndarray:
    """Q1 element mass matrix, the tensor product of 1D P1 mass matrices."""
    _, m1 = _q1_1d(h)
    nl = 2 ** dim
    me = np.ones((nl, nl))
    for a in range(nl):
        for b in range(nl):
            for ax in range(dim):
                me[a, b] *= m1[(a >> ax) & 1, (b >> ax) & 1]
    return me


def _assemble_full(dim: int, nodes: int, elem_mat: np.ndarray, coef: np.ndarray) -> np.ndarray:
    """Assemble element matrices scaled by the element field ``coef`` (shape
    (nodes-1,)*dim, index order [z][y][x]) into stencil planes over ALL nodes:
    returns shape (3**dim,) + (nodes,)*dim."""
    shape = (nodes,) * dim
    planes = np.zeros((3 ** dim,) + shape)
    ne = nodes - 1
    nl = 2 ** dim
    for a in range(nl):
        abits = [(a >> ax) & 1 for ax in range(dim)]
        for b in range(nl):
            bbits = [(b >> ax) & 1 for ax in range(dim)]
            off = tuple(bb - aa for aa, bb in zip(abits, bbits))
            s = plane_index(off)
            # row node = element corner + a ; numpy index order is reversed (z, y, x)
            sl = tuple(slice(abits[ax], abits[ax] + ne) for ax in reversed(range(dim)))
            planes[(s,) + sl] += elem_mat[a, b] * coef
    return planes


def _interior(dim: int, full: np.ndarray) -> np.ndarray:
    inner = tuple(slice(1, -1) for _ in range(dim))
    return full[(Ellipsis,) + inner]


def _eliminate_dirichlet(dim: int, planes_int: np.ndarray) -> np.ndarray:
    """Zero the couplings of interior rows to boundary nodes."""
    n1 = planes_int.shape[-1]
    out = planes_int.copy()
    for s, off in enumerate(_offsets(dim)):
        for ax, o in enumerate(off):
            if o == 0:
                continue
            npax = dim - 1 - ax              # numpy axis of grid axis ``ax``
            idx = [slice(None)] * dim
            idx[npax] = 0 if o < 0 else n1 - 1
            out[(s,) + tuple(idx)] = 0.0
    return out


@dataclasses.dataclass
class Problem:
    """A structured Q1 problem: operator stencil, right-hand side and metadata."""
    dim: int
    nodes: int               # nodes per side, boundary included
    levels: int              # grids in the nested hierarchy (coarsest has 5 nodes per side)
    stencil: np.ndarray      # (3**dim, n) float64, the format described above
    b: np.ndarray            # (n,) float64
    name: str = ""
    kappa: np.ndarray | None = None   # element coefficient field, if any

    @property
    def n1(self) -> int:
        return self.nodes - 2

    @property
    def n(self) -> int:
        return self.n1 ** self.dim


def assemble_diffusion(dim: int, nodes: int, kappa=None, kdiag=None) -> np.ndarray:
    """Stencil planes (3**dim, n) of the Q1 diffusion operator with element
    coefficient field ``kappa`` (default 1) and anisotropy ``kdiag``."""
    h = 1.0 / (nodes - 1)
    ne = nodes - 1
    coef = np.ones((ne,) * dim) if kappa is None else np.asarray(kappa, dtype=np.float64)
    ke = q1_stiffness(dim, h, kdiag)
    full = _assemble_full(dim, nodes, ke, coef)
    planes = _eliminate_dirichlet(dim, _interior(dim, full))
    return planes.reshape(3 ** dim, -1)


def load_vector(dim: int, nodes: int, fvals: np.ndarray) -> np.ndarray:
    """b_i = sum_j M_ij f_j over all nodes j (boundary included), interior rows i."""
    h = 1.0 / (nodes - 1)
    ne = nodes - 1
    full = _assemble_full(dim, nodes, q1_mass(dim, h), np.ones((ne,) * dim))
    b = np.zeros((nodes - 2,) * dim)
    fpad = np.asarray(fvals, dtype=np.float64).reshape((nodes,) * dim)
    for s, off in enumerate(_offsets(dim)):
        src = tuple(slice(1 + off[ax], nodes - 1 + off[ax]) for ax in reversed(range(dim)))
        b += _interior(dim, full[s]) * fpad[src]
    return b.reshape(-1)


def node_coords(dim: int, nodes: int):
    """Meshgrid of node coordinates in [0,1], numpy order (z, y, x)."""
    t = np.linspace(0.0, 1.0, nodes)
    return np.meshgrid(*([t] * dim), indexing="ij")[::-1]   # returns x, y[, z] arrays shaped [z][y][x]


def manufactured_u(dim: int, nodes: int, interior: bool = True) -> np.ndarray:
    """Nodal values of u = prod_k sin(pi x_k)."""
    xs = node_coords(dim, nodes)
    u = np.ones_like(xs[0])
    for x in xs:
        u = u * np.sin(np.pi * x)
    return _interior(dim, u).reshape(-1) if interior else u


def macro_kappa(dim: int, nodes: int, seed: int, cells: int = 16, lo: float = -2.0, hi: float = 4.0) -> np.ndarray:
    """Piecewise-constant coefficient: log10(kappa) uniform in [lo, hi] on a
    cells^dim macro grid (one draw per macro cell, row-major with x fastest);
    element (i, j[, k]) takes macro cell floor(cells*i/(nodes-1)) per axis."""
    ne = nodes - 1
    vals = 10.0 ** (lo + (hi - lo) * uniform(seed, cells ** dim))
    vals = vals.reshape((cells,) * dim)                    # [z][y][x]
    m = (cells * np.arange(ne)) // ne
    return vals[np.ix_(*([m] * dim))]


# ---------------------------------------------------------------------------
# the benchmark workloads
# ---------------------------------------------------------------------------

def poisson_manufactured_2d(nodes: int = 65) -> Problem:
    """2D Poisson, b = M f_I with f = 2 pi^2 sin(pi x) sin(pi y)."""
    f = 2.0 * np.pi ** 2 * manufactured_u(2, nodes, interior=False)
    return Problem(2, nodes, levels_for_nodes(nodes), assemble_diffusion(2, nodes),
                   load_vector(2, nodes, f), name=f"poisson2d_manufactured_{nodes}")


def poisson_manufactured_3d(nodes: int) -> Problem:
    f = 3.0 * np.pi ** 2 * manufactured_u(3, nodes, interior=False)
    return Problem(3, nodes, levels_for_nodes(nodes), assemble_diffusion(3, nodes),
                   load_vector(3, nodes, f), name=f"poisson3d_manufactured_{nodes}")


def poisson_random(dim: int, nodes: int, seed: int) -> Problem:
    """Poisson with an N(0,1) right-hand side (one draw per interior DOF)."""
    st = assemble_diffusion(dim, nodes)
    n = (nodes - 2) ** dim
    return Problem(dim, nodes, levels_for_nodes(nodes), st, normal(seed, n),
                   name=f"poisson{dim}d_random_{nodes}_s{seed}")


def diffusion_macro(dim: int, nodes: int, kappa_seed: int, rhs: str = "ones", rhs_seed: int = 0) -> Problem:
    """Variable-coefficient diffusion with a seeded log-uniform macro-cell kappa.
    ``rhs='ones'`` gives b = M 1 (f = 1); ``rhs='normal'`` gives N(0,1) entries."""
    kap = macro_kappa(dim, nodes, kappa_seed)
    st = assemble_diffusion(dim, nodes, kappa=kap)
    if rhs == "ones":
        b = load_vector(dim, nodes, np.ones((nodes,) * dim))
    else:
        b = normal(rhs_seed, (nodes - 2) ** dim)
    return Problem(dim, nodes, levels_for_nodes(nodes), st, b, kappa=kap,
                   name=f"diffusion{dim}d_{nodes}_k{kappa_seed}")


def anisotropic_2d(nodes: int, kxx: float, kyy: float = 1.0) -> Problem:
    """Example 1's anisotropic operator K = diag(kxx, kyy) with f = 1."""
    st = assemble_diffusion(2, nodes, kdiag=(kxx, kyy))
    b = load_vector(2, nodes, np.ones((nodes, nodes)))
    return Problem(2, nodes, levels_for_nodes(nodes), st, b, name=f"aniso2d_{nodes}_{kxx:g}")


def net_init_params(seed: int = 7, chans=(2, 16, 16, 16, 1)) -> np.ndarray:
    """Initial weights of the learned column's 3x3 network, layer by layer
    W[co][ci][ky][kx]: Kaiming-uniform draws U(-b, b), b = sqrt(6 / (9 ci)),
    from the splitmix64 uniforms above (float32)."""
    parts = []
    for i in range(len(chans) - 1):
        b = np.sqrt(6.0 / (chans[i] * 9))
        u = uniform(seed * 1000 + i, chans[i + 1] * chans[i] * 9)
        parts.append((2.0 * u - 1.0) * b)
    return np.concatenate(parts).astype(np.float32)


def batch_sizes(count: int = 256, seed: int = 4, choices=(33, 65, 129, 257, 513)) -> list[int]:
    """Side lengths of a batch of 2D problems, drawn uniformly from ``choices``."""
    u = uniform(seed, count)
    return [choices[min(int(x * len(choices)), len(choices) - 1)] for x in u]


def batch_problem(index: int, nodes: int) -> Problem:
    """Problem ``index`` of the batched workload: own kappa seed and N(0,1) RHS."""
    return diffusion_macro(2, nodes, kappa_seed=10000 + index, rhs="normal", rhs_seed=20000 + index)
