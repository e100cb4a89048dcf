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


def perturbed(v: np.ndarray, seed: int, rel: float) -> np.ndarray:
    """``v`` with every entry scaled by (1 + rel * g), g a seeded N(0,1) draw
    (seed stream offset so that it never repeats a right-hand side's draw)."""
    return v * (1.0 + rel * normal(7_000_000 + seed, v.size))


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


ALL_FACES = 0x3F


def face_flags(dim: int, faces: int):
    """Per axis (x first): (lo, hi) = 1 where that face is a Dirichlet face.
    Bit 2a of ``faces`` is the low face of axis a, bit 2a+1 the high face."""
    return [((faces >> (2 * a)) & 1, (faces >> (2 * a + 1)) & 1) for a in range(dim)]


def grid_shape(dim: int, nodes: int, faces: int = ALL_FACES):
    """Unknown nodes per axis (x first): nodes minus the Dirichlet faces."""
    return tuple(nodes - lo - hi for lo, hi in face_flags(dim, faces))


@dataclasses.dataclass
class Problem:
    """A structured Q1 problem: operator stencil, right-hand side and metadata.

    Scalar problems (``ncomp == 1``) use the stencil format described above.
    Vector problems (``ncomp == 3``, 3D elasticity) have unknowns
    ``i = a + 3 * node`` (component a fastest, nodes lexicographic over the
    unknown nodes, x fastest) and a stencil of shape ``(3 * 27, n)``: plane
    ``b * 27 + s`` holds, for every row unknown (node, a), the coefficient
    coupling it to unknown (node + offset_s, b)."""
    dim: int
    nodes: int               # nodes per side, boundary included
    levels: int              # grids in the nested hierarchy (coarsest has 5 nodes per side)
    stencil: np.ndarray      # (ncomp * 3**dim, n) float64, the format described above
    b: np.ndarray            # (n,) float64
    name: str = ""
    kappa: np.ndarray | None = None   # element coefficient field, if any
    ncomp: int = 1           # unknowns per node
    faces: int = ALL_FACES   # Dirichlet faces (bit 2a: low face of axis a, 2a+1: high face)

    @property
    def n1(self) -> int:
        if self.faces != ALL_FACES:
            raise AttributeError("n1 is defined for all-Dirichlet grids only; use shape")
        return self.nodes - 2

    @property
    def shape(self):
        return grid_shape(self.dim, self.nodes, self.faces)

    @property
    def n(self) -> int:
        return self.ncomp * int(np.prod(self.shape))


def assemble_diffusion(dim: int, nodes: int, kappa=None, kdiag=None, faces: int = ALL_FACES) -> np.ndarray:
    """Stencil planes (3**dim, n) of the Q1 diffusion operator with element
    coefficient field ``kappa`` (default 1) and anisotropy ``kdiag``; the
    nodes of the Dirichlet faces ``faces`` are eliminated, the other boundary
    nodes are unknowns (natural boundary condition)."""
    h = 1.0 / (nodes - 1)
    ne = nodes - 1
    coef = np.ones((ne,) * dim) if kappa is None else np.asarray(kappa, dtype=np.float64)
    ke = q1_stiffness(dim, h, kdiag)
    full = _assemble_full(dim, nodes, ke, coef)
    if faces == ALL_FACES:
        planes = _eliminate_dirichlet(dim, _interior(dim, full))
    else:
        planes = _eliminate_faces(dim, full, faces)
    return planes.reshape(3 ** dim, -1)


def diffusion_faces(dim: int, nodes: int, faces: int, rhs_seed: int, kappa_seed: int | None = None) -> Problem:
    """Diffusion with Dirichlet data on the faces in ``faces`` only (the
    others carry the natural condition), N(0,1) right-hand side."""
    kap = None if kappa_seed is None else macro_kappa(dim, nodes, kappa_seed)
    st = assemble_diffusion(dim, nodes, kappa=kap, faces=faces)
    n = int(np.prod(grid_shape(dim, nodes, faces)))
    return Problem(dim, nodes, levels_for_nodes(nodes), st, normal(rhs_seed, n), kappa=kap,
                   name=f"diffusion{dim}d_{nodes}_faces{faces:x}", faces=faces)


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


def anisotropic_2d(nodes: int, kxx: float, kyy: float = 1.0, levels: int | None = None) -> Problem:
    """Example 1's anisotropic operator K = diag(kxx, kyy) with f = 1 and zero
    Dirichlet data (the paper states neither; these are the readings)."""
    st = assemble_diffusion(2, nodes, kdiag=(kxx, kyy))
    b = load_vector(2, nodes, np.ones((nodes, nodes)))
    return Problem(2, nodes, levels_for_nodes(nodes) if levels is None else levels, st, b,
                   name=f"aniso2d_{nodes}_{kxx:g}")


def example1(kxx: float, nodes: int = 161, levels: int = 4) -> Problem:
    """Section 3, Example 1: the unit square with 160 x 160 elements and a
    4-grid hierarchy (20 x 20 elements on the coarsest grid), K = diag(kxx, 1)."""
    if (nodes - 1) % (1 << (levels - 1)):
        raise ValueError("nodes - 1 must be divisible by 2^(levels-1)")
    return anisotropic_2d(nodes, kxx, 1.0, levels)


def stencil_csr(prob: Problem):
    """The operator of a scalar stencil problem as a scipy CSR matrix (rows
    and columns over the unknowns, x fastest; sorted columns, the couplings
    to nodes outside the grid of unknowns left out), the input format of the
    algebraic hierarchy."""
    import scipy.sparse as sp
    if prob.ncomp != 1:
        raise ValueError("scalar problems only")
    shape = prob.shape
    dim = prob.dim
    n = int(np.prod(shape))
    idx = np.arange(n)
    coords = [(idx // int(np.prod(shape[:a]))) % shape[a] for a in range(dim)]
    rows, cols, vals = [], [], []
    for s_, off in enumerate(_offsets(dim)):
        ok = np.ones(n, dtype=bool)
        col = np.zeros(n, dtype=np.int64)
        stride = 1
        for a in range(dim):
            c = coords[a] + off[a]
            ok &= (c >= 0) & (c < shape[a])
            col += c * stride
            stride *= shape[a]
        v = prob.stencil[s_]
        keep = ok & (v != 0.0)
        rows.append(idx[keep])
        cols.append(col[keep])
        vals.append(v[keep])
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    A.sort_indices()
    return A


def fracture_kappa(nodes: int, kf: float, km: float = 1.0, delta: float = 1e-4, nfrac: int = 24,
                   seed: int = 11) -> np.ndarray:
    """Element coefficients of a seeded fracture network in the matrix of
    permeability km (the stand-in for Example 2, whose network is not
    published): nfrac straight fractures of thickness delta, centre uniform
    in [0.05, 0.95]^2, length uniform in [0.15, 0.5], direction uniform in
    [0, pi) (five uniforms per fracture, in that order).  Every element a
    fracture crosses (sampled at h/4 along it) takes the element-averaged
    permeability of a layer of thickness delta: arithmetic along a
    conducting fracture (kf >= km), km + (delta/h)(kf - km), harmonic across
    a blocking one, h / ((h - delta)/km + delta/kf)."""
    ne = nodes - 1
    h = 1.0 / ne
    kap = np.full((ne, ne), km)
    keff = km + (delta / h) * (kf - km) if kf >= km else h / ((h - delta) / km + delta / kf)
    u = uniform(seed, 5 * nfrac).reshape(nfrac, 5)
    for cx, cy, ul, ua, _ in u:
        cx, cy = 0.05 + 0.9 * cx, 0.05 + 0.9 * cy
        length, ang = 0.15 + 0.35 * ul, math.pi * ua
        m = int(math.ceil(length / (h / 4))) + 1
        t = np.linspace(-length / 2, length / 2, m)
        x, y = cx + t * math.cos(ang), cy + t * math.sin(ang)
        ok = (x >= 0) & (x < 1) & (y >= 0) & (y < 1)
        ix = np.minimum((x[ok] / h).astype(np.int64), ne - 1)
        iy = np.minimum((y[ok] / h).astype(np.int64), ne - 1)
        kap[iy, ix] = keff
    return kap


def fracture_network(kf: float, nodes: int = 545, km: float = 1.0, delta: float = 1e-4, nfrac: int = 24,
                     seed: int = 11) -> Problem:
    """Example 2's boundary value problem on a seeded network: -div(kappa
    grad p) = 0 on (0,1)^2, p = 1 on the right edge (its nodes eliminated),
    inflow flux g_N = 1 on the left edge, g_N = 0 on top and bottom.  The
    right-hand side is the consistent Neumann load (h per left-edge node, h/2
    at its two corners) plus the Dirichlet lift: the full operator has zero
    row sums, so -A_{I,D} 1 equals the row sums of the reduced operator.
    545 nodes per side give 545 x 544 = 296,480 unknowns (Example 2 has about
    3e5)."""
    kap = fracture_kappa(nodes, kf, km, delta, nfrac, seed)
    faces = 0x2                                   # the high x face (x = 1) is Dirichlet
    st = assemble_diffusion(2, nodes, kappa=kap, faces=faces)
    nx, ny = grid_shape(2, nodes, faces)
    h = 1.0 / (nodes - 1)
    g = np.zeros((ny, nx))
    g[:, 0] = h
    g[0, 0] = g[-1, 0] = h / 2
    b = g.reshape(-1) + st.sum(axis=0)
    levels = 1                                    # the deepest uniform hierarchy (>= 2 elements per side)
    while (nodes - 1) % (1 << levels) == 0 and ((nodes - 1) >> levels) >= 2:
        levels += 1
    return Problem(2, nodes, levels, st, b, name=f"fracture_{nodes}_kf{kf:g}", kappa=kap, faces=faces)


def net_init_params(seed: int = 7, chans=(2, 16, 16, 16, 1), taps: int = 9) -> np.ndarray:
    """Initial weights of the learned column's network, layer by layer
    W[co][ci][taps]: Kaiming-uniform draws U(-b, b), b = sqrt(6 / (taps ci)),
    from the splitmix64 uniforms above (float32); taps = 9 for the 3x3
    network of 2D problems, 27 for the 3x3x3 one of 3D vector problems."""
    parts = []
    for i in range(len(chans) - 1):
        b = np.sqrt(6.0 / (chans[i] * taps))
        u = uniform(seed * 1000 + i, chans[i + 1] * chans[i] * taps)
        parts.append((2.0 * u - 1.0) * b)
    return np.concatenate(parts).astype(np.float32)


def batch_sizes(count: int = 256, seed: int = 4, choices=(33, 65, 129, 257, 513)) -> list[int]:
    """Side lengths of a batch of 2D problems, drawn uniformly from ``choices``."""
    u = uniform(seed, count)
    return [choices[min(int(x * len(choices)), len(choices) - 1)] for x in u]


def batch_problem(index: int, nodes: int) -> Problem:
    """Problem ``index`` of the batched workload: own kappa seed and N(0,1) RHS."""
    return diffusion_macro(2, nodes, kappa_seed=10000 + index, rhs="normal", rhs_seed=20000 + index)


# ---------------------------------------------------------------------------
# 3D linear elasticity (vector Q1)
# ---------------------------------------------------------------------------

def q1_elasticity(h: float, E: float = 1.0, nu: float = 0.3) -> np.ndarray:
    """24 x 24 element stiffness of isotropic linear elasticity on a cube
    element of side h: sum over the 2x2x2 Gauss points of B^T D B |J| w.
    Unknown 3*a + c is component c of local node a (corner bits, x fastest).
    Strains in Voigt order (xx, yy, zz, yz, xz, xy) with engineering shears;
    D from the Lame constants lambda = E nu / ((1+nu)(1-2nu)), mu = E / (2(1+nu))."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[0, 0] = D[1, 1] = D[2, 2] = lam + 2.0 * mu
    D[3, 3] = D[4, 4] = D[5, 5] = mu
    gp = (0.5 - 0.5 / math.sqrt(3.0), 0.5 + 0.5 / math.sqrt(3.0))   # Gauss points on [0, 1]
    K = np.zeros((24, 24))
    for tz in gp:
        for ty in gp:
            for tx in gp:
                t = (tx, ty, tz)
                B = np.zeros((6, 24))
                for a in range(8):
                    bits = [(a >> k) & 1 for k in range(3)]
                    f = [t[k] if bits[k] else 1.0 - t[k] for k in range(3)]
                    df = [1.0 if bits[k] else -1.0 for k in range(3)]
                    # d N_a / d x_k = d N_a / d t_k / h
                    g = [df[k] * f[(k + 1) % 3] * f[(k + 2) % 3] / h for k in range(3)]
                    c = 3 * a
                    B[0, c + 0] = g[0]
                    B[1, c + 1] = g[1]
                    B[2, c + 2] = g[2]
                    B[3, c + 1], B[3, c + 2] = g[2], g[1]
                    B[4, c + 0], B[4, c + 2] = g[2], g[0]
                    B[5, c + 0], B[5, c + 1] = g[1], g[0]
                K += B.T @ D @ B * (h ** 3 / 8.0)          # |J| w = h^3 * (1/2)^3
    return K


def _eliminate_faces(dim: int, planes: np.ndarray, faces: int) -> np.ndarray:
    """Rows of the unknown nodes only (planes over all nodes in, numpy order
    [..., z, y, x]), with the couplings to Dirichlet nodes set to zero."""
    flags = face_flags(dim, faces)
    sl = tuple(slice(lo, planes.shape[-1 - ax] - hi) for ax, (lo, hi) in reversed(list(enumerate(flags))))
    out = planes[(Ellipsis,) + sl].copy()
    nplanes = 3 ** dim
    for q in range(out.shape[0]):
        off = _offsets(dim)[q % nplanes]
        for ax, o in enumerate(off):
            lo, hi = flags[ax]
            if (o < 0 and lo) or (o > 0 and hi):
                npax = out.ndim - 1 - ax
                idx = [slice(None)] * out.ndim
                idx[npax] = 0 if o < 0 else out.shape[npax] - 1
                out[(q,) + tuple(idx[1:])] = 0.0
    return out


def assemble_elasticity(nodes: int, E: float = 1.0, nu: float = 0.3, faces: int = 0x1) -> np.ndarray:
    """Stencil (81, 3 n_nodes) of Q1 elasticity on the unit cube with the
    Dirichlet (clamped) faces in ``faces`` (default: x = 0 only), in the
    vector format of :class:`Problem`."""
    h = 1.0 / (nodes - 1)
    ne = nodes - 1
    K = q1_elasticity(h, E, nu)
    full = np.zeros((3, 27, 3) + (nodes,) * 3)      # [b][s][a][z][y][x]
    for la in range(8):
        abits = [(la >> k) & 1 for k in range(3)]
        sl = tuple(slice(abits[k], abits[k] + ne) for k in (2, 1, 0))
        for lb in range(8):
            bbits = [(lb >> k) & 1 for k in range(3)]
            s = plane_index(tuple(bb - aa for aa, bb in zip(abits, bbits)))
            for a in range(3):
                for b in range(3):
                    full[(b, s, a) + sl] += K[3 * la + a, 3 * lb + b]
    full = full.reshape((81, 3) + (nodes,) * 3)
    # eliminate per (plane, component) and order rows as (node, component)
    planes = np.stack([_eliminate_faces(3, full[:, a], faces) for a in range(3)], axis=-1)   # [q][z][y][x][a]
    return planes.reshape(81, -1)


def elasticity_body_force(nodes: int, force=(0.0, 0.0, -1.0), faces: int = 0x1) -> np.ndarray:
    """b_(node, a) = force_a * integral of the node's hat function, for the
    unknown nodes (the consistent load of a constant body force)."""
    h = 1.0 / (nodes - 1)
    ne = nodes - 1
    full = _assemble_full(3, nodes, q1_mass(3, h), np.ones((ne,) * 3))
    vol = full.sum(axis=0)                                # sum_j M_ij = integral of N_i
    flags = face_flags(3, faces)
    sl = tuple(slice(lo, nodes - hi) for lo, hi in reversed(flags))
    vol = vol[sl].reshape(-1)
    return (vol[:, None] * np.asarray(force, dtype=np.float64)[None, :]).reshape(-1)


def elasticity_cantilever(nodes: int = 65, E: float = 1.0, nu: float = 0.3) -> Problem:
    """The unit cube clamped at x = 0 under the body force (0, 0, -1)."""
    return Problem(3, nodes, levels_for_nodes(nodes), assemble_elasticity(nodes, E, nu),
                   elasticity_body_force(nodes), name=f"elasticity3d_{nodes}", ncomp=3, faces=0x1)
