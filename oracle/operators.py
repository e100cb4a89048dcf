"""Sparse operators of the structured hierarchy (FP64, scipy.sparse).

Section 2.1: nested Q1 spaces V_0 c ... c V_L on uniformly refined grids,
prolongations P_l^L, restrictions R_L^l = (P_l^L)^T with no extra scaling, and
composite transfers formed by successive two-level transfers.  The coarse
operators are Galerkin products A_{j-1} = P_j^T A_j P_j.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def stencil_to_csr(dim: int, shape, planes: np.ndarray, ncomp: int = 1) -> sp.csr_matrix:
    """The matrix whose row (node, a) has entry planes[b * 3**dim + s][row] in
    the column of unknown (node + offset_s, b) (plane numbering x fastest;
    rows and columns a + ncomp * node, nodes lexicographic, x fastest).
    ``shape`` is the number of unknown nodes per axis (x first), or one int for
    a cube.  Entries pointing off the grid of unknowns must be zero and are
    skipped."""
    shape = (shape,) * dim if np.isscalar(shape) else tuple(shape)
    nn = int(np.prod(shape))
    n = ncomp * nn
    S = 3 ** dim
    coords = np.indices(shape[::-1]).reshape(dim, -1)[::-1]    # (x, y[, z]) of every node
    rows, cols, vals = [], [], []
    for b in range(ncomp):
        for s in range(S):
            off = [(s // 3 ** k) % 3 - 1 for k in range(dim)]
            nb = coords + np.array(off)[:, None]
            ok = np.all((nb >= 0) & (nb < np.array(shape)[:, None]), axis=0)
            node = np.zeros(nn, dtype=np.int64)
            stride = 1
            for k in range(dim):
                node += nb[k] * stride
                stride *= shape[k]
            v = planes[b * S + s].reshape(nn, ncomp)            # [node][a]
            if np.any(v[~ok] != 0.0):
                raise ValueError("stencil couples to a node outside the grid of unknowns")
            for a in range(ncomp):
                rows.append(np.arange(nn)[ok] * ncomp + a)
                cols.append(node[ok] * ncomp + b)
                vals.append(v[ok, a])
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    A.sum_duplicates()
    return A


def prolongation_1d(nc: int, lo: int = 1, hi: int = 1) -> sp.csr_matrix:
    """Linear interpolation along one axis between consecutive grids.  The
    coarse grid has nc + lo + hi nodes, of which the first (lo = 1) and the
    last (hi = 1) are Dirichlet nodes and not unknowns; the fine grid has
    twice the intervals.  Coarse node G sits on fine node 2G; a fine node
    between two coarse nodes takes half of each; Dirichlet parents are zero."""
    Nc = nc + lo + hi
    Nf = 2 * Nc - 1
    nf = Nf - lo - hi
    rows, cols, vals = [], [], []
    for c in range(nc):
        G = c + lo                       # global coarse index
        for g, w in ((2 * G - 1, 0.5), (2 * G, 1.0), (2 * G + 1, 0.5)):
            f = g - lo                   # fine unknown index
            if 0 <= f < nf:
                rows.append(f); cols.append(c); vals.append(w)
    return sp.csr_matrix((vals, (rows, cols)), shape=(nf, nc))


def prolongation(dim: int, nc, lo=None, hi=None, ncomp: int = 1) -> sp.csr_matrix:
    """Bilinear (2D) / trilinear (3D) interpolation between consecutive grids,
    the tensor product of 1D interpolations in lexicographic order (x
    fastest); vector unknowns (a + ncomp * node) interpolate componentwise.
    ``nc``: coarse unknown nodes per axis (x first, or one int for a cube);
    ``lo``/``hi``: per-axis Dirichlet flags of the low and high faces
    (default: all faces Dirichlet)."""
    nc = (nc,) * dim if np.isscalar(nc) else tuple(nc)
    lo = (1,) * dim if lo is None else tuple(lo)
    hi = (1,) * dim if hi is None else tuple(hi)
    P = None
    for ax in range(dim):
        p1 = prolongation_1d(nc[ax], lo[ax], hi[ax])
        P = p1 if P is None else sp.kron(p1, P, format="csr")
    if ncomp > 1:
        P = sp.kron(P, sp.identity(ncomp), format="csr")
    return P.tocsr()


def galerkin(A: sp.spmatrix, P: sp.spmatrix) -> sp.csr_matrix:
    """Coarse operator P^T A P."""
    return (P.T @ A @ P).tocsr()
