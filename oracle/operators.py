"""Sparse operators of the structured hierarchy (FP64, scipy.sparse).

Section 2.1: nested Q1 spaces V_0 c ... c V_L on uniformly refined grids,
prolongations P_l^L, restrictions R_L^l = (P_l^L)^T with no extra scaling, and
composite transfers formed by successive two-level transfers.  The coarse
operators are Galerkin products A_{j-1} = P_j^T A_j P_j.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def stencil_to_csr(dim: int, n1: int, planes: np.ndarray) -> sp.csr_matrix:
    """The n x n matrix whose row i has entry planes[s][i] in the column of the
    node at offset s (plane numbering x fastest).  Entries pointing off the
    interior grid must be zero and are skipped."""
    n = n1 ** dim
    rows, cols, vals = [], [], []
    coords = np.indices((n1,) * dim).reshape(dim, -1)[::-1]   # (x, y[, z]) of every row
    idx = np.arange(n)
    for s in range(3 ** dim):
        off = [(s // 3 ** k) % 3 - 1 for k in range(dim)]
        nb = coords + np.array(off)[:, None]
        ok = np.all((nb >= 0) & (nb < n1), axis=0)
        col = np.zeros(n, dtype=np.int64)
        stride = 1
        for k in range(dim):
            col += nb[k] * stride
            stride *= n1
        v = planes[s]
        if np.any(v[~ok] != 0.0):
            raise ValueError("stencil couples to a node outside the interior grid")
        rows.append(idx[ok]); cols.append(col[ok]); vals.append(v[ok])
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    A.sum_duplicates()
    return A


def prolongation_1d(nc: int) -> sp.csr_matrix:
    """Linear interpolation from nc interior coarse nodes to 2*nc+1 interior
    fine nodes: coarse node I sits on fine node 2I+1; the two fine neighbours
    take half of it; boundary parents are zero (homogeneous Dirichlet)."""
    nf = 2 * nc + 1
    rows, cols, vals = [], [], []
    for I in range(nc):
        rows += [2 * I, 2 * I + 1, 2 * I + 2]
        cols += [I, I, I]
        vals += [0.5, 1.0, 0.5]
    return sp.csr_matrix((vals, (rows, cols)), shape=(nf, nc))


def prolongation(dim: int, nc: int) -> sp.csr_matrix:
    """Bilinear (2D) / trilinear (3D) interpolation between consecutive grids,
    the tensor product of 1D interpolations in lexicographic order (x fastest)."""
    p1 = prolongation_1d(nc)
    P = p1
    for _ in range(dim - 1):
        P = sp.kron(p1, P, format="csr")
    return P.tocsr()


def galerkin(A: sp.spmatrix, P: sp.spmatrix) -> sp.csr_matrix:
    """Coarse operator P^T A P."""
    return (P.T @ A @ P).tocsr()
