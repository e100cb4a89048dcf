"""Additive multigrid corrections as separate columns (Section 2.1, Section 2.2).

Hierarchy (Section 2.1): grids j = 0 (coarsest) ... J (finest); P_j maps grid
j-1 to grid j; R_j = P_j^T (no rescaling); coarse operators by Galerkin
products A_{j-1} = P_j^T A_j P_j.

Level operators:
  * smoother on every level j >= 1 (Eq. 2 with M_j = D_j / omega, damped
    Jacobi): starting from c_0 = 0, nu sweeps s <- s + omega D^{-1}(g - A s),
    D the diagonal, or for vector unknowns (elasticity) the block diagonal of
    the 3 x 3 node blocks;
  * the coarsest grid gets S_0 = A_0^{-1}, applied with a dense Cholesky factor.

MG(r) returns the block Z = [z^0 | ... | z^J] of Section 2.2 with
z^l = P_J ... P_{l+1} S_l (P_{l+1}^T ... P_J^T r), coarse column first.  The sum
of the columns is the additive MG correction of Eq. 3.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .operators import galerkin, prolongation, stencil_to_csr


def block_diag_inverse(A: sp.spmatrix, k: int) -> sp.csr_matrix:
    """Inverse of the block diagonal of A (k x k blocks of consecutive unknowns)."""
    n = A.shape[0]
    D = np.empty((n // k, k, k))
    for a in range(k):
        for b in range(k):
            D[:, a, b] = A[np.arange(a, n, k), np.arange(b, n, k)].A1
    nb = n // k
    return sp.bsr_matrix((np.linalg.inv(D), np.arange(nb), np.arange(nb + 1)), shape=(n, n)).tocsr()


class Hierarchy:
    """Nested structured grids below a fine operator given as stencil planes.

    ``n1`` is the number of unknown nodes per axis of an all-Dirichlet cube,
    or, with ``faces`` (bit 2a: low face of axis a is Dirichlet, bit 2a+1: the
    high face), the number of nodes per side of the fine grid is derived from
    ``nodes``.  ``ncomp`` unknowns per node (3 for elasticity) use the
    componentwise transfers and the block (ncomp x ncomp) Jacobi smoother."""

    def __init__(self, dim: int, n1, planes: np.ndarray, levels: int, nu: int = 2, omega: float = 2.0 / 3.0,
                 nodes: int | None = None, faces: int = 0x3F, ncomp: int = 1):
        if levels < 1:
            raise ValueError("levels >= 1")
        self.dim, self.nu, self.omega, self.ncomp = dim, nu, omega, ncomp
        flags = [((faces >> (2 * a)) & 1, (faces >> (2 * a + 1)) & 1) for a in range(dim)]
        lo = [f[0] for f in flags]
        hi = [f[1] for f in flags]
        self.lo = lo                                 # global coordinate of unknown 0 per axis
        if nodes is None:
            if faces != 0x3F:
                raise ValueError("give nodes when some faces are not Dirichlet")
            nodes = n1 + 2
        # nodes per side, fine -> coarse: N_{j-1} = (N_j + 1) / 2
        Ns = [nodes]
        for _ in range(levels - 1):
            if (Ns[-1] - 1) % 2:
                raise ValueError("grid cannot be coarsened")
            Ns.append((Ns[-1] + 1) // 2)
        Ns = Ns[::-1]                                # index j = 0 coarsest
        self.shape = [tuple(N - lo[a] - hi[a] for a in range(dim)) for N in Ns]
        self.n1 = [sh[0] for sh in self.shape]       # per-axis counts of a cube grid
        A = stencil_to_csr(dim, self.shape[-1], planes, ncomp)
        self.A = [None] * levels
        self.P = [None] * levels                     # P[j]: grid j-1 -> grid j (j >= 1)
        self.A[levels - 1] = A
        for j in range(levels - 1, 0, -1):
            self.P[j] = prolongation(dim, self.shape[j - 1], lo, hi, ncomp)
            self.A[j - 1] = galerkin(self.A[j], self.P[j])
        if ncomp == 1:
            self.Dinv = [1.0 / Aj.diagonal() for Aj in self.A]
        else:
            self.Dinv = [block_diag_inverse(Aj, ncomp) for Aj in self.A]
        A0 = self.A[0].toarray()
        self.chol = sla.cholesky(A0, lower=True)      # A_0 = L L^T; raises if not SPD
        self.levels = levels

    @property
    def J(self) -> int:
        return self.levels - 1

    def smooth(self, j: int, g: np.ndarray) -> np.ndarray:
        """Damped Jacobi, nu sweeps from zero (Eq. 2 with c_0 = 0); for vector
        unknowns D is the block diagonal of the node blocks."""
        s = np.zeros_like(g)
        for _ in range(self.nu):
            # M^{-1} = omega D^{-1} of Eq. 2, formed first, then applied
            if self.ncomp > 1:
                s = s + (self.omega * self.Dinv[j]) @ (g - self.A[j] @ s)
            else:
                s = s + self.omega * self.Dinv[j] * (g - self.A[j] @ s)
        return s

    def coarse_solve(self, g: np.ndarray) -> np.ndarray:
        """S_0 g = A_0^{-1} g by forward and backward substitution."""
        y = sla.solve_triangular(self.chol, g, lower=True)
        return sla.solve_triangular(self.chol.T, y, lower=False)

    def level_correction(self, j: int, g: np.ndarray) -> np.ndarray:
        return self.coarse_solve(g) if j == 0 else self.smooth(j, g)

    def restrict_all(self, r: np.ndarray) -> list:
        """R_L^j r for every grid j, by successive two-level restrictions."""
        rs = [None] * self.levels
        rs[self.J] = r
        for j in range(self.J, 0, -1):
            rs[j - 1] = self.P[j].T @ rs[j]
        return rs

    def prolong_to_fine(self, j: int, v: np.ndarray) -> np.ndarray:
        """P_j^L v, by successive two-level prolongations."""
        for i in range(j + 1, self.levels):
            v = self.P[i] @ v
        return v

    def mg_columns(self, r: np.ndarray) -> np.ndarray:
        """Z = [z^0 | ... | z^J], the per-level additive MG corrections of r."""
        rs = self.restrict_all(r)
        Z = np.empty((r.shape[0], self.levels))
        for j in range(self.levels):
            Z[:, j] = self.prolong_to_fine(j, self.level_correction(j, rs[j]))
        return Z

    def additive_mg(self, r: np.ndarray) -> np.ndarray:
        """B r of Eq. 3 (the sum of the level corrections)."""
        return self.mg_columns(r).sum(axis=1)
