"""SSOR smoothing and the multiplicative V-cycle, the paper's comparison
setup (Section 3: symmetric successive over-relaxation as the smoother, 3
pre- and 3 post-smoothing steps in the multiplicative MG, 6 steps on each
level for the additive MG; the multiplicative MG preconditions CG).  The
V-cycle also takes damped-Jacobi smoothers (class Jacobi): the colouring
of the SSOR reading needs grid coordinates, which an algebraic hierarchy
does not have; Jacobi is self-adjoint, so V(nu, nu) with it stays a
symmetric preconditioner.

This is test infrastructure: only tests/, the package's smoke entry point
and bench.py's CPU baseline may use it; the CUDA path shares nothing with it.

Readings (the paper is silent on each; the CUDA path uses the same):
  * ordering: the unknowns are split into 2^dim colours by the parity of
    their global node coordinates (x, y[, z]); no two unknowns of one colour
    are coupled by the 3^dim-point stencil (for vector unknowns the
    components of a node share its colour and are updated together with
    their 3 x 3 node block), so each colour is updated at once, Gauss-Seidel
    across colours; a forward sweep takes colours 0 .. K-1, a backward sweep
    K-1 .. 0, and one SSOR step is a forward then a backward sweep;
  * relaxation omega = 1 (symmetric Gauss-Seidel) unless given;
  * smoothing starts from zero (c_0 = 0, as for the Jacobi smoother of
    Eq. 2), so k SSOR steps are a fixed symmetric operator;
  * V-cycle: nu steps of pre-smoothing, the defect, restriction P^T, the
    cycle on the coarser grid for the defect, prolongation P and correction,
    nu steps of post-smoothing; the coarsest grid is solved exactly.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def colours(dim: int, shape, lo, ncomp: int = 1) -> np.ndarray:
    """Colour of every unknown (x fastest, component fastest for vectors):
    sum over the axes of parity(global coordinate) << axis."""
    axes = [np.arange(shape[a]) + lo[a] for a in range(dim)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")[::-1]   # grids[a] holds the a-coordinate
    col = np.zeros(grids[0].shape, dtype=np.int64)
    for a in range(dim):
        col |= (grids[a] & 1) << a
    col = col.reshape(-1)
    return np.repeat(col, ncomp)


class SSOR:
    """Multicoloured SSOR on one grid: A (CSR), the inverses of the diagonal
    (scalar) or of the node blocks (vector), colour index sets."""

    def __init__(self, A: sp.spmatrix, col: np.ndarray, Dinv: sp.spmatrix, omega: float = 1.0):
        self.A = sp.csr_matrix(A)
        self.omega = omega
        self.K = int(col.max()) + 1 if col.size else 0
        self.idx = [np.where(col == c)[0] for c in range(self.K)]
        self.rows = [self.A[i] for i in self.idx]
        Dinv = sp.csr_matrix(Dinv)
        self.dinv = [Dinv[i][:, i] for i in self.idx]

    def sweep(self, b: np.ndarray, x: np.ndarray, order) -> None:
        """One Gauss-Seidel sweep over the colours in ``order``, in place:
        x_c += omega D_c^{-1} (b_c - A_c x)."""
        for c in order:
            i = self.idx[c]
            x[i] += self.omega * (self.dinv[c] @ (b[i] - self.rows[c] @ x))

    def steps(self, b: np.ndarray, x: np.ndarray, k: int) -> np.ndarray:
        """k SSOR steps (forward then backward sweep each) from x, in place."""
        fwd = list(range(self.K))
        for _ in range(k):
            self.sweep(b, x, fwd)
            self.sweep(b, x, fwd[::-1])
        return x


class Jacobi:
    """Damped Jacobi on one grid as a smoother with a starting iterate:
    k sweeps x <- x + w D^-1 (b - A x), in place (Eq. 2's smoother)."""

    def __init__(self, A: sp.spmatrix, dinv: np.ndarray, w: float):
        self.A = sp.csr_matrix(A)
        self.dinv = dinv
        self.w = w

    def steps(self, b: np.ndarray, x: np.ndarray, k: int) -> np.ndarray:
        for _ in range(k):
            x += self.w * self.dinv * (b - self.A @ x)
        return x


def jacobi_smoothers(H):
    """The damped-Jacobi smoother of every grid of H with the grid's weight
    (H.omegas where the hierarchy sets one per grid, else H.omega)."""
    ws = getattr(H, "omegas", None) or [H.omega] * H.levels
    return [Jacobi(H.A[j], H.Dinv[j], ws[j]) for j in range(H.levels)]


def level_smoothers(H, omega: float = 1.0):
    """SSOR of every grid of the oracle hierarchy H (mg.Hierarchy)."""
    out = []
    for j in range(H.levels):
        col = colours(H.dim, H.shape[j], H.lo, H.ncomp)
        dinv = H.Dinv[j] if H.ncomp > 1 else sp.diags(H.Dinv[j])
        out.append(SSOR(H.A[j], col, dinv, omega))
    return out


def additive_columns(H, smoothers, r: np.ndarray, steps: int) -> np.ndarray:
    """Z = [z^0 | ... | z^J] of Section 2.2 with SSOR^steps from zero as the
    level correction on grids j >= 1 and the exact solve on grid 0."""
    rs = H.restrict_all(r)
    Z = np.empty((r.shape[0], H.levels))
    for j in range(H.levels):
        if j == 0:
            s = H.coarse_solve(rs[0])
        else:
            s = smoothers[j].steps(rs[j], np.zeros_like(rs[j]), steps)
        Z[:, j] = H.prolong_to_fine(j, s)
    return Z


def vcycle(H, smoothers, r: np.ndarray, nu: int, j: int | None = None) -> np.ndarray:
    """B_V r: one multiplicative V(nu, nu) cycle from zero on grid j (finest
    by default) for the right-hand side r."""
    if j is None:
        j = H.J
    if j == 0:
        return H.coarse_solve(r)
    x = smoothers[j].steps(r, np.zeros_like(r), nu)
    d = r - H.A[j] @ x
    x += H.P[j] @ vcycle(H, smoothers, H.P[j].T @ d, nu, j - 1)
    return smoothers[j].steps(r, x, nu)
