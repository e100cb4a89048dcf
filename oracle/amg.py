"""An algebraic hierarchy built by smoothed aggregation (test infrastructure).

Section 2.1 allows the nested spaces to come from agglomeration instead of
nested meshes, and Section 3 (Example 2) builds them with an algebraic
multigrid setup (BoomerAMG, a third-party library).  This module stands in
for that setup with smoothed aggregation as published by Vanek, Mandel and
Brezina (Computing 56, 1996), restated here; the additive corrections on the
resulting hierarchy are those of ``oracle.mg`` unchanged (Eq. 2, Eq. 3).

Only tests/, the package's smoke entry point and bench.py's CPU baseline may
use it; the CUDA library shares no code with it.

Readings (the paper fixes none of them; the library uses the same):
  * strength: the classical signed measure, as the algebraic multigrid
    setup of Section 3 uses: j != i strongly influences i when
    -a_ij > 0 and -a_ij >= theta * max_{k != i} (-a_ik), theta = 0.4 on every
    grid; i and j are strongly coupled when either influences the other
    (the graph is symmetrised).  Positive couplings are weak.  (The scaled
    measure |a_ij| >= theta sqrt(a_ii a_jj) of smoothed aggregation cannot
    see the anisotropy of Example 1's Q1 operator: its corner couplings keep
    the ratio 1/8 at every k_xx, the ratio of every Poisson coupling.)
  * aggregation, unknowns visited in index order, strong neighbours in
    ascending column order:
      1. an unknown whose strong neighbours are all free starts an aggregate
         holding itself and them;
      2. a free unknown joins the aggregate of its first strong neighbour that
         was placed in step 1;
    an unknown with no strong neighbour belongs to no aggregate.  (An unknown
    passed over in step 1 has a neighbour placed in step 1, so every unknown
    with a strong neighbour is placed; the third pass of the published
    method never runs and is left out.)
  * tentative prolongator T: T[i, a] = 1 / sqrt(|aggregate a|) for i in a
    (orthonormal columns spanning the aggregate-wise constants);
  * smoothed prolongator P = (I - (w / rho) D^-1 A) T, w = 4/3, rho the
    Gershgorin bound max_i sum_j |a_ij| / |a_ii| of the spectral radius of
    D^-1 A (w = 0: plain aggregation, P = T);
  * Galerkin coarse operators A_c = P^T A P;
  * the damped Jacobi smoother of grid j takes the weight
    omega_j = min(omega, (4/3) / rho_j), rho_j the Gershgorin bound of
    D_j^-1 A_j, so that omega_j lambda_max(D_j^-1 A_j) <= 4/3 < 2 and every
    level correction stays symmetric positive definite (the coarse operators
    of smoothed aggregation couple more unknowns than the fine Q1 operator
    and can have lambda_max(D^-1 A) above 3, where omega = 2/3 would make
    the nu = 2 correction indefinite); on Q1 fine grids rho = 2 and
    omega_j = omega = 2/3;
  * coarsening stops at <= coarse_size unknowns, at max_levels grids, or
    when an aggregation yields no aggregate or does not reduce the count.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .mg import Hierarchy
from .operators import galerkin


def strength(A: sp.spmatrix, theta: float) -> sp.csr_matrix:
    """Boolean CSR of the strong couplings (diagonal excluded, symmetric)."""
    A = sp.csr_matrix(A)
    n = A.shape[0]
    rows = np.repeat(np.arange(n), np.diff(A.indptr))
    c = np.where(rows != A.indices, -A.data, -np.inf)      # -a_ij off the diagonal
    m = np.full(n, -np.inf)
    np.maximum.at(m, rows, c)                              # max_{k != i} (-a_ik)
    keep = (c > 0.0) & (c >= theta * m[rows])
    D = sp.csr_matrix((np.ones(int(keep.sum())), (rows[keep], A.indices[keep])), shape=(n, n))
    S = ((D + D.T) != 0).tocsr()
    S.sort_indices()
    return S


def aggregate(S: sp.csr_matrix) -> tuple[np.ndarray, int]:
    """The two aggregation passes over the strong-coupling graph S:
    aggregate index of every unknown (-1: none) and the aggregate count."""
    n = S.shape[0]
    nbrs = [S.indices[S.indptr[i]:S.indptr[i + 1]] for i in range(n)]
    agg = np.full(n, -1, dtype=np.int64)
    first = np.zeros(n, dtype=bool)        # placed by pass 1
    na = 0
    for i in range(n):                     # pass 1
        N = nbrs[i]
        if len(N) == 0 or agg[i] >= 0 or np.any(agg[N] >= 0):
            continue
        agg[i] = na
        agg[N] = na
        first[i] = True
        first[N] = True
        na += 1
    for i in range(n):                     # pass 2
        if agg[i] >= 0 or len(nbrs[i]) == 0:
            continue
        for j in nbrs[i]:
            if first[j]:
                agg[i] = agg[j]
                break
    return agg, na


def tentative(agg: np.ndarray, na: int) -> sp.csr_matrix:
    """T with T[i, agg[i]] = 1/sqrt(size of the aggregate); zero rows for
    unknowns outside every aggregate."""
    n = agg.shape[0]
    inside = agg >= 0
    size = np.bincount(agg[inside], minlength=na).astype(np.float64)
    rows = np.arange(n)[inside]
    T = sp.csr_matrix((1.0 / np.sqrt(size[agg[inside]]), (rows, agg[inside])), shape=(n, na))
    T.sort_indices()
    return T


def gershgorin_bound(A: sp.spmatrix) -> float:
    """max_i sum_j |a_ij| / |a_ii| >= the spectral radius of D^-1 A."""
    A = sp.csr_matrix(A)
    return float(np.max(np.asarray(abs(A).sum(axis=1)).ravel() / np.abs(A.diagonal())))


def smoothed_prolongator(A: sp.spmatrix, T: sp.spmatrix, w: float = 4.0 / 3.0) -> sp.csr_matrix:
    """P = (I - (w / rho) D^-1 A) T; w = 0 returns T."""
    T = sp.csr_matrix(T)
    if w == 0.0:
        return T
    A = sp.csr_matrix(A)
    s = w / gershgorin_bound(A)
    P = T - sp.diags(s / A.diagonal()) @ (A @ T)
    P = sp.csr_matrix(P)
    P.sort_indices()
    return P


class AlgebraicHierarchy(Hierarchy):
    """Grids j = 0 (coarsest) .. J (finest) built from the fine matrix alone;
    the level corrections, transfers and columns are those of the structured
    hierarchy (damped Jacobi nu sweeps from zero on every grid >= 1, exact
    coarsest solve, R_j = P_j^T, composite transfers by successive
    two-level transfers)."""

    def __init__(self, A: sp.spmatrix, theta: float = 0.4, w: float = 4.0 / 3.0,
                 max_levels: int = 12, coarse_size: int = 256, nu: int = 2, omega: float = 2.0 / 3.0):
        A = sp.csr_matrix(A, dtype=np.float64)
        A.sort_indices()
        As, Ps, aggs = [A], [], []
        while len(As) < max_levels and As[-1].shape[0] > coarse_size:
            Af = As[-1]
            S = strength(Af, theta)
            agg, na = aggregate(S)
            if na == 0 or na >= Af.shape[0]:
                break
            P = smoothed_prolongator(Af, tentative(agg, na), w)
            Ac = galerkin(Af, P)
            Ac.sort_indices()
            As.append(Ac)
            Ps.append(P)
            aggs.append(agg)
        # index j = 0 coarsest
        self.A = As[::-1]
        self.P = [None] + Ps[::-1]                  # P[j]: grid j-1 -> grid j
        self.aggregates = [None] + aggs[::-1]       # aggregates[j]: unknowns of grid j -> grid j-1
        self.levels = len(self.A)
        self.dim, self.nu, self.omega, self.ncomp = 0, nu, omega, 1
        self.Dinv = [1.0 / Aj.diagonal() for Aj in self.A]
        self.omegas = [min(omega, (4.0 / 3.0) / gershgorin_bound(Aj)) for Aj in self.A]
        self.chol = sla.cholesky(self.A[0].toarray(), lower=True)

    def smooth(self, j: int, g: np.ndarray) -> np.ndarray:
        """Damped Jacobi, nu sweeps from zero (Eq. 2, c_0 = 0) with the grid's
        weight omega_j."""
        s = np.zeros_like(g)
        for _ in range(self.nu):
            s = s + self.omegas[j] * self.Dinv[j] * (g - self.A[j] @ s)
        return s
