"""Algorithm 1 (additive MG multipreconditioned CG), FP64, step by step.

Notation follows Section 2.2: the block of preconditioned residuals Z_k holds
one column per level; alpha = (P_k^T A P_k)^{-1} (P_k^T r_k); x += P_k alpha;
r -= A P_k alpha; the next search block is Z_{k+1} A-orthogonalised against the
stored blocks of the truncation window (classical Gram-Schmidt: every
coefficient block is formed from Z_{k+1}, as the algorithm writes it).

Readings where the paper is silent (each is also used by the CUDA path):
  * the window holds the last m blocks (P_j, A P_j, G_j^+), newest first;
  * A P_{k+1} is formed by the same recurrence as P_{k+1} (one SpMM per step);
  * (P^T A P)^{-1} is a scaled pseudo-inverse with relative eigenvalue cutoff
    tau, after dropping every column i whose A-norm^2 after orthogonalisation
    is <= delta * (its A-norm^2 before), since P^T A P may become singular
    (Section 2.2) -- a dropped column is zeroed and takes no part;
  * stop when ||r_k||_2 <= rtol ||b||_2, tested after each update; the
    iteration count is the number of x updates.
"""
from __future__ import annotations

import dataclasses

import numpy as np


def scaled_pinv(G: np.ndarray, tau: float) -> np.ndarray:
    """G^+ = D V L^+ V^T D with D = diag(G_ii^{-1/2}) on the active columns
    (G_ii > 0), D G D = V L V^T, and L^+ keeping eigenvalues > tau * max."""
    c = G.shape[0]
    act = np.where(np.diag(G) > 0.0)[0]
    out = np.zeros_like(G)
    if act.size == 0:
        return out
    d = 1.0 / np.sqrt(np.diag(G)[act])
    Gh = d[:, None] * G[np.ix_(act, act)] * d[None, :]
    lam, V = np.linalg.eigh(Gh)
    lmax = lam.max()
    keep = lam > tau * lmax
    inv = np.zeros_like(lam)
    inv[keep] = 1.0 / lam[keep]
    sub = (V * inv[None, :]) @ V.T
    out[np.ix_(act, act)] = d[:, None] * sub * d[None, :]
    return out


@dataclasses.dataclass
class Result:
    x: np.ndarray
    iters: int
    res_hist: list          # ||r_k|| / ||b||, k = 0..iters
    alpha_hist: list        # alpha vectors, one per iteration
    dropped: list           # per block, the indices of dropped columns
    blocks: list = None     # (P_k, AP_k) per iteration if keep_blocks
    converged: bool = False


def mpcg(A, b, mg_columns, x0=None, rtol=1e-8, maxit=500, m=5, delta=1e-10, tau=1e-12,
         extra_column=None, keep_blocks=False) -> Result:
    """Solve A x = b by additive-MG MPCG.

    ``mg_columns(r)`` returns the n x c block of level corrections; if
    ``extra_column(r)`` is given its output is appended as one more column."""
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - A @ x
    nb = np.linalg.norm(b)
    res = [np.linalg.norm(r) / nb if nb > 0 else 0.0]
    out = Result(x, 0, res, [], [], [] if keep_blocks else None)
    if res[0] <= rtol:
        out.converged = True
        return out

    def corrections(r):
        Z = mg_columns(r)
        if extra_column is not None:
            Z = np.column_stack([Z, extra_column(r)])
        return Z

    def finish_block(P, AP, zAz):
        pAp = np.einsum("ij,ij->j", P, AP)
        drop = np.where(pAp <= delta * zAz)[0]
        P[:, drop] = 0.0
        AP[:, drop] = 0.0
        G = P.T @ AP
        G = 0.5 * (G + G.T)
        return P, AP, scaled_pinv(G, tau), drop.tolist()

    Z = corrections(r)
    AZ = A @ Z
    zAz = np.einsum("ij,ij->j", Z, AZ)
    P, AP, Gp, dr = finish_block(Z.copy(), AZ.copy(), zAz)
    out.dropped.append(dr)
    window = [(P, AP, Gp)]
    k = 0
    while True:
        g = P.T @ r
        alpha = Gp @ g
        x += P @ alpha
        r -= AP @ alpha
        k += 1
        res.append(np.linalg.norm(r) / nb)
        out.alpha_hist.append(alpha)
        if keep_blocks:
            out.blocks.append((P.copy(), AP.copy()))
        if res[-1] <= rtol or k >= maxit:
            break
        Z = corrections(r)
        AZ = A @ Z
        zAz = np.einsum("ij,ij->j", Z, AZ)
        Pn, APn = Z.copy(), AZ.copy()
        for Pj, APj, Gpj in reversed(window):
            beta = Gpj @ (APj.T @ Z)
            Pn -= Pj @ beta
            APn -= APj @ beta
        P, AP, Gp, dr = finish_block(Pn, APn, zAz)
        out.dropped.append(dr)
        window.append((P, AP, Gp))
        if len(window) > m:
            window.pop(0)
    out.x, out.iters = x, k
    out.converged = res[-1] <= rtol
    return out
