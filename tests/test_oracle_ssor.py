"""Pins of the SSOR smoother and the multiplicative V-cycle oracle
(oracle/ssor.py): each is checked against its definition written out
independently (dense matrices, a plain lexicographic Gauss-Seidel on the
colour-permuted system, the closed-form SSOR splitting, the two-grid
correction), so that a wrong index, order, sign or transfer fails."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import mg as omg
from oracle import pcg as opcg
from oracle import ssor as oss
from paper_2402_12833_gb300 import problems as pb


def _hier(prob, levels=None):
    return omg.Hierarchy(prob.dim, None, prob.stencil, levels or prob.levels, nodes=prob.nodes, faces=prob.faces,
                         ncomp=prob.ncomp)


TINY = {
    "kappa2d_9": lambda: pb.diffusion_macro(2, 9, 5, rhs="normal", rhs_seed=1),
    "kappa2d_9_faces": lambda: pb.diffusion_faces(2, 9, 0x9, rhs_seed=2, kappa_seed=3),
    "kappa3d_5": lambda: pb.diffusion_macro(3, 5, 6, rhs="normal", rhs_seed=2),
    "elast_5": lambda: pb.elasticity_cantilever(nodes=5),
}


@pytest.mark.parametrize("name", list(TINY))
def test_colours_decouple(name):
    """No coupling inside a colour (block-diagonal over the node blocks for
    vector unknowns), and 2^dim colours in use."""
    prob = TINY[name]()
    H = _hier(prob)
    col = oss.colours(prob.dim, H.shape[-1], H.lo, prob.ncomp)
    A = H.A[-1].tocsr()
    for c in range(2 ** prob.dim):
        i = np.where(col == c)[0]
        assert i.size > 0
        sub = A[i][:, i].tocoo()
        node = i // prob.ncomp
        assert np.all(node[sub.row] == node[sub.col]), (name, c)


def _colour_perm(prob, H):
    col = oss.colours(prob.dim, H.shape[-1], H.lo, prob.ncomp)
    return np.argsort(col, kind="stable"), col


@pytest.mark.parametrize("name", ["kappa2d_9", "kappa3d_5", "kappa2d_9_faces"])
@pytest.mark.parametrize("omega", [1.0, 1.3])
def test_one_step_from_zero_is_the_ssor_splitting(name, omega):
    """x = one SSOR step from zero equals M^{-1} b with the SSOR splitting
    M = (D + w L) D^{-1} (D + w U) / (w (2 - w)) of the colour-ordered
    matrix (L, U its strict triangles)."""
    prob = TINY[name]()
    H = _hier(prob)
    perm, col = _colour_perm(prob, H)
    A = H.A[-1].toarray()
    Ap = A[np.ix_(perm, perm)]
    D = np.diag(np.diag(Ap))
    L, U = np.tril(Ap, -1), np.triu(Ap, 1)
    M = (D + omega * L) @ np.linalg.inv(D) @ (D + omega * U) / (omega * (2.0 - omega))
    b = np.random.default_rng(3).standard_normal(A.shape[0])
    S = oss.level_smoothers(H, omega)[-1]
    x = S.steps(b, np.zeros_like(b), 1)
    ref = np.empty_like(b)
    ref[perm] = np.linalg.solve(M, b[perm])
    assert np.allclose(x, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_forward_sweep_is_lexicographic_gauss_seidel_of_the_coloured_system():
    prob = TINY["kappa2d_9"]()
    H = _hier(prob)
    perm, col = _colour_perm(prob, H)
    A = H.A[-1].toarray()
    Ap = A[np.ix_(perm, perm)]
    rng = np.random.default_rng(4)
    b, x0 = rng.standard_normal(A.shape[0]), rng.standard_normal(A.shape[0])
    xp = x0[perm].copy()
    bp = b[perm]
    for i in range(len(xp)):   # textbook Gauss-Seidel, one unknown at a time
        xp[i] += (bp[i] - Ap[i] @ xp) / Ap[i, i]
    S = oss.level_smoothers(H)[-1]
    x = x0.copy()
    S.sweep(b, x, range(S.K))
    assert np.allclose(x[perm], xp, rtol=1e-12, atol=1e-12)


def _dense(op, n):
    return np.stack([op(e) for e in np.eye(n)], axis=1)


@pytest.mark.parametrize("name", list(TINY))
def test_ssor_steps_and_vcycle_are_symmetric(name):
    prob = TINY[name]()
    H = _hier(prob)
    Ss = oss.level_smoothers(H)
    n = H.A[-1].shape[0]
    S3 = _dense(lambda e: Ss[-1].steps(e, np.zeros_like(e), 3), n)
    assert np.abs(S3 - S3.T).max() <= 1e-12 * np.abs(S3).max()
    V = _dense(lambda e: oss.vcycle(H, Ss, e, 3), n)
    assert np.abs(V - V.T).max() <= 1e-12 * np.abs(V).max()
    assert np.linalg.eigvalsh(0.5 * (V + V.T)).min() > 0.0     # SPD: a CG preconditioner


def test_two_grid_cycle_without_smoothing_is_the_coarse_correction():
    """nu = 0: B_V = P A_c^{-1} P^T on two grids."""
    prob = pb.diffusion_macro(2, 9, 5, rhs="normal", rhs_seed=1)
    H = _hier(prob, levels=2)
    Ss = oss.level_smoothers(H)
    r = np.random.default_rng(6).standard_normal(H.A[-1].shape[0])
    P = H.P[1].toarray()
    Ac = P.T @ H.A[-1].toarray() @ P
    ref = P @ np.linalg.solve(Ac, P.T @ r)
    assert np.allclose(oss.vcycle(H, Ss, r, 0), ref, rtol=1e-12, atol=1e-13)


def test_smoothing_reduces_the_energy_error():
    """SSOR steps on A x = b from zero never increase ||x* - x||_A."""
    prob = pb.diffusion_macro(2, 17, 5, rhs="normal", rhs_seed=1)
    H = _hier(prob)
    S = oss.level_smoothers(H)[-1]
    A = H.A[-1]
    xs = np.linalg.solve(A.toarray(), prob.b)
    x = np.zeros_like(prob.b)
    prev = xs @ (A @ xs)
    for _ in range(6):
        S.steps(prob.b, x, 1)
        e = xs - x
        cur = e @ (A @ e)
        assert cur <= prev * (1 + 1e-12)
        prev = cur


def test_vcycle_pcg_solves_tiny_problems_and_beats_additive_pcg():
    """MG(V)-PCG converges to the dense solution; on Example 1's anisotropic
    operator it needs fewer iterations than additive MG-PCG with the same
    work per level (Section 3: 3 + 3 against 6 SSOR steps)."""
    prob = pb.example1(1e-3, nodes=33, levels=3)
    H = _hier(prob)
    Ss = oss.level_smoothers(H)
    A = H.A[-1]
    xv, kv, _ = opcg.pcg(A, prob.b, lambda r: oss.vcycle(H, Ss, r, 3), rtol=1e-10, maxit=500)
    xa, ka, _ = opcg.pcg(A, prob.b, lambda r: oss.additive_columns(H, Ss, r, 6).sum(axis=1), rtol=1e-10, maxit=500)
    xd = np.linalg.solve(A.toarray(), prob.b)
    assert np.linalg.norm(xv - xd) <= 1e-8 * np.linalg.norm(xd)
    assert np.linalg.norm(xa - xd) <= 1e-8 * np.linalg.norm(xd)
    assert kv < ka, (kv, ka)


def test_jacobi_vcycle_is_the_two_grid_error_propagation():
    """Two grids, V(nu, nu) with damped Jacobi: B_V = (I - E) A^-1 with the
    error propagation E = (I - W A)^nu (I - P A_c^-1 P^T A) (I - W A)^nu,
    W = w D^-1 (the product form, formed densely); B_V is symmetric."""
    from oracle import amg as oa
    prob = pb.example1(1e-2, nodes=17, levels=2)
    A = omg.Hierarchy(2, None, prob.stencil, 2, nodes=17).A[-1]
    H = oa.AlgebraicHierarchy(A, max_levels=2, coarse_size=8)
    assert H.levels == 2
    Sm = oss.jacobi_smoothers(H)
    n = A.shape[0]
    Ad = A.toarray()
    W = H.omegas[1] * np.diag(1.0 / np.diag(Ad))
    P = H.P[1].toarray()
    Ac = P.T @ Ad @ P
    S = np.eye(n) - W @ Ad
    nu = 3
    E = np.linalg.matrix_power(S, nu) @ (np.eye(n) - P @ np.linalg.solve(Ac, P.T @ Ad)) @ np.linalg.matrix_power(S, nu)
    B = (np.eye(n) - E) @ np.linalg.inv(Ad)
    Bv = np.stack([oss.vcycle(H, Sm, e, nu) for e in np.eye(n)], axis=1)
    assert np.abs(Bv - B).max() <= 1e-11 * np.abs(B).max()
    assert np.abs(Bv - Bv.T).max() <= 1e-11 * np.abs(Bv).max()
    assert np.linalg.eigvalsh(0.5 * (Bv + Bv.T)).min() > 0


# ---------------------------------------------------------------- planted mistakes
# Plants in the oracle (on the CPU) that a pin above must catch.

def test_planted_forward_only_steps_fail_symmetry_pin(monkeypatch):
    def forward_twice(self, b, x, k):     # the "backward" sweep repeats the forward order
        fwd = list(range(self.K))
        for _ in range(k):
            self.sweep(b, x, fwd)
            self.sweep(b, x, fwd)
        return x
    monkeypatch.setattr(oss.SSOR, "steps", forward_twice)
    with pytest.raises(AssertionError):
        test_ssor_steps_and_vcycle_are_symmetric(list(TINY)[0])


def test_planted_relaxation_squared_fails_splitting_pin(monkeypatch):
    def sweep_w2(self, b, x, order):      # omega^2 instead of omega in the update
        for c in order:
            i = self.idx[c]
            x[i] += self.omega ** 2 * (self.dinv[c] @ (b[i] - self.rows[c] @ x))
    monkeypatch.setattr(oss.SSOR, "sweep", sweep_w2)
    with pytest.raises(AssertionError):
        test_one_step_from_zero_is_the_ssor_splitting("kappa2d_9", 1.3)
