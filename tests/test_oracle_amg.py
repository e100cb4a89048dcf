"""Pins of the algebraic (smoothed-aggregation) hierarchy of the oracle.

Every expected value here is worked out by hand from the definitions in
oracle/amg.py's header (strength, the two aggregation passes, the tentative
and smoothed prolongators, Galerkin products) or is a property the
construction must have (orthonormal tentative columns, constants kept by the
smoothed prolongator of a pure-Neumann operator, lower energy of the smoothed
basis, the A-orthogonality of the exact coarse correction, anisotropy seen
by the strength measure).
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import amg as oa
from oracle import mpcg as ompcg
from paper_2402_12833_gb300 import problems as pb


def lap1d(n, neumann=False):
    A = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]).tolil()
    if neumann:
        A[0, 0] = 1.0
        A[n - 1, n - 1] = 1.0
    return A.tocsr()


def test_strength_hand_examples():
    A = sp.csr_matrix(np.array([[4, -1, -0.3, 0.5], [-1, 4, -2, 0], [-0.3, -2, 4, -1], [0.5, 0, -1, 3.0]]))
    # row maxima of -a_ik: 1, 2, 2, 1; threshold 0.4 of them; +0.5 is a positive coupling
    want = np.array([[0, 1, 0, 0], [1, 0, 1, 0], [0, 1, 0, 1], [0, 0, 1, 0]])
    assert np.array_equal(oa.strength(A, 0.4).toarray().astype(int), want)
    # 0 -> 1 is weak in row 0 (1 < 0.4 * 3) but 1 -> 0 is strong in row 1: symmetrised
    B = sp.csr_matrix(np.array([[4, -1, -3], [-1, 4, -0.2], [-3, -0.2, 5.0]]))
    want = np.array([[0, 1, 1], [1, 0, 0], [1, 0, 0]])
    assert np.array_equal(oa.strength(B, 0.4).toarray().astype(int), want)
    # theta = 0: every negative coupling is strong; theta > 1: none
    assert oa.strength(A, 0.0).nnz == 8
    assert oa.strength(A, 1.01).nnz == 0


def test_aggregation_of_paths():
    # pass 1 from node 0: {0,1}; node 2 sees the placed node 1; node 3 takes
    # {2,3,4}; node 6 takes {5,6,7}; node 9 takes {8,9}
    agg, na = oa.aggregate(oa.strength(lap1d(10), 0.4))
    assert na == 4 and agg.tolist() == [0, 0, 1, 1, 1, 2, 2, 2, 3, 3]
    # n = 6: node 5 is passed over in pass 1 and joins the aggregate of node 4 in pass 2
    agg, na = oa.aggregate(oa.strength(lap1d(6), 0.4))
    assert na == 2 and agg.tolist() == [0, 0, 1, 1, 1, 1]
    # an unknown with no strong neighbour is in no aggregate
    A = sp.block_diag([lap1d(4), sp.csr_matrix([[1.0]])]).tocsr()
    agg, na = oa.aggregate(oa.strength(A, 0.4))
    assert agg.tolist() == [0, 0, 1, 1, -1] and na == 2


def test_tentative_prolongator():
    agg = np.array([0, 0, 1, 1, 1, -1, 2])
    T = oa.tentative(agg, 3).toarray()
    assert np.allclose(T.T @ T, np.eye(3), atol=1e-15)
    # T T^T 1 is 1 on the aggregated unknowns, 0 elsewhere
    assert np.allclose(T @ (T.T @ np.ones(7)), [1, 1, 1, 1, 1, 0, 1], atol=1e-15)
    assert T[2, 1] == pytest.approx(1 / np.sqrt(3), abs=0)


def test_gershgorin_bound():
    assert oa.gershgorin_bound(lap1d(10)) == 2.0
    assert oa.gershgorin_bound(sp.diags([3.0, 5.0])) == 1.0


def test_smoothed_prolongator_hand_columns():
    """1D Dirichlet Laplacian, n = 10, aggregates {0,1}, {2,3,4}, ...: rho = 2,
    so P = (I - (2/3)(1/2) A) T:
    column 0 = (2/3, 2/3, 1/3, 0, ...)/sqrt 2,
    column 1 = (0, 1/3, 2/3, 1, 2/3, 1/3, 0, ...)/sqrt 3."""
    A = lap1d(10)
    agg, na = oa.aggregate(oa.strength(A, 0.4))
    P = oa.smoothed_prolongator(A, oa.tentative(agg, na)).toarray()
    c0 = np.array([2 / 3, 2 / 3, 1 / 3, 0, 0, 0, 0, 0, 0, 0]) / np.sqrt(2)
    c1 = np.array([0, 1 / 3, 2 / 3, 1, 2 / 3, 1 / 3, 0, 0, 0, 0]) / np.sqrt(3)
    assert np.allclose(P[:, 0], c0, atol=1e-15)
    assert np.allclose(P[:, 1], c1, atol=1e-15)
    # w = 0 is plain aggregation
    assert np.array_equal(oa.smoothed_prolongator(A, oa.tentative(agg, na), 0.0).toarray(),
                          oa.tentative(agg, na).toarray())


def test_smoothed_prolongator_keeps_constants_and_lowers_energy():
    # pure-Neumann operator: A 1 = 0, so (I - s D^-1 A) keeps the constant
    A = lap1d(12, neumann=True)
    agg, na = oa.aggregate(oa.strength(A, 0.4))
    T = oa.tentative(agg, na)
    P = oa.smoothed_prolongator(A, T)
    assert np.allclose(P @ (T.T @ np.ones(12)), np.ones(12), atol=1e-14)
    # 2D Poisson: each smoothed basis function has lower energy than the
    # tentative one (a sign error in the smoothing would raise it)
    p = pb.poisson_random(2, 17, 1)
    from oracle.operators import stencil_to_csr
    A2 = stencil_to_csr(2, 15, p.stencil)
    agg, na = oa.aggregate(oa.strength(A2, 0.4))
    T2 = oa.tentative(agg, na)
    P2 = oa.smoothed_prolongator(A2, T2)
    eT = np.einsum("ij,ij->j", T2.toarray(), (A2 @ T2).toarray())
    eP = np.einsum("ij,ij->j", P2.toarray(), (A2 @ P2).toarray())
    assert np.all(eP < eT)


def test_galerkin_of_pair_aggregates():
    """Plain aggregation in pairs of the 1D Laplacian: (T^T A T)_aa =
    (2 - 2 + 2)/2 = 1, (T^T A T)_{a,a+1} = -1/2."""
    from oracle.operators import galerkin
    n = 10
    agg = np.arange(n) // 2
    Ac = galerkin(lap1d(n), oa.tentative(agg, n // 2)).toarray()
    want = np.diag(np.ones(5)) - 0.5 * np.diag(np.ones(4), 1) - 0.5 * np.diag(np.ones(4), -1)
    assert np.allclose(Ac, want, atol=1e-15)


def _example1_matrix(kxx, nodes=41):
    from oracle import mg as omg
    prob = pb.example1(kxx, nodes=nodes, levels=3)
    return prob, omg.Hierarchy(2, None, prob.stencil, prob.levels, nodes=prob.nodes).A[-1]


def test_anisotropy_gives_line_aggregates():
    """k_xx = 1e-6: the x couplings are positive or a quarter of the y
    coupling, so every first aggregate lies in one grid column (same x)."""
    prob, A = _example1_matrix(1e-6)
    H = oa.AlgebraicHierarchy(A, coarse_size=16)
    agg = H.aggregates[H.J]
    n1 = prob.nodes - 2
    x = np.arange(A.shape[0]) % n1
    assert np.all(agg >= 0)
    for a in range(agg.max() + 1):
        assert len(set(x[agg == a])) == 1
    # isotropic: aggregates span both directions
    _, A1 = _example1_matrix(1.0)
    agg1 = oa.AlgebraicHierarchy(A1, coarse_size=16).aggregates[-1]
    assert any(len(set(x[agg1 == a])) > 1 for a in range(agg1.max() + 1))


def test_hierarchy_stopping_rules_and_coarse_operators():
    _, A = _example1_matrix(1e-2, nodes=81)
    H = oa.AlgebraicHierarchy(A, coarse_size=100)
    sizes = [a.shape[0] for a in H.A]
    assert sizes[0] <= 100 < sizes[1] and sizes == sorted(sizes)
    assert all(H.P[j].shape == (sizes[j], sizes[j - 1]) for j in range(1, H.levels))
    for Aj in H.A:                          # symmetric positive definite
        assert abs(Aj - Aj.T).max() <= 1e-14 * abs(Aj).max()
        assert np.linalg.eigvalsh(Aj.toarray()).min() > 0 if Aj.shape[0] <= 2000 else True
    Hm = oa.AlgebraicHierarchy(A, max_levels=2, coarse_size=10)
    assert Hm.levels == 2
    D = sp.diags(np.arange(1.0, 50.0)).tocsr()      # no couplings: one grid
    assert oa.AlgebraicHierarchy(D, coarse_size=10).levels == 1


def test_exact_coarse_column_is_a_projection():
    """Column 0 of MG(r) is P_0^L A_0^{-1} (P_0^L)^T r with A_0 the Galerkin
    operator of the composite prolongation, so (P_0^L)^T (r - A z^0) = 0."""
    _, A = _example1_matrix(1e-3, nodes=41)
    H = oa.AlgebraicHierarchy(A, coarse_size=40)
    assert H.levels >= 3
    r = np.random.default_rng(3).standard_normal(A.shape[0])
    z0 = H.mg_columns(r)[:, 0]
    n0 = H.A[0].shape[0]
    Pc = np.stack([H.prolong_to_fine(0, e) for e in np.eye(n0)], axis=1)
    assert np.abs(Pc.T @ (r - A @ z0)).max() <= 1e-10 * np.abs(Pc.T @ r).max()


def test_algebraic_hierarchy_handles_the_anisotropy():
    """On Example 1 with k_xx = 1e-6 the geometric hierarchy needs hundreds
    of MPCG iterations; the algebraic one follows the strong direction."""
    from oracle import mg as omg
    prob = pb.example1(1e-6, nodes=81, levels=4)
    Og = omg.Hierarchy(2, None, prob.stencil, prob.levels, nodes=prob.nodes)
    A = Og.A[-1]
    kg = ompcg.mpcg(A, prob.b, Og.mg_columns, rtol=1e-8, maxit=3000).iters
    H = oa.AlgebraicHierarchy(A, coarse_size=64)
    res = ompcg.mpcg(A, prob.b, H.mg_columns, rtol=1e-8, maxit=3000)
    assert np.linalg.norm(prob.b - A @ res.x) <= 1.01e-8 * np.linalg.norm(prob.b)
    assert res.iters * 4 < kg, (res.iters, kg)


def test_level_smoothers_stay_positive_definite():
    """Conducting fractures (k_f = 1e4): a coarse operator of the hierarchy
    has lambda_max(D^-1 A) above 3, where the fixed weight 2/3 would exceed 2;
    the grid weights keep omega_j lambda_max <= 4/3 on every grid, and on the
    Q1 fine grid (Gershgorin bound 2) omega_j is the given 2/3."""
    prob = pb.fracture_network(1e4, nodes=129)
    A = pb.stencil_csr(prob)
    H = oa.AlgebraicHierarchy(A)
    assert abs(H.omegas[H.J] - 2.0 / 3.0) <= 1e-15
    lam = []
    for j in range(H.levels):
        d = H.A[j].diagonal()
        At = (H.A[j].toarray() / np.sqrt(d)[:, None]) / np.sqrt(d)[None, :]
        lam.append(np.linalg.eigvalsh(At).max() if H.A[j].shape[0] <= 2500 else 2.0)
        assert H.omegas[j] * lam[-1] <= 4.0 / 3.0 + 1e-12, j
    assert max(lam) * 2.0 / 3.0 > 2.0 * 0.9    # the fixed weight would come close to, or pass, 2


# ---------------------------------------------------------------- planted mistakes
# Each plants a plausible mistake in the oracle (on the CPU) and shows that a
# pin above fails.

def test_planted_smoothing_sign_fails_energy_pin(monkeypatch):
    def plus(A, T, w=4.0 / 3.0):          # P = T + s D^-1 A T (wrong sign)
        T = sp.csr_matrix(T)
        A = sp.csr_matrix(A)
        s = w / oa.gershgorin_bound(A)
        return sp.csr_matrix(T + sp.diags(s / A.diagonal()) @ (A @ T))
    monkeypatch.setattr(oa, "smoothed_prolongator", plus)
    with pytest.raises(AssertionError):
        test_smoothed_prolongator_keeps_constants_and_lowers_energy()


def test_planted_unsymmetrised_strength_fails_hand_pin(monkeypatch):
    real = oa.strength

    def directed(A, theta):               # forgets the symmetrisation
        A = sp.csr_matrix(A)
        n = A.shape[0]
        rows = np.repeat(np.arange(n), np.diff(A.indptr))
        c = np.where(rows != A.indices, -A.data, -np.inf)
        m = np.full(n, -np.inf)
        np.maximum.at(m, rows, c)
        keep = (c > 0.0) & (c >= theta * m[rows])
        S = sp.csr_matrix((np.ones(int(keep.sum()), dtype=bool), (rows[keep], A.indices[keep])), shape=(n, n))
        S.sort_indices()
        return S
    monkeypatch.setattr(oa, "strength", directed)
    with pytest.raises(AssertionError):
        test_strength_hand_examples()
    monkeypatch.setattr(oa, "strength", real)


def test_planted_missing_second_pass_fails_path_pin(monkeypatch):
    def one_pass(S):
        n = S.shape[0]
        nbrs = [S.indices[S.indptr[i]:S.indptr[i + 1]] for i in range(n)]
        agg = np.full(n, -1, dtype=np.int64)
        na = 0
        for i in range(n):
            N = nbrs[i]
            if len(N) == 0 or agg[i] >= 0 or np.any(agg[N] >= 0):
                continue
            agg[i] = na
            agg[N] = na
            na += 1
        return agg, na
    monkeypatch.setattr(oa, "aggregate", one_pass)
    with pytest.raises(AssertionError):
        test_aggregation_of_paths()


def test_planted_unnormalised_tentative_fails_orthonormality_pin(monkeypatch):
    def ones(agg, na):                    # T[i, a] = 1 instead of 1/sqrt(|a|)
        n = agg.shape[0]
        inside = agg >= 0
        return sp.csr_matrix((np.ones(int(inside.sum())), (np.arange(n)[inside], agg[inside])), shape=(n, na))
    monkeypatch.setattr(oa, "tentative", ones)
    with pytest.raises(AssertionError):
        test_tentative_prolongator()
