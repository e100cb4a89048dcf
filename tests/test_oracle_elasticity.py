"""Pins of the elasticity inputs and of the oracle on vector unknowns.

The 3D elasticity configuration (unit cube, Q1 hexahedra, E = 1, nu = 0.3,
clamped at x = 0, body force (0, 0, -1)) is problem data; the oracle applies
the same multigrid method to it with componentwise transfers and a 3 x 3
block Jacobi smoother.  The checks below come from mechanics and linear
algebra, not from the code under test: rigid-body modes, the constant-strain
energy, the patch test, global equilibrium, a brute-force element assembly,
Galerkin = rediscretisation, the block-Jacobi closed form and dense solves.
"""
import numpy as np
import pytest

from oracle import mg as omg
from oracle import mpcg as ompcg
from oracle.operators import prolongation, prolongation_1d, stencil_to_csr
from paper_2402_12833_gb300 import problems as pb

E, NU = 1.0, 0.3


def _elastic_D():
    """Isotropic elasticity matrix (Voigt xx, yy, zz, yz, xz, xy, engineering
    shears) as the inverse of the compliance written with E and nu."""
    C = np.zeros((6, 6))
    C[:3, :3] = -NU / E
    for i in range(3):
        C[i, i] = 1.0 / E
        C[3 + i, 3 + i] = 2.0 * (1.0 + NU) / E           # 1 / G
    return np.linalg.inv(C)


def _rigid_modes(X):
    """Six rigid-body displacement fields at points X (npts, 3), flattened (a fastest)."""
    modes = []
    for a in range(3):
        u = np.zeros_like(X); u[:, a] = 1.0
        modes.append(u.reshape(-1))
    for w in np.eye(3):
        modes.append(np.cross(w, X).reshape(-1))
    return np.array(modes)


def _corners(h):
    return np.array([[(a >> 0) & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], dtype=float) * h


def test_element_matrix_kernel_is_the_rigid_body_modes():
    h = 0.25
    K = pb.q1_elasticity(h, E, NU)
    assert np.abs(K - K.T).max() < 1e-15 * np.abs(K).max()
    ev = np.linalg.eigvalsh(K)
    assert np.all(ev > -1e-14 * ev[-1])
    assert np.sum(ev < 1e-12 * ev[-1]) == 6
    R = _rigid_modes(_corners(h) + 0.3)                  # any origin
    assert np.abs(K @ R.T).max() < 1e-13 * np.abs(K).max()


def test_constant_strain_energy():
    """u = G x (G any 3x3 matrix): u^T K u = h^3 eps^T D eps with eps the Voigt strain."""
    h = 0.5
    K = pb.q1_elasticity(h, E, NU)
    rng = np.random.default_rng(3)
    Gm = rng.standard_normal((3, 3))
    u = (_corners(h) @ Gm.T).reshape(-1)
    eps_t = 0.5 * (Gm + Gm.T)
    eps = np.array([eps_t[0, 0], eps_t[1, 1], eps_t[2, 2], 2 * eps_t[1, 2], 2 * eps_t[0, 2], 2 * eps_t[0, 1]])
    assert np.isclose(u @ K @ u, h ** 3 * eps @ _elastic_D() @ eps, rtol=1e-13)


def _dense_brute_force(nodes, faces):
    """Element-by-element scatter of q1_elasticity into a dense matrix over
    all nodes, then removal of the Dirichlet nodes (unknowns a + 3 node)."""
    h = 1.0 / (nodes - 1)
    K = pb.q1_elasticity(h, E, NU)
    N = nodes
    A = np.zeros((3 * N ** 3, 3 * N ** 3))
    for ez in range(N - 1):
        for ey in range(N - 1):
            for ex in range(N - 1):
                gn = [(ex + (a & 1)) + N * (ey + ((a >> 1) & 1)) + N * N * (ez + ((a >> 2) & 1)) for a in range(8)]
                dofs = np.array([3 * g + c for g in gn for c in range(3)])
                A[np.ix_(dofs, dofs)] += K
    keep = []
    flags = pb.face_flags(3, faces)
    for z in range(N):
        for y in range(N):
            for x in range(N):
                c = (x, y, z)
                if any((flags[a][0] and c[a] == 0) or (flags[a][1] and c[a] == N - 1) for a in range(3)):
                    continue
                keep.append((x + N * y + N * N * z))
    idx = np.array([3 * g + c for g in keep for c in range(3)])
    return A[np.ix_(idx, idx)]


@pytest.mark.parametrize("faces", [0x1, 0x3F, 0x0, 0x5])
def test_stencil_equals_brute_force_assembly(faces):
    nodes = 5
    st = pb.assemble_elasticity(nodes, E, NU, faces=faces)
    A = stencil_to_csr(3, pb.grid_shape(3, nodes, faces), st, ncomp=3).toarray()
    ref = _dense_brute_force(nodes, faces)
    assert A.shape == ref.shape
    assert np.abs(A - ref).max() < 1e-14 * np.abs(ref).max()


def test_patch_test_and_rigid_modes_of_the_free_assembly():
    """No Dirichlet faces: rigid modes give zero force everywhere, and a linear
    field gives zero force at every node off the boundary."""
    nodes = 7
    A = stencil_to_csr(3, (nodes,) * 3, pb.assemble_elasticity(nodes, E, NU, faces=0), ncomp=3)
    t = np.linspace(0.0, 1.0, nodes)
    Z, Y, X = np.meshgrid(t, t, t, indexing="ij")
    P = np.stack([X.reshape(-1), Y.reshape(-1), Z.reshape(-1)], axis=1)
    R = _rigid_modes(P)
    assert np.abs(A @ R.T).max() < 1e-12 * abs(A).max()
    Gm = np.random.default_rng(4).standard_normal((3, 3))
    f = (A @ (P @ Gm.T).reshape(-1)).reshape(nodes, nodes, nodes, 3)
    assert np.abs(f[1:-1, 1:-1, 1:-1]).max() < 1e-12 * abs(A).max()


def test_body_force_total_and_global_equilibrium():
    """sum b_z = -(1 - h/2) (the clamped face's hat functions carry half a slab);
    the solution's reaction at the clamped face balances the whole load."""
    nodes = 9
    h = 1.0 / (nodes - 1)
    prob = pb.elasticity_cantilever(nodes)
    assert np.isclose(prob.b[2::3].sum(), -(1.0 - h / 2.0), rtol=1e-13)
    assert np.all(prob.b[0::3] == 0.0) and np.all(prob.b[1::3] == 0.0)
    A = stencil_to_csr(3, prob.shape, prob.stencil, ncomp=3)
    u = np.linalg.solve(A.toarray(), prob.b)
    full = stencil_to_csr(3, (nodes,) * 3, pb.assemble_elasticity(nodes, E, NU, faces=0), ncomp=3)
    ufull = np.zeros((nodes, nodes, nodes, 3))
    ufull[:, :, 1:, :] = u.reshape(nodes, nodes, nodes - 1, 3)
    fint = (full @ ufull.reshape(-1)).reshape(nodes, nodes, nodes, 3)
    load = pb.elasticity_body_force(nodes, faces=0).reshape(nodes, nodes, nodes, 3)
    reaction = fint[:, :, 0, :] - load[:, :, 0, :]
    assert np.allclose(reaction.sum(axis=(0, 1)), [0.0, 0.0, 1.0], atol=1e-10)
    assert np.abs(fint[:, :, 1:] - load[:, :, 1:]).max() < 1e-10


@pytest.mark.parametrize("lo,hi", [(1, 0), (0, 1), (0, 0), (1, 1)])
def test_prolongation_with_free_faces_interpolates(lo, hi):
    """P c evaluates the coarse Q1 function at the fine unknown nodes, with
    Dirichlet parents zero, for every combination of face types."""
    Nc = 5
    nc = Nc - lo - hi
    P = prolongation_1d(nc, lo, hi).toarray()
    Nf = 2 * Nc - 1
    xc = np.arange(Nc) / (Nc - 1)
    xf = np.arange(Nf) / (Nf - 1)
    B = np.maximum(0.0, 1.0 - np.abs((xf[:, None] - xc[None, :]) * (Nc - 1)))
    B = B[lo:Nf - hi, lo:Nc - hi]
    assert np.allclose(P, B, atol=1e-15)
    # the 3D vector prolongation is the componentwise tensor product
    P3 = prolongation(3, (nc, Nc - 1, Nc), (lo, 1, 0), (hi, 0, 0), ncomp=3).toarray()
    By = np.maximum(0.0, 1.0 - np.abs((xf[:, None] - xc[None, :]) * (Nc - 1)))[1:, 1:]
    Bz = np.maximum(0.0, 1.0 - np.abs((xf[:, None] - xc[None, :]) * (Nc - 1)))
    ref = np.kron(np.kron(np.kron(Bz, By), B), np.eye(3))
    assert np.allclose(P3, ref, atol=1e-15)


def _hier(prob):
    return omg.Hierarchy(3, None, prob.stencil, prob.levels, nodes=prob.nodes, faces=prob.faces, ncomp=3)


def test_galerkin_equals_rediscretisation_elasticity():
    prob = pb.elasticity_cantilever(17)
    H = _hier(prob)
    for j in range(H.levels - 1):
        Nj = (prob.nodes - 1) // 2 ** (H.levels - 1 - j) + 1
        ref = stencil_to_csr(3, pb.grid_shape(3, Nj, 0x1), pb.assemble_elasticity(Nj), ncomp=3)
        assert abs(H.A[j] - ref).max() < 1e-13 * abs(ref).max()
    assert H.A[0].shape == (300, 300)                    # 4 x 5 x 5 nodes x 3


def test_two_sweep_block_jacobi_closed_form():
    prob = pb.elasticity_cantilever(9)
    H = _hier(prob)
    j = H.J
    A = H.A[j].toarray()
    n = A.shape[0]
    D = np.zeros_like(A)
    for i in range(0, n, 3):
        D[i:i + 3, i:i + 3] = A[i:i + 3, i:i + 3]
    Di = np.linalg.inv(D)
    g = pb.normal(5, n)
    w = H.omega
    want = 2 * w * Di @ g - w * w * Di @ (A @ (Di @ g))
    assert np.allclose(H.smooth(j, g), want, rtol=1e-12, atol=1e-12 * abs(want).max())


def test_block_jacobi_smoother_is_spd_at_omega_two_thirds():
    """c_0 = 0 makes S^nu symmetric; it is positive definite when
    omega * lambda_max(D^-1 A) < 2 (here about 1.9)."""
    prob = pb.elasticity_cantilever(9)
    H = _hier(prob)
    for j in range(1, H.levels):
        lam = np.linalg.eigvals((H.Dinv[j] @ H.A[j]).toarray()).real.max()
        assert H.omega * lam < 2.0


def test_tiny_elasticity_solve_equals_dense_solution():
    prob = pb.elasticity_cantilever(9)
    H = _hier(prob)
    A = H.A[-1]
    res = ompcg.mpcg(A, prob.b, H.mg_columns, rtol=1e-12, maxit=500)
    x = np.linalg.solve(A.toarray(), prob.b)
    assert np.linalg.norm(res.x - x) <= 1e-10 * np.linalg.norm(x)
    # the cube sags: every z displacement is negative away from the clamp
    assert x[2::3].max() < 0.0


def test_planted_point_jacobi_fails_block_jacobi_pin(monkeypatch):
    """Plant: the diagonal instead of the 3 x 3 node blocks."""
    import scipy.sparse as sp

    def point_diag(A, k):
        return sp.diags(1.0 / A.diagonal()).tocsr()
    monkeypatch.setattr(omg, "block_diag_inverse", point_diag)
    with pytest.raises(AssertionError):
        test_two_sweep_block_jacobi_closed_form()


@pytest.mark.parametrize("dim,faces", [(2, 0x1), (2, 0x5), (3, 0x1), (3, 0x2A)])
def test_free_faces_galerkin_and_tiny_solve(dim, faces):
    """Diffusion with natural conditions on some faces: Galerkin products equal
    the rediscretised operators, and MPCG reaches the dense solution."""
    nodes = 17 if dim == 2 else 9
    prob = pb.diffusion_faces(dim, nodes, faces, rhs_seed=3)
    H = omg.Hierarchy(dim, None, prob.stencil, prob.levels, nodes=nodes, faces=faces)
    for j in range(H.levels - 1):
        Nj = (nodes - 1) // 2 ** (H.levels - 1 - j) + 1
        ref = stencil_to_csr(dim, pb.grid_shape(dim, Nj, faces), pb.assemble_diffusion(dim, Nj, faces=faces))
        assert abs(H.A[j] - ref).max() < 1e-13 * abs(ref).max()
    A = H.A[-1]
    res = ompcg.mpcg(A, prob.b, H.mg_columns, rtol=1e-12, maxit=500)
    x = np.linalg.solve(A.toarray(), prob.b)
    assert np.linalg.norm(res.x - x) <= 1e-10 * np.linalg.norm(x)


def test_example1_grid_hierarchy_and_pcg_equivalence():
    """Example 1's 160 x 160 elements on 4 grids (20 x 20 coarsest): the
    Galerkin operators equal the rediscretised anisotropic operators, and MPCG
    with the single summed column is additive-MG PCG."""
    from oracle.pcg import pcg
    prob = pb.example1(1e-3)
    H = omg.Hierarchy(2, prob.nodes - 2, prob.stencil, prob.levels)
    assert [N for N in (sh[0] + 2 for sh in H.shape)] == [21, 41, 81, 161]
    for j in range(H.levels - 1):
        Nj = H.shape[j][0] + 2
        ref = stencil_to_csr(2, Nj - 2, pb.assemble_diffusion(2, Nj, kdiag=(1e-3, 1.0)))
        assert abs(H.A[j] - ref).max() < 1e-13 * abs(ref).max()
    A = H.A[-1]
    res = ompcg.mpcg(A, prob.b, lambda r: H.additive_mg(r)[:, None], m=1, rtol=1e-8, maxit=2000)
    x, k, hist = pcg(A, prob.b, H.additive_mg, rtol=1e-8, maxit=2000)
    assert res.iters == k
    assert np.linalg.norm(res.x - x) <= 1e-10 * np.linalg.norm(x)
