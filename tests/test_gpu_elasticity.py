"""Parity of the CUDA path with the FP64 oracle on vector unknowns (3D Q1
elasticity, 3 x 3 block Jacobi) and on grids with free (natural) faces, whose
padded pitches are no longer powers of two.

Tolerances as in the scalar parity tests: operators and kernels to ~1e-13
relative (summation order only), FP64 solves to +-1 iteration and 1e-10 in
the solution, mixed precision by its true FP64 residual and its distance to
the FP64 oracle solution.  The full 65^3 x 3 configuration is checked by its
true residual (computed here in FP64 from the assembled operator) and by the
sag of the clamped cube.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mg as omg
from oracle import mpcg as ompcg
from oracle.operators import stencil_to_csr
from paper_2402_12833_gb300 import problems as pb

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_12833_gb300 import build, mpcg
    build.build()
    mpcg.load()
    return mpcg


PROBS = {
    "elast_9": lambda: pb.elasticity_cantilever(9),
    "elast_17": lambda: pb.elasticity_cantilever(17),
    "diff3d_17_free": lambda: pb.diffusion_faces(3, 17, 0x2A, rhs_seed=4, kappa_seed=8),
    "diff2d_65_x0": lambda: pb.diffusion_faces(2, 65, 0x1, rhs_seed=5, kappa_seed=9),
    "diff2d_33_lo": lambda: pb.diffusion_faces(2, 33, 0x5, rhs_seed=6),
}


def _hier(M, prob, levels=None, **opts):
    st = torch.from_numpy(np.ascontiguousarray(prob.stencil)).cuda()
    return M.Hierarchy(st, prob.dim, prob.nodes, levels or prob.levels, dofs_per_node=prob.ncomp,
                       faces=prob.faces, **opts)


def _oracle(prob, levels=None):
    return omg.Hierarchy(prob.dim, None, prob.stencil, levels or prob.levels, nodes=prob.nodes,
                         faces=prob.faces, ncomp=prob.ncomp)


@pytest.mark.parametrize("name", ["elast_17", "diff3d_17_free", "diff2d_65_x0"])
def test_galerkin_operators_match_oracle(M, name):
    prob = PROBS[name]()
    H = _hier(M, prob)
    O = _oracle(prob)
    S = prob.ncomp * 3 ** prob.dim
    for j in range(prob.levels):
        n = M.mg_level_size(H.h, j)
        assert n == O.A[j].shape[0]
        planes = torch.zeros((S, n), dtype=torch.float64, device="cuda")
        M.mg_get_operator(H.h, j, planes)
        A = stencil_to_csr(prob.dim, O.shape[j], planes.cpu().numpy(), prob.ncomp)
        ref = O.A[j]
        err = abs(A - ref).max()
        assert err <= 1e-13 * abs(ref).max(), (j, err)


@pytest.mark.parametrize("name", ["elast_17", "diff2d_33_lo"])
@pytest.mark.parametrize("ncols", [1, 5, 8, 9])
def test_block_spmm_matches_oracle(M, name, ncols):
    prob = PROBS[name]()
    H = _hier(M, prob)
    O = _oracle(prob)
    for j in (0, prob.levels - 1):
        n = O.A[j].shape[0]
        X = pb.normal(200 + j, n * ncols).reshape(ncols, n)
        Xd = torch.from_numpy(X).cuda()
        Yd = torch.zeros_like(Xd)
        M.mg_apply_operator(H.h, j, Xd, Yd, ncols)
        ref = (O.A[j] @ X.T).T
        scale = abs(O.A[j]).max() * np.abs(X).max()
        assert np.abs(Yd.cpu().numpy() - ref).max() <= 1e-14 * scale * 81


@pytest.mark.parametrize("name", ["elast_9", "elast_17", "diff3d_17_free", "diff2d_65_x0", "diff2d_33_lo"])
def test_mg_columns_match_oracle(M, name):
    """Restriction, (block) Jacobi, coarse solve and prolongation together."""
    prob = PROBS[name]()
    H = _hier(M, prob)
    O = _oracle(prob)
    r = pb.normal(7, prob.n)
    Zd = torch.zeros((prob.levels, prob.n), dtype=torch.float64, device="cuda")
    M.mg_corrections(H.h, torch.from_numpy(r).cuda(), Zd)
    Z = Zd.cpu().numpy().T
    ref = O.mg_columns(r)
    for l in range(prob.levels):
        assert np.abs(Z[:, l] - ref[:, l]).max() <= 1e-12 * np.abs(ref[:, l]).max(), l


@pytest.mark.parametrize("name,m", [("elast_9", 5), ("elast_17", 5), ("elast_17", 1),
                                    ("diff3d_17_free", 5), ("diff2d_65_x0", 5), ("diff2d_33_lo", 2)])
def test_solve_matches_oracle(M, name, m):
    prob = PROBS[name]()
    H = _hier(M, prob, m=m)
    O = _oracle(prob)
    b = torch.from_numpy(prob.b).cuda()
    x = torch.zeros_like(b)
    st, k, rh, ah = H.solve(b, x, rtol=1e-8, maxit=1000)
    ref = ompcg.mpcg(O.A[-1], prob.b, O.mg_columns, m=m, rtol=1e-8, maxit=1000)
    assert st == M.MPCG_OK and ref.converged
    assert abs(k - ref.iters) <= 1, (k, ref.iters)
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - ref.x) <= 1e-10 * np.linalg.norm(ref.x)
    kk = min(k, ref.iters, 6)
    assert np.allclose(rh[:kk + 1], ref.res_hist[:kk + 1], rtol=1e-6)
    assert np.allclose(ah[0], ref.alpha_hist[0], rtol=1e-8, atol=1e-12 * np.abs(ref.alpha_hist[0]).max())


@pytest.mark.parametrize("name", ["elast_17", "diff2d_65_x0"])
def test_mixed_precision_reaches_fp64_tolerance(M, name):
    prob = PROBS[name]()
    H = _hier(M, prob, precision=M.MPCG_MIXED)
    O = _oracle(prob)
    b = torch.from_numpy(prob.b).cuda()
    x = torch.zeros_like(b)
    st, k, rh, ah = H.solve(b, x, rtol=1e-8, maxit=2000)
    assert st == M.MPCG_OK
    xg = x.cpu().numpy()
    tr = np.linalg.norm(prob.b - O.A[-1] @ xg) / np.linalg.norm(prob.b)
    assert tr <= 1e-8
    ref = ompcg.mpcg(O.A[-1], prob.b, O.mg_columns, rtol=1e-12, maxit=2000)
    assert np.linalg.norm(xg - ref.x) <= 1e-5 * np.linalg.norm(ref.x)


def test_vector_problem_argument_checks(M):
    prob = PROBS["elast_9"]()
    st = torch.from_numpy(prob.stencil).cuda()
    with pytest.raises(M.MpcgError):            # 3 unknowns per node in 2D
        M.Hierarchy(st, 2, 9, 2, dofs_per_node=3, faces=0x1)
    with pytest.raises(M.MpcgError):            # 2 unknowns per node
        M.Hierarchy(st, 3, 9, 2, dofs_per_node=2, faces=0x1)
    with pytest.raises(M.MpcgError):            # face bits beyond the six faces
        M.Hierarchy(st, 3, 9, 2, dofs_per_node=3, faces=0x40)


def test_full_size_cantilever_65(M):
    """The 65^3 x 3 configuration (811,200 unknowns) in mixed precision: true
    FP64 residual <= 1e-8, and the displacement field sags everywhere."""
    prob = pb.elasticity_cantilever(65)
    assert prob.n == 811200
    H = _hier(M, prob, precision=M.MPCG_MIXED)
    b = torch.from_numpy(prob.b).cuda()
    x = torch.zeros_like(b)
    st, k, rh, ah = H.solve(b, x, rtol=1e-8, maxit=2000, histories=False)
    assert st == M.MPCG_OK
    xg = x.cpu().numpy()
    A = stencil_to_csr(3, prob.shape, prob.stencil, ncomp=3)
    tr = np.linalg.norm(prob.b - A @ xg) / np.linalg.norm(prob.b)
    assert tr <= 1e-8
    assert xg[2::3].max() < 0.0


def test_mg_columns_full_size_cantilever_65(M):
    """The MG columns of the 65^3 x 3 hierarchy (FP64), where the fine grid's
    second block-Jacobi sweep runs as one launch (residual and block update
    fused): the fine grid's column against the oracle to 1e-12 of its largest
    entry.  The coarser columns go through the Galerkin chain, which the GPU
    and the oracle sum in different orders over four products; the coarse
    solve amplifies those ~1e-15 differences (measured 1.9e-12 on the
    coarsest column), so they are held to 1e-10.  The FP32 instance of the
    fused launch runs in the full-size mixed solve above."""
    prob = pb.elasticity_cantilever(65)
    O = _oracle(prob)
    r = pb.normal(7, prob.n)
    ref = O.mg_columns(r)
    H = _hier(M, prob)
    Zd = torch.zeros((prob.levels, prob.n), dtype=torch.float64, device="cuda")
    M.mg_corrections(H.h, torch.from_numpy(r).cuda(), Zd)
    Z = Zd.cpu().numpy().T
    errs = [np.abs(Z[:, l] - ref[:, l]).max() / np.abs(ref[:, l]).max() for l in range(prob.levels)]
    print("relative column errors, coarse to fine:", errs)
    assert errs[-1] <= 1e-12, errs
    assert max(errs) <= 1e-10, errs
