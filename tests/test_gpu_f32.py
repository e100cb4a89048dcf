"""The FP32 arithmetic of the mixed precision's inner solves against the FP64
oracle, through mg_apply_operator_f32 and mg_corrections_f32.

On scalar grids these kernels stream the symmetric half of each grid's
stencil (the diagonal and the couplings to the later neighbours; a coupling
to an earlier neighbour is read transposed, A(i, i - s) = A(i - s, i), from
the neighbour's entry).  Covered: 2D and 3D, every grid of the hierarchy
(the narrow one-point-per-thread smoothing of the small grids included),
all-Dirichlet grids with power-of-two pitches, a grid whose pitch exceeds its
extent by more than one (Example 1: 159 unknowns per side, pitch 160), free
(natural) faces, ragged column counts, and grids of pitch 4 to 160 (rows
that fill part of a warp, several rows per warp, or more than a warp).

Bars.  SpMM: an output is a sum of at most 27 products of FP32-rounded
operands accumulated in FP32, so |y32 - A x| <= gamma_29 (|A| |x|)
entrywise with gamma_n = n u / (1 - n u) and u = 2^-24 (Higham, Accuracy and
Stability of Numerical Algorithms, 2nd ed., Section 3.1); the bar is 64 u.
A coupling read from the wrong plane, position or neighbour is off by the
size of |a||x| and fails it.  MG columns: two damped-Jacobi sweeps, the
transfers and the coarse solve in FP32 data; the bar is 2e-5 of each
column's largest entry (the observed error is a few 1e-7).
"""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mg as omg
from paper_2402_12833_gb300 import problems as pb

pytestmark = pytest.mark.gpu

U = 2.0 ** -24


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_12833_gb300 import build, mpcg
    build.build()
    mpcg.load()
    return mpcg


PROBS = {
    "poisson2d_65": lambda: pb.poisson_random(2, 65, 1),
    "kappa2d_65": lambda: pb.diffusion_macro(2, 65, 3),
    "example1_1e-3": lambda: pb.example1(1e-3),
    "diff2d_65_x0": lambda: pb.diffusion_faces(2, 65, 0x1, rhs_seed=5, kappa_seed=9),
    "poisson3d_17": lambda: pb.poisson_random(3, 17, 2),
    "kappa3d_33": lambda: pb.diffusion_macro(3, 33, 4, rhs="normal", rhs_seed=6),
    "diff3d_17_free": lambda: pb.diffusion_faces(3, 17, 0x2A, rhs_seed=4, kappa_seed=8),
    "kappa3d_65": lambda: pb.diffusion_macro(3, 65, 5, rhs="normal", rhs_seed=7),
    "diff3d_65_free": lambda: pb.diffusion_faces(3, 65, 0x2A, rhs_seed=8, kappa_seed=10),
}


def _hier(M, prob, **opts):
    st = torch.from_numpy(np.ascontiguousarray(prob.stencil)).cuda()
    return M.Hierarchy(st, prob.dim, prob.nodes, prob.levels, faces=prob.faces, precision=M.MPCG_MIXED, **opts)


def _oracle(prob):
    return omg.Hierarchy(prob.dim, None, prob.stencil, prob.levels, nodes=prob.nodes, faces=prob.faces)


@pytest.mark.parametrize("name", list(PROBS))
@pytest.mark.parametrize("ncols", [1, 6, 13])
def test_f32_block_spmm_matches_oracle(M, name, ncols):
    prob = PROBS[name]()
    H = _hier(M, prob)
    O = _oracle(prob)
    for j in range(prob.levels):
        n = O.A[j].shape[0]
        X = pb.normal(300 + 7 * j + ncols, n * ncols).reshape(ncols, n)
        Xd = torch.from_numpy(X).cuda()
        Yd = torch.zeros_like(Xd)
        M.mg_apply_operator_f32(H.h, j, Xd, Yd, ncols)
        ref = (O.A[j] @ X.T).T
        bound = (abs(O.A[j]) @ np.abs(X).T).T
        err = np.abs(Yd.cpu().numpy() - ref)
        assert np.all(err <= 64 * U * bound), (j, float((err / np.maximum(bound, 1e-300)).max()))


@pytest.mark.parametrize("name", list(PROBS))
def test_f32_mg_columns_match_oracle(M, name):
    prob = PROBS[name]()
    H = _hier(M, prob)
    O = _oracle(prob)
    r = pb.normal(9, prob.n)
    Zd = torch.zeros((prob.levels, prob.n), dtype=torch.float64, device="cuda")
    M.mg_corrections_f32(H.h, torch.from_numpy(r).cuda(), Zd)
    Z = Zd.cpu().numpy().T
    ref = O.mg_columns(r)
    for l in range(prob.levels):
        err = np.abs(Z[:, l] - ref[:, l]).max()
        assert err <= 2e-5 * np.abs(ref[:, l]).max(), (l, err / np.abs(ref[:, l]).max())


def test_f32_calls_need_a_mixed_stencil_hierarchy(M):
    prob = PROBS["poisson2d_65"]()
    st = torch.from_numpy(np.ascontiguousarray(prob.stencil)).cuda()
    H = M.Hierarchy(st, prob.dim, prob.nodes, prob.levels, precision=M.MPCG_FP64)
    X = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    with pytest.raises(M.MpcgError):
        M.mg_apply_operator_f32(H.h, prob.levels - 1, X, X.clone(), 1)
    with pytest.raises(M.MpcgError):
        M.mg_corrections_f32(H.h, X, torch.zeros((prob.levels, prob.n), dtype=torch.float64, device="cuda"))


@pytest.mark.parametrize("name", ["kappa3d_33", "kappa3d_65", "diff3d_65_free"])
def test_f32_spmm_columns_are_independent(M, name):
    """A column's product does not depend on the other columns: the 1-, 5-
    and 6-column products (separate kernel instances) equal the first columns
    of the 12-column product bit for bit."""
    prob = PROBS[name]()
    H = _hier(M, prob)
    for j in range(prob.levels):
        n = M.mg_level_size(H.h, j)
        X = torch.from_numpy(pb.normal(500 + j, 12 * n).reshape(12, n)).cuda()
        Y12 = torch.zeros_like(X)
        M.mg_apply_operator_f32(H.h, j, X, Y12, 12)
        for c in (1, 5, 6):
            Yc = torch.zeros_like(X[:c])
            M.mg_apply_operator_f32(H.h, j, X[:c].contiguous(), Yc, c)
            assert torch.equal(Yc, Y12[:c]), (j, c)


@pytest.mark.parametrize("name", ["kappa3d_65", "diff3d_65_free"])
def test_f32_mixed_solve_reaches_fp64_tolerance(M, name):
    """A mixed solve on a 65^3 grid (fine-grid SpMM with the z^T A z
    partials): the true FP64 residual of its solution, taken with the
    oracle's operator, meets the tolerance."""
    prob = PROBS[name]()
    H = _hier(M, prob)
    O = _oracle(prob)
    b = torch.from_numpy(prob.b).cuda()
    x = torch.zeros_like(b)
    st, k, rh, ah = H.solve(b, x, rtol=1e-8, maxit=2000)
    assert st == M.MPCG_OK
    xg = x.cpu().numpy()
    tr = np.linalg.norm(prob.b - O.A[-1] @ xg) / np.linalg.norm(prob.b)
    assert tr <= 1e-8


@pytest.mark.parametrize("name", ["poisson2d_65", "kappa3d_33", "diff3d_17_free"])
def test_f32_full_stencil_option(M, name):
    """half_stencil = 0: the FP32 kernels read the full stored stencil; the
    products meet the same bar against the oracle on every grid, and the
    mixed solve still reaches the FP64 tolerance."""
    prob = PROBS[name]()
    H = _hier(M, prob, half_stencil=0)
    O = _oracle(prob)
    for j in range(prob.levels):
        n = O.A[j].shape[0]
        X = pb.normal(700 + j, 6 * n).reshape(6, n)
        Yd = torch.zeros((6, n), dtype=torch.float64, device="cuda")
        M.mg_apply_operator_f32(H.h, j, torch.from_numpy(X).cuda(), Yd, 6)
        ref = (O.A[j] @ X.T).T
        bound = (abs(O.A[j]) @ np.abs(X).T).T
        assert np.all(np.abs(Yd.cpu().numpy() - ref) <= 64 * U * bound), j
    b = torch.from_numpy(prob.b).cuda()
    x = torch.zeros_like(b)
    st, k, _, _ = H.solve(b, x, rtol=1e-8, maxit=2000)
    assert st == M.MPCG_OK
    assert np.linalg.norm(prob.b - O.A[-1] @ x.cpu().numpy()) <= 1e-8 * np.linalg.norm(prob.b)
    with pytest.raises(M.MpcgError):
        _hier(M, prob, half_stencil=2)


@functools.lru_cache(maxsize=1)
def _full_size():
    prob = pb.poisson_random(3, 129, 2)
    return prob, _oracle(prob)


def test_f32_full_size_spmm_columns_and_solve(M):
    """The benchmark's workload at full size (3D Poisson 129^3, 2,048,383
    unknowns, 6 grids): the fine-grid SpMM of the FP32 inner iterations with
    its 6 columns, entrywise within 64 u of |A||x| of the oracle's product;
    the 6 FP32 MG columns within 2e-5 of the oracle's; and the mixed solve's
    true FP64 residual, taken with the oracle's operator, below 1e-8."""
    prob, O = _full_size()
    H = _hier(M, prob)
    j = prob.levels - 1
    X = pb.normal(900, 6 * prob.n).reshape(6, prob.n)
    Yd = torch.zeros((6, prob.n), dtype=torch.float64, device="cuda")
    M.mg_apply_operator_f32(H.h, j, torch.from_numpy(X).cuda(), Yd, 6)
    Y = Yd.cpu().numpy()
    del Yd
    for c in range(6):
        ref = O.A[j] @ X[c]
        bound = abs(O.A[j]) @ np.abs(X[c])
        assert np.all(np.abs(Y[c] - ref) <= 64 * U * bound), c
    r = pb.normal(901, prob.n)
    Zd = torch.zeros((prob.levels, prob.n), dtype=torch.float64, device="cuda")
    M.mg_corrections_f32(H.h, torch.from_numpy(r).cuda(), Zd)
    Z = Zd.cpu().numpy().T
    del Zd
    ref = O.mg_columns(r)
    for l in range(prob.levels):
        assert np.abs(Z[:, l] - ref[:, l]).max() <= 2e-5 * np.abs(ref[:, l]).max(), l
    b = torch.from_numpy(prob.b).cuda()
    x = torch.zeros_like(b)
    st, k, _, _ = H.solve(b, x, rtol=1e-8, maxit=200, histories=False)
    assert st == M.MPCG_OK
    assert np.linalg.norm(prob.b - O.A[-1] @ x.cpu().numpy()) <= 1e-8 * np.linalg.norm(prob.b)
