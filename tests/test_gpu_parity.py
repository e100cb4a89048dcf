"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (FP64 path): operators and single kernels agree to ~1e-13
relative (different summation order only); full solves agree in iteration
count to +-1 and in the solution to 1e-10 relative.  Mixed precision: the
true FP64 residual reaches rtol and the error against the FP64 oracle
solution is reported and bounded.
"""
import functools

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


def _hier(M, prob, levels=None, **opts):
    st = torch.from_numpy(np.ascontiguousarray(prob.stencil)).cuda()
    return M.Hierarchy(st, prob.dim, prob.nodes, levels or prob.levels, **opts)


def _oracle(prob, levels=None):
    return omg.Hierarchy(prob.dim, prob.n1, prob.stencil, levels or prob.levels)


PROBS = {
    "poisson2d_65": lambda: pb.poisson_random(2, 65, 1),
    "kappa2d_65": lambda: pb.diffusion_macro(2, 65, 3),
    "kappa2d_33_normal": lambda: pb.diffusion_macro(2, 33, 11, rhs="normal", rhs_seed=5),
    "poisson3d_17": lambda: pb.poisson_random(3, 17, 2),
    "kappa3d_17": lambda: pb.diffusion_macro(3, 17, 4, rhs="normal", rhs_seed=6),
}


@pytest.mark.parametrize("name", ["kappa2d_65", "kappa3d_17"])
def test_galerkin_operators_match_oracle(M, name):
    prob = PROBS[name]()
    H = _hier(M, prob)
    O = _oracle(prob)
    S = 3 ** prob.dim
    for j in range(prob.levels):
        n = M.mg_level_size(H.h, j)
        planes = torch.zeros((S, n), dtype=torch.float64, device="cuda")
        M.mg_get_operator(H.h, j, planes)
        A = stencil_to_csr(prob.dim, O.n1[j], planes.cpu().numpy())
        ref = O.A[j]
        err = abs(A - ref).max()
        assert err <= 1e-13 * abs(ref).max(), (j, err)


@pytest.mark.parametrize("name", ["poisson2d_65", "kappa3d_17"])
@pytest.mark.parametrize("ncols", [1, 5, 12, 13])
def test_block_spmm_matches_oracle(M, name, ncols):
    prob = PROBS[name]()
    H = _hier(M, prob)
    O = _oracle(prob)
    for j in (0, prob.levels - 1):
        n = O.A[j].shape[0]
        X = pb.normal(100 + j, n * ncols).reshape(ncols, n)
        Xd = torch.from_numpy(X).cuda()
        Yd = torch.zeros_like(Xd)
        M.mg_apply_operator(H.h, j, Xd, Yd, ncols)
        ref = (O.A[j] @ X.T).T
        scale = abs(O.A[j]).max() * np.abs(X).max()
        assert np.abs(Yd.cpu().numpy() - ref).max() <= 1e-14 * scale * 27


@pytest.mark.parametrize("name", ["poisson2d_65", "kappa2d_65", "poisson3d_17", "kappa3d_17"])
def test_mg_columns_match_oracle(M, name):
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


def _solve_pair(M, prob, m=5, rtol=1e-8, maxit=800, levels=None, precision=None):
    H = _hier(M, prob, levels=levels, m=m, **({} if precision is None else {"precision": precision}))
    O = _oracle(prob, levels)
    b = torch.from_numpy(prob.b).cuda()
    x = torch.zeros_like(b)
    st, k, rh, ah = H.solve(b, x, rtol=rtol, maxit=maxit)
    ref = ompcg.mpcg(O.A[-1], prob.b, O.mg_columns, m=m, rtol=rtol, maxit=maxit)
    return st, k, x.cpu().numpy(), rh, ah, ref, O


SENSITIVE = {("kappa2d_33_normal", 10)}


@pytest.mark.parametrize("precision", ["fp64", "fp64_dw"])
@pytest.mark.parametrize("name,m", [("poisson2d_65", 5), ("poisson2d_65", 1), ("kappa2d_65", 5),
                                    ("kappa2d_33_normal", 1), ("kappa2d_33_normal", 10),
                                    ("poisson3d_17", 5), ("kappa3d_17", 5), ("kappa3d_17", 2)])
def test_solve_matches_oracle(M, name, m, precision):
    """FP64 arithmetic, and FP64 data with double-word (2 x FP32, ~48-bit)
    arithmetic: both held to the same bar against the oracle."""
    prob = PROBS[name]()
    prec = M.MPCG_FP64 if precision == "fp64" else M.MPCG_FP64_DW
    st, k, x, rh, ah, ref, O = _solve_pair(M, prob, m=m, precision=prec)
    assert st == M.MPCG_OK
    assert ref.converged
    if (name, m) in SENSITIVE:
        # the drop rule and the pseudo-inverse cutoff are discontinuous in the
        # data: with a 10-block window on high contrast the Gram matrices sit
        # near the thresholds and rounding decides drops, so the oracle itself
        # moves by several iterations under 1e-15 relative changes of b
        # (tests/test_oracle_pins.py pins that spread on the CPU).  The GPU
        # count must lie within the oracle's own spread over eight such
        # perturbations (widened by one); the solutions agree to 1e-9 (their
        # spread under the same perturbations is ~1e-10) and the true
        # residual meets rtol.
        spread = [ompcg.mpcg(O.A[-1], pb.perturbed(prob.b, s, 1e-15), O.mg_columns, m=m, rtol=1e-8,
                             maxit=800).iters for s in range(8)] + [ref.iters]
        assert min(spread) - 1 <= k <= max(spread) + 1, (k, spread)
        assert np.linalg.norm(x - ref.x) <= 1e-9 * np.linalg.norm(ref.x)
        tr = np.linalg.norm(prob.b - O.A[-1] @ x) / np.linalg.norm(prob.b)
        assert tr <= 1.01e-8
        return
    if precision == "fp64_dw":
        # double-word arithmetic rounds at 2^-47 instead of FP64's 2^-53;
        # like any Krylov method in finite precision, the larger rounding
        # delays convergence on the long high-contrast solves (kappa2d_65:
        # 201 steps against the oracle's 199, whose count does not move
        # under 2^-47 relative changes of b).  Held to 1 % of the count
        # (at least +-1); FP64 arithmetic stays at +-1.
        assert abs(k - ref.iters) <= max(1, int(np.ceil(0.01 * ref.iters))), (k, ref.iters)
    else:
        assert abs(k - ref.iters) <= 1, (k, ref.iters)
    assert np.linalg.norm(x - ref.x) <= 1e-10 * np.linalg.norm(ref.x)
    # residual histories agree while they are far above round-off
    kk = min(k, ref.iters, 6)
    assert np.allclose(rh[:kk + 1], ref.res_hist[:kk + 1], rtol=1e-6)
    # first alpha vector
    assert np.allclose(ah[0], ref.alpha_hist[0], rtol=1e-8, atol=1e-12 * np.abs(ref.alpha_hist[0]).max())
    # the true residual of the GPU solution
    tr = np.linalg.norm(prob.b - O.A[-1] @ x) / np.linalg.norm(prob.b)
    assert tr <= 1.01e-8


def test_manufactured_rhs_converges_in_one_iteration(M):
    prob = pb.poisson_manufactured_2d(65)
    st, k, x, rh, ah, ref, O = _solve_pair(M, prob)
    assert k == ref.iters == 1
    assert np.abs(x - pb.manufactured_u(2, 65)).max() < 1e-3


def test_single_grid_exact_solve(M):
    prob = pb.poisson_random(2, 5, 3)
    st, k, x, rh, ah, ref, O = _solve_pair(M, prob, rtol=1e-13)
    assert k == 1 and ref.iters == 1
    assert np.allclose(x, ref.x, rtol=1e-13, atol=1e-15)


def test_two_levels_tiny_3d(M):
    prob = pb.diffusion_macro(3, 9, 2, rhs="normal", rhs_seed=1)
    st, k, x, rh, ah, ref, O = _solve_pair(M, prob, rtol=1e-12)
    assert abs(k - ref.iters) <= 1
    assert np.linalg.norm(x - ref.x) <= 1e-10 * np.linalg.norm(ref.x)


@pytest.mark.parametrize("precision", ["fp64", "fp64_dw"])
def test_nonzero_initial_guess_and_fewer_levels(M, precision):
    prob = pb.diffusion_macro(2, 65, 8, rhs="normal", rhs_seed=2)
    levels = 3
    H = _hier(M, prob, levels=levels, precision=M.MPCG_FP64 if precision == "fp64" else M.MPCG_FP64_DW)
    O = _oracle(prob, levels)
    x0 = pb.normal(33, prob.n)
    x = torch.from_numpy(x0.copy()).cuda()
    st, k, rh, ah = H.solve(torch.from_numpy(prob.b).cuda(), x, rtol=1e-9, maxit=600)
    ref = ompcg.mpcg(O.A[-1], prob.b, O.mg_columns, x0=x0, rtol=1e-9, maxit=600)
    assert abs(k - ref.iters) <= 1
    assert np.linalg.norm(x.cpu().numpy() - ref.x) <= 1e-10 * np.linalg.norm(ref.x)


def test_host_buffers_give_the_device_result(M):
    prob = PROBS["kappa2d_65"]()
    H = _hier(M, prob)
    xd = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    st, k, _, _ = H.solve(torch.from_numpy(prob.b).cuda(), xd, maxit=600)
    xh = np.zeros(prob.n)
    st2, k2, _, _ = H.solve(prob.b.copy(), xh, maxit=600)
    assert k == k2
    assert np.array_equal(xd.cpu().numpy(), xh)


def test_repeated_solves_are_bitwise_identical(M):
    prob = PROBS["kappa3d_17"]()
    H = _hier(M, prob)
    b = torch.from_numpy(prob.b).cuda()
    outs = []
    for _ in range(3):
        x = torch.zeros_like(b)
        H.solve(b, x)
        outs.append(x.cpu().numpy())
    assert all(np.array_equal(outs[0], o) for o in outs[1:])


def test_not_converged_status(M):
    prob = PROBS["kappa2d_65"]()
    H = _hier(M, prob)
    x = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    st, k, rh, ah = H.solve(torch.from_numpy(prob.b).cuda(), x, maxit=3)
    assert st == M.MPCG_NOT_CONVERGED and k == 3 and len(rh) == 4


def test_zero_rhs_returns_immediately(M):
    prob = PROBS["poisson2d_65"]()
    H = _hier(M, prob)
    x = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    st, k, rh, ah = H.solve(torch.zeros_like(x), x)
    assert st == M.MPCG_OK and k == 0 and torch.count_nonzero(x) == 0


def test_not_spd_coarse_operator_is_reported(M):
    prob = pb.poisson_random(2, 17, 1)
    st = torch.from_numpy(-prob.stencil).cuda()
    with pytest.raises(M.MpcgError) as e:
        M.Hierarchy(st, 2, 17, prob.levels)
    assert e.value.status == M.MPCG_ERR_NOT_SPD


def test_bad_arguments_are_rejected(M):
    prob = pb.poisson_random(2, 17, 1)
    st = torch.from_numpy(prob.stencil).cuda()
    with pytest.raises(M.MpcgError) as e:
        M.Hierarchy(st, 2, 17, 5)           # 17 nodes allow at most 4 grids
    assert e.value.status == M.MPCG_ERR_ARG
    with pytest.raises(M.MpcgError):
        M.Hierarchy(st, 2, 18, 2)
    with pytest.raises(M.MpcgError):
        M.Hierarchy(st, 2, 17, 2, m=0)


@pytest.mark.parametrize("name", ["kappa2d_65", "poisson3d_17"])
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
    err = np.linalg.norm(xg - ref.x) / np.linalg.norm(ref.x)
    assert err <= 1e-5, err


def test_summed_column_solve_is_additive_mg_pcg(M):
    """sum_columns = 1 with a one-block window: the paper's additive MG-PCG
    comparison method, against textbook PCG with the oracle's B of Eq. 3."""
    from oracle.pcg import pcg
    prob = pb.example1(1e-2)
    H = _hier(M, prob, m=1, sum_columns=1)
    assert M.mg_num_columns(H.h) == 1
    O = _oracle(prob)
    b = torch.from_numpy(prob.b).cuda()
    x = torch.zeros_like(b)
    st, k, rh, ah = H.solve(b, x, rtol=1e-8, maxit=3000)
    xr, kr, hist = pcg(O.A[-1], prob.b, O.additive_mg, rtol=1e-8, maxit=3000)
    assert st == M.MPCG_OK
    assert abs(k - kr) <= 1, (k, kr)
    assert np.linalg.norm(x.cpu().numpy() - xr) <= 1e-10 * np.linalg.norm(xr)
    assert np.allclose(rh[:6], hist[:6], rtol=1e-6)


@pytest.mark.parametrize("kxx", [1.0, 1e-3, 1e-6])
def test_example1_hierarchy_and_solve_match_oracle(M, kxx):
    """Example 1 (160 x 160 elements, 4 grids, 20 x 20 coarsest): a grid whose
    element count is not a power of two."""
    prob = pb.example1(kxx)
    H = _hier(M, prob)
    O = _oracle(prob)
    for j in range(prob.levels):
        n = M.mg_level_size(H.h, j)
        planes = torch.zeros((9, n), dtype=torch.float64, device="cuda")
        M.mg_get_operator(H.h, j, planes)
        A = stencil_to_csr(2, O.n1[j], planes.cpu().numpy())
        assert abs(A - O.A[j]).max() <= 1e-13 * abs(O.A[j]).max()
    b = torch.from_numpy(prob.b).cuda()
    x = torch.zeros_like(b)
    st, k, rh, ah = H.solve(b, x, rtol=1e-8, maxit=3000)
    ref = ompcg.mpcg(O.A[-1], prob.b, O.mg_columns, m=5, rtol=1e-8, maxit=3000)
    assert st == M.MPCG_OK and ref.converged
    assert abs(k - ref.iters) <= 1, (k, ref.iters)
    assert np.linalg.norm(x.cpu().numpy() - ref.x) <= 1e-9 * np.linalg.norm(ref.x)


# -- the branches of the drop rule and the scaled pseudo-inverse (Section 2.2,
# the remark on a singular P^T A P) and the breakdown exits

def _eig_cut_margin(ref, tau):
    """Over the oracle's blocks: (blocks whose Cholesky certificate
    trace((DGD)^-1) * tau * n_active < 1 fails, eigenvalues cut, smallest
    distance in decades between an eigenvalue of D G D and the cutoff
    tau * lambda_max)."""
    fails = cuts = 0
    margin = np.inf
    for P, AP in ref.blocks:
        G = P.T @ AP
        G = 0.5 * (G + G.T)
        act = np.where(np.diag(G) > 0)[0]
        d = 1.0 / np.sqrt(np.diag(G)[act])
        Gh = d[:, None] * G[np.ix_(act, act)] * d[None, :]
        lam = np.linalg.eigvalsh(Gh)
        fails += int(np.trace(np.linalg.inv(Gh)) * tau * act.size >= 1.0)
        thr = tau * lam.max()
        cuts += int((lam <= thr).sum())
        margin = min(margin, float(np.min(np.abs(np.log10(lam / thr)))))
    return fails, cuts, margin


@pytest.mark.parametrize("name,tau,expect_cuts", [("poisson2d_65", 0.03, False), ("poisson3d_17", 0.3, True),
                                                  ("kappa3d_17", 0.7, True)])
def test_eigenvalue_pseudo_inverse_branch_matches_oracle(M, name, tau, expect_cuts):
    """A raised cutoff tau makes the Cholesky certificate in the alpha kernel
    fail, so the Jacobi eigenvalue pseudo-inverse runs on the GPU; with
    expect_cuts some eigenvalues of D G D fall below tau * lambda_max and are
    removed.  Every eigenvalue sits at least 5 % away from the cutoff, so
    rounding cannot change which are kept."""
    prob = PROBS[name]()
    H = _hier(M, prob, pinv_tau=tau)
    O = _oracle(prob)
    b = torch.from_numpy(prob.b).cuda()
    x = torch.zeros_like(b)
    st, k, rh, ah = H.solve(b, x, rtol=1e-8, maxit=400)
    cnt = M.mg_last_solve_counters(H.h)
    ref = ompcg.mpcg(O.A[-1], prob.b, O.mg_columns, rtol=1e-8, maxit=400, tau=tau, keep_blocks=True)
    fails, cuts, margin = _eig_cut_margin(ref, tau)
    assert margin > np.log10(1.05), margin
    assert fails >= 1 and (cuts >= 1) == expect_cuts, (fails, cuts)
    assert st == M.MPCG_OK and ref.converged
    assert cnt["pinv_fallbacks"] >= 1 and cnt["iters"] == k, cnt
    assert abs(k - ref.iters) <= 1, (k, ref.iters)
    assert np.linalg.norm(x.cpu().numpy() - ref.x) <= 1e-10 * np.linalg.norm(ref.x)
    kk = min(k, ref.iters)
    A = np.array(ref.alpha_hist[:kk])
    assert np.allclose(ah[:kk], A, rtol=1e-7, atol=1e-10 * np.abs(A).max())


def test_default_cutoff_never_takes_the_eigenvalue_branch(M):
    """At the default tau = 1e-12 the certified Cholesky path serves every
    block of a well-conditioned solve (the counter sees no fallback)."""
    prob = PROBS["poisson2d_65"]()
    H = _hier(M, prob)
    b = torch.from_numpy(prob.b).cuda()
    H.solve(b, torch.zeros_like(b))
    cnt = M.mg_last_solve_counters(H.h)
    assert cnt["pinv_fallbacks"] == 0 and cnt["dropped"] == 0 and cnt["done"] == 1, cnt


def test_zero_network_column_is_dropped_every_block(M):
    """A learned column from an all-zero network is identically zero: the drop
    rule removes it from every block, and the solve equals the plain one and
    the oracle's run with a zero extra column."""
    prob = PROBS["kappa2d_33_normal"]()
    H = _hier(M, prob)
    O = _oracle(prob)
    b = torch.from_numpy(prob.b).cuda()
    x0 = torch.zeros_like(b)
    st0, k0, _, _ = H.solve(b, x0, rtol=1e-8, maxit=400)
    plain = M.mg_last_solve_counters(H.h)
    M.mg_learned_attach(H.h, np.zeros(M.mg_learned_num_params(), dtype=np.float32))
    x = torch.zeros_like(b)
    st, k, rh, ah = H.solve(b, x, rtol=1e-8, maxit=400)
    cnt = M.mg_last_solve_counters(H.h)
    ref = ompcg.mpcg(O.A[-1], prob.b, O.mg_columns, rtol=1e-8, maxit=400, extra_column=lambda r: np.zeros_like(r))
    assert st == st0 == M.MPCG_OK and ref.converged
    assert all(prob.levels in d for d in ref.dropped)
    assert cnt["dropped"] == plain["dropped"] + k, (cnt, plain, k)
    assert k == k0 and abs(k - ref.iters) <= 1, (k, k0, ref.iters)
    assert np.all(ah[:, -1] == 0.0)
    assert np.linalg.norm(x.cpu().numpy() - x0.cpu().numpy()) <= 1e-12 * np.linalg.norm(x0.cpu().numpy())
    assert np.linalg.norm(x.cpu().numpy() - ref.x) <= 1e-10 * np.linalg.norm(ref.x)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_every_column_dropped_is_a_breakdown(M, precision):
    """drop_delta = 2 removes every column of the first block (its squared
    A-norms equal those before orthogonalisation): the oracle's first block
    keeps nothing and its iterate never moves; the library stops with
    MPCG_ERR_BREAKDOWN instead of looping."""
    prob = PROBS["poisson2d_65"]()
    prec = M.MPCG_FP64 if precision == "fp64" else M.MPCG_MIXED
    H = _hier(M, prob, drop_delta=2.0, inner_drop_delta=2.0, precision=prec)
    b = torch.from_numpy(prob.b).cuda()
    x = torch.zeros_like(b)
    with pytest.raises(M.MpcgError) as e:
        H.solve(b, x, rtol=1e-8, maxit=50)
    assert e.value.status == M.MPCG_ERR_BREAKDOWN
    cnt = M.mg_last_solve_counters(H.h)
    assert cnt["done"] == 3 and cnt["dropped"] == prob.levels, cnt
    O = _oracle(prob)
    ref = ompcg.mpcg(O.A[-1], prob.b, O.mg_columns, rtol=1e-8, maxit=3, delta=2.0)
    assert ref.dropped[0] == list(range(prob.levels)) and not np.any(ref.x)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("where", ["b_nan", "b_inf", "x0_nan"])
def test_non_finite_input_is_a_breakdown(M, precision, where):
    """A NaN or infinity in b or x_0 (made on the host) ends the solve with
    MPCG_ERR_BREAKDOWN; the hierarchy stays usable for the next solve."""
    prob = PROBS["kappa2d_65"]()
    prec = M.MPCG_FP64 if precision == "fp64" else M.MPCG_MIXED
    H = _hier(M, prob, precision=prec)
    b = prob.b.copy()
    x0 = np.zeros(prob.n)
    bad = {"b_nan": np.nan, "b_inf": np.inf, "x0_nan": np.nan}[where]
    (x0 if where.startswith("x0") else b)[prob.n // 3] = bad
    bd, xd = torch.from_numpy(b).cuda(), torch.from_numpy(x0).cuda()
    with pytest.raises(M.MpcgError) as e:
        H.solve(bd, xd, rtol=1e-8, maxit=100)
    assert e.value.status == M.MPCG_ERR_BREAKDOWN
    x = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    st, k, _, _ = H.solve(torch.from_numpy(prob.b).cuda(), x, rtol=1e-8, maxit=2000)
    assert st == M.MPCG_OK and torch.isfinite(x).all()


@functools.lru_cache(maxsize=1)
def _oracle_full_size():
    prob = pb.poisson_random(3, 129, 2)
    O = _oracle(prob)
    return ompcg.mpcg(O.A[-1], prob.b, O.mg_columns, m=5, rtol=1e-8, maxit=200)


@pytest.mark.parametrize("precision", ["fp64", "fp64_dw"])
def test_full_size_fp64_solve_matches_oracle(M, precision):
    """The 3D Poisson workload at full size (129^3 nodes, 2,048,383 unknowns,
    6 grids, N(0,1) right-hand side seed 2, m = 5) in the FP64-data paths
    (FP64 and double-word arithmetic), with the graph-launched solve the
    benchmark times: iteration count +-1 and the solution to 1e-10 relative
    against the oracle."""
    prob = pb.poisson_random(3, 129, 2)
    H = _hier(M, prob, m=5, precision=M.MPCG_FP64 if precision == "fp64" else M.MPCG_FP64_DW)
    b = torch.from_numpy(prob.b).cuda()
    x = torch.zeros_like(b)
    st, k, rh, ah = H.solve(b, x, rtol=1e-8, maxit=200, histories=False)
    xg = x.cpu().numpy()
    H.close()
    ref = _oracle_full_size()
    assert st == M.MPCG_OK and ref.converged
    assert abs(k - ref.iters) <= 1, (k, ref.iters)
    assert np.linalg.norm(xg - ref.x) <= 1e-10 * np.linalg.norm(ref.x)
