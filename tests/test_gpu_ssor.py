"""The SSOR smoother and the multiplicative V-cycle (Section 3's comparison
setup) on the GPU against the oracle (oracle/ssor.py), through the C ABI.

Tolerances (FP64): the level corrections and the V-cycle agree with the
oracle to 1e-12 relative (summation order only; the colour updates are
exact Gauss-Seidel in the same order); solves agree in iteration count to
+-1 and in the solution to 1e-10 relative, like the Jacobi path.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mg as omg
from oracle import mpcg as ompcg
from oracle import pcg as opcg
from oracle import ssor as oss
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


CASES = {
    "kappa2d_33": lambda: pb.diffusion_macro(2, 33, 3, rhs="normal", rhs_seed=2),
    "kappa2d_33_faces": lambda: pb.diffusion_faces(2, 33, 0x9, rhs_seed=3, kappa_seed=4),
    "kappa3d_17": lambda: pb.diffusion_macro(3, 17, 4, rhs="normal", rhs_seed=6),
    "example1_1e-3": lambda: pb.example1(1e-3, nodes=41, levels=3),
    # larger fine grids (16,384 and 32,768 padded points)
    "kappa2d_129": lambda: pb.diffusion_macro(2, 129, 6, rhs="normal", rhs_seed=8),
    "kappa3d_33": lambda: pb.diffusion_macro(3, 33, 7, rhs="normal", rhs_seed=9),
}


def _hier(M, prob, **opts):
    st = torch.from_numpy(np.ascontiguousarray(prob.stencil)).cuda()
    return M.Hierarchy(st, prob.dim, prob.nodes, prob.levels, faces=prob.faces, smoother=M.MPCG_SMOOTHER_SSOR,
                       **opts)


def _oracle(prob):
    H = omg.Hierarchy(prob.dim, None, prob.stencil, prob.levels, nodes=prob.nodes, faces=prob.faces)
    return H, oss.level_smoothers(H)


@pytest.mark.parametrize("name", list(CASES))
def test_ssor_columns_match_oracle(M, name):
    prob = CASES[name]()
    H = _hier(M, prob, nu=6)
    O, Ss = _oracle(prob)
    r = np.random.default_rng(1).standard_normal(prob.n)
    Z = torch.zeros((prob.levels, prob.n), dtype=torch.float64, device="cuda")
    M.mg_corrections(H.h, torch.from_numpy(r).cuda(), Z)
    ref = oss.additive_columns(O, Ss, r, 6)
    got = Z.cpu().numpy().T
    for j in range(prob.levels):
        assert np.abs(got[:, j] - ref[:, j]).max() <= 1e-12 * np.abs(ref[:, j]).max(), j


@pytest.mark.parametrize("name", list(CASES))
def test_vcycle_matches_oracle(M, name):
    prob = CASES[name]()
    H = _hier(M, prob, nu=3, vcycle=1, m=1)
    O, Ss = _oracle(prob)
    r = np.random.default_rng(2).standard_normal(prob.n)
    Z = torch.zeros((1, prob.n), dtype=torch.float64, device="cuda")
    M.mg_corrections(H.h, torch.from_numpy(r).cuda(), Z)
    ref = oss.vcycle(O, Ss, r, 3)
    assert np.abs(Z.cpu().numpy()[0] - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("name", list(CASES))
def test_solves_match_oracle(M, name):
    """MG(V)-PCG, additive-SSOR MG-PCG and additive-SSOR MG-MPCG (m = 5):
    iteration count +-1 and solution to 1e-10 against the oracle."""
    prob = CASES[name]()
    O, Ss = _oracle(prob)
    A = O.A[-1]
    b = torch.from_numpy(prob.b).cuda()
    runs = {
        "v_pcg": (dict(nu=3, vcycle=1, m=1),
                  lambda: opcg.pcg(A, prob.b, lambda r: oss.vcycle(O, Ss, r, 3), rtol=1e-8, maxit=2000)),
        "add_pcg": (dict(nu=6, sum_columns=1, m=1),
                    lambda: opcg.pcg(A, prob.b, lambda r: oss.additive_columns(O, Ss, r, 6).sum(axis=1),
                                     rtol=1e-8, maxit=2000)),
        "add_mpcg": (dict(nu=6, m=5),
                     lambda: (lambda res: (res.x, res.iters, None))(
                         ompcg.mpcg(A, prob.b, lambda r: oss.additive_columns(O, Ss, r, 6), rtol=1e-8, maxit=2000))),
    }
    for key, (opts, ref) in runs.items():
        H = _hier(M, prob, **opts)
        x = torch.zeros_like(b)
        st, k, _, _ = H.solve(b, x, rtol=1e-8, maxit=2000)
        xr, kr, _ = ref()
        assert st == M.MPCG_OK, key
        assert abs(k - kr) <= 1, (key, k, kr)
        err = np.linalg.norm(x.cpu().numpy() - xr) / np.linalg.norm(xr)
        assert err <= 1e-10, (key, err)


def test_mixed_precision_vcycle_reaches_tolerance(M):
    prob = CASES["kappa2d_33"]()
    O, _ = _oracle(prob)
    H = _hier(M, prob, nu=3, vcycle=1, m=1, precision=M.MPCG_MIXED)
    b = torch.from_numpy(prob.b).cuda()
    x = torch.zeros_like(b)
    st, k, _, _ = H.solve(b, x, rtol=1e-8, maxit=2000)
    assert st == M.MPCG_OK
    xg = x.cpu().numpy()
    assert np.linalg.norm(prob.b - O.A[-1] @ xg) / np.linalg.norm(prob.b) <= 1e-8


def test_options_are_checked(M):
    prob = CASES["kappa2d_33"]()
    st = torch.from_numpy(prob.stencil).cuda()
    for bad in (dict(vcycle=1, sum_columns=1), dict(smoother=2), dict(smoother=1, ssor_omega=2.0),
                dict(smoother=1, vcycle=1, sum_columns=1)):
        with pytest.raises(M.MpcgError):
            M.Hierarchy(st, 2, 33, prob.levels, **bad)
    pe = pb.elasticity_cantilever(nodes=9)
    with pytest.raises(M.MpcgError):
        M.Hierarchy(torch.from_numpy(pe.stencil).cuda(), 3, 9, pe.levels, dofs_per_node=3, faces=pe.faces,
                    smoother=M.MPCG_SMOOTHER_SSOR)


@pytest.mark.parametrize("omega", [0.8, 1.4])
def test_ssor_relaxation_factor(M, omega):
    """SSOR with omega != 1 (under- and over-relaxed) against the oracle:
    the level corrections and the V(3,3) cycle to 1e-12."""
    prob = CASES["kappa2d_33"]()
    H = _hier(M, prob, nu=6, ssor_omega=omega)
    O = omg.Hierarchy(prob.dim, None, prob.stencil, prob.levels, nodes=prob.nodes, faces=prob.faces)
    Ss = oss.level_smoothers(O, omega)
    r = np.random.default_rng(7).standard_normal(prob.n)
    Z = torch.zeros((prob.levels, prob.n), dtype=torch.float64, device="cuda")
    M.mg_corrections(H.h, torch.from_numpy(r).cuda(), Z)
    ref = oss.additive_columns(O, Ss, r, 6)
    got = Z.cpu().numpy().T
    for j in range(prob.levels):
        assert np.abs(got[:, j] - ref[:, j]).max() <= 1e-12 * np.abs(ref[:, j]).max(), j
    Hv = _hier(M, prob, nu=3, vcycle=1, m=1, ssor_omega=omega)
    Zv = torch.zeros((1, prob.n), dtype=torch.float64, device="cuda")
    M.mg_corrections(Hv.h, torch.from_numpy(r).cuda(), Zv)
    refv = oss.vcycle(O, Ss, r, 3)
    assert np.abs(Zv.cpu().numpy()[0] - refv).max() <= 1e-12 * np.abs(refv).max()


@pytest.mark.parametrize("name", ["kappa2d_33", "kappa3d_17", "example1_1e-3"])
def test_jacobi_vcycle_matches_oracle(M, name):
    """The V(nu, nu) cycle with damped-Jacobi smoothing (nu = 3, odd: the
    post-smoothing ends in the ping-pong buffer and is copied back) and the
    MG(V)-PCG solve against the oracle."""
    prob = CASES[name]()
    st = torch.from_numpy(np.ascontiguousarray(prob.stencil)).cuda()
    H = M.Hierarchy(st, prob.dim, prob.nodes, prob.levels, faces=prob.faces, nu=3, vcycle=1, m=1)
    O = omg.Hierarchy(prob.dim, None, prob.stencil, prob.levels, nodes=prob.nodes, faces=prob.faces)
    Sm = oss.jacobi_smoothers(O)
    r = np.random.default_rng(3).standard_normal(prob.n)
    Z = torch.zeros((1, prob.n), dtype=torch.float64, device="cuda")
    M.mg_corrections(H.h, torch.from_numpy(r).cuda(), Z)
    ref = oss.vcycle(O, Sm, r, 3)
    assert np.abs(Z.cpu().numpy()[0] - ref).max() <= 1e-12 * np.abs(ref).max()
    b = torch.from_numpy(prob.b).cuda()
    x = torch.zeros_like(b)
    st_, k, _, _ = H.solve(b, x, rtol=1e-8, maxit=2000)
    xr, kr, _ = opcg.pcg(O.A[-1], prob.b, lambda v: oss.vcycle(O, Sm, v, 3), rtol=1e-8, maxit=2000)
    assert st_ == M.MPCG_OK and abs(k - kr) <= 1, (k, kr)
    assert np.linalg.norm(x.cpu().numpy() - xr) <= 1e-10 * np.linalg.norm(xr)
