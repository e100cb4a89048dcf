"""The autotuner on the GPU: tuning times candidate shapes and stores one per
key; the tuned solve still meets the oracle's bar; an extreme shape set by
hand (the most and the fewest blocks the buffers allow) changes the FP64
solve only at rounding level; a cache written by one tuning serves the next
one without timing.  The table is cleared afterwards, so the other tests run
on the fixed rules."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mg as omg
from oracle import mpcg as ompcg
from paper_2402_12833_gb300 import problems as pb

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_12833_gb300 import build, mpcg
    build.build()
    mpcg.load()
    mpcg.mg_autotune_clear()
    yield mpcg
    mpcg.mg_autotune_clear()


@pytest.fixture(scope="module")
def prob():
    return pb.poisson_random(3, 65, 2)


@pytest.fixture(scope="module")
def ref(prob):
    O = omg.Hierarchy(prob.dim, prob.n1, prob.stencil, prob.levels)
    return O, ompcg.mpcg(O.A[-1], prob.b, O.mg_columns, m=5, rtol=1e-8, maxit=300)


def _hier(M, prob, precision):
    st = torch.from_numpy(np.ascontiguousarray(prob.stencil)).cuda()
    return M.Hierarchy(st, prob.dim, prob.nodes, prob.levels, m=5, precision=precision)


@pytest.mark.parametrize("precision", ["mixed", "fp64", "fp64_dw"])
def test_tuned_solve_meets_the_oracle_bar(M, prob, ref, precision, tmp_path):
    O, r = ref
    prec = {"mixed": M.MPCG_MIXED, "fp64": M.MPCG_FP64, "fp64_dw": M.MPCG_FP64_DW}[precision]
    H = _hier(M, prob, prec)
    path = str(tmp_path / "tune.json")
    timed = M.mg_autotune(H.h, path)
    assert timed >= 8, timed   # stream, Gram and SpMM candidates plus two per Jacobi grid
    kind = {"mixed": M.MG_TUNE_F32, "fp64": M.MG_TUNE_F64, "fp64_dw": M.MG_TUNE_DW}[precision]
    npts = (prob.nodes - 1 + 3) // 4 * 4 * (prob.nodes - 1) * (prob.nodes - 1)   # padded fine box
    assert M.mg_autotune_lookup(M.MG_TUNE_STREAM_BLOCKS, M.MG_TUNE_ANY, npts, 1, 0) > 0
    assert M.mg_autotune_lookup(M.MG_TUNE_SPMM_BLOCKS, kind, npts, 1, prob.levels) > 0
    b = torch.from_numpy(prob.b).cuda()
    x = torch.zeros_like(b)
    st, k, _, _ = H.solve(b, x, rtol=1e-8, maxit=300)
    xg = x.cpu().numpy()
    assert st == M.MPCG_OK
    if precision == "mixed":
        assert np.linalg.norm(prob.b - O.A[-1] @ xg) <= 1.01e-8 * np.linalg.norm(prob.b)
        assert np.linalg.norm(xg - r.x) <= 1e-5 * np.linalg.norm(r.x)
    else:
        assert abs(k - r.iters) <= 1 and np.linalg.norm(xg - r.x) <= 1e-10 * np.linalg.norm(r.x)
    # the cache holds every key: the next tuning times nothing
    M.mg_autotune_clear()
    assert M.mg_autotune(H.h, path) == 0
    assert M.mg_autotune_lookup(M.MG_TUNE_STREAM_BLOCKS, M.MG_TUNE_ANY, npts, 1, 0) > 0
    H.close()
    M.mg_autotune_clear()


@pytest.mark.parametrize("blocks", [1, 100000])
def test_extreme_shapes_are_clamped_and_exact(M, prob, ref, blocks):
    """Shapes far outside the safe range are clamped at launch (to 64 points
    per thread, to the buffers' reserve); the FP64 solve is unchanged up to
    rounding."""
    O, r = ref
    npts = (prob.nodes - 1 + 3) // 4 * 4 * (prob.nodes - 1) * (prob.nodes - 1)
    for fn, kind, C in ((M.MG_TUNE_STREAM_BLOCKS, M.MG_TUNE_ANY, 0), (M.MG_TUNE_GRAM_CHUNKS, M.MG_TUNE_ANY, 0),
                        (M.MG_TUNE_SPMM_BLOCKS, M.MG_TUNE_F64, prob.levels)):
        M.mg_autotune_set(fn, kind, npts, 1, C, blocks)
    H = _hier(M, prob, M.MPCG_FP64)
    b = torch.from_numpy(prob.b).cuda()
    x = torch.zeros_like(b)
    st, k, _, _ = H.solve(b, x, rtol=1e-8, maxit=300)
    xg = x.cpu().numpy()
    H.close()
    M.mg_autotune_clear()
    assert st == M.MPCG_OK and abs(k - r.iters) <= 1
    assert np.linalg.norm(xg - r.x) <= 1e-10 * np.linalg.norm(r.x)
