"""The allocation-free stencil product against the allocating one.

mg_stencil_apply_noalloc serves callers that cannot call cudaMalloc (device
memory owned by another framework's pool, or loops that must not call
cudaFree because it synchronises the device).  It keeps its scratch in one
static device array, so this file checks it through the C ABI against
mg_apply_operator on two calls in a row (the second call must not see the
first call's leftovers) and checks that oversized grids are refused.  The
file is named to run last, so that a failure here leaves every other test
already run.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2402_12833_gb300 import problems as pb

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_12833_gb300 import build, mpcg
    build.build()
    return mpcg


def _call(M, prob, X):
    lib = M.load()
    st = torch.from_numpy(np.ascontiguousarray(prob.stencil)).cuda()
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.full_like(Xd, np.nan)
    status = lib.mg_stencil_apply_noalloc(prob.dim, prob.nodes, ctypes.c_void_p(st.data_ptr()),
                                          ctypes.c_void_p(Xd.data_ptr()), ctypes.c_void_p(Yd.data_ptr()),
                                          X.shape[0], None)
    assert status == M.MPCG_OK, M.mpcg_last_error()
    torch.cuda.synchronize()
    return Yd.cpu().numpy()


def _reference(M, prob, X):
    st = torch.from_numpy(np.ascontiguousarray(prob.stencil)).cuda()
    H = M.Hierarchy(st, prob.dim, prob.nodes, prob.levels)
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.zeros_like(Xd)
    M.mg_apply_operator(H.h, prob.levels - 1, Xd, Yd, X.shape[0])
    H.close()
    return Yd.cpu().numpy()


@pytest.mark.parametrize("dim,nodes,ncols", [(3, 17, 5), (2, 65, 12), (3, 33, 3), (2, 161, 4), (3, 13, 2)])
def test_noalloc_matches_allocating_entry_point_twice(lib, dim, nodes, ncols):
    # 161 and 13 nodes: element counts that are not powers of two (Example 1's
    # 160 x 160 elements; 12 = 3 * 2^2), which the hierarchy accepts as well
    if (nodes - 1) & (nodes - 2):
        st = pb.assemble_diffusion(dim, nodes)
        prob = pb.Problem(dim, nodes, 4 if nodes == 161 else 2, st, pb.normal(4, (nodes - 2) ** dim), name="odd")
    else:
        prob = pb.diffusion_macro(dim, nodes, 21, rhs="normal", rhs_seed=4)
    for call in range(2):
        X = pb.normal(500 + call, ncols * prob.n).reshape(ncols, prob.n)
        got = _call(lib, prob, X)
        ref = _reference(lib, prob, X)
        scale = np.abs(prob.stencil).max() * np.abs(X).max()
        assert np.abs(got - ref).max() <= 1e-14 * scale * 27, call


def test_noalloc_smaller_grid_after_larger_one(lib):
    # leftovers of a larger call must not leak into a smaller one
    big = pb.diffusion_macro(3, 33, 3, rhs="normal", rhs_seed=1)
    _call(lib, big, pb.normal(1, 4 * big.n).reshape(4, big.n))
    small = pb.poisson_random(2, 17, 2)
    X = pb.normal(2, 2 * small.n).reshape(2, small.n)
    assert np.allclose(_call(lib, small, X), _reference(lib, small, X), rtol=0, atol=1e-13)


def test_noalloc_rejects_grids_beyond_the_scratch(lib):
    lib_ = lib.load()
    st = torch.zeros(27, 8, dtype=torch.float64, device="cuda")
    X = torch.zeros(8, dtype=torch.float64, device="cuda")
    status = lib_.mg_stencil_apply_noalloc(3, 65, ctypes.c_void_p(st.data_ptr()), ctypes.c_void_p(X.data_ptr()),
                                           ctypes.c_void_p(X.data_ptr()), 1, None)
    assert status == lib.MPCG_ERR_ARG
    assert "scratch" in lib.mpcg_last_error()
    # a good call afterwards clears the message
    small = pb.poisson_random(2, 17, 2)
    _call(lib, small, pb.normal(3, small.n).reshape(1, small.n))
    assert lib.mpcg_last_error() == ""
