"""The library's smoothed-aggregation setup (C++, host only: no GPU needed)
against the oracle's (oracle/amg.py) on the same matrices.

Bars: the same number of grids and grid sizes; the aggregates of every grid
equal (integer work, bit-exact); operators and prolongators within 1e-12 of
their largest entry (the sparse products sum in another order).  Bad
matrices and options are refused with MPCG_ERR_ARG.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import amg as oa
from paper_2402_12833_gb300 import problems as pb


@pytest.fixture(scope="module")
def M():
    from paper_2402_12833_gb300 import build, mpcg
    build.build()
    mpcg._lib = None
    mpcg.load()
    return mpcg


CASES = {
    "example1_1e-6_81": lambda: (pb.stencil_csr(pb.example1(1e-6, nodes=81, levels=3)), dict(coarse_size=64)),
    "example1_1_161": lambda: (pb.stencil_csr(pb.example1(1.0)), dict()),
    "kappa2d_65": lambda: (pb.stencil_csr(pb.diffusion_macro(2, 65, 3)), dict()),
    "poisson3d_17": lambda: (pb.stencil_csr(pb.poisson_random(3, 17, 2)), dict(coarse_size=50)),
    "fracture_129_blocking": lambda: (pb.stencil_csr(pb.fracture_network(1e-4, nodes=129)), dict()),
    "fracture_257_conducting": lambda: (pb.stencil_csr(pb.fracture_network(1e4, nodes=257)), dict()),
    "plain_aggregation": lambda: (pb.stencil_csr(pb.diffusion_macro(2, 65, 5)), dict(w=0.0)),
    "theta_0.25": lambda: (pb.stencil_csr(pb.example1(1e-2, nodes=81, levels=3)), dict(theta=0.25)),
    "two_grids": lambda: (pb.stencil_csr(pb.diffusion_macro(2, 65, 6)), dict(max_levels=2, coarse_size=1024)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_host_setup_matches_oracle(M, name):
    A, amg = CASES[name]()
    O = oa.AlgebraicHierarchy(A, **amg)
    H = M.AmgHost(A, **amg)
    assert H.levels == O.levels
    for j in range(O.levels):
        assert H.size(j) == O.A[j].shape[0]
        rp, ci, va = H.get(j, M.MPCG_AMG_A)
        Aj = sp.csr_matrix((va, ci, rp), shape=O.A[j].shape)
        assert abs(Aj - O.A[j]).max() <= 1e-12 * abs(O.A[j]).max(), j
        if j >= 1:
            assert np.array_equal(H.aggregates(j), O.aggregates[j]), j
            rp, ci, va = H.get(j, M.MPCG_AMG_P)
            Pj = sp.csr_matrix((va, ci, rp), shape=O.P[j].shape)
            assert abs(Pj - O.P[j]).max() <= 1e-12 * abs(O.P[j]).max(), j
    H.close()


def test_host_setup_refuses_bad_input(M):
    A = pb.stencil_csr(pb.example1(1.0, nodes=33, levels=2))
    bad = A.tolil()
    bad[0, 1] = 3.0 * bad[0, 1]
    with pytest.raises(M.MpcgError):
        M.AmgHost(bad.tocsr())
    unsorted = sp.csr_matrix((A.data.copy(), A.indices.copy(), A.indptr.copy()), shape=A.shape)
    i0, i1 = unsorted.indptr[3], unsorted.indptr[4]
    unsorted.indices[i0:i1] = unsorted.indices[i0:i1][::-1]
    unsorted.data[i0:i1] = unsorted.data[i0:i1][::-1]
    with pytest.raises(M.MpcgError):
        M.AmgHost(unsorted)
    for amg in (dict(theta=-0.1), dict(w=2.5), dict(max_levels=0), dict(coarse_size=0)):
        with pytest.raises(M.MpcgError):
            M.AmgHost(A, **amg)
    with pytest.raises(M.MpcgError):                    # 961 unknowns kept on one grid is fine ...
        M.AmgHost(pb.stencil_csr(pb.example1(1.0, nodes=65, levels=2)), max_levels=1)   # ... 3969 is not
    H = M.AmgHost(A, max_levels=1)
    assert H.levels == 1 and H.size(0) == A.shape[0]
    with pytest.raises(M.MpcgError):
        H.aggregates(0)
    assert M.load().mg_amg_host_size(H.h, 5) == -1


def test_device_setup_refuses_bad_requests_before_any_cuda_call(M):
    """mg_hierarchy_setup_algebraic checks options and the matrix before it
    touches a device, so its refusals hold on a machine without a GPU."""
    A = pb.stencil_csr(pb.example1(1.0, nodes=33, levels=2))
    cases = [
        (A, {}, dict(smoother=M.MPCG_SMOOTHER_SSOR)),   # SSOR needs grid coordinates
        (A, dict(theta=2.0), {}),
        (A, dict(coarse_size=5000), {}),
        (A, {}, dict(m=0)),
        (A, {}, dict(vcycle=1, sum_columns=1)),
    ]
    for mat, amg, opts in cases:
        with pytest.raises(M.MpcgError) as e:
            M.AlgebraicHierarchy(mat, **amg, **opts)
        assert e.value.status == M.MPCG_ERR_ARG
    bad = A.tolil()
    bad[1, 0] = 5.0 * bad[1, 0]
    with pytest.raises(M.MpcgError) as e:
        M.AlgebraicHierarchy(bad.tocsr())
    assert e.value.status == M.MPCG_ERR_ARG and "symmetric" in str(e.value)
