"""The sliced-ELLPACK layout the device kernels read, built by the library
on the host: emulating the kernels' indexing (one warp per slice of 32 / g
rows, lane l serving row l / g of the slice, slot k of lane l at
sptr[s] + 32 k + l) must reproduce y = M x for every operator,
prolongator and restriction of a hierarchy; padding entries are column 0,
value 0; g follows the mean-row-length rule."""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2402_12833_gb300 import problems as pb


@pytest.fixture(scope="module")
def M():
    from paper_2402_12833_gb300 import build, mpcg
    build.build()
    mpcg._lib = None
    mpcg.load()
    return mpcg


def _emulate(lg, sptr, col, val, rows, x):
    g, rps = 1 << lg, 32 >> lg
    e = np.arange(sptr[-1])
    s = np.searchsorted(sptr, e, side="right") - 1          # slice of every stored entry
    lane = (e - sptr[s]) % 32
    row = s * rps + lane // g
    keep = row < rows
    return np.bincount(row[keep], weights=val[keep] * x[col[keep]], minlength=rows), row, keep


@pytest.mark.parametrize("make", [
    lambda: (pb.stencil_csr(pb.fracture_network(1e4, nodes=129)), {}),
    lambda: (pb.stencil_csr(pb.example1(1e-6, nodes=81, levels=3)), dict(coarse_size=64)),
    lambda: (pb.stencil_csr(pb.poisson_random(3, 17, 2)), dict(coarse_size=50)),
])
def test_ell_layout_reproduces_the_products(M, make):
    A, amg = make()
    H = M.AmgHost(A, **amg)
    rng = np.random.default_rng(0)
    lgs = set()
    for j in range(H.levels):
        rp, ci, va = H.get(j, M.MPCG_AMG_A)
        mats = {M.MPCG_AMG_A: sp.csr_matrix((va, ci, rp), shape=(H.size(j), H.size(j)))}
        if j >= 1:
            rp, ci, va = H.get(j, M.MPCG_AMG_P)
            P = sp.csr_matrix((va, ci, rp), shape=(H.size(j), H.size(j - 1)))
            mats[M.MPCG_AMG_P] = P
            mats[M.MPCG_AMG_R] = P.T.tocsr()
        for which, Mat in mats.items():
            lg, sptr, col, val = H.ell(j, which)
            rows, cols = Mat.shape
            mean = Mat.nnz / rows
            want_lg = 0
            while want_lg < 5 and (2 << want_lg) <= mean / 6.0:
                want_lg += 1
            assert lg == want_lg
            lgs.add(lg)
            assert np.all(np.diff(sptr) % 32 == 0) and sptr[0] == 0
            assert len(sptr) - 1 == -(-rows // (32 >> lg))
            x = rng.standard_normal(cols)
            y, row, keep = _emulate(lg, sptr, col, val, rows, x)
            ref = Mat @ x
            assert np.abs(y - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max()), (j, which)
            # every stored entry of the matrix appears once; the rest is padding (0, 0)
            assert np.count_nonzero(val) == np.count_nonzero(Mat.data)
            assert np.all(col[val == 0] == 0) or np.all(Mat.data != 0)
            assert np.all(col[~keep] == 0) and np.all(val[~keep] == 0)
    assert 0 in lgs and max(lgs) >= 2                       # both one-lane and grouped rows are exercised
