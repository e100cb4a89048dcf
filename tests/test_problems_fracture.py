"""The Example 2 stand-in's inputs (problems.fracture_network) against the
recipe it states, and the CSR conversion of stencil problems against the
oracle's own conversion."""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle.operators import stencil_to_csr
from paper_2402_12833_gb300 import problems as pb


@pytest.mark.parametrize("kf", [1e-4, 1.0, 1e4])
def test_fracture_permeabilities(kf):
    nodes = 129
    h = 1.0 / (nodes - 1)
    kap = pb.fracture_kappa(nodes, kf)
    vals = set(np.unique(kap).tolist())
    if kf == 1.0:
        assert vals == {1.0}
        return
    keff = 1.0 + (1e-4 / h) * (kf - 1.0) if kf > 1 else h / ((h - 1e-4) / 1.0 + 1e-4 / kf)
    assert vals == {1.0, keff}
    frac = (kap != 1.0).mean()
    assert 0.01 < frac < 0.2          # 24 fractures of length 0.15..0.5 crossing h-wide cells
    assert keff > 100 if kf > 1 else keff < 0.02       # 129 at h = 1/128 for k_f = 1e4; 0.0078 for 1e-4


def test_fracture_rhs_is_neumann_load_plus_lift():
    nodes = 65
    prob = pb.fracture_network(1e4, nodes=nodes)
    A = pb.stencil_csr(prob)
    assert abs(A - A.T).max() <= 1e-12 * abs(A).max()
    nx, ny = prob.shape
    assert (nx, ny) == (nodes - 1, nodes) and prob.faces == 0x2
    h = 1.0 / (nodes - 1)
    g = np.zeros((ny, nx))
    g[:, 0] = h
    g[0, 0] = g[-1, 0] = h / 2
    # the full operator annihilates constants: -A_{I,D} 1 = A 1 on the unknowns
    np.testing.assert_allclose(prob.b - g.reshape(-1), A @ np.ones(A.shape[0]), atol=1e-12)
    assert math.isclose(g.sum(), 1.0, rel_tol=1e-12)       # unit inflow through the left edge


def test_fracture_solution_obeys_the_maximum_principle():
    """p = 1 on the right, inflow on the left, no sources: 1 <= p, and p is
    largest on the inflow edge."""
    prob = pb.fracture_network(1e-4, nodes=65)
    A = pb.stencil_csr(prob)
    p = spla.spsolve(A.tocsc(), prob.b).reshape(prob.shape[::-1])
    assert p.min() >= 1.0 - 1e-10
    assert p[:, 0].max() == pytest.approx(p.max())


@pytest.mark.parametrize("make", [lambda: pb.diffusion_macro(2, 33, 3), lambda: pb.poisson_random(3, 9, 1),
                                  lambda: pb.diffusion_faces(2, 17, 0x5, rhs_seed=1, kappa_seed=2),
                                  lambda: pb.fracture_network(1e-2, nodes=33)])
def test_stencil_csr_equals_the_oracle_conversion(make):
    prob = make()
    A = pb.stencil_csr(prob)
    B = stencil_to_csr(prob.dim, prob.shape, prob.stencil)
    assert A.shape == B.shape and abs(A - B).max() == 0.0
    assert A.has_sorted_indices
