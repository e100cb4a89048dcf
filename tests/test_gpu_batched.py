"""Batched solves: many independent problems per launch, uneven sizes across
concurrent size classes.  A problem solved inside a batch must give the
result of its own single solve (same kernels, same reduction layout: the
comparison is bitwise), and every problem must reach its tolerance."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mg as omg
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _single(M, prob, **opts):
    H = M.Hierarchy(_dev(prob.stencil), prob.dim, prob.nodes, prob.levels, **opts)
    x = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    st, k, _, _ = H.solve(_dev(prob.b), x, rtol=1e-8, maxit=2000, histories=False)
    return k, x.cpu().numpy()


def _true_res(prob, x):
    O = omg.Hierarchy(prob.dim, prob.n1, prob.stencil, prob.levels)
    return np.linalg.norm(prob.b - O.A[-1] @ x) / np.linalg.norm(prob.b)


@pytest.mark.parametrize("nodes,dim", [(33, 2), (9, 3)])
def test_batch_equals_single_solves_bitwise(M, nodes, dim):
    probs = [pb.diffusion_macro(dim, nodes, 300 + i, rhs="normal", rhs_seed=400 + i) for i in range(4)]
    B = M.BatchedHierarchy([_dev(p.stencil) for p in probs], dim, nodes, probs[0].levels)
    b = _dev(np.stack([p.b for p in probs]))
    x = torch.zeros_like(b)
    st, its = B.solve(b, x, rtol=1e-8, maxit=2000)
    assert st == M.MPCG_OK
    X = x.cpu().numpy()
    for i, p in enumerate(probs):
        k, xs = _single(M, p)
        assert its[i] == k
        assert np.array_equal(X[i], xs)


def test_batch_mixed_precision_reaches_tolerance(M):
    probs = [pb.diffusion_macro(2, 65, 500 + i, rhs="normal", rhs_seed=600 + i) for i in range(5)]
    B = M.BatchedHierarchy([_dev(p.stencil) for p in probs], 2, 65, probs[0].levels, precision=M.MPCG_MIXED)
    b = _dev(np.stack([p.b for p in probs]))
    x = torch.zeros_like(b)
    st, its = B.solve(b, x, rtol=1e-8, maxit=3000)
    assert st == M.MPCG_OK
    X = x.cpu().numpy()
    for i, p in enumerate(probs):
        assert _true_res(p, X[i]) <= 1e-8
        k, xs = _single(M, p, precision=M.MPCG_MIXED)
        assert np.linalg.norm(X[i] - xs) <= 1e-6 * np.linalg.norm(xs)


def test_zero_rhs_problem_in_a_batch(M):
    probs = [pb.poisson_random(2, 33, 1), pb.poisson_random(2, 33, 2)]
    probs[1].b = np.zeros_like(probs[1].b)
    B = M.BatchedHierarchy([_dev(p.stencil) for p in probs], 2, 33, probs[0].levels)
    b = _dev(np.stack([p.b for p in probs]))
    x = torch.zeros_like(b)
    st, its = B.solve(b, x)
    assert st == M.MPCG_OK and its[1] == 0 and its[0] > 0
    assert torch.count_nonzero(x[1]) == 0


def test_uneven_batch_in_concurrent_classes(M):
    sizes = {33: 3, 65: 2, 129: 1}
    classes, bs, xs, probs = [], [], [], []
    streams = [torch.cuda.Stream() for _ in sizes]
    for (nodes, cnt), strm in zip(sizes.items(), streams):
        ps = [pb.batch_problem(len(probs) + i, nodes) for i in range(cnt)]
        probs.append(ps)
        classes.append(M.BatchedHierarchy([_dev(p.stencil) for p in ps], 2, nodes, ps[0].levels,
                                          precision=M.MPCG_MIXED, stream=strm.cuda_stream))
        bs.append(_dev(np.stack([p.b for p in ps])))
        xs.append(torch.zeros_like(bs[-1]))
    torch.cuda.synchronize()
    st, its = M.mpcg_solve_batched(classes, bs, xs, rtol=1e-8, maxit=4000)
    assert st == M.MPCG_OK
    for ps, x, it in zip(probs, xs, its):
        X = x.cpu().numpy()
        for i, p in enumerate(ps):
            assert it[i] > 0
            assert _true_res(p, X[i]) <= 1e-8


def _classes(M, sizes, precision, first=0):
    classes, bs, probs = [], [], []
    for nodes, cnt in sizes.items():
        ps = [pb.batch_problem(first + len(probs) * 7 + i, nodes) for i in range(cnt)]
        probs.append(ps)
        strm = torch.cuda.Stream()
        classes.append(M.BatchedHierarchy([_dev(p.stencil) for p in ps], 2, nodes, ps[0].levels,
                                          precision=precision, stream=strm.cuda_stream))
        bs.append(_dev(np.stack([p.b for p in ps])))
    torch.cuda.synchronize()
    return classes, bs, probs


def test_one_graph_batch_equals_per_class_solves(M):
    """mpcg_solve_batched_graph (every class's mixed-precision solve a branch
    of one CUDA graph, one launch) gives bitwise the per-class solves'
    results and iteration counts, on a rebuilt graph and on the cached one,
    with device and with host arrays."""
    sizes = {33: 3, 65: 2, 129: 1}
    classes, bs, probs = _classes(M, sizes, M.MPCG_MIXED)
    ref_x, ref_it = [], []
    for c, b in zip(classes, bs):
        x = torch.zeros_like(b)
        st, it = c.solve(b, x, rtol=1e-8, maxit=4000)
        assert st == M.MPCG_OK
        ref_x.append(x.cpu().numpy())
        ref_it.append(np.array(it))
    for call in range(2):   # the second call reuses the cached graph
        xs = [torch.zeros_like(b) for b in bs]
        st, its = M.mpcg_solve_batched(classes, bs, xs, rtol=1e-8, maxit=4000, one_graph=True)
        assert st == M.MPCG_OK
        for x, it, rx, ri in zip(xs, its, ref_x, ref_it):
            assert np.array_equal(it, ri), (call, it, ri)
            assert np.array_equal(x.cpu().numpy(), rx), call
    # host arrays (staged through each class's buffers)
    bh = [b.cpu().numpy() for b in bs]
    xh = [np.zeros_like(b) for b in bh]
    st, its = M.mpcg_solve_batched(classes, bh, xh, rtol=1e-8, maxit=4000, one_graph=True)
    assert st == M.MPCG_OK
    for x, rx in zip(xh, ref_x):
        assert np.array_equal(x, rx)
    for ps, x in zip(probs, ref_x):
        for i, p in enumerate(ps):
            assert _true_res(p, x[i]) <= 1e-8


def test_one_graph_batch_after_a_class_is_replaced(M):
    """A destroyed class drops the cached graphs that hold it; a new class
    in its place gets a new graph (results equal its own solve)."""
    classes, bs, _ = _classes(M, {33: 2, 65: 1}, M.MPCG_MIXED, first=40)
    xs = [torch.zeros_like(b) for b in bs]
    M.mpcg_solve_batched(classes, bs, xs, rtol=1e-8, maxit=4000, one_graph=True)
    classes[1].close()
    new, nbs, _ = _classes(M, {65: 2}, M.MPCG_MIXED, first=60)
    classes[1], bs[1] = new[0], nbs[0]
    xs = [torch.zeros_like(b) for b in bs]
    st, its = M.mpcg_solve_batched(classes, bs, xs, rtol=1e-8, maxit=4000, one_graph=True)
    assert st == M.MPCG_OK
    x1 = torch.zeros_like(bs[1])
    st1, it1 = classes[1].solve(bs[1], x1, rtol=1e-8, maxit=4000)
    assert np.array_equal(np.array(it1), its[1]) and torch.equal(x1, xs[1])


def test_one_graph_batch_refuses_other_precisions(M):
    """The one-graph entry takes mixed-precision classes only; the general
    entry point runs an FP64 class among them from host threads."""
    classes, bs, probs = _classes(M, {33: 2}, M.MPCG_MIXED, first=80)
    c64, b64, p64 = _classes(M, {65: 1}, M.MPCG_FP64, first=90)
    allc, allb = classes + c64, bs + b64
    xs = [torch.zeros_like(b) for b in allb]
    with pytest.raises(M.MpcgError):
        M.mpcg_solve_batched(allc, allb, xs, rtol=1e-8, maxit=4000, one_graph=True)
    with pytest.raises(M.MpcgError):   # a class twice
        M.mpcg_solve_batched(classes + classes, bs + bs, [xs[0], xs[0]], rtol=1e-8, maxit=4000, one_graph=True)
    st, its = M.mpcg_solve_batched(allc, allb, xs, rtol=1e-8, maxit=4000)
    assert st == M.MPCG_OK
    for ps, x in zip(probs + p64, xs):
        X = x.cpu().numpy()
        for i, p in enumerate(ps):
            assert _true_res(p, X[i]) <= 1e-8


def test_profiled_solve_of_a_batch(M):
    """mpcg_solve_profiled on a batched hierarchy (direct launches with
    per-launch CUDA events) returns one iteration count per problem, those of
    the graph-launched solve, and iterates that agree with it."""
    classes, bs, _ = _classes(M, {65: 3}, M.MPCG_MIXED, first=120)
    c, b = classes[0], bs[0]
    x0 = torch.zeros_like(b)
    st, it = c.solve(b, x0, rtol=1e-8, maxit=4000)
    x1 = torch.zeros_like(b)
    st1, it1, cls, trace = M.mpcg_solve_profiled(c.h, b, x1, 1e-8, 4000)
    assert st1 == st == M.MPCG_OK
    assert np.asarray(it1).shape == (3,)
    assert np.all(np.abs(np.asarray(it1) - np.asarray(it)) <= 1), (it1, it)
    assert torch.linalg.norm(x1 - x0) <= 1e-6 * torch.linalg.norm(x0)
    assert sum(1 for k, _ in trace if k == "check") >= int(np.max(it))
