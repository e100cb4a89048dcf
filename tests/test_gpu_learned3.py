"""The learned column of 3D vector problems (the 3x3x3 network of the
elasticity hierarchy) on the GPU, against the CPU oracle.

As for the 2D network: every layer of the forward pass is checked element
by element from the GPU's own bfloat16 inputs (each output must be the
oracle's bfloat16 rounding of the exact 3x3x3 convolution, or one of its two
neighbours where the FP32 accumulation bound leaves the rounding undecided);
at 65^3 and 129^3 nodes the same check runs on sampled nodes (faces, edges,
corners, tile and row-block boundaries, and random ones).  Weight gradients
are checked entry by entry against the oracle's backward pass on the GPU's
activations, within the accumulation bound of each entry's absolute sum.
The solver with the network attached follows the oracle MPCG using the same
network as its extra column, and training on solver-made pairs lowers the
A-angle loss.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import learned as OL
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


def _hier(M, prob, **opts):
    st = torch.from_numpy(np.ascontiguousarray(prob.stencil)).cuda()
    return M.Hierarchy(st, prob.dim, prob.nodes, prob.levels, dofs_per_node=3, faces=prob.faces, **opts)


def _oracle(prob):
    return omg.Hierarchy(3, None, prob.stencil, prob.levels, nodes=prob.nodes, faces=prob.faces, ncomp=3)


def _zyx(prob):
    return tuple(prob.shape[::-1])


def _bf(x):
    return OL.bf16(np.asarray(x, dtype=np.float32)).astype(np.float64)


def _bounds(z, zabs, K):
    """FP32 accumulation of K exact products: |error| <= (K + 2) 2^-23 sum|w a|."""
    return (K + 2) * 2.0 ** -23 * zabs


def _check_relu_out(z, zabs, K, out):
    """out: GPU bfloat16 outputs after ReLU; returns (ambiguous, flips)."""
    err = _bounds(z, zabs, K)
    lo = _bf(np.maximum(z - err, 0.0))
    hi = _bf(np.maximum(z + err, 0.0))
    bad = (out < lo) | (out > hi)
    assert not bad.any(), (int(bad.sum()), np.argwhere(bad)[:5])
    return int((lo != hi).sum()), int((out != _bf(np.maximum(z, 0.0))).sum())


def _check_forward_full(theta, rhat, acts, y, zyx):
    """acts: (4, nn, 16) of one image, y: (n,) vector layout."""
    Wq = [OL.bf16(W).astype(np.float64) for W in OL.unpack3(theta)]
    A = acts.reshape(4, *zyx, 16).transpose(0, 4, 1, 2, 3).astype(np.float64)
    assert np.array_equal(A[0, :3], OL.to_image3(_bf(rhat), zyx))
    assert not np.any(A[0, 3:])
    amb = flips = 0
    for i in range(3):
        a_in = A[i, :3] if i == 0 else A[i]
        z = OL.conv3(a_in, Wq[i])
        zabs = OL.conv3(np.abs(a_in), np.abs(Wq[i]))
        n_amb, n_flip = _check_relu_out(z, zabs, a_in.shape[0] * 27, A[i + 1])
        amb += n_amb
        flips += n_flip
    z = OL.conv3(A[3], Wq[3])
    err = _bounds(z, OL.conv3(np.abs(A[3]), np.abs(Wq[3])), 16 * 27)
    yi = OL.to_image3(y.astype(np.float64), zyx)
    assert np.all(np.abs(yi - z) <= err + 1e-30), np.max(np.abs(yi - z) / (err + 1e-30))
    # K = 432 products: the worst-case bound leaves about 15 % undecided
    assert amb <= 0.3 * 3 * 16 * A[0, 0].size, amb
    return flips


@pytest.mark.parametrize("nodes", [9, 17, 33])
def test_forward3_matches_oracle_layer_by_layer(M, nodes):
    """Two images, every node and channel of every layer (9: 8 x 9 x 9 nodes,
    17: row blocks of 4 with a ragged last one, 33: 32 x 33 x 33)."""
    prob = pb.elasticity_cantilever(nodes)
    H = _hier(M, prob)
    theta = OL.init_params3(7)
    assert M.mg_learned_num_params_of(H.h) == OL.n_params3() == 16416
    M.mg_learned_attach(H.h, theta)
    assert M.mg_num_columns(H.h) == prob.levels + 1
    R = np.stack([pb.normal(3 + k, prob.n) for k in range(2)])
    R /= np.linalg.norm(R, axis=1, keepdims=True)
    R = R.astype(np.float32)
    nn = prob.n // 3
    Y = torch.zeros((2, prob.n), dtype=torch.float32, device="cuda")
    acts = torch.full((4, 2, nn, 16), np.nan, dtype=torch.float32, device="cuda")
    M.mg_learned_forward_acts(H.h, torch.from_numpy(R).cuda(), Y, acts, 2)
    acts, Yh = acts.cpu().numpy(), Y.cpu().numpy()
    flips = [_check_forward_full(theta, R[k], acts[:, k], Yh[k], _zyx(prob)) for k in range(2)]
    Y2 = torch.zeros_like(Y)
    M.mg_learned_forward(H.h, torch.from_numpy(R).cuda(), Y2, 2)
    assert torch.equal(Y, Y2)
    print("bfloat16 flips per image:", flips)


def _sample_nodes(zyx, count, seed):
    """Nodes (z, y, x) on faces, edges and corners, at the 128-node tile edge
    and the 4-row block edges, and random ones."""
    Z, Y, X = zyx
    rng = np.random.default_rng(seed)
    special = []
    for z in (0, 1, Z // 2, Z - 2, Z - 1):
        for y in (0, 3, 4, Y - 2, Y - 1):
            for x in (0, 1, min(X - 1, 127), X - 1):
                special.append((z, y, x))
    rnd = np.stack([rng.integers(0, Z, count), rng.integers(0, Y, count), rng.integers(0, X, count)], axis=1)
    return np.unique(np.concatenate([np.array(special), rnd]), axis=0)


def _patches(act_img, pts, zyx):
    """(npts, 16, 3, 3, 3) neighbourhoods of nodes pts in act_img ((nn, 16)
    on the device), zero outside the grid; gathered on the device."""
    Z, Y, X = zyx
    off = np.array([(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)])
    c = pts[:, None, :] + off[None, :, :]
    ok = np.all((c >= 0) & (c < np.array(zyx)), axis=2)
    flat = np.where(ok, (c[..., 0] * Y + c[..., 1]) * X + c[..., 2], 0)
    g = act_img[torch.from_numpy(flat.reshape(-1)).cuda()].cpu().numpy().reshape(len(pts), 27, 16)
    g[~ok] = 0.0
    return g.reshape(len(pts), 3, 3, 3, 16).transpose(0, 4, 1, 2, 3).astype(np.float64)


@pytest.mark.parametrize("nodes", [65, 129])
def test_forward3_sampled_at_full_size(M, nodes):
    """65^3 (the cantilever of the elasticity workload) and 129^3 (two
    128-node tile columns, the second one all pads): every layer at sampled
    nodes, from the GPU's own inputs of the layer."""
    prob = pb.elasticity_cantilever(nodes)
    H = _hier(M, prob)
    theta = OL.init_params3(11)
    M.mg_learned_attach(H.h, theta)
    Wq = [OL.bf16(W).astype(np.float64) for W in OL.unpack3(theta)]
    zyx = _zyx(prob)
    nn = prob.n // 3
    r = pb.normal(17, prob.n)
    r = (r / np.linalg.norm(r)).astype(np.float32)
    Y = torch.zeros((1, prob.n), dtype=torch.float32, device="cuda")
    acts = torch.full((4, 1, nn, 16), np.nan, dtype=torch.float32, device="cuda")
    M.mg_learned_forward_acts(H.h, torch.from_numpy(r).cuda(), Y, acts, 1)
    assert not torch.isnan(acts).any()
    # the input layer everywhere
    a0 = acts[0, 0].cpu().numpy()
    assert np.array_equal(a0[:, :3], _bf(r).reshape(nn, 3))
    assert not np.any(a0[:, 3:])
    pts = _sample_nodes(zyx, 400, nodes)
    Yh = Y[0].cpu().numpy()
    Z, Yn, X = zyx
    q = (pts[:, 0] * Yn + pts[:, 1]) * X + pts[:, 2]
    for i in range(4):
        P = _patches(acts[i, 0], pts, zyx)
        if i == 0:
            P = P[:, :3]
        z = np.stack([OL.conv3(P[j], Wq[i])[:, 1, 1, 1] for j in range(len(pts))])
        zabs = np.stack([OL.conv3(np.abs(P[j]), np.abs(Wq[i]))[:, 1, 1, 1] for j in range(len(pts))])
        K = P.shape[1] * 27
        if i < 3:
            out = acts[i + 1, 0][torch.from_numpy(q).cuda()].cpu().numpy().astype(np.float64)
            _check_relu_out(z, zabs, K, out)
        else:
            yv = Yh.reshape(nn, 3)[q].astype(np.float64)
            assert np.all(np.abs(yv - z) <= _bounds(z, zabs, K) + 1e-30)


def _oracle_grad_on3(theta, acts, y, R, E, A, zyx):
    """The oracle's backward pass on the GPU's activations and outputs:
    (gradient, scale, mean loss); scale[i] bounds the rounding of entry i
    (the same sums over absolute values, A y and A e taken as |A| |y| and
    |A| |e|, the FP32 operator's products)."""
    Wq = [OL.bf16(W).astype(np.float64) for W in OL.unpack3(theta)]
    absA = abs(A)
    B = R.shape[0]
    g = np.zeros(OL.n_params3())
    sc = np.zeros(OL.n_params3())
    Ls = 0.0
    for k in range(B):
        Ak = acts[:, k].reshape(4, *zyx, 16).transpose(0, 4, 1, 2, 3).astype(np.float64)
        ins = [Ak[0, :3], Ak[1], Ak[2], Ak[3]]
        yk = y[k].astype(np.float64)
        e = E[k].astype(np.float64)
        Ay, Ae = A @ yk, A @ e
        L, dy = OL.angle_loss(yk, e, Ay, Ae)
        Ls += L / B
        eAy, eAe, yAy = e @ Ay, e @ Ae, yk @ Ay
        k1, k2 = 2.0 * eAy / (eAe * yAy), eAy / yAy
        d = OL.to_image3(dy / B, zyx)
        dabs = OL.to_image3(abs(k1) * (absA @ np.abs(e) + abs(k2) * (absA @ np.abs(yk))) / B, zyx)
        gl, sl = [None] * 4, [None] * 4
        for i in range(3, -1, -1):
            gl[i] = OL.conv3_wgrad(d, ins[i])
            sl[i] = OL.conv3_wgrad(dabs, np.abs(ins[i]))
            if i > 0:
                d = OL.conv3_transpose(d, Wq[i]) * (ins[i] > 0)
                dabs = OL.conv3_transpose(dabs, np.abs(Wq[i])) * (ins[i] > 0)
        g += np.concatenate([x.reshape(-1) for x in gl])
        sc += np.concatenate([x.reshape(-1) for x in sl])
    return g, sc, Ls


@pytest.mark.parametrize("nodes,B", [(9, 3), (17, 2)])
def test_weight_gradients3_match_oracle(M, nodes, B):
    """mg_learned_grad on the 3D network: the training forward layer by
    layer, then every gradient entry against the oracle's backward pass on the
    GPU's activations, within 1e-4 of the entry's absolute sum (the FP32
    gradients enter the tensor cores as bfloat16 hi + lo pairs, 2^-17, and
    accumulate in FP32 over three layers)."""
    prob = pb.elasticity_cantilever(nodes)
    H = _hier(M, prob)
    theta = OL.init_params3(5)
    zyx = _zyx(prob)
    R = np.stack([pb.normal(40 + k, prob.n) for k in range(B)])
    R /= np.linalg.norm(R, axis=1, keepdims=True)
    E = np.stack([pb.normal(50 + k, prob.n) for k in range(B)])
    R, E = R.astype(np.float32), E.astype(np.float32)
    nn = prob.n // 3
    acts = torch.full((4, B, nn, 16), np.nan, dtype=torch.float32, device="cuda")
    Y = torch.zeros((B, prob.n), dtype=torch.float32, device="cuda")
    g_gpu, loss = M.mg_learned_grad(H.h, theta, torch.from_numpy(R).cuda(), torch.from_numpy(E).cuda(), B,
                                    acts_dev=acts, y_dev=Y)
    acts, Yh = acts.cpu().numpy(), Y.cpu().numpy()
    for k in range(B):
        _check_forward_full(theta, R[k], acts[:, k], Yh[k], zyx)
    A = stencil_to_csr(3, prob.shape, prob.stencil, ncomp=3)
    g_orc, scale, L_orc = _oracle_grad_on3(theta, acts, Yh, R, E, A, zyx)
    rel = np.abs(g_gpu - g_orc) / (scale + 1e-30)
    print("largest |error| / scale:", rel.max())
    assert rel.max() <= 1e-4, (int((rel > 1e-4).sum()), rel.max())
    assert abs(loss - L_orc) <= 1e-5 * abs(L_orc)
    for part in np.split(g_gpu, np.cumsum([1296, 6912, 6912])):
        assert np.any(part != 0.0)
    # end to end against the oracle's own forward (independent roundings)
    _, g_ind = OL.batch_grad3(theta, [(R[k].astype(np.float64), E[k].astype(np.float64), A) for k in range(B)], zyx)
    assert np.linalg.norm(g_gpu - g_ind) <= 3e-2 * np.linalg.norm(g_ind)


@pytest.mark.parametrize("B,batch", [(4, 4), (3, 4)])
def test_training3_step_applies_the_gradient(M, B, batch):
    """First Adam step with beta1 = 0 and eps >> |g|: -lr g / (|g| + eps),
    also for a batch shorter than the batch size."""
    prob = pb.elasticity_cantilever(9)
    H = _hier(M, prob)
    theta = OL.init_params3(5)
    R = np.stack([pb.normal(40 + k, prob.n) for k in range(B)])
    R /= np.linalg.norm(R, axis=1, keepdims=True)
    E = np.stack([pb.normal(50 + k, prob.n) for k in range(B)])
    R, E = R.astype(np.float32), E.astype(np.float32)
    Rd, Ed = torch.from_numpy(R).cuda(), torch.from_numpy(E).cuda()
    g_ref, _ = M.mg_learned_grad(H.h, theta, Rd, Ed, B)
    params = theta.copy()
    lr = eps = 1e3
    M.mg_learned_train([H.h], [0] * B, Rd, Ed, params, epochs=1, batch=batch, lr=lr, beta1=0.0, beta2=0.999, eps=eps)
    step = params.astype(np.float64) - theta.astype(np.float64)
    g32 = g_ref.astype(np.float32).astype(np.float64)
    want = -lr * g32 / (np.abs(g32) + eps)
    assert np.all(np.abs(step - want) <= 4 * np.spacing(np.abs(theta).astype(np.float32)).astype(np.float64)
                  + 1e-6 * np.abs(want)), np.max(np.abs(step - want))


def _extra3(theta, zyx):
    def extra(r):
        nr = np.linalg.norm(r)
        y, _ = OL.forward3(theta, OL.to_image3(r / nr, zyx))
        return nr * OL.from_image3(y)
    return extra


@pytest.mark.parametrize("nodes", [9, 17])
def test_solver3_with_learned_column_matches_oracle(M, nodes):
    """FP64 MPCG with the 3D network as the extra column against the oracle
    MPCG with the oracle network: iteration counts within 2 (or 10 %), the
    same FP64 solution tolerance, and the column takes part."""
    prob = pb.elasticity_cantilever(nodes)
    H = _hier(M, prob)
    theta = OL.init_params3(9)
    M.mg_learned_attach(H.h, theta)
    b = torch.from_numpy(prob.b).cuda()
    x = torch.zeros_like(b)
    st, k, rh, ah = H.solve(b, x, rtol=1e-8, maxit=1000)
    O = _oracle(prob)
    ref = ompcg.mpcg(O.A[-1], prob.b, O.mg_columns, rtol=1e-8, maxit=1000, extra_column=_extra3(theta, _zyx(prob)))
    assert st == M.MPCG_OK and ref.converged
    assert abs(k - ref.iters) <= max(2, 0.1 * ref.iters), (k, ref.iters)
    assert np.linalg.norm(prob.b - O.A[-1] @ x.cpu().numpy()) <= 1.01e-8 * np.linalg.norm(prob.b)
    assert np.any(np.abs(ah[:5, -1]) > 0)
    M.mg_learned_detach(H.h)
    assert M.mg_num_columns(H.h) == prob.levels


@pytest.mark.parametrize("precision", ["fp64_dw", "mixed"])
def test_solver3_learned_column_other_precisions(M, precision):
    """The column in the double-word and the mixed-precision solvers reaches
    the FP64 tolerance on 33^3 x 3."""
    prob = pb.elasticity_cantilever(33)
    p = M.MPCG_FP64_DW if precision == "fp64_dw" else M.MPCG_MIXED
    H = _hier(M, prob, precision=p)
    M.mg_learned_attach(H.h, OL.init_params3(2))
    b = torch.from_numpy(prob.b).cuda()
    x = torch.zeros_like(b)
    st, k, _, _ = H.solve(b, x, rtol=1e-8, maxit=3000, histories=False)
    assert st == M.MPCG_OK
    A = stencil_to_csr(3, prob.shape, prob.stencil, ncomp=3)
    assert np.linalg.norm(prob.b - A @ x.cpu().numpy()) <= 1.01e-8 * np.linalg.norm(prob.b)


def test_full_size_cantilever_65_with_learned_column(M):
    """65^3 x 3 (811,200 unknowns), mixed precision with the 3D network as an
    extra column: true FP64 residual <= 1e-8."""
    prob = pb.elasticity_cantilever(65)
    H = _hier(M, prob, precision=M.MPCG_MIXED)
    M.mg_learned_attach(H.h, OL.init_params3(2))
    b = torch.from_numpy(prob.b).cuda()
    x = torch.zeros_like(b)
    st, k, _, _ = H.solve(b, x, rtol=1e-8, maxit=2000, histories=False)
    assert st == M.MPCG_OK
    A = stencil_to_csr(3, prob.shape, prob.stencil, ncomp=3)
    assert np.linalg.norm(prob.b - A @ x.cpu().numpy()) <= 1e-8 * np.linalg.norm(prob.b)
    assert x.cpu().numpy()[2::3].max() < 0.0
    print("iterations with the learned column:", k)


def _pairs3(M, prob, ks, force=None):
    """(r_k/||r_k||, e_k/||r_k||) for iterates x_k of the GPU FP64 solver."""
    H = _hier(M, prob)
    bvec = prob.b if force is None else pb.elasticity_body_force(prob.nodes, force)
    b = torch.from_numpy(bvec).cuda()
    xs = torch.zeros_like(b)
    H.solve(b, xs, rtol=1e-13, maxit=5000, histories=False)
    R, E = [], []
    Ax = torch.empty_like(b)
    for k in ks:
        x = torch.zeros_like(b)
        H.solve(b, x, rtol=1e-30, maxit=k, histories=False)
        M.mg_apply_operator(H.h, prob.levels - 1, x, Ax, 1)
        r = b - Ax
        nr = torch.linalg.norm(r)
        R.append((r / nr).float())
        E.append(((xs - x) / nr).float())
    return H, torch.stack(R).contiguous(), torch.stack(E).contiguous()


def _loss_of(M, H, prob, params, R, E):
    M.mg_learned_attach(H.h, params)
    Y = torch.zeros_like(R)
    M.mg_learned_forward(H.h, R, Y, R.shape[0])
    M.mg_learned_detach(H.h)
    Yd, Ed = Y.double().contiguous(), E.double().contiguous()
    AY, AE = torch.zeros_like(Yd), torch.zeros_like(Ed)
    M.mg_apply_operator(H.h, prob.levels - 1, Yd, AY, Yd.shape[0])
    M.mg_apply_operator(H.h, prob.levels - 1, Ed, AE, Ed.shape[0])
    eay = (Ed * AY).sum(1)
    return float((1.0 - eay * eay / ((Ed * AE).sum(1) * (Yd * AY).sum(1))).mean())


def test_training3_lowers_loss(M):
    """Training on pairs of the 17^3 cantilever under its own load lowers the
    A-angle loss on those pairs and on pairs of the same body under held-out
    loads; the trained column keeps the solver converging.  The solver needs
    about 40 steps here, so pairs come from the first 24 iterates, whose
    errors stay far above the 1e-13 accuracy of the reference solution."""
    prob = pb.elasticity_cantilever(17)
    H, R, E = _pairs3(M, prob, range(1, 25))
    init = OL.init_params3(7)
    params = init.copy()
    loss = M.mg_learned_train([H.h], [0] * R.shape[0], R, E, params, epochs=30, batch=8, lr=1e-3)
    assert loss[-1] < loss[0] - 0.02, loss
    for force in [(1.0, 0.0, 0.0), (0.0, 1.0, 1.0)]:
        Hh, Rh, Eh = _pairs3(M, prob, range(1, 25, 3), force)
        before = _loss_of(M, Hh, prob, init, Rh, Eh)
        after = _loss_of(M, Hh, prob, params, Rh, Eh)
        print("held-out loss", force, before, "->", after)
        assert after < before, (before, after)
    b = torch.from_numpy(prob.b).cuda()
    x = torch.zeros_like(b)
    _, k0, _, _ = H.solve(b, x, rtol=1e-8, maxit=1000, histories=False)
    its = {}
    for name, p in (("initial", init), ("trained", params)):
        M.mg_learned_attach(H.h, p)
        x.zero_()
        st, its[name], _, _ = H.solve(b, x, rtol=1e-8, maxit=1000, histories=False)
        assert st == M.MPCG_OK
    print("iterations: plain", k0, "with the column", its)


def test_tensor_core_wait_timeout3_is_reported_and_recovers(M):
    """The 3D network's kernels with zero polls for their first wait (the
    weight-gradient CTAs own 16 chunks, so they give up inside their chunk
    pipeline and drain the MMAs they issued): MPCG_ERR_TIMEOUT from the
    forward and the training pass; the default limit restores the earlier
    results bitwise."""
    prob = pb.elasticity_cantilever(9)
    H = _hier(M, prob)
    theta = OL.init_params3(7)
    M.mg_learned_attach(H.h, theta)
    R = np.stack([pb.normal(3 + k, prob.n) for k in range(2)])
    R = torch.from_numpy((R / np.linalg.norm(R, axis=1, keepdims=True)).astype(np.float32)).cuda()
    E = torch.from_numpy(np.stack([pb.normal(9 + k, prob.n) for k in range(2)]).astype(np.float32)).cuda()
    Y0 = torch.zeros_like(R)
    M.mg_learned_forward(H.h, R, Y0, 2)
    g0, _ = M.mg_learned_grad(H.h, theta, R, E, 2)
    try:
        M.mg_set_tensor_wait_limit(0)
        for call in (lambda: M.mg_learned_forward(H.h, R, torch.zeros_like(R), 2),
                     lambda: M.mg_learned_grad(H.h, theta, R, E, 2)):
            with pytest.raises(M.MpcgError) as ei:
                call()
            assert ei.value.status == M.MPCG_ERR_TIMEOUT, ei.value
    finally:
        M.mg_set_tensor_wait_limit(M.MG_TENSOR_WAIT_DEFAULT)
    Y1 = torch.zeros_like(R)
    M.mg_learned_forward(H.h, R, Y1, 2)
    assert torch.equal(Y0, Y1)
    g1, _ = M.mg_learned_grad(H.h, theta, R, E, 2)
    assert np.array_equal(g0, g1)
