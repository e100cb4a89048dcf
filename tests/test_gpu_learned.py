"""The learned search column on the GPU, against the CPU oracle.

Forward passes (the tensor-core inference kernel and the training kernels)
are checked layer by layer and element by element: given the GPU's bfloat16
inputs of a layer, every output must be the oracle's bfloat16 rounding of the
exact convolution, except where the FP32 accumulation bound leaves the
rounding undecided (a counted one-ulp flip, which must then be one of the
two neighbours).  Weight gradients are checked element by element against
the oracle's backward pass run on the GPU's own activations, within the FP32
accumulation bound of each entry's absolute sum.  Training runs on the
tensor cores: the forward pass is the fused inference kernel keeping its
activations, the weight and data gradients are tcgen05 GEMMs whose FP32
gradients enter as bfloat16 hi + lo pairs (16 significant bits).  The solver with the network attached is compared with the oracle
MPCG using the same network as its extra column; training on solver-made
(residual, error) pairs must lower the loss on those pairs and on pairs of
held-out coefficient fields, and the trained column must keep the solver
converging.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import learned as OL
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
    return mpcg


def _hier(M, prob, **opts):
    st = torch.from_numpy(np.ascontiguousarray(prob.stencil)).cuda()
    return M.Hierarchy(st, prob.dim, prob.nodes, prob.levels, **opts)


def _bf(x):
    return OL.bf16(np.asarray(x, dtype=np.float32)).astype(np.float64)


def _check_layer(a_in, a_out, W, last):
    """One convolution layer, element by element.  a_in: (cin, H, W) GPU
    inputs (bfloat16 values), a_out: the GPU's outputs ((16, H, W) bfloat16
    after ReLU, or (H, W) FP32 for the last layer), W: bfloat16 weights.
    Returns (ambiguous entries, flips)."""
    z = OL.conv(a_in, W.astype(np.float64))
    zabs = OL.conv(np.abs(a_in), np.abs(W).astype(np.float64))
    # FP32 accumulation of K = cin * 9 exact products: |error| <= K u sum|w a|,
    # taken with u = 2^-23 (truncating adds) plus two spare units
    err = (a_in.shape[0] * 9 + 2) * 2.0 ** -23 * zabs
    if last:
        assert np.all(np.abs(a_out - z[0]) <= err[0] + 1e-30), np.max(np.abs(a_out - z[0]) / (err[0] + 1e-30))
        return 0, 0
    want = _bf(np.maximum(z, 0.0))
    lo = _bf(np.maximum(z - err, 0.0))
    hi = _bf(np.maximum(z + err, 0.0))
    bad = (a_out < lo) | (a_out > hi)
    assert not bad.any(), (int(bad.sum()), np.argwhere(bad)[:5])
    return int((lo != hi).sum()), int((a_out != want).sum())


def _check_forward(theta, rhat, c_orc, acts, y, n1):
    """acts: (4, n1*n1, 16) of one image, y: (n1*n1,).  Returns the flip count."""
    Wq = [OL.bf16(W) for W in OL.unpack(theta)]
    A = acts.reshape(4, n1, n1, 16).transpose(0, 3, 1, 2).astype(np.float64)
    # input channels: bfloat16 of the FP32 residual exactly; the coefficient
    # channel within one bfloat16 ulp of the oracle's (log10 rounding)
    assert np.array_equal(A[0, 0], _bf(rhat.reshape(n1, n1)))
    cw = _bf(c_orc)
    assert np.all(np.abs(A[0, 1] - cw) <= 2.0 ** -7 * np.abs(cw) + 1e-30)
    assert not np.any(A[0, 2:])
    flips = amb = 0
    for i in range(3):
        a_in = A[i, :2] if i == 0 else A[i]
        n_amb, n_flip = _check_layer(a_in, A[i + 1], Wq[i], False)
        amb += n_amb
        flips += n_flip
    _check_layer(A[3], y.reshape(n1, n1).astype(np.float64), Wq[3], True)
    # the worst-case bound leaves a few per cent of the entries undecided
    assert amb <= 0.1 * 3 * 16 * n1 * n1, amb
    return flips


def _cchan(prob):
    centre = 4
    return OL.coefficient_channel(prob.stencil[centre]).reshape(prob.n1, prob.n1)


@pytest.mark.parametrize("nodes", [65, 129])
def test_forward_matches_oracle_layer_by_layer(M, nodes):
    """The tensor-core inference kernel: 2 images, every layer element-wise
    (65^2: one tile column, eight tile rows with a ragged last one; 129^2:
    two tile columns, the second ragged)."""
    prob = pb.diffusion_macro(2, nodes, 21)
    H = _hier(M, prob)
    theta = OL.init_params(7)
    M.mg_learned_attach(H.h, theta)
    R = np.stack([pb.normal(3 + k, prob.n) for k in range(2)])
    R /= np.linalg.norm(R, axis=1, keepdims=True)
    R = R.astype(np.float32)
    Y = torch.zeros((2, prob.n), dtype=torch.float32, device="cuda")
    acts = torch.full((4, 2, prob.n, 16), np.nan, dtype=torch.float32, device="cuda")
    M.mg_learned_forward_acts(H.h, torch.from_numpy(R).cuda(), Y, acts, 2)
    acts = acts.cpu().numpy()
    Yh = Y.cpu().numpy()
    c = _cchan(prob)
    flips = [_check_forward(theta, R[k], c, acts[:, k], Yh[k], prob.n1) for k in range(2)]
    # the plain forward entry point gives the same outputs
    Y2 = torch.zeros_like(Y)
    M.mg_learned_forward(H.h, torch.from_numpy(R).cuda(), Y2, 2)
    assert torch.equal(Y, Y2)
    print("bfloat16 flips per image:", flips)


def _oracle_grad_on(theta, acts, y, R, E, A, n1):
    """The oracle's backward pass on the GPU's activations and outputs:
    (gradient, scale, mean loss), scale[i] = sum of |terms| of entry i with
    |dy| replaced by the magnitude of its terms (the bound of its rounding)."""
    Wq = [OL.bf16(W).astype(np.float64) for W in OL.unpack(theta)]
    B = R.shape[0]
    g = np.zeros(OL.n_params())
    sc = np.zeros(OL.n_params())
    Ls = 0.0
    for k in range(B):
        Ak = acts[:, k].reshape(4, n1, n1, 16).transpose(0, 3, 1, 2).astype(np.float64)
        ins = [Ak[0, :2], Ak[1], Ak[2], Ak[3]]
        yk = y[k].astype(np.float64)
        e = E[k].astype(np.float64)
        Ay, Ae = A @ yk, A @ e
        L, dy = OL.angle_loss(yk, e, Ay, Ae)
        Ls += L / B
        eAy, eAe, yAy = e @ Ay, e @ Ae, yk @ Ay
        k1, k2 = 2.0 * eAy / (eAe * yAy), eAy / yAy
        d = (dy / B).reshape(1, n1, n1)
        dabs = (abs(k1) * (np.abs(Ae) + abs(k2) * np.abs(Ay)) / B).reshape(1, n1, n1)
        gl, sl = [None] * 4, [None] * 4
        for i in range(3, -1, -1):
            gl[i] = OL.conv_wgrad(d, ins[i])
            sl[i] = OL.conv_wgrad(dabs, np.abs(ins[i]))
            if i > 0:
                d = OL.conv_transpose(d, Wq[i]) * (ins[i] > 0)
                dabs = OL.conv_transpose(dabs, np.abs(Wq[i])) * (ins[i] > 0)
        g += OL.pack(gl)
        sc += OL.pack(sl)
    return g, sc, Ls


@pytest.mark.parametrize("nodes,B", [(33, 4), (65, 3)])
def test_weight_gradients_match_oracle(M, nodes, B):
    """mg_learned_grad: the training forward layer by layer (as for the
    inference kernel), then every gradient entry against the oracle's
    backward pass on the GPU's activations, within 1e-4 of the entry's
    absolute sum (FP32 partial sums over 128 points, an FP32 operator in
    A y and A e)."""
    prob = pb.diffusion_macro(2, nodes, 22, rhs="normal", rhs_seed=1)
    H = _hier(M, prob)
    theta = OL.init_params(5)
    R = np.stack([pb.normal(40 + k, prob.n) for k in range(B)])
    R /= np.linalg.norm(R, axis=1, keepdims=True)
    E = np.stack([pb.normal(50 + k, prob.n) for k in range(B)])
    R, E = R.astype(np.float32), E.astype(np.float32)
    acts = torch.full((4, B, prob.n, 16), np.nan, dtype=torch.float32, device="cuda")
    Y = torch.zeros((B, prob.n), dtype=torch.float32, device="cuda")
    g_gpu, loss = M.mg_learned_grad(H.h, theta, torch.from_numpy(R).cuda(), torch.from_numpy(E).cuda(), B,
                                    acts_dev=acts, y_dev=Y)
    acts, Yh = acts.cpu().numpy(), Y.cpu().numpy()
    c = _cchan(prob)
    for k in range(B):
        _check_forward(theta, R[k], c, acts[:, k], Yh[k], prob.n1)
    O = omg.Hierarchy(2, prob.n1, prob.stencil, prob.levels)
    g_orc, scale, L_orc = _oracle_grad_on(theta, acts, Yh, R, E, O.A[-1], prob.n1)
    bad = np.abs(g_gpu - g_orc) > 1e-4 * scale + 1e-30
    assert not bad.any(), (int(bad.sum()), np.max(np.abs(g_gpu - g_orc) / (scale + 1e-30)))
    assert abs(loss - L_orc) <= 1e-5 * abs(L_orc)
    # every layer receives a gradient
    for part in np.split(g_gpu, np.cumsum([288, 2304, 2304])):
        assert np.any(part != 0.0)
    # end to end against the oracle's own forward (independent bfloat16
    # roundings): flips move a few entries, so this is a norm check
    _, g_ind = OL.batch_grad(theta, [(R[k].astype(np.float64), E[k].astype(np.float64), O.A[-1], c.reshape(-1))
                                     for k in range(B)], prob.n1)
    assert np.linalg.norm(g_gpu - g_ind) <= 3e-2 * np.linalg.norm(g_ind)


@pytest.mark.parametrize("B,batch", [(4, 4), (3, 4)])
def test_training_step_applies_the_gradient(M, B, batch):
    """With beta1 = 0 and eps >> |g| the first Adam step of mg_learned_train
    is -lr g / (|g| + eps): the step on one batch recovers the gradient that
    mg_learned_grad returns for that batch (FP32 update arithmetic), also for
    a batch shorter than the batch size (fewer weight-gradient partials)."""
    prob = pb.diffusion_macro(2, 33, 22, rhs="normal", rhs_seed=1)
    H = _hier(M, prob)
    theta = OL.init_params(5)
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


@pytest.mark.parametrize("kind", ["poisson", "kappa"])
def test_solver_with_learned_column_matches_oracle(M, kind):
    """Iteration counts within +-2 where MPCG converges in a few steps; on a
    high-contrast field (>200 truncated-MPCG steps) rare bfloat16 rounding
    flips between FP32 (GPU) and FP64 (oracle) accumulation steer the
    iterates apart, so there only convergence and a 10 % band are required."""
    prob = (pb.poisson_random(2, 65, 7) if kind == "poisson"
            else pb.diffusion_macro(2, 33, 23, rhs="normal", rhs_seed=2))
    H = _hier(M, prob)
    theta = OL.init_params(9)
    M.mg_learned_attach(H.h, theta)
    assert M.mg_num_columns(H.h) == prob.levels + 1
    b = torch.from_numpy(prob.b).cuda()
    x = torch.zeros_like(b)
    st, k, rh, ah = H.solve(b, x, rtol=1e-8, maxit=800)
    O = omg.Hierarchy(2, prob.n1, prob.stencil, prob.levels)
    c = _cchan(prob)

    def extra(r):
        nr = np.linalg.norm(r)
        y, _ = OL.forward(theta, (r / nr).reshape(prob.n1, prob.n1), c)
        return nr * y.reshape(-1)
    ref = ompcg.mpcg(O.A[-1], prob.b, O.mg_columns, rtol=1e-8, maxit=800, extra_column=extra)
    assert st == M.MPCG_OK and ref.converged
    if kind == "poisson":
        assert abs(k - ref.iters) <= 2, (k, ref.iters)
    else:
        assert abs(k - ref.iters) <= 0.1 * ref.iters, (k, ref.iters)
    xg = x.cpu().numpy()
    assert np.linalg.norm(prob.b - O.A[-1] @ xg) <= 1.01e-8 * np.linalg.norm(prob.b)
    # the learned column took part (non-zero weights in the first steps)
    assert np.any(np.abs(ah[:5, -1]) > 0)
    M.mg_learned_detach(H.h)
    assert M.mg_num_columns(H.h) == prob.levels


def test_mixed_precision_with_learned_column(M):
    prob = pb.diffusion_macro(2, 65, 24, rhs="normal", rhs_seed=3)
    H = _hier(M, prob, precision=M.MPCG_MIXED)
    M.mg_learned_attach(H.h, OL.init_params(2))
    b = torch.from_numpy(prob.b).cuda()
    x = torch.zeros_like(b)
    st, k, _, _ = H.solve(b, x, rtol=1e-8, maxit=3000)
    O = omg.Hierarchy(2, prob.n1, prob.stencil, prob.levels)
    assert st == M.MPCG_OK
    assert np.linalg.norm(prob.b - O.A[-1] @ x.cpu().numpy()) <= 1e-8 * np.linalg.norm(prob.b)


def _pairs_from_solver(M, prob, ks):
    """(r_k/||r_k||, e_k/||r_k||) for iterates x_k of the GPU FP64 solver."""
    H = _hier(M, prob)
    b = torch.from_numpy(prob.b).cuda()
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
    return H, torch.stack(R), torch.stack(E)


def _heldout_loss(M, H, prob, params, R, E):
    """Mean A-angle loss of the network with weights params on pairs (R, E)."""
    M.mg_learned_attach(H.h, params)
    Y = torch.zeros_like(R)
    M.mg_learned_forward(H.h, R, Y, R.shape[0])
    M.mg_learned_detach(H.h)
    Yd, Ed = Y.double().contiguous(), E.double().contiguous()
    AY, AE = torch.zeros_like(Yd), torch.zeros_like(Ed)
    M.mg_apply_operator(H.h, prob.levels - 1, Yd, AY, Yd.shape[0])
    M.mg_apply_operator(H.h, prob.levels - 1, Ed, AE, Ed.shape[0])
    eay = (Ed * AY).sum(1)
    loss = 1.0 - eay * eay / ((Ed * AE).sum(1) * (Yd * AY).sum(1))
    return float(loss.mean())


def test_training_lowers_loss_on_held_out_fields(M):
    """Training lowers the A-angle loss on its pairs and on pairs of held-out
    coefficient fields (the quantity it optimises), and the trained column
    lowers the iteration count on the two held-out 65^2 problems: measured
    199 -> 197 and 304 -> 264 (8 % fewer in total).  The gain is held to at
    least 4 % in total and no problem may need more than 2 % more steps (the
    training is deterministic, but rounding-level changes of its pairs move
    the gain by a few per cent)."""
    nodes, train_seeds = 65, range(1000, 1006)
    hs, Rs, Es, owner = [], [], [], []
    for i, sd in enumerate(train_seeds):
        prob = pb.diffusion_macro(2, nodes, sd)
        H, R, E = _pairs_from_solver(M, prob, range(1, 121))
        hs.append(H)
        Rs.append(R)
        Es.append(E)
        owner += [i] * R.shape[0]
    R = torch.cat(Rs).contiguous()
    E = torch.cat(Es).contiguous()
    init = OL.init_params(7)
    params = init.copy()
    loss = M.mg_learned_train([h.h for h in hs], owner, R, E, params, epochs=30, batch=8, lr=1e-3)
    assert loss[-1] < loss[0] - 0.02, loss
    gains, held = [], []
    for sd in (3, 5):
        prob = pb.diffusion_macro(2, nodes, sd)
        H, Rh, Eh = _pairs_from_solver(M, prob, range(1, 121, 4))
        before = _heldout_loss(M, H, prob, init, Rh, Eh)
        after = _heldout_loss(M, H, prob, params, Rh, Eh)
        held.append((before, after))
        b = torch.from_numpy(prob.b).cuda()
        x = torch.zeros_like(b)
        _, k_plain, _, _ = H.solve(b, x, rtol=1e-8, maxit=3000)
        M.mg_learned_attach(H.h, params)
        x = torch.zeros_like(b)
        st, k_learned, _, _ = H.solve(b, x, rtol=1e-8, maxit=3000)
        assert st == M.MPCG_OK
        assert k_learned <= 1.02 * k_plain, (k_plain, k_learned)
        gains.append((k_plain, k_learned))
    print("held-out loss (before, after):", held, "iterations (plain, learned):", gains)
    assert sum(k for _, k in gains) <= 0.96 * sum(k for k, _ in gains), gains
    for before, after in held:
        assert after < before - 0.01, held


def test_tensor_core_wait_timeout_is_reported_and_recovers(M):
    """With zero polls for the first bounded wait, every tensor-core kernel
    gives up: the forward pass, the training pass and a solve with the column
    (its graph built before the change) return MPCG_ERR_TIMEOUT after the
    kernels let their MMAs finish and free tensor memory; with the default
    limit back, the same calls give the earlier results bitwise."""
    prob = pb.diffusion_macro(2, 65, 21, rhs="normal", rhs_seed=4)
    H = _hier(M, prob)
    theta = OL.init_params(7)
    M.mg_learned_attach(H.h, theta)
    R = np.stack([pb.normal(3 + k, prob.n) for k in range(2)])
    R = torch.from_numpy((R / np.linalg.norm(R, axis=1, keepdims=True)).astype(np.float32)).cuda()
    E = torch.from_numpy(np.stack([pb.normal(9 + k, prob.n) for k in range(2)]).astype(np.float32)).cuda()
    b = torch.from_numpy(prob.b).cuda()
    Y0 = torch.zeros_like(R)
    M.mg_learned_forward(H.h, R, Y0, 2)
    g0, l0 = M.mg_learned_grad(H.h, theta, R, E, 2)
    x0 = torch.zeros_like(b)
    st0, k0, _, _ = H.solve(b, x0, rtol=1e-8, maxit=800, histories=False)
    try:
        M.mg_set_tensor_wait_limit(0)
        for call in (lambda: M.mg_learned_forward(H.h, R, torch.zeros_like(R), 2),
                     lambda: M.mg_learned_grad(H.h, theta, R, E, 2),
                     lambda: H.solve(b, torch.zeros_like(b), rtol=1e-8, maxit=800, histories=False)):
            with pytest.raises(M.MpcgError) as ei:
                call()
            assert ei.value.status == M.MPCG_ERR_TIMEOUT, ei.value
    finally:
        M.mg_set_tensor_wait_limit(M.MG_TENSOR_WAIT_DEFAULT)
    Y1 = torch.zeros_like(R)
    M.mg_learned_forward(H.h, R, Y1, 2)
    assert torch.equal(Y0, Y1)
    g1, l1 = M.mg_learned_grad(H.h, theta, R, E, 2)
    assert np.array_equal(g0, g1) and abs(l1 - l0) <= 1e-15
    x1 = torch.zeros_like(b)
    st1, k1, _, _ = H.solve(b, x1, rtol=1e-8, maxit=800, histories=False)
    assert st1 == st0 == M.MPCG_OK and k1 == k0 and torch.equal(x0, x1)
    with pytest.raises(M.MpcgError):
        M.mg_set_tensor_wait_limit(-1)
