"""The learned search column on the GPU, against the CPU oracle.

Forward pass and weight gradients are compared with the oracle's
bfloat16-emulating network (tolerance: a few bfloat16 rounding flips, 1-3 %
in norm); the solver with the network attached is compared with the oracle
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


def _cchan(prob):
    centre = 4
    return OL.coefficient_channel(prob.stencil[centre]).reshape(prob.n1, prob.n1)


def test_forward_matches_oracle(M):
    prob = pb.diffusion_macro(2, 65, 21)
    H = _hier(M, prob)
    theta = OL.init_params(7)
    M.mg_learned_attach(H.h, theta)
    R = np.stack([pb.normal(3 + k, prob.n) for k in range(2)])
    R /= np.linalg.norm(R, axis=1, keepdims=True)
    R = R.astype(np.float32)
    Y = torch.zeros((2, prob.n), dtype=torch.float32, device="cuda")
    M.mg_learned_forward(H.h, torch.from_numpy(R).cuda(), Y, 2)
    c = _cchan(prob)
    for k in range(2):
        want, _ = OL.forward(theta, R[k].reshape(prob.n1, prob.n1), c)
        got = Y[k].cpu().numpy().reshape(prob.n1, prob.n1)
        assert np.linalg.norm(got - want) <= 1e-2 * np.linalg.norm(want)


def test_weight_gradients_match_oracle(M):
    """With beta1 = 0 and eps >> |g| the first Adam step is -lr g / eps, so
    one step on one batch exposes the GPU gradient."""
    prob = pb.diffusion_macro(2, 33, 22, rhs="normal", rhs_seed=1)
    H = _hier(M, prob)
    theta = OL.init_params(5)
    B = 4
    R = np.stack([pb.normal(40 + k, prob.n) for k in range(B)])
    R /= np.linalg.norm(R, axis=1, keepdims=True)
    E = np.stack([pb.normal(50 + k, prob.n) for k in range(B)])
    R, E = R.astype(np.float32), E.astype(np.float32)
    params = theta.copy()
    lr = eps = 1e3
    M.mg_learned_train([H.h], [0] * B, torch.from_numpy(R).cuda(), torch.from_numpy(E).cuda(), params, epochs=1,
                       batch=B, lr=lr, beta1=0.0, beta2=0.999, eps=eps)
    g_gpu = -(params.astype(np.float64) - theta.astype(np.float64)) * eps / lr
    O = omg.Hierarchy(2, prob.n1, prob.stencil, prob.levels)
    A = O.A[-1]
    c = _cchan(prob).reshape(-1)
    _, g_orc = OL.batch_grad(theta, [(R[k].astype(np.float64), E[k].astype(np.float64), A, c) for k in range(B)],
                             prob.n1)
    assert np.linalg.norm(g_gpu - g_orc) <= 3e-2 * np.linalg.norm(g_orc)
    for l in range(4):                       # every layer receives its gradient
        a, b = (np.split(g_gpu, np.cumsum([288, 2304, 2304]))[l], np.split(g_orc, np.cumsum([288, 2304, 2304]))[l])
        assert np.linalg.norm(a - b) <= 5e-2 * np.linalg.norm(b)


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
    leaves the solver converging.  The iteration gain itself is reported,
    not asserted: on two held-out 65^2 problems it moves between about -8 %
    and +1 % with rounding-level changes of the training pairs."""
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
        assert k_learned <= 1.1 * k_plain
        gains.append((k_plain, k_learned))
    print("held-out loss (before, after):", held, "iterations (plain, learned):", gains)
    for before, after in held:
        assert after < before - 0.01, held
