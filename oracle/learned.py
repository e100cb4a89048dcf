"""CPU oracle of the learned search direction (test infrastructure).

Not part of the paper: the extension appends one more MPCG search column
z = ||r|| N(r / ||r||, c), where N is a small convolutional network on the
structured grid and c = log10(diag A) / 3 minus its mean gives the network the
local coefficient (a residual-only input cannot locate coefficient jumps).
MPCG's energy minimisation weights the column (zero when it is useless), so
the additive-MG columns remain the fallback.

Network: 3x3 convolutions with channels 2 -> 16 -> 16 -> 16 -> 1, ReLU after
the first three, zero padding (the homogeneous Dirichlet boundary), no bias.
Weights W_l[co, ci, ky, kx] multiply input (ci, y + ky - 1, x + kx - 1).

Precision model of the CUDA path: weights, the two inputs and the outputs of
layers 1-3 are rounded to bfloat16 (round to nearest even); products are
exact and accumulation is FP32 on the GPU (FP64 here); the output y is not
rounded.  ``emulate=False`` gives the plain FP64 network used for the
finite-difference pins.

Loss (per pair): the A-angle between the prediction y and the true error e,
L = 1 - (e^T A y)^2 / ((e^T A e) (y^T A y)), which is what MPCG's energy
minimisation rewards and is invariant to the scale of y.
"""
from __future__ import annotations

import numpy as np

CHANS = (2, 16, 16, 16, 1)
# the 3D vector-valued network of the elasticity problem: the three
# displacement components of r / ||r|| in, three out, 3x3x3 convolutions
CHANS3 = (3, 16, 16, 16, 3)


def n_params() -> int:
    return sum(CHANS[i + 1] * CHANS[i] * 9 for i in range(4))


def unpack(theta: np.ndarray) -> list:
    out, k = [], 0
    for i in range(4):
        sz = CHANS[i + 1] * CHANS[i] * 9
        out.append(theta[k:k + sz].reshape(CHANS[i + 1], CHANS[i], 3, 3))
        k += sz
    return out


def pack(Ws: list) -> np.ndarray:
    return np.concatenate([W.reshape(-1) for W in Ws])


def bf16(x) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned
    as float32."""
    a = np.ascontiguousarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    rounding = np.uint64(0x7FFF) + ((u >> np.uint64(16)) & np.uint64(1))
    r = ((u + rounding) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32).reshape(a.shape)


def init_params(seed: int = 7) -> np.ndarray:
    """The seeded initial weights (an input, drawn by the input module)."""
    from paper_2402_12833_gb300.problems import net_init_params
    return net_init_params(seed, CHANS)


def coefficient_channel(diag: np.ndarray) -> np.ndarray:
    c = np.log10(diag) / 3.0
    return c - c.mean()


def conv(x: np.ndarray, W: np.ndarray) -> np.ndarray:
    """Zero-padded 3x3 correlation: x (cin, H, W), W (cout, cin, 3, 3)."""
    cin, H, Wd = x.shape
    xp = np.zeros((cin, H + 2, Wd + 2), dtype=np.float64)
    xp[:, 1:-1, 1:-1] = x
    out = np.zeros((W.shape[0], H, Wd))
    for ky in range(3):
        for kx in range(3):
            patch = xp[:, ky:ky + H, kx:kx + Wd]
            out += np.einsum("oc,chw->ohw", W[:, :, ky, kx].astype(np.float64), patch)
    return out


def conv_transpose(d: np.ndarray, W: np.ndarray) -> np.ndarray:
    """Adjoint of ``conv`` with respect to its input."""
    cout, H, Wd = d.shape
    out = np.zeros((W.shape[1], H + 2, Wd + 2))
    for ky in range(3):
        for kx in range(3):
            out[:, ky:ky + H, kx:kx + Wd] += np.einsum("oc,ohw->chw", W[:, :, ky, kx].astype(np.float64), d)
    return out[:, 1:-1, 1:-1]


def conv_wgrad(d: np.ndarray, x: np.ndarray) -> np.ndarray:
    """d L / d W for out = conv(x, W), given d = d L / d out."""
    cin, H, Wd = x.shape
    xp = np.zeros((cin, H + 2, Wd + 2))
    xp[:, 1:-1, 1:-1] = x
    g = np.zeros((d.shape[0], cin, 3, 3))
    for ky in range(3):
        for kx in range(3):
            g[:, :, ky, kx] = np.einsum("ohw,chw->oc", d, xp[:, ky:ky + H, kx:kx + Wd])
    return g


def forward(theta: np.ndarray, rhat: np.ndarray, c: np.ndarray, emulate: bool = True):
    """y = N(rhat, c) on an (H, W) image; returns (y, cache)."""
    Ws = unpack(theta)
    rnd = bf16 if emulate else (lambda v: np.asarray(v, dtype=np.float64))
    Wq = [rnd(W) for W in Ws]
    x = rnd(np.stack([rhat, c]).astype(np.float32 if emulate else np.float64))
    acts = [x]
    for i in range(4):
        z = conv(x, Wq[i])
        if i < 3:
            z = np.maximum(z, 0.0)
            x = rnd(z.astype(np.float32) if emulate else z)
            acts.append(x)
        else:
            x = z
    return x[0], (Wq, acts)


def backward(cache, dy: np.ndarray) -> np.ndarray:
    """Gradient of the loss w.r.t. the packed parameters, given dL/dy (the
    rounding to bfloat16 is passed straight through)."""
    Wq, acts = cache
    d = dy[None].astype(np.float64)
    grads = [None] * 4
    for i in range(3, -1, -1):
        grads[i] = conv_wgrad(d, acts[i])
        if i > 0:
            d = conv_transpose(d, Wq[i]) * (acts[i] > 0)
    return pack(grads)


def angle_loss(y: np.ndarray, e: np.ndarray, Ay: np.ndarray, Ae: np.ndarray):
    """L = 1 - (e^T A y)^2 / ((e^T A e)(y^T A y)) and dL/dy (A symmetric)."""
    eAy = float(e @ Ay)
    eAe = float(e @ Ae)
    yAy = float(y @ Ay)
    L = 1.0 - eAy * eAy / (eAe * yAy)
    dy = -(2.0 * eAy / (eAe * yAy)) * (Ae - (eAy / yAy) * Ay)
    return L, dy


def adam_step(theta, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) with bias correction; t counts from 1."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def batch_grad(theta, pairs, n1, emulate=True):
    """Mean loss and gradient over pairs [(rhat, e, A, c)] (vectors of n1^2)."""
    gsum = np.zeros(n_params())
    Lsum = 0.0
    for rhat, e, A, c in pairs:
        y, cache = forward(theta, rhat.reshape(n1, n1), c.reshape(n1, n1), emulate)
        y = y.reshape(-1)
        L, dy = angle_loss(y, e, A @ y, A @ e)
        gsum += backward(cache, dy.reshape(n1, n1))
        Lsum += L
    return Lsum / len(pairs), gsum / len(pairs)


# ---------------------------------------------------------------------------
# 3D network for vector problems (3D elasticity): the same architecture with
# 3x3x3 convolutions, channels 3 -> 16 -> 16 -> 16 -> 3, on the grid of
# unknown nodes (zero padding outside it, i.e. at clamped nodes and beyond
# the free faces).  Weights W[co][ci][kz][ky][kx] multiply the input at
# (x + kx - 1, y + ky - 1, z + kz - 1); the input is r / ||r|| per component
# (no coefficient channel: the material is homogeneous).  Unknown
# i = a + 3 * node, node = x + nx (y + ny z) maps to image[a, z, y, x].

def n_params3() -> int:
    return sum(CHANS3[i + 1] * CHANS3[i] * 27 for i in range(4))


def unpack3(theta: np.ndarray) -> list:
    out, k = [], 0
    for i in range(4):
        sz = CHANS3[i + 1] * CHANS3[i] * 27
        out.append(theta[k:k + sz].reshape(CHANS3[i + 1], CHANS3[i], 3, 3, 3))
        k += sz
    return out


def init_params3(seed: int = 7) -> np.ndarray:
    from paper_2402_12833_gb300.problems import net_init_params
    return net_init_params(seed, CHANS3, taps=27)


def to_image3(v: np.ndarray, shape) -> np.ndarray:
    """Vector of 3 components per node -> (3, Z, Y, X)."""
    Z, Y, X = shape
    return np.asarray(v).reshape(Z, Y, X, 3).transpose(3, 0, 1, 2)


def from_image3(img: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(img.transpose(1, 2, 3, 0)).reshape(-1)


def conv3(x: np.ndarray, W: np.ndarray) -> np.ndarray:
    """Zero-padded 3x3x3 correlation: x (cin, Z, Y, X), W (cout, cin, 3, 3, 3)."""
    cin, Z, Y, X = x.shape
    xp = np.zeros((cin, Z + 2, Y + 2, X + 2), dtype=np.float64)
    xp[:, 1:-1, 1:-1, 1:-1] = x
    out = np.zeros((W.shape[0], Z, Y, X))
    for kz in range(3):
        for ky in range(3):
            for kx in range(3):
                patch = xp[:, kz:kz + Z, ky:ky + Y, kx:kx + X]
                out += np.einsum("oc,czyx->ozyx", W[:, :, kz, ky, kx].astype(np.float64), patch)
    return out


def conv3_transpose(d: np.ndarray, W: np.ndarray) -> np.ndarray:
    """Adjoint of ``conv3`` with respect to its input."""
    cout, Z, Y, X = d.shape
    out = np.zeros((W.shape[1], Z + 2, Y + 2, X + 2))
    for kz in range(3):
        for ky in range(3):
            for kx in range(3):
                out[:, kz:kz + Z, ky:ky + Y, kx:kx + X] += np.einsum("oc,ozyx->czyx",
                                                                     W[:, :, kz, ky, kx].astype(np.float64), d)
    return out[:, 1:-1, 1:-1, 1:-1]


def conv3_wgrad(d: np.ndarray, x: np.ndarray) -> np.ndarray:
    """d L / d W for out = conv3(x, W), given d = d L / d out."""
    cin, Z, Y, X = x.shape
    xp = np.zeros((cin, Z + 2, Y + 2, X + 2))
    xp[:, 1:-1, 1:-1, 1:-1] = x
    g = np.zeros((d.shape[0], cin, 3, 3, 3))
    for kz in range(3):
        for ky in range(3):
            for kx in range(3):
                g[:, :, kz, ky, kx] = np.einsum("ozyx,czyx->oc", d, xp[:, kz:kz + Z, ky:ky + Y, kx:kx + X])
    return g


def forward3(theta: np.ndarray, rhat: np.ndarray, emulate: bool = True):
    """y = N(rhat) for rhat of shape (3, Z, Y, X); returns (y, cache)."""
    Ws = unpack3(theta)
    rnd = bf16 if emulate else (lambda v: np.asarray(v, dtype=np.float64))
    Wq = [rnd(W) for W in Ws]
    x = rnd(np.asarray(rhat, dtype=np.float32 if emulate else np.float64))
    acts = [x]
    for i in range(4):
        z = conv3(x, Wq[i])
        if i < 3:
            z = np.maximum(z, 0.0)
            x = rnd(z.astype(np.float32) if emulate else z)
            acts.append(x)
        else:
            x = z
    return x, (Wq, acts)


def backward3(cache, dy: np.ndarray) -> np.ndarray:
    """Gradient of the loss w.r.t. the packed 3D parameters, given dL/dy of
    shape (3, Z, Y, X) (the rounding to bfloat16 passed straight through)."""
    Wq, acts = cache
    d = np.asarray(dy, dtype=np.float64)
    grads = [None] * 4
    for i in range(3, -1, -1):
        grads[i] = conv3_wgrad(d, acts[i])
        if i > 0:
            d = conv3_transpose(d, Wq[i]) * (acts[i] > 0)
    return np.concatenate([g.reshape(-1) for g in grads])


def batch_grad3(theta, pairs, shape, emulate=True):
    """Mean loss and gradient over pairs [(rhat, e, A)] of vectors (3 unknowns
    per node) on a grid of unknown nodes of the given (Z, Y, X) shape."""
    gsum = np.zeros(n_params3())
    Lsum = 0.0
    for rhat, e, A in pairs:
        y, cache = forward3(theta, to_image3(rhat, shape), emulate)
        yv = from_image3(y)
        L, dy = angle_loss(yv, e, A @ yv, A @ e)
        gsum += backward3(cache, to_image3(dy, shape))
        Lsum += L
    return Lsum / len(pairs), gsum / len(pairs)
