"""Textbook preconditioned CG (Hestenes-Stiefel recurrence), FP64.

Used only as an independent pin: with the additive MG preconditioner B of
Eq. 3 this is the additive MG-PCG method the paper compares against
(Section 2.1 and Section 3.1); MPCG given the single summed column B r must
reproduce its iterates.
"""
from __future__ import annotations

import numpy as np


def pcg(A, b, precond, x0=None, rtol=1e-8, maxit=500):
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - A @ x
    nb = np.linalg.norm(b)
    res = [np.linalg.norm(r) / nb]
    if res[0] <= rtol:
        return x, 0, res
    z = precond(r)
    p = z.copy()
    rz = r @ z
    k = 0
    while True:
        Ap = A @ p
        a = rz / (p @ Ap)
        x += a * p
        r -= a * Ap
        k += 1
        res.append(np.linalg.norm(r) / nb)
        if res[-1] <= rtol or k >= maxit:
            break
        z = precond(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, k, res
