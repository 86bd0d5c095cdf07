"""Preconditioned conjugate gradients (oracle, test-only).

Textbook PCG for the SPD system A x = b of Sec. 2.3, starting from x_1 = 0,
with the residual r_i = b - A x_i updated recursively.  Stops when
||r||_2 / ||b||_2 <= tol.  The error-tracking benchmark method of Sec. 2.3
(b = A x_true, track ||x_i - x_true||) is available through ``x_true``.

Parity: pinned (tests/test_oracle_cg.py) against a dense Cholesky solve and
the closed-form Wiener filter.
"""
import numpy as np


def pcg(apply_A, b, apply_M=None, tol=1e-8, maxiter=1000, x_true=None):
    b = np.asarray(b, dtype=np.float64)
    if apply_M is None:
        apply_M = lambda v: v
    x = np.zeros_like(b)
    r = b.copy()
    z = apply_M(r)
    p = z.copy()
    rz = float(r @ z)
    bnorm = float(np.linalg.norm(b))
    hist, errs = [], []
    it = 0
    while it < maxiter:
        q = apply_A(p)
        alpha = rz / float(p @ q)
        x += alpha * p
        r -= alpha * q
        it += 1
        rel = float(np.linalg.norm(r)) / bnorm
        hist.append(rel)
        if x_true is not None:
            errs.append(float(np.linalg.norm(x - x_true)))
        if rel <= tol:
            break
        z = apply_M(r)
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, {"iters": it, "rel_res": hist, "err": errs}
