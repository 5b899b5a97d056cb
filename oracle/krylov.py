"""MGCNN as a preconditioner of flexible GMRES (the use of the network inside a
Krylov method, Sec. 2.2: the network approximates A^{-1}, and beyond the
stationary iteration of Eq. 1 it can precondition an outer Krylov solver).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Right-preconditioned flexible GMRES(m): the preconditioner may change from one
application to the next (the mixed-precision network rounds differently for
every input), so the preconditioned directions z_j = M(v_j) are kept and the
update is u += Z y.  Arnoldi with classical Gram-Schmidt applied twice (each
pass projects the new vector against all basis vectors with the coefficients
of that pass), Givens rotations for the least-squares problem, convergence
test ||r|| / ||f|| <= tol on the recursive residual estimate, restarts from the
true residual f - A u.  Written from the textbook definition of the method
(Arnoldi relation A Z_m = V_{m+1} H_m, y = argmin ||beta e_1 - H_m y||).
"""
from __future__ import annotations

from typing import Callable

import numpy as np


def fgmres(apply_A: Callable[[np.ndarray], np.ndarray], precond: Callable[[np.ndarray], np.ndarray],
           f: np.ndarray, u0: np.ndarray | None, tol: float, maxit: int, restart: int):
    """Solve A u = f.  apply_A, precond: maps of arrays of f's shape.

    maxit counts preconditioner applications (inner iterations) over all restarts.
    Returns (u, iters, history) with history[k] = the residual-norm ratio after k
    inner iterations (history[0] = ||f - A u0|| / ||f||): the recursive estimate
    inside a cycle, the TRUE residual after a cycle's last iteration."""
    u = np.zeros_like(f) if u0 is None else u0.astype(np.float64).copy()
    fn = np.linalg.norm(f)
    if fn == 0.0:
        return np.zeros_like(f), 0, [0.0]
    r = f - apply_A(u)
    beta = np.linalg.norm(r)
    hist = [beta / fn]
    it = 0
    while hist[-1] > tol and it < maxit:
        m = min(restart, maxit - it)
        V = [r / beta]
        Z = []
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        k = 0
        for j in range(m):
            z = precond(V[j])
            w = apply_A(z)
            for _ in range(2):                       # classical Gram-Schmidt, twice
                c = np.array([np.vdot(v, w) for v in V])
                for i, v in enumerate(V):
                    w = w - c[i] * v
                H[: j + 1, j] += c
            hn = np.linalg.norm(w)
            H[j + 1, j] = hn
            Z.append(z)
            # apply the previous rotations to column j, then a new one
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            d = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / d, H[j + 1, j] / d
            H[j, j], H[j + 1, j] = d, 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            it += 1
            est = abs(g[j + 1]) / fn
            if est <= tol or it >= maxit or not np.isfinite(est) or j == m - 1:
                break                                # the cycle's last entry is the true residual
            hist.append(est)
            V.append(w / hn)
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):               # back substitution on the rotated H
            y[i] = (g[i] - np.dot(H[i, i + 1:k], y[i + 1:k])) / H[i, i]
        for i in range(k):
            u = u + y[i] * Z[i]
        r = f - apply_A(u)
        beta = np.linalg.norm(r)
        hist.append(beta / fn)
        if not np.isfinite(beta):
            break
    return u, it, hist
