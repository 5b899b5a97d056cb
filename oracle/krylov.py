"""MGCNN as a preconditioner of Krylov methods (the use of the network inside a
Krylov method, Sec. 2.2: the network approximates A^{-1}, and beyond the
stationary iteration of Eq. 1 it can precondition an outer Krylov solver; for
a symmetric problem and the symmetric network, Remark "Symmetric problem"
names MINRES).

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


def pcg(apply_A: Callable[[np.ndarray], np.ndarray], precond: Callable[[np.ndarray], np.ndarray],
        f: np.ndarray, u0: np.ndarray | None, tol: float, maxit: int):
    """Preconditioned conjugate gradients for SPD A and SPD preconditioner M
    (textbook form: z = M r, p = z + beta p, alpha = (r, z) / (p, A p),
    beta = (r_new, z_new) / (r, z)).  Stops when ||r_k|| / ||f|| <= tol on the
    recursively updated residual, or after maxit iterations (one preconditioner
    application each).  Returns (u, iters, history) with history[k] =
    ||r_k|| / ||f|| (history[0] from the true residual f - A u0)."""
    u = np.zeros_like(f) if u0 is None else u0.astype(np.float64).copy()
    fn = np.linalg.norm(f)
    if fn == 0.0:
        return np.zeros_like(f), 0, [0.0]
    r = f - apply_A(u)
    hist = [np.linalg.norm(r) / fn]
    it = 0
    p = None
    rz = 0.0
    while hist[-1] > tol and it < maxit and np.isfinite(hist[-1]):
        z = precond(r)
        rz_new = np.vdot(r, z)
        p = z if p is None else z + (rz_new / rz) * p
        rz = rz_new
        q = apply_A(p)
        alpha = rz / np.vdot(p, q)
        u = u + alpha * p
        r = r - alpha * q
        it += 1
        hist.append(np.linalg.norm(r) / fn)
    return u, it, hist


def minres(apply_A: Callable[[np.ndarray], np.ndarray], precond: Callable[[np.ndarray], np.ndarray],
           f: np.ndarray, u0: np.ndarray | None, tol: float, maxit: int):
    """Preconditioned MINRES for symmetric A and SPD preconditioner M.

    Lanczos on (M A) in the M^{-1} inner product, with the three-term vectors
    kept in both forms (r_k unpreconditioned, y_k = M r_k, beta_k = sqrt((r_k, y_k))),
    the tridiagonal least-squares problem solved by Givens rotations as columns
    arrive, and the iterate updated through the search directions
    w_k = (v_k - eps_k w_{k-2} - delta_k w_{k-1}) / gamma_k.  Iterate k minimises
    ||f - A u||_M over u0 + K_k(M A, M r0) (M-norm: sqrt(r^T M r)).  Stops when
    that norm, relative to its value at u0, is <= tol, or after maxit iterations.
    Returns (u, iters, history) with history[k] = ||r_k||_M / ||r_0||_M from the
    recursion (history[0] = 1)."""
    u = np.zeros_like(f) if u0 is None else u0.astype(np.float64).copy()
    r = f - apply_A(u)
    y = precond(r)
    beta1 = np.sqrt(np.vdot(r, y))
    if beta1 == 0.0:
        return u, 0, [0.0]
    hist = [1.0]
    # Lanczos state: r_prev = r_{k-1}, r_cur = r_k (unpreconditioned), y = M r_k
    r_prev, r_cur = np.zeros_like(f), r
    beta_prev, beta = 0.0, beta1
    # rotation state
    cs, sn = -1.0, 0.0
    dbar, eps = 0.0, 0.0
    phibar = beta1
    w_prev2, w_prev = np.zeros_like(f), np.zeros_like(f)
    it = 0
    while it < maxit:
        v = y / beta                                   # Lanczos vector (M-orthonormal basis of K)
        t = apply_A(v)
        if it > 0:
            t = t - (beta / beta_prev) * r_prev
        alpha = np.vdot(v, t)
        t = t - (alpha / beta) * r_cur
        r_prev, r_cur = r_cur, t
        y = precond(r_cur)
        beta_prev, beta = beta, np.sqrt(np.vdot(r_cur, y))
        # previous rotation on the new column (eps, delta from the last two rotations)
        eps_old = eps
        delta = cs * dbar + sn * alpha
        gbar = sn * dbar - cs * alpha
        eps = sn * beta
        dbar = -cs * beta
        gamma = np.hypot(gbar, beta)
        cs, sn = gbar / gamma, beta / gamma
        phi = cs * phibar
        phibar = sn * phibar
        w = (v - eps_old * w_prev2 - delta * w_prev) / gamma
        w_prev2, w_prev = w_prev, w
        u = u + phi * w
        it += 1
        hist.append(abs(phibar) / beta1)
        if hist[-1] <= tol or not np.isfinite(hist[-1]) or beta == 0.0:
            break
    return u, it, hist
