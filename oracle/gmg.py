"""Classical geometric multigrid (Sec. 2.3; Algorithm 1 applied recursively as a V-cycle).

Settings of Sec. 2.3: halving coarsening, coarse operators by rediscretising the
PDE on the coarse grid (`operator.level_stencils_*`), bilinear transfers and
weighted-Jacobi smoothing.  Restriction is full weighting (1/16)[1 2 1; 2 4 2;
1 2 1] applied as an unpadded stride-2 stencil (coarse node I on fine node
2I + 1, 0-based), prolongation is bilinear interpolation, the transpose stencil
(1/4)[1 2 1; 2 4 2; 1 2 1].  The coarsest (3x3) grid is not solved directly:
it gets nu1 + nu2 Jacobi sweeps (reading; the paper does not say).

The V-cycle acts on the residual equation A e = r from e = 0 and returns e; the
outer loop is the stationary iteration u <- u + V(f - A u) (Eq. 1).
"""
from __future__ import annotations

import numpy as np

from .operator import Stencil, apply

FW = np.array([[1.0, 2.0, 1.0], [2.0, 4.0, 2.0], [1.0, 2.0, 1.0]]) / 16.0
BILINEAR = np.array([[1.0, 2.0, 1.0], [2.0, 4.0, 2.0], [1.0, 2.0, 1.0]]) / 4.0


def jacobi_sweep(st: Stencil, e: np.ndarray, r: np.ndarray, omega: float) -> np.ndarray:
    """e <- e + omega D^{-1} (r - A e)."""
    return e + omega * (r - apply(st, e)) / st.aC


def restrict_fw(d: np.ndarray) -> np.ndarray:
    """r_c[J, I] = sum_ab FW[a, b] d[2J + a, 2I + b] (0-based interior indices)."""
    n = d.shape[0]
    nc = (n - 1) // 2
    rc = np.zeros((nc, nc))
    for a in range(3):
        for b in range(3):
            rc += FW[a, b] * d[a:a + 2 * nc - 1:2, b:b + 2 * nc - 1:2]
    return rc


def prolong_bilinear(ec: np.ndarray, n_fine: int) -> np.ndarray:
    """e[2J + a, 2I + b] += BILINEAR[a, b] e_c[J, I]."""
    nc = ec.shape[0]
    assert n_fine == 2 * nc + 1
    e = np.zeros((n_fine, n_fine))
    for a in range(3):
        for b in range(3):
            e[a:a + 2 * nc - 1:2, b:b + 2 * nc - 1:2] += BILINEAR[a, b] * ec
    return e


def level_omegas(levels: int, omega) -> list[float]:
    """Jacobi weight of every level, finest first.

    `omega` is one weight for every level, or three weights (w_fine, w_mid,
    w_coarsest): w_fine on the finest level, w_coarsest on the coarsest, w_mid
    on every level in between; a one-level hierarchy takes w_fine.  Reading:
    Sec. 2.3 smooths with weighted Jacobi and fixes no weight, so the weight
    may be chosen per level like any other smoother parameter.
    """
    if np.ndim(omega) == 0:
        return [float(omega)] * levels
    w_fine, w_mid, w_coarsest = (float(x) for x in omega)
    if levels == 1:
        return [w_fine]
    return [w_fine] + [w_mid] * (levels - 2) + [w_coarsest]


def _omega_at(omega, level: int) -> float:
    """omega: one weight, or a list with one weight per level."""
    return float(omega) if np.ndim(omega) == 0 else float(omega[level])


def vcycle(stencils: list[Stencil], r: np.ndarray, nu1: int, nu2: int, omega,
           level: int = 0) -> np.ndarray:
    """One V(nu1, nu2) cycle for A_level e = r from e = 0; returns e.

    omega: one Jacobi weight, or a list with one weight per level (finest first)."""
    st = stencils[level]
    om = _omega_at(omega, level)
    e = np.zeros_like(r)
    if level == len(stencils) - 1:
        for _ in range(nu1 + nu2):
            e = jacobi_sweep(st, e, r, om)
        return e
    for _ in range(nu1):
        e = jacobi_sweep(st, e, r, om)
    d = r - apply(st, e)
    ec = vcycle(stencils, restrict_fw(d), nu1, nu2, omega, level + 1)
    e = e + prolong_bilinear(ec, r.shape[0])
    for _ in range(nu2):
        e = jacobi_sweep(st, e, r, om)
    return e


def stationary_solve(stencils: list[Stencil], f: np.ndarray, u0: np.ndarray | None, tol: float,
                     maxit: int, nu1: int = 2, nu2: int = 2, omega=0.8):
    """u^{k+1} = u^k + V(f - A u^k) until ||r||_2/||f||_2 <= tol (checked before each cycle).

    omega: one Jacobi weight, or a list with one weight per level (`level_omegas`).

    Returns (u, iters, relres_history, iterates) with iterates[k] = u^k.
    """
    A = stencils[0]
    u = np.zeros_like(f) if u0 is None else u0.copy()
    fn = np.linalg.norm(f)
    hist, iterates = [], [u.copy()]
    if fn == 0.0:
        return np.zeros_like(f), 0, [0.0], [np.zeros_like(f)]
    for k in range(maxit + 1):
        r = f - apply(A, u)
        rel = np.linalg.norm(r) / fn
        hist.append(rel)
        if rel <= tol or k == maxit:
            return u, k, hist, iterates
        u = u + vcycle(stencils, r, nu1, nu2, omega)
        iterates.append(u.copy())
    raise AssertionError("unreachable")
