"""5-point finite-difference operators on the unit square, zero Dirichlet boundary.

Two discretisations:

* `stencil_div` -- the divergence form -div(k grad u) + b . grad u = f of
  Remark 2.1 (Eq. convection_diffusion_div), with the face coefficient the
  harmonic mean of the two nodal k and first-order upwind convection.
* `stencil_nondiv` -- the paper's non-divergence form -mu Lap u + v . grad u = f
  (Sec. 2.5, Eqs. convection_diffusion and convection_diffusion_kernel): the
  5-point Laplacian scaled by mu at the node plus the upwind kernel
  v_x^+ dx^- + v_x^- dx^+, v_y^+ dy^- + v_y^- dy^+.

Both produce the five coefficient arrays (a_C, a_W, a_E, a_S, a_N) on the n x n
interior nodes with (A u)_p = sum_o a_o(p) u(p + o), neighbours outside the
interior contributing 0 (zero padding, Sec. 2.5).  W/E are i -+ 1, S/N are j -+ 1.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .grid import spacing


@dataclass
class Stencil:
    aC: np.ndarray
    aW: np.ndarray
    aE: np.ndarray
    aS: np.ndarray
    aN: np.ndarray

    @property
    def n(self) -> int:
        return self.aC.shape[0]


def harmonic_mean(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Face coefficient between two nodes: 2 a b / (a + b)."""
    return 2.0 * a * b / (a + b)


def stencil_div(k: np.ndarray, b: tuple[float, float]) -> Stencil:
    """Divergence-form operator from nodal k on the (n+2)^2 nodes incl. the boundary ring.

    a_W = -k_{i-1/2,j}/h^2 - max(b_x,0)/h     a_E = -k_{i+1/2,j}/h^2 + min(b_x,0)/h
    a_S = -k_{i,j-1/2}/h^2 - max(b_y,0)/h     a_N = -k_{i,j+1/2}/h^2 + min(b_y,0)/h
    a_C = (sum of the four face k)/h^2 + (|b_x| + |b_y|)/h
    """
    n = k.shape[0] - 2
    h = spacing(n)
    bx, by = float(b[0]), float(b[1])
    kc = k[1:-1, 1:-1]
    kw = harmonic_mean(kc, k[1:-1, :-2])
    ke = harmonic_mean(kc, k[1:-1, 2:])
    ks = harmonic_mean(kc, k[:-2, 1:-1])
    kn = harmonic_mean(kc, k[2:, 1:-1])
    ih2 = 1.0 / (h * h)
    aW = -kw * ih2 - max(bx, 0.0) / h
    aE = -ke * ih2 + min(bx, 0.0) / h
    aS = -ks * ih2 - max(by, 0.0) / h
    aN = -kn * ih2 + min(by, 0.0) / h
    aC = (kw + ke + ks + kn) * ih2 + (abs(bx) + abs(by)) / h
    return Stencil(aC, aW, aE, aS, aN)


def stencil_nondiv(mu: np.ndarray, v: tuple[float, float]) -> Stencil:
    """Non-divergence operator from nodal mu on the n x n interior nodes (Sec. 2.5).

    (1/h){ (mu/h) [0 -1 0; -1 4 -1; 0 -1 0] + v . K_upwind } written per node:
    the Laplacian part gives -mu/h^2 on each neighbour and 4 mu/h^2 on the
    centre; dx^- = u_i - u_{i-1} weighted by v_x^+, dx^+ = u_{i+1} - u_i by v_x^-,
    and likewise in y.
    """
    n = mu.shape[0]
    h = spacing(n)
    vx, vy = float(v[0]), float(v[1])
    lap = mu / (h * h)
    aW = -lap - max(vx, 0.0) / h
    aE = -lap + min(vx, 0.0) / h
    aS = -lap - max(vy, 0.0) / h
    aN = -lap + min(vy, 0.0) / h
    aC = 4.0 * lap + (max(vx, 0.0) - min(vx, 0.0) + max(vy, 0.0) - min(vy, 0.0)) / h
    return Stencil(aC, aW, aE, aS, aN)


def inject_k(k: np.ndarray) -> np.ndarray:
    """Coarse nodal k by injection: coarse node I is fine node 2I (boundary ring included)."""
    return np.ascontiguousarray(k[::2, ::2])


def restrict_k(k: np.ndarray, mean: str = "log") -> np.ndarray:
    """Coarse nodal k for the divergence form: full weighting around fine node 2I.

    mean="log" (default): log k_c(I, J) = sum_ab w_a w_b log k(2J + a - 1, 2I + b - 1)
    / sum of the weights used; mean="arith": k_c = sum_ab w_a w_b k(...) / sum of
    the weights used; w = (1, 2, 1), over the fine nodes that exist (the boundary
    ring renormalises).
    Reading: Sec. 2.3 rediscretises the PDE on the coarse grid without saying how a
    heterogeneous k gets there, and the setup phase restricts coefficients with a
    strided 3x3 convolution (Eq. setup1).  The geometric average keeps
    rediscretised GMG convergent on smooth lognormal k; the arithmetic average
    (never below the geometric one) gives stiffer coarse operators, which keep the
    coarse-grid correction from over-correcting on piecewise-constant
    high-contrast k, where the geometric one makes GMG diverge.
    """
    if mean not in ("log", "arith"):
        raise ValueError(mean)
    m = k.shape[0]
    mc = (m + 1) // 2
    g = np.pad(np.log(k) if mean == "log" else k, 1)
    mask = np.pad(np.ones_like(k), 1)
    w = np.array([1.0, 2.0, 1.0])
    num = np.zeros((mc, mc))
    den = np.zeros((mc, mc))
    for a in range(3):
        for b in range(3):
            num += w[a] * w[b] * g[a:a + 2 * mc - 1:2, b:b + 2 * mc - 1:2]
            den += w[a] * w[b] * mask[a:a + 2 * mc - 1:2, b:b + 2 * mc - 1:2]
    return np.exp(num / den) if mean == "log" else num / den


def inject_mu(mu: np.ndarray) -> np.ndarray:
    """Coarse interior mu by injection: coarse interior node J (1-based) is fine node 2J."""
    return np.ascontiguousarray(mu[1::2, 1::2])


def level_stencils_div(k: np.ndarray, b, levels: int, mean: str = "log") -> list[Stencil]:
    """Rediscretised operators on every level (Sec. 2.3: coarse operators by discretising
    the PDE on the coarse grid), with k carried to the coarse grid by `restrict_k`
    (`mean`: its averaging, geometric or arithmetic)."""
    out = []
    kl = k
    for _ in range(levels):
        out.append(stencil_div(kl, b))
        kl = restrict_k(kl, mean)
    return out


def level_stencils_nondiv(mu: np.ndarray, v, levels: int) -> list[Stencil]:
    """Rediscretised non-divergence operators, mu injected (the operator at a node
    depends on mu there only, so sampling the coefficient is the rediscretisation)."""
    out = []
    ml = mu
    for _ in range(levels):
        out.append(stencil_nondiv(ml, v))
        ml = inject_mu(ml)
    return out


def apply(st: Stencil, u: np.ndarray) -> np.ndarray:
    """(A u)_p = a_C u_p + a_W u_W + a_E u_E + a_S u_S + a_N u_N with zero padding."""
    up = np.pad(u, 1)
    return (st.aC * u + st.aW * up[1:-1, :-2] + st.aE * up[1:-1, 2:]
            + st.aS * up[:-2, 1:-1] + st.aN * up[2:, 1:-1])


def apply_transpose(st: Stencil, v: np.ndarray) -> np.ndarray:
    """(A^T v)_q = sum_p A[p, q] v_p: the W coefficient of node q+(0,1) multiplies v there, etc."""
    n = st.n
    out = st.aC * v
    out[:, :-1] += st.aW[:, 1:] * v[:, 1:]      # p = q + e_x sees q as its W neighbour
    out[:, 1:] += st.aE[:, :-1] * v[:, :-1]     # p = q - e_x sees q as its E neighbour
    out[:-1, :] += st.aS[1:, :] * v[1:, :]      # p = q + e_y sees q as its S neighbour
    out[1:, :] += st.aN[:-1, :] * v[:-1, :]     # p = q - e_y sees q as its N neighbour
    assert out.shape == (n, n)
    return out


def residual(st: Stencil, f: np.ndarray, u: np.ndarray) -> np.ndarray:
    """r = f - A u (Eq. stationary_iteration)."""
    return f - apply(st, u)


def dense_matrix(st: Stencil) -> np.ndarray:
    """Assemble A as an n^2 x n^2 matrix, row p = j*n + i, by applying it to unit vectors."""
    n = st.n
    N = n * n
    M = np.zeros((N, N))
    e = np.zeros((n, n))
    for q in range(N):
        e.flat[q] = 1.0
        M[:, q] = apply(st, e).ravel()
        e.flat[q] = 0.0
    return M
