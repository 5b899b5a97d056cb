"""Pins for the oracle's classical GMG (Sec. 2.3) and its outer stationary loop (Eq. 1)."""
import os

import numpy as np
import pytest

from oracle import gmg
from oracle import operator as op
from oracle.grid import num_levels
from paper_2312_11093_gb300 import inputs


def cfg0_problem():
    """31x31, h = 1/32, 8x8 board of 4x4-cell blocks with log10 k ~ U(-1, 1),
    b = (1, 0.5), f ~ N(0, 1), seed 0 (block draws first, then f)."""
    n = 31
    rng = np.random.default_rng(0)
    k = inputs.block_board_k(n, rng)
    f = inputs.normal_rhs(n, rng)
    return n, k, (1.0, 0.5), f


def test_transfer_transpose_relation():
    """Full weighting is a quarter of the transpose of bilinear prolongation."""
    rng = np.random.default_rng(5)
    d = rng.standard_normal((15, 15))
    c = rng.standard_normal((7, 7))
    lhs = np.sum(gmg.restrict_fw(d) * c)
    rhs = 0.25 * np.sum(d * gmg.prolong_bilinear(c, 15))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_transfers_on_polynomials():
    """FW keeps a linear field (away from the boundary); bilinear prolongation
    reproduces a linear field at fine nodes whose coarse neighbours are interior."""
    n, nc = 31, 15
    h, hc = 1.0 / (n + 1), 1.0 / (nc + 1)
    x = np.arange(1, n + 1) * h
    X, Y = np.meshgrid(x, x)
    lin = 0.3 + 2 * X - 1.5 * Y
    xc = np.arange(1, nc + 1) * hc
    Xc, Yc = np.meshgrid(xc, xc)
    np.testing.assert_allclose(gmg.restrict_fw(lin), 0.3 + 2 * Xc - 1.5 * Yc, rtol=1e-13)
    e = gmg.prolong_bilinear(0.3 + 2 * Xc - 1.5 * Yc, n)
    np.testing.assert_allclose(e[1:-1, 1:-1], lin[1:-1, 1:-1], rtol=1e-13)


def test_poisson_vcycle_convergence_factor():
    """Constant k, b = 0, V(2,2), omega = 0.8.  The coarsest 3x3 grid is smoothed, not
    solved, so the asymptotic factor is set by its smoothest mode: Jacobi damps it by
    1 - omega * 2 sin^2(pi h_c / 2) per sweep with h_c = 1/4, over 4 sweeps
    (the finer levels contract much faster).  Observed factor within 10% of that."""
    n = 63
    sts = op.level_stencils_div(np.ones((n + 2, n + 2)), (0.0, 0.0), num_levels(n))
    f = np.random.default_rng(1).standard_normal((n, n))
    _, it, hist, _ = gmg.stationary_solve(sts, f, None, 1e-10, 60)
    rate = (hist[-1] / hist[-4]) ** (1 / 3)
    coarse = (1 - 0.8 * 2 * np.sin(np.pi / 8) ** 2) ** 4
    assert abs(rate - coarse) < 0.1 * coarse, (rate, coarse)
    assert it < 30


def test_cfg0_gmg_matches_direct_solve():
    n, k, b, f = cfg0_problem()
    sts = op.level_stencils_div(k, b, num_levels(n))
    u, it, hist, _ = gmg.stationary_solve(sts, f, None, 1e-10, 200)
    assert hist[-1] <= 1e-10 and it < 200
    ustar = np.linalg.solve(op.dense_matrix(sts[0]), f.ravel()).reshape(n, n)
    assert np.linalg.norm(u - ustar) / np.linalg.norm(ustar) < 1e-7


def test_zero_rhs_and_maxit():
    n, k, b, f = cfg0_problem()
    sts = op.level_stencils_div(k, b, num_levels(n))
    u, it, hist, _ = gmg.stationary_solve(sts, np.zeros_like(f), None, 1e-10, 5)
    assert it == 0 and not u.any()
    _, it, hist, _ = gmg.stationary_solve(sts, f, None, 1e-30, 3)
    assert it == 3 and len(hist) == 4


def test_symmetric_vcycle_for_a_symmetric_operator():
    """With b = 0 (A symmetric), Jacobi smoothing and full weighting = 1/4 x the
    bilinear transpose, the V(nu, nu) cycle is a symmetric operator (pre- and
    post-smoothing are adjoint, the coarsest-grid sweeps are a symmetric
    polynomial in D^-1 A times D^-1); V(2, 1) is not."""
    n = 15
    rng = np.random.default_rng(8)
    k = inputs.lognormal_k(n, 0.1, rng)
    sts = op.level_stencils_div(k, (0.0, 0.0), num_levels(n))

    def dense(nu1, nu2):
        B = np.zeros((n * n, n * n))
        for c in range(n * n):
            e = np.zeros(n * n)
            e[c] = 1.0
            B[:, c] = gmg.vcycle(sts, e.reshape(n, n), nu1, nu2, 0.8).ravel()
        return B
    for nu in (1, 2):
        B = dense(nu, nu)
        assert np.abs(B - B.T).max() <= 1e-13 * np.abs(B).max()
    B = dense(2, 1)
    assert np.abs(B - B.T).max() > 1e-3 * np.abs(B).max()


def _paper_gmg_iterations():
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_gmg_iterations.txt")
    out = {}
    for line in open(path):
        line = line.split("#")[0].strip()
        if line:
            n, v = line.split(":")
            out[int(n)] = float(v)
    return out


@pytest.mark.parametrize("n", [31, 63, 127, 255, 511, 1023])
def test_paper_gmg_iteration_counts(n):
    """The paper's GMG column (Table channels_double) on its own test problem: the
    oracle's non-divergence operator (coef = mu / h, Sec. 2.5) with white-noise
    coef in [1e-3, 1], v = (sin 0.5, cos 0.5), f = 1, and GMG with the paper's
    settings (weight 0.67, three pre- and three post-sweeps, level = log2(n+1) - 3,
    the coarsest grid smoothed) needs within 15% of the printed mean iteration
    count to 1e-8 (mean over three draws here up to 255^2 and one draw beyond,
    ten there)."""
    paper = _paper_gmg_iterations()[n]
    v = (np.sin(0.5), np.cos(0.5))
    its = []
    for rep in range(3 if n <= 255 else 1):
        rng = np.random.default_rng(100 * n + rep)
        mu = inputs.paper_white_noise_mu(n, rng)
        sts = op.level_stencils_nondiv(mu, v, num_levels(n) - 2)
        _, it, hist, _ = gmg.stationary_solve(sts, inputs.unit_rhs(n), None, 1e-8, 300, 3, 3, 0.67)
        assert hist[-1] <= 1e-8
        its.append(it)
    assert abs(np.mean(its) - paper) <= 0.15 * paper, (its, paper)


def test_level_omegas_rule():
    """One weight for every level, or (finest, in between, coarsest)."""
    assert gmg.level_omegas(3, 0.8) == [0.8, 0.8, 0.8]
    assert gmg.level_omegas(1, (0.7, 1.3, 1.1)) == [0.7]
    assert gmg.level_omegas(2, (0.7, 1.3, 1.1)) == [0.7, 1.1]
    assert gmg.level_omegas(5, (0.7, 1.3, 1.1)) == [0.7, 1.3, 1.3, 1.3, 1.1]


def _dense_fw(n: int) -> np.ndarray:
    """Full weighting as a dense (nc^2 x n^2) matrix: coarse node (J, I) takes
    fine nodes (2J + a, 2I + b), a, b in {0, 1, 2}, with weights (1 2 1)(1 2 1)^T / 16."""
    nc = (n - 1) // 2
    w = np.array([1.0, 2.0, 1.0])
    R = np.zeros((nc * nc, n * n))
    for J in range(nc):
        for I in range(nc):
            for a in range(3):
                for b in range(3):
                    R[J * nc + I, (2 * J + a) * n + 2 * I + b] = w[a] * w[b] / 16.0
    return R


@pytest.mark.parametrize("nu1,nu2", [(1, 0), (2, 1)])
def test_vcycle_with_level_weights_equals_the_error_propagation_matrix(nu1, nu2):
    """With a different Jacobi weight on every level, one V(nu1, nu2) cycle from
    e = 0 equals (I - E_0) A_0^{-1} r, E the textbook two-grid recursion built
    from dense matrices: S_l = I - omega_l D_l^{-1} A_l, E_L = S_L^(nu1+nu2) on the
    coarsest grid, E_l = S_l^nu2 (I - P (I - E_{l+1}) A_{l+1}^{-1} R A_l) S_l^nu1,
    R full weighting and P = 4 R^T (bilinear interpolation)."""
    n = 15
    rng = np.random.default_rng(8)
    k = np.exp(rng.standard_normal((n + 2, n + 2)))
    sts = op.level_stencils_div(k, (1.0, -0.5), num_levels(n))
    oms = [0.7, 1.3, 1.1]
    assert len(sts) == 3
    A = [op.dense_matrix(st) for st in sts]
    S = [np.eye(a.shape[0]) - om * np.diag(1.0 / np.diag(a)) @ a for a, om in zip(A, oms)]
    E = np.linalg.matrix_power(S[2], nu1 + nu2)
    for lev in (1, 0):
        R = _dense_fw(sts[lev].n)
        P = 4.0 * R.T
        cgc = np.eye(A[lev].shape[0]) - P @ (np.eye(E.shape[0]) - E) @ np.linalg.solve(A[lev + 1], R @ A[lev])
        E = np.linalg.matrix_power(S[lev], nu2) @ cgc @ np.linalg.matrix_power(S[lev], nu1)
    r = rng.standard_normal(n * n)
    expect = (np.eye(n * n) - E) @ np.linalg.solve(A[0], r)
    got = gmg.vcycle(sts, r.reshape(n, n), nu1, nu2, oms).ravel()
    assert np.linalg.norm(got - expect) <= 1e-11 * np.linalg.norm(expect)
