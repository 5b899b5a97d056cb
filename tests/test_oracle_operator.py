"""Pins for the oracle's discretisation (Sec. 2.5, Remark 2.1).

Each check comes from outside the oracle's own formulas: closed-form
eigenvalues, exactness on polynomials, invariants of the matrix, observed
convergence order on a manufactured solution, and the paper's printed
kernels (tests/golden/paper_fd_kernels.txt).
"""
import math
import os

import numpy as np
import pytest

from oracle import operator as op
from oracle.grid import level_sizes, num_levels, spacing

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_fd_kernels.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if not line:
            continue
        k, v = line.split(":")
        vals = [float(t) for t in v.split()]
        out[k.strip()] = np.array(vals).reshape(3, 3) if len(vals) == 9 else vals[0]
    return out


def test_level_rule_matches_paper():
    g = _golden()
    assert num_levels(31) == g["levels_31"]
    assert num_levels(63) == g["levels_63"]
    assert level_sizes(31) == [31, 15, 7, 3]
    assert level_sizes(4095)[-1] == 3 and len(level_sizes(4095)) == 11
    with pytest.raises(ValueError):
        num_levels(32)


@pytest.mark.parametrize("n", [7, 15])
def test_constant_k_laplacian_eigenvalues(n):
    """k = kappa, b = 0: A = kappa * (textbook 5-point Laplacian), eigenvalues
    (4 kappa / h^2)(sin^2(p pi h / 2) + sin^2(q pi h / 2)), p, q = 1..n."""
    kappa = 2.5
    h = spacing(n)
    st = op.stencil_div(np.full((n + 2, n + 2), kappa), (0.0, 0.0))
    ev = np.sort(np.linalg.eigvalsh(op.dense_matrix(st)))
    p = np.arange(1, n + 1)
    s2 = np.sin(p * math.pi * h / 2) ** 2
    ref = np.sort((4 * kappa / h ** 2 * (s2[:, None] + s2[None, :])).ravel())
    np.testing.assert_allclose(ev, ref, rtol=1e-12)


@pytest.mark.parametrize("bx,by", [(1.0, 0.5), (-0.7, 1.3), (0.0, -2.0)])
def test_polynomial_exactness(bx, by):
    """Constant k: centred second differences are exact on quadratics and the
    one-sided upwind difference of x^2 is 2x -+ h.  With p = x^2 + x y + 2 y^2:
      -k Lap p = -6k,  upwind_x = 2x + y - sgn(bx) h,  upwind_y = x + 4y - 2 sgn(by) h.
    Checked on nodes whose four neighbours are interior (zero padding elsewhere)."""
    n, kappa = 15, 1.7
    h = spacing(n)
    st = op.stencil_div(np.full((n + 2, n + 2), kappa), (bx, by))
    x = np.arange(1, n + 1) * h
    X, Y = np.meshgrid(x, x)               # [j, i]: Y varies along rows
    u = X ** 2 + X * Y + 2 * Y ** 2
    Au = op.apply(st, u)
    ref = (-6 * kappa + bx * (2 * X + Y - np.sign(bx) * h)
           + by * (X + 4 * Y - 2 * np.sign(by) * h))
    np.testing.assert_allclose(Au[1:-1, 1:-1], ref[1:-1, 1:-1], rtol=1e-9, atol=1e-9)


def test_symmetry_and_row_sums_variable_k():
    """b = 0: A is symmetric positive definite for any positive k; A 1 vanishes
    except at nodes next to the boundary, where it equals the boundary-face
    conductances over h^2 (which are positive)."""
    n = 15
    rng = np.random.default_rng(3)
    k = 10 ** rng.uniform(-2, 2, size=(n + 2, n + 2))
    st = op.stencil_div(k, (0.0, 0.0))
    M = op.dense_matrix(st)
    np.testing.assert_allclose(M, M.T, rtol=1e-13, atol=0)
    assert np.linalg.eigvalsh(M).min() > 0
    rs = op.apply(st, np.ones((n, n)))
    assert np.allclose(rs[1:-1, 1:-1], 0.0, atol=1e-9 * np.abs(st.aC).max())
    assert (rs[0, :] > 0).all() and (rs[:, 0] > 0).all() and (rs[-1, :] > 0).all()


def test_transpose_apply_matches_dense():
    n = 7
    rng = np.random.default_rng(4)
    st = op.stencil_div(np.exp(rng.standard_normal((n + 2, n + 2))), (1.0, -0.5))
    M = op.dense_matrix(st)
    v = rng.standard_normal((n, n))
    np.testing.assert_allclose(op.apply_transpose(st, v).ravel(), M.T @ v.ravel(), rtol=1e-12)


def _manufactured(n, b):
    """u* = sin(pi x) sin(pi y), k = 1 + 0.5 sin(2 pi x) cos(pi y); f = -div(k grad u*) + b.grad u*."""
    h = spacing(n)
    xs = np.arange(n + 2) * h
    Xn, Yn = np.meshgrid(xs, xs)
    k = 1 + 0.5 * np.sin(2 * np.pi * Xn) * np.cos(np.pi * Yn)
    X, Y = Xn[1:-1, 1:-1], Yn[1:-1, 1:-1]
    pi = np.pi
    u = np.sin(pi * X) * np.sin(pi * Y)
    ux = pi * np.cos(pi * X) * np.sin(pi * Y)
    uy = pi * np.sin(pi * X) * np.cos(pi * Y)
    lap = -2 * pi ** 2 * u
    kk = 1 + 0.5 * np.sin(2 * pi * X) * np.cos(pi * Y)
    kx = pi * np.cos(2 * pi * X) * np.cos(pi * Y)
    ky = -0.5 * pi * np.sin(2 * pi * X) * np.sin(pi * Y)
    f = -(kk * lap + kx * ux + ky * uy) + b[0] * ux + b[1] * uy
    return k, f, u


@pytest.mark.parametrize("b,order", [((0.0, 0.0), 2.0), ((1.0, 0.5), 1.0)])
def test_manufactured_solution_order(b, order):
    """Observed discretisation order: 2 for pure diffusion (centred, harmonic faces),
    1 with first-order upwind convection (Sec. 2.5)."""
    errs, hs = [], []
    for n in (15, 31, 63):
        k, f, ustar = _manufactured(n, b)
        st = op.stencil_div(k, b)
        uh = np.linalg.solve(op.dense_matrix(st), f.ravel()).reshape(n, n)
        errs.append(np.abs(uh - ustar).max())
        hs.append(spacing(n))
    rates = [math.log(errs[i] / errs[i + 1]) / math.log(hs[i] / hs[i + 1]) for i in range(2)]
    assert abs(rates[-1] - order) < 0.25, rates


def test_nondiv_matches_paper_kernels():
    """The paper's operator K = (1/h){coef Lap5 + v_x^+ dx^- + v_x^- dx^+ + v_y^+ dy^- + v_y^- dy^+}
    with coef = mu / h (Sec. 2.5), built from the printed kernels, equals
    `stencil_nondiv` at an interior node.  The printed image rows grow downwards
    (y decreases), the oracle's rows grow with y: flip the kernel vertically."""
    g = _golden()
    n = 7
    h = spacing(n)
    mu = np.full((n, n), 0.37)
    for ang in (g["velocity_angle"], 2.0, 4.0):
        vx, vy = math.sin(ang), math.cos(ang)
        K = (1.0 / h) * ((0.37 / h) * g["laplace5"]
                         + max(vx, 0) * g["dx_minus"] + min(vx, 0) * g["dx_plus"]
                         + max(vy, 0) * g["dy_minus"] + min(vy, 0) * g["dy_plus"])
        Ky = K[::-1, :]
        st = op.stencil_nondiv(mu, (vx, vy))
        j = i = 3
        got = np.array([[0, st.aS[j, i], 0], [st.aW[j, i], st.aC[j, i], st.aE[j, i]], [0, st.aN[j, i], 0]])
        np.testing.assert_allclose(got, Ky, rtol=1e-13, atol=1e-9)


def test_coarse_operator_is_rediscretisation():
    """Constant k: the rediscretised coarse operator is the 2h Laplacian (Sec. 2.3)."""
    n, kappa = 15, 3.0
    sts = op.level_stencils_div(np.full((n + 2, n + 2), kappa), (0.0, 0.0), 3)
    for st, nl in zip(sts, [15, 7, 3]):
        hl = spacing(nl)
        assert st.n == nl
        np.testing.assert_allclose(st.aC, 4 * kappa / hl ** 2, rtol=1e-13)
        np.testing.assert_allclose(st.aW, -kappa / hl ** 2, rtol=1e-13)


def test_coarse_k_restriction():
    """restrict_k keeps a constant k and reproduces a log-linear k exactly at coarse
    nodes whose 3x3 fine neighbourhood exists (full weighting is exact on linear
    functions); coarse node I sits on fine node 2I."""
    m = 17
    np.testing.assert_allclose(op.restrict_k(np.full((m, m), 4.2)), 4.2, rtol=1e-14)
    j, i = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    k = np.exp(0.3 * i - 0.2 * j + 1.0)
    kc = op.restrict_k(k)
    J, I = np.meshgrid(np.arange(kc.shape[0]), np.arange(kc.shape[0]), indexing="ij")
    ref = np.exp(0.3 * 2 * I - 0.2 * 2 * J + 1.0)
    np.testing.assert_allclose(kc[1:-1, 1:-1], ref[1:-1, 1:-1], rtol=1e-13)
    assert kc.shape == (9, 9)


def test_layered_medium_flux_is_exact():
    """Series resistances: for k that varies only in x and is constant on each
    node's dual cell, the exact solution of -(k u_x)_x = 0 rises by
    q (h/2)(1/k_{i-1} + 1/k_i) between neighbouring nodes (the integral of q/k).
    A two-point flux with the harmonic-mean face reproduces that flux exactly, so
    A u vanishes wherever the stencil sees only interior nodes."""
    n = 15
    h = spacing(n)
    rng = np.random.default_rng(3)
    kx = 10.0 ** rng.uniform(-2.0, 2.0, size=n + 2)          # one value per column, boundary ring included
    k = np.tile(kx, (n + 2, 1))
    u = np.zeros(n + 2)
    for i in range(1, n + 2):
        u[i] = u[i - 1] + 0.5 * h * (1.0 / kx[i - 1] + 1.0 / kx[i])
    U = np.tile(u[1:-1], (n, 1))                             # interior values, u(x) only
    Au = op.apply(op.stencil_div(k, (0.0, 0.0)), U)
    scale = np.max(k) / h ** 2 * np.max(np.abs(U))
    assert np.max(np.abs(Au[1:-1, 1:-1])) <= 1e-12 * scale


def test_coarse_k_restriction_weights_on_a_quadratic():
    """Full weighting (1, 2, 1)/4 of a quadratic adds half the squared fine
    spacing per direction: log k = c (i^2 + j^2) restricts to
    c ((2I)^2 + (2J)^2) + c at coarse nodes whose fine neighbourhood exists."""
    m, c = 17, 0.01
    j, i = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    kc = op.restrict_k(np.exp(c * (i ** 2 + j ** 2)))
    J, I = np.meshgrid(np.arange(kc.shape[0]), np.arange(kc.shape[0]), indexing="ij")
    ref = c * ((2 * I) ** 2 + (2 * J) ** 2) + c
    np.testing.assert_allclose(np.log(kc)[1:-1, 1:-1], ref[1:-1, 1:-1], rtol=1e-12, atol=1e-12)


def test_arithmetic_coarse_k_restriction():
    """The arithmetic full weighting keeps a constant k, reproduces a linear k
    exactly and a quadratic k = 1 + c (i^2 + j^2) as 1 + c ((2I)^2 + (2J)^2) + c
    (the (1, 2, 1)/4 average of x^2 is x^2 + 1/2 per direction) at coarse nodes
    whose fine neighbourhood exists; at a ring node it averages the fine nodes that
    exist with their weights renormalised, and it is never below the geometric
    average (AM-GM)."""
    m = 17
    np.testing.assert_allclose(op.restrict_k(np.full((m, m), 4.2), "arith"), 4.2, rtol=1e-14)
    j, i = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    J, I = np.meshgrid(np.arange(9), np.arange(9), indexing="ij")
    kc = op.restrict_k(2.0 + 0.3 * i + 0.2 * j, "arith")
    np.testing.assert_allclose(kc[1:-1, 1:-1], (2.0 + 0.6 * I + 0.4 * J)[1:-1, 1:-1], rtol=1e-13)
    c = 0.01
    kc = op.restrict_k(1.0 + c * (i ** 2 + j ** 2), "arith")
    ref = 1.0 + c * ((2 * I) ** 2 + (2 * J) ** 2) + c
    np.testing.assert_allclose(kc[1:-1, 1:-1], ref[1:-1, 1:-1], rtol=1e-13)
    k = 10.0 ** np.random.default_rng(4).uniform(-2, 2, size=(m, m))
    kc = op.restrict_k(k, "arith")
    # corner coarse node (0, 0): fine nodes (0..1, 0..1) with weights 4, 2, 2, 1
    expect = (4 * k[0, 0] + 2 * k[0, 1] + 2 * k[1, 0] + k[1, 1]) / 9.0
    assert abs(kc[0, 0] - expect) <= 1e-14 * expect
    # edge coarse node (0, 3): fine rows 0..1, columns 5..7
    wv = np.array([[2.0, 4.0, 2.0], [1.0, 2.0, 1.0]])
    expect = np.sum(wv * k[0:2, 5:8]) / np.sum(wv)
    assert abs(kc[0, 3] - expect) <= 1e-14 * expect
    assert np.all(kc >= op.restrict_k(k) * (1 - 1e-14))
    with pytest.raises(ValueError):
        op.restrict_k(k, "harmonic")
