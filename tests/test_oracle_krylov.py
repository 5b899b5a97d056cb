"""Pins for the oracle's flexible GMRES (MGCNN as a Krylov preconditioner).

* Identity preconditioner: after k steps the residual is the minimum of
  ||f - A u|| over u in the Krylov space span{r0, A r0, ..., A^(k-1) r0},
  computed here by brute force (explicit basis + least squares).
* Exact preconditioner (dense inverse): one step.
* The 8-channel GMG V(1,0) network as preconditioner: the converged iterate is
  the dense direct solve, also across restarts.
"""
import numpy as np

from oracle import gmg
from oracle import krylov
from oracle import mgcnn as mg
from oracle import operator as op
from oracle.grid import num_levels
from paper_2312_11093_gb300 import inputs


def _problem(n, seed, b=(1.0, 0.5)):
    rng = np.random.default_rng(seed)
    k = inputs.lognormal_k(n, 0.1, rng)
    f = inputs.normal_rhs(n, rng)
    return op.level_stencils_div(k, b, num_levels(n)), f


def test_identity_preconditioner_is_minimal_residual():
    sts, f = _problem(7, 1, b=(3.0, -2.0))
    A = op.dense_matrix(sts[0])
    apply_A = lambda x: op.apply(sts[0], x)
    u, it, hist = krylov.fgmres(apply_A, lambda v: v.copy(), f, None, 1e-30, 12, 49)
    r0 = f.ravel()
    K = [r0]
    for k in range(1, 13):
        Q, _ = np.linalg.qr(np.stack(K, axis=1))
        y, *_ = np.linalg.lstsq(A @ Q, r0, rcond=None)
        best = np.linalg.norm(r0 - A @ (Q @ y)) / np.linalg.norm(r0)
        # the monomial Krylov basis of the brute force loses digits as k grows
        assert abs(hist[k] - best) <= 1e-8 * max(best, 1e-3), k
        K.append(A @ K[-1])


def test_exact_preconditioner_one_step():
    sts, f = _problem(7, 2)
    Ainv = np.linalg.inv(op.dense_matrix(sts[0]))
    apply_A = lambda x: op.apply(sts[0], x)
    u, it, hist = krylov.fgmres(apply_A, lambda v: (Ainv @ v.ravel()).reshape(v.shape), f, None, 1e-12, 10, 10)
    assert it == 1 and hist[-1] <= 1e-12


def test_v10_network_preconditioner_reaches_direct_solve_with_restarts():
    n = 31
    sts, f = _problem(n, 3)
    w = mg.gmg_v10_weights()
    s = mg.gmg_v10_setup(sts, 0.8)
    apply_A = lambda x: op.apply(sts[0], x)
    B = lambda v: mg.solve_phase(w, s, v)
    ustar = np.linalg.solve(op.dense_matrix(sts[0]), f.ravel()).reshape(n, n)
    for restart in (30, 4):
        u, it, hist = krylov.fgmres(apply_A, B, f, None, 1e-11, 200, restart)
        assert hist[-1] <= 1e-11 and len(hist) == it + 1   # one entry per inner iteration
        assert np.linalg.norm(u - ustar) / np.linalg.norm(ustar) <= 1e-8
        true = np.linalg.norm(f - apply_A(u)) / np.linalg.norm(f)
        assert abs(true - hist[-1]) <= 1e-3 * hist[-1] + 1e-15
    # Krylov acceleration beats the stationary iteration with the same network
    _, it_st, _, _ = gmg.stationary_solve(sts, f, None, 1e-11, 500, 1, 0, 0.8)
    u, it_k, _ = krylov.fgmres(apply_A, B, f, None, 1e-11, 200, 30)
    assert it_k < it_st
