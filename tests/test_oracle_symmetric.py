"""Pins of the oracle's symmetric network variant (Remark "Symmetric problem",
Sec. 3.3) and of its CG / MINRES drivers, against properties fixed by the
mathematics: exact symmetry and positive definiteness of B, agreement with the
general network where the two forms coincide, the textbook BPX operator written
out with dense matrices, and the Krylov optimality of PCG and MINRES iterates
checked by brute-force least squares on tiny problems."""
import numpy as np
import pytest

from oracle import krylov as ok
from oracle import mgcnn as omg
from oracle import operator as oop
from oracle.grid import num_levels
from paper_2312_11093_gb300 import inputs


def dense(apply, N, n):
    M = np.zeros((N, N))
    for i in range(N):
        e = np.zeros(N)
        e[i] = 1.0
        M[:, i] = apply(e.reshape(n, n)).ravel()
    return M


def spd_problem(n, seed):
    rng = np.random.default_rng(seed)
    k = inputs.lognormal_k(n, 0.1, rng)
    sts = oop.level_stencils_div(k, (0.0, 0.0), num_levels(n))
    return rng, sts


@pytest.mark.parametrize("nu", [1, 2])
@pytest.mark.parametrize("C", [4, 8])
def test_symmetric_network_is_symmetric_and_positive_definite(C, nu):
    """B of the tied network equals B^T to rounding and has positive eigenvalues,
    for random weights and random setup tensors of both signs."""
    n = 15
    rng, sts = spd_problem(n, 3 + C + nu)
    w = omg.random_weights(C, nu, nu, rng, scale=0.6)
    s = [rng.standard_normal((C, st.n, st.n)) for st in sts]
    B = dense(lambda r: omg.solve_phase_symmetric(w, s, r), n * n, n)
    assert np.abs(B - B.T).max() <= 1e-14 * np.abs(B).max()
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0.0


def test_symmetric_network_equals_general_form_for_uniform_setup():
    """With a setup tensor that is one scalar per level, s * (K^T x) = K^T (s * x),
    so the symmetric network is the general network (Algorithm 3) with the tied
    weight set."""
    n = 31
    rng, sts = spd_problem(n, 11)
    w = omg.random_weights(8, 2, 2, rng)
    s = [np.full((8, st.n, st.n), rng.uniform(-1.0, 1.0)) for st in sts]
    r = rng.standard_normal((n, n))
    a = omg.solve_phase_symmetric(w, s, r)
    b = omg.solve_phase(omg.symmetric_weights(w), s, r)
    assert np.linalg.norm(a - b) <= 1e-13 * np.linalg.norm(b)


def fw_matrix(n):
    """Full weighting (1/16)[1 2 1; 2 4 2; 1 2 1] from the n^2 fine to the
    ((n-1)/2)^2 coarse grid, coarse node (J, I) centred on fine node (2J+1, 2I+1)."""
    nc = (n - 1) // 2
    R = np.zeros((nc * nc, n * n))
    wts = {0: 4.0, 1: 2.0, 2: 1.0}
    for J in range(nc):
        for I in range(nc):
            for dj in (-1, 0, 1):
                for di in (-1, 0, 1):
                    R[J * nc + I, (2 * J + 1 + dj) * n + 2 * I + 1 + di] = wts[abs(dj) + abs(di)] / 16.0
    return R


@pytest.mark.parametrize("omega,C", [(1.0, 4), (0.7, 2)])
def test_bpx_network_is_the_textbook_bpx_operator(omega, C):
    """The BPX weights and setup turn the symmetric network into
    sum_l 4^l R_l^T (omega D_l^{-1}) R_l + eps^2 sum_l R_l^T R_l, with R_l the
    l-fold full weighting and D_l the diagonal of the level-l operator."""
    n = 15
    rng, sts = spd_problem(n, 21)
    w = omg.bpx_weights(C)
    s = omg.bpx_setup(sts, omega, C)
    B = dense(lambda r: omg.solve_phase_symmetric(w, s, r), n * n, n)
    ref = np.zeros((n * n, n * n))
    Rl = np.eye(n * n)
    nl = n
    for lev, st in enumerate(sts):
        ref += 4.0 ** lev * Rl.T @ np.diag(omega / st.aC.ravel()) @ Rl + omg.BPX_EPS ** 2 * Rl.T @ Rl
        if lev + 1 < len(sts):
            Rl = fw_matrix(nl) @ Rl
            nl = (nl - 1) // 2
    assert np.linalg.norm(B - ref) <= 1e-12 * np.linalg.norm(ref)


def test_bpx_pcg_iterations_do_not_grow_with_the_grid():
    """Grid-independent convergence of CG with the BPX network (the reason for a
    symmetric multilevel preconditioner): the iteration count to 1e-8 barely
    changes from 31^2 to 127^2 while unpreconditioned CG needs several times more."""
    its = []
    for n in (31, 63, 127):
        rng, sts = spd_problem(n, 30 + n)
        f = inputs.normal_rhs(n, rng)
        w, s = omg.bpx_weights(4), omg.bpx_setup(sts, 1.0, 4)
        ap = lambda x: oop.apply(sts[0], x)
        u, it, hist = ok.pcg(ap, lambda r: omg.solve_phase_symmetric(w, s, r), f, None, 1e-8, 400)
        assert hist[-1] <= 1e-8
        assert np.linalg.norm(f - ap(u)) <= 1.1e-8 * np.linalg.norm(f)
        its.append(it)
        _, it_cg, _ = ok.pcg(ap, lambda r: r, f, None, 1e-8, 4000)
        assert it_cg > 3 * it
    assert max(its) - min(its) <= 4


def krylov_basis(apply_MA, z0, k):
    """Orthonormal basis of span{z0, (MA) z0, ..., (MA)^{k-1} z0}."""
    V = [z0 / np.linalg.norm(z0)]
    for _ in range(k - 1):
        w = apply_MA(V[-1])
        for _ in range(2):
            for v in V:
                w = w - np.dot(v, w) * v
        V.append(w / np.linalg.norm(w))
    return np.stack(V, axis=1)


def tiny_spd_system(seed):
    n = 7
    rng, sts = spd_problem(n, seed)
    A = oop.dense_matrix(sts[0])
    w = omg.random_weights(4, 1, 1, rng, scale=0.6)
    s = [rng.standard_normal((4, st.n, st.n)) for st in sts]
    M = dense(lambda r: omg.solve_phase_symmetric(w, s, r), n * n, n)
    M = 0.5 * (M + M.T)
    f = rng.standard_normal(n * n)
    u0 = rng.standard_normal(n * n)
    return n, A, M, f, u0


@pytest.mark.parametrize("k", [1, 2, 4, 7])
def test_pcg_iterate_minimises_the_energy_error(k):
    """PCG's k-th iterate minimises the A-norm of the error over
    u0 + K_k(M A, M r0) (brute force: Galerkin projection on a Krylov basis)."""
    n, A, M, f, u0 = tiny_spd_system(5)
    u, it, _ = ok.pcg(lambda x: A @ x, lambda r: M @ r, f, u0, 0.0, k)
    assert it == k
    r0 = f - A @ u0
    V = krylov_basis(lambda x: M @ (A @ x), M @ r0, k)
    y = np.linalg.solve(V.T @ A @ V, V.T @ r0)
    ref = u0 + V @ y
    assert np.linalg.norm(u - ref) <= 1e-9 * np.linalg.norm(ref)


def test_pcg_identity_preconditioner_solves_the_system():
    n, A, M, f, u0 = tiny_spd_system(6)
    u, it, hist = ok.pcg(lambda x: A @ x, lambda r: r, f, None, 1e-13, 500)
    ref = np.linalg.solve(A, f)
    assert hist[-1] <= 1e-13
    assert np.linalg.norm(u - ref) <= 1e-9 * np.linalg.norm(ref)
    # the history is the norm of the true residual up to rounding
    assert abs(np.linalg.norm(f - A @ u) / np.linalg.norm(f) - hist[-1]) <= 1e-12


@pytest.mark.parametrize("k", [1, 2, 4, 7])
def test_minres_iterate_minimises_the_preconditioned_residual(k):
    """MINRES's k-th iterate minimises ||f - A u||_M over u0 + K_k(M A, M r0), and
    its history entry is that minimum relative to ||r0||_M."""
    n, A, M, f, u0 = tiny_spd_system(7)
    u, it, hist = ok.minres(lambda x: A @ x, lambda r: M @ r, f, u0, 0.0, k)
    assert it == k
    r0 = f - A @ u0
    V = krylov_basis(lambda x: M @ (A @ x), M @ r0, k)
    AV = A @ V
    y = np.linalg.solve(AV.T @ M @ AV, AV.T @ M @ r0)
    ref = u0 + V @ y
    assert np.linalg.norm(u - ref) <= 1e-9 * np.linalg.norm(ref)
    mnorm = lambda v: np.sqrt(v @ M @ v)
    assert abs(hist[-1] - mnorm(f - A @ u) / mnorm(r0)) <= 1e-10


def test_minres_without_preconditioner_is_minimal_residual():
    """With M = I, MINRES on a symmetric matrix and GMRES (the pinned FGMRES with
    an identity preconditioner, no restart) minimise the same 2-norm over the
    same Krylov space: equal iterates."""
    n, A, M, f, u0 = tiny_spd_system(8)
    for k in (1, 3, 6):
        um, _, _ = ok.minres(lambda x: A @ x, lambda r: r, f, u0, 0.0, k)
        ug, _, _ = ok.fgmres(lambda x: A @ x, lambda r: r, f, u0, 0.0, k, k)
        assert np.linalg.norm(um - ug) <= 1e-9 * np.linalg.norm(ug)


def test_zero_rhs_and_exact_guess():
    n, A, M, f, u0 = tiny_spd_system(9)
    u, it, hist = ok.pcg(lambda x: A @ x, lambda r: M @ r, np.zeros_like(f), None, 1e-8, 10)
    assert it == 0 and not u.any() and hist == [0.0]
    x = np.linalg.solve(A, f)
    u, it, hist = ok.minres(lambda x_: A @ x_, lambda r: M @ r, A @ x, x, 1e-8, 10)
    assert it <= 1 and np.linalg.norm(u - x) <= 1e-12 * np.linalg.norm(x)
