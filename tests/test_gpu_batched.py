"""Batched solves of uneven sizes (one CUDA graph launch per batch) against
independent single-problem solves of the same fields with the same network,
and against the oracle."""
import numpy as np
import pytest
import torch

from oracle import mgcnn as omg
from paper_2312_11093_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2312_11093_gb300 import build
    build.build()
    from paper_2312_11093_gb300 import mgcnn
    mgcnn.load()
    return mgcnn


def _weights(M):
    """A convergent 8-channel network: trained weights when present, else random
    weights with a small output layer (the iteration then contracts slowly)."""
    import os
    path = os.path.join(os.path.dirname(M.__file__), "weights", "mgcnn_c8_trained.npy")
    if os.path.exists(path):
        return np.load(path)
    from paper_2312_11093_gb300.train import init_weights
    return init_weights(8, 1, 1, np.random.default_rng(3), out_scale=0.05)


def _fields(sizes, seed):
    rng = np.random.default_rng(seed)
    ks, fs = [], []
    for i, n in enumerate(sizes):
        kind = i % 3
        k = (inputs.lognormal_k(n, 0.1, rng) if kind == 0 else
             inputs.random_blocks_k(n, rng) if kind == 1 else inputs.checkerboard_k(n))
        ks.append(np.ascontiguousarray(k.ravel()))
        fs.append(np.ascontiguousarray(inputs.normal_rhs(n, rng).ravel()))
    return ks, fs


def test_batched_equals_single_problem_solves(M):
    """Same kernels, same arithmetic per pixel (the tile shape does not change the
    summation order): bit-identical iterates.  The single solve sums its norms in
    the fused finest down kernel's order, the batch in the residual kernel's: the
    final relative residuals agree to rounding."""
    sizes = [63, 15, 127, 63, 7, 31, 127, 3, 63]
    ks, fs = _fields(sizes, 1)
    w = _weights(M)
    sv = M.Solver(8, 1, 1, precision="mixed_bf16")
    sv.set_weights(w)
    sv.setup_batched(ks, sizes)
    us = [np.zeros(n * n) for n in sizes]
    st, iters, relres, stat = sv.solve_batched(fs, us, 1e-6, 40)
    for i, n in enumerate(sizes):
        one = M.Solver(8, 1, 1, precision="mixed_bf16")
        one.set_weights(w)
        one.setup(ks[i].copy(), n)
        u = np.zeros(n * n)
        st1, it1, h1 = one.solve(fs[i].copy(), u, 1e-6, 40)
        assert it1 == iters[i], (i, n, it1, iters[i])
        assert np.array_equal(u, us[i]), (i, n)
        assert abs(relres[i] - h1[-1]) <= 1e-13 * h1[-1]
        assert stat[i] == st1


def test_batched_coarse_tail_equals_a_launch_per_level(M):
    """Classes run concurrently, each with its own coarse tail kernel and grid
    barrier; a class with more tiles than the cooperative grid has blocks (24
    problems of 255^2: 768 tiles on level 1) strides them.  Against a launch per
    level: bit-identical iterates."""
    sizes = [255] * 24 + [63] * 30 + [1023] * 2 + [15] * 3
    ks, fs = _fields(sizes, 5)
    w = _weights(M)
    res = {}
    for t in (255, 0):
        sv = M.Solver(8, 1, 1, precision="mixed_bf16")
        sv.set_option(sv.OPT_COARSE_TAIL, t)
        sv.set_weights(w)
        sv.setup_batched(ks, sizes)
        us = [np.zeros(n * n) for n in sizes]
        st, iters, relres, stat = sv.solve_batched(fs, us, 1e-30, 4, per_problem=True)
        res[t] = (list(iters), us, list(stat))
    assert res[255][0] == res[0][0]
    assert res[255][2] == res[0][2]
    for a, b in zip(res[255][1], res[0][1]):
        assert np.array_equal(a, b)


def test_batched_statuses_and_special_cases(M):
    sizes = [31, 31, 15]
    ks, fs = _fields(sizes, 2)
    fs[1] = np.zeros(31 * 31)                   # f = 0: u = 0, no cycles
    fs[2][5] = np.nan                           # non-finite right-hand side
    sv = M.Solver(8, 1, 1, precision="mixed_bf16")
    sv.set_weights(_weights(M))
    sv.setup_batched(ks, sizes)
    us = [np.ones(n * n) for n in sizes]
    with pytest.raises(M.MGCNNError):
        sv.solve_batched(fs, us, 1e-30, 3)
    fs[2][5] = 0.0
    us = [np.ones(n * n) for n in sizes]
    st, iters, relres, stat = sv.solve_batched(fs, us, 1e-30, 3)
    assert st == M.NOT_CONVERGED
    assert list(iters) == [3, 0, 3] and stat[1] == M.OK and not us[1].any()


def test_batched_rejects_unsupported_config(M):
    sv = M.Solver(13, 3, 2, precision="mixed_bf16")
    sv.set_weights(M.gmg_weights(2, 2))
    with pytest.raises(M.MGCNNError) as ei:
        sv.setup_batched([np.ones(9 * 9)], [7])
    assert ei.value.status == M.ERR_SIZE


def test_batched_gmg_v10_equals_single_solves_and_converges(M):
    """Batched setup with the analytic V(1,0) tensors: every problem's iterate is the
    single-problem solve's bit for bit (same kernels, same setup values), and on GRF
    fields the network converges to 1e-6 (checked again by the oracle's residual)."""
    from oracle import operator as oop
    sizes = [63, 127, 31, 63, 255, 127]
    rng = np.random.default_rng(9)
    ks = [np.ascontiguousarray(inputs.lognormal_k(n, 0.1, rng).ravel()) for n in sizes]
    fs = [np.ascontiguousarray(inputs.normal_rhs(n, rng).ravel()) for n in sizes]
    w = M.gmg_v10_weights()
    sv = M.Solver(8, 1, 1, precision="mixed_bf16")
    sv.set_weights(w)
    sv.setup_batched(ks, sizes, gmg_omega=0.8)
    us = [np.zeros(n * n) for n in sizes]
    st, iters, relres, stat = sv.solve_batched(fs, us, 1e-6, 200)
    assert st == M.OK and (stat == M.OK).all()
    for i, n in enumerate(sizes):
        one = M.Solver(8, 1, 1, precision="mixed_bf16")
        one.set_weights(w)
        one.setup_gmg(ks[i], n, 0.8)
        u1 = np.zeros(n * n)
        st1, it1, h1 = one.solve(fs[i].copy(), u1, 1e-6, 200)
        assert it1 == iters[i] and np.array_equal(u1, us[i]), i
        st_ = oop.stencil_div(ks[i].reshape(n + 2, n + 2), (1.0, 0.5))
        r = fs[i].reshape(n, n) - oop.apply(st_, us[i].reshape(n, n))
        assert np.linalg.norm(r) / np.linalg.norm(fs[i]) <= 1.01e-6



@pytest.mark.parametrize("coarse_k", [0, 1])
def test_batched_level_weights_equal_single_solves(M, coarse_k):
    """Batched setup with per-level Jacobi weights (finest, in between, coarsest),
    and either coarse-coefficient rule: each problem gets the weights on its own
    hierarchy, so every iterate equals the single-problem solve with
    mgcnn_setup_gmg_levels bit for bit."""
    sizes = [63, 255, 31, 127, 63]
    rng = np.random.default_rng(19)
    ks = [np.ascontiguousarray(inputs.lognormal_k(n, 0.1, rng).ravel()) for n in sizes]
    fs = [np.ascontiguousarray(inputs.normal_rhs(n, rng).ravel()) for n in sizes]
    om = (0.8, 1.5, 1.0)
    w = M.gmg_v10_weights()
    sv = M.Solver(8, 1, 1, precision="mixed_bf16")
    sv.set_weights(w)
    sv.set_option(sv.OPT_COARSE_K, coarse_k)
    sv.setup_batched(ks, sizes, gmg_omega=om)
    us = [np.zeros(n * n) for n in sizes]
    st, iters, relres, stat = sv.solve_batched(fs, us, 1e-6, 200)
    assert st == M.OK and (stat == M.OK).all()
    for i, n in enumerate(sizes):
        one = M.Solver(8, 1, 1, precision="mixed_bf16")
        one.set_weights(w)
        one.set_option(one.OPT_COARSE_K, coarse_k)
        one.setup_gmg(ks[i], n, om)
        u1 = np.zeros(n * n)
        st1, it1, h1 = one.solve(fs[i].copy(), u1, 1e-6, 200)
        assert it1 == iters[i] and np.array_equal(u1, us[i]), i


def test_batched_divergence_limit(M):
    """A batch mixing GRF problems (which converge) with random-block problems
    (which diverge): with OPT_DIVTOL = 6 every block problem ends with ERR_DIVERGED
    at its first cycle above 1e6, and every GRF problem's iterate is bit for bit the
    one without the limit."""
    sizes = [63, 127, 63, 255, 127, 31]
    rng = np.random.default_rng(23)
    ks, fs = [], []
    for i, n in enumerate(sizes):
        k = inputs.lognormal_k(n, 0.1, rng) if i % 2 == 0 else inputs.random_blocks_k(n, rng)
        ks.append(np.ascontiguousarray(k.ravel()))
        fs.append(np.ascontiguousarray(inputs.normal_rhs(n, rng).ravel()))
    out = {}
    for divtol in (0, 6):
        sv = M.Solver(8, 1, 1, precision="mixed_bf16")
        sv.set_weights(M.gmg_v10_weights())
        sv.set_option(sv.OPT_DIVTOL, divtol)
        sv.setup_batched(ks, sizes, gmg_omega=0.8)
        us = [np.zeros(n * n) for n in sizes]
        st, iters, relres, stat = sv.solve_batched(fs, us, 1e-6, 60, per_problem=True)
        out[divtol] = (iters.copy(), relres.copy(), stat.copy(), us)
    it0, rr0, st0, u0 = out[0]
    it6, rr6, st6, u6 = out[6]
    for i in range(len(sizes)):
        if i % 2 == 0:
            assert st0[i] == st6[i] == M.OK and it0[i] == it6[i] and np.array_equal(u0[i], u6[i]), i
        else:
            assert st6[i] == M.ERR_DIVERGED and rr6[i] > 1e6 and it6[i] < it0[i], i


def _mixture(sizes, seed):
    """Problems over the three coefficient families in turn (GRF, random blocks of
    contrast 1e4, 16 x 16 checkerboard {1, 100})."""
    rng = np.random.default_rng(seed)
    ks, fs = [], []
    for i, n in enumerate(sizes):
        fam = i % 3
        k = (inputs.lognormal_k(n, 0.1, rng) if fam == 0 else
             inputs.random_blocks_k(n, rng) if fam == 1 else inputs.checkerboard_k(n))
        ks.append(np.ascontiguousarray(k.ravel()))
        fs.append(np.ascontiguousarray(inputs.normal_rhs(n, rng).ravel()))
    return ks, fs


def test_batched_krylov_solves_the_three_families(M):
    """Batched FGMRES(30) with the V(1,0) network on the arithmetic coarse
    coefficient: every problem of an uneven three-family batch reaches 1e-6
    (checked by the oracle's FP64 residual), in the iteration count of the
    single-problem FGMRES within two (the dot products sum in another order)."""
    from oracle import operator as oop
    sizes = [63, 127, 31, 255, 63, 127, 31, 63, 255]
    ks, fs = _mixture(sizes, 31)
    om = (0.8, 1.5, 1.0)
    w = M.gmg_v10_weights()
    sv = M.Solver(8, 1, 1, precision="mixed_bf16")
    sv.set_weights(w)
    sv.set_option(sv.OPT_COARSE_K, 1)
    sv.setup_batched(ks, sizes, gmg_omega=om)
    us = [np.zeros(n * n) for n in sizes]
    st, iters, relres, stat = sv.solve_batched_krylov(fs, us, 1e-6, 300, 30)
    assert st == M.OK and (stat == M.OK).all(), stat
    for i, n in enumerate(sizes):
        r = fs[i].reshape(n, n) - oop.apply(oop.stencil_div(ks[i].reshape(n + 2, n + 2), (1.0, 0.5)),
                                            us[i].reshape(n, n))
        true = np.linalg.norm(r) / np.linalg.norm(fs[i])
        assert true <= 1.05e-6 and abs(true - relres[i]) <= 1e-3 * true, (i, true, relres[i])
        one = M.Solver(8, 1, 1, precision="mixed_bf16")
        one.set_weights(w)
        one.set_option(one.OPT_COARSE_K, 1)
        one.setup_gmg(ks[i], n, om)
        u1 = np.zeros(n * n)
        st1, it1, h1 = one.solve_krylov(fs[i].copy(), u1, 1e-6, 300, 30)
        assert st1 == M.OK and abs(it1 - iters[i]) <= 2, (i, it1, iters[i])


def test_batched_krylov_edge_cases(M):
    """A zero right-hand side gives u = 0 in no iterations; maxit = 0 reports
    NOT_CONVERGED with the initial residual; a restart outside 1..64 is an error;
    the stationary batched solve still works on the same setup afterwards."""
    sizes = [31, 63, 31]
    ks, fs = _mixture(sizes, 32)
    fs[2] = np.zeros(31 * 31)
    sv = M.Solver(8, 1, 1, precision="mixed_bf16")
    sv.set_weights(M.gmg_v10_weights())
    sv.setup_batched(ks, sizes, gmg_omega=0.8)
    us = [np.full(n * n, 0.5) for n in sizes]
    st, iters, relres, stat = sv.solve_batched_krylov(fs, us, 1e-6, 0, 30)
    assert st == M.NOT_CONVERGED
    assert stat[2] == M.OK and iters[2] == 0 and not us[2].any()
    assert stat[0] == M.NOT_CONVERGED and iters[0] == 0 and relres[0] > 1e-6
    for bad in (0, 65):
        with pytest.raises(M.MGCNNError) as ei:
            sv.solve_batched_krylov(fs, us, 1e-6, 10, bad)
        assert ei.value.status == M.ERR_ARG
    us = [np.zeros(n * n) for n in sizes]
    st, iters, relres, stat = sv.solve_batched(fs[:1] + fs[1:], us, 1e-6, 200, per_problem=True)
    assert stat[0] == M.OK and stat[2] == M.OK

@pytest.mark.parametrize("cfg", [(0, True), (1, False)])
def test_batched_first_cycle_against_the_oracle(M, cfg):
    """Every problem of an uneven batch over the three coefficient families, one
    cycle from u = 0 (u_1 = B f with the batch's BF16 network and setup network),
    against the oracle's FP64 B f with the same weights: the bar of the
    single-problem mixed test, 5e-2 (BF16 rounding along one cycle)."""
    from oracle import operator as oop
    from oracle.grid import num_levels
    sbd, idiag = cfg
    sizes = [31, 63, 15, 127, 63, 7]
    ks, fs = _fields(sizes, 21)
    w = omg.random_weights(8, 1, 1, np.random.default_rng(22))
    sv = M.Solver(8, 1, 1, precision="mixed_bf16", scale_by_diag=sbd, input_diag=idiag)
    sv.set_weights(M.pack_weights(w, 8, 1, 1))
    sv.setup_batched(ks, sizes)
    us = [np.zeros(n * n) for n in sizes]
    st, iters, relres, stat = sv.solve_batched(fs, us, 0.0, 1, per_problem=True)
    for i, n in enumerate(sizes):
        assert iters[i] == 1 and stat[i] == M.NOT_CONVERGED, i
        sts = oop.level_stencils_div(ks[i].reshape(n + 2, n + 2), (1.0, 0.5), num_levels(n))
        s = omg.setup(w, sts, scale_by_diag=sbd)
        e_ref = omg.solve_phase(w, s, fs[i].reshape(n, n), d_inv=(1.0 / sts[0].aC) if idiag else None)
        err = np.linalg.norm(us[i] - e_ref.ravel()) / np.linalg.norm(e_ref)
        assert err <= 5e-2, (i, n, err)
