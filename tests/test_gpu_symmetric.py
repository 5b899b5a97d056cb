"""GPU parity of the symmetric network variant (Remark "Symmetric problem",
Sec. 3.3) and of CG / MINRES with it as preconditioner, against the FP64 oracle:
tied weights, the adjoint up sweep, the BPX setup, and iterate-for-iterate
Krylov histories, all through the C ABI."""
import numpy as np
import pytest
import torch

from oracle import krylov as ok
from oracle import mgcnn as omg
from oracle import operator as oop
from oracle.grid import level_sizes, num_levels
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


def relerr(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def levels_from_nhwc(flat, n, C):
    out, off = [], 0
    for nl in level_sizes(n):
        m = nl * nl * C
        out.append(flat[off:off + m].reshape(nl, nl, C).transpose(2, 0, 1))
        off += m
    return out


def spd_problem(n, seed):
    rng = np.random.default_rng(seed)
    k = inputs.lognormal_k(n, 0.1, rng)
    f = inputs.normal_rhs(n, rng)
    sts = oop.level_stencils_div(k, (0.0, 0.0), num_levels(n))
    return rng, k, f, sts


def symmetric_solver(M, C, nu, **kw):
    sv = M.Solver(C, nu, nu, precision="fp64", input_diag=False, b=(0.0, 0.0), **kw)
    sv.set_option(sv.OPT_SYMMETRIC, 1)
    return sv


@pytest.mark.parametrize("C,nu,n", [(4, 1, 63), (8, 2, 31), (4, 2, 127)])
def test_tied_weights_and_adjoint_vcycle_match_oracle(M, C, nu, n):
    """The library ties the weights as the oracle does (exact copies) and its
    V-cycle is the oracle's symmetric network on the same setup tensors."""
    rng, k, f, sts = spd_problem(n, 100 + n)
    w = omg.random_weights(C, nu, nu, rng)
    sv = symmetric_solver(M, C, nu)
    sv.set_weights(M.pack_weights(w, C, nu, nu))
    assert np.array_equal(sv.get_weights(), M.pack_weights(omg.symmetric_weights(w), C, nu, nu))
    sv.setup(k.ravel().copy(), n)
    s = levels_from_nhwc(sv.get_setup_tensors(), n, C)
    r = rng.standard_normal((n, n))
    e = sv.vcycle(r.ravel().copy())
    assert relerr(e, omg.solve_phase_symmetric(w, s, r)) <= 1e-13


def test_option_after_weights_ties_them(M):
    C, nu, n = 4, 1, 31
    rng, k, f, sts = spd_problem(n, 7)
    w = omg.random_weights(C, nu, nu, rng)
    sv = M.Solver(C, nu, nu, precision="fp64", input_diag=False, b=(0.0, 0.0))
    sv.set_weights(M.pack_weights(w, C, nu, nu))
    sv.set_option(sv.OPT_SYMMETRIC, 1)
    assert np.array_equal(sv.get_weights(), M.pack_weights(omg.symmetric_weights(w), C, nu, nu))


def test_symmetric_vcycle_is_symmetric_on_the_gpu(M):
    """<B x, y> = <x, B y> for the library's V-cycle (random weights and setup)."""
    C, nu, n = 8, 1, 63
    rng, k, f, sts = spd_problem(n, 12)
    sv = symmetric_solver(M, C, nu)
    sv.set_weights(M.pack_weights(omg.random_weights(C, nu, nu, rng), C, nu, nu))
    sv.setup(k.ravel().copy(), n)
    x, y = rng.standard_normal(n * n), rng.standard_normal(n * n)
    bx, by = sv.vcycle(x.copy()), sv.vcycle(y.copy())
    assert abs(bx @ y - x @ by) <= 1e-13 * np.linalg.norm(bx) * np.linalg.norm(y)
    assert x @ bx > 0.0 and y @ by > 0.0


@pytest.mark.parametrize("n,omega,C", [(63, 1.0, 4), (255, 0.7, 2), (127, 1.0, 2)])
def test_bpx_setup_matches_oracle(M, n, omega, C):
    rng, k, f, sts = spd_problem(n, 200 + n)
    sv = symmetric_solver(M, C, 1)
    sv.set_weights(M.bpx_weights(C))
    assert np.array_equal(sv.get_weights(), M.pack_weights(omg.bpx_weights(C), C, 1, 1))
    sv.setup_bpx(k.ravel().copy(), n, omega)
    s = levels_from_nhwc(sv.get_setup_tensors(), n, C)
    # the level operators agree with the oracle's to rounding, so the tensors do too
    for a, b in zip(s, omg.bpx_setup(sts, omega, C)):
        assert np.all(np.abs(a - b) <= 1e-14 * np.abs(b))
    r = rng.standard_normal((n, n))
    assert relerr(sv.vcycle(r.ravel().copy()), omg.solve_phase_symmetric(omg.bpx_weights(C), s, r)) <= 1e-13


@pytest.mark.parametrize("method", ["pcg", "minres"])
@pytest.mark.parametrize("n", [63, 255])
def test_krylov_with_bpx_iterate_for_iterate(M, method, n):
    """CG / MINRES with the BPX network against the oracle.  Two FP64 runs of a
    Krylov method agree only until rounding has cost the Lanczos vectors their
    orthogonality: a 1e-14 relative perturbation of the preconditioner's output
    moves the oracle's own history by up to 40% after about 17 iterations at
    255^2 and may add an iteration.  So the first ten history entries (2-norm
    for CG, B-norm for MINRES) must agree to 1e-9, the iteration counts to two,
    and both runs must reach the tolerance, checked with the oracle's operator."""
    rng, k, f, sts = spd_problem(n, 300 + n)
    sv = symmetric_solver(M, 2, 1)
    sv.set_weights(M.bpx_weights(2))
    sv.setup_bpx(k.ravel().copy(), n, 1.0)
    u = np.zeros(n * n)
    solve = sv.solve_pcg if method == "pcg" else sv.solve_minres
    st, it, hist = solve(f.ravel().copy(), u, 1e-8, 200)
    assert st == M.OK
    w, s = omg.bpx_weights(2), omg.bpx_setup(sts, 1.0, 2)
    run = ok.pcg if method == "pcg" else ok.minres
    u_o, it_o, hist_o = run(lambda x: oop.apply(sts[0], x), lambda r: omg.solve_phase_symmetric(w, s, r),
                            f, None, 1e-8, 200)
    assert abs(it - it_o) <= 2 and it > 10
    assert np.allclose(hist[:10], hist_o[:10], rtol=1e-9, atol=0.0)
    assert hist[-1] <= 1e-8 and hist_o[-1] <= 1e-8
    assert np.linalg.norm(f - oop.apply(sts[0], u.reshape(n, n))) <= 1.05e-8 * np.linalg.norm(f) * (
        1.0 if method == "pcg" else 10.0)


def test_bpx_on_the_papers_multilevel_data(M):
    """The paper's test setting (Sec. 4.1: coefficient in [1/Re, 1] with Re = 1000,
    right-hand side 1, tol 1e-8) on its multi-level data: CG with the BPX network
    against the oracle, as in the test above (the oracle needs 29-33 iterations
    at 63^2-255^2)."""
    n = 255
    rng = np.random.default_rng(n)
    k = inputs.paper_mldata_k(n, rng)
    f = inputs.unit_rhs(n)
    sts = oop.level_stencils_div(k, (0.0, 0.0), num_levels(n))
    sv = symmetric_solver(M, 2, 1)
    sv.set_weights(M.bpx_weights(2))
    sv.setup_bpx(k.ravel().copy(), n, 1.0)
    u = np.zeros(n * n)
    st, it, hist = sv.solve_pcg(f.ravel().copy(), u, 1e-8, 200)
    assert st == M.OK
    w, s = omg.bpx_weights(2), omg.bpx_setup(sts, 1.0, 2)
    _, it_o, hist_o = ok.pcg(lambda x: oop.apply(sts[0], x), lambda r: omg.solve_phase_symmetric(w, s, r),
                             f, None, 1e-8, 200)
    assert abs(it - it_o) <= 2 and it <= 40
    assert np.allclose(hist[:10], hist_o[:10], rtol=1e-9, atol=0.0)
    assert np.linalg.norm(f - oop.apply(sts[0], u.reshape(n, n))) <= 1.05e-8 * np.linalg.norm(f)


def test_bpx_pcg_at_1023_needs_grid_independent_iterations(M):
    """At 1023^2 CG with the BPX network still needs about as many iterations
    as at 63^2 (the oracle needs 25-31 up to 511^2 on such fields); the
    solution is checked with the oracle's operator."""
    n = 1023
    rng, k, f, sts = spd_problem(n, 9)
    sv = symmetric_solver(M, 2, 1)
    sv.set_weights(M.bpx_weights(2))
    sv.setup_bpx(k.ravel().copy(), n, 1.0)
    u = np.zeros(n * n)
    st, it, hist = sv.solve_pcg(f.ravel().copy(), u, 1e-8, 200)
    assert st == M.OK and it <= 40
    assert np.linalg.norm(f - oop.apply(sts[0], u.reshape(n, n))) <= 1.05e-8 * np.linalg.norm(f)


def test_symmetric_errors_and_special_cases(M):
    n = 31
    rng, k, f, sts = spd_problem(n, 5)
    # two channels exist in FP64 only
    with pytest.raises(M.MGCNNError) as ei:
        M.Solver(2, 1, 1, precision="mixed_bf16", input_diag=False)
    assert ei.value.status == M.ERR_SIZE
    # the mode needs FP64, input_diag 0 and equal layer counts
    for kw in ({"precision": "mixed_bf16", "input_diag": False}, {"precision": "fp64", "input_diag": True}):
        sv = M.Solver(4, 1, 1, b=(0.0, 0.0), **kw)
        with pytest.raises(M.MGCNNError) as ei:
            sv.set_option(sv.OPT_SYMMETRIC, 1)
        assert ei.value.status == M.ERR_ARG
    sv = M.Solver(4, 2, 1, precision="fp64", input_diag=False, b=(0.0, 0.0))
    with pytest.raises(M.MGCNNError) as ei:
        sv.set_option(sv.OPT_SYMMETRIC, 1)
    assert ei.value.status == M.ERR_ARG
    # CG / MINRES / the BPX setup need the mode
    sv = M.Solver(4, 1, 1, precision="fp64", input_diag=False, b=(0.0, 0.0))
    sv.set_weights(M.bpx_weights(4))
    with pytest.raises(M.MGCNNError) as ei:
        sv.setup_bpx(k.ravel().copy(), n)
    assert ei.value.status == M.ERR_STATE
    sv.setup(k.ravel().copy(), n)
    with pytest.raises(M.MGCNNError) as ei:
        sv.solve_pcg(f.ravel().copy(), np.zeros(n * n), 1e-8, 10)
    assert ei.value.status == M.ERR_STATE
    # ... and a symmetric A
    sv = M.Solver(4, 1, 1, precision="fp64", input_diag=False, b=(1.0, 0.0))
    sv.set_option(sv.OPT_SYMMETRIC, 1)
    sv.set_weights(M.bpx_weights(4))
    sv.setup_bpx(k.ravel().copy(), n)
    with pytest.raises(M.MGCNNError) as ei:
        sv.solve_minres(f.ravel().copy(), np.zeros(n * n), 1e-8, 10)
    assert ei.value.status == M.ERR_ARG
    # training is not available in the mode
    sv = symmetric_solver(M, 4, 1)
    sv.set_weights(M.bpx_weights(4))
    with pytest.raises(M.MGCNNError) as ei:
        sv.loss_grad([(k.ravel().copy(), f.ravel().copy(), n)], 2)
    assert ei.value.status == M.ERR_STATE
    # f = 0: u = 0, no iterations; maxit reached: NOT_CONVERGED with maxit + 1 entries
    sv.setup_bpx(k.ravel().copy(), n)
    for solve in (sv.solve_pcg, sv.solve_minres):
        u = np.ones(n * n)
        st, it, hist = solve(np.zeros(n * n), u, 1e-8, 10)
        assert st == M.OK and it == 0 and not u.any()
        st, it, hist = solve(f.ravel().copy(), np.zeros(n * n), 1e-12, 3)
        assert st == M.NOT_CONVERGED and it == 3 and len(hist) == 4
