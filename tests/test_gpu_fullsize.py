"""Full-size (4095^2) checks in the launch configuration the benchmark times.

The oracle cannot run a 4095^2 V-cycle in seconds, so the network is checked
through properties that hold at any size (linearity in the right-hand side,
Sec. 3.1 P2) and through the oracle's own FP64 residual of the final iterate;
the operator on every level and the residual are compared entry by entry.
"""
import numpy as np
import pytest
import torch

from oracle import operator as oop
from oracle.grid import level_sizes, num_levels
from paper_2312_11093_gb300 import inputs

pytestmark = pytest.mark.gpu
N_FULL = 4095


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2312_11093_gb300 import build
    build.build()
    from paper_2312_11093_gb300 import mgcnn
    mgcnn.load()
    return mgcnn


@pytest.fixture(scope="module")
def field():
    """The roofline workload: channelised binary k in {1, 1e3} (GRF corr. 0.02,
    70th percentile), b = (1, 0.5), f ~ N(0, 1)."""
    rng = np.random.default_rng(4)
    k = inputs.channelised_k(N_FULL, rng, 0.02, 0.70, 1.0, 1e3)
    f = inputs.normal_rhs(N_FULL, rng)
    return k, f


def _relerr(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def _weights(M):
    import os
    path = os.path.join(os.path.dirname(M.__file__), "weights", "mgcnn_c8_trained.npy")
    if os.path.exists(path):
        return np.load(path)
    from paper_2312_11093_gb300.train import init_weights
    return init_weights(8, 1, 1, np.random.default_rng(3), out_scale=0.05)


def test_operator_and_residual_full_size(M, field):
    k, f = field
    sv = M.Solver(8, 1, 1, precision="mixed_bf16")
    sv.set_weights(_weights(M))
    kd = torch.from_numpy(k.ravel()).cuda()
    sv.setup(kd, N_FULL)
    sts = oop.level_stencils_div(k, (1.0, 0.5), num_levels(N_FULL))
    for l, (st, nl) in enumerate(zip(sts, level_sizes(N_FULL))):
        got = sv.get_operator(l, nl).reshape(5, nl, nl)
        for g, r in zip(got, [st.aC, st.aW, st.aE, st.aS, st.aN]):
            assert np.max(np.abs(g - r)) <= 1e-14 * np.max(np.abs(st.aC)), l
    u = np.random.default_rng(5).standard_normal((N_FULL, N_FULL)) * 1e-6
    r, n2 = sv.residual(f.ravel().copy(), u.ravel().copy())
    rref = oop.residual(sts[0], f, u)
    assert np.max(np.abs(r - rref.ravel())) <= 1e-13 * np.max(np.abs(rref))
    assert abs(n2 - np.sum(rref ** 2)) <= 1e-12 * np.sum(rref ** 2)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed_bf16", 3e-2)])
def test_vcycle_linearity_full_size(M, field, precision, tol):
    """B(a r1 + b r2) = a B r1 + b B r2 at 4095^2 (exact in FP64 up to rounding;
    the BF16 network rounds each input differently, bounded like its error)."""
    k, f = field
    sv = M.Solver(8, 1, 1, precision=precision)
    sv.set_weights(_weights(M))
    sv.setup(torch.from_numpy(k.ravel()).cuda(), N_FULL)
    g = np.random.default_rng(6).standard_normal(N_FULL * N_FULL)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = lambda: torch.empty(N_FULL * N_FULL, dtype=torch.float64, device="cuda")
    e1 = sv.vcycle(dev(f.ravel()), out()).cpu().numpy()
    e2 = sv.vcycle(dev(g), out()).cpu().numpy()
    e12 = sv.vcycle(dev(2.0 * f.ravel() - 0.5 * g), out()).cpu().numpy()
    assert _relerr(e12, 2.0 * e1 - 0.5 * e2) <= tol


def test_mixed_solve_full_size_residual_in_fp64(M):
    """Mixed-precision solve at 4095^2 -- the benchmark's launch configuration: the
    8-channel network that is GMG V(1,0) on the fused level kernels, a lognormal GRF
    field (corr. 0.05, b = 10(cos t, sin t)); its convergence test is FP64, and the
    oracle recomputes the final residual independently."""
    rng = np.random.default_rng(2)
    t = rng.uniform(0.0, 2.0 * np.pi)
    k = inputs.lognormal_k(N_FULL, 0.05, rng)
    f = inputs.normal_rhs(N_FULL, rng)
    b = (10.0 * np.cos(t), 10.0 * np.sin(t))
    sv = M.Solver(8, 1, 1, precision="mixed_bf16", b=b)
    sv.set_weights(M.gmg_v10_weights())
    sv.setup_gmg(torch.from_numpy(k.ravel()).cuda(), N_FULL, 0.8)
    u = torch.zeros(N_FULL * N_FULL, dtype=torch.float64, device="cuda")
    st, it, hist = sv.solve(torch.from_numpy(f.ravel()).cuda(), u, 1e-6, 150)
    assert st == M.OK
    st_ = oop.stencil_div(k, b)
    rel = np.linalg.norm(oop.residual(st_, f, u.cpu().numpy().reshape(N_FULL, N_FULL))) / np.linalg.norm(f)
    # f - A u cancels: each entry carries rounding of order eps * sum_o |a_o u_o|,
    # a visible fraction of the entry at relres 1e-6, so two FP64 evaluations of
    # the same iterate agree to about 1e-2 in norm
    assert abs(rel - hist[-1]) <= 1e-2 * hist[-1]
    assert rel <= 1.01e-6
