"""Pins for the oracle's MGCNN setup / solve phases (Algorithms 2 and 3).

* P2 (Sec. 3.1): the solve phase is linear in the right-hand side.
* With the GMG-equivalent weights the solve phase reproduces classical GMG
  (Sec. 2.3) iterate for iterate, and the converged solution equals a dense
  direct solve.
* An independent PyTorch-CPU rendering of both algorithms (library conv
  routines, autograd-free) agrees with the oracle.
"""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

from oracle import gmg
from oracle import mgcnn as mg
from oracle import operator as op
from oracle.grid import num_levels
from paper_2312_11093_gb300 import inputs
from test_oracle_gmg import cfg0_problem


def _problem(n, seed, b=(1.0, 0.5)):
    rng = np.random.default_rng(seed)
    k = inputs.lognormal_k(n, 0.1, rng)
    f = inputs.normal_rhs(n, rng)
    return op.level_stencils_div(k, b, num_levels(n)), f


def test_linearity_in_rhs():
    sts, f = _problem(31, 2)
    rng = np.random.default_rng(3)
    w = mg.random_weights(8, 1, 1, rng)
    s = mg.setup(w, sts)
    g = rng.standard_normal(f.shape)
    lhs = mg.solve_phase(w, s, 2.5 * f - 0.75 * g)
    rhs = 2.5 * mg.solve_phase(w, s, f) - 0.75 * mg.solve_phase(w, s, g)
    assert np.linalg.norm(lhs - rhs) <= 1e-13 * np.linalg.norm(lhs)


def test_gmg_equivalence_cfg0():
    """Iterate-for-iterate equality with GMG V(2,2), omega = 0.8, 4 levels, tol 1e-10."""
    n, k, b, f = cfg0_problem()
    sts = op.level_stencils_div(k, b, num_levels(n))
    w = mg.gmg_equivalent_weights(2, 2)
    s = mg.gmg_equivalent_setup(sts, 0.8)
    u_m, it_m, hist_m, its_m = mg.stationary_solve(w, s, sts[0], f, None, 1e-10, 200)
    u_g, it_g, hist_g, its_g = gmg.stationary_solve(sts, f, None, 1e-10, 200, 2, 2, 0.8)
    assert it_m == it_g
    for a, c in zip(its_m[1:], its_g[1:]):
        assert np.linalg.norm(a - c) <= 1e-13 * np.linalg.norm(c)
    ustar = np.linalg.solve(op.dense_matrix(sts[0]), f.ravel()).reshape(n, n)
    assert np.linalg.norm(u_m - ustar) / np.linalg.norm(ustar) < 1e-7


def test_gmg_equivalence_other_sizes_and_sweeps():
    for n, nu1, nu2 in [(15, 1, 1), (63, 3, 2)]:
        sts, f = _problem(n, n, b=(-0.3, 2.0))
        w = mg.gmg_equivalent_weights(nu1, nu2)
        s = mg.gmg_equivalent_setup(sts, 0.7)
        r = f - op.apply(sts[0], np.zeros_like(f))
        e_m = mg.solve_phase(w, s, r)
        e_g = gmg.vcycle(sts, r, nu1, nu2, 0.7)
        assert np.linalg.norm(e_m - e_g) <= 1e-13 * np.linalg.norm(e_g)



@pytest.mark.parametrize("input_diag", [False, True])
def test_networks_with_level_weights_are_gmg_with_level_weights(input_diag):
    """A Jacobi weight per level (finest 0.8, in between 1.3, coarsest 1.0) in the
    setup tensors of the 13-channel V(2,1) network and of the 8-channel V(1,0)
    network gives GMG with the same weight on each level, iterate for iterate."""
    n = 63
    sts, f = _problem(n, 71, b=(2.0, -1.0))
    oms = gmg.level_omegas(len(sts), (0.8, 1.3, 1.0))
    assert oms[0] == 0.8 and oms[-1] == 1.0 and oms[1] == 1.3
    for w, s, nu in ((mg.gmg_equivalent_weights(2, 1), mg.gmg_equivalent_setup(sts, oms, input_diag), (2, 1)),
                     (mg.gmg_v10_weights(), mg.gmg_v10_setup(sts, oms, input_diag), (1, 0))):
        u_m, it_m, _, its_m = mg.stationary_solve(w, s, sts[0], f, None, 1e-9, 200, input_diag=input_diag)
        u_g, it_g, _, its_g = gmg.stationary_solve(sts, f, None, 1e-9, 200, *nu, oms)
        assert it_m == it_g < 200
        for a, c in zip(its_m[1:], its_g[1:]):
            assert np.linalg.norm(a - c) <= 1e-12 * np.linalg.norm(c)

def _torch_setup(w, sts, feat):
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a))
    c = F.conv2d(T(feat)[None], T(w["sw_in"]), T(w["sb_in"]), padding=1)
    outs = []
    for l, st in enumerate(sts):
        z = c
        for i in range(4):
            z = torch.tanh(F.conv2d(z, T(w["sw"][i]), T(w["sb"][i]), padding=1)) + z
        outs.append((z[0] / T(st.aC)).numpy())
        c = F.conv2d(c, T(w["sw_R"]), stride=2)
    return outs


def _torch_solve(w, s, r):
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a))
    L = len(s)
    x = [None] * L
    x[0] = F.conv2d(T(r)[None, None], T(w["w_in"]), padding=1)
    for l in range(L):
        for i in range(w["w_down"].shape[0]):
            x[l] = x[l] + F.conv2d(T(s[l])[None] * x[l], T(w["w_down"][i]), padding=1)
        if l < L - 1:
            x[l + 1] = F.conv2d(x[l], T(w["w_R"]), stride=2)
    for l in reversed(range(L)):
        for i in range(w["w_up"].shape[0]):
            x[l] = x[l] + F.conv2d(T(s[l])[None] * x[l], T(w["w_up"][i]), padding=1)
        if l > 0:
            x[l - 1] = x[l - 1] + F.conv_transpose2d(x[l], T(w["w_P"]), stride=2)
    return F.conv2d(x[0], T(w["w_out"]), padding=1)[0, 0].numpy()


def test_against_pytorch_rendering():
    sts, f = _problem(31, 7)
    w = mg.random_weights(8, 2, 1, np.random.default_rng(8))
    s = mg.setup(w, sts)
    ref = _torch_setup(w, sts, mg.setup_features(sts[0]))
    for a, c in zip(s, ref):
        np.testing.assert_allclose(a, c, rtol=1e-11, atol=0)
    e = mg.solve_phase(w, s, f)
    np.testing.assert_allclose(e, _torch_solve(w, s, f), rtol=1e-10, atol=1e-12 * np.abs(e).max())


def test_setup_features_are_scale_free():
    """Scaling k by a constant leaves the stencil-ratio features unchanged and shifts
    the log feature by log10 of the constant (b = 0)."""
    n = 15
    k = np.exp(np.random.default_rng(9).standard_normal((n + 2, n + 2)))
    f1 = mg.setup_features(op.stencil_div(k, (0, 0)))
    f2 = mg.setup_features(op.stencil_div(100 * k, (0, 0)))
    np.testing.assert_allclose(f1[:4], f2[:4], rtol=1e-13)
    np.testing.assert_allclose(f2[4] - f1[4], 2.0, rtol=1e-12)


@pytest.mark.parametrize("n", [7, 31, 127])
def test_setup_features_do_not_depend_on_the_grid(n):
    """For constant k the 5-point stencil is k/h^2 [-1 -1 4 -1 -1]: the ratio
    features are -1/4 and the log feature log10(h^2 a_C) = log10(4 k) at every
    grid size, so one set of setup weights serves every level and size."""
    kappa = 3.7
    f = mg.setup_features(op.stencil_div(np.full((n + 2, n + 2), kappa), (0, 0)))
    np.testing.assert_allclose(f[:4], -0.25, rtol=1e-13)
    np.testing.assert_allclose(f[4], np.log10(4.0 * kappa), rtol=1e-13)


def test_gmg_equivalence_with_input_normalisation():
    """With B r = Net(D^{-1} r) the finest-level setup tensors absorb the diagonal
    (s[F_J] = omega, s[F_G] = a_C) and the network is still GMG iterate for iterate."""
    n, k, b, f = cfg0_problem()
    sts = op.level_stencils_div(k, b, num_levels(n))
    w = mg.gmg_equivalent_weights(2, 2)
    s = mg.gmg_equivalent_setup(sts, 0.8, input_diag=True)
    u_m, it_m, _, its_m = mg.stationary_solve(w, s, sts[0], f, None, 1e-10, 200, input_diag=True)
    u_g, it_g, _, its_g = gmg.stationary_solve(sts, f, None, 1e-10, 200, 2, 2, 0.8)
    assert it_m == it_g
    for a, c in zip(its_m[1:], its_g[1:]):
        assert np.linalg.norm(a - c) <= 1e-13 * np.linalg.norm(c)


def test_linearity_with_input_normalisation():
    sts, f = _problem(31, 22)
    rng = np.random.default_rng(23)
    w = mg.random_weights(8, 1, 1, rng)
    s = mg.setup(w, sts, scale_by_diag=False)
    d = 1.0 / sts[0].aC
    g = rng.standard_normal(f.shape)
    lhs = mg.solve_phase(w, s, 3.0 * f + g, d_inv=d)
    rhs = 3.0 * mg.solve_phase(w, s, f, d_inv=d) + mg.solve_phase(w, s, g, d_inv=d)
    assert np.linalg.norm(lhs - rhs) <= 1e-13 * np.linalg.norm(lhs)


@pytest.mark.parametrize("input_diag", [False, True])
def test_v10_network_is_gmg_v10(input_diag):
    """The 8-channel, one-down-one-up network with the V(1,0) weights and setup
    tensors reproduces GMG V(1, 0) iterate for iterate (Sec. 2.3), including the
    normalised input B r = Net(D^{-1} r)."""
    for n, b in [(31, (1.0, 0.5)), (63, (-0.3, 2.0))]:
        sts, f = _problem(n, n + 7, b=b)
        w = mg.gmg_v10_weights()
        s = mg.gmg_v10_setup(sts, 0.8, input_diag=input_diag)
        u_m, it_m, _, its_m = mg.stationary_solve(w, s, sts[0], f, None, 1e-9, 200, input_diag=input_diag)
        u_g, it_g, _, its_g = gmg.stationary_solve(sts, f, None, 1e-9, 200, 1, 0, 0.8)
        assert it_m == it_g < 200
        for a, c in zip(its_m[1:], its_g[1:]):
            assert np.linalg.norm(a - c) <= 1e-12 * np.linalg.norm(c)
