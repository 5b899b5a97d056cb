"""Closed-form pins for the composition of the oracle's setup phase (Sec. 3.2,
Algorithm 2): coef_1 = reChannelCNN(features); on every level the setup output
is NonLinearResNet(coef_l) -- four layers z <- tanh(K_i z + b_i) + z (Eq.
resnet_nonlinear) -- followed by the level scaling; the next level's
coefficient is the setup RCNN applied to coef_l itself (not to the setup
output).

The expected values below come from special cases whose answer is known
without running the algorithm:
* with every setup-layer kernel zero, each layer adds tanh(b_i), so the
  output is coef + sum_i tanh(b_i) per channel;
* a reChannel kernel with only a centre tap and a setup RCNN that is a
  one-hot tap make coef_l a pointwise linear map of the features sampled on a
  known sub-lattice (coarse pixel (J, I) reads fine pixel (2J + a, 2I + b));
* centre-tap-only setup layers make the NonLinearResNet a per-pixel map of a
  C-vector (four matrix-vector products), so it commutes with sampling.
A mistake in which tensor is restricted, in where the level scaling sits or in
the layer count changes these values (tests/test_oracle_mutations_all.py
plants each one).
"""
import numpy as np
import pytest

from oracle import mgcnn as mg
from oracle import operator as op
from oracle.grid import num_levels, spacing
from paper_2312_11093_gb300 import inputs

C = 8
LAYERS = 4   # Sec. 3.2: the setup NonLinearResNet has four layers


def _stencils(n, seed, b=(1.0, 0.5)):
    k = inputs.lognormal_k(n, 0.1, np.random.default_rng(seed))
    return op.level_stencils_div(k, b, num_levels(n))


def _centre_only(w, key, rng, scale):
    """Replace a [.., C, Cin, 3, 3] kernel by one with a random centre tap only
    (the setup layers: LAYERS of them, each with a random bias)."""
    shape = w[key].shape if key != "sw" else (LAYERS, C, C, 3, 3)
    if key == "sw":
        w["sb"] = rng.uniform(-1.0, 1.0, (LAYERS, C))
    out = np.zeros(shape)
    out[..., 1, 1] = rng.standard_normal(shape[:-2]) * scale
    w[key] = out


def _pointwise_nl(w, c):
    """The NonLinearResNet of centre-tap-only layers at one pixel: c is [C, ...]."""
    z = c
    for i in range(LAYERS):
        K = w["sw"][i][:, :, 1, 1]
        z = np.tanh(np.tensordot(K, z, axes=([1], [0])) + w["sb"][i].reshape((-1,) + (1,) * (z.ndim - 1))) + z
    return z


def _scale(mode, st, st0):
    if mode == 1:
        return 1.0 / st.aC
    if mode == 2:
        return (spacing(st.n) / spacing(st0.n)) ** 2
    return 1.0


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_zero_setup_kernels_add_tanh_of_the_biases(mode):
    """sw = 0, reChannel kernel 0, centred-delta setup RCNN: coef_l = sb_in on every
    level and every layer adds tanh(b_i), so setup_out_l = (sb_in + sum_i tanh(b_i))
    times the level scale -- the scale applied after the NonLinearResNet."""
    sts = _stencils(31, 1)
    rng = np.random.default_rng(2)
    w = mg.random_weights(C, 1, 1, rng)
    w["sw_in"] = np.zeros_like(w["sw_in"])
    w["sw"] = np.zeros((LAYERS, C, C, 3, 3))
    w["sb_in"] = rng.uniform(-2.0, 2.0, C)
    w["sb"] = rng.uniform(-1.5, 1.5, (LAYERS, C))
    w["sw_R"] = np.zeros((C, C, 3, 3))
    w["sw_R"][np.arange(C), np.arange(C), 1, 1] = 1.0
    s = mg.setup(w, sts, scale_by_diag=mode)
    per_channel = w["sb_in"] + np.tanh(w["sb"]).sum(axis=0)
    assert len(s) == len(sts)
    for st, sl in zip(sts, s):
        expect = per_channel[:, None, None] * _scale(mode, st, sts[0]) * np.ones((1, st.n, st.n))
        np.testing.assert_allclose(sl, expect, rtol=1e-14, atol=0)


def test_constant_features_and_centred_restriction_keep_coef():
    """Constant k, b = 0: the features are the same at every node ([-1/4] * 4 and
    log10(4 k)).  A centre-only reChannel kernel gives a constant coef_1, a
    centred-delta setup RCNN copies it to every level (coef_{l+1} = coef_l), and
    centre-only setup layers map it pointwise, so every level's output is the
    same constant vector (scale mode 0)."""
    n = 63
    kappa = 2.5
    sts = op.level_stencils_div(np.full((n + 2, n + 2), kappa), (0.0, 0.0), num_levels(n))
    rng = np.random.default_rng(4)
    w = mg.random_weights(C, 1, 1, rng)
    _centre_only(w, "sw_in", rng, 0.5)
    _centre_only(w, "sw", rng, 0.4)
    w["sw_R"] = np.zeros((C, C, 3, 3))
    w["sw_R"][np.arange(C), np.arange(C), 1, 1] = 1.0
    feat = np.array([-0.25, -0.25, -0.25, -0.25, np.log10(4.0 * kappa)])
    c1 = w["sw_in"][:, :, 1, 1] @ feat + w["sb_in"]
    keep = {}
    s = mg.setup(w, sts, scale_by_diag=0, keep=keep)
    expect = _pointwise_nl(w, c1)
    for l, (st, sl) in enumerate(zip(sts, s)):
        np.testing.assert_allclose(keep["c"][l], c1[:, None, None] * np.ones((1, st.n, st.n)), rtol=1e-13, atol=1e-14)
        np.testing.assert_allclose(sl, expect[:, None, None] * np.ones((1, st.n, st.n)), rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("tap", [(0, 2), (2, 1), (1, 1)])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_setup_rcnn_restricts_coef_not_the_setup_output(tap, mode):
    """A one-hot setup RCNN at tap (a, b) makes coef_{l+1}[J, I] = coef_l[2J + a, 2I + b];
    with centre-only reChannel and setup layers coef_1 is a pointwise linear map of
    the features and the NonLinearResNet a pointwise map phi, so
    setup_out_l = phi(coef_1 sampled on level l's sub-lattice) x the level scale.
    Restricting setup_out_{l} (= phi(coef_l)) instead would apply phi twice on
    level 2 and give a different value."""
    a, b = tap
    sts = _stencils(63, 5)
    rng = np.random.default_rng(6)
    w = mg.random_weights(C, 1, 1, rng)
    _centre_only(w, "sw_in", rng, 0.6)
    _centre_only(w, "sw", rng, 0.5)
    w["sb"] = rng.uniform(-0.8, 0.8, (LAYERS, C))
    w["sw_R"] = np.zeros((C, C, 3, 3))
    w["sw_R"][np.arange(C), np.arange(C), a, b] = 1.0
    feat = mg.setup_features(sts[0])
    c = np.tensordot(w["sw_in"][:, :, 1, 1], feat, axes=([1], [0])) + w["sb_in"][:, None, None]
    s = mg.setup(w, sts, scale_by_diag=mode)
    for l, st in enumerate(sts):
        if l > 0:
            nc = st.n
            c = c[:, a:a + 2 * nc - 1:2, b:b + 2 * nc - 1:2]
        assert c.shape[1:] == (st.n, st.n)
        expect = _pointwise_nl(w, c) * _scale(mode, st, sts[0])
        np.testing.assert_allclose(s[l], expect, rtol=1e-12, atol=1e-13 * np.abs(expect).max())
    # the two readings differ on level 2 by far more than rounding
    c1 = np.tensordot(w["sw_in"][:, :, 1, 1], feat, axes=([1], [0])) + w["sb_in"][:, None, None]
    n2 = sts[1].n
    wrong = _pointwise_nl(w, _pointwise_nl(w, c1)[:, a:a + 2 * n2 - 1:2, b:b + 2 * n2 - 1:2])
    right = _pointwise_nl(w, c1[:, a:a + 2 * n2 - 1:2, b:b + 2 * n2 - 1:2])
    assert np.abs(wrong - right).max() > 1e-2


def test_setup_output_is_scaled_after_the_nonlinear_resnet():
    """scale_by_diag = 1 divides NL(coef_l) by the level's a_C.  With centre-only
    layers NL is pointwise, so NL(coef_l) / a_C is known; NL(coef_l / a_C) -- the
    scaling moved in front of the tanh layers -- is a different tensor."""
    sts = _stencils(31, 9)
    rng = np.random.default_rng(10)
    w = mg.random_weights(C, 1, 1, rng)
    _centre_only(w, "sw_in", rng, 0.6)
    _centre_only(w, "sw", rng, 0.5)
    w["sw_R"] = np.zeros((C, C, 3, 3))
    w["sw_R"][np.arange(C), np.arange(C), 1, 1] = 1.0
    feat = mg.setup_features(sts[0])
    c = np.tensordot(w["sw_in"][:, :, 1, 1], feat, axes=([1], [0])) + w["sb_in"][:, None, None]
    s = mg.setup(w, sts, scale_by_diag=1)
    np.testing.assert_allclose(s[0], _pointwise_nl(w, c) / sts[0].aC, rtol=1e-12, atol=0)
    other = _pointwise_nl(w, c / sts[0].aC)
    assert np.abs(other - s[0]).max() > 1e-3 * np.abs(s[0]).max()
