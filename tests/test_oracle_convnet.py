"""Pins for the oracle's 3x3 convolution primitives (Sec. 2.4, Eqs. conv and transconv).

The oracle's layers must follow PyTorch semantics (the paper's framework):
they are checked against brute-force loops on tiny inputs, against PyTorch's
own CPU conv2d / conv_transpose2d, and against the transpose identities that
Eq. transconv states (TCNN = K^T of a strided CNN with the same weights).
"""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

from oracle import convnet as cn


def _brute_same(x, W):
    C_in, n, m = x.shape
    C_out = W.shape[0]
    y = np.zeros((C_out, n, m))
    for co in range(C_out):
        for j in range(n):
            for i in range(m):
                acc = 0.0
                for ci in range(C_in):
                    for a in range(3):
                        for b in range(3):
                            jj, ii = j + a - 1, i + b - 1
                            if 0 <= jj < n and 0 <= ii < m:
                                acc += W[co, ci, a, b] * x[ci, jj, ii]
                y[co, j, i] = acc
    return y


def _brute_rcnn(x, W):
    C_in, n, _ = x.shape
    nc = (n - 1) // 2
    y = np.zeros((W.shape[0], nc, nc))
    for co in range(W.shape[0]):
        for J in range(nc):
            for I in range(nc):
                y[co, J, I] = sum(W[co, ci, a, b] * x[ci, 2 * J + a, 2 * I + b]
                                  for ci in range(C_in) for a in range(3) for b in range(3))
    return y


def _brute_tcnn(x, W, n):
    C_in, nc, _ = x.shape
    y = np.zeros((W.shape[1], n, n))
    for ci in range(C_in):
        for co in range(W.shape[1]):
            for J in range(nc):
                for I in range(nc):
                    for a in range(3):
                        for b in range(3):
                            y[co, 2 * J + a, 2 * I + b] += W[ci, co, a, b] * x[ci, J, I]
    return y


@pytest.fixture
def rng():
    return np.random.default_rng(11)


def test_conv_same_brute_force(rng):
    x = rng.standard_normal((2, 5, 5))
    W = rng.standard_normal((3, 2, 3, 3))
    np.testing.assert_allclose(cn.conv_same(x, W), _brute_same(x, W), rtol=1e-13, atol=1e-13)


def test_strided_brute_force(rng):
    x = rng.standard_normal((2, 7, 7))
    W = rng.standard_normal((3, 2, 3, 3))
    np.testing.assert_allclose(cn.rcnn(x, W), _brute_rcnn(x, W), rtol=1e-13, atol=1e-13)
    xc = rng.standard_normal((2, 3, 3))
    Wt = rng.standard_normal((2, 3, 3, 3))
    np.testing.assert_allclose(cn.tcnn(xc, Wt, 7), _brute_tcnn(xc, Wt, 7), rtol=1e-13, atol=1e-13)


def test_against_pytorch(rng):
    x = rng.standard_normal((4, 15, 15))
    W = rng.standard_normal((5, 4, 3, 3))
    bias = rng.standard_normal(5)
    tx, tW = torch.from_numpy(x)[None], torch.from_numpy(W)
    ref = F.conv2d(tx, tW, torch.from_numpy(bias), padding=1)[0].numpy()
    np.testing.assert_allclose(cn.conv_same(x, W, bias), ref, rtol=1e-12, atol=1e-12)
    ref = F.conv2d(tx, tW, stride=2)[0].numpy()
    np.testing.assert_allclose(cn.rcnn(x, W), ref, rtol=1e-12, atol=1e-12)
    xc = rng.standard_normal((4, 7, 7))
    Wt = rng.standard_normal((4, 5, 3, 3))
    ref = F.conv_transpose2d(torch.from_numpy(xc)[None], torch.from_numpy(Wt), stride=2)[0].numpy()
    np.testing.assert_allclose(cn.tcnn(xc, Wt, 15), ref, rtol=1e-12, atol=1e-12)


def test_transpose_identity(rng):
    """<TCNN_W x, y> = <x, RCNN_W y> for the same weight array (Eq. transconv)."""
    C, n = 3, 15
    W = rng.standard_normal((C, C, 3, 3))
    x = rng.standard_normal((C, 7, 7))
    y = rng.standard_normal((C, n, n))
    lhs = np.sum(cn.tcnn(x, W, n) * y)
    rhs = np.sum(x * cn.rcnn(y, W))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_adjoints_and_weight_grads(rng):
    Ci, Co, n = 3, 4, 9
    x = rng.standard_normal((Ci, n, n))
    W = rng.standard_normal((Co, Ci, 3, 3))
    dW = rng.standard_normal((Co, Ci, 3, 3))
    yb = rng.standard_normal((Co, n, n))
    # <K x, y> = <x, K^T y>
    assert np.isclose(np.sum(cn.conv_same(x, W) * yb), np.sum(x * cn.conv_same_adjoint(yb, W)), rtol=1e-12)
    # d/dW <K_W x, y> along dW equals <dW, wgrad>
    assert np.isclose(np.sum(cn.conv_same(x, dW) * yb), np.sum(dW * cn.conv_same_wgrad(yb, x)), rtol=1e-12)
    ybc = rng.standard_normal((Co, 4, 4))
    assert np.isclose(np.sum(cn.rcnn(x, dW) * ybc), np.sum(dW * cn.rcnn_wgrad(ybc, x)), rtol=1e-12)
    xc = rng.standard_normal((Ci, 4, 4))
    dWt = rng.standard_normal((Ci, Co, 3, 3))
    assert np.isclose(np.sum(cn.tcnn(xc, dWt, n) * yb), np.sum(dWt * cn.tcnn_wgrad(xc, yb)), rtol=1e-12)
