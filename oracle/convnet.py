"""3x3 convolution primitives in PyTorch (cross-correlation) semantics, FP64.

Sec. 2.4 uses 3x3 kernels for every layer: same-size convolutions (zero padding
1, Sec. 2.5's zero-padding rule), the stride-2 restriction RCNN and the
transposed convolution TCNN (Eq. transconv, y = K^T x).  The strided layers use
no padding, which makes odd sizes nest: n_c = (n - 1)/2 and coarse node I sits
on fine node 2I + 1 (0-based interior indices).

Tensors are [C, n, n].  Weights:  same/RCNN  W[c_out, c_in, a, b];
TCNN (PyTorch conv_transpose2d layout)  W[c_in, c_out, a, b].
Tap (a, b) reads the source pixel at offset (a - 1, b - 1) for the same
convolution and (2J + a, 2I + b) for RCNN.
"""
from __future__ import annotations

import numpy as np


def conv_same(x: np.ndarray, W: np.ndarray, bias: np.ndarray | None = None) -> np.ndarray:
    """y[co, p] = sum_ci sum_ab W[co, ci, a, b] x[ci, p + (a-1, b-1)] (+ bias[co])."""
    C_in, n, m = x.shape
    C_out = W.shape[0]
    assert W.shape == (C_out, C_in, 3, 3)
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1)))
    y = np.zeros((C_out, n, m))
    for a in range(3):
        for b in range(3):
            y += np.tensordot(W[:, :, a, b], xp[:, a:a + n, b:b + m], axes=([1], [0]))
    if bias is not None:
        y += bias[:, None, None]
    return y


def conv_same_adjoint(ybar: np.ndarray, W: np.ndarray) -> np.ndarray:
    """x_bar[ci, q] = sum_co sum_ab W[co, ci, a, b] y_bar[co, q - (a-1, b-1)] (zero outside)."""
    C_out, n, m = ybar.shape
    C_in = W.shape[1]
    yp = np.pad(ybar, ((0, 0), (1, 1), (1, 1)))
    x = np.zeros((C_in, n, m))
    for a in range(3):
        for b in range(3):
            x += np.tensordot(W[:, :, a, b].T, yp[:, 2 - a:2 - a + n, 2 - b:2 - b + m], axes=([1], [0]))
    return x


def conv_same_wgrad(ybar: np.ndarray, x: np.ndarray) -> np.ndarray:
    """dW[co, ci, a, b] = sum_p y_bar[co, p] x[ci, p + (a-1, b-1)]."""
    C_out, n, m = ybar.shape
    C_in = x.shape[0]
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1)))
    g = np.zeros((C_out, C_in, 3, 3))
    for a in range(3):
        for b in range(3):
            g[:, :, a, b] = np.tensordot(ybar, xp[:, a:a + n, b:b + m], axes=([1, 2], [1, 2]))
    return g


def rcnn(x: np.ndarray, W: np.ndarray) -> np.ndarray:
    """Stride-2 restriction: y[co, J, I] = sum_ci sum_ab W[co, ci, a, b] x[ci, 2J + a, 2I + b]."""
    C_in, n, _ = x.shape
    nc = (n - 1) // 2
    y = np.zeros((W.shape[0], nc, nc))
    for a in range(3):
        for b in range(3):
            y += np.tensordot(W[:, :, a, b], x[:, a:a + 2 * nc - 1:2, b:b + 2 * nc - 1:2], axes=([1], [0]))
    return y


def tcnn(x: np.ndarray, W: np.ndarray, n_fine: int) -> np.ndarray:
    """Stride-2 transposed convolution: y[co, 2J + a, 2I + b] += sum_ci W[ci, co, a, b] x[ci, J, I]."""
    C_in, nc, _ = x.shape
    assert n_fine == 2 * nc + 1
    y = np.zeros((W.shape[1], n_fine, n_fine))
    for a in range(3):
        for b in range(3):
            y[:, a:a + 2 * nc - 1:2, b:b + 2 * nc - 1:2] += np.tensordot(W[:, :, a, b].T, x, axes=([1], [0]))
    return y


def rcnn_wgrad(ybar: np.ndarray, x: np.ndarray) -> np.ndarray:
    """dW[co, ci, a, b] = sum_JI y_bar[co, J, I] x[ci, 2J + a, 2I + b]  (for y = rcnn(x, W))."""
    C_out, nc, _ = ybar.shape
    g = np.zeros((C_out, x.shape[0], 3, 3))
    for a in range(3):
        for b in range(3):
            g[:, :, a, b] = np.tensordot(ybar, x[:, a:a + 2 * nc - 1:2, b:b + 2 * nc - 1:2], axes=([1, 2], [1, 2]))
    return g


def tcnn_wgrad(x: np.ndarray, ybar: np.ndarray) -> np.ndarray:
    """dW[ci, co, a, b] = sum_JI x[ci, J, I] y_bar[co, 2J + a, 2I + b]  (for y = tcnn(x, W))."""
    C_in, nc, _ = x.shape
    g = np.zeros((C_in, ybar.shape[0], 3, 3))
    for a in range(3):
        for b in range(3):
            g[:, :, a, b] = np.tensordot(x, ybar[:, a:a + 2 * nc - 1:2, b:b + 2 * nc - 1:2], axes=([1, 2], [1, 2]))
    return g
