"""Training loss after K unrolled cycles and its hand-written FP64 gradient.

Sec. 3.4, Eq. loss: the network is trained without labels by minimising the
squared residual.  The loss here is the relative form after K stationary
cycles from u = 0 (the paper's own loss is the K = 1 case, unnormalised):

    r_0 = f,   r_{k+1} = r_k - A B_theta(r_k),    L = (1/N) sum_i ||r_K,i||^2 / ||f_i||^2 .

B_theta is the solve phase (Algorithm 3) with setup tensors s_l(theta) from the
setup phase (Algorithm 2); theta is every weight of both phases.

Reverse sweep (g_k = dL/dr_k):
    g_K = 2 r_K / (N ||f||^2)
    g_k = g_{k+1} + B^T(-A^T g_{k+1})
and each cycle contributes the weight gradient of <B_theta(r_k), -A^T g_{k+1}>.
Intermediates of B are recomputed per cycle from the stored r_k (per-cycle
checkpointing).
"""
from __future__ import annotations

import numpy as np

from . import convnet as cn
from . import mgcnn as mg
from .operator import Stencil, apply, apply_transpose

SOLVE_KEYS = ("w_in", "w_down", "w_up", "w_R", "w_P", "w_out")
SETUP_KEYS = ("sw_in", "sb_in", "sw", "sb", "sw_R")


def unrolled_residuals(weights: dict, stencils: list[Stencil], f: np.ndarray, K: int,
                       scale_by_diag: bool = True, input_diag: bool = False):
    """r_0 = f, r_{k+1} = r_k - A B r_k for k < K.  Returns (r list, setup tensors)."""
    s = mg.setup(weights, stencils, scale_by_diag)
    A = stencils[0]
    d_inv = (1.0 / A.aC) if input_diag else None
    rs = [f.copy()]
    for _ in range(K):
        rs.append(rs[-1] - apply(A, mg.solve_phase(weights, s, rs[-1], d_inv=d_inv)))
    return rs, s


def loss(weights: dict, problems: list, K: int, scale_by_diag: bool = True, input_diag: bool = False) -> float:
    """L = (1/N) sum_i ||r_K,i||^2 / ||f_i||^2 over problems [(stencils, f), ...]."""
    total = 0.0
    for stencils, f in problems:
        rs, _ = unrolled_residuals(weights, stencils, f, K, scale_by_diag, input_diag)
        total += float(np.sum(rs[-1] ** 2) / np.sum(f ** 2))
    return total / len(problems)


def _resnet_layer_backward(xbar, x_in, s_l, W, gW, sbar_l):
    """y = x + K(s * x).  Given y_bar, return x_bar; accumulate dK and ds."""
    z = s_l * x_in
    t = cn.conv_same_adjoint(xbar, W)           # K^T y_bar
    gW += cn.conv_same_wgrad(xbar, z)
    sbar_l += x_in * t
    return xbar + s_l * t


def solve_phase_backward(weights: dict, s: list[np.ndarray], r: np.ndarray, ebar: np.ndarray,
                         grads: dict, sbar: list[np.ndarray], d_inv: np.ndarray | None = None) -> np.ndarray:
    """Adjoint of e = B r (Algorithm 3, on D^{-1} r when d_inv is given) at input r
    for output adjoint e_bar.

    Returns r_bar = B^T e_bar; adds the weight gradients into `grads` and the
    setup-tensor gradients into `sbar`.
    """
    keep = {}
    mg.solve_phase(weights, s, r, keep, d_inv=d_inv)
    L = len(s)
    sizes = [t.shape[1] for t in s]
    nu_d = weights["w_down"].shape[0]
    nu_u = weights["w_up"].shape[0]
    # e = W_out * x_fin[0]
    grads["w_out"] += cn.conv_same_wgrad(ebar[None], keep["x_fin"][0])
    xbar_fin = [None] * L
    xbar_fin[0] = cn.conv_same_adjoint(ebar[None], weights["w_out"])
    xbar_down = [np.zeros_like(keep["x_down"][l]) for l in range(L)]
    # up loop in reverse: l = 1..L (0-based 0..L-1)
    for l in range(L):
        xb = xbar_fin[l]
        for i in reversed(range(nu_u)):
            xb = _resnet_layer_backward(xb, keep["up_in"][l][i], s[l], weights["w_up"][i],
                                        grads["w_up"][i], sbar[l])
        # pre-up state = x_down[l] (+ TCNN(x_fin[l+1]) when l < L-1)
        xbar_down[l] += xb
        if l < L - 1:
            xbar_fin[l + 1] = cn.rcnn(xb, weights["w_P"])          # TCNN^T = RCNN, same array
            grads["w_P"] += cn.tcnn_wgrad(keep["x_fin"][l + 1], xb)
    # down loop in reverse: l = L..1
    rbar = None
    for l in reversed(range(L)):
        xb = xbar_down[l]
        for i in reversed(range(nu_d)):
            xb = _resnet_layer_backward(xb, keep["down_in"][l][i], s[l], weights["w_down"][i],
                                        grads["w_down"][i], sbar[l])
        if l > 0:
            # x0[l] = RCNN(x_down[l-1])
            xbar_down[l - 1] += cn.tcnn(xb, weights["w_R"], sizes[l - 1])  # RCNN^T = TCNN
            grads["w_R"] += cn.rcnn_wgrad(xb, keep["x_down"][l - 1])
        else:
            grads["w_in"] += cn.conv_same_wgrad(xb, keep["rin"][None])
            rbar = cn.conv_same_adjoint(xb, weights["w_in"])[0]
            if d_inv is not None:
                rbar = rbar * d_inv
    return rbar


def setup_backward(weights: dict, stencils: list[Stencil], sbar: list[np.ndarray], grads: dict,
                   scale_by_diag: bool = True) -> None:
    """Adjoint of Algorithm 2: from dL/ds_l to the setup weights."""
    keep = {}
    mg.setup(weights, stencils, scale_by_diag, keep)
    L = len(stencils)
    sizes = [st.n for st in stencils]
    cbar = [np.zeros_like(c) for c in keep["c"]]
    for l in reversed(range(L)):
        mode = int(scale_by_diag)
        if mode == 1:
            zb = sbar[l] / stencils[l].aC
        elif mode == 2:
            zb = sbar[l] * (stencils[0].n + 1.0) ** 2 / (stencils[l].n + 1.0) ** 2
        else:
            zb = sbar[l].copy()
        for i in reversed(range(mg.SETUP_LAYERS)):
            t = keep["t"][l][i]
            dpre = zb * (1.0 - t * t)
            grads["sw"][i] += cn.conv_same_wgrad(dpre, keep["z"][l][i])
            grads["sb"][i] += dpre.sum(axis=(1, 2))
            zb = zb + cn.conv_same_adjoint(dpre, weights["sw"][i])
        cbar[l] += zb
        if l > 0:
            # c_l = RCNN_setup(c_{l-1})
            cbar[l - 1] += cn.tcnn(cbar[l], weights["sw_R"], sizes[l - 1])
            grads["sw_R"] += cn.rcnn_wgrad(cbar[l], keep["c"][l - 1])
    grads["sw_in"] += cn.conv_same_wgrad(cbar[0], keep["feat"])
    grads["sb_in"] += cbar[0].sum(axis=(1, 2))


def loss_and_grad(weights: dict, problems: list, K: int, scale_by_diag: bool = True, input_diag: bool = False):
    """Loss and its gradient with respect to every weight (dict of arrays like `weights`)."""
    grads = {k: np.zeros_like(v) for k, v in weights.items()}
    N = len(problems)
    total = 0.0
    for stencils, f in problems:
        A = stencils[0]
        d_inv = (1.0 / A.aC) if input_diag else None
        rs, s = unrolled_residuals(weights, stencils, f, K, scale_by_diag, input_diag)
        fn2 = float(np.sum(f * f))
        total += float(np.sum(rs[-1] ** 2)) / fn2
        g = 2.0 * rs[-1] / (N * fn2)
        sbar = [np.zeros_like(t) for t in s]
        for k in reversed(range(K)):
            ebar = -apply_transpose(A, g)
            g = g + solve_phase_backward(weights, s, rs[k], ebar, grads, sbar, d_inv)
        setup_backward(weights, stencils, sbar, grads, scale_by_diag)
    return total / N, grads
