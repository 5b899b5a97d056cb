"""Pins for the oracle's hand-written FP64 adjoint of the K-cycle loss (Sec. 3.4, Eq. loss).

Checked against central finite differences of the oracle's own loss
(eps = 1e-6 max(1, |theta|), relative error <= 1e-6), against PyTorch CPU
autograd of an independent rendering, and by the dot-product test for B^T.
"""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

from oracle import adjoint as adj
from oracle import mgcnn as mg
from oracle import operator as op
from oracle.grid import num_levels
from paper_2312_11093_gb300 import inputs


def _problems(sizes, seed):
    rng = np.random.default_rng(seed)
    out = []
    for n in sizes:
        k = inputs.lognormal_k(n, 0.1, rng)
        f = inputs.normal_rhs(n, rng)
        out.append((op.level_stencils_div(k, (1.0, 0.5), num_levels(n)), f))
    return out


def test_dot_product_transpose():
    (sts, f), = _problems([15], 1)
    rng = np.random.default_rng(2)
    w = mg.random_weights(4, 1, 1, rng)
    s = mg.setup(w, sts)
    v, wv = rng.standard_normal(f.shape), rng.standard_normal(f.shape)
    grads = {k: np.zeros_like(a) for k, a in w.items()}
    sbar = [np.zeros_like(t) for t in s]
    btw = adj.solve_phase_backward(w, s, v, wv, grads, sbar)
    lhs = np.sum(mg.solve_phase(w, s, v) * wv)
    assert abs(lhs - np.sum(v * btw)) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("scale_by_diag,input_diag", [(1, False), (0, True), (2, True)])
def test_central_differences(scale_by_diag, input_diag):
    probs = _problems([7, 15], 3)
    rng = np.random.default_rng(4)
    w = mg.random_weights(3, 1, 2, rng, scale=0.5)
    K = 2
    kw = dict(scale_by_diag=scale_by_diag, input_diag=input_diag)
    L0, g = adj.loss_and_grad(w, probs, K, **kw)
    assert np.isclose(L0, adj.loss(w, probs, K, **kw), rtol=1e-13)
    checked = 0
    for key in w:
        flat = w[key].reshape(-1)
        for idx in rng.choice(flat.size, size=min(3, flat.size), replace=False):
            eps = 1e-6 * max(1.0, abs(flat[idx]))
            old = flat[idx]
            flat[idx] = old + eps
            lp = adj.loss(w, probs, K, **kw)
            flat[idx] = old - eps
            lm = adj.loss(w, probs, K, **kw)
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            an = g[key].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(abs(fd), 1e-3 * abs(L0)), (key, idx, fd, an)
            checked += 1
    assert checked >= 25


def _torch_loss(wt, probs, K, input_diag=False, setup_scale=1):
    total = 0.0
    for sts, f in probs:
        aC = [torch.from_numpy(st.aC) for st in sts]
        feat = torch.from_numpy(mg.setup_features(sts[0]))[None]
        c = F.conv2d(feat, wt["sw_in"], wt["sb_in"], padding=1)
        s = []
        for l in range(len(sts)):
            z = c
            for i in range(4):
                z = torch.tanh(F.conv2d(z, wt["sw"][i], wt["sb"][i], padding=1)) + z
            if setup_scale == 1:
                s.append(z / aC[l])
            elif setup_scale == 2:
                s.append(z * 4.0 ** l)
            else:
                s.append(z)
            c = F.conv2d(c, wt["sw_R"], stride=2)
        A = sts[0]
        coef = [torch.from_numpy(a) for a in (A.aC, A.aW, A.aE, A.aS, A.aN)]

        def applyA(u):
            up = F.pad(u, (1, 1, 1, 1))
            return (coef[0] * u + coef[1] * up[1:-1, :-2] + coef[2] * up[1:-1, 2:]
                    + coef[3] * up[:-2, 1:-1] + coef[4] * up[2:, 1:-1])

        def B(r):
            L = len(s)
            x = [None] * L
            rin = r / aC[0] if input_diag else r
            x[0] = F.conv2d(rin[None, None], wt["w_in"], padding=1)
            for l in range(L):
                for i in range(wt["w_down"].shape[0]):
                    x[l] = x[l] + F.conv2d(s[l] * x[l], wt["w_down"][i], padding=1)
                if l < L - 1:
                    x[l + 1] = F.conv2d(x[l], wt["w_R"], stride=2)
            for l in reversed(range(L)):
                for i in range(wt["w_up"].shape[0]):
                    x[l] = x[l] + F.conv2d(s[l] * x[l], wt["w_up"][i], padding=1)
                if l > 0:
                    x[l - 1] = x[l - 1] + F.conv_transpose2d(x[l], wt["w_P"], stride=2)
            return F.conv2d(x[0], wt["w_out"], padding=1)[0, 0]

        ft = torch.from_numpy(f)
        r = ft.clone()
        for _ in range(K):
            r = r - applyA(B(r))
        total = total + (r * r).sum() / (ft * ft).sum()
    return total / len(probs)


@pytest.mark.parametrize("setup_scale,input_diag", [(1, False), (0, True), (2, True)])
def test_against_torch_autograd(setup_scale, input_diag):
    probs = _problems([15, 31], 5)
    w = mg.random_weights(4, 2, 1, np.random.default_rng(6), scale=0.5)
    K = 3
    L0, g = adj.loss_and_grad(w, probs, K, scale_by_diag=setup_scale, input_diag=input_diag)
    wt = {k: torch.tensor(v, requires_grad=True) for k, v in w.items()}
    Lt = _torch_loss(wt, probs, K, input_diag, setup_scale)
    Lt.backward()
    assert np.isclose(L0, Lt.item(), rtol=1e-12)
    for k in w:
        gt = wt[k].grad.numpy()
        assert np.linalg.norm(g[k] - gt) <= 1e-9 * max(np.linalg.norm(gt), 1e-30), k
