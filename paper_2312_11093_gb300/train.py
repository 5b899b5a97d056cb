"""Training the MGCNN solver with the library's hand-written adjoint.

`MGCNNLoss` exposes the K-cycle residual loss (Sec. 3.4, Eq. loss, unrolled
over K stationary cycles) as a torch.autograd.Function whose backward is the
CUDA adjoint of libmgcnn.so.  `train()` runs the training recipe of the
8-channel network: batches of 64 problems (32 on 63x63 grids, 32 on 127x127),
k = exp(g) with g a Gaussian random field (squared-exponential covariance,
correlation length 0.1, sigma 1), f ~ N(0, 1), b = (1, 0.5), K = 8, FP32,
Adam with lr 1e-3, a fresh batch every step (Sec. 3.4: "generated randomly
for every batch").
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
if os.path.dirname(HERE) not in sys.path:
    sys.path.insert(0, os.path.dirname(HERE))

from paper_2312_11093_gb300 import inputs, mgcnn  # noqa: E402

WEIGHTS = os.path.join(HERE, "weights", "mgcnn_c8_trained.npy")


def _autograd():
    import torch

    class MGCNNLoss(torch.autograd.Function):
        """loss = MGCNNLoss.apply(weights, solver, problems, K): weights is a float64
        tensor holding the weight blob; backward returns dL/dweights from the CUDA adjoint."""

        @staticmethod
        def forward(ctx, weights, solver, problems, K):
            solver.set_weights(np.ascontiguousarray(weights.detach().cpu().numpy(), dtype=np.float64))
            loss, grad = solver.loss_grad(problems, K, want_grad=True)
            ctx.save_for_backward(torch.from_numpy(grad).to(weights.device))
            return torch.tensor(loss, dtype=torch.float64, device=weights.device)

        @staticmethod
        def backward(ctx, gout):
            (grad,) = ctx.saved_tensors
            return gout * grad, None, None, None

    return MGCNNLoss


def init_weights(C: int, nu_d: int, nu_u: int, rng: np.random.Generator, out_scale: float = 0.1,
                 setup_out: float = 0.01) -> np.ndarray:
    """Random initial weights, uniform with PyTorch's default fan-in bound.

    The output layer is shrunk (out_scale) and the setup network starts near zero
    (its input layer and biases times setup_out), so the setup tensors, and with
    them every s-scaled path of the solve phase, start small: the initial solve
    network is its unscaled skip/transfer paths, A B has O(1) entries with the
    normalised input, and the unrolled cycles start from a loss near 1 at every
    training size, also when the setup tensors carry the per-level factor
    (h_l/h_1)^2."""
    F, S = mgcnn.FEATURES, mgcnn.SETUP_LAYERS

    def u(*shape, fan):
        b = 1.0 / np.sqrt(fan)
        return rng.uniform(-b, b, size=shape)
    w = {"w_in": u(C, 1, 3, 3, fan=9), "w_down": u(nu_d, C, C, 3, 3, fan=9 * C),
         "w_up": u(nu_u, C, C, 3, 3, fan=9 * C), "w_R": u(C, C, 3, 3, fan=9 * C),
         "w_P": u(C, C, 3, 3, fan=9 * C), "w_out": out_scale * u(1, C, 3, 3, fan=9 * C),
         "sw_in": setup_out * u(C, F, 3, 3, fan=9 * F), "sb_in": setup_out * u(C, fan=9 * F),
         "sw": u(S, C, C, 3, 3, fan=9 * C), "sb": setup_out * u(S, C, fan=9 * C), "sw_R": u(C, C, 3, 3, fan=9 * C)}
    return mgcnn.pack_weights(w, C, nu_d, nu_u)


def make_batch(step: int, sizes=(63, 127), per_size: int = 32, corr_len: float = 0.1):
    rng = np.random.default_rng(1000 + step)
    probs = []
    for n in sizes:
        for _ in range(per_size):
            k = inputs.lognormal_k(n, corr_len, rng)
            f = inputs.normal_rhs(n, rng)
            probs.append((np.ascontiguousarray(k.ravel()), np.ascontiguousarray(f.ravel()), n))
    return probs


def train(steps: int = 2000, K: int = 8, lr: float = 1e-3, C: int = 8, seed: int = 0, log_every: int = 50,
          out: str | None = WEIGHTS, precision: str = "mixed_bf16", per_size: int = 32, setup_scale: int = 2):
    sv = mgcnn.Solver(C, 1, 1, precision=precision, b=(1.0, 0.5), scale_by_diag=setup_scale, input_diag=True)
    sv.set_weights(init_weights(C, 1, 1, np.random.default_rng(seed)))
    hist = []
    t0 = time.time()
    for s in range(steps):
        loss = sv.train_step(make_batch(s, per_size=per_size), K, lr)
        if not np.isfinite(loss):
            raise RuntimeError(f"loss became non-finite at step {s}")
        hist.append(loss)
        if s % log_every == 0 or s == steps - 1:
            print(json.dumps({"step": s, "loss": loss, "elapsed_s": round(time.time() - t0, 1)}), flush=True)
    w = sv.get_weights()
    if out:
        os.makedirs(os.path.dirname(out), exist_ok=True)
        np.save(out, w)
    return w, hist


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--K", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--per-size", type=int, default=32)
    ap.add_argument("--out", default=WEIGHTS)
    args = ap.parse_args()
    train(args.steps, args.K, args.lr, per_size=args.per_size, out=args.out)
