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
# weights trained on the paper's own test family (PAPER_SCHEDULE, workload "paper")
PAPER_WEIGHTS = os.path.join(HERE, "weights", "mgcnn_c8_paper_problem.npy")


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
                 setup_out: float = 0.01, mg_transfers: bool = False) -> np.ndarray:
    """Random initial weights, uniform with PyTorch's default fan-in bound.

    The output layer is shrunk (out_scale) and the setup network starts near zero
    (its input layer and biases times setup_out), so the setup tensors, and with
    them every s-scaled path of the solve phase, start small: the initial solve
    network is its unscaled skip/transfer paths, A B has O(1) entries with the
    normalised input, and the unrolled cycles start from a loss near 1 at every
    training size, also when the setup tensors carry the per-level factor
    (h_l/h_1)^2.

    mg_transfers: start RCNN and TCNN from the classical transfers on every
    channel (full weighting scaled to sum 4 -- the ratio of neighbouring levels'
    diagonals, which the normalised input leaves to the network -- and bilinear
    interpolation), plus 0.1x the random weights."""
    F, S = mgcnn.FEATURES, mgcnn.SETUP_LAYERS

    def u(*shape, fan):
        b = 1.0 / np.sqrt(fan)
        return rng.uniform(-b, b, size=shape)
    w = {"w_in": u(C, 1, 3, 3, fan=9), "w_down": u(nu_d, C, C, 3, 3, fan=9 * C),
         "w_up": u(nu_u, C, C, 3, 3, fan=9 * C), "w_R": u(C, C, 3, 3, fan=9 * C),
         "w_P": u(C, C, 3, 3, fan=9 * C), "w_out": out_scale * u(1, C, 3, 3, fan=9 * C),
         "sw_in": setup_out * u(C, F, 3, 3, fan=9 * F), "sb_in": setup_out * u(C, fan=9 * F),
         "sw": u(S, C, C, 3, 3, fan=9 * C), "sb": setup_out * u(S, C, fan=9 * C), "sw_R": u(C, C, 3, 3, fan=9 * C)}
    if mg_transfers:
        stencil = np.outer([1.0, 2.0, 1.0], [1.0, 2.0, 1.0]) / 4.0
        w["w_R"] *= 0.1
        w["w_P"] *= 0.1
        for ch in range(C):
            w["w_R"][ch, ch] += stencil
            w["w_P"][ch, ch] += stencil
    return mgcnn.pack_weights(w, C, nu_d, nu_u)


def make_batch(step: int, sizes=(63, 127), per_size=32, corr_len: float = 0.1):
    """Fresh problems for one step: per_size (an int, or one count per size) problems
    of each size, GRF coefficients, white-noise right-hand sides."""
    rng = np.random.default_rng(1000 + step)
    counts = per_size if isinstance(per_size, (list, tuple)) else [per_size] * len(sizes)
    probs = []
    for n, m in zip(sizes, counts):
        for _ in range(m):
            k = inputs.lognormal_k(n, corr_len, rng)
            f = inputs.normal_rhs(n, rng)
            probs.append((np.ascontiguousarray(k.ravel()), np.ascontiguousarray(f.ravel()), n))
    return probs


PAPER_V = (float(np.sin(0.5)), float(np.cos(0.5)))


def make_paper_batch(step: int, sizes=(31, 63, 127, 255), per_size=(16, 8, 4, 2), corr_len: float = 0.0):
    """Fresh problems of the paper's own test family (Sec. 4.1: the non-divergence
    operator with white-noise coef in [1e-3, 1], mu = coef h, v = (sin 0.5, cos 0.5)),
    white-noise right-hand sides; the coefficient array is mu on the n^2 interior nodes."""
    rng = np.random.default_rng(2000 + step)
    counts = per_size if isinstance(per_size, (list, tuple)) else [per_size] * len(sizes)
    probs = []
    for n, m in zip(sizes, counts):
        for _ in range(m):
            mu = inputs.paper_white_noise_mu(n, rng)
            f = inputs.normal_rhs(n, rng)
            probs.append((np.ascontiguousarray(mu.ravel()), np.ascontiguousarray(f.ravel()), n))
    return probs


# Training schedule.  The 63^2 / 127^2 recipe alone (5-6 levels) gives weights
# that diverge on 9-11 levels, and continuing from them on larger grids starts
# from exploding losses.  Every batch therefore mixes the sizes of the paper's
# progressive schedule (Appendix A, Table training_settings: 31^2 ... 511^2, the
# batch halving as the size doubles): 16 x 63^2 + 8 x 127^2 + 4 x 255^2 + 2 x 511^2,
# K = 8, Adam at lr 1e-4, then 3e-5 (the paper decays its rate stepwise; at 1e-3
# the K-cycle loss of this mix blows up within the first hundred steps).
SCHEDULE = [((63, 127, 255, 511), (16, 8, 4, 2), 1500, 1e-4), ((63, 127, 255, 511), (16, 8, 4, 2), 500, 3e-5)]
# The paper's own test family (make_paper_batch): the sizes of its progressive
# schedule up to 255^2 in every batch, 1200 steps at lr 1e-4, then 300 at 3e-5.
PAPER_SCHEDULE = [((31, 63, 127, 255), (16, 8, 4, 2), 1200, 1e-4), ((31, 63, 127, 255), (16, 8, 4, 2), 300, 3e-5)]
# The recipe on 63^2 / 127^2 only (batch 64, 2000 steps, lr 1e-3).
RECIPE_63_127 = [((63, 127), (32, 32), 2000, 1e-3)]


def slow_modes(weights: np.ndarray, problems, iters: int = 30, C: int = 8, precision: str = "mixed_bf16",
               seed: int = 0):
    """For each problem (k, f, n): the dominant mode of the residual iteration
    r <- (I - A B) r of the current network (power iteration from a random start,
    normalised every step).  Unrolled-loss training with white-noise right-hand
    sides weighs each eigenmode of I - A B by about 1/N, so a single slow mode
    barely shows in the loss yet decides the asymptotic rate of Eq. 1."""
    rng = np.random.default_rng(seed)
    sv = mgcnn.Solver(C, 1, 1, precision=precision, b=(1.0, 0.5), input_diag=True)
    sv.set_weights(weights)
    modes = []
    for k, _, n in problems:
        sv.setup(k, n)
        r = rng.standard_normal(n * n)
        r /= np.linalg.norm(r)
        for _ in range(iters):
            e = sv.vcycle(r)
            r, _ = sv.residual(r, e)
            nr = np.linalg.norm(r)
            if not np.isfinite(nr) or nr == 0.0:
                break
            r /= nr
        modes.append(np.ascontiguousarray(r))
    sv.close()
    return modes


def train(steps: int | None = None, K: int = 8, lr: float | None = None, C: int = 8, seed: int = 0,
          log_every: int = 50, out: str | None = WEIGHTS, precision: str = "mixed_bf16", per_size=None,
          setup_scale: int = 0, mg_transfers: bool = True, schedule=None, snapshot_every: int = 25,
          spike: float = 50.0, max_restarts: int = 8, init: np.ndarray | None = None, hard_every: int = 0,
          hard_sizes=(63, 127, 255, 511), workload: str = "grf"):
    """Run the schedule (or a single phase when steps/lr/per_size are given) and
    return (weights, loss history).

    Safeguard against blow-ups: the K-cycle loss of a network whose cycle stops
    contracting on one problem grows like rho^K, and Adam does not come back from
    there.  Every snapshot_every steps the weights are copied to the host when the
    step's loss is finite and within `spike` x the median of the last 20 losses;
    a loss outside that band restores the last snapshot in a fresh context (fresh
    Adam moments) and halves the phase's learning rate.

    hard_every > 0: every hard_every steps draw one fresh training problem per
    size in hard_sizes and replace its right-hand side by the slowest residual
    mode of the current network (`slow_modes`); these problems join every batch
    until the next refresh, so the loss sees the mode that limits Eq. 1.
    init: start from these weights instead of the random initialisation.
    workload: "grf" (lognormal k, divergence form, b = (1, 0.5)) or "paper" (the
    paper's non-divergence test family, make_paper_batch)."""
    paper = workload == "paper"
    if paper and hard_every:
        raise ValueError("hard_every draws divergence-form problems: use it with the grf workload")
    batch_fn = make_paper_batch if paper else make_batch
    if schedule is None:
        schedule = SCHEDULE if steps is None else [((63, 127), per_size or (32, 32), steps, lr or 1e-3)]

    def fresh(weights):
        sv = mgcnn.Solver(C, 1, 1, precision=precision, b=PAPER_V if paper else (1.0, 0.5),
                          pde="nondiv" if paper else "div", scale_by_diag=setup_scale, input_diag=True)
        sv.set_weights(weights)
        return sv

    w0 = init if init is not None else init_weights(C, 1, 1, np.random.default_rng(seed), mg_transfers=mg_transfers)
    sv = fresh(w0)
    snap, snap_step = sv.get_weights(), 0
    hard = []
    hist = []
    t0 = time.time()
    step, restarts = 0, 0
    for sizes, counts, nsteps, plr in schedule:
        for _ in range(nsteps):
            if hard_every and step % hard_every == 0:
                base = batch_fn(500000 + step, hard_sizes, 1)
                modes = slow_modes(sv.get_weights(), base, C=C, precision=precision, seed=step)
                hard = [(k, v, n) for (k, _, n), v in zip(base, modes)]
            try:
                loss = sv.train_step(batch_fn(step, sizes, counts) + hard, K, plr)
            except mgcnn.MGCNNError as err:
                if err.status != mgcnn.ERR_NONFINITE:
                    raise
                loss = float("inf")
            recent = hist[-20:]
            bad = not np.isfinite(loss) or (len(recent) >= 5 and loss > spike * float(np.median(recent)))
            if bad:
                restarts += 1
                if restarts > max_restarts:
                    raise RuntimeError(f"loss blew up {restarts} times (last at step {step})")
                sv.close()
                sv = fresh(snap)
                plr *= 0.5
                print(json.dumps({"step": step, "restart_from": snap_step, "loss": loss, "lr": plr}), flush=True)
                step += 1
                continue
            hist.append(loss)
            if step % snapshot_every == 0:
                snap, snap_step = sv.get_weights(), step
            if step % log_every == 0:
                print(json.dumps({"step": step, "sizes": list(sizes), "loss": loss, "lr": plr,
                                  "elapsed_s": round(time.time() - t0, 1)}), flush=True)
            step += 1
    w = sv.get_weights()
    sv.close()
    if out:
        os.makedirs(os.path.dirname(out), exist_ok=True)
        np.save(out, w)
    return w, hist


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    ap.add_argument("--workload", default="grf", choices=["grf", "paper"],
                    help="grf: the lognormal divergence-form family (SCHEDULE); paper: the paper's own "
                         "non-divergence test family (PAPER_SCHEDULE)")
    args = ap.parse_args()
    if args.workload == "paper":
        train(schedule=PAPER_SCHEDULE, workload="paper", out=args.out or PAPER_WEIGHTS)
    else:
        train(out=args.out or WEIGHTS)
