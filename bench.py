"""Benchmark: MGCNN solves/s to relative residual 1e-6 at 4095^2 on GB300.

One step = one whole solve through the C ABI: mgcnn_setup (operators on every
level + setup network, or the analytic GMG-equivalent setup) followed by
mgcnn_solve from u = 0 to ||f - A u||/||f|| <= tol (FP64 residual, BF16
tensor-core V-cycle).  Inputs are resident in HBM when the timed region
starts; the working set (> 2 GB per cycle) is far larger than L2.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
instead (bounded sample, see `cpu_reference`).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2312_11093_gb300 import inputs  # noqa: E402

WEIGHTS_DIR = os.path.join(ROOT, "paper_2312_11093_gb300", "weights")
TRAINED = os.path.join(WEIGHTS_DIR, "mgcnn_c8_trained.npy")
METRIC = "solves/s to rel-res 1e-6 at 4095^2 (setup + solve), mixed BF16 MGCNN"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")


# --------------------------------------------------------------------------- workload
def make_workload(name: str, n: int, seed: int):
    """Seeded synthetic problem.  Returns (k nodal (n+2)^2, f n^2, b)."""
    rng = np.random.default_rng(seed)
    if name == "channelised":
        # binary k in {1, 1e3}: GRF (corr. length 0.02) above its 70th percentile is high-k
        k = inputs.channelised_k(n, rng, 0.02, 0.70, 1.0, 1e3)
        b = (1.0, 0.5)
    elif name == "grf":
        # lognormal GRF, corr. length 0.05, sigma 1; b = 10 (cos t, sin t), t ~ U(0, 2 pi)
        t = rng.uniform(0.0, 2.0 * math.pi)
        k = inputs.lognormal_k(n, 0.05, rng)
        b = (10.0 * math.cos(t), 10.0 * math.sin(t))
    else:
        raise ValueError(name)
    f = inputs.normal_rhs(n, rng)
    return np.ascontiguousarray(k.ravel()), np.ascontiguousarray(f.ravel()), b


def make_batch_workload(count: int, seed: int, sizes=(63, 127, 255, 511, 1023), families: int = 3):
    """Uneven batch: n ~ U{sizes}; k family ~ U{lognormal GRF (corr. 0.1, sigma 1),
    random blocks on a 16x16 board with log10 k ~ U(-2, 2), 16x16 checkerboard {1, 100}}
    (the first `families` of them); b = (1, 0.5); f ~ N(0, 1)."""
    rng = np.random.default_rng(seed)
    ns = [int(x) for x in rng.choice(sizes, size=count)]
    fam = rng.integers(0, families, size=count)
    ks, fs = [], []
    for n, fm in zip(ns, fam):
        if fm == 0:
            k = inputs.lognormal_k(n, 0.1, rng)
        elif fm == 1:
            k = inputs.random_blocks_k(n, rng)
        else:
            k = inputs.checkerboard_k(n)
        ks.append(np.ascontiguousarray(k.ravel()))
        fs.append(np.ascontiguousarray(inputs.normal_rhs(n, rng).ravel()))
    return ns, ks, fs


def network(kind: str):
    """(channels, nu_d, nu_u, blob, gmg) for the solve network: the trained 8-channel
    network, the 8-channel network that is GMG V(1,0) (same shape, same fused
    kernels, analytic setup tensors), or the 13-channel network that is GMG V(2,2)."""
    from paper_2312_11093_gb300 import mgcnn
    if kind == "gmg":
        return 13, 3, 2, mgcnn.gmg_weights(2, 2), True
    if kind == "gmg_v10":
        return 8, 1, 1, mgcnn.gmg_v10_weights(), True
    if not os.path.exists(TRAINED):
        raise SystemExit(f"no trained weights at {TRAINED}: train them (python -m paper_2312_11093_gb300.train) "
                         "or pick --net gmg_v10")
    blob = np.load(TRAINED)
    return 8, 1, 1, np.ascontiguousarray(blob, dtype=np.float64), False


def parse_omega(text: str):
    """'0.8' -> 0.8 (every level); '0.8,1.5,1.0' -> (finest, in between, coarsest)."""
    parts = [float(x) for x in str(text).split(",")]
    if len(parts) == 1:
        return parts[0]
    if len(parts) != 3:
        raise SystemExit("--omega takes one weight or three (finest,in-between,coarsest)")
    return tuple(parts)


def omega_record(omega, net: str):
    """The Jacobi weights of the analytic network, as the bench line records them."""
    if net not in ("gmg", "gmg_v10"):
        return None
    if isinstance(omega, tuple):
        return {"finest": omega[0], "in_between": omega[1], "coarsest": omega[2]}
    return omega


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=lambda: self.lines.extend(self.proc.stdout), daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            self.proc.wait(timeout=5)
            self.t.join(timeout=5)

    def summary(self):
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = max(smax, float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax or None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- roofline helpers
def algorithmic_bytes(kind: str, n: int, cp: int) -> float:
    """Bytes a launch of `kind` must move (each operand once): the finest level's
    kernel classes, or the fused kernels of a coarser level l ("down<l>",
    "up<l>", level size n_l = (n_{l-1} - 1) / 2)."""
    # per level unknown, BF16 with cp channels: down = x_in, s in; x_down and the
    # coarse x out (6.5 cp bytes); up = x_down, s and the coarse x_fin (hi + lo
    # parts) in; x_fin (hi + lo) out (9 cp bytes)
    down_l, up_l = 6.5 * cp, 9.0 * cp
    if kind == "tail":
        # the coarse tail kernel: down and up of every level from the first with
        # n_l <= 255 (level 1 at the earliest, at most 8 levels) to the coarsest
        sizes = [n]
        while sizes[-1] > 3:
            sizes.append((sizes[-1] - 1) // 2)
        tail = [nl for lvl, nl in enumerate(sizes) if lvl >= 1 and nl <= 255][-8:]
        return sum((down_l + up_l) * nl * nl for nl in tail)
    for pre in ("down", "up"):
        if kind.startswith(pre) and kind[len(pre):].isdigit() and int(kind[len(pre):]) > 0:
            nl = n
            for _ in range(int(kind[len(pre):])):
                nl = (nl - 1) // 2
            return (down_l if pre == "down" else up_l) * nl * nl
    N = n * n
    return {
        "residual": 60.0 * N,                    # u, f (FP64) + 5 stencil arrays in, FP32 r out
        "resnet": 6.0 * cp * N,                  # x, s in; y out (BF16, cp channels)
        "restrict": 2.0 * cp * N + 0.5 * cp * N,  # fine x in, coarse y out
        "prolong": 4.5 * cp * N,                 # fine y in/out, coarse x in
        "in": (4.0 + 2.0 * cp) * N,              # FP32 r in, BF16 x out
        "out": (2.0 * cp + 16.0) * N,            # BF16 x in, FP64 u in/out
        # fused level kernels at the finest level (8 channels):
        "down0": (4.0 + 2.0 * cp + 2.0 * cp + 0.5 * cp) * N,  # r (FP32), s in; x_down, coarse x out
        "up0": (2.0 * cp + 2.0 * cp + 1.0 * cp + 16.0) * N,   # x_down, s, coarse x (hi + lo), u in; u out
    }[kind]


# the sources whose hash identifies a kernel's build (its file and the headers that
# shape it)
KERNEL_SOURCE = {"residual_kernel": ("operator.cu", "ops.cuh", "fpconv.cuh"),
                 "down_kernel": ("mixed_fused.cu", "mixed.cuh", "tma.cuh", "ops.cuh"),
                 "up_kernel": ("mixed_fused.cu", "mixed.cuh", "tma.cuh", "ops.cuh")}


def kernel_source_hash(kernel: str) -> str:
    h = hashlib.sha1()
    for f in KERNEL_SOURCE[kernel]:
        h.update(open(os.path.join(ROOT, "paper_2312_11093_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:12]


def _profile_fields(kernel: str, workload: str):
    """The fields recorded for (kernel, workload) in the committed ncu summary, if
    it was taken on the current source of that kernel (source hash recorded beside
    the numbers)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path) or kernel not in KERNEL_SOURCE:
        return None
    h = kernel_source_hash(kernel)
    for ln in open(path):
        parts = ln.split()
        if len(parts) >= 4 and parts[0] == kernel and parts[1] == workload and parts[2] == h:
            return parts[3:]
    return None


def traffic_record(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary (current source only)."""
    f = _profile_fields(kernel, workload)
    return float(f[0]) if f else None


def sm_pipes_record(kernel: str, workload: str):
    """The SM-side limits of the same capture: busy fraction of the shared-memory
    data pipe and the fraction of cycles with an instruction issued."""
    f = _profile_fields(kernel, workload)
    if not f or len(f) < 3:
        return None
    return {"shared_memory_data_pipe_busy": float(f[1]), "issue_active": float(f[2]),
            "source": f"ncu --set full capture, profiles/{kernel}_{workload}.md"}


# --------------------------------------------------------------------------- CPU oracle
def _oracle_net(net, sts, omega=0.8):
    import oracle.gmg as ogmg
    import oracle.mgcnn as omg
    oms = ogmg.level_omegas(len(sts), omega)
    if net == "gmg":
        return omg.gmg_equivalent_weights(2, 2), omg.gmg_equivalent_setup(sts, oms), False
    if net == "gmg_v10":
        return omg.gmg_v10_weights(), omg.gmg_v10_setup(sts, oms), False
    w = unpack_blob(np.load(TRAINED), 8, 1, 1)
    return w, omg.setup(w, sts, scale_by_diag=False), True


def _oracle_solve(job):
    """One complete FP64 oracle solve in a worker process: input generation, then
    (timed) the operators on every level, the network's setup and the stationary
    iteration from u = 0 to ||f - A u|| / ||f|| <= tol.  Returns (seconds, cycles,
    final relative residual)."""
    workload, net, n, seed, tol, omega = job
    import oracle.mgcnn as omg
    import oracle.operator as oop
    from oracle.grid import num_levels
    k, f, b = make_workload(workload, n, seed)
    m = n + 2
    t0 = time.perf_counter()
    sts = oop.level_stencils_div(k.reshape(m, m), b, num_levels(n))
    w, s, diag = _oracle_net(net, sts, omega)
    _, iters, hist, _ = omg.stationary_solve(w, s, sts[0], f.reshape(n, n), None, tol, 300, input_diag=diag)
    return time.perf_counter() - t0, int(iters), float(hist[-1])


def host_cores() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def cpu_reference(workload: str, net: str, n_full: int = 4095, n_sample: int = 1023, count: int | None = None,
                  tol: float = 1e-6, seed0: int = 500, omega=0.8):
    """The FP64 oracle timed on this host's cores: `count` complete solves of the same
    workload family at n_sample^2 (each its own seeded problem), run one per core in
    spawned worker processes (one BLAS thread each), wall clock around all of them.
    Only the grid size is extrapolated: the rate at n_sample^2 is divided by
    (n_full / n_sample)^2, the oracle's cost per cycle being proportional to the
    unknown count and its cycle count (classical-GMG-like) nearly independent of n."""
    import multiprocessing as mp
    cores = host_cores()
    count = count or cores
    workers = max(1, min(count, cores))
    jobs = [(workload, net, n_sample, seed0 + i, tol, omega) for i in range(count)]
    saved = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    os.environ.update({v: "1" for v in saved})      # inherited by the workers only
    try:
        with mp.get_context("spawn").Pool(workers) as pool:
            pool.map(_oracle_solve, [(workload, net, 31, 1, tol, omega)] * workers)   # start-up, untimed
            t0 = time.perf_counter()
            res = pool.map(_oracle_solve, jobs, chunksize=1)
            wall = time.perf_counter() - t0
    finally:
        for v, old in saved.items():
            if old is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = old
    scale = (n_full / n_sample) ** 2
    per = [r[0] for r in res]
    cyc = [r[1] for r in res]
    value = count / wall / scale
    return {"value": value, "unit": "solves/s", "cores": workers, "kind": "oracle",
            "sample": (f"{count} complete FP64 numpy-oracle solves at {n_sample}^2 (setup + stationary iteration "
                       f"to {tol:g}, {min(cyc)}-{max(cyc)} cycles), {workers} at a time in worker processes with one "
                       f"BLAS thread each: {wall:.1f} s wall, {statistics.median(per):.1f} s median per solve; "
                       f"rate divided by {scale:.2f} = ({n_full}/{n_sample})^2 for {n_full}^2 (only the grid size "
                       f"is extrapolated)"),
            "measured": {"n": n_sample, "solves": count, "wall_s": wall, "cycles_median": statistics.median(cyc),
                         "solve_s_median": statistics.median(per), "relres_max": max(r[2] for r in res),
                         "solves_per_s_at_n": count / wall},
            "seconds_per_solve": 1.0 / value}


def unpack_blob(blob, C, nd, nu):
    from paper_2312_11093_gb300.mgcnn import FEATURES, SETUP_LAYERS, WEIGHT_ORDER
    shapes = {"w_in": (C, 1, 3, 3), "w_down": (nd, C, C, 3, 3), "w_up": (nu, C, C, 3, 3), "w_R": (C, C, 3, 3),
              "w_P": (C, C, 3, 3), "w_out": (1, C, 3, 3), "sw_in": (C, FEATURES, 3, 3), "sb_in": (C,),
              "sw": (SETUP_LAYERS, C, C, 3, 3), "sb": (SETUP_LAYERS, C), "sw_R": (C, C, 3, 3)}
    out, o = {}, 0
    for key in WEIGHT_ORDER:
        sz = int(np.prod(shapes[key]))
        out[key] = np.asarray(blob[o:o + sz]).reshape(shapes[key])
        o += sz
    return out


def pinned_copy(a: np.ndarray) -> np.ndarray:
    """A copy of `a` in page-locked host memory (numpy view of a pinned torch tensor)."""
    import torch
    t = torch.empty(a.size, dtype=torch.float64, pin_memory=True)
    out = t.numpy()
    out[:] = a.ravel()
    pinned_copy.keep.append(t)      # the tensor owns the memory
    return out


pinned_copy.keep = []


def pinned_zeros(count: int, dev) -> np.ndarray:
    """A zeroed page-locked host array, written by a copy from the device so that
    the device has reached its pages once (a host buffer's first transfers here
    run several times slower than later ones), like a buffer the caller reuses."""
    import torch
    t = torch.empty(count, dtype=torch.float64, pin_memory=True)
    t.copy_(torch.zeros(count, dtype=torch.float64, device=dev))
    pinned_copy.keep.append(t)
    return t.numpy()


# --------------------------------------------------------------------------- ranks
def max_over_ranks(ms: float, world: int, device) -> float:
    """The slowest rank's time: each rank (one GPU) runs its own replica of the
    workload, and the job is done when the last one is."""
    if world <= 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, solves_per_rank: int, ms: float) -> float:
    """Solves per second of the whole job: every rank finished solves_per_rank
    solves in (at most) ms milliseconds."""
    return world * solves_per_rank * 1e3 / ms


def rank_seed(base: int, rank: int) -> int:
    """Each rank draws its own problems (weak scaling, independent replicas)."""
    return base + 1000 * rank


# --------------------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--n", type=int, default=4095)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--net", default=None, choices=["trained", "gmg_v10", "gmg"])
    ap.add_argument("--workload", default=None, choices=["channelised", "grf", "batched256"])
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--maxit", type=int, default=100, help="cycle limit of the batched solves")
    ap.add_argument("--batch-solver", default="stationary", choices=["stationary", "krylov"],
                    help="solver of the batched workload line (the default line reports both)")
    ap.add_argument("--batch-restart", type=int, default=12, help="restart length of the batched FGMRES")
    ap.add_argument("--divtol", type=int, default=6,
                    help="batched solves stop a problem as diverged once ||r||/||f|| > 10^divtol (0: never)")
    ap.add_argument("--tile", type=int, default=-1, choices=[-1, 0, 1, 2, 3, 4, 5, 6, 7],
                    help="tile shape of the fused kernels: -1 autotuned, 0 16x32, 1 8x32, 2 16x16, 3 32x32, 4 24x32, "
                         "5 24x30 (up) + 24x32 (down), 6 32x30 (up) + 24x32 (down), 7 22x30 (up) + 24x32 (down)")
    ap.add_argument("--coarse-tail", type=int, default=-1,
                    help="largest grid side of the coarse levels run as one cooperative kernel "
                         "(0: a launch per level; -1: the library default)")
    ap.add_argument("--omega", default="0.8,1.5,1.0",
                    help="Jacobi weight(s) of the analytic networks: one for every level, or finest,in-between,coarsest")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched and channelised workloads reported beside the headline")
    ap.add_argument("--krylov", action="store_true", help="also time flexible GMRES with the network as preconditioner")
    ap.add_argument("--paper-table", action="store_true",
                    help="also record iterations against n (31..4095) on the paper's own test problem")
    ap.add_argument("--bpx", action="store_true",
                    help="also time CG with the symmetric network in its BPX form (same k field, b = 0, FP64, tol 1e-8)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    args.omega = parse_omega(args.omega)
    net = args.net or ("trained" if os.path.exists(TRAINED) else "gmg_v10")
    workload = args.workload or "grf"
    args.net_resolved = net

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        t0 = time.perf_counter()
        # each step is one complete oracle solve at 1023^2, run one per host core
        ns = min(args.n, 1023)
        base = cpu_reference(workload, net, args.n, n_sample=ns, count=args.steps, tol=args.tol, omega=args.omega)
        wall = base["measured"]["wall_s"]
        v = base["value"]
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
                          "steps": args.steps, "warmup": 0, "ms_per_step": 1e3 * wall / args.steps,
                          "step": f"one complete FP64 oracle solve at {ns}^2 (steps run concurrently, one per core)",
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic", "config": {"workload": f"{workload}_{args.n}", "net": net, "tol": args.tol,
                                     "omega": omega_record(args.omega, net)},
                          "cpu_baseline": base,
                          "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                          "wall_s": time.perf_counter() - t0}))
        return

    if workload == "batched256":
        return bench_batched(args, rank, world, local)

    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2312_11093_gb300 import mgcnn

    n, tol = args.n, args.tol
    C, nd, nu, blob, is_gmg = network(net)
    k_h, f_h, b = make_workload(workload, n, rank_seed(4, rank))
    dev = torch.device("cuda", local)
    k_d = torch.from_numpy(k_h).to(dev)
    f_d = torch.from_numpy(f_h).to(dev)
    u_d = torch.zeros(n * n, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def make_solver(prec):
        sv = mgcnn.Solver(C, nd, nu, precision=prec, b=b, stream=stream)
        sv.set_weights(blob)
        if args.tile >= 0:
            sv.set_option(sv.OPT_TILE, args.tile)
        if args.coarse_tail >= 0:
            sv.set_option(sv.OPT_COARSE_TAIL, args.coarse_tail)
        return sv

    def step(sv, k, f, u):
        if is_gmg:
            sv.setup_gmg(k, n, args.omega)
        else:
            sv.setup(k, n)
        if isinstance(u, np.ndarray):
            u[:] = 0.0
        else:
            u.zero_()
        return sv.solve(f, u, tol, 300)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    sv = make_solver("mixed_bf16")
    for _ in range(args.warmup):
        st, iters, hist = step(sv, k_d, f_d, u_d)
    launches0 = mgcnn.kernel_launches()
    with ClockSampler(local) as clk:
        barrier()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            st, iters, hist = step(sv, k_d, f_d, u_d)
        ev1.record(stream)
        barrier()
    launches = (mgcnn.kernel_launches() - launches0) // args.steps
    ms = ev0.elapsed_time(ev1)

    # Kernel timing for the roofline: the solve above is one device-side graph
    # per solve, which per-kernel events cannot bracket, so the same steps run
    # again with the library's event brackets on (host-driven cycle loop, every
    # kernel a plain launch on `stream`); the bracketed durations give each
    # kernel class's average launch time.
    sv.profile_read()
    sv.profile(True)
    barrier()
    pv0 = torch.cuda.Event(enable_timing=True)
    pv1 = torch.cuda.Event(enable_timing=True)
    pv0.record(stream)
    for _ in range(args.steps):
        step(sv, k_d, f_d, u_d)
    pv1.record(stream)
    barrier()
    prof = sv.profile_read()
    sv.profile(False)
    profiled_ms_per_step = pv0.elapsed_time(pv1) / args.steps
    ms = max_over_ranks(ms, world, dev)
    ms_per_step = ms / args.steps
    value = whole_job_rate(world, 1, ms_per_step)
    relres_mixed = float(hist[-1])
    u_mixed = u_d.clone()

    # solve-only time (setup excluded), as the paper splits them
    if is_gmg:
        sv.setup_gmg(k_d, n, args.omega)
    else:
        sv.setup(k_d, n)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    u_d.zero_()
    sv.solve(f_d, u_d, tol, 300)
    torch.cuda.synchronize(dev)
    solve_only_ms = (time.perf_counter() - t0) * 1e3

    # end to end through the C ABI with host buffers in pinned memory: the library
    # copies k, f and the initial guess in and the solution out inside the timed
    # region; each step gets its own zeroed initial guess, prepared beforehand
    # (as many steps as the device-timed region: single host-to-device copies
    # here occasionally take ten times their usual 0.7 ms, so few steps would
    # make the mean depend on whether one of them lands in the region)
    e2e_steps = max(3, args.steps)
    k_p, f_p = pinned_copy(k_h), pinned_copy(f_h)
    u_p = [pinned_zeros(n * n, dev) for _ in range(e2e_steps + 1)]

    def e2e_step(u):
        if is_gmg:
            sv.setup_gmg(k_p, n, args.omega)
        else:
            sv.setup(k_p, n)
        return sv.solve(f_p, u, tol, 300)
    e2e_step(u_p[-1])
    barrier()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        e2e_step(u_p[i])
    barrier()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / e2e_steps
    h2d = k_p.nbytes + f_p.nbytes + u_p[0].nbytes
    d2h = u_p[0].nbytes
    del k_p, f_p, u_p
    pinned_copy.keep.clear()

    # roofline of the dominant kernel (largest share of timed kernel time)
    cp = 8 if C <= 8 else 16
    dom = max(prof, key=lambda kk: prof[kk][0])
    dom_ms, dom_cnt = prof[dom]
    with open(PEAKS) as fh:
        peaks = json.load(fh)
    peak = float(peaks["hbm_gbs"])
    achieved = algorithmic_bytes(dom, n, cp) / (dom_ms / dom_cnt * 1e-3) / 1e9 if dom_cnt else None
    kname = {"residual": "residual_kernel", "resnet": "resnet_mma_kernel", "restrict": "rcnn_mma_kernel",
             "prolong": "tcnn_add_kernel16", "in": "in_kernel16", "out": "out_kernel16"}.get(
                 dom, "down_kernel" if dom.startswith("down") else "up_kernel")
    roofline = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "peak_source": "MEASURED_PEAKS.json hbm_gbs",
                "traffic": traffic_record(kname, f"{workload}_{n}"),
                "sm_pipes": sm_pipes_record(kname, f"{workload}_{n}"),
                "algorithmic_bytes_per_launch": algorithmic_bytes(dom, n, cp),
                "avg_launch_ms": dom_ms / dom_cnt if dom_cnt else None,
                "timing": "CUDA events around each finest-level launch, second timed pass of the same steps "
                          "(host-driven loop)",
                "profiled_ms_per_step": profiled_ms_per_step,
                "kernel_ms_per_step": {kk: round(v[0] / args.steps, 4) for kk, v in prof.items()},
                "launches_per_step": {kk: v[1] // args.steps for kk, v in prof.items()},
                "achieved_gbs": {kk: round(algorithmic_bytes(kk, n, cp) * v[1] / (v[0] * 1e-3) / 1e9, 1)
                                 for kk, v in prof.items() if v[1] and v[0] > 0}}

    result = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
              "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
              "config": {"workload": f"{workload}_{n}", "n": n, "tol": tol, "net": net, "omega": omega_record(args.omega, net),
                         "channels": C,
                         "down_layers": nd, "up_layers": nu, "b": list(b), "l2": "inputs larger than L2",
                         "tile": "autotuned" if args.tile < 0 else ["16x32", "8x32", "16x16", "32x32", "24x32", "24x30 up, 24x32 down",
                                                      "32x30 up, 24x32 down", "22x30 up, 24x32 down"][args.tile],
                         "parallelism": "replicas" if world > 1 else "single"},
              "iters": iters, "relres": relres_mixed, "solve_only_ms": solve_only_ms,
              "e2e": {"value": world * 1e3 / e2e_ms, "unit": "solves/s", "h2d_bytes_per_step": h2d,
                      "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
              "gpu_launches": int(launches), "roofline": roofline, "clocks": clk.summary()}

    if not args.no_fp64 and rank == 0:
        sv64 = make_solver("fp64")
        u64 = torch.zeros_like(u_d)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        st64, it64, h64 = step(sv64, k_d, f_d, u64)
        torch.cuda.synchronize(dev)
        t64 = time.perf_counter() - t0
        err = float(torch.linalg.norm(u_mixed - u64) / torch.linalg.norm(u64))
        result["fp64"] = {"value": 1.0 / t64, "unit": "solves/s", "iters": it64, "relres": float(h64[-1]),
                          "mixed_vs_fp64_rel_err": err, "mixed_speedup": value / world * t64}
        sv64.close()
    if not args.no_fp64 and rank == 0:
        # classical GMG comparator (Sec. 2.3): FP64 V(2,2), omega 0.8, same operators and tolerance;
        # beside it the same cycle with the per-level weights of the analytic network
        svg = make_solver("fp64")
        svg.setup_gmg(k_d, n, 0.8) if is_gmg else svg.setup(k_d, n)
        ug = torch.zeros_like(u_d)
        gmg_runs = [("gmg", 0.8, "V(2,2) weighted Jacobi 0.8, FP64")]
        if isinstance(args.omega, tuple):
            gmg_runs.append(("gmg_levels", args.omega, "V(2,2) weighted Jacobi %g finest, %g in between, %g coarsest, "
                                                       "FP64" % args.omega))
        for key, om, cycle in gmg_runs:
            try:                       # untimed first call: allocates the comparator's level buffers
                svg.gmg_solve(f_d, ug, tol, 2, 2, 2, om)
            except mgcnn.MGCNNError:
                pass
            ug.zero_()
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            try:
                stg, itg, hg = svg.gmg_solve(f_d, ug, tol, 300, 2, 2, om)
                tg = time.perf_counter() - t0
                result[key] = {"value": 1.0 / tg, "unit": "solves/s", "iters": itg, "relres": float(hg[-1]),
                               "converged": bool(stg == mgcnn.OK), "cycle": cycle}
            except mgcnn.MGCNNError as err:
                result[key] = {"converged": False, "error": str(err)[:120], "cycle": cycle}
        svg.close()
    if args.krylov and rank == 0:
        # the same network as the preconditioner of flexible GMRES(30), same tolerance
        uk = torch.zeros_like(u_d)

        def kstep():
            if is_gmg:
                sv.setup_gmg(k_d, n, args.omega)
            else:
                sv.setup(k_d, n)
            uk.zero_()
            return sv.solve_krylov(f_d, uk, tol, 300, 30)
        kstep()
        ksteps = max(2, min(args.steps, 5))
        kv0 = torch.cuda.Event(enable_timing=True)
        kv1 = torch.cuda.Event(enable_timing=True)
        barrier()
        kv0.record(stream)
        for _ in range(ksteps):
            kst, kit, kh = kstep()
        kv1.record(stream)
        barrier()
        kms = kv0.elapsed_time(kv1) / ksteps
        result["krylov"] = {"value": 1e3 / kms, "unit": "solves/s", "ms_per_step": kms, "iters": kit,
                            "relres": float(kh[-1]), "converged": bool(kst == mgcnn.OK),
                            "method": "flexible GMRES(30), the network as right preconditioner, setup + solve"}
    if args.bpx and rank == 0:
        # the symmetric variant: CG preconditioned by the BPX network on the symmetric
        # problem of the same coefficient field (b = 0), the paper's FP64 tolerance
        svb = mgcnn.Solver(2, 1, 1, precision="fp64", input_diag=False, b=(0.0, 0.0), stream=stream)
        svb.set_option(svb.OPT_SYMMETRIC, 1)
        svb.set_weights(mgcnn.bpx_weights(2))
        ub = torch.zeros_like(u_d)

        def bstep():
            svb.setup_bpx(k_d, n, 1.0)
            ub.zero_()
            return svb.solve_pcg(f_d, ub, 1e-8, 300)
        bstep()
        bsteps = max(2, min(args.steps, 3))
        bv0 = torch.cuda.Event(enable_timing=True)
        bv1 = torch.cuda.Event(enable_timing=True)
        barrier()
        bv0.record(stream)
        for _ in range(bsteps):
            bst, bit, bh = bstep()
        bv1.record(stream)
        barrier()
        bms = bv0.elapsed_time(bv1) / bsteps
        result["bpx_pcg"] = {"value": 1e3 / bms, "unit": "solves/s", "ms_per_step": bms, "iters": bit,
                             "relres": float(bh[-1]), "tol": 1e-8, "converged": bool(bst == mgcnn.OK),
                             "method": "CG, symmetric network as BPX preconditioner (C = 2, FP64), b = 0, "
                                       "setup + solve"}
        # MINRES with the same preconditioner (its history is the B-norm ratio)
        svb.setup_bpx(k_d, n, 1.0)
        ub.zero_()
        barrier()
        bv0.record(stream)
        mst, mit, mh = svb.solve_minres(f_d, ub, 1e-8, 300)
        bv1.record(stream)
        barrier()
        mms = bv0.elapsed_time(bv1)
        result["bpx_minres"] = {"value": 1e3 / mms, "unit": "solves/s", "ms_per_step": mms, "iters": mit,
                                "relres_bnorm": float(mh[-1]), "tol": 1e-8, "converged": bool(mst == mgcnn.OK),
                                "method": "MINRES, same preconditioner and problem, solve only"}
        svb.close()
    if args.paper_table and rank == 0:
        result["paper_problem"] = run_paper_table(dev, stream, mgcnn, args.omega)
    sv.close()
    if not args.no_extras and rank == 0 and world == 1:
        # the other two GPU workloads: the uneven batch over three coefficient
        # families, and the channelised field at 4095^2 (FP64 MGCNN, mixed MGCNN,
        # GMG, per-level achieved bandwidth)
        result["batched"] = run_batched(args, rank, world, dev, mgcnn, quiet=True)
        if args.batch_solver == "stationary":
            result["batched_krylov"] = run_batched(args, rank, world, dev, mgcnn, quiet=True, solver="krylov")
        result["channelised"] = run_channelised(n, dev, stream, mgcnn, C, nd, nu, blob, is_gmg, tol, args.omega)
        if is_gmg:
            result["high_contrast_krylov"] = run_high_contrast(n, dev, stream, mgcnn, C, nd, nu, blob, args.omega, tol)
        result["setup_network"] = time_setup_network(n, dev, stream, mgcnn, k_d, b)
    if not args.no_cpu and rank == 0 and world == 1:
        # one wave of complete oracle solves at 511^2, one per host core (about 15-30 s)
        result["cpu_baseline"] = cpu_reference(workload, net, n, n_sample=min(n, 511), tol=tol, omega=args.omega)
    if rank == 0:
        print(json.dumps(result))
    if world > 1:
        torch.distributed.destroy_process_group()


def bench_batched(args, rank, world, local):
    """The batched workload as the bench line itself (--workload batched256)."""
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2312_11093_gb300 import mgcnn
    res = run_batched(args, rank, world, torch.device("cuda", local), mgcnn, solver=args.batch_solver)
    if rank == 0:
        print(json.dumps(res))
    if world > 1:
        torch.distributed.destroy_process_group()


def run_batched(args, rank, world, dev, mgcnn, quiet=False, solver="stationary"):
    """256 uneven problems per step (setup + solve of the whole batch), tile shapes
    autotuned at setup; solves/s = problems that reach the tolerance / step time.
    solver "stationary": the stationary iteration, one CUDA graph launch per batch;
    "krylov": batched FGMRES(--batch-restart) with the network on the arithmetic
    coarse coefficient as preconditioner, at most 300 inner iterations."""
    krylov = solver == "krylov"
    import torch
    # all three coefficient families of the workload; a problem that does not reach
    # the tolerance within the cycle limit is a failure (counted, not a solve)
    net = args.net or ("trained" if os.path.exists(TRAINED) else "gmg_v10")
    C, nd, nu, blob, is_gmg = network(net)
    ns, ks, fs = make_batch_workload(args.batch, rank_seed(3, rank), families=3)
    fam = np.random.default_rng(rank_seed(3, rank))
    fam.choice((63, 127, 255, 511, 1023), size=args.batch)
    family = fam.integers(0, 3, size=args.batch)     # the same draws as make_batch_workload
    kd = [torch.from_numpy(k).to(dev) for k in ks]
    fd = [torch.from_numpy(f).to(dev) for f in fs]
    ud = [torch.zeros(n * n, dtype=torch.float64, device=dev) for n in ns]
    sv = mgcnn.Solver(C, nd, nu, precision="mixed_bf16")
    sv.set_weights(blob)
    if args.divtol > 0:
        # a problem whose ||r||/||f|| exceeds 10^divtol is stopped as diverged (a failure)
        sv.set_option(sv.OPT_DIVTOL, args.divtol)
    if krylov:
        sv.set_option(sv.OPT_COARSE_K, 1)
    maxit = 300 if krylov else args.maxit

    def solve(ff, uu):
        if krylov:
            return sv.solve_batched_krylov(ff, uu, args.tol, maxit, args.batch_restart, per_problem=True)
        return sv.solve_batched(ff, uu, args.tol, maxit, per_problem=True)

    def step(kk, ff, uu):
        sv.setup_batched(kk, ns, gmg_omega=args.omega if is_gmg else None)
        for u in uu:
            u.zero_() if hasattr(u, "zero_") else u.fill(0.0)
        return solve(ff, uu)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        st, iters, relres, stat = step(kd, fd, ud)
    launches0 = mgcnn.kernel_launches()
    stream = torch.cuda.current_stream(dev)
    steps = args.steps if not quiet else max(3, min(args.steps, 5))
    with ClockSampler(dev.index or 0) as clk:
        barrier()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        # the batch runs on the library's own streams and each call returns after
        # its work has finished, so events on this stream bracket all of it
        ev0.record(stream)
        for _ in range(steps):
            st, iters, relres, stat = step(kd, fd, ud)
        ev1.record(stream)
        barrier()
        ms = ev0.elapsed_time(ev1) / steps
    launches = (mgcnn.kernel_launches() - launches0) // steps
    ms = max_over_ranks(ms, world, dev)
    # end to end with pinned host buffers (zeroed initial guesses prepared beforehand)
    e2e_steps = 2
    kp = [pinned_copy(k) for k in ks]
    fp = [pinned_copy(f) for f in fs]
    ups = [[pinned_zeros(n * n, dev) for n in ns] for _ in range(e2e_steps + 1)]

    def e2e_step(uu):
        sv.setup_batched(kp, ns, gmg_omega=args.omega if is_gmg else None)
        return solve(fp, uu)
    e2e_step(ups[-1])
    barrier()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        e2e_step(ups[i])
    barrier()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / e2e_steps
    del kp, fp, ups
    pinned_copy.keep.clear()
    sv.close()
    unknowns = int(sum(n * n for n in ns))
    done = int((stat == 0).sum())   # problems that reached the tolerance count as solves
    res = {"metric": "solves/s to rel-res 1e-6, batch of uneven sizes (setup + solve)",
           "value": whole_job_rate(world, done, ms), "unit": "solves/s", "n_gpus": world, "steps": steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
           "config": {"workload": f"batched{args.batch}_63-1023_mixture", "problems": args.batch,
                      "unknowns": unknowns, "tol": args.tol, "net": net, "omega": omega_record(args.omega, net),
                      "maxit": maxit, "divtol": 10.0 ** args.divtol if args.divtol > 0 else None,
                      "solver": (f"flexible GMRES({args.batch_restart}), the network on the arithmetic coarse "
                                 "coefficient as preconditioner" if krylov else "stationary iteration"),
                      "l2": "inputs larger than L2", "parallelism": "replicas" if world > 1 else "single"},
           "iters_max": int(iters.max()), "iters_mean": float(iters.mean()),
           "converged": done, "failed": int((stat != 0).sum()),
           "failed_by_status": {nm: int((stat == code).sum()) for nm, code in
                                (("not_converged", mgcnn.NOT_CONVERGED), ("nonfinite", mgcnn.ERR_NONFINITE),
                                 ("diverged", mgcnn.ERR_DIVERGED))},
           "converged_by_family": {nm: f"{int(((stat == 0) & (family == i)).sum())}/{int((family == i).sum())}"
                                   for i, nm in enumerate(("grf", "blocks_1e4", "checkerboard_100"))},
           "relres_max_converged": float(relres[stat == 0].max()) if (stat == 0).any() else None,
           "e2e": {"value": world * done * 1e3 / e2e_ms, "unit": "solves/s",
                   "h2d_bytes_per_step": int(sum(k.nbytes for k in ks) + 2 * sum(f.nbytes for f in fs)),
                   "d2h_bytes_per_step": int(sum(f.nbytes for f in fs)), "ms_per_step": e2e_ms},
           "gpu_launches": int(launches), "clocks": clk.summary(), "roofline": None}
    return res


def run_paper_table(dev, stream, mgcnn, omega, sizes=(31, 63, 127, 255, 511, 1023, 2047, 4095), tol=1e-8):
    """Iterations against n on the paper's own test problem (Sec. 4.1: the
    non-divergence operator with white-noise coef in [1e-3, 1], v = (sin 0.5,
    cos 0.5), f = 1, tol 1e-8), the shape of its Table channels_double: classical
    GMG with the paper's GMG settings (weight 0.67, V(3,3), two levels fewer than
    MGCNN) and the mixed 8-channel V(1,0) network with per-level weights as the
    FGMRES(30) preconditioner (its stationary iteration diverges on this
    problem).  One draw per size; time from CUDA events, setup included."""
    import torch
    v = (math.sin(0.5), math.cos(0.5))
    rows = []
    for n in sizes:
        rng = np.random.default_rng(100 * n)
        mu = torch.from_numpy(np.ascontiguousarray(inputs.paper_white_noise_mu(n, rng).ravel())).to(dev)
        f = torch.from_numpy(np.ascontiguousarray(inputs.unit_rhs(n).ravel())).to(dev)
        u = torch.zeros(n * n, dtype=torch.float64, device=dev)
        L = int(round(math.log2(n + 1))) - 1
        row = {"n": n}
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        # classical GMG, the paper's settings
        sg = mgcnn.Solver(8, 1, 1, pde="nondiv", b=v, levels=max(1, L - 2), stream=stream)
        sg.set_weights(np.zeros(sg.weight_count))
        torch.cuda.synchronize(dev)
        e0.record(stream)
        sg.setup(mu, n)
        st, it, h = sg.gmg_solve(f, u, tol, 400, 3, 3, 0.67)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        row["gmg_v33"] = {"iters": it, "converged": bool(st == mgcnn.OK), "ms": e0.elapsed_time(e1)}
        sg.close()
        # the mixed network as the FGMRES preconditioner
        sk = mgcnn.Solver(8, 1, 1, precision="mixed_bf16", pde="nondiv", b=v, stream=stream)
        sk.set_weights(mgcnn.gmg_v10_weights())
        u.zero_()
        torch.cuda.synchronize(dev)
        e0.record(stream)
        sk.setup_gmg(mu, n, omega)
        st, it, h = sk.solve_krylov(f, u, tol, 400, 30)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        row["mgcnn_v10_fgmres"] = {"iters": it, "converged": bool(st == mgcnn.OK), "ms": e0.elapsed_time(e1)}
        sk.close()
        rows.append(row)
    return {"problem": "Sec. 4.1 test problem: non-divergence form, white-noise coef in [1e-3, 1], "
                       "v = (sin 0.5, cos 0.5), f = 1, one draw per size", "tol": tol, "rows": rows}


def time_setup_network(n, dev, stream, mgcnn, k_d, b, reps=5):
    """The learned network's setup phase (Algorithm 2: features, reChannel, four
    tanh ResNet layers and the setup RCNN per level, fused BF16 kernels) on the
    bench's coefficient field, with randomly initialised weights (no trained
    weights here): the cost the analytic GMG setup of the headline replaces."""
    import torch
    from paper_2312_11093_gb300.train import init_weights
    sv = mgcnn.Solver(8, 1, 1, precision="mixed_bf16", b=b, stream=stream)
    sv.set_weights(init_weights(8, 1, 1, np.random.default_rng(1)))
    sv.setup(k_d, n)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        sv.setup(k_d, n)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / reps
    sv.close()
    return {"ms_per_setup": ms, "reps": reps,
            "what": "mgcnn_setup at %d^2: operators on every level plus the setup network, random weights" % n}


def run_channelised(n, dev, stream, mgcnn, C, nd, nu, blob, is_gmg, tol, omega, maxit=60):
    """The channelised binary field (k in {1, 1e3}) at n^2: the mixed and the FP64
    MGCNN (same network) and classical GMG V(2,2), each from u = 0 for at most
    `maxit` cycles; per-level CUDA-event times and algorithmic GB/s of the mixed
    cycle's fused kernels over the first cycles."""
    import torch
    k_h, f_h, b = make_workload("channelised", n, 4)
    k_d = torch.from_numpy(k_h).to(dev)
    f_d = torch.from_numpy(f_h).to(dev)
    out = {"workload": f"channelised_{n}", "tol": tol, "maxit": maxit,
           "note": "relres is the last recorded ||r||/||f||; converged means it reached tol within maxit"}

    def run(prec):
        sv = mgcnn.Solver(C, nd, nu, precision=prec, b=b, stream=stream)
        sv.set_weights(blob)
        sv.setup_gmg(k_d, n, omega) if is_gmg else sv.setup(k_d, n)
        u = torch.zeros(n * n, dtype=torch.float64, device=dev)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        try:
            st, it, hist = sv.solve(f_d, u, tol, maxit)
            rec = {"iters": it, "relres": float(hist[-1]), "converged": bool(st == mgcnn.OK)}
        except mgcnn.MGCNNError as err:
            rec = {"converged": False, "error": str(err)[:100]}
        torch.cuda.synchronize(dev)
        rec["ms"] = (time.perf_counter() - t0) * 1e3
        return sv, rec

    sv, out["mixed"] = run("mixed_bf16")
    cp = 8 if C <= 8 else 16
    sv.profile_read()
    sv.profile(True)
    u = torch.zeros(n * n, dtype=torch.float64, device=dev)
    try:
        sv.solve(f_d, u, 0.0, 3)      # three cycles, every launch bracketed
    except mgcnn.MGCNNError:
        pass
    prof = sv.profile_read()
    sv.profile(False)
    sv.close()
    peak = float(json.load(open(PEAKS))["hbm_gbs"]) if os.path.exists(PEAKS) else None
    levels = {}
    for kk, (t, cnt) in prof.items():
        if cnt and t > 0:
            gbs = algorithmic_bytes(kk, n, cp) * cnt / (t * 1e-3) / 1e9
            levels[kk] = {"us_per_launch": round(1e3 * t / cnt, 2), "gbs": round(gbs, 1),
                          "frac_of_measured_hbm": round(gbs / peak, 3) if peak else None}
    out["mixed"]["per_level"] = levels
    sv64, out["fp64"] = run("fp64")
    ug = torch.zeros(n * n, dtype=torch.float64, device=dev)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    try:
        stg, itg, hg = sv64.gmg_solve(f_d, ug, tol, maxit, 2, 2, 0.8)
        out["gmg"] = {"iters": itg, "relres": float(hg[-1]), "converged": bool(stg == mgcnn.OK),
                      "cycle": "V(2,2) weighted Jacobi 0.8, FP64"}
    except mgcnn.MGCNNError as err:
        out["gmg"] = {"converged": False, "error": str(err)[:100], "cycle": "V(2,2) weighted Jacobi 0.8, FP64"}
    torch.cuda.synchronize(dev)
    out["gmg"]["ms"] = (time.perf_counter() - t0) * 1e3
    sv64.close()
    if is_gmg:
        # the mixed and the FP64 network with the arithmetic coarse coefficient as the
        # preconditioner of flexible GMRES(30), where every stationary solve diverges
        out["mixed_krylov"] = krylov_solve_record(mgcnn, n, k_d, f_d, b, dev, stream, C, nd, nu, blob, omega, tol)
        out["fp64_krylov"] = krylov_solve_record(mgcnn, n, k_d, f_d, b, dev, stream, C, nd, nu, blob, omega, tol,
                                                 precision="fp64", warm=False)
    return out


def krylov_solve_record(mgcnn, n, k_d, f_d, b, dev, stream, C, nd, nu, blob, omega, tol, maxit=300, restart=30,
                        precision="mixed_bf16", warm=True):
    """One setup + FGMRES(restart) solve with the analytic network (mixed or FP64)
    on the arithmetic coarse coefficient (MGCNN_OPT_COARSE_K = 1), timed with CUDA
    events (after one untimed run when `warm`); the final relative residual
    recomputed in FP64."""
    import torch
    sv = mgcnn.Solver(C, nd, nu, precision=precision, b=b, stream=stream)
    sv.set_weights(blob)
    sv.set_option(sv.OPT_COARSE_K, 1)
    u = torch.zeros(n * n, dtype=torch.float64, device=dev)

    def once():
        sv.setup_gmg(k_d, n, omega)
        u.zero_()
        return sv.solve_krylov(f_d, u, tol, maxit, restart)
    if warm:
        once()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    st, it, hist = once()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    r = torch.empty_like(u)
    _, rn2 = sv.residual(f_d, u, r)
    fn = float(torch.linalg.norm(f_d))
    sv.close()
    return {"iters": it, "converged": bool(st == mgcnn.OK), "ms": e0.elapsed_time(e1),
            "relres_fp64": float(np.sqrt(rn2)) / fn,
            "method": f"flexible GMRES({restart}), {'mixed' if precision == 'mixed_bf16' else 'FP64'} V(1,0) network "
                      "as right preconditioner, arithmetic coarse k, setup + solve"}


def run_high_contrast(n, dev, stream, mgcnn, C, nd, nu, blob, omega, tol):
    """Single solves at n^2 of the batched workload's two high-contrast families
    (random blocks with contrast 1e4, 16 x 16 checkerboard {1, 100}; b = (1, 0.5)),
    on which the stationary iteration diverges, by FGMRES(30) with the mixed network."""
    import torch
    rng = np.random.default_rng(5)
    fields = {"blocks_1e4": inputs.random_blocks_k(n, rng), "checkerboard_100": inputs.checkerboard_k(n)}
    f_d = torch.from_numpy(np.ascontiguousarray(inputs.normal_rhs(n, rng).ravel())).to(dev)
    out = {"n": n, "tol": tol, "b": [1.0, 0.5]}
    for name, k in fields.items():
        k_d = torch.from_numpy(np.ascontiguousarray(k.ravel())).to(dev)
        out[name] = krylov_solve_record(mgcnn, n, k_d, f_d, (1.0, 0.5), dev, stream, C, nd, nu, blob, omega, tol)
    return out


if __name__ == "__main__":
    main()
