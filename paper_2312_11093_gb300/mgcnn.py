"""ctypes binding of libmgcnn.so (C ABI in include/mgcnn.h).

Argument marshalling only: every computation runs in the CUDA library.  Arrays
may be numpy float64 arrays (host memory; the library copies them to and from
the device) or float64 torch tensors on the GPU (used in place).  If the
library has not been built the import of this module fails loudly: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_size_t, c_void_p

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libmgcnn.so")

OK, NOT_CONVERGED = 0, 1
ERR_ARG, ERR_SIZE, ERR_STATE, ERR_NOMEM, ERR_CUDA, ERR_NONFINITE, ERR_TIMEOUT, ERR_DIVERGED = -1, -2, -3, -4, -5, -6, -7, -8
PREC = {"fp64": 0, "mixed_bf16": 1}
PDE = {"div": 0, "nondiv": 1}
SETUP_LAYERS = 4
FEATURES = 5


class Config(ctypes.Structure):
    _fields_ = [("channels", c_int), ("down_layers", c_int), ("up_layers", c_int), ("precision", c_int),
                ("pde", c_int), ("scale_by_diag", c_int), ("input_diag", c_int), ("levels", c_int),
                ("bx", c_double), ("by", c_double)]


class MGCNNError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} [{status}]")
        self.status = status


_lib = None


def load() -> ctypes.CDLL:
    """Load libmgcnn.so (raises if it is missing -- build it with build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: the CUDA library must be built "
                          "(python -c 'import __graft_entry__ as g; g.build()')")
    L = ctypes.CDLL(LIB_PATH)
    dp = POINTER(c_double)
    sig = {
        "mgcnn_weight_count": (c_size_t, [POINTER(Config)]),
        "mgcnn_create": (c_int, [POINTER(Config), POINTER(c_void_p)]),
        "mgcnn_destroy": (None, [c_void_p]),
        "mgcnn_set_stream": (c_int, [c_void_p, c_void_p]),
        "mgcnn_set_weights": (c_int, [c_void_p, c_void_p, c_size_t]),
        "mgcnn_setup": (c_int, [c_void_p, c_void_p, c_int]),
        "mgcnn_setup_gmg": (c_int, [c_void_p, c_void_p, c_int, c_double]),
        "mgcnn_setup_gmg_levels": (c_int, [c_void_p, c_void_p, c_int, c_void_p]),
        "mgcnn_setup_tensor_count": (c_size_t, [c_void_p]),
        "mgcnn_set_setup_tensors": (c_int, [c_void_p, c_void_p, c_size_t]),
        "mgcnn_get_setup_tensors": (c_int, [c_void_p, c_void_p, c_size_t]),
        "mgcnn_get_operator": (c_int, [c_void_p, c_int, c_void_p, c_size_t]),
        "mgcnn_residual": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, dp]),
        "mgcnn_vcycle": (c_int, [c_void_p, c_void_p, c_void_p]),
        "mgcnn_solve": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_int, POINTER(c_int), c_void_p]),
        "mgcnn_loss_grad": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_int, dp, c_void_p]),
        "mgcnn_adam_step": (c_int, [c_void_p, c_void_p, c_double, c_double, c_double, c_double]),
        "mgcnn_train_step": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_int, c_double, dp, c_void_p]),
        "mgcnn_get_weights": (c_int, [c_void_p, c_void_p, c_size_t]),
        "mgcnn_set_option": (c_int, [c_void_p, c_int, c_int]),
        "mgcnn_gmg_solve": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_int, c_int, c_int, c_double,
                                    POINTER(c_int), c_void_p]),
        "mgcnn_gmg_solve_levels": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_int, c_int, c_int, c_void_p,
                                    POINTER(c_int), c_void_p]),
        "mgcnn_setup_batched": (c_int, [c_void_p, c_int, c_void_p, c_void_p]),
        "mgcnn_setup_batched_gmg": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_double]),
        "mgcnn_setup_batched_gmg_levels": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
        "mgcnn_solve_batched_krylov": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_double, c_int, c_int, c_void_p,
                                               c_void_p, c_void_p]),
        "mgcnn_check_wait_timeout": (c_int, [c_void_p]),
        "mgcnn_solve_krylov": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_int, c_int, c_void_p, c_void_p]),
        "mgcnn_setup_bpx": (c_int, [c_void_p, c_void_p, c_int, c_double]),
        "mgcnn_solve_pcg": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_int, POINTER(c_int), c_void_p]),
        "mgcnn_solve_minres": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_int, POINTER(c_int), c_void_p]),
        "mgcnn_solve_batched": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_double, c_int, c_void_p, c_void_p,
                                        c_void_p]),
        "mgcnn_kernel_launches": (ctypes.c_longlong, []),
        "mgcnn_profile": (c_int, [c_void_p, c_int]),
        "mgcnn_profile_read": (c_int, [c_void_p, c_void_p, c_void_p, c_int]),
        "mgcnn_status_string": (c_char_p, [c_int]),
        "mgcnn_last_error": (c_char_p, [c_void_p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _level_weights(omega) -> np.ndarray:
    """(finest, in between, coarsest) Jacobi weights as 3 contiguous doubles."""
    w = np.ascontiguousarray(np.asarray(omega, dtype=np.float64).ravel())
    if w.size != 3:
        raise ValueError("per-level Jacobi weights are (finest, in between, coarsest)")
    return w


def _ptr(a, n: int | None = None, writable: bool = False) -> int:
    """Raw pointer of a float64 numpy array or torch tensor (checked for dtype, layout, size)."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"] or (writable and not a.flags["WRITEABLE"]):
            raise TypeError("arrays must be C-contiguous float64")
        if n is not None and a.size != n:
            raise ValueError(f"array has {a.size} entries, expected {n}")
        return a.ctypes.data
    import torch
    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("tensors must be contiguous float64")
        if n is not None and a.numel() != n:
            raise ValueError(f"tensor has {a.numel()} entries, expected {n}")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def kernel_launches() -> int:
    """Kernels launched by libmgcnn.so in this process so far."""
    return int(load().mgcnn_kernel_launches())


def weight_count(channels: int, down_layers: int = 1, up_layers: int = 1) -> int:
    cfg = Config(channels, down_layers, up_layers, 0, 0, 0, 1, 0, 0.0, 0.0)
    return int(load().mgcnn_weight_count(ctypes.byref(cfg)))


WEIGHT_ORDER = ("w_in", "w_down", "w_up", "w_R", "w_P", "w_out", "sw_in", "sb_in", "sw", "sb", "sw_R")


def pack_weights(w: dict, channels: int, down_layers: int, up_layers: int) -> np.ndarray:
    """Flatten a dict of weight arrays into the blob layout of mgcnn_weight_count.

    Missing setup entries are zero (for runs that supply setup tensors directly)."""
    C, F, S = channels, FEATURES, SETUP_LAYERS
    shapes = {"w_in": (C, 1, 3, 3), "w_down": (down_layers, C, C, 3, 3), "w_up": (up_layers, C, C, 3, 3),
              "w_R": (C, C, 3, 3), "w_P": (C, C, 3, 3), "w_out": (1, C, 3, 3), "sw_in": (C, F, 3, 3),
              "sb_in": (C,), "sw": (S, C, C, 3, 3), "sb": (S, C), "sw_R": (C, C, 3, 3)}
    parts = []
    for k in WEIGHT_ORDER:
        a = np.asarray(w[k], dtype=np.float64) if k in w else np.zeros(shapes[k])
        if a.shape != shapes[k]:
            raise ValueError(f"{k}: shape {a.shape}, expected {shapes[k]}")
        parts.append(a.ravel())
    blob = np.ascontiguousarray(np.concatenate(parts))
    assert blob.size == weight_count(C, down_layers, up_layers)
    return blob


GMG_CHANNELS = 13


def gmg_weights(nu1: int = 2, nu2: int = 2) -> np.ndarray:
    """Weight blob (C = 13, nu_d = nu1 + 1, nu_u = nu2) whose solve phase, with the setup
    tensors of mgcnn_setup_gmg, is classical GMG V(nu1, nu2) (Sec. 2.3).

    Channels: 0-4 copies of the correction e used by the Jacobi update (taps C, W, E,
    S, N), 5-9 copies used by the defect, 10 and 11 the level right-hand side (Jacobi
    and defect copies), 12 the defect.  A Jacobi layer adds tap o of channel o and
    the centre of channel 10 into every e copy; the defect layer adds tap o of
    channel 5 + o and the centre of channel 11 into channel 12.  RCNN carries the
    defect into both right-hand-side copies by full weighting; TCNN adds the
    bilinear interpolation of channel 0 into every e copy."""
    C = GMG_CHANNELS
    taps = [(1, 1), (1, 0), (1, 2), (0, 1), (2, 1)]          # C, W, E, S, N
    jac = np.zeros((C, C, 3, 3))
    for t in range(10):
        for o, (a, b) in enumerate(taps):
            jac[t, o, a, b] = 1.0
        jac[t, 10, 1, 1] = 1.0
    dfc = np.zeros((C, C, 3, 3))
    for o, (a, b) in enumerate(taps):
        dfc[12, 5 + o, a, b] = 1.0
    dfc[12, 11, 1, 1] = 1.0
    stencil121 = np.outer([1.0, 2.0, 1.0], [1.0, 2.0, 1.0])
    R = np.zeros((C, C, 3, 3))
    R[10, 12] = R[11, 12] = stencil121 / 16.0
    P = np.zeros((C, C, 3, 3))
    P[0, :10] = stencil121 / 4.0
    w_in = np.zeros((C, 1, 3, 3))
    w_in[10, 0, 1, 1] = w_in[11, 0, 1, 1] = 1.0
    w_out = np.zeros((1, C, 3, 3))
    w_out[0, 0, 1, 1] = 1.0
    w = {"w_in": w_in, "w_down": np.stack([jac] * nu1 + [dfc]), "w_up": np.stack([jac] * nu2),
         "w_R": R, "w_P": P, "w_out": w_out}
    return pack_weights(w, C, nu1 + 1, nu2)


def gmg_v10_weights() -> np.ndarray:
    """Weight blob (C = 8, nu_d = nu_u = 1) whose solve phase, with the setup tensors of
    mgcnn_setup_gmg on such a context, is classical GMG V(1, 0) (Sec. 2.3).

    Channels T_W, T_E, T_S, T_N, F_G, F_J (copies of the level right-hand side), D
    (defect), E (correction).  The down layer sums the off-centre taps of T_o and the
    centre of F_G into D and the centre of F_J into E; the up layer is zero (the
    identity); RCNN carries D by full weighting into every rhs copy; TCNN adds the
    bilinear interpolation of E into E; the output reads E."""
    C = 8
    taps = [(1, 0), (1, 2), (0, 1), (2, 1)]                  # W, E, S, N
    down = np.zeros((C, C, 3, 3))
    for ch, (a, b) in enumerate(taps):
        down[6, ch, a, b] = 1.0
    down[6, 4, 1, 1] = 1.0
    down[7, 5, 1, 1] = 1.0
    stencil121 = np.outer([1.0, 2.0, 1.0], [1.0, 2.0, 1.0])
    R = np.zeros((C, C, 3, 3))
    R[:6, 6] = stencil121 / 16.0
    P = np.zeros((C, C, 3, 3))
    P[7, 7] = stencil121 / 4.0
    w_in = np.zeros((C, 1, 3, 3))
    w_in[:6, 0, 1, 1] = 1.0
    w_out = np.zeros((1, C, 3, 3))
    w_out[0, 7, 1, 1] = 1.0
    w = {"w_in": w_in, "w_down": down[None], "w_up": np.zeros((1, C, C, 3, 3)), "w_R": R, "w_P": P,
         "w_out": w_out}
    return pack_weights(w, C, 1, 1)


BPX_EPS = 2.0 ** -26   # MGCNN_BPX_EPS of the C header


def bpx_weights(channels: int = 4, layers: int = 1) -> np.ndarray:
    """Weight blob of the BPX network for a symmetric context (channels >= 2,
    down_layers = up_layers = `layers`): reChannel-in puts eps r into channel 0,
    the first down layer copies channel 0 (scaled by the setup tensor of
    mgcnn_setup_bpx) into channel 1, RCNN carries channel 0 by full weighting.
    The tied up, TCNN and out entries are filled in by the library."""
    C = channels
    w_in = np.zeros((C, 1, 3, 3))
    w_in[0, 0, 1, 1] = BPX_EPS
    down = np.zeros((layers, C, C, 3, 3))
    down[0, 1, 0, 1, 1] = 1.0
    R = np.zeros((C, C, 3, 3))
    R[0, 0] = np.outer([1.0, 2.0, 1.0], [1.0, 2.0, 1.0]) / 16.0
    return pack_weights({"w_in": w_in, "w_down": down, "w_R": R}, C, layers, layers)


class Solver:
    """One MGCNN context: weights, a setup for one coefficient field, solves."""

    def __init__(self, channels: int = 8, down_layers: int = 1, up_layers: int = 1, precision: str = "fp64",
                 pde: str = "div", scale_by_diag: int = 0, input_diag: bool = True, levels: int = 0,
                 b=(1.0, 0.5), stream=None):
        """Defaults are the learned network's configuration: unscaled setup tensors and
        the network applied to D^{-1} r (see include/mgcnn.h, mgcnn_config)."""
        self._L = load()
        self.cfg = Config(channels, down_layers, up_layers, PREC[precision], PDE[pde], int(scale_by_diag),
                          int(input_diag), levels, float(b[0]), float(b[1]))
        h = c_void_p()
        st = self._L.mgcnn_create(ctypes.byref(self.cfg), ctypes.byref(h))
        if st != OK:
            raise MGCNNError(st, "mgcnn_create failed: " + self._L.mgcnn_status_string(st).decode())
        self._h = h
        self.n = 0
        if stream is not None:
            self.set_stream(stream)

    # -- plumbing -------------------------------------------------------------
    def _check(self, st: int, what: str, ok=(OK,)) -> int:
        if st not in ok:
            msg = self._L.mgcnn_last_error(self._h).decode()
            raise MGCNNError(st, f"{what}: {self._L.mgcnn_status_string(st).decode()}: {msg}")
        return st

    def close(self):
        if getattr(self, "_h", None):
            self._L.mgcnn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, an int handle, or None (legacy default stream)."""
        handle = getattr(stream, "cuda_stream", stream)
        self._check(self._L.mgcnn_set_stream(self._h, c_void_p(handle or 0)), "mgcnn_set_stream")

    # -- ABI ------------------------------------------------------------------
    @property
    def weight_count(self) -> int:
        return int(self._L.mgcnn_weight_count(ctypes.byref(self.cfg)))

    def set_weights(self, blob):
        self._check(self._L.mgcnn_set_weights(self._h, _ptr(blob, self.weight_count), self.weight_count),
                    "mgcnn_set_weights")

    def setup(self, coeff, n: int):
        self._check(self._L.mgcnn_setup(self._h, _ptr(coeff), int(n)), "mgcnn_setup")
        self.n = int(n)

    def setup_gmg(self, coeff, n: int, omega=0.8):
        """Operators + analytic GMG-equivalent setup tensors (13 channels, or the
        8-channel V(1,0) network).  omega: one Jacobi weight, or three (finest
        level, levels in between, coarsest level)."""
        if np.ndim(omega) == 0:
            st = self._L.mgcnn_setup_gmg(self._h, _ptr(coeff), int(n), float(omega))
            self._check(st, "mgcnn_setup_gmg")
        else:
            w = _level_weights(omega)
            self._check(self._L.mgcnn_setup_gmg_levels(self._h, _ptr(coeff), int(n), w.ctypes.data),
                        "mgcnn_setup_gmg_levels")
        self.n = int(n)

    # -- training (Sec. 3.4) ---------------------------------------------------
    def _problems(self, problems):
        """[(k, f, n), ...] -> ctypes arrays of pointers and sizes (arrays are kept alive by the caller).
        k: nodal k on (n+2)^2 nodes, or mu on the n^2 interior nodes for the non-divergence form."""
        m = len(problems)
        div = self.cfg.pde == PDE["div"]
        kp = (c_void_p * m)(*[_ptr(k, (n + 2) * (n + 2) if div else n * n) for k, f, n in problems])
        fp = (c_void_p * m)(*[_ptr(f, n * n) for k, f, n in problems])
        ns = (c_int * m)(*[int(n) for k, f, n in problems])
        return m, kp, fp, ns

    def loss_grad(self, problems, K: int, want_grad: bool = True):
        """Loss after K cycles from u = 0 (mean of ||r_K||^2/||f||^2) and its gradient."""
        m, kp, fp, ns = self._problems(problems)
        loss = c_double(0.0)
        grad = np.zeros(self.weight_count) if want_grad else None
        self._check(self._L.mgcnn_loss_grad(self._h, m, kp, fp, ns, int(K), ctypes.byref(loss),
                                            grad.ctypes.data if want_grad else None), "mgcnn_loss_grad")
        return loss.value, grad

    def adam_step(self, grad, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
        self._check(self._L.mgcnn_adam_step(self._h, _ptr(grad, self.weight_count), lr, beta1, beta2, eps),
                    "mgcnn_adam_step")

    def train_step(self, problems, K: int, lr: float) -> float:
        m, kp, fp, ns = self._problems(problems)
        loss = c_double(0.0)
        self._check(self._L.mgcnn_train_step(self._h, m, kp, fp, ns, int(K), float(lr), ctypes.byref(loss), None),
                    "mgcnn_train_step")
        return loss.value

    def get_weights(self) -> np.ndarray:
        w = np.empty(self.weight_count)
        self._check(self._L.mgcnn_get_weights(self._h, w.ctypes.data, w.size), "mgcnn_get_weights")
        return w

    def gmg_solve(self, f, u, tol: float, maxit: int, nu1: int = 2, nu2: int = 2, omega=0.8):
        """Classical GMG V(nu1, nu2) on this context's operators, in place on u.
        omega: one Jacobi weight, or three (finest, in between, coarsest).
        Returns (status, iters, relres[0..iters])."""
        N = self.n * self.n
        it = c_int(0)
        hist = np.zeros(maxit + 1)
        if np.ndim(omega) == 0:
            name = "mgcnn_gmg_solve"
            st = self._L.mgcnn_gmg_solve(self._h, _ptr(f, N), _ptr(u, N, True), float(tol), int(maxit), int(nu1),
                                         int(nu2), float(omega), ctypes.byref(it), hist.ctypes.data)
        else:
            name = "mgcnn_gmg_solve_levels"
            w = _level_weights(omega)
            st = self._L.mgcnn_gmg_solve_levels(self._h, _ptr(f, N), _ptr(u, N, True), float(tol), int(maxit),
                                                int(nu1), int(nu2), w.ctypes.data, ctypes.byref(it), hist.ctypes.data)
        self._check(st, name, ok=(OK, NOT_CONVERGED))
        return st, it.value, hist[: it.value + 1]

    # -- batched solves -----------------------------------------------------------
    def setup_batched(self, coeffs, ns, gmg_omega=None):
        """coeffs[i]: nodal k of problem i ((n_i+2)^2 doubles), ns[i] = n_i.  With
        gmg_omega (one Jacobi weight, or finest / in between / coarsest), the
        analytic setup of the 8-channel GMG V(1,0) network."""
        m = len(coeffs)
        kp = (c_void_p * m)(*[_ptr(k, (n + 2) * (n + 2)) for k, n in zip(coeffs, ns)])
        nn = (c_int * m)(*[int(n) for n in ns])
        if gmg_omega is None:
            self._check(self._L.mgcnn_setup_batched(self._h, m, kp, nn), "mgcnn_setup_batched")
        elif np.ndim(gmg_omega) == 0:
            self._check(self._L.mgcnn_setup_batched_gmg(self._h, m, kp, nn, float(gmg_omega)),
                        "mgcnn_setup_batched_gmg")
        else:
            w = _level_weights(gmg_omega)
            self._check(self._L.mgcnn_setup_batched_gmg_levels(self._h, m, kp, nn, w.ctypes.data),
                        "mgcnn_setup_batched_gmg_levels")
        self.batch_sizes = [int(n) for n in ns]

    def solve_batched(self, rhs, us, tol: float, maxit: int, per_problem: bool = False):
        """Solves every problem in place on us[i].  Returns (status, iters, relres, statuses).
        per_problem: a problem whose iteration became non-finite, or rose above the
        divergence limit (OPT_DIVTOL), is reported in its entry of `statuses` (and the
        overall status) instead of raising."""
        m = len(rhs)
        fp = (c_void_p * m)(*[_ptr(f, n * n) for f, n in zip(rhs, self.batch_sizes)])
        up = (c_void_p * m)(*[_ptr(u, n * n, True) for u, n in zip(us, self.batch_sizes)])
        iters = np.zeros(m, dtype=np.int32)
        relres = np.zeros(m)
        stat = np.zeros(m, dtype=np.int32)
        st = self._L.mgcnn_solve_batched(self._h, m, fp, up, float(tol), int(maxit), iters.ctypes.data,
                                         relres.ctypes.data, stat.ctypes.data)
        self._check(st, "mgcnn_solve_batched",
                    ok=(OK, NOT_CONVERGED, ERR_NONFINITE, ERR_DIVERGED) if per_problem else (OK, NOT_CONVERGED))
        return st, iters, relres, stat

    def solve_batched_krylov(self, rhs, us, tol: float, maxit: int, restart: int = 30, per_problem: bool = False):
        """Flexible GMRES(restart) of every problem in place on us[i], the batch's
        network as preconditioner.  Returns (status, iters, relres, statuses);
        per_problem as in solve_batched."""
        m = len(rhs)
        fp = (c_void_p * m)(*[_ptr(f, n * n) for f, n in zip(rhs, self.batch_sizes)])
        up = (c_void_p * m)(*[_ptr(u, n * n, True) for u, n in zip(us, self.batch_sizes)])
        iters = np.zeros(m, dtype=np.int32)
        relres = np.zeros(m)
        stat = np.zeros(m, dtype=np.int32)
        st = self._L.mgcnn_solve_batched_krylov(self._h, m, fp, up, float(tol), int(maxit), int(restart),
                                                iters.ctypes.data, relres.ctypes.data, stat.ctypes.data)
        self._check(st, "mgcnn_solve_batched_krylov",
                    ok=(OK, NOT_CONVERGED, ERR_NONFINITE, ERR_DIVERGED) if per_problem else (OK, NOT_CONVERGED))
        return st, iters, relres, stat

    # class index -> name; the finest level's fused kernels are "down0" / "up0",
    # level l >= 1 "down<l>" / "up<l>", the coarse tail kernel "tail" (slot 21 is unused)
    PROFILE_KINDS = (("residual", "resnet", "restrict", "prolong", "in", "out", "down0", "up0") +
                     ("tail",) + tuple(f"down{l}" for l in range(1, 13)) + ("",) + tuple(f"up{l}" for l in range(1, 13)))
    OPT_FUSED = 1
    OPT_DEVICE_LOOP = 2
    OPT_TILE = 3
    OPT_SYMMETRIC = 4
    OPT_FUSED_RESIDUAL = 5
    OPT_COARSE_TAIL = 6
    OPT_DIVTOL = 7
    OPT_COARSE_K = 8

    def set_option(self, option: int, value: int):
        self._check(self._L.mgcnn_set_option(self._h, int(option), int(value)), "mgcnn_set_option")

    def profile(self, enable: bool = True):
        self._check(self._L.mgcnn_profile(self._h, int(enable)), "mgcnn_profile")

    def profile_read(self) -> dict:
        """{kind: (total_ms, launches)} since the last read."""
        k = len(self.PROFILE_KINDS)
        ms = np.zeros(k)
        cnt = np.zeros(k, dtype=np.int64)
        self._check(self._L.mgcnn_profile_read(self._h, ms.ctypes.data, cnt.ctypes.data, k), "mgcnn_profile_read")
        return {name: (float(ms[i]), int(cnt[i])) for i, name in enumerate(self.PROFILE_KINDS) if name}

    def setup_tensor_count(self) -> int:
        return int(self._L.mgcnn_setup_tensor_count(self._h))

    def set_setup_tensors(self, s):
        m = self.setup_tensor_count()
        self._check(self._L.mgcnn_set_setup_tensors(self._h, _ptr(s, m), m), "mgcnn_set_setup_tensors")

    def get_setup_tensors(self, out=None):
        m = self.setup_tensor_count()
        out = np.empty(m) if out is None else out
        self._check(self._L.mgcnn_get_setup_tensors(self._h, _ptr(out, m, True), m), "mgcnn_get_setup_tensors")
        return out

    def get_operator(self, level: int, n_l: int, out=None):
        m = 5 * n_l * n_l
        out = np.empty(m) if out is None else out
        self._check(self._L.mgcnn_get_operator(self._h, int(level), _ptr(out, m, True), m), "mgcnn_get_operator")
        return out

    def residual(self, f, u, r=None):
        N = self.n * self.n
        r = np.empty(N) if r is None else r
        nrm = c_double(0.0)
        self._check(self._L.mgcnn_residual(self._h, _ptr(f, N), _ptr(u, N), _ptr(r, N, True), ctypes.byref(nrm)),
                    "mgcnn_residual")
        return r, nrm.value

    def vcycle(self, r, e=None):
        N = self.n * self.n
        e = np.empty(N) if e is None else e
        self._check(self._L.mgcnn_vcycle(self._h, _ptr(r, N), _ptr(e, N, True)), "mgcnn_vcycle")
        return e

    def setup_bpx(self, coeff, n: int, omega: float = 1.0):
        """Operators + the setup tensors that make the symmetric network BPX."""
        self._check(self._L.mgcnn_setup_bpx(self._h, _ptr(coeff), int(n), float(omega)), "mgcnn_setup_bpx")
        self.n = int(n)

    def _solve_sym(self, fn, name, f, u, tol, maxit):
        N = self.n * self.n
        it = c_int(0)
        hist = np.zeros(maxit + 1)
        st = fn(self._h, _ptr(f, N), _ptr(u, N, True), float(tol), int(maxit), ctypes.byref(it), hist.ctypes.data)
        self._check(st, name, ok=(OK, NOT_CONVERGED))
        return st, it.value, hist[: it.value + 1]

    def solve_pcg(self, f, u, tol: float, maxit: int):
        """CG with the symmetric network as preconditioner, in place on u.
        Returns (status, iters, ||r_k|| / ||f|| for k = 0..iters)."""
        return self._solve_sym(self._L.mgcnn_solve_pcg, "mgcnn_solve_pcg", f, u, tol, maxit)

    def solve_minres(self, f, u, tol: float, maxit: int):
        """MINRES with the symmetric network as preconditioner, in place on u.
        Returns (status, iters, ||r_k||_B / ||r_0||_B for k = 0..iters)."""
        return self._solve_sym(self._L.mgcnn_solve_minres, "mgcnn_solve_minres", f, u, tol, maxit)

    def solve_krylov(self, f, u, tol: float, maxit: int, restart: int = 30):
        """Flexible GMRES with the network as preconditioner, in place on u.
        Returns (status, iters, relres[0..iters])."""
        N = self.n * self.n
        it = c_int(0)
        hist = np.zeros(maxit + 1)
        st = self._L.mgcnn_solve_krylov(self._h, _ptr(f, N), _ptr(u, N, True), float(tol), int(maxit), int(restart),
                                        ctypes.byref(it), hist.ctypes.data)
        self._check(st, "mgcnn_solve_krylov", ok=(OK, NOT_CONVERGED))
        return st, it.value, hist[: it.value + 1]

    def solve(self, f, u, tol: float, maxit: int, relres=None, raise_on_limit: bool = False):
        """Stationary iteration in place on u.  Returns (status, iters, relres[0..iters])."""
        N = self.n * self.n
        it = c_int(0)
        hist = np.zeros(maxit + 1) if relres is None else relres
        st = self._L.mgcnn_solve(self._h, _ptr(f, N), _ptr(u, N, True), float(tol), int(maxit), ctypes.byref(it),
                                 _ptr(hist, None, True))
        self._check(st, "mgcnn_solve", ok=(OK,) if raise_on_limit else (OK, NOT_CONVERGED))
        return st, it.value, hist[: it.value + 1]
