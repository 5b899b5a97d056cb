"""MGCNN setup and solve phases in FP64 (Sec. 3.2, Algorithm 2; Sec. 3.3, Algorithm 3).

Weights (a dict of float64 arrays; C channels, F = 5 setup features,
nu_d / nu_u layers in ResNetDown / ResNetUp, S = 4 setup layers):

  solve phase                                     setup phase
  w_in   [C, 1, 3, 3]   reChannelCNN rhs -> C     sw_in [C, F, 3, 3], sb_in [C]
  w_down [nu_d, C, C, 3, 3]                        sw    [S, C, C, 3, 3], sb [S, C]
  w_up   [nu_u, C, C, 3, 3]                        sw_R  [C, C, 3, 3]   setup RCNN
  w_R    [C, C, 3, 3]   RCNN   [c_out, c_in]
  w_P    [C, C, 3, 3]   TCNN   [c_in, c_out]
  w_out  [1, C, 3, 3]   reChannelCNN C -> sol

One set serves every level (P3, Sec. 3.1).  The solve phase has no bias and
no activation (P2), so B is linear in the right-hand side.

Readings where the paper is silent (each is listed in the design notes):
* setup input: the scale-free stencil [a_W, a_E, a_S, a_N]/a_C and
  log10(h^2 a_C) (Remark "Matrix coefficients as input"), F = 5;
* setup output scaling (`scale_by_diag`): 1 (True) divides setup_out_l by a_C
  of the level-l rediscretised operator (k restricted as in
  operator.restrict_k), a Jacobi-like D^{-1} that gives B the units of A^{-1};
  2 multiplies it by (h_l / h_1)^2 = 4^(l-1), the coefficient-free part of that
  ratio between levels (a coarse diagonal is 4x smaller per level), for use
  with the normalised input below; 0 (False) leaves it unscaled;
* the setup RCNN has its own weights, no bias; every setup layer is
  tanh(K z + b) + z (Eq. resnet_nonlinear), the last one included;
* input normalisation: Sec. 2.5 removes the 1/h factor of the stencil so that
  the network works on an O(1) operator at every grid size.  For a
  heterogeneous divergence-form operator the pointwise analogue is the
  diagonal: with `d_inv` = 1/a_C (finest level) the solve phase is applied to
  D^{-1} r, i.e. B r = Net(D^{-1} r).  Without it the ResNet skip paths give B
  an O(1) multiple of the identity while A ~ k/h^2, and A B grows like n^2.
"""
from __future__ import annotations

import numpy as np

from . import convnet as cn
from .grid import spacing
from .operator import Stencil, apply

SETUP_LAYERS = 4
FEATURES = 5


def random_weights(C: int, nu_d: int, nu_u: int, rng: np.random.Generator, scale: float = 0.3) -> dict:
    """Random weights of the right shapes (test inputs; not a trained solver)."""
    def r(*shape, fan):
        return rng.standard_normal(shape) * (scale / np.sqrt(fan))
    return {
        "w_in": r(C, 1, 3, 3, fan=9), "w_down": r(nu_d, C, C, 3, 3, fan=9 * C),
        "w_up": r(nu_u, C, C, 3, 3, fan=9 * C), "w_R": r(C, C, 3, 3, fan=9 * C),
        "w_P": r(C, C, 3, 3, fan=9 * C), "w_out": r(1, C, 3, 3, fan=9 * C),
        "sw_in": r(C, FEATURES, 3, 3, fan=9 * FEATURES), "sb_in": r(C, fan=1),
        "sw": r(SETUP_LAYERS, C, C, 3, 3, fan=9 * C), "sb": r(SETUP_LAYERS, C, fan=1),
        "sw_R": r(C, C, 3, 3, fan=9 * C),
    }


def setup_features(st: Stencil) -> np.ndarray:
    """[a_W/a_C, a_E/a_C, a_S/a_C, a_N/a_C, log10(h^2 a_C)] on the finest grid, shape [5, n, n]."""
    h = spacing(st.n)
    return np.stack([st.aW / st.aC, st.aE / st.aC, st.aS / st.aC, st.aN / st.aC,
                     np.log10(h * h * st.aC)])


def setup(weights: dict, stencils: list[Stencil], scale_by_diag: bool = True, keep: dict | None = None):
    """Algorithm 2.  Returns setup_outs[l], each [C, n_l, n_l].

    coef_1 = reChannelCNN(features); for each level: setup_out_l =
    NonLinearResNet(coef_l) (4 x [z <- tanh(K_i z + b_i) + z]), then
    coef_{l+1} = RCNN(coef_l).  If `keep` is a dict, the intermediates needed by
    the adjoint are stored in it.
    """
    L = len(stencils)
    feat = setup_features(stencils[0])
    c = cn.conv_same(feat, weights["sw_in"], weights["sb_in"])
    outs, cs, zs, ts = [], [], [], []
    for l in range(L):
        cs.append(c)
        z = c
        zl, tl = [], []
        for i in range(SETUP_LAYERS):
            zl.append(z)
            t = np.tanh(cn.conv_same(z, weights["sw"][i], weights["sb"][i]))
            tl.append(t)
            z = t + z
        zs.append(zl)
        ts.append(tl)
        mode = int(scale_by_diag)
        if mode == 1:
            outs.append(z / stencils[l].aC)
        elif mode == 2:
            outs.append(z * (spacing(stencils[l].n) / spacing(stencils[0].n)) ** 2)
        else:
            outs.append(z)
        if l < L - 1:
            c = cn.rcnn(c, weights["sw_R"])
    if keep is not None:
        keep.update(feat=feat, c=cs, z=zs, t=ts)
    return outs


def solve_phase(weights: dict, s: list[np.ndarray], r: np.ndarray, keep: dict | None = None,
                d_inv: np.ndarray | None = None) -> np.ndarray:
    """Algorithm 3: one application e = B r of the solve network.

    x_1 = reChannelCNN(r) (of D^{-1} r when d_inv is given); down loop:
    x_l <- ResNetDown(s_l, x_l) then x_{l+1} = RCNN(x_l); up loop:
    x_l <- ResNetUp(s_l, x_l) then x_{l-1} <- x_{l-1} + TCNN(x_l);
    sol = reChannelCNN(x_1).  Each ResNet layer is y = K (s_l * x) + x
    (Eq. heteroresnet).
    """
    L = len(s)
    sizes = [t.shape[1] for t in s]
    nu_d = weights["w_down"].shape[0]
    nu_u = weights["w_up"].shape[0]
    x = [None] * L
    x0, down_in, x_down, up_in, x_fin = [None] * L, [], [None] * L, [None] * L, [None] * L
    rin = r if d_inv is None else r * d_inv
    x[0] = cn.conv_same(rin[None], weights["w_in"])
    for l in range(L):
        x0[l] = x[l]
        ins = []
        for i in range(nu_d):
            ins.append(x[l])
            x[l] = x[l] + cn.conv_same(s[l] * x[l], weights["w_down"][i])
        down_in.append(ins)
        x_down[l] = x[l]
        if l < L - 1:
            x[l + 1] = cn.rcnn(x[l], weights["w_R"])
    for l in reversed(range(L)):
        ins = []
        for i in range(nu_u):
            ins.append(x[l])
            x[l] = x[l] + cn.conv_same(s[l] * x[l], weights["w_up"][i])
        up_in[l] = ins
        x_fin[l] = x[l]
        if l > 0:
            x[l - 1] = x[l - 1] + cn.tcnn(x[l], weights["w_P"], sizes[l - 1])
    e = cn.conv_same(x[0], weights["w_out"])[0]
    if keep is not None:
        keep.update(x0=x0, down_in=down_in, x_down=x_down, up_in=up_in, x_fin=x_fin, rin=rin)
    return e


# --------------------------------------------------------------------------
# Symmetric variant (Remark "Symmetric problem", Sec. 3.3): the network is made
# a symmetric operator by sharing weights between ResNetDown and ResNetUp and
# between RCNN and TCNN.  Reading: "sharing" means each up map is the adjoint of
# the matching down map, so that B = W_out M_1 W_in with M_l = U_l (I + P M_{l+1} R) D_l
# has U_l = D_l^T, P = R^T and W_out = W_in^T:
#   down layer   x <- x + K (s * x)            (Eq. heteroresnet, unchanged)
#   up layer     x <- x + s * (K^T x)          (its adjoint: the conv with K's
#                                               channels swapped and taps flipped,
#                                               the setup tensor applied after it)
#   TCNN         the transposed conv with the RCNN weights (exactly R^T)
#   reChannel-out the adjoint of reChannel-in
# The up layers run in the reverse order of the down layers.  Then
#   M_L = D_L^T D_L,   M_l = D_l^T (I + R^T M_{l+1} R) D_l,
# so every M_l is symmetric positive semidefinite and B = W_in^T M_1 W_in is
# symmetric positive definite whenever the down layers are nonsingular and W_in
# is injective -- for any weights and setup tensors -- which is what CG and
# MINRES need from a preconditioner.  No input normalisation (D^{-1} r would
# break the symmetry).
# --------------------------------------------------------------------------
def adjoint_kernel(W: np.ndarray) -> np.ndarray:
    """Weights of the adjoint of a same-size conv: W'[ci, co, a, b] = W[co, ci, 2-a, 2-b]."""
    return np.ascontiguousarray(W.transpose(1, 0, 2, 3)[:, :, ::-1, ::-1])


def symmetric_weights(weights: dict) -> dict:
    """The weight set of the symmetric variant as a plain weight dict: the up,
    TCNN and reChannel-out weights replaced by the tied ones (w_up[i] = the
    adjoint kernel of w_down[nu - 1 - i], w_P = w_R, w_out = the adjoint of
    w_in).  Setup weights are kept."""
    nu = weights["w_down"].shape[0]
    w = dict(weights)
    w["w_up"] = np.stack([adjoint_kernel(weights["w_down"][nu - 1 - i]) for i in range(nu)])
    w["w_P"] = weights["w_R"].copy()
    w["w_out"] = adjoint_kernel(weights["w_in"])
    return w


def solve_phase_symmetric(weights: dict, s: list[np.ndarray], r: np.ndarray) -> np.ndarray:
    """e = B r of the symmetric variant (tied weights taken from `weights`' down,
    RCNN and reChannel-in entries; its up, TCNN and out entries are ignored)."""
    L = len(s)
    sizes = [t.shape[1] for t in s]
    Kd = weights["w_down"]
    nu = Kd.shape[0]
    x = [None] * L
    x[0] = cn.conv_same(r[None], weights["w_in"])
    for l in range(L):
        for i in range(nu):
            x[l] = x[l] + cn.conv_same(s[l] * x[l], Kd[i])
        if l < L - 1:
            x[l + 1] = cn.rcnn(x[l], weights["w_R"])
    for l in reversed(range(L)):
        for i in reversed(range(nu)):
            x[l] = x[l] + s[l] * cn.conv_same_adjoint(x[l], Kd[i])
        if l > 0:
            x[l - 1] = x[l - 1] + cn.tcnn(x[l], weights["w_R"], sizes[l - 1])
    return cn.conv_same_adjoint(x[0], weights["w_in"])[0]


# Additive multilevel (BPX) preconditioner as a symmetric network.  With
# channel 0 a carrier of the (restricted) residual and channel 1 its scaled copy,
#   x_0 = eps r (reChannel-in),  down layer: x[1] += s[0] * x[0],  RCNN: x[0] <- FW x[0],
# the state after level l's down layer holds eps R_l r and sqrt(omega 4^l / a_C,l) R_l r
# (R_l = FW applied l times, R_0 = I) when s_l[0] = sqrt(omega 4^l / a_C,l) / eps.
# The tied up sweep adds the adjoints, so
#   B = sum_l 4^l R_l^T (omega D_l^{-1}) R_l  +  eps^2 sum_l R_l^T R_l,
# the BPX form sum_l P_l D_l^{-1} P_l^T with P_l = 4^l R_l^T (bilinear
# prolongation) and Jacobi-scaled levels (D_l: diagonal of the rediscretised
# level-l operator), plus a term eps^2 a_C,l / (omega 4^l) times the level's
# smoother term, at most 4 eps^2 k (n+1)^2 / omega: below 1e-6 with eps = 2^-26
# up to 4095^2 for k <= 50.  Channels 2.. stay zero.
BPX_EPS = 2.0 ** -26


def bpx_weights(C: int = 4, nu: int = 1) -> dict:
    """Weights of the BPX network (C >= 2 channels, nu down layers of which the
    first carries the smoother copy); setup weights zero."""
    z = lambda *shape: np.zeros(shape)
    w = {"w_in": z(C, 1, 3, 3), "w_down": z(nu, C, C, 3, 3), "w_up": z(nu, C, C, 3, 3),
         "w_R": z(C, C, 3, 3), "w_P": z(C, C, 3, 3), "w_out": z(1, C, 3, 3),
         "sw_in": z(C, FEATURES, 3, 3), "sb_in": z(C), "sw": z(SETUP_LAYERS, C, C, 3, 3),
         "sb": z(SETUP_LAYERS, C), "sw_R": z(C, C, 3, 3)}
    w["w_in"][0, 0, 1, 1] = BPX_EPS
    w["w_down"][0, 1, 0, 1, 1] = 1.0
    w["w_R"][0, 0] = np.array([[1.0, 2.0, 1.0], [2.0, 4.0, 2.0], [1.0, 2.0, 1.0]]) / 16.0
    return symmetric_weights(w)


def bpx_setup(stencils: list[Stencil], omega: float = 1.0, C: int = 4) -> list[np.ndarray]:
    """Setup tensors of the BPX network: s_l[0] = sqrt(omega 4^l / a_C,l) / eps, others 0."""
    out = []
    for lev, st in enumerate(stencils):
        s = np.zeros((C, st.n, st.n))
        s[0] = np.sqrt(omega * 4.0 ** lev / st.aC) / BPX_EPS
        out.append(s)
    return out


def stationary_solve(weights: dict, s: list[np.ndarray], A: Stencil, f: np.ndarray,
                     u0: np.ndarray | None, tol: float, maxit: int, input_diag: bool = False):
    """Eq. 1 with B = solve_phase: u^{k+1} = u^k + B (f - A u^k)
    (B r = Net(D^{-1} r) when input_diag).

    Stops when ||r^k||_2 / ||f||_2 <= tol (checked before each cycle) or k = maxit.
    Returns (u, iters, relres_history, iterates) with iterates[k] = u^k.
    """
    u = np.zeros_like(f) if u0 is None else u0.copy()
    fn = np.linalg.norm(f)
    if fn == 0.0:
        return np.zeros_like(f), 0, [0.0], [np.zeros_like(f)]
    hist, iterates = [], [u.copy()]
    for k in range(maxit + 1):
        r = f - apply(A, u)
        rel = np.linalg.norm(r) / fn
        hist.append(rel)
        if rel <= tol or k == maxit:
            return u, k, hist, iterates
        u = u + solve_phase(weights, s, r, d_inv=(1.0 / A.aC) if input_diag else None)
        iterates.append(u.copy())
    raise AssertionError("unreachable")


# --------------------------------------------------------------------------
# Weights that turn the solve phase into classical GMG V(2,2) (weighted Jacobi,
# full-weighting restriction, bilinear prolongation, rediscretised A_l).
#
# Any stencil acting on e rewrites in source-side form:
#   sum_o a_o(p) e(p+o) = sum_o  ~a_o(q) e(q)  with q = p + o, ~a_o(q) = a_o(q - o),
# so a setup tensor that multiplies a layer's input (Eq. heteroresnet) carries
# the variable coefficient and the 3x3 kernel only selects the tap o.
# Channels (13): E_C E_W E_E E_S E_N  (copies of e for the Jacobi update)
#                G_C G_W G_E G_S G_N  (copies of e for the defect)
#                F_J F_G              (copies of the level right-hand side)
#                D                    (defect)
# --------------------------------------------------------------------------
GMG_CHANNELS = 13
_E = [0, 1, 2, 3, 4]
_G = [5, 6, 7, 8, 9]
_FJ, _FG, _D = 10, 11, 12
# offsets o = (dy, dx) for C, W, E, S, N and the 3x3 tap that reads p + o
_OFFS = [(0, 0), (0, -1), (0, 1), (-1, 0), (1, 0)]
_TAPS = [(dy + 1, dx + 1) for dy, dx in _OFFS]


def gmg_equivalent_weights(nu1: int = 2, nu2: int = 2) -> dict:
    """Solve-phase weights (C = 13) for GMG V(nu1, nu2): ResNetDown = nu1 Jacobi layers
    and one defect layer, ResNetUp = nu2 Jacobi layers, RCNN = full weighting of the
    defect into both rhs copies, TCNN = bilinear interpolation of E_C into every e copy."""
    C = GMG_CHANNELS
    KJ = np.zeros((C, C, 3, 3))
    for t in _E + _G:
        for ch, (a, b) in zip(_E, _TAPS):
            KJ[t, ch, a, b] = 1.0
        KJ[t, _FJ, 1, 1] = 1.0
    KD = np.zeros((C, C, 3, 3))
    for ch, (a, b) in zip(_G, _TAPS):
        KD[_D, ch, a, b] = 1.0
    KD[_D, _FG, 1, 1] = 1.0
    fw = np.array([[1.0, 2.0, 1.0], [2.0, 4.0, 2.0], [1.0, 2.0, 1.0]]) / 16.0
    bil = np.array([[1.0, 2.0, 1.0], [2.0, 4.0, 2.0], [1.0, 2.0, 1.0]]) / 4.0
    R = np.zeros((C, C, 3, 3))
    R[_FJ, _D] = fw
    R[_FG, _D] = fw
    P = np.zeros((C, C, 3, 3))
    for t in _E + _G:
        P[_E[0], t] = bil
    w_in = np.zeros((C, 1, 3, 3))
    w_in[_FJ, 0, 1, 1] = 1.0
    w_in[_FG, 0, 1, 1] = 1.0
    w_out = np.zeros((1, C, 3, 3))
    w_out[0, _E[0], 1, 1] = 1.0
    return {"w_in": w_in, "w_down": np.stack([KJ] * nu1 + [KD]), "w_up": np.stack([KJ] * nu2),
            "w_R": R, "w_P": P, "w_out": w_out}


def _shift_to_source(a: np.ndarray, dy: int, dx: int) -> np.ndarray:
    """out[q] = a[q - o] for o = (dy, dx), zero where q - o is outside the grid."""
    n = a.shape[0]
    out = np.zeros_like(a)
    qy = slice(max(dy, 0), n + min(dy, 0))
    qx = slice(max(dx, 0), n + min(dx, 0))
    py = slice(max(-dy, 0), n + min(-dy, 0))
    px = slice(max(-dx, 0), n + min(-dx, 0))
    out[qy, qx] = a[py, px]
    return out


def _level_weight(omega, lev: int) -> float:
    """omega: one Jacobi weight, or a list with one weight per level (finest first)."""
    return float(omega) if np.ndim(omega) == 0 else float(omega[lev])


def gmg_equivalent_setup(stencils: list[Stencil], omega=0.8, input_diag: bool = False) -> list[np.ndarray]:
    """Setup tensors for `gmg_equivalent_weights` on every level:
    s[E_o](q) = -omega a_o(q-o)/a_C(q-o),  s[F_J] = omega/a_C,
    s[G_o](q) = -a_o(q-o),                 s[F_G] = 1,  s[D] = 0.
    With input_diag the finest level's rhs copies hold D^{-1} r, so there
    s[F_J] = omega and s[F_G] = a_C (the same Jacobi update and defect).
    omega: one weight, or one per level (level l's tensors use omega[l])."""
    outs = []
    for lev, st in enumerate(stencils):
        omega_l = _level_weight(omega, lev)
        n = st.n
        s = np.zeros((GMG_CHANNELS, n, n))
        coeffs = [st.aC, st.aW, st.aE, st.aS, st.aN]
        for k, ((dy, dx), a) in enumerate(zip(_OFFS, coeffs)):
            s[_E[k]] = _shift_to_source(-omega_l * a / st.aC, dy, dx)
            s[_G[k]] = _shift_to_source(-a, dy, dx)
        if input_diag and lev == 0:
            s[_FJ] = omega_l
            s[_FG] = st.aC
        else:
            s[_FJ] = omega_l / st.aC
            s[_FG] = 1.0
        outs.append(s)
    return outs



# --------------------------------------------------------------------------
# An 8-channel network (one ResNetDown and one ResNetUp layer, the learned
# network's shape) that is classical GMG V(1, 0) (Sec. 2.3).  The one down
# layer does the single pre-smoothing sweep from e = 0 and forms the defect in
# the same pass: with e = omega D^{-1} r,
#   d(p) = r(p) - sum_o a_o(p) e(p + o) = (1 - omega) r(p) - sum_{o != C} omega a_o(p) r(p+o) / a_C(p+o),
# whose off-centre coefficients are again source-side setup tensors
# (~a_o(q) = -omega a_o(q - o) / a_C(q)).  The up layer is the identity
# (no post-smoothing), the TCNN adds the bilinear interpolation of the coarse
# correction into the correction channel.
# Channels (8): T_W T_E T_S T_N (rhs copies read by the defect's off-centre
#               taps), F_G (rhs copy, defect centre), F_J (rhs copy, Jacobi),
#               D (defect), E (correction)
# --------------------------------------------------------------------------
V10_CHANNELS = 8
_T10 = [0, 1, 2, 3]
_FG10, _FJ10, _D10, _E10 = 4, 5, 6, 7


def gmg_v10_weights() -> dict:
    """Solve-phase weights (C = 8, one down and one up layer) for GMG V(1, 0)."""
    C = V10_CHANNELS
    KD = np.zeros((C, C, 3, 3))
    for ch, (a, b) in zip(_T10, _TAPS[1:]):
        KD[_D10, ch, a, b] = 1.0
    KD[_D10, _FG10, 1, 1] = 1.0
    KD[_E10, _FJ10, 1, 1] = 1.0
    fw = np.array([[1.0, 2.0, 1.0], [2.0, 4.0, 2.0], [1.0, 2.0, 1.0]]) / 16.0
    bil = np.array([[1.0, 2.0, 1.0], [2.0, 4.0, 2.0], [1.0, 2.0, 1.0]]) / 4.0
    R = np.zeros((C, C, 3, 3))
    for ch in _T10 + [_FG10, _FJ10]:
        R[ch, _D10] = fw
    P = np.zeros((C, C, 3, 3))
    P[_E10, _E10] = bil
    w_in = np.zeros((C, 1, 3, 3))
    for ch in _T10 + [_FG10, _FJ10]:
        w_in[ch, 0, 1, 1] = 1.0
    w_out = np.zeros((1, C, 3, 3))
    w_out[0, _E10, 1, 1] = 1.0
    return {"w_in": w_in, "w_down": KD[None], "w_up": np.zeros((1, C, C, 3, 3)),
            "w_R": R, "w_P": P, "w_out": w_out}


def gmg_v10_setup(stencils: list[Stencil], omega=0.8, input_diag: bool = False) -> list[np.ndarray]:
    """Setup tensors for `gmg_v10_weights` on every level:
    s[T_o](q) = -omega a_o(q-o)/a_C(q),  s[F_G] = 1 - omega,  s[F_J] = omega/a_C,  s[D] = s[E] = 0.
    With input_diag the finest level's rhs copies hold D^{-1} r, so there
    s[T_o](q) = -omega a_o(q-o), s[F_G] = (1 - omega) a_C, s[F_J] = omega.
    omega: one weight, or one per level (level l's tensors use omega[l])."""
    outs = []
    for lev, st in enumerate(stencils):
        omega_l = _level_weight(omega, lev)
        n = st.n
        s = np.zeros((V10_CHANNELS, n, n))
        normalised = input_diag and lev == 0
        for ch, (dy, dx), a in zip(_T10, _OFFS[1:], [st.aW, st.aE, st.aS, st.aN]):
            shifted = _shift_to_source(-omega_l * a, dy, dx)
            s[ch] = shifted if normalised else shifted / st.aC
        s[_FG10] = (1.0 - omega_l) * st.aC if normalised else 1.0 - omega_l
        s[_FJ10] = omega_l if normalised else omega_l / st.aC
        outs.append(s)
    return outs
