"""Mistakes planted in a temporary copy of the oracle package (CPU only, the
repository is not touched) each make a pin fail: the pins are not vacuous.
Each entry: oracle file, source edit, and the pin files run against the copy."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

OP = ["test_oracle_operator.py"]
GMG = ["test_oracle_gmg.py"]
CONV = ["test_oracle_convnet.py"]
NET = ["test_oracle_mgcnn.py"]
KRY = ["test_oracle_krylov.py"]
ADJ = ["test_oracle_adjoint.py"]
SETUP = ["test_oracle_setup.py"]

MUTATIONS = {
    "face k arithmetic instead of harmonic": ("operator.py", "return 2.0 * a * b / (a + b)", "return 0.5 * (a + b)", OP),
    "upwind on the wrong side (x)": ("operator.py", "aW = -kw * ih2 - max(bx, 0.0) / h", "aW = -kw * ih2 + min(bx, 0.0) / h", OP),
    "convection missing from a_C": ("operator.py", "aC = (kw + ke + ks + kn) * ih2 + (abs(bx) + abs(by)) / h",
                                    "aC = (kw + ke + ks + kn) * ih2", OP),
    "non-div centre 3 mu": ("operator.py", "aC = 4.0 * lap +", "aC = 3.0 * lap +", OP),
    "coarse log k unweighted": ("operator.py", "w = np.array([1.0, 2.0, 1.0])\n    num", "w = np.array([1.0, 1.0, 1.0])\n    num", OP),
    "apply: N neighbour from the S side": ("operator.py", "+ st.aS * up[:-2, 1:-1] + st.aN * up[2:, 1:-1])",
                                           "+ st.aS * up[2:, 1:-1] + st.aN * up[:-2, 1:-1])", OP),
    "Jacobi without omega": ("gmg.py", "return e + omega * (r - apply(st, e)) / st.aC", "return e + (r - apply(st, e)) / st.aC", GMG),
    "restriction weights /8": ("gmg.py", "FW = np.array([[1.0, 2.0, 1.0], [2.0, 4.0, 2.0], [1.0, 2.0, 1.0]]) / 16.0",
                               "FW = np.array([[1.0, 2.0, 1.0], [2.0, 4.0, 2.0], [1.0, 2.0, 1.0]]) / 8.0", GMG),
    "no post-smoothing": ("gmg.py", "    for _ in range(nu2):\n        e = jacobi_sweep(st, e, r, om)\n    return e",
                          "    return e", GMG),
    "conv taps not centred": ("convnet.py", "y += np.tensordot(W[:, :, a, b], xp[:, a:a + n, b:b + m], axes=([1], [0]))",
                              "y += np.tensordot(W[:, :, a, b], xp[:, b:b + n, a:a + m], axes=([1], [0]))", CONV),
    "TCNN weight not transposed": ("convnet.py",
                                   "y[:, a:a + 2 * nc - 1:2, b:b + 2 * nc - 1:2] += np.tensordot(W[:, :, a, b].T, x, axes=([1], [0]))",
                                   "y[:, a:a + 2 * nc - 1:2, b:b + 2 * nc - 1:2] += np.tensordot(W[:, :, a, b], x, axes=([1], [0]))", CONV),
    "ResNet skip dropped": ("mgcnn.py", "x[l] = x[l] + cn.conv_same(s[l] * x[l], weights[\"w_down\"][i])",
                            "x[l] = cn.conv_same(s[l] * x[l], weights[\"w_down\"][i])", NET),
    "setup tensor after the conv": ("mgcnn.py", "x[l] = x[l] + cn.conv_same(s[l] * x[l], weights[\"w_up\"][i])",
                                    "x[l] = x[l] + s[l] * cn.conv_same(x[l], weights[\"w_up\"][i])", NET),
    "U-net skip of the TCNN dropped": ("mgcnn.py",
                                       "x[l - 1] = x[l - 1] + cn.tcnn(x[l], weights[\"w_P\"], sizes[l - 1])",
                                       "x[l - 1] = cn.tcnn(x[l], weights[\"w_P\"], sizes[l - 1])", NET),
    "setup tanh without skip": ("mgcnn.py", "            z = t + z\n", "            z = t\n", NET),
    "FGMRES Givens sign": ("krylov.py", "H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]",
                           "H[i + 1, j] = sn[i] * H[i, j] + cs[i] * H[i + 1, j]", KRY),
    "non-div upwind on the wrong side (y)": ("operator.py", "aS = -lap - max(vy, 0.0) / h", "aS = -lap + min(vy, 0.0) / h", OP),
    "coarse log k not renormalised at the ring": ("operator.py",
                                                  "den += w[a] * w[b] * mask[a:a + 2 * mc - 1:2, b:b + 2 * mc - 1:2]",
                                                  "den += w[a] * w[b]", OP),
    "bilinear prolongation /2": ("gmg.py", "BILINEAR = np.array([[1.0, 2.0, 1.0], [2.0, 4.0, 2.0], [1.0, 2.0, 1.0]]) / 4.0",
                                 "BILINEAR = np.array([[1.0, 2.0, 1.0], [2.0, 4.0, 2.0], [1.0, 2.0, 1.0]]) / 2.0", GMG),
    "setup features not scale-free": ("mgcnn.py", "np.log10(h * h * st.aC)])", "np.log10(st.aC)])", NET),
    "V(1,0) setup: 1 + omega": ("mgcnn.py", "s[_FG10] = (1.0 - omega_l) * st.aC if normalised else 1.0 - omega_l",
                                "s[_FG10] = (1.0 + omega_l) * st.aC if normalised else 1.0 + omega_l", NET),
    "input normalisation multiplies by D": ("mgcnn.py", "rin = r if d_inv is None else r * d_inv",
                                            "rin = r if d_inv is None else r / d_inv", NET),
    "FGMRES update with unpreconditioned directions": ("krylov.py", "u = u + y[i] * Z[i]", "u = u + y[i] * V[i]", KRY),
    "RCNN taps offset by one": ("convnet.py",
                                "y += np.tensordot(W[:, :, a, b], x[:, a:a + 2 * nc - 1:2, b:b + 2 * nc - 1:2], axes=([1], [0]))",
                                "y += np.tensordot(W[:, :, a, b], x[:, b:b + 2 * nc - 1:2, a:a + 2 * nc - 1:2], axes=([1], [0]))",
                                CONV),
    "level rule off by one": ("grid.py", "    return m - 1\n", "    return m\n", OP),
    "GMG-equivalent Jacobi copies not divided by a_C": ("mgcnn.py",
                                                        "s[_E[k]] = _shift_to_source(-omega_l * a / st.aC, dy, dx)",
                                                        "s[_E[k]] = _shift_to_source(-omega_l * a, dy, dx)", NET),
    "GMG-equivalent defect copies with the wrong sign": ("mgcnn.py", "s[_G[k]] = _shift_to_source(-a, dy, dx)",
                                                         "s[_G[k]] = _shift_to_source(a, dy, dx)", NET),
    "adjoint: s gradient drops x": ("adjoint.py", "sbar_l += x_in * t", "sbar_l += t", ADJ),
    "adjoint: tanh derivative": ("adjoint.py", "dpre = zb * (1.0 - t * t)", "dpre = zb * (1.0 - t)", ADJ),
    "adjoint: TCNN gradient from the wrong state": ("adjoint.py",
                                                    "grads[\"w_P\"] += cn.tcnn_wgrad(keep[\"x_fin\"][l + 1], xb)",
                                                    "grads[\"w_P\"] += cn.tcnn_wgrad(keep[\"x_down\"][l + 1], xb)", ADJ),
    "adjoint: input normalisation not applied": ("adjoint.py", "                rbar = rbar * d_inv\n",
                                                 "                rbar = rbar\n", ADJ),
    "adjoint: skip path dropped": ("adjoint.py", "return xbar + s_l * t", "return s_l * t", ADJ),
    "setup RCNN restricts the NonLinearResNet output": ("mgcnn.py", "c = cn.rcnn(c, weights[\"sw_R\"])",
                                                       "c = cn.rcnn(z, weights[\"sw_R\"])", SETUP),
    "setup RCNN restricts the scaled setup output": ("mgcnn.py", "c = cn.rcnn(c, weights[\"sw_R\"])",
                                                    "c = cn.rcnn(outs[-1], weights[\"sw_R\"])", SETUP),
    "level scaling in front of the NonLinearResNet": (
        "mgcnn.py",
        [("        z = c\n        zl, tl = [], []\n",
          "        z = c / stencils[l].aC if int(scale_by_diag) == 1 else c\n        zl, tl = [], []\n"),
         ("outs.append(z / stencils[l].aC)", "outs.append(z)")],
        None, SETUP),
    "three setup layers": ("mgcnn.py", "SETUP_LAYERS = 4", "SETUP_LAYERS = 3", SETUP),
    "setup bias outside the tanh": ("mgcnn.py", "t = np.tanh(cn.conv_same(z, weights[\"sw\"][i], weights[\"sb\"][i]))",
                                    "t = np.tanh(cn.conv_same(z, weights[\"sw\"][i])) + weights[\"sb\"][i][:, None, None]",
                                    SETUP),
    "coarsest level takes the in-between weight": ("gmg.py", "return [w_fine] + [w_mid] * (levels - 2) + [w_coarsest]",
                                                   "return [w_fine] + [w_mid] * (levels - 1)", GMG),
    "V-cycle smooths every level with the finest weight": ("gmg.py", "om = _omega_at(omega, level)",
                                                           "om = _omega_at(omega, 0)", GMG),
    "V(1,0) setup uses the finest weight on every level": (
        "mgcnn.py", "omega_l = _level_weight(omega, lev)\n        n = st.n\n        s = np.zeros((V10_CHANNELS",
        "omega_l = _level_weight(omega, 0)\n        n = st.n\n        s = np.zeros((V10_CHANNELS", NET),
    "GMG-equivalent setup uses the finest weight on every level": (
        "mgcnn.py", "omega_l = _level_weight(omega, lev)\n        n = st.n\n        s = np.zeros((GMG_CHANNELS",
        "omega_l = _level_weight(omega, 0)\n        n = st.n\n        s = np.zeros((GMG_CHANNELS", NET),
    "arithmetic coarse k averages log k": ("operator.py", "g = np.pad(np.log(k) if mean == \"log\" else k, 1)",
                                           "g = np.pad(np.log(k), 1)", OP),
    "arithmetic coarse k returned as a geometric mean": (
        "operator.py", "return np.exp(num / den) if mean == \"log\" else num / den", "return np.exp(num / den)", OP),
}


def run_against_mutant(tmp_path, fname, old, new, files):
    """`old` is one source fragment replaced by `new`, or a list of (old, new)
    pairs applied together (then `new` is None)."""
    shutil.copytree(os.path.join(ROOT, "oracle"), tmp_path / "oracle")
    p = tmp_path / "oracle" / fname
    src = p.read_text()
    for o, w in (old if new is None else [(old, new)]):
        assert src.count(o) == 1, o
        src = src.replace(o, w)
    p.write_text(src)
    # the copy comes first on the path: the subprocess starts in it, and the
    # repository follows for everything else
    env = dict(os.environ, PYTHONPATH=str(tmp_path) + os.pathsep + ROOT)
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
                           "--rootdir", ROOT, *[os.path.join(ROOT, "tests", f) for f in files]], cwd=str(tmp_path),
                          env=env, capture_output=True, text=True, timeout=600)


@pytest.mark.parametrize("name", list(MUTATIONS))
def test_planted_mistake_fails_a_pin(tmp_path, name):
    r = run_against_mutant(tmp_path, *MUTATIONS[name])
    assert r.returncode == 1, r.stdout[-1500:] + r.stderr[-1500:]    # 1: tests ran and failed


def test_the_copy_is_what_the_pins_import(tmp_path):
    """Control: a copy whose oracle raises on import makes the pin run fail to collect."""
    r = run_against_mutant(tmp_path, "grid.py", "from __future__ import annotations",
                           "from __future__ import annotations\nraise ImportError('planted')", OP)
    assert r.returncode != 0 and "planted" in (r.stdout + r.stderr)
