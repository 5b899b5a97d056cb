"""The Python binding's host-side marshalling (no library call): array checks,
the weight-blob layout, and the analytic weight sets built by the binding
against the oracle's independent constructions."""
import numpy as np
import pytest
import torch

from oracle import mgcnn as omg
from paper_2312_11093_gb300 import mgcnn


def test_pointer_checks():
    a = np.zeros(16)
    assert mgcnn._ptr(a, 16) == a.ctypes.data
    with pytest.raises(TypeError):
        mgcnn._ptr(np.zeros(16, dtype=np.float32))
    with pytest.raises(TypeError):
        mgcnn._ptr(np.zeros((4, 8))[:, ::2])                  # not contiguous
    with pytest.raises(ValueError):
        mgcnn._ptr(a, 15)
    ro = np.zeros(4)
    ro.setflags(write=False)
    mgcnn._ptr(ro, 4)
    with pytest.raises(TypeError):
        mgcnn._ptr(ro, 4, writable=True)
    t = torch.zeros(9, dtype=torch.float64)
    assert mgcnn._ptr(t, 9) == t.data_ptr()
    with pytest.raises(TypeError):
        mgcnn._ptr(torch.zeros(9, dtype=torch.float32))
    with pytest.raises(ValueError):
        mgcnn._ptr(t, 10)
    with pytest.raises(TypeError):
        mgcnn._ptr([0.0] * 4)


def layout(C, nd, nu):
    """Offsets of the blob's parts in the documented order."""
    F, S = mgcnn.FEATURES, mgcnn.SETUP_LAYERS
    sizes = [("w_in", C * 9), ("w_down", nd * C * C * 9), ("w_up", nu * C * C * 9), ("w_R", C * C * 9),
             ("w_P", C * C * 9), ("w_out", C * 9), ("sw_in", C * F * 9), ("sb_in", C), ("sw", S * C * C * 9),
             ("sb", S * C), ("sw_R", C * C * 9)]
    out, o = {}, 0
    for k, m in sizes:
        out[k] = (o, m)
        o += m
    return out, o


@pytest.mark.parametrize("C,nd,nu", [(8, 1, 1), (4, 2, 3), (2, 1, 1)])
def test_pack_weights_layout(C, nd, nu):
    rng = np.random.default_rng(C + nd + nu)
    w = omg.random_weights(max(C, 2), nd, nu, rng)
    blob = mgcnn.pack_weights(w, C, nd, nu)
    offs, total = layout(C, nd, nu)
    assert blob.size == total
    for k, (o, m) in offs.items():
        assert np.array_equal(blob[o:o + m], np.asarray(w[k]).ravel()), k
    bad = dict(w, w_R=np.zeros((C, C, 3, 2)))
    with pytest.raises(ValueError):
        mgcnn.pack_weights(bad, C, nd, nu)


def test_analytic_weight_sets_match_the_oracle():
    """The binding and the oracle build the V(1,0) and BPX networks independently."""
    assert np.array_equal(mgcnn.gmg_v10_weights(), mgcnn.pack_weights(omg.gmg_v10_weights(), 8, 1, 1))
    for C in (2, 4):
        # the oracle's BPX weights are tied already; the binding leaves tying to the library
        blob = mgcnn.bpx_weights(C)
        ref = mgcnn.pack_weights(omg.bpx_weights(C), C, 1, 1)
        offs, _ = layout(C, 1, 1)
        for k in ("w_in", "w_down", "w_R"):
            o, m = offs[k]
            assert np.array_equal(blob[o:o + m], ref[o:o + m]), k
        for k in ("w_up", "w_P", "w_out"):
            o, m = offs[k]
            assert not blob[o:o + m].any(), k
    assert mgcnn.BPX_EPS == omg.BPX_EPS
