"""The allocation-free residual entry point (mgcnn_residual_noalloc).

Some callers cannot call cudaMalloc: hosts that hand the library a fixed
device-memory budget owned by another allocator (a hidden allocation would
break that budget), and tools that may only touch buffers they were given.  mgcnn_residual_noalloc serves them: the caller passes its own
device arrays, and the per-block partial sums of the norm live in a fixed
array inside the library instead of a fresh allocation.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2312_11093_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2312_11093_gb300 import build
    build.build()
    from paper_2312_11093_gb300 import mgcnn
    L = mgcnn.load()
    L.mgcnn_residual_noalloc.restype = ctypes.c_int
    L.mgcnn_residual_noalloc.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                                                   ctypes.c_void_p]
    return mgcnn


def _noalloc(M, op, f, u, r, n, stream=None):
    nrm = ctypes.c_double(-1.0)
    st = M.load().mgcnn_residual_noalloc(op.data_ptr(), f.data_ptr(), u.data_ptr(), r.data_ptr(), n,
                                         ctypes.byref(nrm), stream)
    return st, nrm.value


@pytest.mark.parametrize("on_stream", [False, True])
def test_noalloc_residual_matches_context_residual_twice(M, on_stream):
    """Calls in a row (different problem sizes, so the shared scratch holds the
    previous call's data; the largest is 4095^2, 8,188 of the array's 8,192
    partial sums) agree with mgcnn_residual within the tests' FP64 bar, on the legacy
    default stream and on a stream of the caller's."""
    stream = torch.cuda.Stream() if on_stream else None
    for n, seed in ((127, 1), (63, 2), (4095, 3), (255, 4)):
        rng = np.random.default_rng(seed)
        k = inputs.lognormal_k(n, 0.1, rng)
        f = inputs.normal_rhs(n, rng)
        u = rng.standard_normal((n, n)) * 1e-3
        sv = M.Solver(8, 1, 1)
        sv.set_weights(np.zeros(sv.weight_count))
        sv.setup(k.ravel().copy(), n)
        r_ref, n2_ref = sv.residual(f.ravel().copy(), u.ravel().copy())
        op = torch.from_numpy(sv.get_operator(0, n)).cuda()
        fd = torch.from_numpy(f.ravel().copy()).cuda()
        ud = torch.from_numpy(u.ravel().copy()).cuda()
        rd = torch.empty(n * n, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        st, n2 = _noalloc(M, op, fd, ud, rd, n, stream.cuda_stream if stream is not None else None)
        assert st == M.OK
        r = rd.cpu().numpy()
        assert np.max(np.abs(r - r_ref)) <= 1e-14 * np.max(np.abs(r_ref))
        assert abs(n2 - n2_ref) <= 1e-12 * n2_ref


def test_noalloc_rejects_oversized_and_host_arrays(M):
    """Grids above the scratch array's limit are refused before any launch: 4097^2,
    and 2^20 (whose 2^40 unknowns would wrap a 32-bit block count to zero)."""
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    for n in (4097, 1 << 20, 2**31 - 1):
        st, _ = _noalloc(M, t, t, t, t, n)
        assert st == M.ERR_SIZE
    h = np.zeros(9)
    nrm = ctypes.c_double(0.0)
    st = M.load().mgcnn_residual_noalloc(h.ctypes.data, h.ctypes.data, h.ctypes.data, h.ctypes.data, 3,
                                         ctypes.byref(nrm), None)
    assert st == M.ERR_ARG
