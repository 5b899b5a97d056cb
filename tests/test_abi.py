"""The C ABI library loads and exports every entry point that include/*.h declares
(CPU only: no compute call, no device needed)."""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(mgcnn_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2312_11093_gb300 import build
    build.build()
    from paper_2312_11093_gb300 import mgcnn
    return mgcnn.load()


def test_header_declares_the_paper_entry_points():
    names = _declared()
    for n in ("mgcnn_setup", "mgcnn_solve", "mgcnn_create", "mgcnn_set_weights", "mgcnn_vcycle"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_weight_count_matches_layout(lib):
    from paper_2312_11093_gb300 import mgcnn
    for C, nd, nu in [(8, 1, 1), (13, 3, 2), (4, 2, 1)]:
        expect = 9 * C + 9 * C * C * (nd + nu + 2) + 9 * C + 9 * C * 5 + C + 4 * (9 * C * C + C) + 9 * C * C
        assert mgcnn.weight_count(C, nd, nu) == expect
    assert mgcnn.weight_count(7, 1, 1) == 0   # unsupported channel count


def test_status_strings(lib):
    assert lib.mgcnn_status_string(0) == b"MGCNN_OK"
    assert lib.mgcnn_status_string(-6) == b"MGCNN_ERR_NONFINITE"
    assert lib.mgcnn_status_string(-8) == b"MGCNN_ERR_DIVERGED"
    assert lib.mgcnn_status_string(-9) == b"MGCNN_UNKNOWN_STATUS"


def test_v10_blob_matches_oracle_construction():
    """The binding's V(1,0) weight blob equals the oracle's construction packed in
    the library's layout (host logic only)."""
    import numpy as np

    from oracle import mgcnn as omg
    from paper_2312_11093_gb300 import mgcnn
    ref = mgcnn.pack_weights(omg.gmg_v10_weights(), omg.V10_CHANNELS, 1, 1)
    assert np.array_equal(mgcnn.gmg_v10_weights(), ref)


def test_bpx_eps_matches_the_header():
    """The BPX weights of the Python binding use the header's MGCNN_BPX_EPS."""
    import re
    from paper_2312_11093_gb300 import mgcnn
    text = open(os.path.join(ROOT, "include", "mgcnn.h")).read()
    m = re.search(r"#define MGCNN_BPX_EPS (\S+)", text)
    assert m and float.fromhex(m.group(1)) == mgcnn.BPX_EPS


def test_product_code_does_not_use_the_oracle():
    """Only tests/, __graft_entry__.smoke() and bench.py's CPU legs may use oracle/:
    nothing in the package imports it, and bench.py imports it only inside the
    functions that time it on the host (the worker that runs one oracle solve
    and its network helper)."""
    pkg = os.path.join(ROOT, "paper_2312_11093_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f), errors="replace").read()
                assert not re.search(r"^\s*(import oracle|from oracle)", text, re.M), f
    lines = open(os.path.join(ROOT, "bench.py")).read().splitlines()
    current = None
    for line in lines:
        m = re.match(r"def (\w+)\(", line)
        if m:
            current = m.group(1)
        if re.match(r"\s*(import oracle|from oracle)", line):
            assert current in ("cpu_reference", "_oracle_solve", "_oracle_net"), line
