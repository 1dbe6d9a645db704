"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every function include/foeed.h declares (no GPU calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b(\w+)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "defined")))


def test_header_declares_the_abi():
    names = declared_functions()
    for n in ["foeed_inpaint", "eed_inpaint", "foeed_step", "eed_step", "foeed_workspace_bytes",
              "foeed_errors", "foeed_errors_workspace_bytes", "foeed_last_error", "foeed_version"]:
        assert n in names


def test_library_builds_and_exports_every_declared_symbol():
    import paper_2006_10406_gb300 as fg
    L = fg.lib()
    for n in declared_functions():
        assert hasattr(L, n), f"missing export {n}"
    assert b"sm_103a" in L.foeed_version()


def test_workspace_sizes_are_consistent():
    import paper_2006_10406_gb300 as fg
    a = fg.workspace_bytes(2048, 2048, fg.F32)
    b = fg.workspace_bytes(2048, 2048, fg.F64)
    assert a >= 3 * 2048 * 2048 * 4 + 2048 * 2048
    assert b >= 3 * 2048 * 2048 * 8 + 2048 * 2048
    assert fg.workspace_bytes(1, 1) > 0
    assert fg.lib().foeed_workspace_bytes(0, 5, 0) == 0


def test_no_gpu_raises_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import numpy as np
    import paper_2006_10406_gb300 as fg
    with pytest.raises(fg.FoeedError):
        fg.foeed_inpaint(np.zeros((4, 4)), np.zeros((4, 4), np.uint8), 0.1, 1.0, 2, 1)


def test_product_package_does_not_reference_the_oracle():
    pkg = os.path.join(ROOT, "paper_2006_10406_gb300")
    for dp, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dp, fn)).read()
                assert "import oracle" not in text and "from oracle" not in text, fn
                assert "liboracle" not in text and "foeed_oracle" not in text, fn
