"""The C-ABI library loads without a GPU and exports every symbol include/nd.h declares;
the Python binding declares exactly those symbols."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    src = open(os.path.join(ROOT, "include", "nd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nd_[A-Za-z0-9_]+)\s*\(", src)))


def test_library_exports_header():
    from paper_1010_5636_gb300 import build
    lib_path = build.build()
    L = ctypes.CDLL(lib_path)
    syms = header_symbols()
    assert len(syms) >= 20
    missing = [s for s in syms if not hasattr(L, s)]
    assert not missing, missing


def test_binding_matches_header():
    import paper_1010_5636_gb300 as nd
    assert nd.declared_symbols() == header_symbols()


def test_zolotarev_host_call_runs_without_gpu():
    """nd_zolotarev is host code: it must work on a machine without a GPU."""
    import paper_1010_5636_gb300 as nd
    sig, b, delta = nd.nd_zolotarev(8, 1e-3)
    assert len(sig) == 8 and all(s > 0 for s in sig) and 0 < delta < 1e-3


def test_create_without_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1010_5636_gb300 as nd
    with pytest.raises(nd.NdError):
        nd.nd_create((4, 4, 4, 4), stream=ctypes.c_void_p(0))
