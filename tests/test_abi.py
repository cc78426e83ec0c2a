"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/attn.h (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "attn.h")).read()
    return sorted(set(re.findall(r"ATTN_API\s+[\w\s\*]+?\b(attn_\w+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_2507_21236_gb300 import build, attn

    path = build()
    lib = ctypes.CDLL(path)
    names = declared()
    assert len(names) >= 30
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the binding wraps exactly the declared entry points
    assert sorted(attn.exported_symbols()) == names
    assert attn.load().attn_version().decode().startswith("attn-gb300")


def test_no_gpu_means_loud_error():
    """Without a GPU the library reports ATTN_ECUDA instead of computing on the CPU."""
    import torch
    from paper_2507_21236_gb300 import attn

    if torch.cuda.is_available():
        return
    attn.load()
    try:
        attn.attn_create()
    except attn.AttnError as e:
        assert e.status == 3
    else:
        raise AssertionError("attn_create succeeded without a GPU")
