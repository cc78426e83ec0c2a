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


def test_config_struct_layout_matches_the_header():
    """attn_config_default writes exactly sizeof(attn_config) bytes (memset + fields): a
    guard-filled buffer shows where the C struct ends, which must be where the binding's
    ctypes struct ends, with every field at the offset the defaults land on."""
    from paper_2507_21236_gb300 import attn

    attn.load()
    n = ctypes.sizeof(attn.attn_config)
    buf = (ctypes.c_ubyte * (n + 64))(*([0xAB] * (n + 64)))
    assert attn.load().attn_config_default(ctypes.cast(buf, ctypes.POINTER(attn.attn_config))) == 0
    raw = bytes(buf)
    end = len(raw)
    while end > 0 and raw[end - 1] == 0xAB:
        end -= 1
    assert end <= n and raw[n:] == b"\xab" * 64
    cfg = attn.attn_config.from_buffer_copy(raw[:n])
    assert (cfg.lanczos_depth, cfg.lanczos_tol, cfg.de_max_iter, cfg.de_rel_dev, cfg.s_ttn) == (20, 1e-13, 20, 1e-12, 1)
    assert (cfg.matvec_dtype, cfg.refine_steps, cfg.refine_tol, cfg.use_graphs, cfg.refine_inner, cfg.f64_split) == \
        (attn.ATTN_F64, 3, 1e-10, 0, 16, 0)
    # the C memset covers the whole struct: the zeroed tail reaches the binding's size
    assert all(b == 0 for b in raw[end:n]) and (cfg.de_method, cfg.tc_schedule, cfg.lanczos_basis) == (0, 0, 0)
