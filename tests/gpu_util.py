"""Helpers shared by the GPU tests: build/load libattn, device buffers."""
import numpy as np


def lib_and_ctx(cfg_updates=None):
    import torch
    from paper_2507_21236_gb300 import attn, build

    build()
    attn.load()
    cfg = attn.attn_config_default()
    for k, v in (cfg_updates or {}).items():
        setattr(cfg, k, v)
    ctx = attn.attn_create(cfg, torch.cuda.current_stream().cuda_stream)
    return attn, ctx


def dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
