"""Shared helpers for the tests (host-side marshalling only)."""
import re
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def to_dev(x, device="cuda"):
    """uint32 numpy array -> int32 CUDA tensor with the same bits."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.uint32).view(np.int32)).to(device)


def to_host(t):
    """int32/uint32 tensor -> uint32 numpy array with the same bits."""
    import torch
    if t.dtype != torch.int32:
        t = t.view(torch.int32)
    return t.detach().cpu().numpy().view(np.uint32)


def header_functions():
    """Names of every function declared in include/*.h."""
    names = []
    inc = os.path.join(ROOT, "include")
    for fn in sorted(os.listdir(inc)):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(inc, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        text = re.sub(r"#[^\n]*", "", text)
        for m in re.finditer(r"\b([A-Za-z_][A-Za-z0-9_]*)\s*\(([^;{}]*)\)\s*;", text):
            if m.group(1) not in ("sizeof",):
                names.append(m.group(1))
    return names
