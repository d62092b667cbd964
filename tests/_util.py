import numpy as np


def rel_l2(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def max_rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def cuda(*arrs):
    import torch
    out = []
    for a in arrs:
        if a is None:
            out.append(None)
        else:
            a = np.ascontiguousarray(a)
            dt = torch.float64 if a.dtype.kind == "f" else (torch.int32 if a.dtype == np.int32 else torch.int64)
            out.append(torch.as_tensor(a, dtype=dt).cuda())
    return out
