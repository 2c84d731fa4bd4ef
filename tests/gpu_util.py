"""Helpers shared by the GPU tests (no test cases here)."""
import numpy as np
import torch

DEV = torch.device("cuda:0")


def dt(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def npy(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def max_rel(a, b, floor=1e-300):
    """max |a - b| / max(max |b|, floor).  The floor matters only when every
    reference value is far below the physical scale (e.g. all weights
    underflow: FP32 exp flushes below 2^-126 where FP64 does not)."""
    return float(np.abs(a - b).max() / max(np.abs(b).max(), floor))


def phi_floor(p, sigma):
    """1e-12 of the natural size of Phi, |p|^2 / sigma."""
    return 1e-12 * float(np.abs(p).max()) ** 2 / sigma


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
