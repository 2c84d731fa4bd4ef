"""Helpers shared by the GPU tests (no test cases here)."""
import numpy as np
import torch

DEV = torch.device("cuda:0")


def dt(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def npy(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def max_rel(a, b):
    """max |a - b| / max |b|"""
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
