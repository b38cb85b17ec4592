"""Helpers for the GPU parity tests: torch device buffers around the C ABI."""
import numpy as np
import torch


def dev(x, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def f32(x):
    """Round to FP32 and back: the exact values the GPU receives."""
    return np.asarray(x, dtype=np.float32).astype(np.float64)
