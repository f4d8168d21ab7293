"""Shared helpers of the GPU parity tests (not collected as tests)."""
import numpy as np
import torch


def to_dev(a, device=0):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64).cuda(device)


def to_np(t):
    return t.detach().cpu().numpy()


def projector_dist(P, Q):
    """||(I - Q Q^T) P||_2 for orthonormal P, Q of equal rank: the sine of the
    largest principal angle, i.e. ||P P^T - Q Q^T||_2.  Computed from the
    residual of projecting P onto range(Q), which keeps full relative accuracy
    for tiny angles (1 - cos^2 would not)."""
    return float(np.linalg.norm(P - Q @ (Q.T @ P), 2))


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
