"""Shared set-up for the GPU parity tests: the same seeded inputs on both sides.

Measurements y are formed by the FP64 checker and handed to the CUDA path, so
both sides see identical data; nothing flows from the CUDA path into the checker.
"""
from __future__ import annotations

import numpy as np
import torch

from paper_2412_08264_gb300 import api
from oracle.bilevel import BilevelProblem

DEV = torch.device("cuda:0")


def packed(arrs, dtype):
    return torch.tensor(np.concatenate([np.asarray(a).ravel() for a in arrs]), dtype=dtype, device=DEV)


def split(t: torch.Tensor, sizes):
    out, pos = [], 0
    a = t.double().cpu().numpy()
    for h, w in sizes:
        out.append(a[pos:pos + h * w].reshape(h, w))
        pos += h * w
    return out


def r32(a):
    """Round to FP32 and back: the checker then sees exactly the FP32 path's inputs."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def make(wl, precision="fp32", max_recycle=8, max_basis=40, oracle=None):
    wl.precision = precision
    prob = oracle or BilevelProblem(wl)
    dt = torch.float32 if precision == "fp32" else torch.float64
    if precision == "fp32":
        prob.ys = [r32(y) for y in prob.ys]
        for ll, y in zip(prob.lowers, prob.ys):
            ll.y = y
        prob.x_star = [r32(x) for x in prob.x_star]
    P = api.from_workload(wl, packed(prob.ys, dt), packed(wl.x_star, dt), max_recycle=max_recycle,
                          max_basis=max_basis, precision=precision)
    return P, prob, dt


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def max_elem(a, b):
    """Largest element-wise deviation relative to the largest reference magnitude: a bar on every
    element (tile seams, image borders), which a norm ratio over many elements can dilute."""
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
