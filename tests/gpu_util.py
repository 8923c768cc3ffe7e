"""Shared helpers for the GPU parity tests (CUDA path vs the CPU oracle)."""
import numpy as np


def bz_module():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2103_14890_gb300 import build, binding
    build.build()
    binding.load()
    return binding


def to_dev(a, precision):
    import torch
    dt = torch.float64 if precision == "fp64" else torch.float32
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)


def as_input(a, precision):
    """The exact values the device sees, in FP64 (the oracle gets the same)."""
    return a if precision == "fp64" else a.astype(np.float32).astype(np.float64)


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
