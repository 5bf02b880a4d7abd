"""Helpers shared by the GPU parity tests (device buffers through torch; the solver runs in
libtobk.so).  Nothing here computes any part of the method."""
import numpy as np
import pytest


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1909_13585_gb300 as pkg
    pkg.load()
    return torch, pkg


def to_dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel_err(a, b):
    a = np.asarray(a); b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
