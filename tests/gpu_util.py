"""Helpers for the GPU parity tests (no solver arithmetic here)."""
import numpy as np
import pytest


def lib_or_skip():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_05395_gb300 import build
    build.build()
    import paper_2107_05395_gb300 as sb
    return sb, torch


def relerr_per_system(x, ref):
    """e_m = ||x_m - ref_m||_2 / ||ref_m||_2 per system (absolute where ref_m = 0)."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    num = np.linalg.norm(x - ref, axis=0)
    den = np.linalg.norm(ref, axis=0)
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), num)


def to_dev(a, torch, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def to_host(t):
    return t.detach().cpu().numpy()
