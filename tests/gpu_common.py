"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2007_03847_gb300 as fmc
    fmc.build()
    return fmc


def normwise_rel(a, b):
    """max |a - b| / max |b| over the whole array."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (den if den > 0 else 1.0))


def traj_errors(gpu_traj, ref_traj, n):
    """Normwise relative error of delta and of omega, separately."""
    ed = normwise_rel(gpu_traj[..., :n], ref_traj[..., :n])
    ew = normwise_rel(gpu_traj[..., n:], ref_traj[..., n:])
    return ed, ew
