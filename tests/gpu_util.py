"""Helpers shared by the GPU parity tests (marshalling and error norms only)."""
import numpy as np


def rel_l1(got, ref):
    """Per-variable relative L1 error sum|got - ref| / sum|ref| (absolute where ref is ~0)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    out = []
    for v in range(ref.shape[0]):
        den = np.abs(ref[v]).sum()
        num = np.abs(got[v] - ref[v]).sum()
        out.append(num / den if den > 1e-300 else num)
    return np.array(out)


def rel_max(got, ref):
    """Per-variable element-wise error max|got - ref| / max|ref| (absolute where ref is ~0): a wrong
    cell, a bad corner or a wrong ghost column shows here even when it is lost in a global L1 norm."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    out = []
    for v in range(ref.shape[0]):
        den = np.abs(ref[v]).max() if ref.shape[1] else 0.0
        num = np.abs(got[v] - ref[v]).max() if ref.shape[1] else 0.0
        out.append(num / den if den > 1e-300 else num)
    return np.array(out)


def to_device(Q, dtype):
    import torch

    t = torch.tensor(np.ascontiguousarray(Q), dtype=torch.float32 if dtype == 0 else torch.float64, device="cuda")
    return t


def rounded(Q, dtype):
    """The values the device sees: FP32 runs give the oracle the same rounded inputs."""
    return np.asarray(Q, dtype=np.float32).astype(np.float64) if dtype == 0 else np.asarray(Q, dtype=np.float64)
