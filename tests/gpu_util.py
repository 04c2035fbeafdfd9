"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import torch

# Tolerances on the relative L2 error against the FP64 oracle: FP32 paths
# 1e-5, FP64 paths 1e-12 (the parity bar of the method's north star).
TOL32 = 1e-5
TOL64 = 1e-12


def rel_l2(got, want) -> float:
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    den = np.linalg.norm(want.ravel())
    num = np.linalg.norm((got - want).ravel())
    return float(num / den) if den > 0 else float(num)


def rounded(x, dt):
    """The values the GPU sees, as FP64 arrays for the oracle."""
    return np.asarray(x, dtype=np.float32 if dt == torch.float32 else np.float64).astype(np.float64)


def dev(x, dt):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dt, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def tol(dt):
    return TOL32 if dt == torch.float32 else TOL64
