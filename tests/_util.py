"""Shared helpers of the GPU parity tests (no method arithmetic here)."""
import numpy as np


def rel_fro(got, ref) -> float:
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.linalg.norm(ref)
    if den == 0.0:
        return float(np.linalg.norm(got))
    return float(np.linalg.norm(got - ref) / den)


def to_np(t):
    return t.detach().cpu().numpy()
