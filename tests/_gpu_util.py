"""Helpers shared by the GPU parity tests (no scheme arithmetic: marshalling and comparisons)."""
import numpy as np

TOL_FP64 = 1e-10      # relative max-norm, FP64 path vs oracle
TOL_MIXED = 1e-8      # relative max-norm, mixed path vs oracle
TIE = 1e-12


def torch_dev():
    import torch
    return torch.device("cuda:0")


def to_dev(a, dtype=None):
    import torch
    dtype = dtype or torch.float64
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=torch_dev())


def policies_agree(p_gpu, p_orc, V):
    """Identical policies except at near-ties: where they differ, the GPU's control value must
    be within the tie window of the oracle's choice (V: oracle control values, (K, N))."""
    p_gpu = np.asarray(p_gpu, dtype=np.int64)
    p_orc = np.asarray(p_orc, dtype=np.int64)
    diff = np.nonzero(p_gpu != p_orc)[0]
    if len(diff) == 0:
        return True, 0
    vg = V[p_gpu[diff], diff]
    vo = V[p_orc[diff], diff]
    ok = np.abs(vg - vo) <= 2 * TIE * np.maximum(1.0, np.abs(vo))
    return bool(np.all(ok)), len(diff)


def rel_maxnorm(a, b):
    return float(np.max(np.abs(a - b)) / max(1e-300, np.max(np.abs(b))))
