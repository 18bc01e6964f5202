"""Helpers shared by the GPU parity tests: inputs from synth/, expected values
from oracle/, the device path through the C ABI binding."""
import json
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

_COEFFS = None


def coeffs(L):
    """w_1..w_L of the committed oracle-learned artefact."""
    global _COEFFS
    if _COEFFS is None:
        with open(os.path.join(GOLDEN, "ifnso_coeffs.json")) as f:
            _COEFFS = json.load(f)
    return np.array(_COEFFS["L"][str(L)]["w"])


def lib():
    from paper_2602_02500_gb300 import _build

    _build.build()
    from paper_2602_02500_gb300 import ifnso

    return ifnso


def to_dev(M, dtype):
    """Device copy of M; BF16 rows are padded to a multiple of 8 elements (the
    16-byte row pitch TMA needs) and the view of the first cols columns returned."""
    import torch

    M = np.asarray(M, dtype=np.float32)
    t = torch.tensor(M, device="cuda")
    if dtype != "bf16":
        return t
    r, c = M.shape
    ld = (c + 7) // 8 * 8
    buf = torch.zeros((r, ld), dtype=torch.bfloat16, device="cuda")
    buf[:, :c] = t.to(torch.bfloat16)
    return buf[:, :c]


def to_np(t):
    return t.float().double().cpu().numpy()


def rel(a, b):
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(np.asarray(a, dtype=np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def sym_upper(G, block=256):
    """The symmetric matrix a BF16 plan keeps on its upper block x block blocks
    (element (i, j) with i // block > j // block is read at (j, i))."""
    G = np.array(G, dtype=np.float64, copy=True)
    n = G.shape[0]
    bi = np.arange(n)[:, None] // block
    bj = np.arange(n)[None, :] // block
    low = bi > bj
    G[low] = G.T[low]
    return G


def block_max_rel(a, b, block=256):
    """Largest per-block relative Frobenius error over the block x block tiles
    of the output: ||a_t - b_t||_F / max(||b_t||_F, ||b||_F sqrt(|t| / |b|)).
    A tile whose reference is smaller than the average tile is measured
    against the average tile's norm, so that a wrong output tile (1/352 of a
    2048 x 5632 matrix) shows its own error instead of being averaged away."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    tot = np.linalg.norm(b)
    worst = 0.0
    for i in range(0, b.shape[0], block):
        for j in range(0, b.shape[1], block):
            bt = b[i:i + block, j:j + block]
            at = a[i:i + block, j:j + block]
            den = max(np.linalg.norm(bt), tot * np.sqrt(bt.size / b.size), 1e-300)
            worst = max(worst, float(np.linalg.norm(at - bt) / den))
    return worst
