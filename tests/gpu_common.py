"""Helpers shared by the GPU parity tests (imported by them only)."""
import numpy as np


def block_rel_err(gpu: np.ndarray, ref: np.ndarray, block_axes: int) -> float:
    """max over blocks of max|gpu - ref| / max|ref|, blocks being the leading `block_axes` axes (0/0 counts as 0)."""
    g = gpu.reshape(gpu.shape[:block_axes] + (-1,)).astype(np.float64)
    r = ref.reshape(ref.shape[:block_axes] + (-1,)).astype(np.float64)
    num = np.max(np.abs(g - r), axis=-1)
    den = np.max(np.abs(r), axis=-1)
    out = np.where(den > 0, num / np.where(den > 0, den, 1.0), np.where(num > 0, np.inf, 0.0))
    return float(np.max(out)) if out.size else 0.0


def ps_blocks(p: np.ndarray, l_max: int) -> np.ndarray:
    """[n_c, F] packed or full power spectrum -> [n_c, l_max+1, per_l] for per-(centre, l) blocks."""
    return p.reshape(p.shape[0], l_max + 1, -1)
