"""Binned (blocking) error estimates for correlated Monte Carlo series."""
import numpy as np


def mean_err(x, n_bins: int = 40):
    """Mean and its standard error from n_bins equal blocks of the series."""
    x = np.asarray(x, dtype=np.float64)
    m = len(x) // n_bins
    if m < 1:
        raise ValueError("series too short")
    blocks = x[: m * n_bins].reshape(n_bins, m).mean(axis=1)
    return float(blocks.mean()), float(blocks.std(ddof=1) / np.sqrt(n_bins))
