"""Negative-correlation (NC) loss of Eq. 3, per trace, in FP64 (test infrastructure only).

L_NC(sim, meas) = -Cov(sim, meas) / (sigma_sim sigma_meas) for one sensor trace;
a candidate pose set is scored by the mean over its (unmasked) element traces.
A trace with zero variance scores 0.  Pinned in tests by its defining
invariances: -1 for a trace against itself, +1 against its negative, unchanged by
positive scaling and by offsets of either trace, and equal to numpy's
correlation coefficient (np.corrcoef) with the sign flipped.
"""
from __future__ import annotations

import numpy as np


def nc(sim, meas) -> float:
    s = np.asarray(sim, dtype=np.float64)
    m = np.asarray(meas, dtype=np.float64)
    s = s - s.mean()
    m = m - m.mean()
    den = np.sqrt((s * s).sum() * (m * m).sum())
    return float(-(s * m).sum() / den) if den > 0 else 0.0


def nc_scores(sim, meas, mask=None):
    """sim [K][E][Nt], meas [E][Nt] -> [K] mean NC over kept elements."""
    sim = np.asarray(sim)
    K, E, _ = sim.shape
    keep = np.ones(E, dtype=bool) if mask is None else np.asarray(mask).astype(bool)
    out = np.zeros(K)
    for k in range(K):
        vals = [nc(sim[k, j], meas[j]) for j in range(E) if keep[j]]
        out[k] = float(np.mean(vals)) if vals else 0.0
    return out
