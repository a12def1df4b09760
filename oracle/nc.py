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


def nc_grad(sim, meas):
    """d nc(sim, meas) / d sim.  With s~ and m~ the centred traces and
    rho = <s~, m~> / (|s~| |m~|), the centring drops out of the derivative (the
    centred traces sum to zero) and
        d nc / d sim_n = -(m~_n / |m~| - rho s~_n / |s~|) / |s~|.
    Zero for a trace with zero variance (where nc is defined as 0).  Pinned by
    central differences of nc and by the invariances of nc: the gradient sums to
    zero (offsets) and is orthogonal to sim (positive scaling)."""
    s = np.asarray(sim, dtype=np.float64)
    m = np.asarray(meas, dtype=np.float64)
    s = s - s.mean()
    m = m - m.mean()
    ns, nm = np.sqrt((s * s).sum()), np.sqrt((m * m).sum())
    if ns == 0 or nm == 0:
        return np.zeros_like(s)
    rho = (s * m).sum() / (ns * nm)
    return -(m / nm - rho * s / ns) / ns


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
