"""Textbook Adam steps for the volume and the per-frame twists (test infrastructure only).

Adam (Kingma and Ba) is the optimiser the paper uses for the Stage 1 / Stage 5
objective (Eq. 2) and, by its Algorithm 1, for the rigid parameters of Stage 4.
Parameters: m <- b1 m + (1-b1) g; v <- b2 v + (1-b2) g^2;
theta <- theta - lr (m / (1-b1^k)) / (sqrt(v / (1-b2^k)) + eps) at step k >= 1.

For the twists the update is a twist dxi = -lr m_hat / (sqrt(v_hat) + eps),
applied on the left of the current pose and then reset to zero (the pose is
re-based every step, so the gradient is always taken at xi = 0); rotation and
translation components have their own learning rates because their units
differ (rad, mm).  Frames flagged fixed (the gauge frame) are not moved.  The
optional non-negativity projection of the volume follows the paper's remark
that photoacoustic initial pressures are positive.

Pinned by closed forms of the moment recurrences (geometric sums, eps = 0):
the first step moves every parameter by exactly -lr sign(g); a constant
gradient keeps doing so at every step (bias corrections); alternating +-g gives
steps lr (1-b1)/(1+b1) and -lr (1-b1+b1^2)/(1+b1+b1^2) at k = 2, 3; g then 0
gives -lr [b1/(1+b1)] / sqrt(b2/(1+b2)) at k = 2 (separates b1 from b2); a fixed
frame keeps its pose while its moments advance.  Planted mistakes (swapped
betas, |g| in place of g^2, missing or frozen bias corrections, swapped
rotation and translation rates, a right-hand retraction) each fail one of these.
"""
from __future__ import annotations

import numpy as np

from .rigid import apply_twist


def adam_volume(p0, grad, m, v, k, lr, b1=0.9, b2=0.999, eps=1e-8, nonneg=False):
    p0 = np.asarray(p0, dtype=np.float64)
    grad = np.asarray(grad, dtype=np.float64)
    m = b1 * np.asarray(m, dtype=np.float64) + (1 - b1) * grad
    v = b2 * np.asarray(v, dtype=np.float64) + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** k)
    vh = v / (1 - b2 ** k)
    out = p0 - lr * mh / (np.sqrt(vh) + eps)
    if nonneg:
        out = np.maximum(out, 0.0)
    return out, m, v


def adam_poses(poses, grad6, m, v, k, lr_rot, lr_trans, b1=0.9, b2=0.999, eps=1e-8,
               fixed=None):
    poses = np.asarray(poses, dtype=np.float64)
    grad6 = np.asarray(grad6, dtype=np.float64)
    m = b1 * np.asarray(m, dtype=np.float64) + (1 - b1) * grad6
    v = b2 * np.asarray(v, dtype=np.float64) + (1 - b2) * grad6 * grad6
    mh = m / (1 - b1 ** k)
    vh = v / (1 - b2 ** k)
    lr = np.array([lr_rot] * 3 + [lr_trans] * 3)
    dxi = -lr * mh / (np.sqrt(vh) + eps)
    out = poses.copy()
    for f in range(len(poses)):
        if fixed is not None and fixed[f]:
            continue
        out[f] = apply_twist(poses[f], dxi[f])
    return out, m, v, dxi
