"""Rigid-body pieces of the oracle (test infrastructure only).

* ``so3_exp``: Rodrigues' formula for the exponential of a rotation vector.
  Pinned against ``scipy.linalg.expm`` of the skew matrix.
* ``apply_twist``: the left perturbation used for the per-frame pose
  parameters (reading of the Stage 4 rigid parameters as an se(3) twist):
  ``R <- Exp(w) R``, ``t <- Exp(w) t + v``, so every element moves as
  ``x <- Exp(w) x + v`` about the world origin.
* ``kabsch``: least-squares rotation and translation between matched point
  sets (Stage 3, "the Kabsch algorithm is applied to solve the rigid
  transformation").  Pinned by exact recovery of noise-free transforms and by an
  independent quaternion (Horn) solution written in the tests.
* ``ransac_consensus``: Stage 3's modified RANSAC: every candidate subset is
  first checked for pairwise edge lengths against the template (the geometric
  consistency pre-check), then fitted by Kabsch and scored by inlier count; the
  best hypothesis is refitted on its inliers.  The random subsets are inputs
  (drawn by the caller), so the result is deterministic.  Thresholds are not
  given by the paper; they are arguments.  Pinned by recovery with injected
  outliers.
"""
from __future__ import annotations

import numpy as np


def skew(w):
    w = np.asarray(w, dtype=np.float64)
    return np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])


def so3_exp(w) -> np.ndarray:
    w = np.asarray(w, dtype=np.float64)
    th = float(np.linalg.norm(w))
    K = skew(w)
    if th < 1e-12:
        return np.eye(3) + K + 0.5 * K @ K
    return np.eye(3) + np.sin(th) / th * K + (1.0 - np.cos(th)) / th ** 2 * K @ K


def apply_twist(pose, xi) -> np.ndarray:
    """pose [3][4] (or [F][3][4]) with twist xi = (w, v) applied on the left."""
    pose = np.asarray(pose, dtype=np.float64)
    xi = np.asarray(xi, dtype=np.float64)
    if pose.ndim == 3:
        return np.stack([apply_twist(p, x) for p, x in zip(pose, xi)])
    E = so3_exp(xi[:3])
    out = np.empty((3, 4))
    out[:, :3] = E @ pose[:, :3]
    out[:, 3] = E @ pose[:, 3] + xi[3:]
    return out


def kabsch(P, Q, weights=None):
    """(R, t) minimising sum_i w_i |R P_i + t - Q_i|^2, det R = +1."""
    P = np.asarray(P, dtype=np.float64)
    Q = np.asarray(Q, dtype=np.float64)
    w = np.ones(len(P)) if weights is None else np.asarray(weights, dtype=np.float64)
    w = w / w.sum()
    pc = (w[:, None] * P).sum(0)
    qc = (w[:, None] * Q).sum(0)
    H = ((P - pc) * w[:, None]).T @ (Q - qc)
    U, _, Vt = np.linalg.svd(H)
    D = np.diag([1.0, 1.0, np.sign(np.linalg.det(Vt.T @ U.T)) or 1.0])
    R = Vt.T @ D @ U.T
    return R, qc - R @ pc


def edges_consistent(template, observed, idx, tol) -> bool:
    """Pairwise distances within the subset agree with the template to ``tol`` mm."""
    for a in range(len(idx)):
        for b in range(a + 1, len(idx)):
            dt = np.linalg.norm(template[idx[a]] - template[idx[b]])
            do = np.linalg.norm(observed[idx[a]] - observed[idx[b]])
            if abs(dt - do) > tol:
                return False
    return True


def ransac_consensus(template, observed, subsets, edge_tol, inlier_tol):
    """Returns (R, t, inlier mask, index of the winning subset or -1)."""
    template = np.asarray(template, dtype=np.float64)
    observed = np.asarray(observed, dtype=np.float64)
    best, best_k, best_mask = -1, -1, None
    for k, idx in enumerate(subsets):
        idx = list(idx)
        if not edges_consistent(template, observed, idx, edge_tol):
            continue
        R, t = kabsch(template[idx], observed[idx])
        res = np.linalg.norm(template @ R.T + t - observed, axis=1)
        mask = res < inlier_tol
        cnt = int(mask.sum())
        if cnt > best:
            best, best_k, best_mask = cnt, k, mask
    if best_k < 0 or best < 3:
        return np.eye(3), np.zeros(3), np.zeros(len(template), dtype=bool), -1
    R, t = kabsch(template[best_mask], observed[best_mask])
    return R, t, best_mask, best_k
