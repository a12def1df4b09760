"""One gradient step of the Eq. 2 data term, composed from the oracle's pieces
(test infrastructure only).

Algorithm 1 updates the volume (Stages 1 and 5) and the rigid frame parameters
(Stage 4) by gradient steps on L = 1/2 |mask (A(p0; poses) - S)|^2; the paper's
optimiser is Adam.  ``gradient_step`` evaluates, in this order and at the
pre-update point:

1. element positions x_fj = R_f e_j + t_f (``element_positions``);
2. the forward s = A(p0; poses) (``forward``);
3. the loss head g = mask (s - S), L = 1/2 sum g^2 (``loss``);
4. the volume gradient A^T g (``adjoint``) unless the volume is frozen, and the
   twist gradient (w, v) of every frame (``pose_grad``) unless the poses are
   frozen;
5. Adam on the twists with the left retraction (``adam.adam_poses``; frame 0 is
   not moved when it is the gauge) and Adam on the volume (``adam.adam_volume``,
   optionally projected onto p0 >= 0).

Frozen parts keep their parameters and their moments untouched.  The step count
k is the number of the step being taken (1 for the first).  The volume is held
in FP64 between steps; the forward and the pose gradient read it as the FP32
input array they take.

Parity status: composed only of pinned functions (the operator pins, the
closed-form Adam pins of ``adam.py`` and the retraction pins of ``rigid.py``).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import adam as _adam
from . import adjoint, element_positions, forward, loss, pose_grad


@dataclasses.dataclass
class AdamState:
    m_vol: np.ndarray
    v_vol: np.ndarray
    m_pose: np.ndarray
    v_pose: np.ndarray
    step: int = 0
    lr_vol: float = 1e-3
    lr_rot: float = 1e-4
    lr_trans: float = 1e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    nonneg: bool = False
    fix_frame0: bool = False
    freeze_poses: bool = False
    freeze_volume: bool = False

    @classmethod
    def zeros(cls, geom, **kw):
        nvox = int(geom["nx"]) * int(geom["ny"]) * int(geom["nz"])
        F = int(geom["n_frames"])
        return cls(np.zeros(nvox), np.zeros(nvox), np.zeros((F, 6)), np.zeros((F, 6)), **kw)

    def copy(self):
        return dataclasses.replace(self, m_vol=self.m_vol.copy(), v_vol=self.v_vol.copy(),
                                   m_pose=self.m_pose.copy(), v_pose=self.v_pose.copy())


def gradient_step(geom, p0, poses, elem, meas, mask, state: AdamState):
    """Returns (p0', poses', state', L at the pre-update point)."""
    p0 = np.asarray(p0, dtype=np.float64)
    poses = np.asarray(poses, dtype=np.float64)
    st = state.copy()
    xw = element_positions(geom, elem, poses)
    s = forward(geom, p0.astype(np.float32), xw)
    L, g = loss(geom, s, meas, mask)
    k = st.step + 1
    st.step = k
    p_out, pose_out = p0.copy(), poses.copy()
    if not st.freeze_poses:
        grad6, _ = pose_grad(geom, p0.astype(np.float32), g, xw)
        fixed = np.zeros(len(poses), dtype=bool)
        if st.fix_frame0 and len(poses):
            fixed[0] = True
        pose_out, st.m_pose, st.v_pose, _ = _adam.adam_poses(
            poses, grad6, st.m_pose, st.v_pose, k, st.lr_rot, st.lr_trans, st.beta1, st.beta2, st.eps, fixed)
    if not st.freeze_volume:
        vgrad = adjoint(geom, g, xw).reshape(-1)
        flat, st.m_vol, st.v_vol = _adam.adam_volume(p0.reshape(-1), vgrad, st.m_vol, st.v_vol, k, st.lr_vol,
                                                     st.beta1, st.beta2, st.eps, st.nonneg)
        p_out = flat.reshape(p0.shape)
    return p_out, pose_out, st, L
