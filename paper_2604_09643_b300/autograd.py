"""torch.autograd binding of the radiation operator (Section 2: the forward and
backward operators wrapped as a torch.autograd.Function so that gradients flow
to the source intensity P_c and to the sensor coordinates).

``radiate(p0, xi, base_pose, elem, geom, context)`` returns the traces
s = A(p0; Exp(xi) * base_pose) (float32 [F][E][Nt]).  The per-frame pose is the
base pose with the left twist xi = (w, v) applied (R <- Exp(w) R,
t <- Exp(w) t + v), so optimising xi moves every element of a frame rigidly,
the kinematic constraint of Stage 4.  Backward:

* dL/dp0 = A^T g              (pasfm_adjoint, at the twisted poses);
* dL/dxi = J_l(w)^T (g_w - v x g_v), g_v   (pasfm_pose_grad, then pasfm_twist_grad).

The time of flight is recomputed from the poses in every call; no system matrix
is stored.  Every step runs in the CUDA library; this module only wires calls.
"""
from __future__ import annotations

import torch

from . import binding


class Radiation(torch.autograd.Function):
    @staticmethod
    def forward(fctx, p0, xi, base_pose, elem, geom, context):
        posed = context.apply_twists(base_pose.contiguous(), xi.detach().contiguous())
        sig = context.forward(geom, p0.detach().contiguous(), elem, posed)
        fctx.save_for_backward(p0.detach(), xi.detach(), posed, elem)
        fctx.geom = geom
        fctx.context = context
        return sig

    @staticmethod
    def backward(fctx, gsig):
        p0, xi, posed, elem = fctx.saved_tensors
        ctx, geom = fctx.context, fctx.geom
        g = gsig.detach().to(torch.float32).contiguous()
        gp0 = gxi = None
        if fctx.needs_input_grad[0]:
            gp0 = ctx.adjoint(geom, elem, posed, g).to(p0.dtype)
        if fctx.needs_input_grad[1]:
            g6 = ctx.pose_grad(geom, p0.contiguous(), elem, posed, g)
            gxi = ctx.twist_grad(xi.contiguous(), g6)
        return gp0, gxi, None, None, None, None


def radiate(p0, xi, base_pose, elem, geom, context: binding.Context):
    """Differentiable traces for volume p0 [nz][ny][nx] and frame twists xi [F][6]."""
    return Radiation.apply(p0, xi, base_pose, elem, geom, context)
