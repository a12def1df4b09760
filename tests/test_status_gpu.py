"""Device-side failure reporting through the context's status word.

Every TMA-staged copy is awaited with a bounded wait.  The context's wait limit
(pasfm_set_wait_limit) set to 0 makes each such wait report PASFM_STATUS_TIMEOUT
at once; the kernels then skip their compute, let the copies in flight land with
the full bound and exit, and pasfm_status returns PASFM_ETIMEOUT.  Nothing faults
or hangs: the copies are ordinary in-bounds loads that complete within
microseconds.  Afterwards the default limit is restored and the same context
computes correct results again.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2604_09643_b300 import binding
from tests.parity_cases import REL_L2_POSE, REL_L2_SIG, pose_residual, rel_l2, residual, tma_case

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def test_wait_timeout_is_reported_and_the_context_recovers(cuda_device):
    geom, p0, elem, poses = tma_case()  # nx % 4 == 0, Nt % 4 == 0, FP32: every kernel stages with TMA
    g = residual(geom, seed=31)
    dp0, delem, dpose, dg = _dev(p0), _dev(elem), _dev(poses), _dev(g)
    w = torch.zeros((3,) + p0.shape, dtype=torch.float32, device="cuda")
    with binding.Context(0) as ctx:
        ctx.set_wait_limit(0)
        calls = {
            "forward": lambda: ctx.forward(geom, dp0, delem, dpose),
            "adjoint": lambda: ctx.adjoint(geom, delem, dpose, dg),
            "pose_grad": lambda: ctx.pose_grad(geom, dp0, delem, dpose, dg),
            "tgv_grad": lambda: ctx.tgv_grad(geom, dp0, w, 0.5, 0.2, 0.05),
        }
        for name, call in calls.items():
            call()
            rc, bits = ctx.status()
            assert rc == -4 and bits & binding.STATUS_TIMEOUT, (name, rc, bits)
            rc, bits = ctx.status()  # reading clears the word
            assert rc == 0 and bits == 0, (name, rc, bits)

        ctx.set_wait_limit(-1)  # back to the default bound
        xw = oracle.element_positions(geom, elem, poses)
        sig = ctx.forward(geom, dp0, delem, dpose).cpu().numpy()
        vol = ctx.adjoint(geom, delem, dpose, dg).cpu().numpy()
        gp = pose_residual(geom, p0, elem, poses)
        g6 = ctx.pose_grad(geom, dp0, delem, dpose, _dev(gp)).cpu().numpy()
        rc, bits = ctx.status()
        assert rc == 0 and bits == 0, (rc, bits)
    assert rel_l2(sig, oracle.forward(geom, p0, xw)) < REL_L2_SIG
    assert rel_l2(vol, oracle.adjoint(geom, g, xw)) < REL_L2_SIG
    ref6, _ = oracle.pose_grad(geom, p0, gp, xw)
    for f in range(geom["n_frames"]):
        assert rel_l2(g6[f, :3], ref6[f, :3]) < REL_L2_POSE and rel_l2(g6[f, 3:], ref6[f, 3:]) < REL_L2_POSE

