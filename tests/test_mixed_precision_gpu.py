"""BF16 / FP16 storage of the volume and the signals (GPU).

Time of flight and accumulation stay FP32 and the pose-gradient reduction FP64;
only storage is 16-bit.  The kernel error is measured against the FP64 oracle
fed the same rounded inputs (relative L2 <= 1e-3 required; the FP32 tolerances
1e-5 / 1e-4 hold in practice and are asserted).  The end-to-end error against
unrounded inputs is dominated by the rounding itself (about 1e-3 for BF16,
1e-4 for FP16) and is checked to be of that order only.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2604_09643_b300 import binding
from tests.parity_cases import REL_L2_POSE, REL_L2_SIG, pose_residual, rel_l2, residual, tma_case

pytestmark = pytest.mark.gpu

DTYPES = {"bf16": torch.bfloat16, "f16": torch.float16}


def _rounded(a, dt):
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dt)
    return t, t.float().numpy()


@pytest.fixture(scope="module")
def setup(cuda_device):
    geom, p0, elem, poses = tma_case()
    xw = oracle.element_positions(geom, elem, poses)
    ctx = binding.Context(0)
    yield geom, p0, elem, poses, xw, ctx
    ctx.close()


@pytest.mark.parametrize("dt", sorted(DTYPES))
def test_forward_16bit_volume(setup, dt):
    geom, p0, elem, poses, xw, ctx = setup
    t16, p0r = _rounded(p0, DTYPES[dt])
    got = ctx.forward(geom, t16.cuda(), torch.tensor(elem).cuda(), torch.tensor(poses).cuda()).cpu().numpy()
    kern = rel_l2(got, oracle.forward(geom, p0r, xw))
    e2e = rel_l2(got, oracle.forward(geom, p0, xw))
    print(f"{dt} forward: kernel {kern:.2e}, end to end {e2e:.2e}")
    assert kern < REL_L2_SIG
    assert e2e < (1e-2 if dt == "bf16" else 1e-3)


@pytest.mark.parametrize("dt", sorted(DTYPES))
def test_adjoint_16bit_signals(setup, dt):
    geom, p0, elem, poses, xw, ctx = setup
    g = residual(geom, seed=51)
    g16, gr = _rounded(g, DTYPES[dt])
    got = ctx.adjoint(geom, torch.tensor(elem).cuda(), torch.tensor(poses).cuda(), g16.cuda()).cpu().numpy()
    kern = rel_l2(got, oracle.adjoint(geom, gr, xw))
    print(f"{dt} adjoint: kernel {kern:.2e}, end to end {rel_l2(got, oracle.adjoint(geom, g, xw)):.2e}")
    assert kern < REL_L2_SIG


@pytest.mark.parametrize("dt", sorted(DTYPES))
def test_pose_grad_16bit_storage(setup, dt):
    geom, p0, elem, poses, xw, ctx = setup
    p16, p0r = _rounded(p0, DTYPES[dt])
    g16, gr = _rounded(pose_residual(geom, p0r, elem, poses), DTYPES[dt])
    got = ctx.pose_grad(geom, p16.cuda(), torch.tensor(elem).cuda(), torch.tensor(poses).cuda(),
                        g16.cuda()).cpu().numpy()
    ref, _ = oracle.pose_grad(geom, p0r, gr, xw)
    full, _ = oracle.pose_grad(geom, p0, pose_residual(geom, p0, elem, poses), xw)
    worst = lambda r, blk: max(rel_l2(got[f, blk], r[f, blk]) for f in range(geom["n_frames"]))
    print(f"{dt} pose gradient: kernel rotation {worst(ref, slice(0, 3)):.2e} translation "
          f"{worst(ref, slice(3, 6)):.2e}; end to end rotation {worst(full, slice(0, 3)):.2e} "
          f"translation {worst(full, slice(3, 6)):.2e}")
    for f in range(geom["n_frames"]):
        assert rel_l2(got[f, :3], ref[f, :3]) < REL_L2_POSE
        assert rel_l2(got[f, 3:], ref[f, 3:]) < REL_L2_POSE


@pytest.mark.parametrize("dt", sorted(DTYPES))
def test_step_16bit_storage(setup, dt):
    """One pasfm_step with 16-bit volume and measurements: the loss at the starting
    point matches the oracle on the rounded inputs, the volume stays 16-bit."""
    geom, p0, elem, poses, xw, ctx = setup
    p16, p0r = _rounded(p0, DTYPES[dt])
    m16, mr = _rounded(0.8 * oracle.forward(geom, p0, xw), DTYPES[dt])
    p = p16.cuda().clone()
    L = torch.zeros((), dtype=torch.float64, device="cuda")
    adam = binding.AdamState(geom, "cuda", lr_vol=1e-3, freeze_poses=True)
    ctx.step(geom, p, torch.tensor(poses).cuda(), torch.tensor(elem).cuda(), m16.cuda(), adam, loss_out=L)
    torch.cuda.synchronize()
    Lref, _ = oracle.loss(geom, oracle.forward(geom, p0r, xw), mr)
    assert abs(float(L) - Lref) <= 1e-5 * Lref
    assert p.dtype == DTYPES[dt] and torch.isfinite(p.float()).all()
    assert ctx.status()[0] == 0
