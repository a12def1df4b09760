"""TGV regulariser on the GPU (through the C ABI) against the FP64 oracle of oracle/tgv.py."""
import numpy as np
import pytest
import torch

from oracle import tgv as otgv
from paper_2604_09643_b300 import binding, synth
from tests.parity_cases import REL_L2_SIG, rel_l2

pytestmark = pytest.mark.gpu

A1, A0, EPS = 0.8, 0.3, 0.05


def _case(shape, spacing, seed):
    geom = synth.make_geom(shape, spacing, 1, 1, 16)
    rng = np.random.default_rng(seed)
    u = rng.uniform(0, 1, size=shape).astype(np.float32)
    w = rng.normal(0, 3.0, size=(3,) + tuple(shape)).astype(np.float32)
    return geom, u, w


# shapes: TMA path (nx % 4 == 0) over several tiles; ragged non-TMA path; a single partial tile
CASES = [((20, 24, 64), 0.1, 1), ((13, 22, 37), (0.12, 0.1, 0.15), 2), ((3, 2, 5), 0.2, 3)]


@pytest.mark.parametrize("shape,spacing,seed", CASES)
def test_tgv_matches_oracle(cuda_device, shape, spacing, seed):
    geom, u, w = _case(shape, spacing, seed)
    sp = (geom["dx"], geom["dy"], geom["dz"])
    J, gu, gw = otgv.energy_and_grad(u, w, sp, A1, A0, EPS)
    with binding.Context(0) as ctx:
        e, gu_d, gw_d = ctx.tgv_grad(geom, torch.tensor(u, device="cuda"), torch.tensor(w, device="cuda"),
                                     A1, A0, EPS)
        assert ctx.status() == (0, 0)
    assert abs(float(e) - J) <= 1e-6 * abs(J)
    assert rel_l2(gu_d.cpu().numpy(), gu) < REL_L2_SIG
    assert rel_l2(gw_d.cpu().numpy(), gw) < REL_L2_SIG


def test_tgv_accumulates_and_reads_16bit_volumes(cuda_device):
    geom, u, w = _case((16, 20, 48), 0.1, 4)
    ub = torch.tensor(u, device="cuda").to(torch.bfloat16)
    ur = ub.float().cpu().numpy()
    _, gu, gw = otgv.energy_and_grad(ur, w, (0.1, 0.1, 0.1), A1, A0, EPS)
    base = np.random.default_rng(5).normal(size=u.shape).astype(np.float32)
    with binding.Context(0) as ctx:
        acc = torch.tensor(base, device="cuda")
        _, acc, gw_d = ctx.tgv_grad(geom, ub, torch.tensor(w, device="cuda"), A1, A0, EPS, grad_u=acc,
                                    accumulate=True)
    assert rel_l2(acc.cpu().numpy() - base, gu) < REL_L2_SIG
    assert rel_l2(gw_d.cpu().numpy(), gw) < REL_L2_SIG


def test_tgv_step_adds_the_regulariser(cuda_device):
    """pasfm_step_tgv = pasfm_step's data gradient + the TGV gradient, then Adam on p0
    and w: checked against the same composition of separate calls and a host Adam."""
    s = synth.single_frame()
    geom, p0, elem, poses = s.geom, s.p0, s.elem, s.poses
    rng = np.random.default_rng(6)
    w0 = rng.normal(0, 1.0, size=(3,) + p0.shape).astype(np.float32)
    init = (0.5 * p0 + 0.05).astype(np.float32)
    lr_vol, lr_w = 1e-2, 5e-3
    with binding.Context(0) as ctx:
        T = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
        meas = ctx.forward(geom, T(p0), T(elem), T(poses))
        # reference: separate calls
        sig = ctx.forward(geom, T(init), T(elem), T(poses))
        _, g = ctx.loss(geom, sig, meas)
        gvol = ctx.adjoint(geom, T(elem), T(poses), g)
        _, gvol, gw = ctx.tgv_grad(geom, T(init), T(w0), A1, A0, EPS, grad_u=gvol, accumulate=True)
        # fused step
        p = T(init)
        adam = binding.AdamState(geom, "cuda", lr_vol=lr_vol, freeze_poses=True)
        st = binding.TgvState(geom, "cuda", A1, A0, EPS, lr_w=lr_w, w=T(w0))
        ctx.step(geom, p, T(poses), T(elem), meas, adam, tgv=st)
        assert ctx.status() == (0, 0)
    # first Adam step: x - lr g / (|g| + eps) with eps = 1e-8
    ref_p = init - lr_vol * gvol.cpu().numpy() / (np.abs(gvol.cpu().numpy()) + 1e-8)
    ref_w = w0 - lr_w * gw.cpu().numpy() / (np.abs(gw.cpu().numpy()) + 1e-8)
    assert np.abs(p.cpu().numpy() - ref_p).max() < 1e-5
    assert np.abs(st.w.cpu().numpy() - ref_w).max() < 1e-5
