"""torch.autograd.Function over (p0, frame twists) against the oracle (GPU).

The volume gradient is compared with the oracle adjoint of the oracle residual;
the twist gradient with central finite differences of the oracle loss, the
twist being applied with scipy's matrix exponential (independent of both the
kernel's and the oracle's Rodrigues formulas).  Twists are large (0.2 rad,
0.3 mm) so that the left Jacobian of SO(3) in the chain rule matters.
"""
import math

import numpy as np
import pytest
import scipy.linalg
import torch

import oracle
from paper_2604_09643_b300 import binding, synth
from paper_2604_09643_b300.autograd import radiate
from tests.parity_cases import REL_L2_POSE, rel_l2

pytestmark = pytest.mark.gpu


def _twist(pose, xi):
    K = np.array([[0, -xi[2], xi[1]], [xi[2], 0, -xi[0]], [-xi[1], xi[0], 0]])
    E = scipy.linalg.expm(K)
    out = np.empty((3, 4))
    out[:, :3] = E @ pose[:, :3]
    out[:, 3] = E @ pose[:, 3] + xi[3:]
    return out


def _case(kernel="sphere"):
    geom = synth.make_geom((24, 28, 32), 0.1, 36, 2, 1024, kernel=kernel,
                           sigma=0.05 if kernel == "gauss" else None)
    rng = np.random.default_rng(60)
    p0 = synth.vessel_tree_phantom(geom, 8, rng) + rng.uniform(0, 0.05, size=(24, 28, 32)).astype(np.float32)
    elem = synth.planar_array(6, 6, 0.5)
    base = synth.sweep_poses(2, 0.4, synth.top_face_z(geom) + 4.0, np.random.default_rng(61))
    xi = np.array([[0.2, -0.1, 0.15, 0.3, -0.2, 0.1], [-0.12, 0.18, -0.05, -0.1, 0.25, -0.2]])
    truth = synth.perturb_poses(np.stack([_twist(base[f], xi[f]) for f in range(2)]),
                                np.random.default_rng(62), 0.4, 0.05, keep_first=False)
    meas = oracle.forward(geom, p0, oracle.element_positions(geom, elem, truth)).astype(np.float32)
    return geom, p0.astype(np.float32), elem, base, xi, meas


def _oracle_loss(geom, p0, elem, base, xi, meas):
    posed = np.stack([_twist(base[f], xi[f]) for f in range(len(base))])
    s = oracle.forward(geom, p0, oracle.element_positions(geom, elem, posed))
    r = s - meas
    return 0.5 * math.fsum((r * r).ravel()), r, posed


@pytest.mark.parametrize("kernel", ["sphere", "gauss"])
def test_autograd_gradients_match_oracle(cuda_device, kernel):
    geom, p0, elem, base, xi, meas = _case(kernel)
    with binding.Context(0) as ctx:
        tp0 = torch.tensor(p0, device="cuda", requires_grad=True)
        txi = torch.tensor(xi, device="cuda", requires_grad=True)
        sig = radiate(tp0, txi, torch.tensor(base, device="cuda"), torch.tensor(elem, device="cuda"), geom, ctx)
        loss = 0.5 * ((sig.double() - torch.tensor(meas, device="cuda").double()) ** 2).sum()
        loss.backward()
        gp0 = tp0.grad.cpu().numpy()
        gxi = txi.grad.cpu().numpy()
        assert ctx.status()[0] == 0
    L0, r, posed = _oracle_loss(geom, p0, elem, base, xi, meas)
    assert abs(float(loss.detach()) - L0) <= 1e-5 * L0
    ref_p0 = oracle.adjoint(geom, r, oracle.element_positions(geom, elem, posed))
    assert rel_l2(gp0, ref_p0) < 2e-5  # residual of two FP32 traces, then the adjoint
    # small step for the sphere: its loss is only piecewise smooth (support-edge
    # kinks), and a 1e-8 rad / mm step lets few pairs straddle a kink while FP64
    # round-off stays near 1e-6 relative; the Gaussian pulse is smooth up to its
    # e^-8 truncation
    eps = 1e-8 if kernel == "sphere" else 1e-6
    for f in range(2):
        fd = np.zeros(6)
        for k in range(6):
            xp, xm = xi.copy(), xi.copy()
            xp[f, k] += eps
            xm[f, k] -= eps
            fd[k] = (_oracle_loss(geom, p0, elem, base, xp, meas)[0]
                     - _oracle_loss(geom, p0, elem, base, xm, meas)[0]) / (2 * eps)
        assert rel_l2(gxi[f, :3], fd[:3]) < REL_L2_POSE, (f, gxi[f], fd)
        assert rel_l2(gxi[f, 3:], fd[3:]) < REL_L2_POSE, (f, gxi[f], fd)


def test_apply_twists_matches_expm(cuda_device):
    base = synth.sweep_poses(3, 0.4, 8.0, np.random.default_rng(63))
    xi = np.random.default_rng(64).normal(scale=0.5, size=(3, 6))
    xi[1, :3] = 1e-9  # near-zero rotation takes the series branch
    with binding.Context(0) as ctx:
        got = ctx.apply_twists(torch.tensor(base, device="cuda"), torch.tensor(xi, device="cuda")).cpu().numpy()
    ref = np.stack([_twist(base[f], xi[f]) for f in range(3)])
    assert np.abs(got - ref).max() < 1e-13
