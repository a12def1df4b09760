"""pasfm_step (Algorithm 1's Stage 1 / 4 / 5 updates: forward, loss head, adjoint,
pose gradient, Adam on p0 and on the frame twists with the left retraction)
against the FP64 oracle's composition of the same steps (``oracle.step``), on the
same seeded inputs, for three consecutive steps.

The GPU and the oracle each run their own trajectory from the same starting point;
after every step the test compares the loss at the pre-update point, the volume
and its Adam moments, and the poses and their moments.  Tolerances follow from the
operators' own bounds:

* the adjoint (volume gradient) is within REL_L2_SIG of the oracle, so the first
  moment m is too, and the second moment v (quadratic in g) within twice that;
* the pose gradient is within REL_L2_POSE per rotation / translation block, so
  the twist moments are too (v within twice that), and so is each frame's
  cumulative pose change;
* the loss L = 1/2 |r|^2 moves by at most |r| |ds| <= REL_L2_SIG |s| |r| when the
  forward s moves by |ds|;
* Adam divides by sqrt(v) + eps: where a gradient component is near zero its
  update would hinge on its rounding, so eps is set to a thousandth of the RMS
  volume gradient of the first step (computed by the oracle), which makes the
  update Lipschitz in g with constant lr / eps; every pose-gradient component of
  these cases is at least 0.6% of its block, far from zero.

Flags: the inlier mask of Eq. 4, the projection p0 >= 0, the gauge frame
(frame 0 fixed) and each of the two freezes are exercised.

The uniform sphere's pose gradient jumps where a sample boundary crosses a
sphere's edge, and the FP32 path places boundaries to ~3e-7 mm; on this case's
residual (which holds the volume's dense random background) such one-sided choices
move a frame's gradient by more than 1e-4.  Where poses are updated, each step's
inlier mask is then, for the sphere, the set of traces without a nonzero boundary
term within EPS_STRICT of an edge at the oracle's current state, so that every kept
trace has a single admissible gradient (the parity tests cover the band of the
others).  Both sides get the same mask.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import step as ostep
from paper_2604_09643_b300 import binding, synth
from tests.parity_cases import REL_L2_POSE, REL_L2_SIG, gaussian, ragged_case, rel_l2, tma_case

pytestmark = pytest.mark.gpu

EPS_STRICT = 1e-6  # mm; as in the parity tests

N_STEPS = 3
CASES = {"sphere_ragged": ragged_case, "gauss_tma": gaussian(tma_case, 0.05)}
MODES = {
    # joint update with the inlier mask, the non-negativity projection and the gauge frame
    "joint_mask_nonneg_fix0": dict(nonneg=True, fix_frame0=True, masked=True),
    "volume_only": dict(freeze_poses=True, masked=False),
    "poses_only": dict(freeze_volume=True, fix_frame0=True, masked=True),
}


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _problem(make):
    geom, truth, elem, poses = make()
    meas = oracle.forward(geom, truth, oracle.element_positions(geom, elem, poses)).astype(np.float32)
    rng = np.random.default_rng(7)
    p0 = (0.5 * truth + rng.uniform(0, 0.01, truth.shape)).astype(np.float32)
    start = synth.perturb_poses(poses, np.random.default_rng(8), 0.3, 0.03, keep_first=True)
    mask = (np.random.default_rng(9).uniform(size=(geom["n_frames"], geom["n_elem"])) > 0.25).astype(np.uint8)
    return geom, elem, meas, p0, start, mask


@pytest.mark.parametrize("mode", sorted(MODES))
@pytest.mark.parametrize("case", sorted(CASES))
def test_step_matches_oracle_over_three_steps(cuda_device, case, mode):
    geom, elem, meas, p0, start, mask = _problem(CASES[case])
    opts = dict(MODES[mode])
    masked = opts.pop("masked")
    mask = mask if masked else None
    # eps: a thousandth of the first step's RMS volume gradient (oracle)
    xw = oracle.element_positions(geom, elem, start)
    _, g = oracle.loss(geom, oracle.forward(geom, p0, xw), meas, mask)
    eps = 1e-3 * float(np.sqrt(np.mean(oracle.adjoint(geom, g, xw) ** 2)))
    hyper = dict(lr_vol=1e-2, lr_rot=2e-4, lr_trans=2e-3, beta1=0.8, beta2=0.95, eps=eps)

    ost = ostep.AdamState.zeros(geom, **hyper, **opts)
    op0, oposes = p0.astype(np.float64), start.copy()

    gp0, gposes = _dev(p0), _dev(start)
    gelem, gmeas = _dev(elem), _dev(meas)
    adam = binding.AdamState(geom, "cuda", **hyper, **opts)
    L = torch.zeros((), dtype=torch.float64, device="cuda")
    F = geom["n_frames"]
    with binding.Context(0) as ctx:
        for k in range(1, N_STEPS + 1):
            xw_k = oracle.element_positions(geom, elem, oposes)
            s_ref = oracle.forward(geom, op0.astype(np.float32), xw_k)
            mask_k = mask
            if geom.get("kernel", "sphere") == "sphere" and not opts.get("freeze_poses"):
                _, g_k = oracle.loss(geom, s_ref, meas, mask)
                F_, E_ = geom["n_frames"], geom["n_elem"]
                _, _, n = oracle.element_gradient_bounds(geom, op0.astype(np.float32), g_k, xw_k,
                                                         np.arange(F_ * E_), EPS_STRICT, counts=True)
                # the clean rows are the inlier mask here (with the random one on top, a frame of
                # this 33-element case can lose all its traces)
                mask_k = (n == 0).reshape(F_, E_).astype(np.uint8)
                assert mask_k[1:].any(axis=1).all(), (case, mode, k)  # every moving frame keeps traces
            gmask = None if mask_k is None else _dev(mask_k)
            r_ref = s_ref - meas if mask_k is None else (s_ref - meas) * mask_k[:, :, None]
            op0, oposes, ost, Lref = ostep.gradient_step(geom, op0, oposes, elem, meas, mask_k, ost)
            ctx.step(geom, gp0, gposes, gelem, gmeas, adam, mask=gmask, loss_out=L)
            rc, bits = ctx.status()
            assert rc == 0 and bits == 0, (rc, bits)
            assert adam.step == ost.step == k
            tag = (case, mode, k)

            tolL = REL_L2_SIG * np.linalg.norm(s_ref) * np.linalg.norm(r_ref)
            assert abs(float(L) - Lref) <= tolL, (tag, float(L), Lref, tolL)

            got_p0 = gp0.cpu().numpy().astype(np.float64)
            if opts.get("freeze_volume"):
                assert np.array_equal(got_p0, p0.astype(np.float64)), tag
                assert not adam.m_vol.any() and not adam.v_vol.any(), tag
            else:
                assert rel_l2(got_p0, op0) < REL_L2_SIG, (tag, rel_l2(got_p0, op0))
                # the cumulative update itself, not only the parameter
                assert rel_l2(got_p0 - p0, op0 - p0) < REL_L2_POSE, (tag, rel_l2(got_p0 - p0, op0 - p0))
                assert rel_l2(adam.m_vol.cpu().numpy(), ost.m_vol) < REL_L2_SIG, tag
                assert rel_l2(adam.v_vol.cpu().numpy(), ost.v_vol) < 2 * REL_L2_SIG, tag
                if opts.get("nonneg"):
                    assert got_p0.min() >= 0.0 and (op0 == 0.0).any(), tag  # the projection is active

            got_pose = gposes.cpu().numpy()
            if opts.get("freeze_poses"):
                assert np.array_equal(got_pose, start), tag
                assert not adam.m_pose.any() and not adam.v_pose.any(), tag
                continue
            mp, vp = adam.m_pose.cpu().numpy(), adam.v_pose.cpu().numpy()
            worst = max(rel_l2(mp[f, blk], ost.m_pose[f, blk]) for f in range(F) for blk in (slice(0, 3), slice(3, 6))
                        if not (f == 0 and opts.get("fix_frame0")))
            print(f"{case} {mode} step {k}: worst twist first-moment error {worst:.2e}")
            for f in range(F):
                for blk in (slice(0, 3), slice(3, 6)):
                    assert rel_l2(mp[f, blk], ost.m_pose[f, blk]) < REL_L2_POSE, (tag, f, blk)
                    assert rel_l2(vp[f, blk], ost.v_pose[f, blk]) < 2 * REL_L2_POSE, (tag, f, blk)
                if f == 0 and opts.get("fix_frame0"):
                    assert np.array_equal(got_pose[0], start[0]), tag  # the gauge frame does not move
                    continue
                assert rel_l2(got_pose[f] - start[f], oposes[f] - start[f]) < REL_L2_POSE, (tag, f)
