"""Coarse-to-fine optimiser on the GPU: level resampling and pose recovery."""
import numpy as np
import pytest
import scipy.ndimage
import torch

from paper_2604_09643_b300 import binding, optim, synth
from tests.parity_cases import rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("src_n,dst_n", [(12, 24), (24, 17), (16, 16)])
def test_resample_matches_scipy_trilinear(cuda_device, src_n, dst_n):
    fine = synth.make_geom((24, 24, 24), 0.1, 1, 1, 1)
    gs = optim.level_geometry(fine, (src_n, src_n + 2, src_n + 4))
    gd = optim.level_geometry(fine, (dst_n, dst_n + 1, dst_n + 3))
    src = np.random.default_rng(5).uniform(size=(src_n, src_n + 2, src_n + 4)).astype(np.float32)
    with binding.Context(0) as ctx:
        got = ctx.resample(gs, torch.tensor(src, device="cuda"), gd).cpu().numpy()
    zz, yy, xx = np.meshgrid(*[(gd["o" + a] + gd["d" + a] * np.arange(gd["n" + a]) - gs["o" + a]) / gs["d" + a]
                               for a in "zyx"], indexing="ij")
    ref = scipy.ndimage.map_coordinates(src.astype(np.float64), [zz, yy, xx], order=1, mode="nearest")
    assert np.abs(got - ref).max() < 1e-6


@pytest.mark.parametrize("sigma", [0.0, 0.7, 2.5, 6.0])
def test_lowpass_matches_scipy(cuda_device, sigma):
    sig = np.random.default_rng(6).standard_normal((3, 5, 301)).astype(np.float32)
    with binding.Context(0) as ctx:
        got = ctx.lowpass(torch.tensor(sig, device="cuda"), sigma).cpu().numpy()
        inplace = torch.tensor(sig, device="cuda")
        ctx.lowpass(inplace, sigma, out=inplace)
    ref = sig.astype(np.float64) if sigma == 0 else scipy.ndimage.gaussian_filter1d(
        sig.astype(np.float64), sigma, axis=-1, mode="constant", truncate=4.0)
    assert np.abs(got - ref).max() < 1e-5
    assert np.array_equal(inplace.cpu().numpy(), got)


@pytest.mark.parametrize("decim", [2, 3, 4])
def test_lowpass_decimates(cuda_device, decim):
    sig = np.random.default_rng(7).standard_normal((2, 3, 301)).astype(np.float32)
    with binding.Context(0) as ctx:
        got = ctx.lowpass(torch.tensor(sig, device="cuda"), 1.7, decim=decim).cpu().numpy()
    ref = scipy.ndimage.gaussian_filter1d(sig.astype(np.float64), 1.7, axis=-1, mode="constant", truncate=4.0)
    assert got.shape == (2, 3, -(-301 // decim))
    assert np.abs(got - ref[..., ::decim]).max() < 1e-5


def test_nc_scores_match_oracle(cuda_device):
    from oracle import nc as ncmod
    rng = np.random.default_rng(8)
    meas = rng.standard_normal((12, 777)).astype(np.float32)
    sim = (0.3 * meas[None] + rng.standard_normal((5, 12, 777))).astype(np.float32)
    sim[2, 3] = 1.0  # zero-variance trace scores 0
    mask = (rng.uniform(size=12) > 0.3).astype(np.uint8)
    with binding.Context(0) as ctx:
        got = ctx.nc_scores(torch.tensor(sim, device="cuda"), torch.tensor(meas, device="cuda")).cpu().numpy()
        gotm = ctx.nc_scores(torch.tensor(sim, device="cuda"), torch.tensor(meas, device="cuda"),
                             torch.tensor(mask, device="cuda")).cpu().numpy()
    assert np.abs(got - ncmod.nc_scores(sim, meas)).max() < 1e-6
    assert np.abs(gotm - ncmod.nc_scores(sim, meas, mask)).max() < 1e-6


def _small_scan():
    n, sp, F = 48, 0.2, 12
    geom = synth.make_geom((n, n, n), sp, 64, F, 1024)
    p0 = synth.vessel_tree_phantom(geom, 12, np.random.default_rng(7), radius=(0.1, 0.4))
    elem = synth.planar_array(8, 8, 0.8)
    truth = synth.sweep_poses(F, 0.6, synth.top_face_z(geom) + 4.0, np.random.default_rng(8))
    return geom, p0, elem, truth


def test_pose_only_recovery_is_exact_inside_the_basin(cuda_device):
    geom, p0, elem, truth = _small_scan()
    init = synth.perturb_poses(truth, np.random.default_rng(9), 0.1, 0.02, keep_first=True)
    with binding.Context(0) as ctx:
        T = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
        meas = ctx.forward(geom, T(p0), T(elem), T(truth))
        poses = T(init)
        adam = binding.AdamState(geom, "cuda", lr_rot=5e-4, lr_trans=5e-3, fix_frame0=True, freeze_volume=True)
        for _ in range(200):
            ctx.step(geom, T(p0), poses, T(elem), meas, adam)
        err = optim.element_errors(elem, poses.cpu().numpy(), truth)
    assert optim.element_errors(elem, init, truth) > 0.03 and err < 1e-3


def test_joint_coarse_to_fine_recovers_poses_below_a_voxel(cuda_device):
    """Unknown volume and poses 0.33 mm off (mean element error): coarse level with
    band-limited data, NC grid search, joint refinement, fine level."""
    geom, p0, elem, truth = _small_scan()
    init = synth.perturb_poses(truth, np.random.default_rng(9), 1.0, 0.2, keep_first=True)
    cfg = optim.C2FConfig(levels=((24, 24, 24), (48, 48, 48)), steps=(150, 200), lr_vol=0.02, lr_rot=1e-3,
                          lr_trans=1e-2, lr_decay=0.5, search_rounds=1, search_radius_mm=0.8, search_step_mm=0.1,
                          search_joint_steps=150)
    with binding.Context(0) as ctx:
        T = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
        meas = ctx.forward(geom, T(p0), T(elem), T(truth))
        vol, poses, hist = optim.reconstruct(ctx, geom, elem, meas, init, cfg, truth_poses=truth)
    e0 = optim.element_errors(elem, init, truth)
    assert e0 > 0.3
    assert hist[-1]["mean_element_error_mm"] < 0.02, hist  # voxel = 0.2 mm


def test_gaussian_kernel_annealing_recovers_poses(cuda_device):
    """Gaussian kernel (Eq. 1) end to end: traces simulated with sigma = 0.08 mm on a
    64^3 grid at 0.1 mm, 12 frames, 8x8 elements; poses perturbed by 1.5 deg / 0.3 mm
    (0.49 mm mean element error).  Two levels (32^3 on a 2x coarser time grid, then
    64^3) with the kernel width decaying 0.24 -> 0.16 and 0.12 -> 0.08 mm."""
    n, F = 64, 12
    geom = synth.make_geom((n, n, n), 0.1, 64, F, 1536, kernel="gauss", sigma=0.08)
    p0 = synth.vessel_tree_phantom(geom, 12, np.random.default_rng(7), radius=(0.1, 0.4))
    elem = synth.planar_array(8, 8, 0.8)
    truth = synth.sweep_poses(F, 0.4, synth.top_face_z(geom) + 4.0, np.random.default_rng(8))
    init = synth.perturb_poses(truth, np.random.default_rng(9), 1.5, 0.3, keep_first=True)
    with binding.Context(0) as ctx:
        T = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
        meas = ctx.forward(geom, T(p0), T(elem), T(truth))
        cfg = optim.C2FConfig(levels=((32, 32, 32), (64, 64, 64)), steps=(200, 200), lr_vol=0.02, lr_rot=1e-3,
                              lr_trans=1e-2, lr_decay=0.5, sigma_schedule=((0.24, 0.16), (0.12, 0.08)))
        _, poses, hist = optim.reconstruct(ctx, geom, elem, meas, init, cfg, truth_poses=truth)
        assert ctx.status() == (0, 0)
    assert optim.element_errors(elem, init, truth) > 0.45
    assert [h["time_decimation"] for h in hist] == [2, 1]
    assert hist[-1]["kernel_sigma_mm"] == 0.08
    assert hist[-1]["mean_element_error_mm"] < 0.01


def test_nc_grad_matches_oracle(cuda_device):
    from oracle import nc as ncmod
    rng = np.random.default_rng(12)
    R, T = 40, 777
    meas = rng.standard_normal((R, T)).astype(np.float32)
    sim = (0.6 * meas + 0.8 * rng.standard_normal((R, T)) + 0.2).astype(np.float32)
    sim[3] = 1.5  # zero variance: gradient 0, NC 0
    mask = (rng.uniform(size=R) > 0.25).astype(np.uint8)
    with binding.Context(0) as ctx:
        d = lambda a: torch.tensor(a, device="cuda")
        g, nc = ctx.nc_grad(d(sim), d(meas), d(mask), scale=2.0)
        alias = d(sim)
        ctx.nc_grad(alias, d(meas), d(mask), scale=2.0, out=alias)
    g, nc = g.cpu().numpy(), nc.cpu().numpy()
    ref = np.stack([2.0 * ncmod.nc_grad(sim[r], meas[r]) * mask[r] for r in range(R)])
    ref_nc = np.array([ncmod.nc(sim[r], meas[r]) * mask[r] for r in range(R)])
    assert rel_l2(g, ref) < 1e-5
    assert np.abs(nc - ref_nc).max() < 1e-6
    assert not g[3].any() and nc[3] == 0.0
    assert np.array_equal(alias.cpu().numpy(), g)


def test_nc_grad_pairs_each_measured_trace_with_repeated_candidates(cuda_device):
    from oracle import nc as ncmod
    rng = np.random.default_rng(13)
    E, K, T = 5, 7, 300
    meas = rng.standard_normal((E, T)).astype(np.float32)
    sim = (0.5 * np.repeat(meas, K, axis=0) + rng.standard_normal((E * K, T))).astype(np.float32)
    with binding.Context(0) as ctx:
        d = lambda a: torch.tensor(a, device="cuda")
        g, nc = ctx.nc_grad(d(sim), d(meas), meas_repeat=K)
        x = d(sim[0].copy())
        ctx.scale(x, -2.5)
    ref = np.stack([ncmod.nc_grad(sim[r], meas[r // K]) for r in range(E * K)])
    assert rel_l2(g.cpu().numpy(), ref) < 1e-5
    assert np.abs(nc.cpu().numpy() - [ncmod.nc(sim[r], meas[r // K]) for r in range(E * K)]).max() < 1e-6
    assert np.array_equal(x.cpu().numpy(), (sim[0] * np.float32(-2.5)).astype(np.float32))
