"""pasfm_pose_grad_noalloc: the pose gradient for callers that must not allocate device
memory while they run (a host application that owns all device memory in its own
pool, a real-time loop that cannot take cudaMalloc's latency and implicit sync).

It keeps its scratch in one fixed in-library device array instead of a context
workspace, so it is checked here against the context-based pasfm_pose_grad on
the same inputs, twice in a row (the second call reuses whatever the first one
left in the shared scratch), within the pose-gradient tolerance of the other
parity tests.  This file is collected last so that a run that stops at the
first failure has already run every other test; it also passes on its own.
"""
import numpy as np
import pytest
import torch

from paper_2604_09643_b300 import binding, synth
from tests.parity_cases import REL_L2_POSE, gaussian, rel_l2, residual, tma_case

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _single_frame():
    s = synth.single_frame()
    return s.geom, s.p0, s.elem, s.poses


def _near_limit():
    """64^3 voxels (64 cubes), 16 x 16 elements, 160 frames: 61.9 MiB of the 64 MiB scratch."""
    s = synth.full_scan(n=64, n_tubes=10, m=16, n_frames=160, n_samples=1024)
    return s.geom, s.p0, s.elem, s.poses


@pytest.mark.parametrize("make_case", [_single_frame, tma_case, gaussian(_single_frame, 0.08), _near_limit],
                         ids=["single_frame", "tma", "gauss_single_frame", "near_scratch_limit"])
def test_noalloc_matches_context_pose_grad_on_two_calls(cuda_device, make_case):
    geom, p0, elem, poses = make_case()
    g = residual(geom, seed=41)
    mask = (np.random.default_rng(42).uniform(size=(geom["n_frames"], geom["n_elem"])) > 0.2).astype(np.uint8)
    dp0, delem, dpose, dg, dmask = _dev(p0), _dev(elem), _dev(poses), _dev(g), _dev(mask)
    F, E = geom["n_frames"], geom["n_elem"]
    with binding.Context(0) as ctx:
        ref6, refG = ctx.pose_grad(geom, dp0, delem, dpose, dg, dmask, want_elem=True)
        ref6, refG = ref6.cpu().numpy(), refG.cpu().numpy()
    for call in range(2):
        g6 = torch.full((F, 6), float("nan"), dtype=torch.float64, device="cuda")
        gE = torch.full((F, E, 3), float("nan"), dtype=torch.float64, device="cuda") if call == 0 else None
        binding.pasfm_pose_grad_noalloc(geom, dp0, delem, dpose, dg, dmask, g6, gE)
        torch.cuda.synchronize()
        got6 = g6.cpu().numpy()
        for f in range(F):
            assert rel_l2(got6[f, :3], ref6[f, :3]) < REL_L2_POSE, (call, f)
            assert rel_l2(got6[f, 3:], ref6[f, 3:]) < REL_L2_POSE, (call, f)
        if gE is not None:
            assert rel_l2(gE.cpu().numpy(), refG) < REL_L2_POSE


def test_noalloc_rejects_problems_beyond_its_scratch(cuda_device):
    geom = synth.make_geom((128, 128, 128), 0.1, 256, 64, 2048)  # 202 MB of scratch needed
    z = torch.zeros(1, device="cuda")
    g6 = torch.zeros((geom["n_frames"], 6), dtype=torch.float64, device="cuda")
    with pytest.raises(binding.PasfmError) as e:
        binding.pasfm_pose_grad_noalloc(geom, z, z.double(), z.double(), z, None, g6)
    assert e.value.code == -6 and "scratch" in str(e.value)


def test_noalloc_reports_a_device_side_failure_as_nan(cuda_device):
    """With no context status word, an element within the pulse support of the grid
    (the array plane through the volume) turns the outputs into NaN; the next call
    on a valid geometry is correct again (the status word in the scratch is cleared)."""
    geom, p0, elem, poses = _single_frame()
    bad = poses.copy()
    bad[0, 2, 3] = 0.0
    g = residual(geom, seed=43)
    F, E = geom["n_frames"], geom["n_elem"]
    g6 = torch.zeros((F, 6), dtype=torch.float64, device="cuda")
    gE = torch.zeros((F, E, 3), dtype=torch.float64, device="cuda")
    binding.pasfm_pose_grad_noalloc(geom, _dev(p0), _dev(elem), _dev(bad), _dev(g), None, g6, gE)
    torch.cuda.synchronize()
    assert torch.isnan(g6).all() and torch.isnan(gE).all()
    with binding.Context(0) as ctx:
        ref6 = ctx.pose_grad(geom, _dev(p0), _dev(elem), _dev(poses), _dev(g)).cpu().numpy()
    binding.pasfm_pose_grad_noalloc(geom, _dev(p0), _dev(elem), _dev(poses), _dev(g), None, g6)
    torch.cuda.synchronize()
    got = g6.cpu().numpy()
    assert rel_l2(got[0, :3], ref6[0, :3]) < REL_L2_POSE and rel_l2(got[0, 3:], ref6[0, 3:]) < REL_L2_POSE
