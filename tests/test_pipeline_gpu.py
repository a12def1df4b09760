"""The PA-SFM pipeline (Algorithm 1, Stages 1-5) end to end on the GPU."""
import numpy as np
import pytest

from paper_2604_09643_b300 import binding, pipeline, synth

pytestmark = pytest.mark.gpu


def test_two_view_bowl_recovers_view_b(cuda_device):
    """64^3 at 0.2 mm at the centre of a 512-element half of a 60 mm hemispherical
    bowl; view B turned 90 deg with a prior 1.3 mm off (mean element error)."""
    scan = synth.two_view_scan(n=64, spacing=0.2)
    with binding.Context(0) as ctx:
        res, p0, poses = pipeline.run(ctx, scan, pipeline.PipelineConfig())
        assert ctx.status() == (0, 0)
    assert res["prior_element_error_mm"] > 1.0
    assert res["stages2to4"]["stage2_within_inlier_tol"] > 0.9
    assert res["stages2to4"]["stage3_element_error_mm"] < 0.05
    assert res["final_element_error_mm"] < 0.01
    assert res["stage5"]["mip_psnr_db"] > res["stage1"]["mip_psnr_db"]
    assert poses.shape == (2, 3, 4) and np.allclose(poses[0], scan.poses[0])


def test_three_views_of_a_sparse_cap_array(cuda_device):
    """33 elements on a 40-degree spherical cap at 60 mm, three views 30 deg apart,
    located against a 0.4 mm reference map."""
    scan = synth.two_view_scan(n=32, spacing=0.4, elem=synth.cap_array(33), n_views=3, view_b_deg=30.0)
    cfg = pipeline.PipelineConfig(stage1_steps=1500, search_radius_mm=2.0, inlier_tol_mm=0.5, edge_tol_mm=0.5,
                                  top_k=8)
    with binding.Context(0) as ctx:
        res, _, poses = pipeline.run(ctx, scan, cfg)
        assert ctx.status() == (0, 0)
    assert res["prior_element_error_mm"] > 1.0
    assert min(res["stages2to4"]["stage3_inliers"]) >= 25
    assert res["final_element_error_mm"] < 0.02
    assert poses.shape == (3, 3, 4)
