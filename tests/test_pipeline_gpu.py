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
