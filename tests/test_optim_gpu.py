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
