"""Host-side pieces of the coarse-to-fine optimiser (CPU): pyramid geometry and the
Stage 3 rigid consensus against the oracle's independent Kabsch / RANSAC."""
import numpy as np
import pytest

from oracle import rigid
from paper_2604_09643_b300 import optim, synth


def test_level_geometry_keeps_the_world_box():
    g = synth.make_geom((256, 256, 256), 0.1, 256, 4, 2048)
    for n in (64, 128, 256):
        lg = optim.level_geometry(g, (n, n, n))
        for ax in "xyz":
            lo = lg["o" + ax] - 0.5 * lg["d" + ax]
            hi = lo + lg["n" + ax] * lg["d" + ax]
            assert abs(lo - (g["o" + ax] - 0.05)) < 1e-12 and abs(hi - (-lo)) < 1e-12
        assert abs(lg["a0_mm"] - 0.5 * 25.6 / n) < 1e-12
        # pi/6 fill factor of the inscribed sphere is level-invariant
        assert abs(4 / 3 * np.pi * lg["a0_mm"] ** 3 / lg["dx"] ** 3 - np.pi / 6) < 1e-12


def test_kabsch_matches_oracle():
    rng = np.random.default_rng(0)
    P = rng.normal(size=(20, 3))
    R = rigid.so3_exp(rng.normal(size=3))
    Q = P @ R.T + rng.normal(size=3) + 0.01 * rng.normal(size=(20, 3))
    w = rng.uniform(0.5, 2, size=20)
    r1, t1 = optim.kabsch(P, Q, w)
    r2, t2 = rigid.kabsch(P, Q, w)
    assert np.abs(r1 - r2).max() < 1e-12 and np.abs(t1 - t2).max() < 1e-12


def test_ransac_matches_oracle_on_the_same_subsets():
    rng = np.random.default_rng(1)
    tmpl = synth.planar_array(8, 8, 0.6)
    R = rigid.so3_exp([0.05, -0.1, 0.2])
    obs = tmpl @ R.T + np.array([0.3, -0.2, 9.0]) + 0.005 * rng.normal(size=(64, 3))
    bad = rng.choice(64, size=12, replace=False)
    obs[bad] += rng.normal(scale=0.5, size=(12, 3))
    subsets = [rng.choice(64, size=3, replace=False) for _ in range(100)]
    r1, t1, m1, k1 = optim.ransac(tmpl, obs, subsets, 0.05, 0.05)
    r2, t2, m2, k2 = rigid.ransac_consensus(tmpl, obs, subsets, 0.05, 0.05)
    assert k1 == k2 >= 0 and np.array_equal(m1, m2)
    assert np.abs(r1 - r2).max() < 1e-12 and np.abs(t1 - t2).max() < 1e-12
    assert not m1[bad].any()


def test_element_errors():
    poses = synth.sweep_poses(3, 0.3, 8.0, np.random.default_rng(2))
    elem = synth.planar_array(4, 4, 0.5)
    assert optim.element_errors(elem, poses, poses) == 0.0
    moved = poses.copy()
    moved[:, 0, 3] += 0.1
    assert abs(optim.element_errors(elem, poses, moved) - 0.1) < 1e-12


@pytest.mark.parametrize("d_coarse,decim,tol", [(0.2, 1, 2e-3), (0.2, 2, 2e-3), (0.4, 4, 1e-2)])
def test_gauss_level_transfer_keeps_the_signals(d_coarse, decim, tol):
    """A smooth source on a 0.1 mm grid of sigma = 0.08 mm Gaussians, its traces
    low-passed and decimated as the coarse-to-fine optimiser does, against the
    same source on a coarser grid (sigma scaled with the spacing, amplitudes
    rescaled, time grid decimated), both through the FP64 oracle."""
    import scipy.ndimage

    import oracle

    h = 1.5 / 40.0

    def traces(spacing, sigma, fs, nt):
        n = int(round(3.6 / spacing)) + 1
        geom = synth.make_geom((n, n, n), spacing, 1, 1, nt, kernel="gauss", sigma=sigma, fs=fs)
        geom["t0_us"] = 6.0 / 1.5
        x, y, z = synth.voxel_axes(geom)
        zz, yy, xx = np.meshgrid(z, y, x, indexing="ij")
        f = np.exp(-(xx ** 2 + yy ** 2 + zz ** 2) / (2 * 0.4 ** 2)).astype(np.float32)
        return oracle.forward(geom, f, np.array([[[0.7, -0.4, 10.0]]]))[0, 0]

    s_fine, s_coarse = 0.08, 0.08 * d_coarse / 0.1
    fine = traces(0.1, s_fine, 40.0, 400)
    coarse = traces(d_coarse, s_coarse, 40.0 / decim, -(-400 // decim))
    lp = optim.gauss_lowpass_samples(s_coarse, s_fine, h, decim)
    fine_lp = scipy.ndimage.gaussian_filter1d(fine, lp, mode="constant", truncate=6.0)[::decim]
    fac = optim.gauss_amplitude_factor(s_fine, 0.1, s_coarse, d_coarse)
    assert np.linalg.norm(fine_lp - fac * coarse) / np.linalg.norm(fine_lp) < tol


def test_time_decimation_factor():
    fine = synth.make_geom((64, 64, 64), 0.1, 4, 1, 100, kernel="gauss", sigma=0.05)
    cfg = optim.C2FConfig()
    for n, k in ((64, 1), (32, 2), (16, 4), (21, 2)):
        assert optim.time_decimation(fine, optim.level_geometry(fine, (n, n, n)), cfg) == k
    assert optim.time_decimation(synth.make_geom((64, 64, 64), 0.1, 4, 1, 100),
                                 optim.level_geometry(fine, (16, 16, 16)), cfg) == 1


def test_search_grids():
    """Full grid: every offset at step_mm within the radius.  Coarse to fine: 5-point
    grids whose spacing halves from radius / 2 down to step_mm, so the union of the
    nested grids reaches every offset of the full grid from the right centre, with
    far fewer candidates."""
    full = optim.search_grids(1.2, 0.15, False)
    assert len(full) == 1 and len(full[0]) == 17
    np.testing.assert_allclose(full[0][[0, -1]], [-1.2, 1.2])
    grids = optim.search_grids(1.2, 0.15, True)
    np.testing.assert_allclose([g[1] - g[0] for g in grids], [0.6, 0.3, 0.15])
    assert all(len(g) == 5 and abs(g[2]) < 1e-12 for g in grids)
    assert sum(len(g) ** 3 for g in grids) == 375
    # nested reach: the sum of one offset per level covers the full grid's span
    assert abs(sum(g[-1] for g in grids) - 2.1) < 1e-9
    # a radius already at the step: one 5-point grid at step_mm
    one = optim.search_grids(0.1, 0.1, True)
    assert len(one) == 1 and abs(one[0][1] - one[0][0] - 0.1) < 1e-12


def test_stage2_top_k_selection_deduplicates_and_pads():
    """Stage 2's coarse-to-fine search evaluates overlapping 3x3x3 neighbourhoods, so a
    position can appear several times; the Top-K keeps each once, best score first, and
    pads with the last distinct one when too few remain."""
    from paper_2604_09643_b300.pipeline import select_top
    a, b, c = np.array([0.0, 0, 0]), np.array([0.25, 0, 0]), np.array([0, 0.25, 0])
    cands = np.stack([b, a, c, a + 1e-9, b, c])
    scores = np.array([-0.5, -0.9, -0.1, -0.8, -0.5, -0.2])
    top = select_top(cands, scores, 4, distinct=True)
    assert np.allclose(top, [a, b, c, c])                        # a (twice), b (twice), c (twice): 3 distinct
    assert np.allclose(select_top(cands, scores, 2, distinct=True), [a, b])
    # without de-duplication the repeats stay, in score order
    assert np.allclose(select_top(cands, scores, 4), [a, a + 1e-9, b, b])
    # where the grids coincide (no repeats) both options give the same list
    uniq = np.stack([a, b, c])
    s3 = np.array([0.3, -0.1, 0.2])
    assert np.array_equal(select_top(uniq, s3, 3, distinct=True), select_top(uniq, s3, 3))
