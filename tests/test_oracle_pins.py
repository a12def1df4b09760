"""The FP64 oracle against closed forms, identities and finite differences (CPU)."""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import adam, rigid
from tests import oracle_checks as oc


def test_pulse_exact_closed_form():
    assert oc.check_closed_form() < 1e-12


def test_pulse_quadrature():
    assert oc.check_quadrature() < 1e-9


def test_pulse_derivative_fd():
    assert oc.check_pulse_dd() < 1e-6


def test_point_sampling_flag():
    assert oc.check_point_sampling() < 1e-13


def test_voxel_layout_and_superposition():
    assert oc.check_superposition() < 1e-12


def test_adjoint_identity():
    assert oc.check_adjoint_identity() < 1e-12


def test_rigid_invariance():
    assert oc.check_rigid_invariance() < 1e-12


def test_pose_gradient_fd():
    rot, trans, elem = oc.check_pose_fd()
    assert rot < 1e-6 and trans < 1e-6 and elem < 1e-6, (rot, trans, elem)


def test_pose_gradient_fd_masked():
    rot, trans, elem = oc.check_pose_fd(use_mask=True, seed=11)
    assert rot < 1e-6 and trans < 1e-6 and elem < 1e-6, (rot, trans, elem)


@pytest.mark.parametrize("sigma", [None, 0.06])
def test_volume_gradient_fd(sigma):
    assert oc.check_p0_gradient_fd(sigma=sigma) < 1e-9


# ---- Gaussian kernel (Eq. 1, Appendix A Eq. gaussian_far_field)

def test_gauss_pulse_solves_the_wave_equation():
    inside, outside = oc.check_wave_equation_gauss()
    assert inside < 1e-8          # far-field form = exact solution at r >= 3 mm, sigma <= 0.08 mm
    assert outside < 2.3e-3       # what the 4-sigma truncation drops: 4 exp(-7.5) of the peak


def test_gauss_pulse_quadrature():
    assert oc.check_quadrature_gauss() < 1e-9


def test_gauss_pulse_derivative_fd():
    assert oc.check_pulse_dd(gauss=True) < 1e-6


def test_gauss_adjoint_identity_and_rigid_invariance():
    assert oc.check_adjoint_identity(sigma=0.06) < 1e-12
    assert oc.check_rigid_invariance(sigma=0.06) < 1e-12


@pytest.mark.parametrize("use_mask", [False, True])
def test_gauss_pose_gradient_fd(use_mask):
    rot, trans, elem = oc.check_pose_fd(sigma=0.06, use_mask=use_mask, seed=11 if use_mask else 9)
    assert rot < 1e-6 and trans < 1e-6 and elem < 1e-6


def test_big_ball_converges_to_pi_over_6():
    r2, l2_coarse = oc.check_big_ball(spacing=0.2)
    r1, l2_fine = oc.check_big_ball(spacing=0.1)
    assert abs(r1 - 1.0) < 0.02, r1
    assert l2_fine < 0.06, l2_fine
    assert l2_fine < l2_coarse, (l2_fine, l2_coarse)


def test_loss_head():
    assert oc.check_loss() < 1e-14


# ---------------------------------------------------------------- rigid / Adam

def test_so3_exp_matches_expm():
    rng = np.random.default_rng(0)
    for _ in range(20):
        w = rng.normal(size=3) * rng.uniform(1e-9, 3.0)
        ref = scipy.linalg.expm(rigid.skew(w))
        assert np.abs(rigid.so3_exp(w) - ref).max() < 1e-13


def _horn(P, Q):
    """Quaternion (Horn 1987) least-squares rotation, independent of the SVD route."""
    pc, qc = P.mean(0), Q.mean(0)
    S = (P - pc).T @ (Q - qc)
    Sxx, Sxy, Sxz, Syx, Syy, Syz, Szx, Szy, Szz = S.ravel()
    N = np.array([[Sxx + Syy + Szz, Syz - Szy, Szx - Sxz, Sxy - Syx],
                  [Syz - Szy, Sxx - Syy - Szz, Sxy + Syx, Szx + Sxz],
                  [Szx - Sxz, Sxy + Syx, -Sxx + Syy - Szz, Syz + Szy],
                  [Sxy - Syx, Szx + Sxz, Syz + Szy, -Sxx - Syy + Szz]])
    w, V = np.linalg.eigh(N)
    q0, qx, qy, qz = V[:, -1]
    R = np.array([[q0 * q0 + qx * qx - qy * qy - qz * qz, 2 * (qx * qy - q0 * qz), 2 * (qx * qz + q0 * qy)],
                  [2 * (qy * qx + q0 * qz), q0 * q0 - qx * qx + qy * qy - qz * qz, 2 * (qy * qz - q0 * qx)],
                  [2 * (qz * qx - q0 * qy), 2 * (qz * qy + q0 * qx), q0 * q0 - qx * qx - qy * qy + qz * qz]])
    return R, qc - R @ pc


def test_kabsch_exact_and_matches_horn():
    rng = np.random.default_rng(1)
    P = rng.normal(size=(12, 3)) * 3
    R = rigid.so3_exp(rng.normal(size=3))
    t = rng.normal(size=3) * 5
    Rk, tk = rigid.kabsch(P, P @ R.T + t)
    assert np.abs(Rk - R).max() < 1e-12 and np.abs(tk - t).max() < 1e-12
    Q = P @ R.T + t + 0.05 * rng.normal(size=P.shape)
    Rk, tk = rigid.kabsch(P, Q)
    Rh, th = _horn(P, Q)
    assert np.abs(Rk - Rh).max() < 1e-10 and np.abs(tk - th).max() < 1e-10


def test_ransac_rejects_outliers():
    rng = np.random.default_rng(2)
    tmpl = np.stack(np.meshgrid(np.arange(5), np.arange(5), indexing="ij"), -1).reshape(-1, 2) * 0.6
    tmpl = np.concatenate([tmpl, np.zeros((25, 1))], axis=1)
    R = rigid.so3_exp([0.1, -0.2, 0.3])
    t = np.array([1.0, 2.0, 8.0])
    obs = tmpl @ R.T + t
    bad = rng.choice(25, size=6, replace=False)
    obs[bad] += rng.normal(size=(6, 3)) * 2.0
    subsets = [rng.choice(25, size=3, replace=False) for _ in range(200)]
    Rr, tr, mask, k = rigid.ransac_consensus(tmpl, obs, subsets, edge_tol=0.05, inlier_tol=0.1)
    truth = np.ones(25, dtype=bool)
    truth[bad] = False
    assert k >= 0 and np.array_equal(mask, truth)
    assert np.abs(Rr - R).max() < 1e-12 and np.abs(tr - t).max() < 1e-12


def test_adam_first_step_is_signed_lr():
    rng = np.random.default_rng(3)
    p = rng.normal(size=100)
    g = rng.normal(size=100)
    out, m, v = adam.adam_volume(p, g, np.zeros(100), np.zeros(100), 1, lr=0.01, eps=0.0)
    assert np.abs(out - (p - 0.01 * np.sign(g))).max() < 1e-15
    # projected variant clips at zero
    out2, _, _ = adam.adam_volume(p, g, np.zeros(100), np.zeros(100), 1, lr=0.01, eps=0.0, nonneg=True)
    assert np.all(out2 >= 0) and np.allclose(out2, np.maximum(out, 0))


def test_adam_pose_first_step_moves_by_signed_lr():
    poses = np.tile(np.eye(3, 4), (3, 1, 1))
    poses[:, 2, 3] = 10.0
    g6 = np.array([[1, -2, 3, -4, 5, -6], [0.5, 0.5, -0.5, 1, 1, 1], [1, 1, 1, 1, 1, 1]], float)
    out, m, v, dxi = adam.adam_poses(poses, g6, np.zeros((3, 6)), np.zeros((3, 6)), 1,
                                     lr_rot=1e-3, lr_trans=1e-2, eps=0.0,
                                     fixed=np.array([0, 0, 1], bool))
    expect = -np.sign(g6) * np.array([1e-3] * 3 + [1e-2] * 3)
    assert np.abs(dxi - expect).max() < 1e-15
    assert np.array_equal(out[2], poses[2])
    E = scipy.linalg.expm(rigid.skew(expect[0, :3]))
    assert np.abs(out[0][:, :3] - E).max() < 1e-14
    assert np.abs(out[0][:, 3] - (E @ poses[0, :, 3] + expect[0, 3:])).max() < 1e-13
    assert math.isclose(np.linalg.det(out[1][:, :3]), 1.0, rel_tol=1e-14)


# Multi-step Adam pins.  Adam (Kingma and Ba 2015, Algorithm 1) keeps
# m_k = b1 m_{k-1} + (1 - b1) g_k and v_k = b2 v_{k-1} + (1 - b2) g_k^2 from zero and
# steps by -lr m_k / (1 - b1^k) / sqrt(v_k / (1 - b2^k)) (eps = 0).  For the gradient
# sequences below the moments are geometric sums with closed forms:
#  - constant g:        m_k = (1 - b1^k) g, v_k = (1 - b2^k) g^2, so every step is -lr sign(g);
#  - alternating g, -g: m_2 = -(1 - b1)^2 g, m_3 = (1 - b1)(1 - b1 + b1^2) g, v_k = (1 - b2^k) g^2,
#    so step 2 is +lr (1 - b1) / (1 + b1) sign(g) and step 3 -lr (1 - b1 + b1^2) / (1 + b1 + b1^2) sign(g);
#  - g then 0:          m_2 = b1 (1 - b1) g, v_2 = b2 (1 - b2) g^2, so step 2 is
#    -lr [b1 / (1 + b1)] / sqrt(b2 / (1 + b2)) sign(g).
# The last one separates b1 from b2; the first needs the bias corrections at every k
# and v built from g^2 (|g| != 1).
ADAM_B1, ADAM_B2 = 0.8, 0.95


def _adam_seq(grads, lr=0.1, b1=ADAM_B1, b2=ADAM_B2):
    """Parameter after each step of the volume Adam on one scalar, from 0."""
    p, m, v, out = np.zeros(1), np.zeros(1), np.zeros(1), []
    for k, g in enumerate(grads, start=1):
        p, m, v = adam.adam_volume(p, np.array([g]), m, v, k, lr=lr, b1=b1, b2=b2, eps=0.0)
        out.append(float(p[0]))
    return np.diff(np.concatenate([[0.0], out]))  # the steps


def test_adam_constant_gradient_steps_by_lr_every_step():
    for g in (3.0, -0.25):
        steps = _adam_seq([g] * 4)
        assert np.abs(steps - (-0.1 * np.sign(g))).max() < 1e-14


def test_adam_alternating_gradient_closed_form():
    b1 = ADAM_B1
    steps = _adam_seq([2.0, -2.0, 2.0])
    assert abs(steps[0] + 0.1) < 1e-15
    assert abs(steps[1] - 0.1 * (1 - b1) / (1 + b1)) < 1e-14
    assert abs(steps[2] + 0.1 * (1 - b1 + b1 * b1) / (1 + b1 + b1 * b1)) < 1e-14


def test_adam_gradient_then_zero_separates_the_betas():
    b1, b2 = ADAM_B1, ADAM_B2
    steps = _adam_seq([-5.0, 0.0])
    assert abs(steps[1] - 0.1 * (b1 / (1 + b1)) / math.sqrt(b2 / (1 + b2))) < 1e-14


def test_adam_pose_moments_follow_the_same_closed_forms():
    """The twist Adam keeps per-component moments like the volume's; rotation and
    translation take their own rates."""
    b1, b2 = ADAM_B1, ADAM_B2
    poses = np.tile(np.eye(3, 4), (1, 1, 1))
    m, v = np.zeros((1, 6)), np.zeros((1, 6))
    seq = [np.array([[2.0, -5.0, 1.5, -2.0, -5.0, 0.7]]), np.array([[-2.0, 0.0, 1.5, 2.0, 0.0, 0.7]])]
    dxis = []
    for k, g6 in enumerate(seq, start=1):
        poses, m, v, dxi = adam.adam_poses(poses, g6, m, v, k, lr_rot=1e-3, lr_trans=1e-2, b1=b1, b2=b2, eps=0.0)
        dxis.append(dxi[0])
    lr = np.array([1e-3] * 3 + [1e-2] * 3)
    alt = (1 - b1) / (1 + b1)
    zero = (b1 / (1 + b1)) / math.sqrt(b2 / (1 + b2))
    expect2 = lr * np.array([alt, zero, -1.0, -alt, zero, -1.0])
    assert np.abs(dxis[0] - (-lr * np.sign(seq[0][0]))).max() < 1e-17
    assert np.abs(dxis[1] - expect2).max() < 1e-16


def test_retraction_closed_forms():
    """The left retraction of the twist (w, v): about z by theta the rotation is
    [[c, -s, 0], [s, c, 0], [0, 0, 1]] applied on the left of both R and t; a pure
    translation adds v to t and leaves R alone."""
    rng = np.random.default_rng(8)
    pose = np.zeros((3, 4))
    pose[:, :3] = rigid.so3_exp(rng.normal(size=3))
    pose[:, 3] = rng.normal(size=3) * 4
    th = 0.3
    Rz = np.array([[math.cos(th), -math.sin(th), 0.0], [math.sin(th), math.cos(th), 0.0], [0.0, 0.0, 1.0]])
    out = rigid.apply_twist(pose, [0.0, 0.0, th, 0.0, 0.0, 0.0])
    assert np.abs(out[:, :3] - Rz @ pose[:, :3]).max() < 1e-15
    assert np.abs(out[:, 3] - Rz @ pose[:, 3]).max() < 1e-14
    v = np.array([0.1, -0.2, 0.3])
    out = rigid.apply_twist(pose, np.concatenate([np.zeros(3), v]))
    assert np.array_equal(out[:, :3], pose[:, :3]) and np.abs(out[:, 3] - (pose[:, 3] + v)).max() < 1e-15


def test_adam_pose_fixed_frame_keeps_pose_but_updates_moments():
    poses = np.tile(np.eye(3, 4), (2, 1, 1))
    g6 = np.array([[1.0, 2, 3, 4, 5, 6], [1.0, 2, 3, 4, 5, 6]])
    out, m, v, _ = adam.adam_poses(poses, g6, np.zeros((2, 6)), np.zeros((2, 6)), 1, 1e-3, 1e-2,
                                   fixed=np.array([True, False]))
    assert np.array_equal(out[0], poses[0]) and not np.array_equal(out[1], poses[1])
    assert np.array_equal(m[0], m[1]) and np.array_equal(v[0], v[1]) and np.abs(m[0]).min() > 0


def test_kink_band_reduces_to_strict_gradient_and_contains_it():
    """The one-sided-ambiguity band of the element gradient: with eps = 0 it is the
    strict gradient; with eps > 0 it contains the strict value and its width grows
    with eps."""
    import oracle
    geom, elem, poses = oc.small_geom(shape=(6, 6, 6), spacing=0.2, m=3, n_frames=2, n_samples=320)
    rng = np.random.default_rng(30)
    p0 = rng.uniform(0.2, 1, size=(6, 6, 6)).astype(np.float32)
    g = rng.standard_normal((2, 9, 320))
    xw = oracle.element_positions(geom, elem, poses)
    rows = np.arange(18)
    strict = oracle.element_gradient_rows(geom, p0, g, xw, rows)
    mid0, half0 = oracle.element_gradient_bounds(geom, p0, g, xw, rows, 0.0)
    assert np.abs(mid0 - strict).max() <= 1e-13 * np.abs(strict).max() and half0.max() == 0.0
    mid1, half1 = oracle.element_gradient_bounds(geom, p0, g, xw, rows, 1e-3)
    mid2, half2, n2 = oracle.element_gradient_bounds(geom, p0, g, xw, rows, 5e-3, counts=True)
    assert np.all(np.abs(strict - mid1) <= half1 * (1 + 1e-12) + 1e-15)
    assert half2.sum() >= half1.sum() > 0.0
    # the count of ambiguous boundaries: none at eps = 0; a row without any has a
    # zero-width band centred on the strict gradient
    _, _, n0 = oracle.element_gradient_bounds(geom, p0, g, xw, rows, 0.0, counts=True)
    assert not n0.any() and n2.sum() > 0
    clean = n2 == 0
    assert np.all((half2[clean] == 0.0)) and np.all(half2[~clean].sum(axis=1) > 0.0)
    assert np.abs(mid2[clean] - strict[clean]).max(initial=0.0) <= 1e-13 * np.abs(strict).max()


def test_nc_loss_invariances():
    from oracle import nc as ncmod
    rng = np.random.default_rng(40)
    a = rng.standard_normal(500)
    b = rng.standard_normal(500)
    assert abs(ncmod.nc(a, a) + 1.0) < 1e-14
    assert abs(ncmod.nc(a, -a) - 1.0) < 1e-14
    assert abs(ncmod.nc(3.0 * a + 2.0, b - 5.0) - ncmod.nc(a, b)) < 1e-14
    assert abs(ncmod.nc(a, b) + np.corrcoef(a, b)[0, 1]) < 1e-14
    assert ncmod.nc(np.ones(10), a[:10]) == 0.0



def test_nc_gradient_pins():
    from oracle import nc as ncmod
    rng = np.random.default_rng(41)
    a = rng.standard_normal(300) + 0.3
    b = 0.5 * a + rng.standard_normal(300)
    g = ncmod.nc_grad(a, b)
    assert abs(g.sum()) < 1e-13 * np.abs(g).sum()          # offsets of sim do not change nc
    assert abs(np.dot(g, a)) < 1e-13 * np.abs(g * a).sum()  # nor does positive scaling
    h = 1e-6
    for n in rng.integers(0, 300, size=8):
        ap, am = a.copy(), a.copy()
        ap[n] += h
        am[n] -= h
        fd = (ncmod.nc(ap, b) - ncmod.nc(am, b)) / (2 * h)
        assert abs(fd - g[n]) < 1e-7 * np.abs(g).max()
    assert not ncmod.nc_grad(np.ones(10), a[:10]).any()


# ---- TGV regulariser (Stages 1 and 5, Eq. 2)

def test_tgv_matches_sparse_matrix_formulation():
    assert oc.check_tgv_sparse() < 1e-12


def test_tgv_gradient_fd():
    assert oc.check_tgv_fd() < 1e-7


def test_tgv_constant_field():
    assert oc.check_tgv_constant() < 1e-14
