"""Checks that pin the FP64 oracle to things other than itself.

Each ``check_*`` returns an error figure; ``test_oracle_pins.py`` asserts the
thresholds and ``test_oracle_mutants.py`` shows that oracle builds with planted
mistakes (a dropped term, a flipped sign, a transposed operand, a swapped index)
fail at least one of them.  Pins used:

* exact rational values of the Appendix A uniform-sphere closed form, averaged
  over each sample interval (``golden/pulse_worked_example.json``);
* numerical quadrature of the same continuous pulse at random distances;
* central finite differences of the pulse in the distance;
* the point-sample flag against the closed form evaluated at the sample time;
* voxel indexing and superposition: a few isolated voxels against the exact
  single-voxel values at distances computed from the documented grid layout;
* the adjoint identity <A x, y> = <x, A^T y>;
* invariance of every signal when one rigid motion moves volume and array;
* central finite differences of L = 1/2 |A(p0; poses) - S|^2 in the twist
  components and in the element positions;
* convergence of a voxelised ball to pi/6 times the ball's own closed-form pulse
  (each voxel sphere fills pi/6 of its cell).

For the Gaussian kernel (Eq. 1, Appendix A Eq. gaussian_far_field):

* the exact solution of the 3-D wave equation for a Gaussian initial pressure,
  from Poisson's spherical-means formula p = d/dt [t M(ct)] evaluated by
  numerical quadrature (no closed form involved), against the point-sampled
  pulse;
* quadrature of the truncated far-field pulse over each sample interval against
  the interval averages;
* central finite differences of the pulse in the distance;
* the adjoint identity, rigid invariance and loss finite differences as above.
"""
from __future__ import annotations

import importlib.util
import json
import math
import os
from fractions import Fraction as Fr

import numpy as np
import scipy.integrate
import scipy.linalg
import scipy.ndimage

import oracle
from paper_2604_09643_b300 import synth

_GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden_module():
    spec = importlib.util.spec_from_file_location(
        "make_pulse_worked_example", os.path.join(_GOLDEN, "make_pulse_worked_example.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _scalar_geom(c, fs, a0, t0, n_samples=100000, sigma=None):
    g = synth.make_geom((1, 1, 1), 1.0, 1, 1, n_samples, fs=float(fs), c=float(c),
                        a0=float(a0), t0=float(t0))
    if sigma is not None:
        g.update(kernel="gauss", sigma_mm=float(sigma))
    return g


GAUSS_TRUNC = 4.0  # support half-width in units of sigma (reading: the paper states none)


def _gauss_far_field(r, tau, sigma):
    """Outgoing Gaussian pulse at distance r and tau = c t, truncated at 4 sigma."""
    w = r - tau
    return w / (2 * r) * math.exp(-w * w / (2 * sigma * sigma)) if abs(w) <= GAUSS_TRUNC * sigma else 0.0


def _poisson_gauss(r, t, c, sigma):
    """Pressure at distance r, time t for p(x, 0) = exp(-|x|^2 / (2 sigma^2)),
    p_t(x, 0) = 0, from Poisson's formula p = d/dt [t M(ct)], with M(R) the mean of
    the initial field over the sphere of radius R about the observation point.
    M and dM/dR are integrated numerically over u = cos(polar angle)."""
    R = c * t
    f = lambda u: math.exp(-(r * r + R * R - 2 * r * R * u) / (2 * sigma * sigma))
    dfdR = lambda u: -(R - r * u) / (sigma * sigma) * f(u)
    # the integrand is concentrated near u = 1 when R ~ r; give quad the scale
    pts = [max(-1.0, 1.0 - (8 * sigma) ** 2 / max(2 * r * R, 1e-300))]
    M = 0.5 * scipy.integrate.quad(f, -1, 1, points=pts, epsabs=1e-15, epsrel=1e-12, limit=400)[0]
    dM = 0.5 * scipy.integrate.quad(dfdR, -1, 1, points=pts, epsabs=1e-15, epsrel=1e-12, limit=400)[0]
    return M + t * c * dM


def check_wave_equation_gauss(seed=12):
    """Returns (max |oracle - Poisson| / peak inside the 4-sigma support,
    max |Poisson| / peak outside it).  The point-sampled Gaussian pulse is the
    far-field form, which differs from the exact solution only by the inward
    wave (exp(-(r + ct)^2 / 2 sigma^2), nil at r >= 3 mm) and the truncation."""
    rng = np.random.default_rng(seed)
    c, fs = 1.5, 40.0
    inside, outside = 0.0, 0.0
    for _ in range(6):
        sigma = float(rng.choice([0.03, 0.05, 0.08]))
        r = float(rng.uniform(3.0, 12.0))
        t0 = float(rng.uniform(0.0, 0.3))
        geom = _scalar_geom(c, fs, 0.05, t0, sigma=sigma)
        peak = sigma / (2 * r) * math.exp(-0.5)
        h = c / fs
        n0 = int(math.floor((r - 6 * sigma - c * t0) / h))
        n1 = int(math.ceil((r + 6 * sigma - c * t0) / h))
        for n in range(n0, n1 + 1):
            t = t0 + n / fs
            exact = _poisson_gauss(r, t, c, sigma)
            got = oracle.pulse(geom, r, n, point_sampling=True)
            w = abs(c * t - r)
            if w < GAUSS_TRUNC * sigma:
                inside = max(inside, abs(got - exact) / peak)
            else:
                outside = max(outside, abs(exact) / peak)
                if w > GAUSS_TRUNC * sigma:  # truncated: the oracle must give exactly zero
                    inside = max(inside, abs(got) / peak)
    return inside, outside


def check_quadrature_gauss(seed=13) -> float:
    """Interval averages against quadrature of the truncated far-field pulse."""
    rng = np.random.default_rng(seed)
    worst = 0.0
    c, fs = 1.5, 40.0
    h = c / fs
    for _ in range(10):
        sigma = float(rng.choice([0.02, 0.04, 0.08, 0.15]))
        t0, r = float(rng.uniform(0, 0.5)), float(rng.uniform(3.0, 20.0))
        geom = _scalar_geom(c, fs, 0.05, t0, sigma=sigma)
        rho = GAUSS_TRUNC * sigma
        peak = sigma / (2 * r) * math.exp(-0.5)
        for n in range(int(math.floor((r - rho - c * t0) / h)) - 2, int(math.ceil((r + rho - c * t0) / h)) + 3):
            ta, tb = c * (t0 + (n - 0.5) / fs), c * (t0 + (n + 0.5) / fs)
            pts = [x for x in (r - rho, r, r + rho) if ta < x < tb]
            val = scipy.integrate.quad(lambda tau: _gauss_far_field(r, tau, sigma), ta, tb, points=pts or None,
                                       epsabs=1e-15, epsrel=1e-12, limit=200)[0] / h
            worst = max(worst, abs(oracle.pulse(geom, r, n) - val) / peak)
    return worst


def check_closed_form() -> float:
    """Max |oracle - exact| / max|exact| over the golden worked example."""
    with open(os.path.join(_GOLDEN, "pulse_worked_example.json")) as fh:
        data = json.load(fh)
    worst = 0.0
    for case in data["cases"]:
        geom = _scalar_geom(Fr(case["c_mm_per_us"]), Fr(case["fs_mhz"]), Fr(case["a0_mm"]),
                            Fr(case["t0_us"]))
        r = float(Fr(case["r_mm"]))
        exact = {int(n): Fr(v[0]) for n, v in case["samples"].items()}
        scale = float(max(abs(v) for v in exact.values()))
        for n, v in exact.items():
            worst = max(worst, abs(oracle.pulse(geom, r, n) - float(v)) / scale)
    return worst


def _quad_sample(r, n, c, fs, a0, t0):
    """Average of the continuous closed-form pressure over sample n (quadrature in t)."""
    def p(t):
        tau = c * t
        return (r - tau) / (2 * r) if (r - a0) <= tau <= (r + a0) else 0.0
    ta, tb = t0 + (n - 0.5) / fs, t0 + (n + 0.5) / fs
    pts = [x for x in ((r - a0) / c, (r + a0) / c) if ta < x < tb]
    val, _ = scipy.integrate.quad(p, ta, tb, points=pts or None, epsabs=1e-14, epsrel=1e-12,
                                  limit=200)
    return val * fs


def check_quadrature(seed=5) -> float:
    rng = np.random.default_rng(seed)
    worst = 0.0
    for _ in range(12):
        c, fs, a0, t0 = 1.5, 40.0, float(rng.choice([0.05, 0.1, 0.2])), float(rng.uniform(0, 0.5))
        r = float(rng.uniform(3.0, 20.0))
        geom = _scalar_geom(c, fs, a0, t0)
        h = c / fs
        n0 = int(math.floor((r - a0 - c * t0) / h)) - 2
        n1 = int(math.ceil((r + a0 - c * t0) / h)) + 2
        scale = a0 / (2 * r)
        for n in range(n0, n1 + 1):
            worst = max(worst, abs(oracle.pulse(geom, r, n) - _quad_sample(r, n, c, fs, a0, t0)) / scale)
    return worst


def check_pulse_dd(seed=6, gauss=False) -> float:
    """Max relative gap between pulse_dd and a central difference of pulse."""
    rng = np.random.default_rng(seed)
    worst = 0.0
    eps = 1e-7
    for _ in range(20):
        a0 = float(rng.choice([0.05, 0.1]))
        sigma = float(rng.choice([0.02, 0.05])) if gauss else None
        geom = _scalar_geom(1.5, 40.0, a0, 0.0, sigma=sigma)
        rho = GAUSS_TRUNC * sigma if gauss else a0
        r = float(rng.uniform(3.0, 15.0))
        h = 1.5 / 40.0
        ns = range(int((r - rho) / h) - 1, int((r + rho) / h) + 2)
        scale = max(abs(oracle.pulse_dd(geom, r, n)) for n in ns) + 1e-300
        for n in ns:
            fd = (oracle.pulse(geom, r + eps, n) - oracle.pulse(geom, r - eps, n)) / (2 * eps)
            worst = max(worst, abs(fd - oracle.pulse_dd(geom, r, n)) / scale)
    return worst


def check_point_sampling() -> float:
    geom = _scalar_geom(1.5, 40.0, 0.1, 0.0)
    worst = 0.0
    for r in (5.0, 6.31, 11.007):
        for n in range(int((r - 0.2) / 0.0375), int((r + 0.2) / 0.0375) + 1):
            tau = 1.5 * n / 40.0
            ref = (r - tau) / (2 * r) if abs(tau - r) <= 0.1 else 0.0
            worst = max(worst, abs(oracle.pulse(geom, r, n, point_sampling=True) - ref))
    return worst / (0.1 / 10.0)


def small_geom(shape=(5, 6, 7), spacing=0.25, m=2, n_frames=2, n_samples=256, a0=None, seed=0, sigma=None):
    """Small volume with an m x m array 3 mm above it and slightly tilted frames
    (Gaussian kernel of width ``sigma`` if given)."""
    geom = synth.make_geom(shape, spacing, m * m, n_frames, n_samples, a0=a0)
    if sigma is not None:
        geom.update(kernel="gauss", sigma_mm=float(sigma))
    rng = np.random.default_rng(seed)
    elem = synth.planar_array(m, m, 0.7)
    poses = np.zeros((n_frames, 3, 4))
    for f in range(n_frames):
        poses[f, :, :3] = synth.axis_angle_matrix(synth.random_unit(rng), rng.uniform(0, 0.3))
        poses[f, :, 3] = [rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5),
                          synth.top_face_z(geom) + 3.0]
    return geom, elem, poses


def check_superposition() -> float:
    """Isolated voxels vs exact single-voxel values at independently computed distances."""
    gm = _golden_module()
    geom, elem, poses = small_geom(shape=(4, 5, 6), spacing=0.3, a0=0.15, n_samples=400)
    p0 = np.zeros((4, 5, 6), dtype=np.float32)
    picks = [((0, 0, 0), 1.0), ((3, 4, 5), 0.5), ((1, 3, 2), 0.75), ((2, 0, 5), 0.25)]
    for (iz, iy, ix), a in picks:
        p0[iz, iy, ix] = a
    xw = oracle.element_positions(geom, elem, poses)
    sig = oracle.forward(geom, p0, xw)
    c, fs, a0, t0 = Fr(1.5), Fr(40), Fr(geom["a0_mm"]), Fr(0)
    worst, scale = 0.0, 0.0
    for f in range(geom["n_frames"]):
        for j in range(geom["n_elem"]):
            R, t = poses[f, :, :3], poses[f, :, 3]
            x = R @ elem[j] + t
            ref = np.zeros(geom["n_samples"])
            for (iz, iy, ix), a in picks:
                r = np.array([geom["ox"] + geom["dx"] * ix, geom["oy"] + geom["dy"] * iy,
                              geom["oz"] + geom["dz"] * iz])
                d = Fr(float(np.linalg.norm(x - r)))
                for n in range(geom["n_samples"]):
                    v = gm.exact_sample(d, n, c, fs, a0, t0)
                    if v:
                        ref[n] += a * float(v)
            worst = max(worst, float(np.abs(sig[f, j] - ref).max()))
            scale = max(scale, float(np.abs(ref).max()))
    return worst / scale


def check_adjoint_identity(seed=7, sigma=None) -> float:
    geom, elem, poses = small_geom(shape=(6, 7, 8), spacing=0.2, m=3, n_frames=2, n_samples=320, sigma=sigma)
    rng = np.random.default_rng(seed)
    xw = oracle.element_positions(geom, elem, poses)
    x = rng.uniform(0, 1, size=(6, 7, 8)).astype(np.float32)
    x2 = rng.uniform(0, 1, size=(6, 7, 8)).astype(np.float32)
    y = oracle.forward(geom, x2, xw) + rng.standard_normal((2, 9, 320))
    Ax = oracle.forward(geom, x, xw)
    Aty = oracle.adjoint(geom, y, xw)
    lhs = math.fsum((Ax * y).ravel())
    rhs = math.fsum((x.astype(np.float64) * Aty).ravel())
    return abs(lhs - rhs) / max(abs(lhs), abs(rhs))


def check_rigid_invariance(seed=8, sigma=None) -> float:
    geom, elem, poses = small_geom(shape=(6, 6, 5), spacing=0.2, m=3, n_frames=2, n_samples=320, sigma=sigma)
    rng = np.random.default_rng(seed)
    p0 = rng.uniform(0, 1, size=(5, 6, 6)).astype(np.float32)
    G = synth.axis_angle_matrix(synth.random_unit(rng), math.radians(rng.uniform(5, 30)))
    gt = rng.uniform(-5, 5, size=3)
    vol_pose = np.concatenate([G, gt[:, None]], axis=1)
    moved = poses.copy()
    for f in range(len(poses)):
        moved[f, :, :3] = G @ poses[f, :, :3]
        moved[f, :, 3] = G @ poses[f, :, 3] + gt
    s0 = oracle.forward(geom, p0, oracle.element_positions(geom, elem, poses))
    s1 = oracle.forward(geom, p0, oracle.element_positions(geom, elem, moved), vol_pose=vol_pose)
    return float(np.linalg.norm(s1 - s0) / np.linalg.norm(s0))


def _twist_pose(pose, xi):
    E = scipy.linalg.expm(np.array([[0, -xi[2], xi[1]], [xi[2], 0, -xi[0]], [-xi[1], xi[0], 0]]))
    out = np.empty((3, 4))
    out[:, :3] = E @ pose[:, :3]
    out[:, 3] = E @ pose[:, 3] + xi[3:]
    return out


def _loss_at(geom, p0, elem, poses, meas, mask=None):
    xw = np.einsum("fab,jb->fja", poses[:, :, :3], elem) + poses[:, None, :, 3]
    s = oracle.forward(geom, p0, xw)
    r = s - meas
    if mask is not None:
        r = r * mask[:, :, None]
    return 0.5 * math.fsum((r * r).ravel())


def check_pose_fd(seed=9, eps=1e-6, use_mask=False, sigma=None):
    """Returns (max rel err rotation block, translation block, element gradient)."""
    geom, elem, poses = small_geom(shape=(4, 5, 5), spacing=0.25, m=2, n_frames=2, n_samples=256, sigma=sigma)
    rng = np.random.default_rng(seed)
    p0 = rng.uniform(0.2, 1, size=(4, 5, 5)).astype(np.float32)
    meas = 0.02 * rng.standard_normal((2, 4, 256))
    mask = np.array([[1, 0, 1, 1], [1, 1, 1, 0]], dtype=np.uint8) if use_mask else None
    xw = oracle.element_positions(geom, elem, poses)
    s = oracle.forward(geom, p0, xw)
    _, g = oracle.loss(geom, s, meas)  # unmasked residual: the mask is applied by pose_grad
    grad6, G = oracle.pose_grad(geom, p0, g, xw, mask)
    errs = [0.0, 0.0]
    for f in range(2):
        fd = np.zeros(6)
        for k in range(6):
            xi = np.zeros(6)
            xi[k] = eps
            pp, pm = poses.copy(), poses.copy()
            pp[f] = _twist_pose(poses[f], xi)
            pm[f] = _twist_pose(poses[f], -xi)
            fd[k] = (_loss_at(geom, p0, elem, pp, meas, mask)
                     - _loss_at(geom, p0, elem, pm, meas, mask)) / (2 * eps)
        for b, sl in enumerate((slice(0, 3), slice(3, 6))):
            errs[b] = max(errs[b], float(np.linalg.norm(fd[sl] - grad6[f, sl]) / np.linalg.norm(fd[sl])))
    # element positions directly: move one element of frame 0 along each axis
    ge = 0.0
    for j in range(geom["n_elem"]):
        fdj = np.zeros(3)
        for a in range(3):
            xp, xm = xw.copy(), xw.copy()
            xp[0, j, a] += eps
            xm[0, j, a] -= eps
            lp = 0.5 * np.sum(((oracle.forward(geom, p0, xp) - meas) * (1 if mask is None else mask[:, :, None])) ** 2)
            lm = 0.5 * np.sum(((oracle.forward(geom, p0, xm) - meas) * (1 if mask is None else mask[:, :, None])) ** 2)
            fdj[a] = (lp - lm) / (2 * eps)
        denom = max(np.linalg.norm(fdj), 1e-300)
        if np.linalg.norm(fdj) > 0 or np.linalg.norm(G[0, j]) > 0:
            ge = max(ge, float(np.linalg.norm(fdj - G[0, j]) / max(denom, np.linalg.norm(G[0, j]))))
    return errs[0], errs[1], ge


def check_p0_gradient_fd(seed=14, sigma=None) -> float:
    """The volume gradient of L = 1/2 |A p0 - S|^2 is A^T (A p0 - S): central
    differences of L in single voxels (exact for a quadratic up to rounding)
    against the oracle adjoint of the residual."""
    geom, elem, poses = small_geom(shape=(4, 5, 5), spacing=0.25, m=2, n_frames=2, n_samples=256, sigma=sigma)
    rng = np.random.default_rng(seed)
    p0 = rng.uniform(0.2, 1, size=(4, 5, 5))
    meas = 0.02 * rng.standard_normal((2, 4, 256))
    xw = oracle.element_positions(geom, elem, poses)
    _, g = oracle.loss(geom, oracle.forward(geom, p0.astype(np.float32), xw), meas)
    grad = oracle.adjoint(geom, g, xw)
    worst = 0.0
    eps = 1e-3
    for _ in range(8):
        i = tuple(int(rng.integers(0, n)) for n in p0.shape)
        pp, pm = p0.copy(), p0.copy()
        # steps exactly representable around float32 voxel values
        pp[i] = np.float32(p0[i]) + eps
        pm[i] = np.float32(p0[i]) - eps
        lp = 0.5 * math.fsum(((oracle.forward(geom, pp.astype(np.float32), xw) - meas) ** 2).ravel())
        lm = 0.5 * math.fsum(((oracle.forward(geom, pm.astype(np.float32), xw) - meas) ** 2).ravel())
        dp = float(np.float32(pp[i])) - float(np.float32(pm[i]))
        fd = (lp - lm) / dp
        worst = max(worst, abs(fd - grad[i]) / np.abs(grad).max())
    return worst


def check_big_ball(spacing=0.1, radius=1.0, dist=10.0):
    """Returns (ratio of projections, low-passed relative L2) of a voxelised ball
    against pi/6 times the ball's closed-form pulse (quadrature)."""
    n = int(round(2 * radius / spacing)) + 1
    geom = synth.make_geom((n, n, n), spacing, 1, 1, 0, fs=40.0, c=1.5)
    c, fs = 1.5, 40.0
    t0 = (dist - radius - 0.5) / c
    nt = int(math.ceil((2 * radius + 1.0) / (c / fs))) + 1
    geom["t0_us"], geom["n_samples"] = t0, nt
    x, y, z = synth.voxel_axes(geom)
    zz, yy, xx = np.meshgrid(z, y, x, indexing="ij")
    p0 = ((xx ** 2 + yy ** 2 + zz ** 2) <= radius ** 2).astype(np.float32)
    xw = np.array([[[0.0, 0.0, dist]]])
    s = oracle.forward(geom, p0, xw)[0, 0]
    ball = np.array([_quad_sample(dist, k, c, fs, radius, t0) for k in range(nt)]) * math.pi / 6
    ratio = float(np.dot(s, ball) / np.dot(ball, ball))
    lp = lambda v: scipy.ndimage.gaussian_filter1d(v, 3.0)
    l2 = float(np.linalg.norm(lp(s) - lp(ball)) / np.linalg.norm(lp(ball)))
    return ratio, l2


def check_loss(seed=10) -> float:
    geom, _, _ = small_geom(n_samples=64)
    rng = np.random.default_rng(seed)
    s = rng.standard_normal((2, 4, 64))
    S = rng.standard_normal((2, 4, 64))
    mask = (rng.uniform(size=(2, 4)) > 0.3).astype(np.uint8)
    L, g = oracle.loss(geom, s, S, mask)
    ref_g = (s - S) * mask[:, :, None]
    ref_L = 0.5 * math.fsum((ref_g ** 2).ravel())
    return max(abs(L - ref_L) / ref_L, float(np.abs(g - ref_g).max()))


# ----------------------------------------------------------------------------- TGV regulariser

def _tgv_sparse(u, w, spacing, alpha1, alpha0, eps):
    """The same energy and gradients from explicit sparse difference matrices
    (Kronecker products of 1-D forward-difference matrices) and their transposes."""
    import scipy.sparse as sp

    nz, ny, nx = u.shape

    def d1(n, h):
        m = sp.lil_matrix((n, n))
        for i in range(n - 1):
            m[i, i], m[i, i + 1] = -1.0 / h, 1.0 / h
        return m.tocsr()

    I = lambda n: sp.identity(n, format="csr")
    D = [sp.kron(I(nz), sp.kron(I(ny), d1(nx, spacing[0]))),
         sp.kron(I(nz), sp.kron(d1(ny, spacing[1]), I(nx))),
         sp.kron(d1(nz, spacing[2]), sp.kron(I(ny), I(nx)))]
    uf = u.ravel().astype(np.float64)
    wf = [w[b].ravel().astype(np.float64) for b in range(3)]
    r = [D[a] @ uf - wf[a] for a in range(3)]
    phi1 = np.sqrt(sum(x * x for x in r) + eps * eps)
    E = [[0.5 * (D[a] @ wf[b] + D[b] @ wf[a]) for b in range(3)] for a in range(3)]
    phi2 = np.sqrt(sum(E[a][b] ** 2 for a in range(3) for b in range(3)) + eps * eps)
    J = alpha1 * phi1.sum() + alpha0 * phi2.sum()
    gu = sum(D[a].T @ (alpha1 * r[a] / phi1) for a in range(3))
    gw = [-(alpha1 * r[b] / phi1) + sum(D[a].T @ (alpha0 * E[a][b] / phi2) for a in range(3)) for b in range(3)]
    return J, gu.reshape(u.shape), np.stack([g.reshape(u.shape) for g in gw])


def _tgv_case(seed=30, shape=(4, 5, 6)):
    rng = np.random.default_rng(seed)
    u = rng.uniform(0, 1, size=shape)
    w = rng.normal(0, 2.0, size=(3,) + shape)
    return u, w, (0.1, 0.12, 0.15), 0.7, 0.4, 0.05


def check_tgv_sparse(seed=30) -> float:
    """Max relative gap between the oracle and the sparse-matrix formulation."""
    from oracle import tgv
    u, w, sp_, a1, a0, eps = _tgv_case(seed)
    J, gu, gw = tgv.energy_and_grad(u, w, sp_, a1, a0, eps)
    J2, gu2, gw2 = _tgv_sparse(u, w, sp_, a1, a0, eps)
    return max(abs(J - J2) / abs(J2), float(np.abs(gu - gu2).max() / np.abs(gu2).max()),
               float(np.abs(gw - gw2).max() / np.abs(gw2).max()))


def check_tgv_fd(seed=31, h=1e-6) -> float:
    """Central differences of J in random entries of u and w against the gradients."""
    from oracle import tgv
    u, w, sp_, a1, a0, eps = _tgv_case(seed)
    _, gu, gw = tgv.energy_and_grad(u, w, sp_, a1, a0, eps)
    rng = np.random.default_rng(seed + 1)
    worst = 0.0
    scale = max(np.abs(gu).max(), np.abs(gw).max())
    for _ in range(12):
        i = tuple(int(rng.integers(0, n)) for n in u.shape)
        up, um = u.copy(), u.copy()
        up[i] += h
        um[i] -= h
        fd = (tgv.energy_and_grad(up, w, sp_, a1, a0, eps)[0] - tgv.energy_and_grad(um, w, sp_, a1, a0, eps)[0]) / (2 * h)
        worst = max(worst, abs(fd - gu[i]) / scale)
        b = int(rng.integers(0, 3))
        wp, wm = w.copy(), w.copy()
        wp[(b,) + i] += h
        wm[(b,) + i] -= h
        fd = (tgv.energy_and_grad(u, wp, sp_, a1, a0, eps)[0] - tgv.energy_and_grad(u, wm, sp_, a1, a0, eps)[0]) / (2 * h)
        worst = max(worst, abs(fd - gw[(b,) + i]) / scale)
    return worst


def check_tgv_constant() -> float:
    """A constant field with w = 0 has only the smoothing floor: J = N (alpha1 + alpha0) eps,
    zero gradients."""
    from oracle import tgv
    u = np.full((3, 4, 5), 0.7)
    w = np.zeros((3, 3, 4, 5))
    J, gu, gw = tgv.energy_and_grad(u, w, (0.1, 0.1, 0.1), 0.7, 0.4, 0.05)
    return max(abs(J - 60 * 1.1 * 0.05) / (60 * 1.1 * 0.05), float(np.abs(gu).max()), float(np.abs(gw).max()))
