"""Seeded synthetic inputs for the radiation operator: phantoms, arrays, trajectories.

This module holds no arithmetic of the method itself (no pulse, no time of
flight, no gradient).  It only draws the inputs that both the CUDA path and the
FP64 oracle consume, so that the two can be fed identical arrays:

* source volumes ``p0[nz][ny][nx]`` (float32): random cylinders (the
  single-frame workload) or a vessel tree of tubes along cubic Bezier curves,
  max-combined and Gaussian-smoothed (the full-scan workloads);
* planar element templates ``elem[E][3]`` (float64, mm, array frame, centred,
  z = 0), standing for the sensor coordinates x_s of Eq. 1 and the rigid
  template X_template of Stage 3;
* per-frame rigid poses ``pose[F][3][4] = [R | t]`` (float64) with the world
  position of element j in frame f being ``R e_j + t`` (the rigid model of
  Stage 4);
* the acquisition scalars (sampling rate, sound speed, sphere radius).

Units are mm, microseconds and MHz.  The volume is centred on the world origin
with voxel centres at ``(k - (N-1)/2) * spacing``; the array plane sits a fixed
standoff above the top face of the volume, facing it.  Seeds are fixed per
workload (phantom 0, trajectory 1, noise 2, arrival stream 3) plus ten times
the workload index, so every run sees the same arrays.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy import ndimage
from scipy.spatial import cKDTree

SEED_PHANTOM, SEED_TRAJ, SEED_NOISE, SEED_STREAM = 0, 1, 2, 3

C_MM_PER_US = 1.5
FS_MHZ = 40.0
STANDOFF_MM = 5.0


@dataclasses.dataclass
class Scan:
    """One synthetic acquisition: geometry scalars, volume, template and poses."""

    geom: dict
    p0: np.ndarray          # float32 [nz][ny][nx]
    elem: np.ndarray        # float64 [E][3], array frame
    poses: np.ndarray       # float64 [F][3][4], true poses
    name: str = ""
    poses_init: np.ndarray | None = None  # perturbed starting poses (reconstruction)

    @property
    def n_vox(self) -> int:
        return int(self.p0.size)

    @property
    def pairs(self) -> int:
        """Voxel-element pairs per operator application, summed over frames."""
        return self.n_vox * self.geom["n_elem"] * self.geom["n_frames"]


def make_geom(shape, spacing, n_elem, n_frames, n_samples, *, fs=FS_MHZ,
              c=C_MM_PER_US, a0=None, t0=0.0, kernel="sphere", sigma=None) -> dict:
    """Acquisition scalars for a grid of ``shape = (nz, ny, nx)`` centred at 0.
    ``kernel`` names the voxel pulse: "sphere" (radius a0) or "gauss" (width sigma, mm)."""
    nz, ny, nx = (int(s) for s in shape)
    if np.isscalar(spacing):
        dz = dy = dx = float(spacing)
    else:
        dz, dy, dx = (float(s) for s in spacing)
    if a0 is None:
        a0 = 0.5 * min(dx, dy, dz)
    if kernel not in ("sphere", "gauss") or (kernel == "gauss" and not (sigma and sigma > 0)):
        raise ValueError("kernel must be 'sphere', or 'gauss' with sigma > 0")
    return dict(nx=nx, ny=ny, nz=nz, dx=dx, dy=dy, dz=dz,
                ox=-0.5 * (nx - 1) * dx, oy=-0.5 * (ny - 1) * dy,
                oz=-0.5 * (nz - 1) * dz,
                n_elem=int(n_elem), n_frames=int(n_frames),
                n_samples=int(n_samples), fs_mhz=float(fs), t0_us=float(t0),
                c_mm_per_us=float(c), a0_mm=float(a0),
                kernel=kernel, sigma_mm=float(sigma) if kernel == "gauss" else 0.0)


def voxel_axes(geom):
    """Voxel-centre coordinates along x, y, z (float64)."""
    x = geom["ox"] + geom["dx"] * np.arange(geom["nx"])
    y = geom["oy"] + geom["dy"] * np.arange(geom["ny"])
    z = geom["oz"] + geom["dz"] * np.arange(geom["nz"])
    return x, y, z


def top_face_z(geom) -> float:
    return geom["oz"] + (geom["nz"] - 1) * geom["dz"] + 0.5 * geom["dz"]


def planar_array(m_x: int, m_y: int | None = None, pitch: float = 1.0) -> np.ndarray:
    """Centred m_x x m_y planar element grid at z = 0 in the array frame."""
    m_y = m_x if m_y is None else m_y
    a = (np.arange(m_x) - 0.5 * (m_x - 1)) * pitch
    b = (np.arange(m_y) - 0.5 * (m_y - 1)) * pitch
    bb, aa = np.meshgrid(b, a, indexing="ij")
    return np.stack([aa.ravel(), bb.ravel(), np.zeros(aa.size)], axis=1).astype(np.float64)


def axis_angle_matrix(axis, angle) -> np.ndarray:
    """Rotation matrix of ``angle`` radians about ``axis`` (input drawing only)."""
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis)
    k = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(angle) * k + (1 - math.cos(angle)) * (k @ k)


def euler_xyz(rx, ry, rz) -> np.ndarray:
    return (axis_angle_matrix([0, 0, 1], rz) @ axis_angle_matrix([0, 1, 0], ry)
            @ axis_angle_matrix([1, 0, 0], rx))


def random_unit(rng) -> np.ndarray:
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


# ---------------------------------------------------------------------------
# phantoms
# ---------------------------------------------------------------------------

def cylinders_phantom(geom, n_cyl, rng, inner=4.0, radius=(0.2, 0.4)) -> np.ndarray:
    """Binary volume of ``n_cyl`` infinite cylinders (amplitude 1)."""
    x, y, z = voxel_axes(geom)
    zz, yy, xx = np.meshgrid(z, y, x, indexing="ij")
    pts = np.stack([xx, yy, zz], axis=-1)
    out = np.zeros(xx.shape, dtype=np.float32)
    for _ in range(n_cyl):
        c = rng.uniform(-inner / 2, inner / 2, size=3)
        u = random_unit(rng)
        r = rng.uniform(*radius)
        rel = pts - c
        dist = np.linalg.norm(np.cross(rel, u), axis=-1)
        out[dist <= r] = 1.0
    return out


def _bezier(ctrl, t):
    s = 1.0 - t
    return ((s ** 3)[:, None] * ctrl[0] + (3 * s * s * t)[:, None] * ctrl[1]
            + (3 * s * t * t)[:, None] * ctrl[2] + (t ** 3)[:, None] * ctrl[3])


def vessel_tree_phantom(geom, n_tubes, rng, radius=(0.05, 0.4), amp=(0.5, 1.0),
                        inner=0.9, blur_sigma_vox=0.5) -> np.ndarray:
    """Max-combined tubes along random cubic Bezier curves, then Gaussian blur."""
    nx, ny, nz = geom["nx"], geom["ny"], geom["nz"]
    d = np.array([geom["dx"], geom["dy"], geom["dz"]])
    o = np.array([geom["ox"], geom["oy"], geom["oz"]])
    half = 0.5 * inner * np.array([nx - 1, ny - 1, nz - 1]) * d
    dims = np.array([nx, ny, nz])
    out = np.zeros((nz, ny, nx), dtype=np.float32)
    for _ in range(n_tubes):
        ctrl = rng.uniform(-half, half, size=(4, 3))
        r = rng.uniform(*radius)
        a = np.float32(rng.uniform(*amp))
        length = sum(np.linalg.norm(ctrl[k + 1] - ctrl[k]) for k in range(3))
        step = 0.5 * min(r, float(d.min()))
        m = max(8, int(math.ceil(length / step)) + 1)
        pts = _bezier(ctrl, np.linspace(0.0, 1.0, m))
        kr = np.ceil(r / d).astype(int)
        offs = np.stack(np.meshgrid(*[np.arange(-k, k + 1) for k in kr], indexing="ij"),
                        axis=-1).reshape(-1, 3)
        base = np.rint((pts - o) / d).astype(int)
        cand = (base[:, None, :] + offs[None, :, :]).reshape(-1, 3)
        cand = cand[np.all((cand >= 0) & (cand < dims), axis=1)]
        # unique voxels, in (x, y, z) lexicographic order
        lin = np.unique((cand[:, 0] * dims[1] + cand[:, 1]) * dims[2] + cand[:, 2])
        cand = np.stack([lin // (dims[1] * dims[2]), (lin // dims[2]) % dims[1], lin % dims[2]], axis=1)
        if cand.size == 0:
            continue
        centres = o + cand * d
        # distance from each candidate voxel centre to the nearest sampled curve point
        best, _ = cKDTree(pts).query(centres, k=1)
        sel = cand[best <= r]
        cur = out[sel[:, 2], sel[:, 1], sel[:, 0]]
        out[sel[:, 2], sel[:, 1], sel[:, 0]] = np.maximum(cur, a)
    if blur_sigma_vox and blur_sigma_vox > 0:
        out = ndimage.gaussian_filter(out, sigma=blur_sigma_vox, mode="constant").astype(np.float32)
    return out


# ---------------------------------------------------------------------------
# trajectories
# ---------------------------------------------------------------------------

def smooth_jitter(n_frames, rng, peak_rad, n_terms=3):
    """Per-axis sum of low-frequency sinusoids, scaled to ``peak_rad`` peak."""
    t = np.linspace(0.0, 1.0, n_frames)
    out = np.zeros((n_frames, 3))
    for ax in range(3):
        sig = np.zeros(n_frames)
        for _ in range(n_terms):
            freq = rng.uniform(0.3, 2.0)
            ph = rng.uniform(0, 2 * math.pi)
            sig += rng.uniform(0.3, 1.0) * np.sin(2 * math.pi * freq * t + ph)
        peak = np.abs(sig).max()
        out[:, ax] = sig / peak * peak_rad if peak > 0 else 0.0
    return out


def sweep_poses(n_frames, step_mm, plane_z, rng, jitter_deg=2.0):
    """Frames translating along x in fixed steps, centred, with smooth tilt jitter."""
    ang = smooth_jitter(n_frames, rng, math.radians(jitter_deg))
    poses = np.zeros((n_frames, 3, 4))
    for f in range(n_frames):
        poses[f, :, :3] = euler_xyz(*ang[f])
        poses[f, :, 3] = [(f - 0.5 * (n_frames - 1)) * step_mm, 0.0, plane_z]
    return poses


def perturb_poses(poses, rng, rot_sigma_deg, trans_sigma_mm, keep_first=True):
    """Left-multiply each pose by a random rigid motion about the array centre."""
    out = poses.copy()
    for f in range(len(poses)):
        if keep_first and f == 0:
            continue
        dr = euler_xyz(*rng.normal(0.0, math.radians(rot_sigma_deg), size=3))
        out[f, :, :3] = dr @ poses[f, :, :3]
        out[f, :, 3] = poses[f, :, 3] + rng.normal(0.0, trans_sigma_mm, size=3)
    return out


# ---------------------------------------------------------------------------
# named workloads
# ---------------------------------------------------------------------------

def single_frame(seed_offset=0) -> Scan:
    """32^3 at 0.2 mm, 4 cylinders, 8x8 array at 1.0 mm, 1 perturbed frame, 512 samples."""
    geom = make_geom((32, 32, 32), 0.2, 64, 1, 512, a0=0.1)
    rng = np.random.default_rng(SEED_PHANTOM + 10 * 1 + seed_offset)
    p0 = cylinders_phantom(geom, 4, rng)
    elem = planar_array(8, 8, 1.0)
    trng = np.random.default_rng(SEED_TRAJ + 10 * 1 + seed_offset)
    rot = axis_angle_matrix(random_unit(trng), math.radians(trng.uniform(0.0, 1.0)))
    t = random_unit(trng) * trng.uniform(0.0, 0.3)
    pose = np.zeros((1, 3, 4))
    pose[0, :, :3] = rot
    pose[0, :, 3] = np.array([0.0, 0.0, top_face_z(geom) + STANDOFF_MM]) + t
    return Scan(geom, p0, elem, pose, name="single_frame_32^3_8x8_512")


def full_scan(n=128, spacing=0.1, n_tubes=40, m=16, pitch=0.6, n_frames=64,
              n_samples=2048, step_mm=0.3, workload=2, seed_offset=0) -> Scan:
    """Vessel-tree volume, m x m array, smooth x-sweep of n_frames frames."""
    shape = (n, n, n) if np.isscalar(n) else tuple(n)
    geom = make_geom(shape, spacing, m * m, n_frames, n_samples)
    rng = np.random.default_rng(SEED_PHANTOM + 10 * workload + seed_offset)
    p0 = vessel_tree_phantom(geom, n_tubes, rng)
    elem = planar_array(m, m, pitch)
    trng = np.random.default_rng(SEED_TRAJ + 10 * workload + seed_offset)
    poses = sweep_poses(n_frames, step_mm, top_face_z(geom) + STANDOFF_MM, trng)
    return Scan(geom, p0, elem, poses,
                name=f"full_scan_{'x'.join(map(str, shape))}_{m}x{m}_{n_frames}f_{n_samples}")


def reconstruction_scan(n=256, n_frames=200, seed_offset=0) -> Scan:
    """256^3 at 0.1 mm, 150 tubes, 16x16 at 0.6 mm, 200 frames with noisy initial poses."""
    s = full_scan(n=n, spacing=0.1 * 256 / n, n_tubes=150, m=16, pitch=0.6,
                  n_frames=n_frames, n_samples=2048, step_mm=25.6 / n_frames,
                  workload=3, seed_offset=seed_offset)
    nrng = np.random.default_rng(SEED_NOISE + 30 + seed_offset)
    s.poses_init = perturb_poses(s.poses, nrng, 1.5, 0.5, keep_first=True)
    s.name = f"reconstruction_{n}^3_16x16_{n_frames}f"
    return s


def mixed_precision_scan(n_frames=400, seed_offset=0) -> Scan:
    """256x256x128 at 0.1 mm, 32x32 at 0.3 mm, 400 frames, 3072 samples."""
    return full_scan(n=(128, 256, 256), spacing=0.1, n_tubes=150, m=32, pitch=0.3,
                     n_frames=n_frames, n_samples=3072, step_mm=0.3, workload=4,
                     seed_offset=seed_offset)


def hemisphere_array(n_total=1024, radius=60.0, keep_half=True) -> np.ndarray:
    """Elements spread evenly (Fibonacci spiral) over the hemisphere of `radius` mm
    facing its centre from above (z > 0), centre at the origin of the array frame.
    With keep_half only the elements with azimuth in [0, pi) are kept: the
    512-element half of a 1024-element bowl."""
    k = np.arange(n_total) + 0.5
    z = 1.0 - k / n_total                     # cos(polar angle) uniform in (0, 1): even area on the hemisphere
    phi = np.mod(math.pi * (3.0 - math.sqrt(5.0)) * k, 2 * math.pi)
    r = np.sqrt(1.0 - z * z)
    pts = radius * np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)
    if keep_half:
        pts = pts[phi < math.pi]
    return pts


def cap_array(n_elem=33, radius=60.0, half_angle_deg=40.0, seed=0) -> np.ndarray:
    """A sparse array of n_elem elements spread over a spherical cap of `radius` mm
    and the given half-angle about +z, facing its centre (the origin)."""
    rng = np.random.default_rng(SEED_TRAJ + 70 + seed)
    cmin = math.cos(math.radians(half_angle_deg))
    z = rng.uniform(cmin, 1.0, size=n_elem)
    phi = rng.uniform(0, 2 * math.pi, size=n_elem)
    r = np.sqrt(1.0 - z * z)
    return radius * np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def two_view_scan(n=128, spacing=0.1, n_tubes=40, elem=None, view_b_deg=90.0, prior_rot_deg=0.5,
                  prior_trans_mm=0.5, n_samples=768, n_views=2, seed_offset=0) -> Scan:
    """Views of a vessel-tree volume at the centre of a hemispherical bowl: view 0
    at the known pose (identity), view k the same probe turned by k * view_b_deg
    about the bowl axis plus a small random tilt and offset.  poses_init holds the
    priors (truth perturbed by prior_rot_deg / prior_trans_mm; view 0 exact).  The
    record starts when the nearest voxel's pulse can first arrive."""
    elem = hemisphere_array() if elem is None else np.asarray(elem, dtype=np.float64)
    geom = make_geom((n, n, n), spacing, len(elem), n_views, n_samples)
    rng = np.random.default_rng(SEED_PHANTOM + 80 + seed_offset)
    p0 = vessel_tree_phantom(geom, n_tubes, rng)
    trng = np.random.default_rng(SEED_TRAJ + 80 + seed_offset)
    poses = np.zeros((n_views, 3, 4))
    poses[0, :, :3] = np.eye(3)
    for k in range(1, n_views):
        poses[k, :, :3] = axis_angle_matrix(random_unit(trng), math.radians(trng.uniform(0.5, 1.5))) @ \
            axis_angle_matrix([0.0, 0.0, 1.0], math.radians(k * view_b_deg))
        poses[k, :, 3] = random_unit(trng) * trng.uniform(0.2, 0.6)
    half_diag = 0.5 * math.sqrt(3.0) * n * spacing
    d_min = float(np.linalg.norm(elem, axis=1).min()) - half_diag - 1.0
    geom["t0_us"] = max(0.0, d_min) / geom["c_mm_per_us"]
    nrng = np.random.default_rng(SEED_NOISE + 80 + seed_offset)
    init = poses.copy()
    init[1:] = perturb_poses(poses[1:], nrng, prior_rot_deg, prior_trans_mm, keep_first=False)
    return Scan(geom, p0, elem, poses, name=f"two_view_{n}^3_{len(elem)}elem", poses_init=init)


def random_like_signals(geom, rng, dtype=np.float32) -> np.ndarray:
    """Standard-normal array shaped like the signals [F][E][Nt]."""
    return rng.standard_normal((geom["n_frames"], geom["n_elem"],
                                geom["n_samples"])).astype(dtype)


def request_stream(n_requests=200, rate_per_s=4.0, seed=SEED_STREAM + 50):
    """Seeded Poisson stream of reconstruction requests of mixed sizes."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for k in range(n_requests):
        t += rng.exponential(1.0 / rate_per_s)
        reqs.append(dict(
            id=k, arrival_s=t,
            n=int(rng.choice([64, 96, 128, 192, 256])),
            n_frames=int(rng.integers(16, 257)),
            m=int(rng.choice([8, 16, 32])),
            pitch=float(rng.uniform(0.3, 1.0)),
            n_samples=int(rng.choice([1024, 2048, 3072])),
            n_tubes=int(rng.integers(10, 151)),
            seed=int(rng.integers(0, 2 ** 31 - 1)),
        ))
    return reqs
