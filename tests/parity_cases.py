"""Seeded workloads shared by the GPU parity tests (inputs only; no arithmetic of the method
beyond calls into the FP64 oracle)."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2604_09643_b300 import synth

REL_L2_SIG = 1e-5    # signals and volumes, FP32 path vs FP64 oracle
REL_L2_POSE = 1e-4   # pose gradients, rotation and translation blocks separately


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def ragged_case(seed=0, cut=False):
    """Ragged everything: 29 x 37 x 20 grid (not a multiple of any cube or of 4),
    33 elements (one warp + 1), 3 frames, Nt = 1001 (not a multiple of 4).  With
    ``cut`` the record starts after the nearest arrivals and ends (Nt = 61)
    before the farthest ones, so pulses cross both ends of the record."""
    geom = synth.make_geom((20, 37, 29), 0.1, 33, 3, 1001)
    rng = np.random.default_rng(100 + seed)
    p0 = synth.vessel_tree_phantom(geom, 6, rng, radius=(0.05, 0.2))
    p0 += rng.uniform(0, 0.05, size=p0.shape).astype(np.float32)  # dense background
    elem = synth.planar_array(11, 3, 0.45)
    trng = np.random.default_rng(200 + seed)
    poses = synth.sweep_poses(3, 0.4, synth.top_face_z(geom) + 2.5, trng, jitter_deg=3.0)
    if cut:
        geom["t0_us"] = 2.8 / geom["c_mm_per_us"]
        geom["n_samples"] = 61
    return geom, p0, elem, poses


def tma_case(seed=0):
    """Aligned case that takes the TMA paths: 40 x 48 x 32 grid (nx % 4 == 0),
    64 elements, 2 frames, Nt = 1024."""
    geom = synth.make_geom((32, 48, 40), 0.1, 64, 2, 1024)
    rng = np.random.default_rng(300 + seed)
    p0 = synth.vessel_tree_phantom(geom, 10, rng)
    p0 += rng.uniform(0, 0.02, size=p0.shape).astype(np.float32)
    elem = synth.planar_array(8, 8, 0.6)
    trng = np.random.default_rng(400 + seed)
    poses = synth.sweep_poses(2, 0.3, synth.top_face_z(geom) + 5.0, trng)
    return geom, p0, elem, poses


def wide_window_case(seed=0):
    """The largest forward window of 16^3 cubes: 0.17 mm spacing (cube diagonal 2.2 mm
    of distance range, 118 samples, plus S = 6 slots and the margin: W = 128, the
    16^3 cap) on an aligned 28 x 24 x 20 grid, 40 elements, 2 frames, Nt = 1024."""
    geom = synth.make_geom((20, 24, 28), 0.17, 40, 2, 1024)
    rng = np.random.default_rng(700 + seed)
    p0 = synth.vessel_tree_phantom(geom, 6, rng)
    p0 += rng.uniform(0, 0.02, size=p0.shape).astype(np.float32)
    elem = synth.planar_array(8, 5, 0.6)
    trng = np.random.default_rng(800 + seed)
    poses = synth.sweep_poses(2, 0.3, synth.top_face_z(geom) + 3.0, trng)
    return geom, p0, elem, poses


def coarse_window_case(seed=0):
    """The largest forward window of 8^3 cubes and the largest sphere slot count at once:
    0.557 mm spacing (a0 = 0.2785 mm, S = 16; an 8^3 cube's 181-sample distance range
    plus the slots and the margin: W = 200, the 8^3 cap) on a 12 x 12 x 10 grid, 25
    elements, 2 frames, Nt = 800."""
    geom = synth.make_geom((10, 12, 12), 0.557, 25, 2, 800)
    rng = np.random.default_rng(900 + seed)
    p0 = rng.uniform(0, 1, size=(10, 12, 12)).astype(np.float32)
    elem = synth.planar_array(5, 5, 1.0)
    trng = np.random.default_rng(1000 + seed)
    poses = synth.sweep_poses(2, 0.5, synth.top_face_z(geom) + 4.0, trng)
    return geom, p0, elem, poses


def aniso_case(seed=0):
    """Anisotropic voxels (dz, dy, dx) = (0.12, 0.1, 0.08) mm on a 24 x 30 x 20 grid (x
    fastest, nx % 4 == 0), 36 elements, 2 frames, Nt = 1024: every axis has its own
    spacing, so a swapped axis or spacing anywhere shows."""
    geom = synth.make_geom((20, 30, 24), (0.12, 0.1, 0.08), 36, 2, 1024)
    rng = np.random.default_rng(1100 + seed)
    p0 = synth.vessel_tree_phantom(geom, 6, rng)
    p0 += rng.uniform(0, 0.02, size=p0.shape).astype(np.float32)
    elem = synth.planar_array(6, 6, 0.5)
    trng = np.random.default_rng(1200 + seed)
    poses = synth.sweep_poses(2, 0.3, synth.top_face_z(geom) + 3.0, trng)
    return geom, p0, elem, poses


def coarse_case(seed=0):
    """Coarse grid (0.3 mm, a0 = 0.15 mm, 2 a0 / h = 8 exactly): 10 slots per pair
    and 8^3 cubes."""
    geom = synth.make_geom((18, 20, 22), 0.3, 25, 2, 800)
    rng = np.random.default_rng(500 + seed)
    p0 = rng.uniform(0, 1, size=(18, 20, 22)).astype(np.float32)
    elem = synth.planar_array(5, 5, 1.0)
    trng = np.random.default_rng(600 + seed)
    poses = synth.sweep_poses(2, 0.5, synth.top_face_z(geom) + 4.0, trng)
    return geom, p0, elem, poses


def residual(geom, seed=1, scale=1.0):
    """White-noise trace residual [F][E][Nt]."""
    rng = np.random.default_rng(seed)
    return (scale * rng.standard_normal((geom["n_frames"], geom["n_elem"], geom["n_samples"]))).astype(np.float32)


def pose_residual(geom, p0, elem, poses, seed=5, rot_deg=0.5, trans_mm=0.05):
    """The residual the method itself produces: traces at the given poses minus
    traces at slightly perturbed poses (computed by the oracle)."""
    rng = np.random.default_rng(seed)
    pert = synth.perturb_poses(poses, rng, rot_deg, trans_mm, keep_first=False)
    a = oracle.forward(geom, p0, oracle.element_positions(geom, elem, poses))
    b = oracle.forward(geom, p0, oracle.element_positions(geom, elem, pert))
    return (a - b).astype(np.float32)


def gaussian(case, sigma):
    """The same inputs with the Gaussian kernel of width ``sigma`` (mm) instead of the sphere."""
    def make(*a, **kw):
        geom, p0, elem, poses = case(*a, **kw)
        return dict(geom, kernel="gauss", sigma_mm=float(sigma)), p0, elem, poses
    return make


def sphere(case, a0):
    """The same inputs with a uniform-sphere voxel of radius ``a0`` (mm)."""
    def make(*a, **kw):
        geom, p0, elem, poses = case(*a, **kw)
        return dict(geom, a0_mm=float(a0)), p0, elem, poses
    return make
