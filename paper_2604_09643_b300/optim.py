"""Coarse-to-fine joint reconstruction of the source volume and the frame poses.

The paper's pipeline (Algorithm 1) reconstructs P_c with Adam on the Eq. 2
data term, localises sensors from gradients of the radiation engine (Stage 2),
snaps noisy sensor estimates onto the rigid array template with a RANSAC whose
subsets are pre-checked on pairwise edge lengths before a Kabsch fit (Stage 3),
and refines the rigid parameters with an inlier-masked loss (Stage 4, Eq. 4).
Here those pieces drive a joint optimisation over every frame:

* Levels: the volume estimate lives on a pyramid of grids over the same world
  box (for example 64^3 -> 128^3 -> 256^3), each with sphere radius a0 = spacing / 2.
  A coarse level has wider pulses, which smooths the loss like the paper's
  decaying kernel width.  Since (4/3) pi a0^3 / spacing^3 = pi / 6 on every level,
  the estimate carries over by trilinear resampling without rescaling.
* Gaussian kernel (Eq. 1): each level runs one or more widths sigma, largest
  first (the dynamic smoothing of Stage 2).  The measurements, simulated or
  recorded at the finest width, are low-passed in time by a Gaussian of width
  sqrt(sigma^2 - sigma_fine^2), which turns their pulses into exactly the
  pulses of width sigma; voxel amplitudes are rescaled by (sigma_old / sigma_new)^3
  (spacing_new / spacing_old)^3 at each change so the represented field is kept.
* Steps: each is one ``pasfm_step``: forward, inlier-masked loss head, fused
  adjoint + pose gradient, Adam on the volume (projected to p0 >= 0) and on the
  frame twists.  Frame 0 is the gauge, held at its known pose like the paper's
  Pose A.
* Coarse search (Stage 2): on the coarsest level, after its joint steps, each
  frame's translation is re-chosen from a cubic grid of candidates scored by
  the NC loss of Eq. 3 against that frame's (band-limited) traces, Top-1, and
  joint steps resume; this widens the capture range beyond what gradients alone
  reach (about half a pulse width per level).
* Rigid consensus, every ``refine_every`` steps:
  1. Each element proposes a position one fixed-length step down its own
     gradient (the per-sensor gradient step of Stage 2).
  2. Per frame, RANSAC over 3-element subsets runs the edge-length pre-check,
     then a Kabsch fit, to pick the rigid pose most elements agree with.
  3. Its inliers become the loss mask of Eq. 4.
  4. A frame whose consensus pose moves its elements by more than
     ``reset_mm`` from the current pose is reset to the consensus pose (rigid
     outlier rejection).

The paper leaves the thresholds, step sizes, iteration counts and the subset
sampler unstated; they are fields of :class:`C2FConfig`.
"""
from __future__ import annotations

import dataclasses
import itertools
import math
import time

import numpy as np
import torch

from . import binding


# ----------------------------------------------------------------------------- rigid-body pieces

def kabsch(src, dst, weights=None):
    """Rotation R and translation t minimising sum w |R src_i + t - dst_i|^2 (det R = +1)."""
    src = np.asarray(src, dtype=np.float64)
    dst = np.asarray(dst, dtype=np.float64)
    w = np.ones(len(src)) if weights is None else np.asarray(weights, dtype=np.float64)
    w = w / w.sum()
    cs = w @ src
    cd = w @ dst
    cov = (src - cs).T @ ((dst - cd) * w[:, None])
    u, _, vt = np.linalg.svd(cov)
    d = 1.0 if np.linalg.det(vt.T @ u.T) >= 0 else -1.0
    rot = vt.T @ np.diag([1.0, 1.0, d]) @ u.T
    return rot, cd - rot @ cs


def edge_precheck(template, observed, subset, tol_mm):
    """True when every pairwise distance in the subset matches the template within tol."""
    s = list(subset)
    for a in range(len(s)):
        for b in range(a + 1, len(s)):
            lt = math.dist(template[s[a]], template[s[b]])
            lo = math.dist(observed[s[a]], observed[s[b]])
            if abs(lt - lo) > tol_mm:
                return False
    return True


def ransac(template, observed, subsets, edge_tol_mm, inlier_tol_mm):
    """Stage 3 consensus over the given subsets.  Returns (R, t, inlier mask, winning
    subset index or -1); the winner is the first subset with the most inliers, and
    the returned fit is refitted on its inliers."""
    template = np.asarray(template, dtype=np.float64)
    observed = np.asarray(observed, dtype=np.float64)
    best_n, best_i, best_mask = -1, -1, None
    for i, sub in enumerate(subsets):
        if not edge_precheck(template, observed, sub, edge_tol_mm):
            continue
        rot, tr = kabsch(template[list(sub)], observed[list(sub)])
        err = np.linalg.norm(template @ rot.T + tr - observed, axis=1)
        inl = err < inlier_tol_mm
        if int(inl.sum()) > best_n:
            best_n, best_i, best_mask = int(inl.sum()), i, inl
    if best_i < 0 or best_n < 3:
        return np.eye(3), np.zeros(3), np.zeros(len(template), dtype=bool), -1
    rot, tr = kabsch(template[best_mask], observed[best_mask])
    return rot, tr, best_mask, best_i


# ----------------------------------------------------------------------------- levels

def level_geometry(geom, shape):
    """Grid of `shape` = (nz, ny, nx) covering the same world box as `geom`'s voxels,
    with a0 = half the smallest spacing (the inscribed sphere)."""
    nz, ny, nx = (int(s) for s in shape)
    out = dict(geom)
    for ax, n in (("x", nx), ("y", ny), ("z", nz)):
        lo = geom["o" + ax] - 0.5 * geom["d" + ax]
        ext = geom["n" + ax] * geom["d" + ax]
        d = ext / n
        out["n" + ax] = n
        out["d" + ax] = d
        out["o" + ax] = lo + 0.5 * d
    out["a0_mm"] = 0.5 * min(out["dx"], out["dy"], out["dz"])
    return out


@dataclasses.dataclass
class C2FConfig:
    levels: tuple = ((64, 64, 64), (128, 128, 128), (256, 256, 256))
    steps: tuple = (100, 100, 100)
    lr_vol: float = 0.02
    lr_rot: float = 2e-3
    lr_trans: float = 2e-2
    lr_decay: float = 0.5          # learning-rate factor applied per level
    init_value: float = 0.0
    nonneg: bool = True
    fix_frame0: bool = True
    lowpass: tuple | None = None   # per-level time low-pass sigma (samples); None: (a0_l - a0_fine) / h
    volume_only: tuple | None = None  # per-level steps with poses frozen before the joint steps
    reference_steps: int = 0       # coarsest level: volume from the gauge frame alone (Stage 1)
    register_steps: int = 0        # coarsest level: poses against that map, volume frozen (Stages 2-4)
    search_rounds: int = 0         # coarsest level: Stage 2 grid searches after its joint steps
    search_radius_mm: float = 0.8  # half-width of the cubic translation grid
    search_step_mm: float = 0.1
    search_coarse_to_fine: bool = True  # shrinking 5-point grids instead of the full grid
    search_joint_steps: int = 150  # joint steps after each search round
    search_batch: int = 512        # candidates per forward call
    refine_every: int = 0          # 0 disables the rigid-consensus pass
    elem_step_mm: float = 0.05
    edge_tol_mm: float = 0.05
    inlier_tol_mm: float = 0.1
    reset_mm: float = 0.3
    n_subsets: int = 64
    seed: int = 0
    # Gaussian kernel (Eq. 1): per-level widths (mm), each level's joint steps split evenly
    # over its widths, widest first (the dynamic smoothing of Stage 2); None: one
    # width per level, the data's width scaled by the level's spacing (at most SIGMA_MAX_SAMPLES sample pitches)
    sigma_schedule: tuple | None = None
    decimate_time: bool = True     # Gaussian kernel: coarse levels on a time grid coarser by their spacing ratio
    # TGV regulariser of Stages 1 and 5 (alpha1, alpha0, eps, lr_w), or None; its auxiliary
    # field starts at zero on every level
    tgv: tuple | None = None


SIGMA_MAX_SAMPLES = 3.75  # widest Gaussian the compiled kernels take, in sample pitches (8 sigma / h <= 30)


def gauss_widths(geom_fine, geom, cfg, li):
    """The Gaussian widths (mm) of level `li`, largest first."""
    if cfg.sigma_schedule is not None:
        return tuple(float(x) for x in cfg.sigma_schedule[li])
    h = geom["c_mm_per_us"] / geom["fs_mhz"]
    return (min(SIGMA_MAX_SAMPLES * h, geom_fine["sigma_mm"] * geom["dx"] / geom_fine["dx"]),)


def time_decimation(geom_fine, geom, cfg):
    """Power-of-two factor by which a Gaussian level's time grid is coarser than the
    data's: the level's spacing ratio rounded down (1 when disabled or for the sphere)."""
    if not cfg.decimate_time or geom_fine.get("kernel", "sphere") != "gauss":
        return 1
    ratio = geom["dx"] / geom_fine["dx"]
    k = 1
    while 2 * k <= ratio + 1e-9:
        k *= 2
    return k


def gauss_lowpass_samples(sigma_level, sigma_data, h_data, decim):
    """Low-pass width (data samples) that turns data pulses of width sigma_data,
    averaged over one sample, into pulses of width sigma_level averaged over
    `decim` samples.  Variances add (a sample average over a width b adds
    b^2 / 12), so the filter supplies sigma_level^2 + (decim h)^2 / 12 minus
    sigma_data^2 + h^2 / 12."""
    var = (sigma_level ** 2 - sigma_data ** 2) / h_data ** 2 + (decim ** 2 - 1) / 12.0
    return math.sqrt(var) if var > 0 else 0.0


def gauss_amplitude_factor(sig_old, d_old, sig_new, d_new):
    """Rescaling of voxel amplitudes that keeps a sum of Gaussians on a grid the same
    field when the width or the spacing changes: a voxel of amplitude p and width
    sigma on spacing D stands for a density p (2 pi)^(3/2) sigma^3 / D^3."""
    return (sig_old / sig_new) ** 3 * (d_new / d_old) ** 3


def element_errors(elem, poses_a, poses_b):
    """Mean distance (mm) between element positions under two pose sets."""
    pa = np.einsum("fab,jb->fja", poses_a[:, :, :3], elem) + poses_a[:, None, :, 3]
    pb = np.einsum("fab,jb->fja", poses_b[:, :, :3], elem) + poses_b[:, None, :, 3]
    return float(np.linalg.norm(pa - pb, axis=-1).mean())


def rigid_consensus(ctx, geom, p0, poses, elem, meas, mask, cfg: C2FConfig, rng):
    """One Stage 2/3 pass; returns (new inlier mask, poses) on the device."""
    F, E = geom["n_frames"], geom["n_elem"]
    sig = ctx.forward(geom, p0, elem, poses)
    _, g = ctx.loss(geom, sig, meas, mask)
    _, G = ctx.pose_grad(geom, p0, elem, poses, g, mask, want_elem=True)
    G = G.cpu().numpy()
    P = poses.cpu().numpy()
    tmpl = elem.cpu().numpy()
    x = np.einsum("fab,jb->fja", P[:, :, :3], tmpl) + P[:, None, :, 3]
    new_mask = np.ones((F, E), dtype=np.uint8)
    first = 1 if cfg.fix_frame0 else 0
    for f in range(first, F):
        gn = np.linalg.norm(G[f], axis=1)
        if gn.max() <= 0:
            continue
        prop = x[f] - cfg.elem_step_mm * G[f] / gn.max()
        subsets = [rng.choice(E, size=3, replace=False) for _ in range(cfg.n_subsets)]
        rot, tr, inl, k = ransac(tmpl, prop, subsets, cfg.edge_tol_mm, cfg.inlier_tol_mm)
        if k < 0:
            continue
        new_mask[f] = inl.astype(np.uint8)
        cons = tmpl @ rot.T + tr
        if np.linalg.norm(cons - x[f], axis=1).max() > cfg.reset_mm:
            P[f, :, :3] = rot
            P[f, :, 3] = tr
    poses.copy_(torch.from_numpy(P))
    return torch.from_numpy(new_mask).to(poses.device), poses


def search_grids(radius_mm, step_mm, coarse_to_fine):
    """Per-axis offset grids of a translation search: the full grid of half-width
    radius_mm at step_mm, or (coarse_to_fine) shrinking 5-point grids -- spacing
    radius/2, then half the previous spacing around the best offset so far -- down to
    step_mm."""
    if not coarse_to_fine:
        return [np.arange(-radius_mm, radius_mm + 1e-9, step_mm)]
    grids, r = [], radius_mm
    while True:
        s = max(r / 2, step_mm)
        grids.append(np.arange(-2, 3) * s)
        if s <= step_mm * (1 + 1e-9):
            return grids
        r = s


def search_translations(ctx, geom, p0, poses, elem, meas, radius_mm, step_mm, first_frame=1, batch=512,
                        mask=None, coarse_to_fine=True):
    """Stage 2 coarse search: for every frame from `first_frame` on, translation
    offsets are scored by the NC loss of Eq. 3 (candidates are evaluated as extra
    frames of one forward call) and the frame takes the best candidate (Top-1).  The
    offsets are the cubic grid of half-width radius_mm at step_mm, or with
    coarse_to_fine shrinking 5-point grids around the best offset so far (375
    candidates for a 1.2 mm radius at 0.15 mm against 4913).  Returns the per-frame
    best scores."""
    P = poses.cpu().numpy()
    dev = poses.device
    best_scores = []
    grids = search_grids(radius_mm, step_mm, coarse_to_fine)
    for f in range(first_frame, geom["n_frames"]):
        best, best_pose = math.inf, None
        centre = P[f].copy()
        for ax in grids:
            offs = np.array(list(itertools.product(ax, ax, ax)))
            for c0 in range(0, len(offs), batch):
                o = offs[c0:c0 + batch]
                cand = np.repeat(centre[None], len(o), axis=0)
                cand[:, :, 3] += o
                gk = dict(geom, n_frames=len(o))
                sim = ctx.forward(gk, p0, elem, torch.from_numpy(cand).to(dev))
                sc = ctx.nc_scores(sim, meas[f], None if mask is None else mask[f]).cpu().numpy()
                i = int(np.argmin(sc))
                if sc[i] < best:
                    best, best_pose = float(sc[i]), cand[i]
            if best_pose is not None:  # no finite score (no signal at any candidate): keep the pose
                centre = best_pose.copy()
        if best_pose is not None:
            P[f] = best_pose
        best_scores.append(best)
    poses.copy_(torch.from_numpy(P).to(dev))
    return best_scores


def reconstruct(ctx: binding.Context, geom_fine, elem, meas, poses_init, cfg: C2FConfig = C2FConfig(),
                truth_poses=None, log=None):
    """Joint coarse-to-fine reconstruction.  meas: float [F][E][Nt] on the device.
    Returns (p0 on the finest level, poses [F][3][4] float64, history list)."""
    dev = ctx.device
    poses = torch.as_tensor(np.asarray(poses_init, dtype=np.float64)).to(dev).contiguous()
    elem_d = torch.as_tensor(np.asarray(elem, dtype=np.float64)).to(dev).contiguous()
    elem_np = np.asarray(elem, dtype=np.float64)
    rng = np.random.default_rng(cfg.seed)
    history = []
    p0, prev_geom, mask = None, None, None
    loss = torch.zeros((), dtype=torch.float64, device=dev)
    h = geom_fine["c_mm_per_us"] / geom_fine["fs_mhz"]
    gauss = geom_fine.get("kernel", "sphere") == "gauss"
    for li, (shape, n_steps) in enumerate(zip(cfg.levels, cfg.steps)):
        geom = level_geometry(geom_fine, shape)
        decim = time_decimation(geom_fine, geom, cfg)
        if decim > 1:
            geom["fs_mhz"] = geom_fine["fs_mhz"] / decim
            geom["n_samples"] = -(-geom_fine["n_samples"] // decim)
        widths = gauss_widths(geom_fine, geom, cfg, li) if gauss else (None,)
        if gauss:
            geom["sigma_mm"] = widths[0]
        if p0 is None:
            p0 = torch.full(tuple(shape), cfg.init_value, dtype=torch.float32, device=dev)
        else:
            p0 = ctx.resample(prev_geom, p0, geom)
            if gauss:
                ctx.scale(p0, gauss_amplitude_factor(prev_geom["sigma_mm"], prev_geom["dx"], geom["sigma_mm"],
                                                     geom["dx"]))
        if gauss:
            # a Gaussian pulse of width s low-passed by a Gaussian of width t is one of width sqrt(s^2 + t^2)
            sigma = (cfg.lowpass[li] if cfg.lowpass is not None
                     else gauss_lowpass_samples(geom["sigma_mm"], geom_fine["sigma_mm"], h, decim))
        else:
            sigma = (cfg.lowpass[li] if cfg.lowpass is not None
                     else max(0.0, (geom["a0_mm"] - geom_fine["a0_mm"]) / h))
        meas_l = ctx.lowpass(meas, sigma, decim=decim) if (sigma > 0 or decim > 1) else meas
        decay = cfg.lr_decay ** li
        t0 = time.perf_counter()
        if li == 0 and cfg.reference_steps:
            # Stage 1: reference map from the gauge frame's traces only
            ref_mask = torch.zeros((geom["n_frames"], geom["n_elem"]), dtype=torch.uint8, device=dev)
            ref_mask[0] = 1
            radam = binding.AdamState(geom, dev, lr_vol=cfg.lr_vol, nonneg=cfg.nonneg, freeze_poses=True)
            for _ in range(cfg.reference_steps):
                ctx.step(geom, p0, poses, elem_d, meas_l, radam, mask=ref_mask, loss_out=loss)
        if li == 0 and cfg.register_steps:
            # Stages 2-4: every frame registered against the map, volume frozen
            gadam = binding.AdamState(geom, dev, lr_rot=cfg.lr_rot, lr_trans=cfg.lr_trans,
                                      fix_frame0=cfg.fix_frame0, freeze_volume=True)
            for _ in range(cfg.register_steps):
                ctx.step(geom, p0, poses, elem_d, meas_l, gadam, mask=mask, loss_out=loss)
        n_vol = cfg.volume_only[li] if cfg.volume_only is not None else 0
        if n_vol:
            vadam = binding.AdamState(geom, dev, lr_vol=cfg.lr_vol * decay, nonneg=cfg.nonneg, freeze_poses=True)
            for _ in range(n_vol):
                ctx.step(geom, p0, poses, elem_d, meas_l, vadam, mask=mask, loss_out=loss)
        adam = binding.AdamState(geom, dev, lr_vol=cfg.lr_vol * decay, lr_rot=cfg.lr_rot * decay,
                                 lr_trans=cfg.lr_trans * decay, nonneg=cfg.nonneg, fix_frame0=cfg.fix_frame0)
        reg = binding.TgvState(geom, dev, *cfg.tgv) if cfg.tgv is not None else None
        phase_len = max(1, -(-n_steps // len(widths)))
        for k in range(n_steps):
            if gauss and k > 0 and k % phase_len == 0:
                # next, narrower width: keep the represented field, band-limit the data to match
                w_new = widths[min(k // phase_len, len(widths) - 1)]
                if w_new != geom["sigma_mm"]:
                    ctx.scale(p0, gauss_amplitude_factor(geom["sigma_mm"], geom["dx"], w_new, geom["dx"]))
                    geom = dict(geom, sigma_mm=w_new)
                    lp = (gauss_lowpass_samples(w_new, geom_fine["sigma_mm"], h, decim)
                          if cfg.lowpass is None else cfg.lowpass[li])
                    meas_l = ctx.lowpass(meas, lp, decim=decim) if (lp > 0 or decim > 1) else meas
                    sigma = lp
                    adam = binding.AdamState(geom, dev, lr_vol=cfg.lr_vol * decay, lr_rot=cfg.lr_rot * decay,
                                             lr_trans=cfg.lr_trans * decay, nonneg=cfg.nonneg,
                                             fix_frame0=cfg.fix_frame0)
            ctx.step(geom, p0, poses, elem_d, meas_l, adam, mask=mask, loss_out=loss, tgv=reg)
            if cfg.refine_every and (k + 1) % cfg.refine_every == 0:
                mask, poses = rigid_consensus(ctx, geom, p0, poses, elem_d, meas_l, mask, cfg, rng)
        n_search = 0
        if li == 0:
            for _ in range(cfg.search_rounds):
                search_translations(ctx, geom, p0, poses, elem_d, meas_l, cfg.search_radius_mm,
                                    cfg.search_step_mm, first_frame=1 if cfg.fix_frame0 else 0,
                                    batch=cfg.search_batch, mask=mask, coarse_to_fine=cfg.search_coarse_to_fine)
                adam = binding.AdamState(geom, dev, lr_vol=cfg.lr_vol * decay, lr_rot=cfg.lr_rot * decay,
                                         lr_trans=cfg.lr_trans * decay, nonneg=cfg.nonneg,
                                         fix_frame0=cfg.fix_frame0)
                for _ in range(cfg.search_joint_steps):
                    ctx.step(geom, p0, poses, elem_d, meas_l, adam, mask=mask, loss_out=loss)
                n_search += cfg.search_joint_steps
        torch.cuda.synchronize(dev)
        extra = (cfg.reference_steps + cfg.register_steps) if li == 0 else 0
        rec = {"level": li, "shape": list(shape), "steps": n_steps + n_vol + extra + n_search, "lowpass_sigma": sigma,
               "kernel_sigma_mm": geom.get("sigma_mm") if gauss else None, "time_decimation": decim,
               "loss": float(loss),
               "seconds": time.perf_counter() - t0}
        if truth_poses is not None:
            rec["mean_element_error_mm"] = element_errors(elem_np, poses.cpu().numpy(), np.asarray(truth_poses))
        history.append(rec)
        if log:
            log(rec)
        prev_geom = geom
    return p0, poses, history
