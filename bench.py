"""Benchmark: gradient steps/s of the differentiable acoustic radiation operator on B300.

One step = one pasfm_step on the full-scan workload (128^3 voxels at 0.1 mm,
vessel-tree phantom of 40 tubes, 16x16 elements at 0.6 mm, 64 frames on a smooth
sweep, 2048 samples at 40 MHz): element positions, forward, fused loss head,
adjoint and pose gradient (one fused kernel), Adam on the volume and on the
frame twists.  Inputs are synthetic and seeded; the iterate starts from a
dense volume and perturbed poses, the measurements are the forward of the true
volume and poses.

Prints ONE JSON line (rank 0).  --impl reference times the FP64 CPU oracle on a
bounded sample of the same step.  Under torchrun (--gpus N > 1) every rank runs
its own replica scan (weak scaling; the step has no cross-rank exchange).
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "grad steps/s"
UNIT = "steps/s"
WORKLOAD = "full_scan_128^3_0.1mm_vessel40_16x16_0.6mm_64f_2048s"


# Algorithmic FP32 flops per voxel-element pair (frozen before tuning;
# m = 2 a0 / h + 1 in-support samples per pair, FMA = 2 flops).
def flops_fwd(m):
    return 18 + 8 * m


def flops_adj(m):
    return 18 + 8 * m


def flops_pose(m):
    return 26 + 13 * m


# Gaussian kernel (Eq. 1): m = 8 sigma / h + 1 in-support samples per pair; three
# exp2 per pair and the two-multiply ratio recurrence per sample boundary.
def flops_fwd_gauss(m):
    return 28 + 5 * m


def flops_adj_gauss(m):
    return 30 + 5 * m


def flops_pose_gauss(m):
    return 37 + 10 * m


def peaks():
    p = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
    except (OSError, ValueError):
        pass
    sm_mhz = float(p.get("sm_max_mhz", 2032.0))
    # FP32 non-tensor peak: 148 SMs x 128 FP32 lanes x 2 flops x max SM clock
    fp32_tflops = 148 * 128 * 2 * sm_mhz * 1e6 / 1e12
    return dict(hbm_gbs=float(p.get("hbm_gbs", 6400.0)), fp32_tflops=fp32_tflops, sm_max_mhz=sm_mhz,
                source="measured" if p else "fallback")


# sources that define each measured kernel (traffic counters are valid only for these bytes)
KERNEL_SOURCES = {
    "fwd_cube": ("kernels.cuh", "pasfm_dev.cuh", "kernels_s.cu"),
    "bwd_cube": ("kernels.cuh", "pasfm_dev.cuh", "kernels_s.cu"),
    "fwd_reduce": ("aux.cu", "pasfm_dev.cuh"),
    "tgv": ("tgv.cu", "pasfm_dev.cuh"),
}


def _code_only(text):
    """Source text without comments and blank lines, so that editing a comment does not
    invalidate counters taken on the same code."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = (re.sub(r"(^|\s)(//|#(?!include|define|if|endif|else|elif|pragma|undef)).*$", "", ln).rstrip()
             for ln in text.splitlines())
    return "\n".join(ln for ln in lines if ln.strip())


def kernel_src_hash(kernel="bwd_cube"):
    """Hash of the code (comments stripped) of the sources that define `kernel` (a
    KERNEL_SOURCES key, '_gauss' suffix ignored) and of the build script that holds their
    compiler flags."""
    h = hashlib.sha256()
    for fn in KERNEL_SOURCES[kernel.replace("_gauss", "")]:
        with open(os.path.join(ROOT, "paper_2604_09643_b300", "csrc", fn), encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    with open(os.path.join(ROOT, "paper_2604_09643_b300", "build.py"), encoding="utf-8") as fh:
        h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def pipes_for(kernel):
    """Executed pipe figures (ncu) of `kernel` from the committed summaries, if taken on
    these sources."""
    try:
        with open(os.path.join(ROOT, "profiles", "pipes.json")) as fh:
            t = json.load(fh)
    except (OSError, ValueError):
        return None
    e = t.get(kernel)
    if not e or e.get("src_sha") != kernel_src_hash(kernel):
        return None
    return {k: v for k, v in e.items() if k != "src_sha"}


def traffic_for(kernel):
    """DRAM bytes per launch from the committed ncu summary, if taken on these sources."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            t = json.load(fh)
    except (OSError, ValueError):
        return None
    e = t.get(kernel)
    if not e or e.get("src_sha") != kernel_src_hash(kernel):
        return None
    return e.get("bytes_per_launch")


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except OSError:
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.remove(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [v for v in (num(r[1]) for r in rows) if v is not None]
        mx = [v for v in (num(r[2]) for r in rows) if v is not None]
        pw = [v for v in (num(r[3]) for r in rows) if v is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_median": statistics.median(pw) if pw else None, "reasons": reasons,
                "samples": len(rows)}


# ----------------------------------------------------------------------------- workload

WORKLOAD_MIXED = "mixed_precision_256x256x128_0.1mm_vessel150_32x32_0.3mm_400f_3072s"


def make_workload(seed_offset=0, n_frames=64, workload="full_scan", sigma=None):
    from paper_2604_09643_b300 import synth

    if workload == "mixed_precision":
        scan = synth.mixed_precision_scan(n_frames=n_frames, seed_offset=seed_offset)
    else:
        scan = synth.full_scan(seed_offset=seed_offset, n_frames=n_frames)
    if sigma:
        scan.geom.update(kernel="gauss", sigma_mm=float(sigma))
    rng = np.random.default_rng(synth.SEED_NOISE + 20 + seed_offset)
    # dense starting iterate: damped truth plus a uniform background
    p_init = (0.5 * scan.p0 + rng.uniform(0.02, 0.08, size=scan.p0.shape)).astype(np.float32)
    poses_init = synth.perturb_poses(scan.poses, rng, 0.5, 0.1, keep_first=True)
    return scan, p_init, poses_init


def fwd_smem_bytes_per_pair(geom):
    """Algorithmic shared-memory bytes per voxel-element pair of the forward: the load and
    store (4 bytes each) of every window slot the pair writes -- S - 1 slots of the
    running-sum window for 3 <= S <= 8, the S slot weights themselves otherwise (the
    wider pulses, whose running sums would round too coarsely, and the dipole of S = 2),
    with S = floor(2 sup / h) + 2 slots and sup = a0 or 4 sigma."""
    h = geom["c_mm_per_us"] / geom["fs_mhz"]
    sup = 4 * geom["sigma_mm"] if geom.get("kernel") == "gauss" else geom["a0_mm"]
    S = int(np.floor(2 * sup / h)) + 2
    return 8 * (S - 1 if 3 <= S <= 8 else S)


def pairs_and_m(geom):
    h = geom["c_mm_per_us"] / geom["fs_mhz"]
    sup = 4 * geom["sigma_mm"] if geom.get("kernel") == "gauss" else geom["a0_mm"]
    m = 2 * sup / h + 1
    pairs = geom["nx"] * geom["ny"] * geom["nz"] * geom["n_elem"] * geom["n_frames"]
    return pairs, m


# ----------------------------------------------------------------------------- CPU oracle timing

def oracle_step_sample(scan, p_init, poses_init, n_elem_sample):
    """Time the oracle on one frame and `n_elem_sample` elements of the step; returns
    seconds and the fraction of the full step's pairs it covered."""
    import oracle

    geom = dict(scan.geom, n_frames=1, n_elem=n_elem_sample)
    elem = scan.elem[:n_elem_sample]
    xw = oracle.element_positions(geom, elem, poses_init[:1])
    meas = np.random.default_rng(0).standard_normal((1, n_elem_sample, geom["n_samples"]))
    t = time.perf_counter()
    s = oracle.forward(geom, p_init, xw)
    _, g = oracle.loss(geom, s, meas)
    oracle.adjoint(geom, g, xw)
    oracle.pose_grad(geom, p_init, g, xw)
    dt = time.perf_counter() - t
    frac = n_elem_sample / (scan.geom["n_elem"] * scan.geom["n_frames"])
    return dt, frac


def cpu_baseline(scan, p_init, poses_init, n_elem_sample=256):
    import oracle

    dt, frac = oracle_step_sample(scan, p_init, poses_init, n_elem_sample)
    step_s = dt / frac
    return {"value": 1.0 / step_s, "unit": UNIT, "cores": oracle.threads_used(), "kind": "oracle",
            "sample": f"1 of {scan.geom['n_frames']} frames x {n_elem_sample} of {scan.geom['n_elem']} "
                      f"elements of one step (forward, loss, adjoint, pose gradient in FP64): "
                      f"{dt:.2f} s, scaled by the pair count", "seconds_per_step": step_s}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle

    scan, p_init, poses_init = make_workload()
    n_sample = 16
    for _ in range(args.warmup):
        oracle_step_sample(scan, p_init, poses_init, n_sample)
    times = []
    for _ in range(args.steps):
        dt, frac = oracle_step_sample(scan, p_init, poses_init, n_sample)
        times.append(dt / frac)
    step_s = sum(times) / len(times)
    value = 1.0 / step_s
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": WORKLOAD, "sample": f"1 frame x {n_sample} elements per step, scaled by pairs"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads_used(), "kind": "oracle",
                            "sample": f"each step: 1 of 64 frames x {n_sample} of 256 elements, scaled by pairs"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


# ----------------------------------------------------------------------------- GPU arm

def run_native(args):
    import torch
    import torch.distributed as dist

    from paper_2604_09643_b300 import binding, replicas

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    frames = args.frames if args.frames else (400 if args.workload == "mixed_precision" else 64)
    scan, p_init, poses_init = make_workload(seed_offset=rank, n_frames=frames, workload=args.workload,
                                             sigma=args.sigma if args.kernel == "gauss" else None)
    store = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[args.storage]
    geom = scan.geom
    pairs, m = pairs_and_m(geom)

    def to_dev(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    ctx = binding.Context(local)
    elem = to_dev(scan.elem)
    meas = ctx.forward(geom, to_dev(scan.p0), elem, to_dev(scan.poses)).to(store)
    ctx.reserve(geom)
    p0 = to_dev(p_init).to(store)
    poses = to_dev(poses_init)
    adam = binding.AdamState(geom, dev, lr_vol=2e-3, lr_rot=2e-4, lr_trans=2e-3, nonneg=True, fix_frame0=True)
    loss = torch.zeros((), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    warmup = max(args.warmup, 3)

    def step():
        ctx.step(geom, p0, poses, elem, meas, adam, loss_out=loss)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    rc, bits = ctx.status()
    if rc != 0:
        raise RuntimeError(f"device status {bits:#x} after warm-up")

    # ---- device-timed region (inputs resident in HBM)
    ctx.timing(True)
    ctx.timing_reset()
    l0 = ctx.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = ctx.launch_count() - l0
    ms = ev0.elapsed_time(ev1)
    per_kernel = {}
    for name in ("fwd_cube", "fwd_reduce", "bwd_cube", "diff_rows", "sum_parts", "pose_rows", "grad6", "adam_vol",
                 "adam_pose", "elem_pos", "loss_sum"):
        t, n = ctx.timing_read(name)
        if n:
            per_kernel[name] = {"ms_total": t, "launches": n, "ms_avg": t / n}
    ctx.timing(False)
    ctx.timing_reset()
    clocks = clk.summary()
    rc, bits = ctx.status()
    if rc != 0:
        raise RuntimeError(f"device status {bits:#x} in the timed region")

    ms = replicas.max_over_ranks(ms, dev)
    ms_per_step = ms / args.steps
    value = replicas.job_throughput(args.steps, ms / 1e3, world)

    # ---- end to end through the public API with host buffers: every step's measurements
    # are copied from pinned host memory (on a copy stream, into the buffer the step before
    # last used, so the copy overlaps the previous step) and its loss and poses read back
    meas_host = meas.cpu().pin_memory()
    loss_host = torch.zeros((), dtype=torch.float64).pin_memory()
    poses_host = torch.zeros(poses.shape, dtype=poses.dtype).pin_memory()
    meas_dev = [torch.empty_like(meas), torch.empty_like(meas)]
    copy_stream = torch.cuda.Stream(dev)
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    used = [torch.cuda.Event(), torch.cuda.Event()]
    e2e_steps = max(3, args.steps // 2)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(copy_stream):
        meas_dev[0].copy_(meas_host, non_blocking=True)
        copied[0].record(copy_stream)
    for k in range(e2e_steps):
        b = k & 1
        if k + 1 < e2e_steps:  # next step's copy into the other buffer, once its last step is done
            with torch.cuda.stream(copy_stream):
                if k >= 1:
                    copy_stream.wait_event(used[b ^ 1])
                meas_dev[b ^ 1].copy_(meas_host, non_blocking=True)
                copied[b ^ 1].record(copy_stream)
        stream.wait_event(copied[b])
        ctx.step(geom, p0, poses, elem, meas_dev[b], adam, loss_out=loss)
        used[b].record(stream)
        loss_host.copy_(loss, non_blocking=True)
        poses_host.copy_(poses, non_blocking=True)
        stream.synchronize()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = replicas.max_over_ranks(e2e_s, dev)
    e2e = {"value": replicas.job_throughput(e2e_steps, e2e_s, world), "unit": UNIT,
           "h2d_bytes_per_step": int(meas.numel() * meas.element_size()),
           "d2h_bytes_per_step": int(loss.element_size() + poses.numel() * poses.element_size())}

    # ---- roofline of the dominant kernel (algorithmic flops / live CUDA-event duration)
    pk = peaks()
    dom = max(per_kernel, key=lambda k: per_kernel[k]["ms_total"])
    gauss = args.kernel == "gauss"
    # the committed DRAM counters are per launch of the full-scan workload at its 64 frames;
    # other workloads and cut-down profiling cases report none
    captured = args.workload == "full_scan" and geom["n_frames"] == 64
    meas_mib = meas.numel() * meas.element_size() / 2**20
    resid_mib = meas.numel() * 4 / 2**20
    f_fwd, f_adj, f_pose = ((flops_fwd_gauss, flops_adj_gauss, flops_pose_gauss) if gauss
                            else (flops_fwd, flops_adj, flops_pose))
    fpp = {"bwd_cube": f_adj(m) + f_pose(m), "fwd_cube": f_fwd(m)}.get(dom)
    roofline = None
    if fpp:
        launches_per_step = per_kernel[dom]["launches"] / args.steps
        flops_per_launch = pairs * fpp / launches_per_step
        achieved = flops_per_launch / (per_kernel[dom]["ms_avg"] * 1e-3) / 1e12
        roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": pk["fp32_tflops"],
                    "unit": "TFLOP/s", "frac": achieved / pk["fp32_tflops"], "traffic": traffic_for(dom + ("_gauss" if gauss else "")) if captured else None,
                    "peak_source": f"FP32 148 SM x 128 lanes x 2 flops x {pk['sm_max_mhz']:.0f} MHz "
                                   f"({pk['source']} clock)",
                    "flops_per_pair": fpp, "pairs_per_launch": pairs / launches_per_step,
                    "executed": pipes_for(dom + ("_gauss" if gauss else "")),
                    "note": "achieved and frac count the frozen algorithmic flops per pair; the kernels' "
                            "rewritten slot sums execute fewer FP32 operations, so frac can pass 1.0 and "
                            "does not place the kernel on its roofline: `executed` does (ncu, same "
                            "sources): the share of cycles the FMA pipe is busy, with issue and warp "
                            "occupancy"}
    step_flops = pairs * (f_fwd(m) + f_adj(m) + f_pose(m))
    # achieved DRAM bandwidth of the kernels whose per-launch traffic ncu measured on these sources
    hbm = {}
    for name in ("fwd_cube", "bwd_cube", "fwd_reduce"):
        tb = traffic_for(name + ("_gauss" if gauss else "")) if captured else None
        if tb and name in per_kernel:
            gbs = tb / (per_kernel[name]["ms_avg"] * 1e-3) / 1e9
            hbm[name] = {"traffic_bytes": tb, "gbs": gbs, "frac": gbs / pk["hbm_gbs"]}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.storage == "f32" else f"f32 (volume and measurements stored {args.storage})",
        "data": "synthetic",
        "config": {"workload": (WORKLOAD if args.workload == "full_scan" else WORKLOAD_MIXED)
                   + (f"_gauss_sigma{args.sigma:g}mm" if gauss else ""),
                   "kernel": "gauss" if gauss else "sphere",
                   "voxels": [geom["nz"], geom["ny"], geom["nx"]],
                   "elements": geom["n_elem"], "frames": geom["n_frames"], "samples": geom["n_samples"],
                   "global_batch": world, "parallelism": f"replicas{world}",
                   "l2": f"inputs larger than L2 ({meas_mib:.0f} MiB measurements, {resid_mib:.0f} MiB residual, "
                         "per-cube partial traces written and read per step)"},
        "pairs_per_s": value * pairs,
        "step_tflops": step_flops * value / world / 1e12,
        "fp32_frac_step": step_flops * value / world / 1e12 / pk["fp32_tflops"],
        "roofline": roofline,
        "hbm": {"peak_gbs": pk["hbm_gbs"], "peak_source": pk["source"], "kernels": hbm},
        "per_kernel_ms": {k: round(v["ms_avg"], 4) for k, v in per_kernel.items()},
        "clocks": clocks,
        "gpu_launches": launches,
        "e2e": e2e,
        "final_loss": float(loss.item()),
    }
    if args.frames:
        out["config"]["workload"] += f" (profiling case: {args.frames} frames, not a bench line)"
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "full_scan" and not gauss:
        out["cpu_baseline"] = cpu_baseline(scan, p_init, poses_init)
    # measured FP32 FMA throughput of this GPU (after the timed region), scalar and packed:
    # context for the derived roofline peak
    out["fp32_probe_tflops"] = {"ffma": binding.fp32_probe(local, packed=False),
                                "ffma2": binding.fp32_probe(local, packed=True)}
    # packed half-precision FMA rates (half2, bfloat162): what half-precision slot arithmetic
    # could gain over the packed FP32 the kernels use
    out["half_probe_tflops"] = {"hfma2_f16": binding.fp32_probe(local, packed=2),
                                "hfma2_bf16": binding.fp32_probe(local, packed=3)}
    # and the shared-memory read-modify-write rate of the forward's window pattern, the
    # forward's own roofline: algorithmic shared bytes = read + write of its window slots
    # (S - 1 per pair for 3 <= S <= 8, else S; 4 bytes each way)
    smem_tbs = binding.smem_probe(local)
    out["smem_rmw_probe_tbs"] = smem_tbs
    if "fwd_cube" in per_kernel:
        bpp = fwd_smem_bytes_per_pair(geom)
        launches_f = per_kernel["fwd_cube"]["launches"] / args.steps
        tbs = pairs * bpp / launches_f / (per_kernel["fwd_cube"]["ms_avg"] * 1e-3) / 1e12
        out["roofline_fwd"] = {"bound": "smem", "kernel": "fwd_cube", "achieved": tbs, "peak": smem_tbs,
                               "unit": "TB/s", "frac": tbs / smem_tbs, "bytes_per_pair": bpp,
                               "peak_source": "measured: pasfm_smem_probe",
                               "executed": pipes_for("fwd_cube" + ("_gauss" if gauss else ""))}
    if rank == 0:
        print(json.dumps(out))
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


# ----------------------------------------------------------------------------- serving stream

WORKLOAD_SERVING = "serving_poisson4_mixed_scans_64-256^3_0.1mm_8x8-32x32_16-256f_1024-3072s"


def run_serving(args):
    """Continuous batching over the first requests of the seeded Poisson stream (mean 4
    scans/s): requests arrive at their stream times, are admitted by free HBM, run
    `--serve-steps` gradient steps each with their state resident, and the line reports
    the aggregate steps/s with the p50/p99 step latency."""
    import torch

    from paper_2604_09643_b300 import binding, serve, synth

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    specs = synth.request_stream(rate_per_s=args.serve_rate)[:args.serve_requests]
    with binding.Context(0) as ctx:
        reqs = [serve.request_from_spec(sp, ctx, steps=args.serve_steps) for sp in specs]
        warm = serve.request_from_spec(dict(specs[0], id=-1, arrival_s=0.0, n=64, n_frames=8, m=8),
                                       ctx, steps=max(args.warmup, 3))
    torch.cuda.synchronize()
    srv = serve.Server(device=0, mode=args.serve_mode)
    srv.submit(warm)
    srv.run()
    srv = serve.Server(device=0, mode=args.serve_mode, max_iteration_pairs=args.serve_max_pairs,
                       iteration_pairs=args.serve_iteration_pairs or None)
    for r in reqs:
        srv.submit(r)
    with ClockSampler(0) as clk:
        srv.run()
        torch.cuda.synchronize()
    rep = srv.report()
    pairs = sum(sp["n"] ** 3 * sp["m"] ** 2 * sp["n_frames"] for sp in specs) * args.serve_steps
    span = max(sp["arrival_s"] for sp in specs) or 1.0
    offered = len(specs) * args.serve_steps / span  # steps/s asked for while the requests arrive
    out = {"metric": METRIC, "value": rep["steps_per_s"], "unit": UNIT, "n_gpus": 1, "steps": rep["steps"],
           "warmup": max(args.warmup, 3), "ms_per_step": 1e3 / rep["steps_per_s"] if rep["steps_per_s"] else None,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic",
           "config": {"workload": WORKLOAD_SERVING.replace("poisson4", f"poisson{args.serve_rate:g}"),
                      "requests": len(specs), "steps_per_request": args.serve_steps,
                      "scheduling": args.serve_mode, "max_iteration_pairs": args.serve_max_pairs,
                      "iteration_pairs": (args.serve_iteration_pairs or None) if args.serve_mode == "batched"
                      else None,
                      "arrivals": f"seeded Poisson stream, mean {args.serve_rate:g} scans/s, first requests in "
                                  "arrival order",
                      "l2": "inputs larger than L2 (each scan's measurements 64 MiB-2.4 GiB)"},
           "offered_steps_per_s": offered, "arrival_span_s": span, "iterations": rep["iterations"],
           "step_ms_p50": rep["step_ms_p50"], "step_ms_p99": rep["step_ms_p99"],
           "queue_wait_s_p50": rep["queue_wait_s_p50"], "queue_wait_s_p99": rep["queue_wait_s_p99"],
           "completed": rep["completed"], "rejected": rep["rejected"], "failed": rep["failed"],
           "wall_s": rep["wall_s"], "pairs_per_s": pairs / rep["wall_s"] if rep["wall_s"] else None,
           "clocks": clk.summary(), "gpu_launches": rep["gpu_launches"],
           "e2e": None, "e2e_note": "measurements are simulated on the device before the stream starts"}
    print(json.dumps(out))
    return 0


# ----------------------------------------------------------------------------- TGV regulariser

WORKLOAD_TGV = "tgv_256^3_0.1mm"
TGV_BYTES_PER_VOXEL = 36  # read u 4 + w 12, read-modify-write grad_u 8, write grad_w 12


def run_tgv(args):
    """HBM roofline of the TGV regulariser kernel on a 256^3 volume (u, w, gradients:
    604 MiB, larger than L2): K timed launches of pasfm_tgv_grad accumulating into the
    volume gradient as pasfm_step_tgv does."""
    import torch

    from paper_2604_09643_b300 import binding

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    n = 256
    geom = {"nx": n, "ny": n, "nz": n, "dx": 0.1, "dy": 0.1, "dz": 0.1, "ox": 0.0, "oy": 0.0, "oz": 0.0,
            "n_elem": 1, "n_frames": 1, "n_samples": 1, "fs_mhz": 40.0, "t0_us": 0.0, "c_mm_per_us": 1.5,
            "a0_mm": 0.05}
    gen = torch.Generator(device=dev).manual_seed(0)
    u = torch.rand((n, n, n), device=dev, generator=gen)
    w = torch.randn((3, n, n, n), device=dev, generator=gen)
    gu = torch.zeros((n, n, n), device=dev)
    gw = torch.empty((3, n, n, n), device=dev)
    e = torch.zeros((), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    with binding.Context(0) as ctx:
        def launch():
            binding.pasfm_tgv_grad(ctx.handle, geom, u, w, 0.8, 0.3, 0.05, gu, 1, gw, e)
        for _ in range(max(args.warmup, 3)):
            launch()
        torch.cuda.synchronize()
        ctx.timing(True)
        ctx.timing_reset()
        l0 = ctx.launch_count()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(0) as clk:
            ev0.record(stream)
            for _ in range(args.steps):
                launch()
            ev1.record(stream)
            torch.cuda.synchronize()
        t_k, n_k = ctx.timing_read("tgv")
        launches = ctx.launch_count() - l0
        ctx.timing(False)
        rc, bits = ctx.status()
        if rc != 0:
            raise RuntimeError(f"device status {bits:#x}")
    ms = ev0.elapsed_time(ev1) / args.steps
    pk = peaks()
    nvox = n ** 3
    achieved = TGV_BYTES_PER_VOXEL * nvox / (t_k / n_k * 1e-3) / 1e9
    out = {"metric": "TGV voxels/s", "value": nvox / (ms * 1e-3), "unit": "voxels/s", "n_gpus": 1,
           "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOAD_TGV, "note": "regulariser kernel alone; not the bench line",
                      "l2": "inputs larger than L2 (604 MiB touched per launch)"},
           "roofline": {"bound": "hbm", "kernel": "tgv", "achieved": achieved, "peak": pk["hbm_gbs"],
                        "unit": "GB/s", "frac": achieved / pk["hbm_gbs"],
                        "traffic": traffic_for("tgv"), "bytes_per_voxel": TGV_BYTES_PER_VOXEL,
                        "peak_source": pk["source"]},
           "clocks": clk.summary(), "gpu_launches": launches}
    print(json.dumps(out))
    return 0


# ----------------------------------------------------------------------------- two-view pipeline

def run_two_view(args):
    """The PA-SFM pipeline (Stages 1-5) on two views of a 128^3 vessel volume at the
    centre of a 512-element half of a 60 mm hemispherical bowl (view B turned 90 deg,
    prior off by 0.5 deg / 0.5 mm per axis), or with --array cap33 on three views of
    a 33-element spherical-cap array over a 32^3 grid at 0.4 mm."""
    import torch

    from paper_2604_09643_b300 import binding, pipeline, synth

    torch.cuda.set_device(0)
    if args.array == "cap33":
        # 33 elements see too little for a fine reference map; the views are located on a 0.4 mm grid
        scan = synth.two_view_scan(n=32, spacing=0.4, elem=synth.cap_array(33), n_views=3, view_b_deg=30.0)
        name = "pipeline_32^3_0.4mm_cap33_60mm_3views"
        cfg = pipeline.PipelineConfig(stage1_steps=1500, search_radius_mm=2.0, inlier_tol_mm=0.5, edge_tol_mm=0.5,
                                      top_k=8)
    else:
        scan = synth.two_view_scan(n=128, spacing=0.1)
        name = "pipeline_128^3_0.1mm_bowl512_60mm_2views"
        cfg = pipeline.PipelineConfig(stage1_steps=900, stage5_steps=900)
    with binding.Context(0) as ctx:
        l0 = ctx.launch_count()
        with ClockSampler(0) as clk:
            t0 = time.perf_counter()
            res, _, _ = pipeline.run(ctx, scan, cfg)
            wall = time.perf_counter() - t0
        launches = ctx.launch_count() - l0
        rc, bits = ctx.status()
        if rc != 0:
            raise RuntimeError(f"device status {bits:#x}")
    out = {"metric": "pipeline seconds", "value": wall, "unit": "s", "n_gpus": 1, "steps": 1, "warmup": 0,
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": name, "note": "Algorithm 1 end to end; not the bench line"},
           "results": res, "clocks": clk.summary(), "gpu_launches": launches}
    print(json.dumps(out))
    return 0


# ----------------------------------------------------------------------------- joint reconstruction

WORKLOAD_RECON = "reconstruction_256^3_0.1mm_vessel150_16x16_0.6mm_200f_2048s_c2f_64-128-256"


def run_reconstruction(args):
    """Coarse-to-fine joint reconstruction of volume and poses on the 256^3, 200-frame
    scan whose initial poses carry N(0, 1.5 deg) rotation and N(0, 0.5 mm) translation
    noise per axis (frame 0 exact): levels 64^3 -> 128^3 -> 256^3, joint Adam steps on
    each, one Stage 2 translation search on the coarsest level.  Reports the steps/s
    over the whole schedule and the mean element error after each level."""
    import torch

    from paper_2604_09643_b300 import binding, optim, synth

    torch.cuda.set_device(0)
    scan = synth.reconstruction_scan()
    geom = scan.geom
    steps = tuple(int(x) for x in args.recon_steps.split(","))
    with binding.Context(0) as ctx:
        dev = ctx.device
        meas = ctx.forward(geom, torch.as_tensor(scan.p0).to(dev), torch.as_tensor(scan.elem).to(dev),
                           torch.as_tensor(scan.poses).to(dev))
        cfg = optim.C2FConfig(levels=((64, 64, 64), (128, 128, 128), (256, 256, 256)), steps=steps,
                              lr_vol=0.02, lr_rot=1e-3, lr_trans=1e-2, lr_decay=0.5,
                              search_rounds=args.recon_search, search_radius_mm=1.2, search_step_mm=0.15,
                              search_joint_steps=steps[0])
        torch.cuda.synchronize()
        l0 = ctx.launch_count()
        with ClockSampler(0) as clk:
            t0 = time.perf_counter()
            p0, poses, hist = optim.reconstruct(ctx, geom, scan.elem, meas, scan.poses_init, cfg,
                                                truth_poses=scan.poses)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
        launches = ctx.launch_count() - l0
        rc, bits = ctx.status()
        if rc != 0:
            raise RuntimeError(f"device status {bits:#x}")
        vol_err = float(np.linalg.norm(p0.cpu().numpy() - scan.p0) / np.linalg.norm(scan.p0))
    n_steps = sum(h["steps"] for h in hist)
    out = {"metric": METRIC, "value": n_steps / wall, "unit": UNIT, "n_gpus": 1, "steps": n_steps, "warmup": 0,
           "ms_per_step": 1e3 * wall / n_steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOAD_RECON, "levels": [list(l) for l in cfg.levels], "steps": list(steps),
                      "search_rounds": args.recon_search,
                      "note": "mixed-level steps/s over the whole schedule, incl. the search; not a bench line"},
           "initial_mean_element_error_mm": optim.element_errors(scan.elem, scan.poses_init, scan.poses),
           "levels": [{k: h[k] for k in ("level", "shape", "steps", "seconds", "mean_element_error_mm",
                                          "lowpass_sigma", "loss")} for h in hist],
           "final_mean_element_error_mm": hist[-1]["mean_element_error_mm"],
           "volume_rel_l2_error": vol_err, "wall_s": wall, "clocks": clk.summary(), "gpu_launches": launches}
    print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--frames", type=int, default=0,
                    help="override the frame count (only for small ncu captures; not a bench line)")
    ap.add_argument("--workload", choices=["full_scan", "mixed_precision", "serving", "reconstruction", "tgv",
                                           "two_view"],
                    default="full_scan",
                    help="full_scan: the benchmark; mixed_precision: 256x256x128, 32x32 elements, 400 frames; "
                         "serving: continuous batching over the seeded request stream; reconstruction: "
                         "coarse-to-fine joint volume + pose recovery on 256^3 with 200 frames")
    ap.add_argument("--recon-steps", default="100,100,100", help="reconstruction: joint steps per level")
    ap.add_argument("--array", choices=["bowl512", "cap33"], default="bowl512", help="two_view: array geometry")
    ap.add_argument("--recon-search", type=int, default=1, help="reconstruction: Stage 2 search rounds")
    ap.add_argument("--kernel", choices=["sphere", "gauss"], default="sphere",
                    help="voxel pulse: uniform sphere (a0 = spacing / 2) or the Gaussian of Eq. 1")
    ap.add_argument("--sigma", type=float, default=0.05, help="Gaussian width (mm) for --kernel gauss")
    ap.add_argument("--serve-requests", type=int, default=12, help="serving: requests taken from the stream")
    ap.add_argument("--serve-steps", type=int, default=4, help="serving: gradient steps per request")
    ap.add_argument("--serve-mode", choices=["batched", "streams"], default="batched",
                    help="serving: one batched step over the resident scans per iteration, or each scan's own "
                         "steps on its own stream")
    ap.add_argument("--serve-max-pairs", type=float, default=None,
                    help="serving: cap on an iteration's voxel-element pairs (resident scans' steps together)")
    ap.add_argument("--serve-iteration-pairs", type=float, default=1e12,
                    help="serving (batched): pair budget of one iteration, filled fair-share (0: every "
                         "resident scan in every iteration)")
    ap.add_argument("--serve-rate", type=float, default=4.0, help="serving: mean arrival rate (scans/s)")
    ap.add_argument("--storage", choices=["f32", "bf16", "f16"], default="f32",
                    help="storage type of the volume and the measurements (arithmetic stays FP32)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "reconstruction":
        return run_reconstruction(args)
    if args.workload == "tgv":
        return run_tgv(args)
    if args.workload == "two_view":
        return run_two_view(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
