"""Continuous-batching reconstruction server over the radiation operator.

Freehand scans arrive as requests, each asking for a number of gradient steps of
the joint volume + pose reconstruction.  The server:

* admits a waiting request when its device footprint fits the free HBM (minus a
  reserve), refuses with a status one that could never fit or that does not fit
  while no scan is running, and otherwise keeps it queued until running scans
  finish and release memory (cached blocks are returned to the driver when a
  request waits for memory);
* keeps every admitted scan resident: its volume, poses, measurements, Adam
  state and a private library context (workspace);
* runs iterations: each is ONE batched gradient step over the resident scans that
  still owe steps (all of them, or with an iteration budget the least-served ones that
  fit: fair share by voxel-element pairs) (pasfm_step_batch), in which the scans sharing a kernel
  instantiation run their forward, reduction and fused adjoint / pose gradient as
  one persistent launch per phase, so their work overlaps on the device; up to
  ``inflight`` iterations are enqueued at a time, and arrivals join at the next
  iteration (continuous batching rather than a queue drained one by one);
* times every iteration with CUDA events (a scan's step latency is the duration
  of the iteration that carried it), records queue wait, and reports p50/p99 step
  latency and aggregate steps/s;
* isolates failures: a scan whose loss turns non-finite or whose device status
  word is set is stopped and released while the others continue.

``mode="streams"`` keeps the earlier scheduling for comparison: each scan steps
with its own pasfm_step calls on its own stream, ``inflight`` steps enqueued per
scan, and the device interleaves the scans' kernels.

A scan's tiles are the same in every batch, and every scan has private workspaces,
so its result does not depend on what else is running (bit-identical).
"""
from __future__ import annotations

import dataclasses
import time
from collections import deque

import numpy as np
import torch

from . import binding

ADMIT, WAIT, REJECT = "admit", "wait", "reject"


def admission(footprint, free, total, reserve):
    """Decision for one request given device memory figures (bytes)."""
    if footprint + reserve > total:
        return REJECT
    if footprint + reserve > free:
        return WAIT
    return ADMIT


def step_pairs(geom):
    """Voxel-element pairs one gradient step of a scan processes (its share of an iteration)."""
    return int(geom["nx"]) * int(geom["ny"]) * int(geom["nz"]) * int(geom["n_elem"]) * int(geom["n_frames"])


def footprint_bytes(geom):
    """Device bytes a resident scan needs: library workspace plus its arrays."""
    import ctypes
    g = binding.make_geom(geom)
    ws = ctypes.c_size_t(0)
    binding._check(binding.lib().pasfm_workspace_size(ctypes.byref(g), ctypes.byref(ws)))
    nvox = geom["nx"] * geom["ny"] * geom["nz"]
    F, E, T = geom["n_frames"], geom["n_elem"], geom["n_samples"]
    arrays = nvox * 4 * 3 + F * E * T * 4 + F * 96 * 3 + E * 24 + 1024
    return int(ws.value + arrays)


@dataclasses.dataclass
class Request:
    """One reconstruction request: measurements, array template, starting point."""
    id: int
    arrival_s: float
    geom: dict
    elem: np.ndarray
    meas: np.ndarray | torch.Tensor   # float32 [F][E][Nt] (host or device)
    poses_init: np.ndarray
    steps: int = 20
    p0_init: np.ndarray | None = None
    lr_vol: float = 0.02
    lr_rot: float = 1e-3
    lr_trans: float = 1e-2


@dataclasses.dataclass
class Result:
    id: int
    status: str
    steps: int
    p0: np.ndarray | None
    poses: np.ndarray | None
    final_loss: float
    queue_wait_s: float
    step_ms: list
    admitted_s: float = 0.0
    finished_s: float = 0.0
    launches: int = 0


def request_from_spec(spec: dict, context, *, steps=4, spacing_mm=0.1, standoff_mm=4.0,
                      rot_sigma_deg=0.5, trans_sigma_mm=0.05) -> Request:
    """A reconstruction request from one entry of a request stream (volume side ``n``,
    ``n_frames``, an ``m`` x ``m`` array at ``pitch`` mm, ``n_samples``, ``n_tubes``,
    ``seed``): a vessel-tree phantom, a sweep trajectory, measurements simulated by
    ``context.forward`` on its device at the true poses, and perturbed starting poses."""
    from . import synth

    n, F, m, T = int(spec["n"]), int(spec["n_frames"]), int(spec["m"]), int(spec["n_samples"])
    geom = synth.make_geom((n, n, n), spacing_mm, m * m, F, T)
    rng = np.random.default_rng(int(spec["seed"]))
    p0 = synth.vessel_tree_phantom(geom, int(spec["n_tubes"]), rng)
    elem = synth.planar_array(m, m, float(spec["pitch"]))
    poses = synth.sweep_poses(F, n * spacing_mm / F, synth.top_face_z(geom) + standoff_mm, rng)  # spans the volume
    d = context.device
    meas = context.forward(geom, torch.as_tensor(p0).to(d), torch.as_tensor(elem).to(d),
                           torch.as_tensor(poses).to(d))
    init = synth.perturb_poses(poses, rng, rot_sigma_deg, trans_sigma_mm, keep_first=True)
    return Request(int(spec["id"]), float(spec["arrival_s"]), geom, elem, meas, init, steps=steps,
                   p0_init=np.full(p0.shape, 0.05, np.float32))


class _Scan:
    def __init__(self, req: Request, device, now, stream=None):
        self.req = req
        self.ctx = binding.Context(device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device)
        self.admitted_s = now
        d = self.ctx.device
        with torch.cuda.stream(self.stream):
            g = req.geom
            shape = (g["nz"], g["ny"], g["nx"])
            self.p0 = (torch.zeros(shape, dtype=torch.float32, device=d) if req.p0_init is None
                       else torch.as_tensor(np.ascontiguousarray(req.p0_init, dtype=np.float32)).to(d))
            self.poses = torch.as_tensor(np.ascontiguousarray(req.poses_init, dtype=np.float64)).to(d)
            self.elem = torch.as_tensor(np.ascontiguousarray(req.elem, dtype=np.float64)).to(d)
            self.meas = torch.as_tensor(req.meas).to(d, torch.float32).contiguous()
            self.adam = binding.AdamState(g, d, lr_vol=req.lr_vol, lr_rot=req.lr_rot, lr_trans=req.lr_trans,
                                          nonneg=True, fix_frame0=True)
            self.loss = torch.zeros((), dtype=torch.float64, device=d)
        self.ctx.reserve(req.geom)
        self.issued = 0
        self.served_pairs = 0   # voxel-element pairs of the steps issued so far (fair share)
        self.events = deque()   # (start, end) per step still running, oldest first
        self.step_ms = []
        self.failed = None

    def issue(self):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(self.stream)
        self.ctx.step(self.req.geom, self.p0, self.poses, self.elem, self.meas, self.adam, loss_out=self.loss,
                      stream=self.stream)
        e.record(self.stream)
        self.events.append((s, e))
        self.issued += 1

    def poll(self):
        while self.events and self.events[0][1].query():
            s, e = self.events.popleft()
            self.step_ms.append(s.elapsed_time(e))

    def done(self):
        return self.issued >= self.req.steps and not self.events

    def finish(self, now, wait_s, shared_stream=False):
        # every step's end event has completed (done()); on a stream shared with other
        # scans' later iterations, read the status on the current stream instead of
        # waiting for those
        if not shared_stream:
            self.stream.synchronize()
        rc, bits = self.ctx.status(None if shared_stream else self.stream)
        loss = float(self.loss.item())
        status = "ok"
        if rc != 0:
            status = f"failed: device status {bits:#x}"
        elif not np.isfinite(loss):
            status = "failed: non-finite loss"
        ok = status == "ok"
        res = Result(self.req.id, status, self.issued, self.p0.cpu().numpy() if ok else None,
                     self.poses.cpu().numpy() if ok else None, loss, wait_s, list(self.step_ms),
                     self.admitted_s, now, self.ctx.launch_count())
        self.release()
        return res

    def release(self):
        self.ctx.close()
        self.p0 = self.poses = self.elem = self.meas = self.adam = self.loss = None


def issue_iteration(scans, stream):
    """One batched gradient step over `scans` on `stream`: every scan's step is timed by
    the iteration's events (shared), and its pending-event queue gets them."""
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record(stream)
    binding.step_batch([x.ctx for x in scans], [x.req.geom for x in scans], [x.p0 for x in scans],
                       [x.poses for x in scans], [x.elem for x in scans], [x.meas for x in scans],
                       [x.adam for x in scans], loss_outs=[x.loss for x in scans], stream=stream)
    e.record(stream)
    for x in scans:
        x.events.append((s, e))
        x.issued += 1
        x.served_pairs += step_pairs(x.req.geom)


def fair_share(due, budget):
    """The scans of the next iteration: the least-served first (pairs of the steps issued
    so far, then arrival order), first fit into `budget` pairs; the least-served scan is
    always taken, so a scan larger than the budget runs alone in its turn and none starves."""
    pick, total = [], 0
    for x in sorted(due, key=lambda x: (x.served_pairs, x.req.arrival_s, x.req.id)):
        c = step_pairs(x.req.geom)
        if pick and total + c > budget:
            continue
        pick.append(x)
        total += c
    return pick


class Server:
    """Admit, run and retire reconstruction requests on one GPU."""

    def __init__(self, device=0, reserve_bytes=2 << 30, max_active=16, inflight=2, mem_info=None,
                 clock=time.perf_counter, mode="batched", max_iteration_pairs=None, iteration_pairs=None):
        """max_iteration_pairs: optional cap on the voxel-element pairs of all resident scans'
        steps together: a request that would pass it waits, unless nothing is running; it
        bounds the step latency at the cost of queue wait (None: up to max_active scans).
        iteration_pairs: optional budget of one batched iteration; each iteration then takes
        the least-served resident scans that fit (fair share by pairs), so small scans step
        in most iterations while a large one steps when its turn comes (None: every
        resident scan that owes a step, every iteration)."""
        if mode not in ("batched", "streams"):
            raise ValueError("mode must be 'batched' or 'streams'")
        self.max_iteration_pairs = max_iteration_pairs
        self.iteration_pairs = iteration_pairs
        self.device = torch.device("cuda", device) if isinstance(device, int) else device
        self.reserve = reserve_bytes
        self.max_active = max_active
        self.inflight = inflight
        self.mode = mode
        self.mem_info = mem_info or (lambda: torch.cuda.mem_get_info(self.device))
        self.clock = clock
        self.queue = deque()
        self.active = []
        self.results = []
        self.iterations = 0
        self.t0 = None
        self._stream = None

    def submit(self, req: Request):
        self.queue.append(req)

    def _now(self):
        return self.clock() - self.t0

    def _admit(self):
        while self.queue and len(self.active) < self.max_active:
            req = self.queue[0]
            if req.arrival_s > self._now():
                return
            if (self.max_iteration_pairs is not None and self.active and
                    sum(step_pairs(x.req.geom) for x, _ in self.active) + step_pairs(req.geom)
                    > self.max_iteration_pairs):
                return  # the iteration is full: wait for a resident scan to finish
            free, total = self.mem_info()
            need = footprint_bytes(req.geom)
            dec = admission(need, free, total, self.reserve)
            if dec == REJECT:
                self.queue.popleft()
                self.results.append(Result(req.id, f"rejected: needs {need} bytes, device has {total}", 0,
                                           None, None, float("nan"), self._now() - req.arrival_s, []))
                continue
            if dec == WAIT and torch.cuda.memory_reserved(self.device) > torch.cuda.memory_allocated(self.device):
                # retired scans' blocks may still sit in the caching allocator: hand them back
                # to the driver (this synchronises, so only when a request is waiting for memory)
                torch.cuda.empty_cache()
                free, total = self.mem_info()
                dec = admission(need, free, total, self.reserve)
            if dec == WAIT:
                if not self.active:
                    # nothing running will free memory for it: waiting could last forever
                    self.queue.popleft()
                    self.results.append(Result(req.id, f"rejected: needs {need} bytes, {free} free with no scan "
                                                       f"running", 0, None, None, float("nan"),
                                               self._now() - req.arrival_s, []))
                    continue
                return
            self.queue.popleft()
            if self.mode == "batched" and self._stream is None:
                self._stream = torch.cuda.Stream(self.device)
            stream = self._stream if self.mode == "batched" else None
            self.active.append((_Scan(req, self.device, self._now(), stream), self._now() - req.arrival_s))

    def _issue(self):
        if self.mode == "streams":
            for scan, _ in self.active:
                scan.poll()
                while scan.issued < scan.req.steps and len(scan.events) < self.inflight:
                    scan.issue()
            return
        # batched: keep up to `inflight` iterations enqueued; an iteration takes every
        # resident scan that still owes a step and has fewer than `inflight` in flight
        while True:
            for scan, _ in self.active:
                scan.poll()
            due = [scan for scan, _ in self.active
                   if scan.issued < scan.req.steps and len(scan.events) < self.inflight]
            if not due:
                return
            if self.iteration_pairs is not None:
                due = fair_share(due, self.iteration_pairs)
            issue_iteration(due, self._stream)
            self.iterations += 1

    def run(self, max_seconds=None):
        """Serve until the queue and the active set are empty (or max_seconds)."""
        self.t0 = self.clock()
        while self.queue or self.active:
            self._admit()
            self._issue()
            keep = []
            for scan, wait in self.active:
                scan.poll()
                if scan.done():
                    self.results.append(scan.finish(self._now(), wait, shared_stream=self.mode == "batched"))
                else:
                    keep.append((scan, wait))
            self.active = keep
            if not self.active and self.queue:
                delay = self.queue[0].arrival_s - self._now()
                if delay > 0:
                    time.sleep(min(delay, 0.05))
            elif self.active:
                time.sleep(0.0005)
            if max_seconds is not None and self._now() > max_seconds:
                break
        return self.results

    def report(self):
        ok = [r for r in self.results if r.status == "ok"]
        lat = [m for r in ok for m in r.step_ms]
        waits = [r.queue_wait_s for r in ok]
        wall = max((r.finished_s for r in ok), default=0.0)
        steps = sum(r.steps for r in ok)
        pct = lambda v, q: float(np.percentile(v, q)) if v else None
        return {"mode": self.mode, "iterations": self.iterations if self.mode == "batched" else None,
                "requests": len(self.results), "completed": len(ok),
                "rejected": sum(r.status.startswith("rejected") for r in self.results),
                "failed": sum(r.status.startswith("failed") for r in self.results),
                "steps": steps, "wall_s": wall, "steps_per_s": steps / wall if wall > 0 else None,
                "gpu_launches": sum(r.launches for r in self.results),
                "step_ms_p50": pct(lat, 50), "step_ms_p99": pct(lat, 99),
                "queue_wait_s_p50": pct(waits, 50), "queue_wait_s_p99": pct(waits, 99)}
