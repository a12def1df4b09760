"""pasfm_step_batch: the serving loop's batched gradient step over resident scans.

Each scan's tiles in a batched launch are exactly the blocks of its own pasfm_step
launches, so a scan's results must be bit-identical to pasfm_step's whatever else is
in the batch.  The scans of one group (same kernel instantiation and profile) share
one persistent launch per phase, and their work overlaps on the device.
"""
import numpy as np
import pytest
import torch

from paper_2604_09643_b300 import binding, synth
from tests.parity_cases import gaussian, ragged_case, tma_case

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _scan(make, seed, mask=False, **adam_kw):
    geom, truth, elem, poses = make()
    with binding.Context(0) as ctx:
        meas = ctx.forward(geom, _dev(truth), _dev(elem), _dev(poses))
    rng = np.random.default_rng(seed)
    p0 = (0.5 * truth + rng.uniform(0, 0.01, truth.shape)).astype(np.float32)
    start = synth.perturb_poses(poses, np.random.default_rng(seed + 1), 0.3, 0.03, keep_first=True)
    m = None
    if mask:
        m = (np.random.default_rng(seed + 2).uniform(size=(geom["n_frames"], geom["n_elem"])) > 0.3).astype(np.uint8)
    kw = dict(lr_vol=1e-2, lr_rot=2e-4, lr_trans=2e-3, nonneg=True, fix_frame0=True)
    kw.update(adam_kw)
    return dict(geom=geom, elem=elem, meas=meas, p0=p0, start=start, mask=m, adam=kw)


def _scans():
    return [
        _scan(tma_case, 1),                                           # sphere, TMA paths
        _scan(lambda: tma_case(seed=3), 11, mask=True),               # same group, masked
        _scan(ragged_case, 21),                                       # same instantiation, unaligned (plain loads)
        _scan(gaussian(tma_case, 0.05), 31),                          # another group (Gaussian, S = 12)
        _scan(lambda: tma_case(seed=5), 41, freeze_poses=True),       # another backward mode (adjoint only)
        _scan(lambda: ragged_case(seed=2), 51, freeze_volume=True),   # pose gradient only
    ]


def _state(sc):
    return dict(p0=_dev(sc["p0"]), pose=_dev(sc["start"]), elem=_dev(sc["elem"]),
                mask=None if sc["mask"] is None else _dev(sc["mask"]),
                adam=binding.AdamState(sc["geom"], "cuda", **sc["adam"]),
                loss=torch.zeros((), dtype=torch.float64, device="cuda"))


def _snapshot(st):
    a = st["adam"]
    return [t.clone() for t in (st["p0"], st["pose"], a.m_vol, a.v_vol, a.m_pose, a.v_pose, st["loss"])]


@pytest.mark.parametrize("chunked", [False, True])
def test_batch_is_bit_identical_to_single_steps(cuda_device, chunked):
    """Two batched steps of six scans in four groups (two instantiations, two backward
    modes, TMA and plain-load staging, a mask) against pasfm_step scan by scan; with
    `chunked` every context's partial budget forces one frame per forward and backward
    launch, so the batch runs several frame-chunk rounds."""
    scans = _scans()
    ref, bat = [], []
    for sc in scans:
        st = _state(sc)
        with binding.Context(0) as ctx:
            if chunked:
                ctx.set_partial_budget(1)
            for _ in range(2):
                ctx.step(sc["geom"], st["p0"], st["pose"], st["elem"], sc["meas"], st["adam"], mask=st["mask"],
                         loss_out=st["loss"])
            assert ctx.status() == (0, 0)
        ref.append(_snapshot(st))
    states = [_state(sc) for sc in scans]
    ctxs = [binding.Context(0) for _ in scans]
    try:
        if chunked:
            for c in ctxs:
                c.set_partial_budget(1)
        for _ in range(2):
            binding.step_batch(ctxs, [sc["geom"] for sc in scans], [st["p0"] for st in states],
                               [st["pose"] for st in states], [st["elem"] for st in states],
                               [sc["meas"] for sc in scans], [st["adam"] for st in states],
                               masks=[st["mask"] for st in states], loss_outs=[st["loss"] for st in states])
        for c in ctxs:
            assert c.status() == (0, 0)
    finally:
        for c in ctxs:
            c.close()
    for i, st in enumerate(states):
        assert st["adam"].step == 2
        for a, b in zip(ref[i], _snapshot(st)):
            assert torch.equal(a, b), i


def test_one_launch_per_phase_and_overlapping_scans(cuda_device):
    """Three scans of one group: one forward, one reduction and one backward launch per
    step (recorded on the first scan's context), and the per-scan [first tile start,
    last tile end] intervals on the device intersect pairwise."""
    scans = [_scan(tma_case, 61), _scan(lambda: tma_case(seed=7), 71), _scan(lambda: tma_case(seed=8), 81)]
    states = [_state(sc) for sc in scans]
    ctxs = [binding.Context(0) for _ in scans]
    trace = torch.zeros((3, 2), dtype=torch.int64, device="cuda")
    try:
        ctxs[0].timing(True)
        binding.step_batch(ctxs, [sc["geom"] for sc in scans], [st["p0"] for st in states],
                           [st["pose"] for st in states], [st["elem"] for st in states],
                           [sc["meas"] for sc in scans], [st["adam"] for st in states], trace=trace)
        torch.cuda.synchronize()
        assert ctxs[0].timing_read("fwd_cube_batch")[1] == 1
        assert ctxs[0].timing_read("fwd_reduce_batch")[1] == 1
        assert ctxs[0].timing_read("bwd_cube_batch")[1] == 1
        assert ctxs[0].timing_read("fwd_cube")[1] == 0 and ctxs[0].timing_read("bwd_cube")[1] == 0
    finally:
        for c in ctxs:
            c.close()
    iv = trace.cpu().numpy().astype(np.uint64)
    assert np.all(iv[:, 1] > iv[:, 0]), iv
    for a in range(3):
        for b in range(a + 1, 3):
            assert max(iv[a, 0], iv[b, 0]) < min(iv[a, 1], iv[b, 1]), (a, b, iv)


def test_batch_argument_errors(cuda_device):
    sc = _scan(tma_case, 91)
    st = _state(sc)
    with binding.Context(0) as ctx:
        with pytest.raises(binding.PasfmError) as e:   # one context for two scans
            binding.step_batch([ctx, ctx], [sc["geom"]] * 2, [st["p0"]] * 2, [st["pose"]] * 2, [st["elem"]] * 2,
                               [sc["meas"]] * 2, [st["adam"]] * 2)
        assert e.value.code == -1
        binding.step_batch([], [], [], [], [], [], [])  # no scans: nothing to do
