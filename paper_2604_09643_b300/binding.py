"""ctypes binding of ``libpasfm.so`` (the C ABI in ``include/pasfm.h``).

Argument marshalling only: every function here checks tensor placement, dtype
and contiguity, passes ``data_ptr()`` and the current CUDA stream to the
library, and turns a negative return code into :class:`PasfmError`.  No step
of the operator runs in Python, and there is no CPU fallback: if the library
cannot be loaded, every call raises.

The low-level functions carry the ABI's names (``pasfm_forward`` ...).
:class:`Context` wraps them with allocation of outputs for convenience.
"""
from __future__ import annotations

import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libpasfm.so")

PASFM_F32, PASFM_BF16, PASFM_F16 = 0, 1, 2
ADAM_NONNEG, ADAM_FIX_FRAME0, ADAM_FREEZE_POSES, ADAM_FREEZE_VOLUME = 1, 2, 4, 8
STATUS_ELEMENT_INSIDE, STATUS_TIMEOUT, STATUS_INDEX_CLAMPED = 1, 2, 4

_DTYPE_CODE = {torch.float32: PASFM_F32, torch.bfloat16: PASFM_BF16, torch.float16: PASFM_F16}


class PasfmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"pasfm error {code}: {msg}")
        self.code = code


class PasfmGeom(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("n_elem", ctypes.c_int32), ("n_frames", ctypes.c_int32), ("n_samples", ctypes.c_int32),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("ox", ctypes.c_double), ("oy", ctypes.c_double), ("oz", ctypes.c_double),
                ("fs_mhz", ctypes.c_double), ("t0_us", ctypes.c_double),
                ("c_mm_per_us", ctypes.c_double), ("a0_mm", ctypes.c_double),
                ("dtype_vol", ctypes.c_int32), ("dtype_sig", ctypes.c_int32),
                ("kernel", ctypes.c_int32), ("reserved", ctypes.c_int32), ("sigma_mm", ctypes.c_double)]


KERNEL_CODE = {"sphere": 0, "gauss": 1}   # PASFM_KERNEL_SPHERE, PASFM_KERNEL_GAUSS


class PasfmAdam(ctypes.Structure):
    _fields_ = [("m_vol", ctypes.c_void_p), ("v_vol", ctypes.c_void_p),
                ("m_pose", ctypes.c_void_p), ("v_pose", ctypes.c_void_p),
                ("step", ctypes.c_int64),
                ("lr_vol", ctypes.c_double), ("lr_rot", ctypes.c_double), ("lr_trans", ctypes.c_double),
                ("beta1", ctypes.c_double), ("beta2", ctypes.c_double), ("eps", ctypes.c_double),
                ("flags", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class PasfmTgv(ctypes.Structure):
    _fields_ = [("w", ctypes.c_void_p), ("m_w", ctypes.c_void_p), ("v_w", ctypes.c_void_p),
                ("alpha1", ctypes.c_double), ("alpha0", ctypes.c_double), ("eps", ctypes.c_double),
                ("lr_w", ctypes.c_double)]


_lib = None
_VP, _I, _SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
_G = ctypes.POINTER(PasfmGeom)
_SIGS = {
    "pasfm_create": ([ctypes.POINTER(_VP), _I], _I),
    "pasfm_destroy": ([_VP], _I),
    "pasfm_workspace_size": ([_G, ctypes.POINTER(_SZ)], _I),
    "pasfm_reserve": ([_VP, _G], _I),
    "pasfm_set_partial_budget": ([_VP, _SZ], _I),
    "pasfm_set_wait_limit": ([_VP, ctypes.c_int64], _I),
    "pasfm_element_positions": ([_VP, _G, _VP, _VP, _VP, _VP], _I),
    "pasfm_forward": ([_VP, _G, _VP, _VP, _VP, _VP, _VP], _I),
    "pasfm_adjoint": ([_VP, _G, _VP, _VP, _VP, _VP, _VP], _I),
    "pasfm_pose_grad": ([_VP, _G, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP], _I),
    "pasfm_loss": ([_VP, _G, _VP, _VP, _VP, _VP, _VP, _VP], _I),
    "pasfm_step": ([_VP, _G, _VP, _VP, _VP, _VP, _VP, ctypes.POINTER(PasfmAdam), _VP, _VP], _I),
    "pasfm_tgv_grad": ([_VP, _G, _VP, _VP, ctypes.c_double, ctypes.c_double, ctypes.c_double, _VP, _I, _VP, _VP,
                        _VP], _I),
    "pasfm_step_batch": ([_I, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP], _I),
    "pasfm_step_tgv": ([_VP, _G, _VP, _VP, _VP, _VP, _VP, ctypes.POINTER(PasfmAdam), ctypes.POINTER(PasfmTgv),
                        _VP, _VP, _VP], _I),
    "pasfm_apply_twists": ([_VP, _I, _VP, _VP, _VP, _VP], _I),
    "pasfm_twist_grad": ([_VP, _I, _VP, _VP, _VP, _VP], _I),
    "pasfm_resample": ([_VP, _G, _VP, _G, _VP, _VP], _I),
    "pasfm_lowpass": ([_VP, ctypes.c_int64, _I, ctypes.c_double, _I, _VP, _VP, _VP], _I),
    "pasfm_nc_scores": ([_VP, _I, _I, _I, _VP, _VP, _I, _VP, _VP, _VP], _I),
    "pasfm_nc_grad": ([_VP, ctypes.c_int64, _I, _VP, _VP, _I, _I, _VP, ctypes.c_double, _VP, _VP, _VP], _I),
    "pasfm_scale": ([_VP, ctypes.c_int64, ctypes.c_double, _VP, _VP], _I),
    "pasfm_fp32_probe": ([_I, _I, ctypes.POINTER(ctypes.c_double)], _I),
    "pasfm_smem_probe": ([_I, ctypes.POINTER(ctypes.c_double)], _I),
    "pasfm_pose_grad_noalloc": ([_G, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP], _I),
    "pasfm_status": ([_VP, _VP, ctypes.POINTER(ctypes.c_uint32)], _I),
    "pasfm_timing_enable": ([_VP, _I], _I),
    "pasfm_timing_reset": ([_VP], _I),
    "pasfm_timing_read": ([_VP, ctypes.c_char_p, ctypes.POINTER(ctypes.c_double),
                           ctypes.POINTER(ctypes.c_int64)], _I),
    "pasfm_launch_count": ([_VP], ctypes.c_int64),
    "pasfm_last_error": ([], ctypes.c_char_p),
    "pasfm_abi_version": ([], _I),
}


def lib():
    """Load libpasfm.so (raises if it was not built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run `python -m paper_2604_09643_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def symbols():
    """Names of the ABI functions this binding declares."""
    return sorted(_SIGS)


def _check(rc):
    if rc != 0:
        raise PasfmError(rc, lib().pasfm_last_error().decode(errors="replace"))
    return rc


def make_geom(geom: dict, dtype_vol=torch.float32, dtype_sig=torch.float32) -> PasfmGeom:
    g = PasfmGeom()
    for k in ("nx", "ny", "nz", "n_elem", "n_frames", "n_samples"):
        setattr(g, k, int(geom[k]))
    for k in ("dx", "dy", "dz", "ox", "oy", "oz", "fs_mhz", "t0_us", "c_mm_per_us", "a0_mm"):
        setattr(g, k, float(geom[k]))
    g.dtype_vol = _DTYPE_CODE[dtype_vol]
    g.dtype_sig = _DTYPE_CODE[dtype_sig]
    g.kernel = KERNEL_CODE[geom.get("kernel", "sphere")]
    g.sigma_mm = float(geom.get("sigma_mm", 0.0))
    return g


def _ptr(t, dtype=None, name="tensor", allow_none=False):
    if t is None:
        if allow_none:
            return None
        raise ValueError(f"{name} is required")
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype not in (dtype if isinstance(dtype, tuple) else (dtype,)):
        raise ValueError(f"{name} has dtype {t.dtype}, expected {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream, device):
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return ctypes.c_void_p(stream.cuda_stream)


_VOL = (torch.float32, torch.bfloat16, torch.float16)


# ----------------------------------------------------------------------------- ABI-named calls

def pasfm_element_positions(ctx, geom, elem, pose, xw_out, stream=None):
    g = make_geom(geom)
    _check(lib().pasfm_element_positions(ctx, ctypes.byref(g), _ptr(elem, torch.float64, "elem"),
                                         _ptr(pose, torch.float64, "pose"), _ptr(xw_out, torch.float64, "xw_out"),
                                         _stream(stream, xw_out.device)))


def pasfm_forward(ctx, geom, p0, elem, pose, sig_out, stream=None):
    g = make_geom(geom, dtype_vol=p0.dtype)
    _check(lib().pasfm_forward(ctx, ctypes.byref(g), _ptr(p0, _VOL, "p0"), _ptr(elem, torch.float64, "elem"),
                               _ptr(pose, torch.float64, "pose"), _ptr(sig_out, torch.float32, "sig_out"),
                               _stream(stream, sig_out.device)))


def pasfm_adjoint(ctx, geom, elem, pose, g_sig, vol_out, stream=None):
    g = make_geom(geom, dtype_sig=g_sig.dtype)
    _check(lib().pasfm_adjoint(ctx, ctypes.byref(g), _ptr(elem, torch.float64, "elem"),
                               _ptr(pose, torch.float64, "pose"), _ptr(g_sig, _VOL, "g"),
                               _ptr(vol_out, torch.float32, "vol_out"), _stream(stream, vol_out.device)))


def pasfm_pose_grad(ctx, geom, p0, elem, pose, g_sig, mask, grad6_out, gelem_out=None, stream=None):
    g = make_geom(geom, dtype_vol=p0.dtype, dtype_sig=g_sig.dtype)
    _check(lib().pasfm_pose_grad(ctx, ctypes.byref(g), _ptr(p0, _VOL, "p0"), _ptr(elem, torch.float64, "elem"),
                                 _ptr(pose, torch.float64, "pose"), _ptr(g_sig, _VOL, "g"),
                                 _ptr(mask, torch.uint8, "mask", allow_none=True),
                                 _ptr(grad6_out, torch.float64, "grad6_out"),
                                 _ptr(gelem_out, torch.float64, "gelem_out", allow_none=True),
                                 _stream(stream, grad6_out.device)))


def pasfm_loss(ctx, geom, sig, meas, mask, g_out, loss_out, stream=None):
    g = make_geom(geom, dtype_sig=meas.dtype)
    _check(lib().pasfm_loss(ctx, ctypes.byref(g), _ptr(sig, torch.float32, "sig"), _ptr(meas, _VOL, "meas"),
                            _ptr(mask, torch.uint8, "mask", allow_none=True), _ptr(g_out, torch.float32, "g_out"),
                            _ptr(loss_out, torch.float64, "loss_out"), _stream(stream, loss_out.device)))


def pasfm_step(ctx, geom, p0, pose, elem, meas, mask, adam: PasfmAdam, loss_out=None, stream=None):
    g = make_geom(geom, dtype_vol=p0.dtype, dtype_sig=meas.dtype)
    _check(lib().pasfm_step(ctx, ctypes.byref(g), _ptr(p0, _VOL, "p0"), _ptr(pose, torch.float64, "pose"),
                            _ptr(elem, torch.float64, "elem"), _ptr(meas, _VOL, "meas"),
                            _ptr(mask, torch.uint8, "mask", allow_none=True), ctypes.byref(adam),
                            _ptr(loss_out, torch.float64, "loss_out", allow_none=True),
                            _stream(stream, p0.device)))


def pasfm_tgv_grad(ctx, geom, p0, w, alpha1, alpha0, eps, grad_u, accumulate, grad_w, energy_out=None,
                   stream=None):
    g = make_geom(geom, dtype_vol=p0.dtype)
    _check(lib().pasfm_tgv_grad(ctx, ctypes.byref(g), _ptr(p0, _VOL, "p0"), _ptr(w, torch.float32, "w"),
                                float(alpha1), float(alpha0), float(eps), _ptr(grad_u, torch.float32, "grad_u"),
                                int(bool(accumulate)), _ptr(grad_w, torch.float32, "grad_w"),
                                _ptr(energy_out, torch.float64, "energy_out", allow_none=True),
                                _stream(stream, p0.device)))


def pasfm_step_tgv(ctx, geom, p0, pose, elem, meas, mask, adam: PasfmAdam, tgv, loss_out=None, tgv_out=None,
                   stream=None):
    g = make_geom(geom, dtype_vol=p0.dtype, dtype_sig=meas.dtype)
    _check(lib().pasfm_step_tgv(ctx, ctypes.byref(g), _ptr(p0, _VOL, "p0"), _ptr(pose, torch.float64, "pose"),
                                _ptr(elem, torch.float64, "elem"), _ptr(meas, _VOL, "meas"),
                                _ptr(mask, torch.uint8, "mask", allow_none=True), ctypes.byref(adam),
                                None if tgv is None else ctypes.byref(tgv),
                                _ptr(loss_out, torch.float64, "loss_out", allow_none=True),
                                _ptr(tgv_out, torch.float64, "tgv_out", allow_none=True),
                                _stream(stream, p0.device)))


def pasfm_pose_grad_noalloc(geom, p0, elem, pose, g_sig, mask, grad6_out, gelem_out=None, stream=None):
    """Pose gradient without any device allocation (fixed in-library scratch)."""
    g = make_geom(geom, dtype_vol=p0.dtype, dtype_sig=g_sig.dtype)
    _check(lib().pasfm_pose_grad_noalloc(ctypes.byref(g), _ptr(p0, _VOL, "p0"), _ptr(elem, torch.float64, "elem"),
                                         _ptr(pose, torch.float64, "pose"), _ptr(g_sig, _VOL, "g"),
                                         _ptr(mask, torch.uint8, "mask", allow_none=True),
                                         _ptr(grad6_out, torch.float64, "grad6_out"),
                                         _ptr(gelem_out, torch.float64, "gelem_out", allow_none=True),
                                         _stream(stream, grad6_out.device)))


def fp32_probe(device=0, packed=False):
    """Measured FMA throughput of the device in TFLOP/s: scalar FP32 (packed False / 0),
    packed two-wide FP32 (True / 1), packed half2 (2) or bfloat162 (3)."""
    v = ctypes.c_double()
    mode = int(packed) if not isinstance(packed, bool) else int(packed)
    _check(lib().pasfm_fp32_probe(int(device), mode, ctypes.byref(v)))
    return v.value


def smem_probe(device=0):
    """Measured shared-memory read-modify-write throughput of the device in TB/s."""
    v = ctypes.c_double()
    _check(lib().pasfm_smem_probe(int(device), ctypes.byref(v)))
    return v.value


def pasfm_status(ctx, stream=None, device=None):
    bits = ctypes.c_uint32(0)
    rc = lib().pasfm_status(ctx, _stream(stream, device), ctypes.byref(bits))
    return rc, int(bits.value)


# ----------------------------------------------------------------------------- convenience

class Context:
    """Owns one ``pasfm_ctx`` (workspace + status word) on one device.

    Use one Context per concurrently running stream."""

    def __init__(self, device=0):
        if isinstance(device, torch.device):
            device = device.index or 0
        self.device = torch.device("cuda", int(device))
        h = ctypes.c_void_p()
        _check(lib().pasfm_create(ctypes.byref(h), int(device)))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            lib().pasfm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- calls -----------------------------------------------------------------
    def reserve(self, geom, dtype_vol=torch.float32, dtype_sig=torch.float32):
        g = make_geom(geom, dtype_vol, dtype_sig)
        _check(lib().pasfm_reserve(self.handle, ctypes.byref(g)))

    def set_partial_budget(self, nbytes):
        _check(lib().pasfm_set_partial_budget(self.handle, int(nbytes)))

    def set_wait_limit(self, cycles):
        """Bound (SM clock cycles) of the kernels' wait for each TMA-staged copy; a
        negative value restores the default, 0 makes every such wait time out at once."""
        _check(lib().pasfm_set_wait_limit(self.handle, int(cycles)))

    def element_positions(self, geom, elem, pose, out=None, stream=None):
        F, E = geom["n_frames"], geom["n_elem"]
        out = torch.empty((F, E, 3), dtype=torch.float64, device=self.device) if out is None else out
        pasfm_element_positions(self.handle, geom, elem, pose, out, stream)
        return out

    def forward(self, geom, p0, elem, pose, out=None, stream=None):
        shape = (geom["n_frames"], geom["n_elem"], geom["n_samples"])
        out = torch.empty(shape, dtype=torch.float32, device=self.device) if out is None else out
        pasfm_forward(self.handle, geom, p0, elem, pose, out, stream)
        return out

    def adjoint(self, geom, elem, pose, g_sig, out=None, stream=None):
        shape = (geom["nz"], geom["ny"], geom["nx"])
        out = torch.empty(shape, dtype=torch.float32, device=self.device) if out is None else out
        pasfm_adjoint(self.handle, geom, elem, pose, g_sig, out, stream)
        return out

    def pose_grad(self, geom, p0, elem, pose, g_sig, mask=None, want_elem=False, stream=None):
        F, E = geom["n_frames"], geom["n_elem"]
        g6 = torch.empty((F, 6), dtype=torch.float64, device=self.device)
        ge = torch.empty((F, E, 3), dtype=torch.float64, device=self.device) if want_elem else None
        pasfm_pose_grad(self.handle, geom, p0, elem, pose, g_sig, mask, g6, ge, stream)
        return (g6, ge) if want_elem else g6

    def loss(self, geom, sig, meas, mask=None, g_out=None, stream=None):
        g_out = torch.empty_like(sig) if g_out is None else g_out
        L = torch.empty((), dtype=torch.float64, device=self.device)
        pasfm_loss(self.handle, geom, sig, meas, mask, g_out, L, stream)
        return L, g_out

    def step(self, geom, p0, pose, elem, meas, adam: "AdamState", mask=None, loss_out=None, stream=None,
             tgv: "TgvState | None" = None, tgv_out=None):
        """One pasfm_step, or pasfm_step_tgv when a TGV state is given."""
        if tgv is None:
            pasfm_step(self.handle, geom, p0, pose, elem, meas, mask, adam.c, loss_out, stream)
        else:
            pasfm_step_tgv(self.handle, geom, p0, pose, elem, meas, mask, adam.c, tgv.c, loss_out, tgv_out, stream)

    def tgv_grad(self, geom, p0, w, alpha1, alpha0, eps, grad_u=None, accumulate=False, stream=None):
        """TGV energy (device double) and gradients (grad_u [nz][ny][nx], grad_w [3][nz][ny][nx])."""
        shape = (geom["nz"], geom["ny"], geom["nx"])
        grad_u = torch.zeros(shape, dtype=torch.float32, device=self.device) if grad_u is None else grad_u
        grad_w = torch.empty((3,) + shape, dtype=torch.float32, device=self.device)
        energy = torch.zeros((), dtype=torch.float64, device=self.device)
        pasfm_tgv_grad(self.handle, geom, p0, w, alpha1, alpha0, eps, grad_u, accumulate, grad_w, energy, stream)
        return energy, grad_u, grad_w

    def apply_twists(self, pose, xi, out=None, stream=None):
        """pose (F,3,4) with left twists xi (F,6) applied: (Exp(w) R, Exp(w) t + v)."""
        out = torch.empty_like(pose) if out is None else out
        _check(lib().pasfm_apply_twists(self.handle, int(pose.shape[0]), _ptr(pose, torch.float64, "pose"),
                                        _ptr(xi, torch.float64, "xi"), _ptr(out, torch.float64, "out"),
                                        _stream(stream, self.device)))
        return out

    def twist_grad(self, xi, grad6, out=None, stream=None):
        """Gradient in twist coordinates from the gradient at the twisted pose."""
        out = torch.empty_like(grad6) if out is None else out
        _check(lib().pasfm_twist_grad(self.handle, int(xi.shape[0]), _ptr(xi, torch.float64, "xi"),
                                      _ptr(grad6, torch.float64, "grad6"), _ptr(out, torch.float64, "out"),
                                      _stream(stream, self.device)))
        return out

    def resample(self, src_geom, src, dst_geom, out=None, stream=None):
        """Trilinear resampling of a float volume onto another voxel grid."""
        shape = (dst_geom["nz"], dst_geom["ny"], dst_geom["nx"])
        out = torch.empty(shape, dtype=torch.float32, device=self.device) if out is None else out
        gs, gd = make_geom(src_geom), make_geom(dst_geom)
        _check(lib().pasfm_resample(self.handle, ctypes.byref(gs), _ptr(src, torch.float32, "src"),
                                    ctypes.byref(gd), _ptr(out, torch.float32, "out"), _stream(stream, self.device)))
        return out

    def lowpass(self, sig, sigma, out=None, stream=None, decim=1):
        """Gaussian low-pass (sigma in input samples) of every trace of sig [..., Nt],
        keeping every `decim`-th sample: out [..., ceil(Nt / decim)]."""
        T = int(sig.shape[-1])
        n_out = -(-T // int(decim))
        out = torch.empty(*sig.shape[:-1], n_out, dtype=torch.float32, device=sig.device) if out is None else out
        rows = sig.numel() // T if sig.numel() else 0
        _check(lib().pasfm_lowpass(self.handle, int(rows), T, float(sigma), int(decim),
                                   _ptr(sig, torch.float32, "sig"), _ptr(out, torch.float32, "out"),
                                   _stream(stream, self.device)))
        return out

    def nc_grad(self, sim, meas, mask=None, scale=1.0, out=None, stream=None, meas_repeat=1):
        """Gradient of the summed NC loss (Eq. 3) w.r.t. sim [..., Nt] and the per-row NC
        values; sim row r is paired with meas row r // meas_repeat; mask per sim row or None."""
        T = int(sim.shape[-1])
        rows = sim.numel() // T if sim.numel() else 0
        if meas.numel() // max(T, 1) * int(meas_repeat) != rows:
            raise ValueError("meas must hold one trace per meas_repeat rows of sim")
        out = torch.empty_like(sim) if out is None else out
        nc = torch.zeros(sim.shape[:-1], dtype=torch.float64, device=self.device)
        _check(lib().pasfm_nc_grad(self.handle, int(rows), T, _ptr(sim, torch.float32, "sim"), _ptr(meas, _VOL, "meas"),
                                   _DTYPE_CODE[meas.dtype], int(meas_repeat),
                                   _ptr(mask, torch.uint8, "mask", allow_none=True), float(scale),
                                   _ptr(out, torch.float32, "out"), _ptr(nc, torch.float64, "nc"),
                                   _stream(stream, self.device)))
        return out, nc

    def scale(self, x, alpha, stream=None):
        """x *= alpha in place (float32 device tensor)."""
        _check(lib().pasfm_scale(self.handle, int(x.numel()), float(alpha), _ptr(x, torch.float32, "x"),
                                 _stream(stream, self.device)))
        return x

    def nc_scores(self, sim, meas, mask=None, out=None, stream=None):
        """NC-loss scores of candidate trace sets sim [K][E][Nt] against meas [E][Nt]."""
        K, E, T = (int(x) for x in sim.shape)
        out = torch.empty(K, dtype=torch.float64, device=self.device) if out is None else out
        _check(lib().pasfm_nc_scores(self.handle, K, E, T, _ptr(sim, torch.float32, "sim"), _ptr(meas, _VOL, "meas"),
                                     _DTYPE_CODE[meas.dtype], _ptr(mask, torch.uint8, "mask", allow_none=True),
                                     _ptr(out, torch.float64, "out"), _stream(stream, self.device)))
        return out

    def status(self, stream=None):
        return pasfm_status(self.handle, stream, self.device)

    def timing(self, enable=True):
        _check(lib().pasfm_timing_enable(self.handle, int(bool(enable))))

    def timing_reset(self):
        _check(lib().pasfm_timing_reset(self.handle))

    def timing_read(self, kernel="*"):
        ms, n = ctypes.c_double(0.0), ctypes.c_int64(0)
        _check(lib().pasfm_timing_read(self.handle, kernel.encode(), ctypes.byref(ms), ctypes.byref(n)))
        return float(ms.value), int(n.value)

    def launch_count(self):
        return int(lib().pasfm_launch_count(self.handle))


def step_batch(ctxs, geoms, p0s, poses, elems, meas, adams, masks=None, loss_outs=None, trace=None, stream=None):
    """pasfm_step_batch: one gradient step for each scan i (its own Context, geometry,
    volume, poses, template, measurements, AdamState, optional mask and loss output),
    the hot kernels of scans sharing an instantiation batched into one launch per phase.
    trace: optional int64 device tensor [n][2] of per-scan first-start / last-end times (ns)."""
    n = len(ctxs)
    if not all(len(x) == n for x in (geoms, p0s, poses, elems, meas, adams)):
        raise ValueError("every per-scan list needs one entry per scan")
    if n == 0:
        return
    device = ctxs[0].device
    G = (PasfmGeom * n)(*[make_geom(g, dtype_vol=p.dtype, dtype_sig=m.dtype) for g, p, m in zip(geoms, p0s, meas)])
    handles = (_VP * n)(*[c.handle for c in ctxs])
    states = (PasfmAdam * n)(*[a.c for a in adams])
    arr = lambda xs, dt, what, none=False: (_VP * n)(*[_ptr(x, dt, what, allow_none=none) for x in xs])
    mk = arr(masks, torch.uint8, "mask", True) if masks is not None else None
    lo = arr(loss_outs, torch.float64, "loss_out", True) if loss_outs is not None else None
    tr = None
    if trace is not None:
        if trace.dtype != torch.int64 or tuple(trace.shape) != (n, 2) or not trace.is_cuda:
            raise ValueError("trace must be an int64 CUDA tensor of shape (n, 2)")
        tr = ctypes.c_void_p(trace.data_ptr())
    rc = lib().pasfm_step_batch(n, handles, G, arr(p0s, _VOL, "p0"), arr(poses, torch.float64, "pose"),
                                arr(elems, torch.float64, "elem"), arr(meas, _VOL, "meas"), mk, states, lo, tr,
                                _stream(stream, device))
    for a, st in zip(adams, states):   # the library advanced each state's step count
        a.c.step = st.step
    _check(rc)


class TgvState:
    """Device-resident auxiliary field w of the TGV regulariser with its Adam moments."""

    def __init__(self, geom, device, alpha1, alpha0, eps=1e-3, lr_w=1e-2, w=None):
        shape = (3, geom["nz"], geom["ny"], geom["nx"])
        self.w = torch.zeros(shape, dtype=torch.float32, device=device) if w is None else w
        self.m_w = torch.zeros(shape, dtype=torch.float32, device=device)
        self.v_w = torch.zeros(shape, dtype=torch.float32, device=device)
        self.c = PasfmTgv(self.w.data_ptr(), self.m_w.data_ptr(), self.v_w.data_ptr(), float(alpha1), float(alpha0),
                          float(eps), float(lr_w))


class AdamState:
    """Device-resident Adam moments for a volume and F frame twists."""

    def __init__(self, geom, device, lr_vol=1e-2, lr_rot=1e-3, lr_trans=1e-2, beta1=0.9, beta2=0.999,
                 eps=1e-8, nonneg=False, fix_frame0=False, freeze_poses=False, freeze_volume=False):
        nvox = geom["nx"] * geom["ny"] * geom["nz"]
        F = geom["n_frames"]
        self.m_vol = torch.zeros(nvox, dtype=torch.float32, device=device)
        self.v_vol = torch.zeros(nvox, dtype=torch.float32, device=device)
        self.m_pose = torch.zeros((F, 6), dtype=torch.float64, device=device)
        self.v_pose = torch.zeros((F, 6), dtype=torch.float64, device=device)
        flags = ((ADAM_NONNEG if nonneg else 0) | (ADAM_FIX_FRAME0 if fix_frame0 else 0)
                 | (ADAM_FREEZE_POSES if freeze_poses else 0) | (ADAM_FREEZE_VOLUME if freeze_volume else 0))
        self.c = PasfmAdam(self.m_vol.data_ptr(), self.v_vol.data_ptr(), self.m_pose.data_ptr(),
                           self.v_pose.data_ptr(), 0, lr_vol, lr_rot, lr_trans, beta1, beta2, eps, flags, 0)

    @property
    def step(self):
        return int(self.c.step)
